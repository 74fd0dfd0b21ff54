// Host side of the TMA helpers: the tensor-map encoder, reached through the
// runtime's driver entry-point query (no link against the driver library).
#include <cudaTypedefs.h>

#include <mutex>

#include "tma.cuh"

namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_once;

struct SmemEntry {
    const void *kernel;
    size_t bytes;
};
SmemEntry g_smem[256];
int g_smem_n = 0;
std::mutex g_smem_mutex;
}  // namespace

cudaError_t dfs_allow_smem(const void *kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    std::lock_guard<std::mutex> lock(g_smem_mutex);
    int i = 0;
    while (i < g_smem_n && g_smem[i].kernel != kernel) ++i;
    if (i < g_smem_n && g_smem[i].bytes >= bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e) return e;
    if (i == g_smem_n) {
        if (g_smem_n == 256) return cudaSuccess;   // table full: keep setting each time
        g_smem[g_smem_n++] = {kernel, bytes};
    } else {
        g_smem[i].bytes = bytes;
    }
    return cudaSuccess;
}

cudaError_t dfs_encode_tensor_map_2d(CUtensorMap *map, const void *base, uint64_t width,
                                     uint64_t height, uint64_t pitch_bytes, uint32_t box_w,
                                     uint32_t box_h) {
    std::call_once(g_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        else
            cudaGetLastError();
    });
    if (!g_encode) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {width, height};
    cuuint64_t strides[1] = {pitch_bytes};
    cuuint32_t box[2] = {box_w, box_h};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(base), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t dfs_encode_tensor_map_3d_f32(CUtensorMap *map, const void *base, const uint64_t dims[3],
                                         const uint64_t strides_bytes[2], const uint32_t box[3],
                                         int swizzle128) {
    std::call_once(g_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        else
            cudaGetLastError();
    });
    if (!g_encode) return cudaErrorNotSupported;
    cuuint64_t d[3] = {dims[0], dims[1], dims[2]};
    cuuint64_t st[2] = {strides_bytes[0], strides_bytes[1]};
    cuuint32_t bx[3] = {box[0], box[1], box[2]};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), d, st,
                          bx, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}
