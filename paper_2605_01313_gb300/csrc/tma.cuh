// Tensor-memory-accelerator (TMA) loads and mbarrier waits in inline PTX for
// sm_103a, plus the host-side tensor-map encoder (driver entry point).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

// Status word values written by kernels (plan-owned device int).
#define DFS_STATUS_OK 0
#define DFS_STATUS_TIMEOUT 1

// Cycles a thread waits on an mbarrier before it gives up (about 1 s at 2 GHz).
#define DFS_WAIT_CYCLES 2000000000LL

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Make barrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// One arrival (no transaction bytes), release semantics at CTA scope.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier, for at most `budget` SM cycles
// (DFS_WAIT_CYCLES by default).  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  long long budget = DFS_WAIT_CYCLES) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > budget) return false;
    }
    return true;
}

// 2-D tiled TMA load of one box into shared memory, completing on `bar`.
// x (the innermost coordinate) times the element size must be a multiple of 16
// bytes; callers guarantee it.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Asynchronous 8-byte copy global -> shared (both 8-byte aligned), completed by
// the commit/wait groups below (this thread's copies only).
__device__ __forceinline__ void cp_async_8(void *smem_dst, const void *gmem_src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}
// Asynchronous 16-byte copy global -> shared (both 16-byte aligned), cached in
// L2 only.
__device__ __forceinline__ void cp_async_16(void *smem_dst, const void *gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}
// Arrive on an mbarrier once every cp.async this thread issued before has
// landed; .noinc: the barrier's expected arrival count already includes it.
__device__ __forceinline__ void cp_async_mbar_arrive_noinc(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// Wait until every cp.async this thread issued has landed (committed or not).
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
// Wait until at most N of this thread's committed groups are still pending.
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Host: raise a kernel's dynamic shared-memory limit to at least `bytes`,
// calling cudaFuncSetAttribute only the first time a larger size is needed (so
// that launches recorded into a CUDA graph make no attribute calls).
cudaError_t dfs_allow_smem(const void *kernel, size_t bytes);

// Host: encode a 2-D tensor map of 8-byte elements (rows of `width` elements,
// `height` rows, row pitch `pitch_bytes`) with box `box_w` x `box_h`.
// Returns cudaErrorNotSupported when the driver offers no encoder.
cudaError_t dfs_encode_tensor_map_2d(CUtensorMap *map, const void *base, uint64_t width,
                                     uint64_t height, uint64_t pitch_bytes, uint32_t box_w,
                                     uint32_t box_h);

// Host: encode a 3-D tensor map of FP32 elements (dims[0] innermost; strides of
// dims 1 and 2 in bytes), box box[0] x box[1] x box[2], optionally with the
// 128-byte swizzle (box[0] x 4 must then be at most 128 bytes).  Elements
// outside the dims read as zero.
cudaError_t dfs_encode_tensor_map_3d_f32(CUtensorMap *map, const void *base, const uint64_t dims[3],
                                         const uint64_t strides_bytes[2], const uint32_t box[3],
                                         int swizzle128);

// 3-D tiled TMA load of one box, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
