// FMA-rate probe (include/dfsnufft_probe.h): independent FMA chains per thread,
// enough CTAs to fill every SM, timed with CUDA events.
#include "common.cuh"
#include "dfsnufft_probe.h"
#include "tma.cuh"

namespace {

template <typename R>
__global__ void __launch_bounds__(256) k_fma_chains(R *sink, int iters, R a, R b) {
    R x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (R)(threadIdx.x + k) * (R)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
        }
    }
    R s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == (R)-12345) sink[blockIdx.x] = s;   // keeps the chains live
}

template <typename R>
int probe(double target_ms, double *out) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
        return DFSNUFFT_ERR_CUDA;
    R *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(R) * 4096)) return DFSNUFFT_ERR_OOM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = sms * 8, threads = 256;
    int iters = 64;
    double flops = 0, ms_best = 0;
    int rc = DFSNUFFT_OK;
    for (int round = 0; round < 12; ++round) {
        cudaEventRecord(e0, 0);
        k_fma_chains<R><<<blocks, threads>>>(sink, iters, (R)0.9999999, (R)1e-7);
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = DFSNUFFT_ERR_CUDA;
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < 0.5 * target_ms && iters < (1 << 24)) {
            iters = (int)(iters * (ms > 0.01 ? 0.9 * target_ms / ms : 16.0));
            if (iters < 1) iters = 1;
            continue;
        }
        double f = 2.0 * 16.0 * 8.0 * (double)iters * blocks * threads;
        if (flops == 0 || f / ms > flops / ms_best) {
            flops = f;
            ms_best = ms;
        }
        if (round >= 6) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc) return rc;
    if (ms_best <= 0) return DFSNUFFT_ERR_CUDA;
    *out = flops / (ms_best * 1e-3);
    return DFSNUFFT_OK;
}

}  // namespace

extern "C" int dfsnufft_probe_fma_rate(int dtype, double target_ms, double *flops_per_s) {
    if (!flops_per_s || !(target_ms > 0)) return DFSNUFFT_ERR_INVALID_ARG;
    if (dtype == DFSNUFFT_F64) return probe<double>(target_ms, flops_per_s);
    if (dtype == DFSNUFFT_F32) return probe<float>(target_ms, flops_per_s);
    return DFSNUFFT_ERR_INVALID_ARG;
}

namespace {

// One thread waits, bounded, on a barrier no one arrives on.
__global__ void k_wait_nobody(long long cycles, int *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    if (!mbar_wait_bounded(&bar, 0, cycles)) atomicExch(status, DFS_STATUS_TIMEOUT);
}

}  // namespace

extern "C" int dfsnufft_selftest_wait_timeout(long long cycles, int *device_status,
                                              double *elapsed_ms) {
    if (!device_status || cycles < 1 || cycles > 4000000000LL) return DFSNUFFT_ERR_INVALID_ARG;
    int *d = nullptr;
    if (cudaMalloc(&d, sizeof(int))) return DFSNUFFT_ERR_OOM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = DFSNUFFT_OK;
    float ms = 0;
    if (cudaMemset(d, 0, sizeof(int)) || cudaEventCreate(&e0) || cudaEventCreate(&e1) ||
        cudaEventRecord(e0, 0)) {
        rc = DFSNUFFT_ERR_CUDA;
    } else {
        k_wait_nobody<<<1, 32>>>(cycles, d);
        if (cudaGetLastError() || cudaEventRecord(e1, 0) || cudaEventSynchronize(e1) ||
            cudaEventElapsedTime(&ms, e0, e1) ||
            cudaMemcpy(device_status, d, sizeof(int), cudaMemcpyDeviceToHost))
            rc = DFSNUFFT_ERR_CUDA;
    }
    if (elapsed_ms) *elapsed_ms = ms;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d);
    return rc;
}
