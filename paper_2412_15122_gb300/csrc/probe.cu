// Measurement probes.  The issue rate of the min-plus step min(a + b, c) on the
// CUDA cores, the ceiling of the cold blocked Floyd-Warshall (whose inner
// loop is an 8 x 8 register tile of these steps per thread).  The probe runs
// the same 8 x 8 register tile with no memory traffic: each iteration does 64
// dependent-free add-min steps and moves the row operands by one (8 adds),
// so nothing is loop-invariant.
#include <cuda_runtime.h>

#include <algorithm>

#include "apsp.h"
#include "common.cuh"

namespace {

template <typename T> __global__ void __launch_bounds__(256) k_probe_addmin(T *out, int iters, T seed) {
    using M = apsp::MinPlus<T>;
    T a[8], b[8], acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        a[r] = seed + (T)((threadIdx.x + r) & 7);
        b[r] = seed + (T)(r * 3);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[r][q] = (T)(1 << 29);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[r][q] = M::add_min(a[r], b[q], acc[r][q]);
#pragma unroll
        for (int r = 0; r < 8; ++r) a[r] = a[r] + (T)1;
    }
    T m = acc[0][0];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 8; ++q) m = M::mn(m, acc[r][q]);
    if (m == (T)-7) out[0] = m;   // never true; keeps the work live
}

template <typename T> apsp_status probe(double *rate) {
    int dev = 0, sms = 1, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return APSP_E_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_addmin<T>, 256, 0) != cudaSuccess)
        return APSP_E_CUDA;
    const int grid = std::max(1, per_sm) * sms;
    const int iters = 4096;
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return APSP_E_NOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 0.f;
    apsp_status st = APSP_OK;
    for (int rep = 0; rep < 4; ++rep) {   // the first launch is a warm-up
        cudaEventRecord(e0);
        k_probe_addmin<T><<<grid, 256>>>(out, iters, (T)rep);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = APSP_E_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (st != APSP_OK) return st;
    if (cudaGetLastError() != cudaSuccess) return APSP_E_CUDA;
    *rate = (double)grid * 256.0 * iters * 64.0 / (best * 1e-3);
    return APSP_OK;
}

// L2 read probe: a buffer of a quarter of L2 (a power of two), warmed by a
// first launch, then read by every thread with 16-byte coalesced loads, 8 in
// flight, `reps` rounds; each load's index wraps with a mask.
__global__ void __launch_bounds__(256) k_probe_l2(const int4 *buf, int64_t mask4, int reps, int *out) {
    int acc = 0;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        int4 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = __ldcg(buf + ((tid + (int64_t)(r * 8 + q) * stride) & mask4));
#pragma unroll
        for (int q = 0; q < 8; ++q) acc ^= v[q].x ^ v[q].y ^ v[q].z ^ v[q].w;
    }
    if (acc == 0x7f3a5c1d) out[0] = acc;   // keeps the loads live
}

apsp_status probe_l2(double *gbs) {
    int dev = 0, sms = 1, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return APSP_E_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    int64_t bytes = 1 << 20;
    while (bytes * 2 <= (int64_t)l2 / 4) bytes *= 2;   // well inside L2
    int4 *buf = nullptr;
    int *out = nullptr;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) return APSP_E_NOMEM;
    if (cudaMalloc(&out, sizeof(int)) != cudaSuccess) {
        cudaFree(buf);
        return APSP_E_NOMEM;
    }
    cudaMemset(buf, 1, bytes);
    const int grid = 4 * sms, reps = 64;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 0.f;
    apsp_status st = APSP_OK;
    for (int rep = 0; rep < 4; ++rep) {   // the first launch warms L2
        cudaEventRecord(e0);
        k_probe_l2<<<grid, 256>>>(buf, bytes / 16 - 1, reps, out);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = APSP_E_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(out);
    if (st != APSP_OK) return st;
    if (cudaGetLastError() != cudaSuccess) return APSP_E_CUDA;
    *gbs = (double)grid * 256.0 * reps * 8.0 * 16.0 / (best * 1e-3) / 1e9;
    return APSP_OK;
}

// Self-test of the bounded grid barrier that the cooperative repair kernel
// uses: with `lose` set the last CTA leaves without arriving, so the others'
// wait can only end by its time limit, recording ERR_TIMEOUT.
__global__ void k_selftest_barrier(apsp::Ctl *ctl, int lose) {
    if (lose && blockIdx.x == gridDim.x - 1) return;
    apsp::grid_barrier(ctl, apsp::NoLeader{});
}

}  // namespace

extern "C" apsp_status apsp_selftest_barrier_timeout(int32_t lose_cta, int32_t *status_out) {
    if (!status_out) return APSP_E_ARG;
    apsp::Ctl *ctl = nullptr;
    if (cudaMalloc(&ctl, sizeof(apsp::Ctl)) != cudaSuccess) return APSP_E_NOMEM;
    cudaError_t e = cudaMemset(ctl, 0, sizeof(apsp::Ctl));
    int lose = lose_cta ? 1 : 0;
    void *args[] = {(void *)&ctl, (void *)&lose};
    if (e == cudaSuccess) e = cudaLaunchCooperativeKernel((void *)k_selftest_barrier, dim3(2), dim3(32), args, 0, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    uint32_t err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, &ctl->err, sizeof(err), cudaMemcpyDeviceToHost);
    cudaFree(ctl);
    if (e != cudaSuccess) return APSP_E_CUDA;
    *status_out = (err & apsp::ERR_TIMEOUT) ? APSP_E_TIMEOUT : APSP_OK;
    return APSP_OK;
}

extern "C" apsp_status apsp_probe_l2_read_gbs(double *gbs) {
    if (!gbs) return APSP_E_ARG;
    return probe_l2(gbs);
}

extern "C" apsp_status apsp_probe_addmin_rate(apsp_dtype dtype, double *pair_ops_per_s) {
    if (!pair_ops_per_s || (dtype != APSP_I32 && dtype != APSP_F32)) return APSP_E_ARG;
    return dtype == APSP_F32 ? probe<float>(pair_ops_per_s) : probe<int32_t>(pair_ops_per_s);
}
