// apsp_add_node_noalloc: node insertion on a caller-owned APSP matrix that
// allocates no memory at all.
//
// Some callers cannot allocate device memory when they need this operation:
// a request handler that must never block on cudaMalloc (it synchronises the
// whole device), code running inside a framework that hands out all device
// memory from its own fixed pool, or a caller with a hard memory budget.  For
// them this entry point keeps its scratch (the new node's masked weights and
// the two min-reduction vectors) in one file-scope device array of fixed size,
// loaded with the library and held by every GPU that loads it until the
// process exits.  The caller still owns and passes the matrix and the inputs.
//
// Host code must not hand the array's symbol to a kernel: on the host it is
// only a stand-in, not a device address.  The device address is fetched once
// per device with cudaGetSymbolAddress (with that device current) by the first
// call made on that device; that first call should therefore happen before
// any CUDA stream capture.
//
// Every call shares the same array and it keeps the previous call's contents,
// so each call re-initialises all of it before use.  Calls whose work
// overlaps on the GPU (different streams, or several host threads) race on
// the array and give undefined results; serialise them.
#include <cuda_runtime.h>

#include <mutex>

#include "apsp.h"
#include "kernels.cuh"

namespace {

constexpr int kMaxSlots = APSP_NOALLOC_MAX_SLOTS;
// w_in, w_out (masked weights) and vin, vout (ordered reduction keys).
static __device__ __align__(256) int32_t g_insert_scratch[4 * kMaxSlots];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int32_t *g_scratch_dev[kMaxDevices] = {};

apsp_status scratch_address(int32_t **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return APSP_E_CUDA;
    if (dev >= kMaxDevices) return APSP_E_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_insert_scratch) != cudaSuccess || !p) return APSP_E_CUDA;
        g_scratch_dev[dev] = (int32_t *)p;
    }
    *out = g_scratch_dev[dev];
    return APSP_OK;
}

// Masks the new node's weights (dead slots, p itself, and negative or NaN
// weights read as missing edges) and resets the reduction keys.
template <typename T>
__global__ void k_na_prep(const int32_t *alive, const T *in_w, const T *out_w, int span, int n_slots, int p,
                          T *w_in, T *w_out, int32_t *vin_k, int32_t *vout_k) {
    using M = apsp::MinPlus<T>;
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= span) return;
    T wi = M::inf(), wo = M::inf();
    if (j < n_slots && j != p && alive[j]) {
        T a = in_w[j], b = out_w[j];
        if (a >= (T)0) wi = a < M::inf() ? a : M::inf();   // false for NaN
        if (b >= (T)0) wo = b < M::inf() ? b : M::inf();
        if (wi == (T)0) wi = (T)0;
        if (wo == (T)0) wo = (T)0;
    }
    w_in[j] = wi;
    w_out[j] = wo;
    vin_k[j] = M::key(M::inf());
    vout_k[j] = M::key(M::inf());
}

// Theorem 3 sweep plus row / column p, without the weight matrix or the
// transposed copy (the caller owns only D).
template <typename T>
__global__ void __launch_bounds__(256) k_na_relax(T *D, int64_t ld, int span, int p, const int32_t *alive,
                                                  const int32_t *vin_k, const int32_t *vout_k) {
    using M = apsp::MinPlus<T>;
    using V4 = typename M::V4;
    for (int r = blockIdx.x; r < span; r += gridDim.x) {
        T *Dr = D + (int64_t)r * ld;
        if (r == p) {
            for (int c = threadIdx.x; c < span; c += blockDim.x) Dr[c] = c == p ? (T)0 : M::unkey(vout_k[c]);
            continue;
        }
        if (!alive[r]) continue;
        const T vi = M::unkey(vin_k[r]);
        if (M::finite(vi)) {
            for (int c4 = threadIdx.x; c4 < span / 4; c4 += blockDim.x) {
                V4 v = *reinterpret_cast<const V4 *>(Dr + 4 * c4);
                T dv[4] = {v.x, v.y, v.z, v.w};
                bool any = false;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    T cand = vi + M::unkey(vout_k[4 * c4 + e]);
                    if (cand < dv[e]) { dv[e] = cand; any = true; }
                }
                if (any) {
                    V4 nv; nv.x = dv[0]; nv.y = dv[1]; nv.z = dv[2]; nv.w = dv[3];
                    *reinterpret_cast<V4 *>(Dr + 4 * c4) = nv;
                }
            }
        }
        __syncthreads();  // the vector holding column p may have been written above
        if (threadIdx.x == 0) Dr[p] = vi;
    }
}

template <typename T>
apsp_status run(T *D, int64_t ld, int n_slots, const int32_t *alive, const T *in_w, const T *out_w, int p,
                cudaStream_t s) {
    int32_t *scr = nullptr;
    apsp_status st = scratch_address(&scr);
    if (st != APSP_OK) return st;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int span = n_slots;
    T *w_in = reinterpret_cast<T *>(scr);
    T *w_out = reinterpret_cast<T *>(scr + kMaxSlots);
    int32_t *vin_k = scr + 2 * kMaxSlots;
    int32_t *vout_k = scr + 3 * kMaxSlots;
    k_na_prep<T><<<(span + 255) / 256, 256, 0, s>>>(alive, in_w, out_w, span, n_slots, p, w_in, w_out, vin_k, vout_k);
    apsp::Dev<T> d{};
    d.D = D;
    d.ld = ld;
    d.span = span;
    d.alive = const_cast<int32_t *>(alive);
    d.w_in = w_in;
    d.w_out = w_out;
    d.vin_k = vin_k;
    d.vout_k = vout_k;
    const int bands = (span + apsp::INS_CB - 1) / apsp::INS_CB;
    int ranges = (3 * sms + bands - 1) / bands;
    ranges = ranges < 1 ? 1 : (ranges > (span + 7) / 8 ? (span + 7) / 8 : ranges);
    const int rows_per = (span + ranges - 1) / ranges;
    dim3 g(bands, (span + rows_per - 1) / rows_per);
    apsp::k_insert_reduce<T><<<g, 256, 0, s>>>(d, rows_per);
    k_na_relax<T><<<span < sms * 4 ? span : sms * 4, 256, 0, s>>>(D, ld, span, p, alive, vin_k, vout_k);
    return cudaGetLastError() == cudaSuccess ? APSP_OK : APSP_E_CUDA;
}

}  // namespace

extern "C" apsp_status apsp_add_node_noalloc(void *D, int64_t ld, int32_t n_slots, const int32_t *alive,
                                             apsp_dtype dtype, const void *in_w, const void *out_w, int32_t p,
                                             void *cuda_stream) {
    if (!D || !alive || !in_w || !out_w) return APSP_E_ARG;
    if (dtype != APSP_I32 && dtype != APSP_F32) return APSP_E_ARG;
    if (n_slots < 4 || n_slots % 4 != 0 || ld < n_slots || ld % 4 != 0) return APSP_E_ARG;
    if (n_slots > kMaxSlots) return APSP_E_CAPACITY;
    if (p < 0 || p >= n_slots) return APSP_E_NODE;
    if (((uintptr_t)D & 15u) != 0) return APSP_E_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (dtype == APSP_F32)
        return run<float>((float *)D, ld, n_slots, alive, (const float *)in_w, (const float *)out_w, p, s);
    return run<int32_t>((int32_t *)D, ld, n_slots, alive, (const int32_t *)in_w, (const int32_t *)out_w, p, s);
}
