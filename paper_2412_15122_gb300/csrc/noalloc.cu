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
// only a stand-in, not a device address.  Every call looks the device address
// up with cudaGetSymbolAddress on the current device (no allocation, no wait).
// The first lookup on a device, or the first after its context was reset,
// loads the library's device code; make that first call before any CUDA
// stream capture.
//
// Every call shares the same array and it keeps the previous call's contents,
// so each call re-initialises all of it before use.  Calls whose work
// overlaps on the GPU (different streams, or several host threads) race on
// the array and give undefined results; serialise them.
//
// Only live slots other than p are read: row and column p and every dead
// slot's row and column may hold anything (INT32_MAX, negative values, NaN)
// and do not reach the result.  Row p is written over all n_slots columns
// (missing at dead slots), column p at live rows; every other entry of a dead
// slot keeps its contents.
#include <cuda_runtime.h>

#include "apsp.h"
#include "kernels.cuh"

namespace {

constexpr int kMaxSlots = APSP_NOALLOC_MAX_SLOTS;
// w_in, w_out (masked weights) and vin, vout (ordered reduction keys).
static __device__ __align__(256) int32_t g_insert_scratch[4 * kMaxSlots];

apsp_status scratch_address(int32_t **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_insert_scratch) != cudaSuccess || !p) return APSP_E_CUDA;
    *out = (int32_t *)p;
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

// An entry of D as the reductions read it: a live column other than p keeps
// its value (int32 values >= INF read as missing), any other column is
// missing, whatever the caller's matrix holds there.
template <typename T> __device__ __forceinline__ T na_entry(T x, bool live);
template <> __device__ __forceinline__ int32_t na_entry<int32_t>(int32_t x, bool live) {
    return live ? min(x, apsp::INF_I32) : apsp::INF_I32;
}
template <> __device__ __forceinline__ float na_entry<float>(float x, bool live) {
    return live ? x : apsp::MinPlus<float>::inf();
}

constexpr int NA_CB = 512;   // columns per CTA: 16 per lane, as 4 vectors of 4

// Corollaries 1 and 2 in one pass over the live block of D:
//   out[c] = min over live t != p of w(p, t) + D[t][c]   (column reduction)
//   in[t]  = min over live c != p of D[t][c] + w(c, p)   (row reduction)
// Rows and columns that are dead or p are skipped by mask, so the caller's
// values there never enter a sum.  Grid: column bands x row ranges; partial
// minima meet through atomicMin on ordered keys.
template <typename T>
__global__ void __launch_bounds__(256) k_na_reduce(const T *D, int64_t ld, int span, int p, const int32_t *alive,
                                                   const T *w_in, const T *w_out, int32_t *vin_k, int32_t *vout_k,
                                                   int rows_per_cta) {
    using M = apsp::MinPlus<T>;
    using V4 = typename M::V4;
    __shared__ T red[8][NA_CB];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c0 = blockIdx.x * NA_CB;
    const int r0 = blockIdx.y * rows_per_cta;
    const int r1 = min(span, r0 + rows_per_cta);
    T win[16], col[16];
    bool cok[16], vin4[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        vin4[q] = c0 + q * 128 + lane * 4 < span;   // span is a multiple of 4
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = c0 + q * 128 + lane * 4 + e;
            cok[q * 4 + e] = c < span && c != p && alive[c] != 0;
            win[q * 4 + e] = c < span ? w_in[c] : M::inf();
            col[q * 4 + e] = M::inf();
        }
    }
    for (int row = r0 + w; row < r1; row += 8) {
        if (row == p || alive[row] == 0) continue;   // uniform across the warp
        const T wo = w_out[row];
        const T *Dr = D + (int64_t)row * ld + c0 + lane * 4;
        V4 v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (vin4[q]) v[q] = *reinterpret_cast<const V4 *>(Dr + q * 128);
        T racc = M::inf();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!vin4[q]) continue;
            const T e4[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const T x = na_entry<T>(e4[e], cok[q * 4 + e]);
                col[q * 4 + e] = M::add_min(wo, x, col[q * 4 + e]);
                racc = M::add_min(x, win[q * 4 + e], racc);
            }
        }
        racc = apsp::warp_min(racc);
        if (lane == 0 && M::finite(racc)) atomicMin(&vin_k[row], M::key(racc));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) red[w][q * 128 + lane * 4 + e] = col[q * 4 + e];
    __syncthreads();
    for (int c = threadIdx.x; c < NA_CB; c += blockDim.x) {
        T m = red[0][c];
#pragma unroll
        for (int k = 1; k < 8; ++k) m = M::mn(m, red[k][c]);
        if (c0 + c < span && M::finite(m)) atomicMin(&vout_k[c0 + c], M::key(m));
    }
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
                    // missing for dead columns and p: those entries stay as they are
                    const T o = M::unkey(vout_k[4 * c4 + e]);
                    if (!M::finite(o)) continue;
                    const T cand = M::add(vi, o);
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
    const int bands = (span + NA_CB - 1) / NA_CB;
    int ranges = (3 * sms + bands - 1) / bands;
    ranges = ranges < 1 ? 1 : (ranges > (span + 7) / 8 ? (span + 7) / 8 : ranges);
    const int rows_per = (span + ranges - 1) / ranges;
    dim3 g(bands, (span + rows_per - 1) / rows_per);
    k_na_reduce<T><<<g, 256, 0, s>>>(D, ld, span, p, alive, w_in, w_out, vin_k, vout_k, rows_per);
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
