// Kernels of the warm-start APSP update path (sm_103a).
//
// Data layout (device, per graph): W, D and (directed graphs) DT = D^T, each a
// row-major ld x ld matrix (ld a multiple of 128, rows 512-byte aligned), plus
// per-slot vectors of ld elements.  `span` (a multiple of 32, <= ld) bounds
// the slots ever used; rows / columns past the live ones hold "missing" so
// every sweep can run on whole 128-bit vectors without tail handling.
//
// Every sweep reads rows with 128-bit coalesced loads and writes only the
// 16-byte vectors that changed; the transposed copy DT receives the changed
// entries as scattered 4-byte stores (few per update) and gives the column
// access that detection and re-relaxation need as contiguous rows.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "fw_tiles.cuh"
#include "mlp.cuh"

namespace apsp {

// Host callbacks around each launch (launch counting and CUDA-event timing).
struct Hook {
    void (*pre)(void *, const char *);
    void (*post)(void *, const char *);
    void *ctx;
    void begin(const char *n) const { if (pre) pre(ctx, n); }
    void end(const char *n) const { if (post) post(ctx, n); }
};

template <typename T> struct Dev {
    T *W, *D, *DT;            // DT == nullptr for undirected graphs (D is symmetric)
    int64_t ld;
    int span;
    int undirected;
    int32_t *alive;           // 1 = live slot
    T *w_in, *w_out;          // masked weights of a new node
    int32_t *vin_k, *vout_k;  // Corollary 2 / Corollary 1 vectors as ordered keys
    T *x, *x2, *y, *y2;       // staged rows / columns of the current update
    int32_t *rlist;           // prepass row list
    int4 *hrows;              // detection: flagged rows (row, first unit, units, batch mask)
    int4 *hunits;             // detection: flagged units (row, batch, row entry, position in the row)
    int4 *hralloc;            // detection: per flagged row (first item, first unit, pairs)
    int32_t *rowcnt;          // detection: listed pairs per (row, batch), DET_MAXB a row
    uint32_t *bmask;          // detection: exact mask per (row, batch), 32 words (one per lane), bmask_nb batches a row
    int32_t bmask_nb;
    long long *hbase;         // detection: first pair slot per unit (-1: none)
    int4 *items;              // (row, first pair, pair count | row's pair count << 8, row's first pair)
    int32_t *icand;           // node insertion: candidate rows of Corollary 1 [0, ld), columns of Corollary 2 [ld, 2 ld)
    int4 *p1u;                // first-pass units: (row, first pair, pairs <= P1_PAIRS, 0)
    int32_t *pairs;           // affected column per pair, grouped by row (columns ascending)
    int32_t *pmin;            // per pair: first-pass minimum as an ordered key
    uint8_t *pstamp;          // per pair: last pass that lowered it (0: none yet)
    uint8_t *rstamp;          // per row (ld): last pass that lowered one of its pairs
    int32_t *units;           // work units of passes >= 2: item | intermediate segment << 24
    Ctl *ctl;
    int64_t pair_cap;
    int32_t item_cap;
    int32_t unit_cap;
    int32_t p1u_cap;
};

template <typename T> __device__ __forceinline__ T col_src(const Dev<T> &d, int row_of_T, int i) {
    // D[i][row_of_T] read through the transposed copy (contiguous in i)
    return d.DT ? d.DT[(int64_t)row_of_T * d.ld + i] : d.D[(int64_t)row_of_T * d.ld + i];
}

template <typename T> __device__ __forceinline__ T warp_min(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = MinPlus<T>::mn(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Append flagged slot i to `list` with one atomic per warp.
__device__ __forceinline__ void warp_append(bool flag, int i, int32_t *list, int32_t *count) {
    unsigned m = __ballot_sync(0xffffffffu, flag);
    if (!m) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (flag) list[base + __popc(m & ((1u << lane) - 1))] = i;
}

// Rows of up to ROW_NV * 1024 elements are swept by 256 threads that first
// load their whole share of the row (ROW_NV 16-byte vectors each) so every
// load of the row is in flight at once, then consume it.
constexpr int ROW_NV = 20;
static_assert(ROW_NV * 1024 >= 18432, "a row of the largest capacity must fit");

template <typename V4>
__device__ __forceinline__ void load_row_regs(V4 (&rv)[ROW_NV], const V4 *row, int nv4) {
#pragma unroll
    for (int k = 0; k < ROW_NV; ++k) {
        const int c4 = threadIdx.x + 256 * k;
        if (c4 < nv4) rv[k] = row[c4];
    }
}

// Warp-per-row sweeps.  A warp walks a row in batches of SWEEP_B 16-byte
// vectors per lane (SWEEP_B * 512 bytes in flight per warp), calling
// f(c4, v) for every vector; no CTA-wide barriers are involved.
constexpr int SWEEP_B = 8;

template <typename V4, int B = SWEEP_B, typename F>
__device__ __forceinline__ void warp_row_sweep(const V4 *row, int nv4, F &&f) {
    const int lane = threadIdx.x & 31;
    for (int base = 0; base < nv4; base += 32 * B) {
        V4 v[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int c4 = base + b * 32 + lane;
            if (c4 < nv4) v[b] = __ldcs(row + c4);
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int c4 = base + b * 32 + lane;
            if (c4 < nv4) f(c4, v[b]);
        }
    }
}

__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Exclusive prefix of v over the lanes of a warp; *total = sum over the warp.
__device__ __forceinline__ int warp_exclusive_scan(int v, int *total) {
    const int lane = threadIdx.x & 31;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    *total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// Stages a vector of `span` elements into shared memory (all threads of the
// CTA); each thread issues up to 8 loads before its first store.
template <typename T> __device__ __forceinline__ void stage_vec(T *dst, const T *src, int span) {
    using V4 = typename MinPlus<T>::V4;
    const int nv = span / 4;
    for (int base = 0; base < nv; base += 8 * (int)blockDim.x) {
        V4 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int c4 = base + k * blockDim.x + threadIdx.x;
            if (c4 < nv) v[k] = __ldcg(reinterpret_cast<const V4 *>(src) + c4);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int c4 = base + k * blockDim.x + threadIdx.x;
            if (c4 < nv) reinterpret_cast<V4 *>(dst)[c4] = v[k];
        }
    }
}

// --------------------------------------------------------------------------
// Small utilities
// --------------------------------------------------------------------------

template <typename T> __global__ void k_fill(T *p, T v, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// Normalise an n x n input block in place: missing -> INF, diagonal 0,
// -0.0 -> +0.0; flag negative weights, NaN and (undirected) asymmetry.
template <typename T> __device__ __forceinline__ T sanitize_val(T w, uint32_t &err) {
    if constexpr (std::is_same<T, int32_t>::value) {
        if (w < 0) err |= ERR_NEGATIVE;
        return w > (T)INF_I32 ? (T)INF_I32 : w;
    } else {
        if (w != w) err |= ERR_NAN;
        else if (w < (T)0) err |= ERR_NEGATIVE;
        return w == (T)0 ? (T)0 : w;
    }
}

template <typename T> __global__ void k_sanitize(T *M, int64_t ld, int n, int check_sym, Ctl *ctl) {
    uint32_t err = 0;
    int64_t tot = (int64_t)n * n;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(idx / n), j = (int)(idx % n);
        T w = sanitize_val<T>(M[(int64_t)i * ld + j], err);
        if (i == j) w = (T)0;
        if (check_sym && i != j) {
            uint32_t e2 = 0;
            T w2 = sanitize_val<T>(M[(int64_t)j * ld + i], e2);
            if (!(w2 == w)) err |= ERR_NOT_SYMMETRIC;
        }
        M[(int64_t)i * ld + j] = w;
    }
    if (err) atomicOr(&ctl->err, err);
}

// DT[j][i] = D[i][j] for i, j < span (span a multiple of 32).
template <typename T> __global__ void k_transpose(const T *__restrict__ D, T *__restrict__ DT, int64_t ld, int span) {
    __shared__ T tile[32][33];
    int tiles = span / 32;
    for (int t = blockIdx.x; t < tiles * tiles; t += gridDim.x) {
        int bi = t / tiles, bj = t % tiles;
        for (int r = threadIdx.y; r < 32; r += blockDim.y)
            tile[r][threadIdx.x] = D[(int64_t)(bi * 32 + r) * ld + bj * 32 + threadIdx.x];
        __syncthreads();
        for (int r = threadIdx.y; r < 32; r += blockDim.y)
            DT[(int64_t)(bj * 32 + r) * ld + bi * 32 + threadIdx.x] = tile[threadIdx.x][r];
        __syncthreads();
    }
}

// --------------------------------------------------------------------------
// Floyd-Warshall, one launch per phase (cold solver at init / recompute)
// --------------------------------------------------------------------------

template <typename T, typename M = MinPlus<T>>
__global__ void __launch_bounds__(FW_THREADS) k_fw_p1(T *D, int64_t ld, int kb) {
    __shared__ FwDiagSmem<T> sm;
    fw_close_diag<T, M>(D + (int64_t)kb * FW_B * ld + (int64_t)kb * FW_B, ld, sm);
}

template <typename T, typename M = MinPlus<T>>
__global__ void __launch_bounds__(FW_THREADS, 2) k_fw_p2(T *D, int64_t ld, int kb, int nb) {
    __shared__ FwSmem<T> sm;
    fw_phase2_tile<T, M>(D, ld, kb, nb, blockIdx.x, sm);
}

template <typename T, typename M = MinPlus<T>>
__global__ void __launch_bounds__(FW_THREADS, 2) k_fw_p3(T *D, int64_t ld, int kb, int nb) {
    __shared__ FwSmem<T> sm;
    fw_phase3_tile<T, M>(D, ld, kb, nb, blockIdx.x, sm);
}

__device__ __forceinline__ int32_t max_of(int32_t a, int32_t b) { return max(a, b); }
__device__ __forceinline__ float max_of(float a, float b) { return fmaxf(a, b); }

// --------------------------------------------------------------------------
// Adding a node p (Section 3.1)
// --------------------------------------------------------------------------

// Which rows (columns) of D can attain the new node's minima.  With t0 the
// slot of the lightest out-edge of p and E0 = max over live j of D[t0][j],
// every column j has out[j] <= w(p, t0) + D[t0][j] <= w(p, t0) + E0, while a
// row t contributes w(p, t) + D[t][j] >= w(p, t) (D >= 0).  Rows with
// w(p, t) > w(p, t0) + E0 therefore never attain a minimum and Corollary 1
// needs only the rows with w(p, t) <= w(p, t0) + E0; likewise Corollary 2
// needs only the columns r with w(r, p) <= w(r1, p) + E1, r1 the lightest
// in-edge and E1 = max over live i of D[i][r1].  The comparisons are exact
// (int64 for int32 weights; for fp32 the bound is rounded up, which keeps a
// superset of the rows) and rounding is monotone, so the minima over
// the candidates are bit-identical to the minima over all rows.  When some
// live node is unreachable the bound is infinite and every row stays a
// candidate.  One CTA (k_insert_cand) builds both lists.
constexpr int INS_CAND_THREADS = 1024;   // the one block of k_insert_cand

// Bound w(p, t0) + E0 of insert_candidates and its test, without fp64 (slow on
// this GPU): int64 for int32 weights, rounded up for fp32.
template <typename T> struct CandBound;
template <> struct CandBound<int32_t> {
    using B = long long;
    __device__ static B make(bool none, int32_t w, int32_t e) {
        return none ? -1ll : (e >= INF_I32 ? 0x7fffffffffffffffll : (B)w + (B)e);
    }
    __device__ static bool keep(int32_t w, B t) { return (B)w <= t; }
};
template <> struct CandBound<float> {
    using B = float;
    __device__ static B make(bool none, float w, float e) { return none ? -1.0f : __fadd_ru(w, e); }
    __device__ static bool keep(float w, B t) { return w <= t; }
};

template <typename T>
__device__ void insert_candidates(const Dev<T> &d, int p) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    constexpr int U = 3;   // vectors per thread held at once (span <= 12288 in one round)
    __shared__ int nsel[2];
    __shared__ T emax[2][INS_CAND_THREADS / 32];
    const int nv = d.span / 4, lane = threadIdx.x & 31, w = threadIdx.x >> 5;   // span is a multiple of 32
    const unsigned long long ao = *(volatile const unsigned long long *)&d.ctl->ins_amin_out;
    const unsigned long long ai = *(volatile const unsigned long long *)&d.ctl->ins_amin_in;
    const int t0 = ao ? (int)(uint32_t)(~ao) : -1, r1 = ai ? (int)(uint32_t)(~ai) : -1;
    if (threadIdx.x < 2) nsel[threadIdx.x] = 0;
    const V4 *row0 = reinterpret_cast<const V4 *>(d.D + (int64_t)max(t0, 0) * d.ld);
    const V4 *col1 = reinterpret_cast<const V4 *>((d.DT ? d.DT : d.D) + (int64_t)max(r1, 0) * d.ld);
    const int4 *al4 = reinterpret_cast<const int4 *>(d.alive);
    const V4 *wo4 = reinterpret_cast<const V4 *>(d.w_out);
    const V4 *wi4 = reinterpret_cast<const V4 *>(d.w_in);
    // the two lightest weights, in flight with the first vectors
    const T wt0 = __ldcg(d.w_out + max(t0, 0)), wr1 = __ldcg(d.w_in + max(r1, 0));
    T e0 = (T)0, e1 = (T)0;
    // E0 = max over live j of D[t0][j], E1 = max over live i of D[i][r1];
    // U vectors of each array per thread are in flight together
    for (int c0 = 0; c0 < nv; c0 += U * (int)blockDim.x) {
        int4 a[U];
        V4 x[U], y[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c4 = c0 + u * blockDim.x + threadIdx.x;
            if (c4 < nv) {
                a[u] = __ldcg(al4 + c4);
                x[u] = __ldcg(row0 + c4);
                y[u] = __ldcg(col1 + c4);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c4 = c0 + u * blockDim.x + threadIdx.x;
            if (c4 >= nv) continue;
            const int j = 4 * c4;
            const bool l0 = a[u].x && j != p, l1 = a[u].y && j + 1 != p, l2 = a[u].z && j + 2 != p, l3 = a[u].w && j + 3 != p;
            e0 = max_of(max_of(max_of(e0, l0 ? x[u].x : (T)0), max_of(l1 ? x[u].y : (T)0, l2 ? x[u].z : (T)0)),
                        l3 ? x[u].w : (T)0);
            e1 = max_of(max_of(max_of(e1, l0 ? y[u].x : (T)0), max_of(l1 ? y[u].y : (T)0, l2 ? y[u].z : (T)0)),
                        l3 ? y[u].w : (T)0);
        }
    }
    // the weights the compaction tests, in flight during the reduction
    V4 wo[U], wi[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int c4 = u * blockDim.x + threadIdx.x;
        if (c4 < nv) {
            wo[u] = __ldcg(wo4 + c4);
            wi[u] = __ldcg(wi4 + c4);
        }
    }
    if (t0 < 0) e0 = (T)0;
    if (r1 < 0) e1 = (T)0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e0 = max_of(e0, __shfl_xor_sync(0xffffffffu, e0, o));
        e1 = max_of(e1, __shfl_xor_sync(0xffffffffu, e1, o));
    }
    if (lane == 0) {
        emax[0][w] = e0;
        emax[1][w] = e1;
    }
    __syncthreads();
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
        e0 = max_of(e0, emax[0][k]);
        e1 = max_of(e1, emax[1][k]);
    }
    using CB = CandBound<T>;
    const typename CB::B thr_o = CB::make(t0 < 0, wt0, e0), thr_i = CB::make(r1 < 0, wr1, e1);
    const unsigned below = (1u << lane) - 1u;
    for (int c0 = 0; c0 < nv; c0 += U * (int)blockDim.x) {
        if (c0 > 0) {   // spans above U * 4 * blockDim.x slots
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int c4 = c0 + u * blockDim.x + threadIdx.x;
                if (c4 < nv) {
                    wo[u] = __ldcg(wo4 + c4);
                    wi[u] = __ldcg(wi4 + c4);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c4 = c0 + u * blockDim.x + threadIdx.x;
            const bool in = c4 < nv;
            const T wov[4] = {wo[u].x, wo[u].y, wo[u].z, wo[u].w}, wiv[4] = {wi[u].x, wi[u].y, wi[u].z, wi[u].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const bool so = in && M::finite(wov[e]) && CB::keep(wov[e], thr_o);
                const bool si = in && M::finite(wiv[e]) && CB::keep(wiv[e], thr_i);
                const unsigned bo = __ballot_sync(0xffffffffu, so), bi = __ballot_sync(0xffffffffu, si);
                if (!(bo | bi)) continue;
                int baseo = 0, basei = 0;
                if (lane == 0) {
                    if (bo) baseo = atomicAdd(&nsel[0], __popc(bo));
                    if (bi) basei = atomicAdd(&nsel[1], __popc(bi));
                }
                baseo = __shfl_sync(0xffffffffu, baseo, 0);
                basei = __shfl_sync(0xffffffffu, basei, 0);
                if (so) d.icand[baseo + __popc(bo & below)] = 4 * c4 + e;
                if (si) d.icand[d.ld + basei + __popc(bi & below)] = 4 * c4 + e;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        d.ctl->ins_nout = nsel[0];
        d.ctl->ins_nin = nsel[1];
        // the candidates' rows and columns cost at most an eighth of a full pass
        d.ctl->ins_narrow = (int64_t)(nsel[0] + nsel[1]) * 8 <= (int64_t)d.span;
    }
}

// Mask the new node's weights (dead slots and p itself -> missing), validate
// them, and reset the two reduction vectors.  With `cand` (min-plus graphs),
// also the argmin of each weight vector, for k_insert_cand.  With `fetch` (a
// device view of mapped host memory, 2 * cap elements), also copy the raw
// vectors there for the host's weight mirror, so a device-input add needs no
// separate device-to-host copies.
template <typename T>
__global__ void k_insert_prep(Dev<T> d, const T *in_raw, const T *out_raw, int cap, int p, int cand, T *fetch) {
    pdl_enter();
    using M = MinPlus<T>;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (fetch)
        for (int t = j; t < cap; t += gridDim.x * blockDim.x) {
            fetch[t] = in_raw[t];
            fetch[cap + t] = out_raw[t];
        }
    uint32_t err = 0;
    T wi = M::inf(), wo = M::inf();
    if (j < d.span) {
        if (j < cap && j != p && d.alive[j]) {
            wi = sanitize_val<T>(in_raw[j], err);
            wo = sanitize_val<T>(out_raw[j], err);
            if (err) { wi = M::inf(); wo = M::inf(); }
        }
        d.w_in[j] = wi;
        d.w_out[j] = wo;
        d.vin_k[j] = M::key(M::inf());
        d.vout_k[j] = M::key(M::inf());
        if (err) atomicOr(&d.ctl->err, err);
    }
    if (!cand) return;
    unsigned long long ko = M::finite(wo) ? ~(((unsigned long long)(uint32_t)M::key(wo) << 32) | (uint32_t)j) : 0ull;
    unsigned long long ki = M::finite(wi) ? ~(((unsigned long long)(uint32_t)M::key(wi) << 32) | (uint32_t)j) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ko = max(ko, __shfl_xor_sync(0xffffffffu, ko, o));
        ki = max(ki, __shfl_xor_sync(0xffffffffu, ki, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (ko) atomicMax(&d.ctl->ins_amin_out, ko);
        if (ki) atomicMax(&d.ctl->ins_amin_in, ki);
    }
}

// The reduction's candidates (insert_candidates), one CTA of INS_CAND_THREADS.
template <typename T>
__global__ void __launch_bounds__(INS_CAND_THREADS) k_insert_cand(Dev<T> d, int p) {
    pdl_enter();
    insert_candidates<T>(d, p);
}

// One pass over D computing both vectors of the new node (when the
// candidate bound leaves too many rows):
//   out[r] = min_t w(p, t) + D[t][r]     (Corollary 1, column reduction)
//   in[t]  = min_r D[t][r] + w(r, p)     (Corollary 2, row reduction)
// Grid: (column band of INS_CB columns) x (row range); the launcher picks the
// number of row ranges so the grid is one wave over the SMs.  Each lane owns
// 16 columns; partial results meet in global memory through atomicMin on
// ordered keys (one per row per band, one per column per row range).
constexpr int INS_CB = 512;

// The same two reductions over the candidates only (insert_candidates):
// CTA (band, k) takes candidates k, k + gridDim.y, ... (a warp each); a
// candidate row t adds w(p, t) + D[t][band] to out[band], a candidate column
// r adds D[band][r] + w(r, p) (row r of Dt) to in[band].  Partial minima
// meet through atomicMin on ordered keys as in the full pass.
template <typename T>
__device__ void insert_reduce_candidates(const Dev<T> &d, T (*red)[INS_CB]) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c0 = blockIdx.x * INS_CB;
    const int nout = *(volatile const int32_t *)&d.ctl->ins_nout;
    const int nc = nout + *(volatile const int32_t *)&d.ctl->ins_nin;
    T ao[16], ai[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) ao[e] = ai[e] = M::inf();
    for (int k = blockIdx.y + gridDim.y * w; k < nc; k += gridDim.y * (blockDim.x >> 5)) {
        const bool out = k < nout;
        const int s = out ? __ldcg(d.icand + k) : __ldcg(d.icand + d.ld + (k - nout));
        const T wt = out ? __ldcg(d.w_out + s) : __ldcg(d.w_in + s);
        const T *src = (out || !d.DT ? d.D : d.DT) + (int64_t)s * d.ld + c0 + lane * 4;
        V4 v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (c0 + q * 128 + lane * 4 < d.span) v[q] = __ldcg(reinterpret_cast<const V4 *>(src + q * 128));
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (c0 + q * 128 + lane * 4 >= d.span) continue;
            const T e4[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (out) ao[q * 4 + e] = M::add_min(wt, e4[e], ao[q * 4 + e]);
                else ai[q * 4 + e] = M::add_min(e4[e], wt, ai[q * 4 + e]);
            }
        }
    }
    for (int side = 0; side < 2; ++side) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int e = 0; e < 4; ++e) red[w][q * 128 + lane * 4 + e] = side ? ai[q * 4 + e] : ao[q * 4 + e];
        __syncthreads();
        for (int c = threadIdx.x; c < INS_CB; c += blockDim.x) {
            T m = red[0][c];
#pragma unroll
            for (int k = 1; k < 8; ++k) m = M::mn(m, red[k][c]);
            if (c0 + c < d.span && M::finite(m)) atomicMin(side ? &d.vin_k[c0 + c] : &d.vout_k[c0 + c], M::key(m));
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_insert_reduce(Dev<T> d, int rows_per_cta) {
    pdl_enter();
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    __shared__ T red[8][INS_CB];
    if (*(volatile const int32_t *)&d.ctl->ins_narrow) {
        insert_reduce_candidates<T>(d, red);
        return;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c0 = blockIdx.x * INS_CB;
    const int r0 = blockIdx.y * rows_per_cta;
    const int r1 = min(d.span, r0 + rows_per_cta);
    T win[16], col[16];
    bool cin[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        cin[q] = c0 + q * 128 + lane * 4 < d.span;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            int c = c0 + q * 128 + lane * 4 + e;
            win[q * 4 + e] = c < d.span ? d.w_in[c] : M::inf();
            col[q * 4 + e] = M::inf();
        }
    }
    // Two rows per warp and step, all eight loads issued before any use.  No
    // per-row liveness test: a dead row has w_out = missing and an all-missing
    // row of D, so it changes neither reduction.
    for (int row = r0 + w; row < r1; row += 16) {
        const int rows2 = row + 8 < r1 ? 2 : 1;
        V4 v[2][4];
        T wo[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            wo[h] = M::inf();
            if (h < rows2) {
                const int r = row + 8 * h;
                wo[h] = d.w_out[r];
                const T *Dr = d.D + (int64_t)r * d.ld + c0 + lane * 4;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (cin[q]) v[h][q] = *reinterpret_cast<const V4 *>(Dr + q * 128);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h >= rows2) break;
            T racc = M::inf();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (!cin[q]) continue;
                T e4[4] = {v[h][q].x, v[h][q].y, v[h][q].z, v[h][q].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    col[q * 4 + e] = M::add_min(wo[h], e4[e], col[q * 4 + e]);
                    racc = M::add_min(e4[e], win[q * 4 + e], racc);
                }
            }
            racc = warp_min(racc);
            if (lane == 0 && M::finite(racc)) atomicMin(&d.vin_k[row + 8 * h], M::key(racc));
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) red[w][q * 128 + lane * 4 + e] = col[q * 4 + e];
    __syncthreads();
    for (int c = threadIdx.x; c < INS_CB; c += blockDim.x) {
        T m = red[0][c];
#pragma unroll
        for (int k = 1; k < 8; ++k) m = M::mn(m, red[k][c]);
        if (c0 + c < d.span && M::finite(m)) atomicMin(&d.vout_k[c0 + c], M::key(m));
    }
}

// Row p = out (Corollary 1), column p = in (Corollary 2), D[p][p] = 0, the
// weights of p, and p becomes live (entry c of each).
template <typename T>
__device__ __forceinline__ void insert_finish_entry(const Dev<T> &d, int p, int c) {
    using M = MinPlus<T>;
    const T o = c == p ? (T)0 : M::unkey(d.vout_k[c]);
    const T in = c == p ? (T)0 : M::unkey(d.vin_k[c]);
    d.D[(int64_t)p * d.ld + c] = o;
    d.D[(int64_t)c * d.ld + p] = in;
    d.W[(int64_t)p * d.ld + c] = c == p ? (T)0 : d.w_out[c];
    d.W[(int64_t)c * d.ld + p] = c == p ? (T)0 : d.w_in[c];
    if (d.DT) {
        d.DT[(int64_t)c * d.ld + p] = o;
        d.DT[(int64_t)p * d.ld + c] = in;
    }
    if (c == p) d.alive[p] = 1;
}

// Theorem 3 sweep: D[i][j] = min(D[i][j], in[i] + out[j]).  One warp per
// row; out[] is staged once per CTA in shared memory.  Each lane streams 8
// vectors at a time and only builds a 32-bit mask of the entries that
// improve; those few entries are then written one by one (the new value is
// in[i] + out[j]; the row data is no longer needed).  A dead row and p
// itself have in[] = missing, so one load decides whether a row is swept.
// Row p and column p are never improved by the sweep (their candidates are
// missing) and row p is never read by it, so the same launch writes them
// (insert_finish_entry) while the rows are swept.
template <typename T>
__global__ void __launch_bounds__(256, 4) k_insert_relax(Dev<T> d, int p, int ranges, int rows_per) {
    pdl_enter();
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int span = d.span;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < span; c += gridDim.x * blockDim.x)
        insert_finish_entry<T>(d, p, c);
    // vout_k holds ordered keys whose bit patterns are the values themselves
    T *so = reinterpret_cast<T *>(smem_raw);
    V4 *so4w = reinterpret_cast<V4 *>(smem_raw);
    const V4 *src4 = reinterpret_cast<const V4 *>(d.vout_k);
    const int nv4 = span / 4;
    for (int c = threadIdx.x; c < nv4; c += blockDim.x) so4w[c] = src4[c];
    __syncthreads();
    const V4 *so4 = reinterpret_cast<const V4 *>(so);
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    // Row order: k_insert_reduce read every one of its `ranges` row ranges in
    // ascending order at once, so its last rows -- the ends of all ranges --
    // are what L2 still holds.  Take those first: k walks the ranges
    // interleaved, from each range's end backwards.
    const int cover = ranges * rows_per;
    for (int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < cover; k += nwarps) {
        const int row = (k % ranges) * rows_per + (rows_per - 1 - k / ranges);
        if (row >= span) continue;
        const T vi = M::unkey(d.vin_k[row]);
        if (!M::finite(vi)) continue;
        T *Dr = d.D + (int64_t)row * d.ld;
        const V4 *Dr4 = reinterpret_cast<const V4 *>(Dr);
        for (int c0 = 0; c0 < nv4; c0 += 32 * SWEEP_B) {
            V4 v[SWEEP_B];
#pragma unroll
            for (int bb = 0; bb < SWEEP_B; ++bb) {
                const int c4 = c0 + bb * 32 + lane;
                if (c4 < nv4) v[bb] = Dr4[c4];
            }
            unsigned mask = 0;
#pragma unroll
            for (int bb = 0; bb < SWEEP_B; ++bb) {
                const int c4 = c0 + bb * 32 + lane;
                if (c4 < nv4) {
                    const V4 o = so4[c4];
                    mask |= ((unsigned)(vi + o.x < v[bb].x) | (unsigned)(vi + o.y < v[bb].y) << 1 |
                             (unsigned)(vi + o.z < v[bb].z) << 2 | (unsigned)(vi + o.w < v[bb].w) << 3) << (4 * bb);
                }
            }
            while (mask) {
                const int bit = __ffs(mask) - 1;
                mask &= mask - 1;
                const int j = 4 * (c0 + (bit >> 2) * 32 + lane) + (bit & 3);
                const T cand = vi + so[j];
                Dr[j] = cand;
                if (d.DT) d.DT[(int64_t)j * d.ld + row] = cand;
            }
        }
    }
}

// --------------------------------------------------------------------------
// Edge decrease u -> v to weight w (exact direct relaxation)
//   D'[i][j] = min(D[i][j], D[i][u] + w + D[v][j])   (+ (v,u) if undirected)
// A row can change only if D[i][u] + w < D[i][v], which the prepass tests.
// --------------------------------------------------------------------------

template <typename T>
__global__ void k_dec_prepass(Dev<T> d, int u, int v, T w) {
    pdl_enter();
    using M = MinPlus<T>;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        d.W[(int64_t)u * d.ld + v] = w;
        if (d.undirected) d.W[(int64_t)v * d.ld + u] = w;
    }
    bool in_r = false;
    if (i < d.span) {
        d.y[i] = d.D[(int64_t)v * d.ld + i];
        if (d.undirected) d.y2[i] = d.D[(int64_t)u * d.ld + i];
        if (d.alive[i]) {
            T xi = col_src(d, u, i);    // D[i][u]
            T xv = col_src(d, v, i);    // D[i][v]
            d.x[i] = xi;
            in_r = M::add(xi, w) < xv;
            if (d.undirected) {
                d.x2[i] = xv;
                in_r = in_r || (M::add(xv, w) < xi);
            }
        }
    }
    warp_append(in_r, i, d.rlist, &d.ctl->r_count);
}

template <typename T>
__global__ void __launch_bounds__(256, 3) k_dec_sweep(Dev<T> d, T w) {
    pdl_enter();
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    const int nrows = *(volatile int32_t *)&d.ctl->r_count;
    const V4 *y4 = reinterpret_cast<const V4 *>(d.y);
    const V4 *y24 = reinterpret_cast<const V4 *>(d.y2);
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < nrows; r += nwarps) {
        const int i = d.rlist[r];
        const T a1 = M::add(d.x[i], w);
        const T a2 = d.undirected ? M::add(d.x2[i], w) : M::inf();
        T *Dr = d.D + (int64_t)i * d.ld;
        warp_row_sweep<V4>(reinterpret_cast<const V4 *>(Dr), d.span / 4, [&](int c4, V4 v) {
            V4 yv = y4[c4];
            T dv[4] = {v.x, v.y, v.z, v.w};
            T yy[4] = {yv.x, yv.y, yv.z, yv.w};
            T yy2[4] = {M::inf(), M::inf(), M::inf(), M::inf()};
            if (d.undirected) {
                V4 t = y24[c4];
                yy2[0] = t.x; yy2[1] = t.y; yy2[2] = t.z; yy2[3] = t.w;
            }
            bool any = false;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                T cand = M::mn(a1 + yy[e], a2 + yy2[e]);
                if (cand < dv[e]) {
                    dv[e] = cand;
                    any = true;
                    if (d.DT) d.DT[(int64_t)(4 * c4 + e) * d.ld + i] = cand;
                }
            }
            if (any) {
                V4 nv; nv.x = dv[0]; nv.y = dv[1]; nv.z = dv[2]; nv.w = dv[3];
                reinterpret_cast<V4 *>(Dr)[c4] = nv;
            }
        });
    }
}

// --------------------------------------------------------------------------
// Affected-pair detection
//   removal of k (Section 3.2, Corollary 3): (i, j) is listed unless
//       D[i][j] < D[i][k] + D[k][j];
//   increase of a tight edge (u, v) of old weight w0: the same test with the
//       path through the edge, D[i][u] + w0 + D[v][j] (and through (v, u) for
//       undirected graphs).
// Pairs whose direct edge is itself a shortest path (W[i][j] == D[i][j], the
// edge not being the changed one) are dropped: that path avoids k / (u, v).
// Listed pairs get an achievable upper bound written into D (the direct edge,
// or the old path with the new edge weight), are compacted per row into
// `pairs`, and are cut into work items of ITEM_PAIRS pairs.
// --------------------------------------------------------------------------

// Clears the per-update row change stamp of slot i.
template <typename T> __device__ __forceinline__ void clear_repair_scratch(const Dev<T> &d, int i) {
    d.rstamp[i] = 0;
}

template <typename T>
__device__ __forceinline__ void k_inc_prepass_body(Dev<T> d, int u, int v, T w_old, T w_new) {
    using M = MinPlus<T>;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool tight_edge = M::tight(w_old, d.D[(int64_t)u * d.ld + v]);
    if (i == 0) {
        d.W[(int64_t)u * d.ld + v] = w_new;
        if (d.undirected) d.W[(int64_t)v * d.ld + u] = w_new;
        if (!tight_edge) d.ctl->trivial = 1;
    }
    bool in_r = false;
    if (i < d.span) {
        clear_repair_scratch(d, i);
        d.y[i] = d.D[(int64_t)v * d.ld + i];
        if (d.undirected) d.y2[i] = d.D[(int64_t)u * d.ld + i];
        if (tight_edge && d.alive[i]) {
            T xi = col_src(d, u, i);   // D[i][u]
            T xv = col_src(d, v, i);   // D[i][v]
            d.x[i] = xi;
            in_r = M::finite(xi) && M::tight(M::add(xi, w_old), xv);
            if (d.undirected) {
                d.x2[i] = xv;
                in_r = in_r || (M::finite(xv) && M::tight(M::add(xv, w_old), xi));
            }
        }
    }
    warp_append(in_r, i, d.rlist, &d.ctl->r_count);
}

template <typename T>
__global__ void k_inc_prepass(Dev<T> d, int u, int v, T w_old, T w_new) {
    pdl_enter();
    k_inc_prepass_body<T>(d, u, v, w_old, w_new);
}

constexpr int DET_MAXB = 32;    // 1024-column batches a row may have (rows <= 32768 columns)

template <typename T> __device__ __forceinline__ T unreachable_leg();
template <> __device__ __forceinline__ int32_t unreachable_leg<int32_t>() { return INF_I32 + 1; }
template <> __device__ __forceinline__ float unreachable_leg<float>() { return __int_as_float(0x7f800000); }

// Affected-pair detection.
// kind 0: removal of node a (rows: every live row != a).  Affected pairs are
//   exactly the need_update_list of Section 3.2: (i, j), i != j, both != a,
//   listed unless D[i][j] < D[i][a] + D[a][j] (Corollary 3).
// kind 1: increase of edge a -> b from w_old to w_new (rows: prepass list):
//   the same test with the path through the old edge.
// For an exact APSP matrix a path through the removed node / old edge is
// never shorter than the stored distance, so "listed" means equal (within
// the fp32 slack).  The staged legs are y = D[a][.] (removal) or D[b][.]
// (increase; y2 = D[a][.] for the reverse direction of an undirected edge).
//
// k_det_scan streams every row once with nothing but a cheap screen per
// entry and records, per row, the 1024-column batches where an entry may be
// tight; three short kernels then apply the exact test to those batches only
// and commit each row's pairs (in column order) with their starting upper
// bounds.

// Exact mask of batch c0 (vectors [c0, c0 + 256) of row i): bit 4 bb + e of
// lane l is entry 4 (c0 + 32 bb + l) + e.
template <typename T, bool TWO>
__device__ __forceinline__ unsigned det_exact_mask(const Dev<T> &d, const typename MinPlus<T>::V4 (&v)[SWEEP_B],
                                                   int c0, T s1, T s2, bool use1, bool use2, int i, int a, int kind) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    const int lane = threadIdx.x & 31;
    const int nv4 = d.span / 4;
    const V4 *y4 = reinterpret_cast<const V4 *>(d.y);
    const V4 *y24 = reinterpret_cast<const V4 *>(d.y2);
    const int ci = i >> 2, cia = i & 3;
    const int ca = kind == 0 ? (a >> 2) : -1, caa = a & 3;
    unsigned mask = 0;
#pragma unroll
    for (int bb = 0; bb < SWEEP_B; ++bb) {
        const int c4 = c0 + bb * 32 + lane;
        if (c4 < nv4) {
            unsigned m = 0;
            if (use1) {
                const V4 y = __ldcg(y4 + c4);
                m |= (unsigned)M::slack_tight(M::slack(s1 + M::leg(y.x), v[bb].x)) |
                     (unsigned)M::slack_tight(M::slack(s1 + M::leg(y.y), v[bb].y)) << 1 |
                     (unsigned)M::slack_tight(M::slack(s1 + M::leg(y.z), v[bb].z)) << 2 |
                     (unsigned)M::slack_tight(M::slack(s1 + M::leg(y.w), v[bb].w)) << 3;
            }
            if (TWO && use2) {
                const V4 y = __ldcg(y24 + c4);
                m |= (unsigned)M::slack_tight(M::slack(s2 + M::leg(y.x), v[bb].x)) |
                     (unsigned)M::slack_tight(M::slack(s2 + M::leg(y.y), v[bb].y)) << 1 |
                     (unsigned)M::slack_tight(M::slack(s2 + M::leg(y.z), v[bb].z)) << 2 |
                     (unsigned)M::slack_tight(M::slack(s2 + M::leg(y.w), v[bb].w)) << 3;
            }
            if (c4 == ci) m &= ~(1u << cia);
            if (c4 == ca) m &= ~(1u << caa);
            mask |= m << (4 * bb);
        }
    }
    return mask;
}

// Optional direct-edge filter: of the tight entries in `mask` (batch c0 of row
// i, values v), drop those whose direct edge is itself a shortest path,
// W[i][j] == D[i][j].  That edge avoids the removed node (and, for an
// increase, differs from the changed edge, whose W already holds the new,
// larger weight), so by Theorem theo_algo12 such a pair keeps its distance:
// a sufficient test for leaving Corollary 3's pair out of Algorithm 12's list.
template <typename T>
__device__ __forceinline__ unsigned det_filter_direct(const Dev<T> &d, unsigned mask,
                                                      const typename MinPlus<T>::V4 (&v)[SWEEP_B], int i, int c0) {
    using V4 = typename MinPlus<T>::V4;
    const int lane = threadIdx.x & 31;
    const V4 *Wr4 = reinterpret_cast<const V4 *>(d.W + (int64_t)i * d.ld);
    V4 w[SWEEP_B];
#pragma unroll
    for (int bb = 0; bb < SWEEP_B; ++bb)
        if ((mask >> (4 * bb)) & 15u) w[bb] = __ldcg(Wr4 + c0 + bb * 32 + lane);
#pragma unroll
    for (int bb = 0; bb < SWEEP_B; ++bb) {
        if (!((mask >> (4 * bb)) & 15u)) continue;
        unsigned drop = (unsigned)(w[bb].x == v[bb].x) | (unsigned)(w[bb].y == v[bb].y) << 1 |
                        (unsigned)(w[bb].z == v[bb].z) << 2 | (unsigned)(w[bb].w == v[bb].w) << 3;
        mask &= ~(drop << (4 * bb));
    }
    return mask;
}

// Starting upper bound of listed pair (i, j): the direct edge, and for an
// increase also the path through the edge at its new weight.
template <typename T, bool TWO>
__device__ __forceinline__ T det_init(const Dev<T> &d, int kind, T w_ij, int j, T wn_x, T wn_x2) {
    using M = MinPlus<T>;
    if (kind != 1) return w_ij;
    return M::mn(w_ij, M::mn(M::add(wn_x, M::mn(d.y[j], M::inf())),
                             M::add(wn_x2, TWO ? M::mn(d.y2[j], M::inf()) : M::inf())));
}

template <typename T>
__device__ __forceinline__ void det_write_pair(const Dev<T> &d, int i, int j, long long slot, T init) {
    d.pairs[slot] = j;
    d.pmin[slot] = MinPlus<T>::key(init);
    d.pstamp[slot] = 0;
    d.D[(int64_t)i * d.ld + j] = init;
    if (d.DT) d.DT[(int64_t)j * d.ld + i] = init;
}

// The rows the scan flagged are committed by two kernels so that a row with
// many flagged batches is spread over as many warps:
//   k_det_alloc  one lane per flagged row (32 rows a warp, one reservation
//                per warp): the row's pairs, work items and re-relaxation
//                units, and each flagged batch's first pair slot (column order);
//   k_det_write  one warp per (row, flagged batch): its pairs, written at the
//                batch's slots with their starting upper bounds.
template <typename T>
__global__ void __launch_bounds__(256) k_det_alloc(Dev<T> d) {
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int n_rows = *(volatile const int32_t *)&d.ctl->hit_rows;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    int rows_hit = 0;
    for (int r0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; r0 < n_rows; r0 += nwarps * 32) {
        const int r = r0 + lane;
        int4 re = make_int4(0, 0, 0, 0);   // (row, first unit, units, batch mask)
        int cnt[DET_MAXB];                  // the row's per-batch counts (flagged batches only)
        int n = 0;
        if (r < n_rows) re = __ldcg(d.hrows + r);
        {
            const int4 *rc4 = reinterpret_cast<const int4 *>(d.rowcnt + (int64_t)re.x * DET_MAXB);
#pragma unroll
            for (int q = 0; q < DET_MAXB / 4; ++q) {
                int4 c4 = make_int4(0, 0, 0, 0);
                if (r < n_rows && (((unsigned)re.w >> (4 * q)) & 15u)) c4 = __ldcg(rc4 + q);
                cnt[4 * q] = ((unsigned)re.w >> (4 * q)) & 1u ? c4.x : 0;
                cnt[4 * q + 1] = ((unsigned)re.w >> (4 * q + 1)) & 1u ? c4.y : 0;
                cnt[4 * q + 2] = ((unsigned)re.w >> (4 * q + 2)) & 1u ? c4.z : 0;
                cnt[4 * q + 3] = ((unsigned)re.w >> (4 * q + 3)) & 1u ? c4.w : 0;
            }
#pragma unroll
            for (int q = 0; q < DET_MAXB; ++q) n += cnt[q];
        }
        const int nit = (n + ITEM_PAIRS - 1) / ITEM_PAIRS;
        const int nseg = (n + YSEG - 1) / YSEG;
        const int nun = nit * nseg;
        const int nh = (n + P1_PAIRS - 1) / P1_PAIRS;
        int tn, tit, tun, th;
        const int on = warp_exclusive_scan(n, &tn);
        const int oit = warp_exclusive_scan(nit, &tit);
        const int oun = warp_exclusive_scan(nun, &tun);
        const int oh = warp_exclusive_scan(nh, &th);
        unsigned long long old = 0;
        int ub = 0, hb = 0;
        if (lane == 0 && tn > 0) {
            old = atomicAdd(&d.ctl->alloc, ((unsigned long long)tn << 24) | (unsigned long long)tit);
            ub = atomicAdd(&d.ctl->unit_alloc, tun);
            hb = atomicAdd(&d.ctl->p1_alloc, th);
        }
        old = __shfl_sync(0xffffffffu, old, 0);
        ub = __shfl_sync(0xffffffffu, ub, 0);
        hb = __shfl_sync(0xffffffffu, hb, 0);
        if (tn == 0) continue;
        const long long pbw = (long long)(old >> 24);
        const int ibw = (int)(old & 0xFFFFFFull);
        if (pbw + tn > d.pair_cap || ibw + tit > d.item_cap || (long long)ub + tun > d.unit_cap ||
            (long long)hb + th > d.p1u_cap) {
            if (lane == 0) atomicOr(&d.ctl->overflow, 1);
            continue;   // these rows' units write nothing (their slots stay -1)
        }
        const long long pb = pbw + on;
        if (n > 0) {
            ++rows_hit;
            long long q = pb;
            int u = re.y;
#pragma unroll
            for (int b = 0; b < DET_MAXB; ++b) {
                if (((unsigned)re.w >> b) & 1u) d.hbase[u++] = q;
                q += cnt[b];
            }
        }
        // the row's items and unit range; its units are written by the
        // warps of k_det_write, each a share
        if (r < n_rows) d.hralloc[r] = make_int4(ibw + oit, ub + oun, n, 0);
        for (int t = 0; t < 32; ++t) {
            const int nt = __shfl_sync(0xffffffffu, n, t);
            if (nt == 0) continue;
            const int it = __shfl_sync(0xffffffffu, re.x, t);
            const long long pbt = __shfl_sync(0xffffffffu, pb, t);
            const int ibt = ibw + __shfl_sync(0xffffffffu, oit, t);
            const int nitt = (nt + ITEM_PAIRS - 1) / ITEM_PAIRS;
            for (int k = lane; k < nitt; k += 32)
                d.items[ibt + k] = make_int4(it, (int)pbt + k * ITEM_PAIRS, min(ITEM_PAIRS, nt - k * ITEM_PAIRS) | (nt << 8), (int)pbt);
            const int hbt = hb + __shfl_sync(0xffffffffu, oh, t);
            const int nht = (nt + P1_PAIRS - 1) / P1_PAIRS;
            for (int k = lane; k < nht; k += 32)
                d.p1u[hbt + k] = make_int4(it, (int)pbt + k * P1_PAIRS, min(P1_PAIRS, nt - k * P1_PAIRS), 0);
        }
    }
    if (rows_hit) atomicAdd(&d.ctl->n_rows, rows_hit);
}

// With the direct-edge filter on, the exact per-batch counts of the scan are
// recounted after the filter (one warp per flagged (row, batch)) before the
// reservation, so k_det_alloc and k_det_write see the same, filtered pairs.
template <typename T, bool TWO>
__global__ void __launch_bounds__(256, 2) k_det_recount(Dev<T> d, int kind, int a, T w_old) {
    pdl_enter();
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    const int lane = threadIdx.x & 31;
    const int n_units = *(volatile const int32_t *)&d.ctl->hit_units;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int nv4 = d.span / 4;
    for (int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n_units; u += nwarps) {
        const int4 ue = __ldcg(d.hunits + u);
        const int i = ue.x;
        const int c0 = ue.y * 32 * SWEEP_B;
        const T xi = __ldcg(d.x + i);
        const T x2i = TWO ? __ldcg(d.x2 + i) : M::inf();
        const V4 *Dr4 = reinterpret_cast<const V4 *>(d.D + (int64_t)i * d.ld);
        V4 v[SWEEP_B];
#pragma unroll
        for (int bb = 0; bb < SWEEP_B; ++bb) {
            const int c4 = c0 + bb * 32 + lane;
            if (c4 < nv4) v[bb] = __ldcg(Dr4 + c4);
        }
        const T s1 = kind == 0 ? xi : M::add(xi, w_old);
        const T s2 = M::add(x2i, w_old);
        const bool use1 = M::finite(s1), use2 = TWO && M::finite(s2);
        unsigned mask = det_exact_mask<T, TWO>(d, v, c0, s1, s2, use1, use2, i, a, kind);
        mask = det_filter_direct<T>(d, mask, v, i, c0);
        const int c = warp_sum(__popc(mask));
        if (lane == 0) d.rowcnt[(int64_t)i * DET_MAXB + ue.y] = c;
    }
}

// FILTER: 0 the exact mask (Corollary 3), 1 minus direct-edge pairs, 2 the
// mask that k_det_alg12 left in umask for this unit.
// Removal: node k's row and column become missing, slot k dead (entry t).
template <typename T>
__device__ __forceinline__ void tombstone_entry(const Dev<T> &d, int k, int t) {
    const T inf = MinPlus<T>::inf();
    d.D[(int64_t)k * d.ld + t] = inf;
    d.D[(int64_t)t * d.ld + k] = inf;
    d.W[(int64_t)k * d.ld + t] = inf;
    d.W[(int64_t)t * d.ld + k] = inf;
    if (d.DT) {
        d.DT[(int64_t)k * d.ld + t] = inf;
        d.DT[(int64_t)t * d.ld + k] = inf;
    }
    if (t == 0) d.alive[k] = 0;
}

// For a removal (kind 0) the same launch also tombstones node a: nothing
// here reads row or column a (column a is never listed) and no listed pair
// lies in them.
template <typename T, bool TWO, int FILTER>
__device__ __forceinline__ void k_det_write_body(Dev<T> d, int kind, int a, T w_old, T w_new,
                                                                      const uint32_t *umask) {
    if (kind == 0)
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < d.span; t += gridDim.x * blockDim.x)
            tombstone_entry<T>(d, a, t);
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    __shared__ int32_t hbuf[8][32 * SWEEP_B * 4];
    const int lane = threadIdx.x & 31;
    int32_t *hb = hbuf[threadIdx.x >> 5];
    const int n_units = *(volatile const int32_t *)&d.ctl->hit_units;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int nv4 = d.span / 4;
    for (int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n_units; u += nwarps) {
        const int4 ue = __ldcg(d.hunits + u);   // (row, batch, row entry, position among the row's units)
        const long long base = __ldcg(d.hbase + u);
        const int i = ue.x;
        const int c0 = ue.y * 32 * SWEEP_B;
        if (base >= 0) {
            // this unit's share of the row's re-relaxation units
            const int4 ra = __ldcg(d.hralloc + ue.z);   // (first item, first unit, pairs)
            const int k = __ldcg(&d.hrows[ue.z].z);
            const int nit = (ra.z + ITEM_PAIRS - 1) / ITEM_PAIRS, nseg = (ra.z + YSEG - 1) / YSEG;
            const int nun = nit * nseg;
            const int lo = (int)((long long)nun * ue.w / k), hi = (int)((long long)nun * (ue.w + 1) / k);
            for (int t = lo + lane; t < hi; t += 32)
                d.units[ra.y + t] = (int32_t)((unsigned)(ra.x + t / nseg) | ((unsigned)(t % nseg) << 24));
        }
        const T xi = __ldcg(d.x + i);
        const T x2i = TWO ? __ldcg(d.x2 + i) : M::inf();
        if (base < 0) continue;   // a row that did not fit
        unsigned mask;
        if (FILTER == 2) {
            mask = __ldcg(umask + (int64_t)u * 32 + lane);
        } else if (FILTER == 0) {
            mask = __ldcg(d.bmask + ((int64_t)i * d.bmask_nb + ue.y) * 32 + lane);   // left by k_det_scan
        } else {
            const V4 *Dr4 = reinterpret_cast<const V4 *>(d.D + (int64_t)i * d.ld);
            V4 v[SWEEP_B];
#pragma unroll
            for (int bb = 0; bb < SWEEP_B; ++bb) {
                const int c4 = c0 + bb * 32 + lane;
                if (c4 < nv4) v[bb] = __ldcg(Dr4 + c4);
            }
            const T s1 = kind == 0 ? xi : M::add(xi, w_old);
            const T s2 = M::add(x2i, w_old);
            const bool use1 = M::finite(s1), use2 = TWO && M::finite(s2);
            mask = det_exact_mask<T, TWO>(d, v, c0, s1, s2, use1, use2, i, a, kind);
            mask = det_filter_direct<T>(d, mask, v, i, c0);
        }
        int tot;
        int off = warp_exclusive_scan(__popc(mask), &tot);
        __syncwarp();   // the previous unit's buffer reads are done
        for (unsigned m = mask; m; m &= m - 1) {
            const int bit = __ffs(m) - 1;
            hb[off++] = 4 * (c0 + (bit >> 2) * 32 + lane) + (bit & 3);
        }
        __syncwarp();
        const T wn_x = kind == 1 ? M::add(xi, w_new) : M::inf();
        const T wn_x2 = kind == 1 ? M::add(x2i, w_new) : M::inf();
        const T *Wr = d.W + (int64_t)i * d.ld;
        for (int h = 0; h < tot; h += 256) {
            int jj[8];
            T ww[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int t = h + lane + 32 * q;
                jj[q] = t < tot ? hb[t] : -1;
                if (jj[q] >= 0) ww[q] = __ldg(Wr + jj[q]);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (jj[q] >= 0)
                    det_write_pair<T>(d, i, jj[q], base + h + lane + 32 * q, det_init<T, TWO>(d, kind, ww[q], jj[q], wn_x, wn_x2));
        }
    }
}

template <typename T, bool TWO, int FILTER>
__global__ void __launch_bounds__(256, FILTER == 1 ? 2 : 4) k_det_write(Dev<T> d, int kind, int a, T w_old, T w_new,
                                                                      const uint32_t *umask) {
    pdl_enter();
    k_det_write_body<T, TWO, FILTER>(d, kind, a, w_old, w_new, umask);
}

// One warp per row, rows assigned round-robin; the legs are staged once per
// CTA in shared memory (the removed node's own column as unreachable, so its
// D[a][a] = 0 never makes a row look tight).  A lane streams 8 vectors at a
// time and keeps only the maximum of d - y (int32: a batch holds a tight
// entry iff that maximum reaches s; fp32: with twice the slack, so rounding
// can only flag extra batches).  A warp keeps the rows it flags in lane
// registers (lane t: its t-th flagged row and batch mask) and appends them
// to the hit list with one atomic when it is done or holds 32.
template <typename T, bool TWO>
__device__ __forceinline__ void k_det_scan_body(Dev<T> d, int kind, int a, T w_old) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // an increase whose prepass found no candidate row (a non-tight edge) has nothing to scan
    if (kind == 1 && *(volatile const int32_t *)&d.ctl->r_count == 0) return;
    const int span = d.span;
    T *ys = reinterpret_cast<T *>(smem_raw);
    T *y2s = ys + span;
    // a removal stages row a of D itself and publishes the legs for the later
    // kernels: y = D[a][.] (a grid-stride share per CTA), x[i] = D[i][a] by the
    // warp that scans row i; the repair's row stamps are cleared here too
    stage_vec<T>(ys, kind == 0 ? d.D + (int64_t)a * d.ld : d.y, span);
    if (TWO) stage_vec<T>(y2s, d.y2, span);
    __syncthreads();
    if (kind == 0)
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < span; c += gridDim.x * blockDim.x) {
            d.y[c] = ys[c];
            clear_repair_scratch(d, c);
        }
    for (int c = threadIdx.x; c < span; c += blockDim.x) {
        ys[c] = kind == 0 && c == a ? unreachable_leg<T>() : M::leg(ys[c]);
        if (TWO) y2s[c] = M::leg(y2s[c]);
    }
    __syncthreads();
    const V4 *ys4 = reinterpret_cast<const V4 *>(ys);
    const V4 *y2s4 = reinterpret_cast<const V4 *>(y2s);
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int nrows = kind == 0 ? span : *(volatile int32_t *)&d.ctl->r_count;
    const int nv4 = span / 4;
    int nh = 0, hrow = 0;
    unsigned hmask = 0;
    auto flush = [&]() {
        // lane t < nh holds a flagged row: one row entry and one unit per
        // flagged batch, the row's units contiguous and in column order
        const int k = lane < nh ? __popc(hmask) : 0;
        int nu;
        const int uoff = warp_exclusive_scan(k, &nu);
        int rbase = 0, ubase = 0;
        if (lane == 0) {
            rbase = atomicAdd(&d.ctl->hit_rows, nh);
            ubase = atomicAdd(&d.ctl->hit_units, nu);
        }
        rbase = __shfl_sync(0xffffffffu, rbase, 0);
        ubase = __shfl_sync(0xffffffffu, ubase, 0);
        if (lane < nh) {
            d.hrows[rbase + lane] = make_int4(hrow, ubase + uoff, k, (int)hmask);
            int q = ubase + uoff, pos = 0;
            for (unsigned m = hmask; m; m &= m - 1) {
                d.hunits[q] = make_int4(hrow, __ffs(m) - 1, rbase + lane, pos++);
                d.hbase[q] = -1;
                ++q;
            }
        }
        nh = 0;
    };
    const int r0 = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int i_next = r0 < nrows ? (kind == 0 ? r0 : d.rlist[r0]) : 0;
    T x_next = r0 < nrows ? (kind == 0 ? col_src(d, a, i_next) : d.x[i_next]) : M::inf();
    T x2_next = TWO && r0 < nrows ? d.x2[i_next] : M::inf();
    for (int r = r0; r < nrows; r += nwarps) {
        const int i = i_next;
        const T xi = x_next;  // missing for a dead row, so it is skipped below
        const T x2i = x2_next;
        if (r + nwarps < nrows) {
            i_next = kind == 0 ? r + nwarps : d.rlist[r + nwarps];
            x_next = kind == 0 ? col_src(d, a, i_next) : d.x[i_next];
            if (TWO) x2_next = d.x2[i_next];
        }
        if (kind == 0 && lane == 0) d.x[i] = xi;
        if (kind == 0 && i == a) continue;
        const T s1 = kind == 0 ? xi : M::add(xi, w_old);
        const T s2 = M::add(x2i, w_old);
        const bool use1 = M::finite(s1), use2 = TWO && M::finite(s2);
        if (!use1 && !use2) continue;
        const V4 *Dr4 = reinterpret_cast<const V4 *>(d.D + (int64_t)i * d.ld);
        unsigned bmask = 0;
        for (int c0 = 0, bi = 0; c0 < nv4; c0 += 32 * SWEEP_B, ++bi) {
            V4 v[SWEEP_B];
#pragma unroll
            for (int bb = 0; bb < SWEEP_B; ++bb) {
                const int c4 = c0 + bb * 32 + lane;
                if (c4 < nv4) v[bb] = __ldcs(Dr4 + c4);
            }
            T b1 = M::screen_floor(), b2 = M::screen_floor();
#pragma unroll
            for (int bb = 0; bb < SWEEP_B; ++bb) {
                const int c4 = c0 + bb * 32 + lane;
                if (c4 < nv4) {
                    const V4 y = ys4[c4];
                    b1 = max_of(b1, max_of(max_of(M::screen_bound(v[bb].x, y.x), M::screen_bound(v[bb].y, y.y)),
                                           max_of(M::screen_bound(v[bb].z, y.z), M::screen_bound(v[bb].w, y.w))));
                    if (TWO && use2) {
                        const V4 z = y2s4[c4];
                        b2 = max_of(b2, max_of(max_of(M::screen_bound(v[bb].x, z.x), M::screen_bound(v[bb].y, z.y)),
                                               max_of(M::screen_bound(v[bb].z, z.z), M::screen_bound(v[bb].w, z.w))));
                    }
                }
            }
            const bool maybe = (use1 && s1 <= b1) || (TWO && use2 && s2 <= b2);
            if (__ballot_sync(0xffffffffu, maybe)) {
                // the batch's exact mask (the same test and bit layout as
                // det_exact_mask; column a is staged unreachable, column i is
                // taken out): its count for the reservation, the mask itself
                // for k_det_write, which then need not read the batch again
                unsigned mk = 0;
#pragma unroll
                for (int bb = 0; bb < SWEEP_B; ++bb) {
                    const int c4 = c0 + bb * 32 + lane;
                    if (c4 < nv4) {
                        unsigned m = 0;
                        if (use1) {
                            const V4 y = ys4[c4];
                            m |= (unsigned)M::slack_tight(M::slack(s1 + y.x, v[bb].x)) |
                                 (unsigned)M::slack_tight(M::slack(s1 + y.y, v[bb].y)) << 1 |
                                 (unsigned)M::slack_tight(M::slack(s1 + y.z, v[bb].z)) << 2 |
                                 (unsigned)M::slack_tight(M::slack(s1 + y.w, v[bb].w)) << 3;
                        }
                        if (TWO && use2) {
                            const V4 y = y2s4[c4];
                            m |= (unsigned)M::slack_tight(M::slack(s2 + y.x, v[bb].x)) |
                                 (unsigned)M::slack_tight(M::slack(s2 + y.y, v[bb].y)) << 1 |
                                 (unsigned)M::slack_tight(M::slack(s2 + y.z, v[bb].z)) << 2 |
                                 (unsigned)M::slack_tight(M::slack(s2 + y.w, v[bb].w)) << 3;
                        }
                        if (c4 == (i >> 2)) m &= ~(1u << (i & 3));   // the diagonal is never a pair
                        mk |= m << (4 * bb);
                    }
                }
                const int c = warp_sum(__popc(mk));
                if (c > 0) {
                    bmask |= 1u << bi;
                    if (lane == 0) d.rowcnt[(int64_t)i * DET_MAXB + bi] = c;
                    d.bmask[((int64_t)i * d.bmask_nb + bi) * 32 + lane] = mk;
                }
            }
        }
        if (bmask) {
            if (lane == nh) {
                hrow = i;
                hmask = bmask;
            }
            if (++nh == 32) flush();
        }
    }
    if (nh) flush();
}

template <typename T, bool TWO>
__global__ void __launch_bounds__(256, 4) k_det_scan(Dev<T> d, int kind, int a, T w_old) {
    pdl_enter();
    k_det_scan_body<T, TWO>(d, kind, a, w_old);
}


// --------------------------------------------------------------------------
// Repair: cooperative persistent kernel that decides warm or cold on the
// device and then either re-relaxes the affected pairs to a fixed point or
// recomputes D by blocked Floyd-Warshall.
//
// Warm (restricted re-relaxation, replacing Algorithm 5's per-row Dijkstra).
// Every listed pair (i, j) starts at an achievable upper bound (its direct
// edge, or a path through the new edge weight); unlisted pairs are exact.
//
// Pass 1 sets every listed pair to min over all x of D[i][x] + D[x][j],
// reading only the starting values (results go to `pmin`, D is untouched), so
// the pass is one read-only sweep taken in chunks of x that keep the touched
// rows and columns in L2.  After it, a pair is exact unless the predecessor
// of j on its new shortest path from i is itself a listed target of row i:
// otherwise that predecessor y has D[i][y] exact and D[y][j] <= W[y][j].
//
// Passes >= 2 therefore only relax each row through its own listed targets,
//     D[i][j] = min(D[i][j], min over listed y of D[i][y] + D[y][j]),
// a Bellman-Ford over the row's list with any achievable D[y][j] <= W[y][j]
// as the arc length.  Semi-naive: after pass 2 (which takes every y) a pair
// is re-examined only through y lowered in the previous pass, and only y
// with D[i][y] < D[i][j] can help (weights are non-negative).  A pass that
// lowers nothing leaves every row at its fixed point, which is exact.
// Rows never wait for each other: concurrent readers see either value of a
// pair being lowered, and both are achievable upper bounds.
// --------------------------------------------------------------------------

struct RepairCfg {
    int mode;            // apsp_dispatch
    float delta;         // Algorithm 5's threshold on Cost
    int n_live_before;   // N of Eq. (equ:cost_defi)
    int has_model;
    const float *model;  // cost-model parameters (device), may be null
    float feat_type;     // update-type feature
    float feat_dw;       // relative weight change
    int32_t *grown_flag; // per-row flags (ld int32) for Algorithm 12's list; null: not measured
    int list_mode;       // apsp_list_mode: 1 drops direct-edge pairs (det_filter_direct), 2 applies Algorithm 12 (k_det_alg12)
    uint32_t *umask;     // list mode 2: surviving mask per flagged unit (32 words each)
};

// Algorithm 12's need_update_list, measured once the repair is done.  A
// listed pair belongs to it iff its distance grew: by Theorem theo_algo12 the
// removed node (or, for an increase, the old edge) was then needed by every
// shortest path.  The old distance of a listed pair is its tight sum through
// the staged legs (removal: D[i][k] + D[k][j]; increase: D[i][u] + w_old +
// D[v][j], or the reverse orientation of an undirected edge).  One warp per
// work item; int32 exact, fp32 "grew" beyond the tightness slack.
template <typename T, bool TWO>
__global__ void __launch_bounds__(256) k_grown_count(Dev<T> d, int kind, T w_old, int32_t *rflag) {
    pdl_enter();
    using M = MinPlus<T>;
    const int lane = threadIdx.x & 31;
    const unsigned long long alloc = *(volatile const unsigned long long *)&d.ctl->alloc;
    if (*(volatile const int32_t *)&d.ctl->overflow) return;
    const int n_items = (int)(alloc & 0xFFFFFFull);
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < n_items; it += nwarps) {
        const int4 item = __ldcg(d.items + it);
        const int i = item.x, cnt = item.z & 0xff;
        bool grown = false;
        if (lane < cnt) {
            const int j = __ldcg(d.pairs + item.y + lane);
            const T xi = __ldcg(d.x + i);
            T old = M::add(kind == 0 ? xi : M::add(xi, w_old), __ldcg(d.y + j));
            if (TWO) old = M::mn(old, M::add(M::add(__ldcg(d.x2 + i), w_old), __ldcg(d.y2 + j)));
            const T now = __ldcg(d.D + (int64_t)i * d.ld + j);
            grown = !M::tight(now, old);
        }
        const unsigned b = __ballot_sync(0xffffffffu, grown);
        if (lane == 0 && b) {
            atomicAdd(&d.ctl->grown_pairs, (unsigned long long)__popc(b));
            if (atomicExch(rflag + i, 1) == 0) atomicAdd(&d.ctl->grown_rows, 1);
        }
    }
}

template <typename T>
__device__ void repair_warm(Dev<T> &d) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    Ctl *ctl = d.ctl;
    const int lane = threadIdx.x & 31;
    const int span = d.span;
    const int64_t ld = d.ld;
    const T *cols = d.DT ? d.DT : d.D;   // row j of `cols` is column j of D
    const long long n_units = *(volatile const int32_t *)&ctl->unit_alloc;

    const int wq = (int)((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % QUEUES) * 32;

    // Pass 1 ran in k_repair_p1 (repair_p1.cuh): pmin holds every listed
    // pair's minimum over all x.  The control block was cleared before the
    // update, so the state the passes below start from (no stop, no pair
    // lowered, empty work queues) needs no barrier.
    int pass = 1;
    auto leader = [&]() {
        volatile Ctl *cv = ctl;
        const int par = pass & 1;
        cv->stop = pass >= 2 && cv->changed[par] == 0;
        cv->changed[par ^ 1] = 0;
        for (int q = 0; q < QUEUES; ++q) cv->qn[par ^ 1][32 * q] = 0;
        cv->passes = pass;
        cv->t_end = globaltimer_ns();
    };
    // Passes >= 2: one warp per unit = (work item, segment of YSEG of the
    // row's listed targets y).  Lane u holds intermediates y = segment[u +
    // 32b] with D[i][y]; pairs are taken four at a time, every lane gathering
    // D[y][j] = cols[j][y] for its y (16 gathers in flight), and a transpose
    // reduction leaves pair t's minimum in lane t.  Pass 2 reads D[i][.] of
    // listed pairs from pmin and stores every pair; later passes take only
    // y lowered in the previous pass and store only pairs they lower.
    // Stores are atomic minima (the segments of one item share its pairs).
    //
    // Gathers that cannot lower the pair are skipped (int32).  Every value
    // in D during the repair is the length of a path in the updated graph,
    // hence >= the new distance >= the old one (a removal or an increase
    // never shortens a path), and the old matrix obeys the triangle
    // inequality through the staged legs: with ly = D[a][.] (removal of a;
    // D[v][.] for an increase of u -> v) and lx = D[.][a] (D[.][u]),
    //     D[y][j] >= ly[j] - ly[y]   and   D[y][j] >= lx[y] - lx[j].
    // So y can lower pair j only if dy - ly[y] < cur - ly[j] and
    // dy + lx[y] < cur + lx[j]; a skipped candidate is >= cur and the
    // stored minimum is the same as without the test.  Values are <= INF =
    // 2^30 - 1, so both sides fit in int32.
    constexpr int YB = YSEG / 32;
    constexpr bool PRUNE = std::is_same<T, int32_t>::value;
    for (pass = 2; pass <= MAX_PASSES && !*(volatile int32_t *)&ctl->stop; ++pass) {
        const int par = pass & 1;
        bool changed = false;
        unsigned long long evals = 0;
        while (true) {
            int tq = 0;
            if (lane == 0) tq = atomicAdd(&ctl->qn[par][wq], 1);
            tq = __shfl_sync(0xffffffffu, tq, 0);
            const long long un = (long long)(wq >> 5) + (long long)QUEUES * tq;
            if (un >= n_units) break;
            const int code = __ldcg(d.units + un);
            const int4 item = __ldcg(d.items + (code & 0xFFFFFF));
            const int seg = (int)((unsigned)code >> 24);
            const int i = item.x;
            // a row is revisited only if it was lowered in the previous pass
            // (a stamp of this pass means the same: its units run only then)
            if (pass > 2 && (int)__ldcg(d.rstamp + i) < pass - 1) continue;
            const int cnt = item.z & 0xff, nrow = item.z >> 8;
            const bool mine = lane < cnt;
            const T *Di = d.D + (int64_t)i * ld;
            int j = 0;
            T cur = (T)0;   // pairs past cnt: no y passes dy < 0, so they load nothing
            T cly = (T)0, clx = (T)0;   // cur - ly[j], cur + lx[j]
            if (mine) {
                j = __ldcg(d.pairs + item.y + lane);
                cur = pass == 2 ? M::unkey(__ldcg(d.pmin + item.y + lane)) : __ldcg(Di + j);
                if (PRUNE) {
                    cly = cur - __ldg(d.y + j);
                    clx = cur + __ldg(d.x + j);
                }
            }
            const int ybeg = seg * YSEG, yend = min(nrow, ybeg + YSEG);
            int yv[YB];
            T dyv[YB], ayv[YB], byv[YB];   // dy, dy - ly[y], dy + lx[y]
#pragma unroll
            for (int b = 0; b < YB; ++b) {
                const int yi = ybeg + 32 * b + lane;
                yv[b] = 0;
                dyv[b] = M::inf();
                if (yi < yend) {
                    yv[b] = __ldcg(d.pairs + item.w + yi);
                    if (pass == 2) dyv[b] = M::unkey(__ldcg(d.pmin + item.w + yi));
                    else if ((int)__ldcg(d.pstamp + item.w + yi) >= pass - 1) dyv[b] = __ldcg(Di + yv[b]);
                }
                if (PRUNE) {
                    ayv[b] = dyv[b];
                    byv[b] = dyv[b];
                    if (dyv[b] < M::inf()) {
                        ayv[b] -= __ldg(d.y + yv[b]);
                        byv[b] += __ldg(d.x + yv[b]);
                    }
                }
            }
            bool any_y = false;
#pragma unroll
            for (int b = 0; b < YB; ++b) any_y |= dyv[b] < M::inf();
            if (seg == 0 && lane == 0) evals += cnt;
            if (pass > 2 && !__any_sync(0xffffffffu, any_y)) continue;   // pass 2 stores every pair
            const int nb = (yend - ybeg + 31) >> 5;   // y blocks holding data (warp-uniform)
            T acc[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) acc[q] = M::inf();
#pragma unroll
            for (int q = 0; q < 32; q += 4) {
                if (q < cnt) {
                    const T *cr[4];
                    T cq[4], qa[4], qb[4];
#pragma unroll
                    for (int u4 = 0; u4 < 4; ++u4) {
                        const int jj = __shfl_sync(0xffffffffu, j, q + u4);
                        cq[u4] = __shfl_sync(0xffffffffu, cur, q + u4);
                        if (PRUNE) {
                            qa[u4] = __shfl_sync(0xffffffffu, cly, q + u4);
                            qb[u4] = __shfl_sync(0xffffffffu, clx, q + u4);
                        }
                        cr[u4] = cols + (int64_t)jj * ld;
                    }
                    T v[4][YB];
#pragma unroll
                    for (int u4 = 0; u4 < 4; ++u4)
#pragma unroll
                        for (int b = 0; b < YB; ++b) {
                            bool use = b < nb && dyv[b] < cq[u4];
                            if (PRUNE) use = use && ayv[b] < qa[u4] && byv[b] < qb[u4];
                            v[u4][b] = use ? __ldcg(cr[u4] + yv[b]) : M::inf();
                        }
#pragma unroll
                    for (int u4 = 0; u4 < 4; ++u4)
#pragma unroll
                        for (int b = 0; b < YB; ++b) acc[q + u4] = M::add_min(dyv[b], v[u4][b], acc[q + u4]);
                }
            }
            // transpose reduction: after the step over lane bit s, acc[k]
            // (k < s) holds the partial minimum of pair (lane's high bits) + k
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                const bool hi = lane & s;
#pragma unroll
                for (int k = 0; k < s; ++k) {
                    const T send = hi ? acc[k] : acc[k + s];
                    const T keep = hi ? acc[k + s] : acc[k];
                    acc[k] = M::mn(keep, __shfl_xor_sync(0xffffffffu, send, s));
                }
            }
            const T best = acc[0];
            const bool lower = mine && M::lowers(best, cur);
            if (mine && (pass == 2 || lower)) {
                const int32_t key = M::key(M::mn(best, cur));
                atomicMin(reinterpret_cast<int32_t *>(d.D + (int64_t)i * ld + j), key);
                if (d.DT) atomicMin(reinterpret_cast<int32_t *>(d.DT + (int64_t)j * ld + i), key);
            }
            if (lower) {
                d.pstamp[item.y + lane] = (uint8_t)pass;
                changed = true;
            }
            if (__any_sync(0xffffffffu, lower) && lane == 0) d.rstamp[i] = (uint8_t)pass;
        }
        if (changed) *(volatile int32_t *)&ctl->changed[par] = 1;
        if (evals) atomicAdd(&ctl->pairs_evaluated, evals);
        if (!grid_barrier(ctl, leader)) return;
    }
    if (pass > MAX_PASSES && !*(volatile int32_t *)&ctl->stop && blockIdx.x == 0 && threadIdx.x == 0)
        atomicOr(&ctl->err, ERR_PASSES);
}

template <typename T>
__device__ void repair_cold(Dev<T> &d, unsigned char *smem) {
    using V4 = typename MinPlus<T>::V4;
    Ctl *ctl = d.ctl;
    const int nb = (d.span + FW_B - 1) / FW_B;
    const int64_t rows = (int64_t)nb * FW_B;
    // D = W (dead rows / columns are missing in W as well)
    const int64_t tot4 = rows * d.ld / 4;
    const V4 *src = reinterpret_cast<const V4 *>(d.W);
    V4 *dst = reinterpret_cast<V4 *>(d.D);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot4; t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = __ldcg(src + t);
    if (!grid_barrier(ctl, NoLeader{})) return;
    FwSmem<T> &fs = *reinterpret_cast<FwSmem<T> *>(smem);
    FwDiagSmem<T> &ds = *reinterpret_cast<FwDiagSmem<T> *>(smem);
    for (int kb = 0; kb < nb; ++kb) {
        if (blockIdx.x == 0) fw_close_diag<T>(d.D + (int64_t)kb * FW_B * d.ld + (int64_t)kb * FW_B, d.ld, ds);
        if (!grid_barrier(ctl, NoLeader{})) return;
        if (nb > 1) {
            for (int t = blockIdx.x; t < 2 * (nb - 1); t += gridDim.x) fw_phase2_tile<T>(d.D, d.ld, kb, nb, t, fs);
            if (!grid_barrier(ctl, NoLeader{})) return;
            for (int t = blockIdx.x; t < (nb - 1) * (nb - 1); t += gridDim.x) fw_phase3_tile<T>(d.D, d.ld, kb, nb, t, fs);
            if (!grid_barrier(ctl, NoLeader{})) return;
        }
    }
    if (d.DT) {
        T (*tile)[33] = reinterpret_cast<T (*)[33]>(smem);
        const int tiles = d.span / 32;
        const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
        for (int t = blockIdx.x; t < tiles * tiles; t += gridDim.x) {
            int bi = t / tiles, bj = t % tiles;
            for (int r = ty; r < 32; r += 8) tile[r][tx] = __ldcg(d.D + (int64_t)(bi * 32 + r) * d.ld + bj * 32 + tx);
            __syncthreads();
            for (int r = ty; r < 32; r += 8) d.DT[(int64_t)(bj * 32 + r) * d.ld + bi * 32 + tx] = tile[tx][r];
            __syncthreads();
        }
    }
}


// Warm / cold decision for the current update, computed identically by
// every CTA of both repair kernels from the control block (deterministic
// arithmetic, so all of them agree).  Returns -1 when there is nothing to
// repair, 0 for warm, else the cold reason (1 Cost rule, 2 model, 3 forced,
// 4 scratch overflow).
__device__ inline int repair_decide(const Ctl *ctl, const RepairCfg &cfg, float *cost, float *pw, float *pc,
                                    int *n_items) {
    const int trivial = *(volatile const int32_t *)&ctl->trivial;
    const unsigned long long alloc = *(volatile const unsigned long long *)&ctl->alloc;
    const int ovf = *(volatile const int32_t *)&ctl->overflow;
    const int rows = *(volatile const int32_t *)&ctl->n_rows;
    *n_items = (int)(alloc & 0xFFFFFFull);
    *pw = *pc = 0.f;
    *cost = 0.f;
    if (trivial || (*n_items == 0 && !ovf)) return -1;
    *cost = (float)rows / (float)max(1, cfg.n_live_before - 1);
    if (ovf) return 4;
    if (cfg.mode == 2) return 3;
    if (cfg.mode == 1) return 0;
    if (cfg.mode == 3 && cfg.has_model) {
        const float n = (float)max(2, cfg.n_live_before);
        const float np = (float)(alloc >> 24);
        float feat[MLP_IN] = {cfg.feat_type, log2f(n), cfg.feat_dw, np / (n * n), *cost, (float)rows / n};
        __shared__ float out[MLP_OUT];
        mlp_predict_cta(cfg.model, feat, out);
        *pw = out[0];
        *pc = out[1];
        return *pc < *pw ? 2 : 0;
    }
    return *cost > cfg.delta ? 1 : 0;
}

__device__ inline void repair_record(Ctl *ctl, int reason, float cost, float pw, float pc) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->cost = cost;
        ctl->cold_reason = reason < 0 ? 0 : reason;
        ctl->model_warm = pw;
        ctl->model_cold = pc;
        ctl->path = reason < 0 ? PATH_TRIVIAL : (reason ? PATH_COLD : PATH_WARM);
        ctl->n_items = (int)(ctl->alloc & 0xFFFFFFull);
        ctl->n_pairs = ctl->alloc >> 24;
    }
}

// Repair (cooperative launch, after k_repair_p1): the warm / cold decision,
// then either the re-relaxation passes >= 2 or the persistent blocked
// Floyd-Warshall.  One kernel holds both, so an update that stays warm
// launches no cold kernel; the first pass, which wants the shared memory for
// its copy ring, is the separate k_repair_p1.
template <typename T>
__device__ __forceinline__ void repair_main_body(Dev<T> d, const RepairCfg &cfg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float cost, pw, pc;
    int n_items;
    const int reason = repair_decide(d.ctl, cfg, &cost, &pw, &pc, &n_items);
    repair_record(d.ctl, reason, cost, pw, pc);
    if (reason < 0) return;
    if (reason > 0) {
        repair_cold<T>(d, smem_raw);
        return;
    }
    repair_warm<T>(d);
}

template <typename T>
__global__ void __launch_bounds__(256, 2) k_repair_main(Dev<T> d, RepairCfg cfg) {
    repair_main_body<T>(d, cfg);
}

}  // namespace apsp
