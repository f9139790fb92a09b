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
    int4 *items;              // (row, first pair, pair count | row's pair count << 8, row's first pair)
    int32_t *pairs;           // affected column per pair, grouped by row (columns ascending)
    int32_t *pmin;            // per pair: first-pass minimum as an ordered key
    uint8_t *pstamp;          // per pair: last pass that lowered it (0: none yet)
    uint8_t *rstamp;          // per row (ld): last pass that lowered one of its pairs
    int32_t *units;           // work units of passes >= 2: item | intermediate segment << 24
    Ctl *ctl;
    int64_t pair_cap;
    int32_t item_cap;
    int32_t unit_cap;
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

template <typename T> __global__ void __launch_bounds__(FW_THREADS) k_fw_p1(T *D, int64_t ld, int kb) {
    __shared__ FwDiagSmem<T> sm;
    fw_close_diag<T>(D + (int64_t)kb * FW_B * ld + (int64_t)kb * FW_B, ld, sm);
}

template <typename T> __global__ void __launch_bounds__(FW_THREADS, 2) k_fw_p2(T *D, int64_t ld, int kb, int nb) {
    __shared__ FwSmem<T> sm;
    fw_phase2_tile<T>(D, ld, kb, nb, blockIdx.x, sm);
}

template <typename T> __global__ void __launch_bounds__(FW_THREADS, 2) k_fw_p3(T *D, int64_t ld, int kb, int nb) {
    __shared__ FwSmem<T> sm;
    fw_phase3_tile<T>(D, ld, kb, nb, blockIdx.x, sm);
}

// --------------------------------------------------------------------------
// Adding a node p (Section 3.1)
// --------------------------------------------------------------------------

// Mask the new node's weights (dead slots and p itself -> missing), validate
// them, and reset the two reduction vectors.
template <typename T>
__global__ void k_insert_prep(Dev<T> d, const T *in_raw, const T *out_raw, int cap, int p) {
    using M = MinPlus<T>;
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d.span) return;
    uint32_t err = 0;
    T wi = M::inf(), wo = M::inf();
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

// One pass over D computing both vectors of the new node:
//   out[r] = min_t w(p, t) + D[t][r]     (Corollary 1, column reduction)
//   in[t]  = min_r D[t][r] + w(r, p)     (Corollary 2, row reduction)
// Grid: (column band of INS_CB columns) x (row range); the launcher picks the
// number of row ranges so the grid is one wave over the SMs.  Each lane owns
// 16 columns; partial results meet in global memory through atomicMin on
// ordered keys (one per row per band, one per column per row range).
constexpr int INS_CB = 512;

template <typename T>
__global__ void __launch_bounds__(256) k_insert_reduce(Dev<T> d, int rows_per_cta) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    __shared__ T red[8][INS_CB];
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
#pragma unroll 2
    for (int row = r0 + w; row < r1; row += 8) {
        if (!d.alive[row]) continue;
        const T wo = d.w_out[row];
        const T *Dr = d.D + (int64_t)row * d.ld + c0 + lane * 4;
        V4 v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (cin[q]) v[q] = *reinterpret_cast<const V4 *>(Dr + q * 128);
        T racc = M::inf();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!cin[q]) continue;
            T e4[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                col[q * 4 + e] = M::add_min(wo, e4[e], col[q * 4 + e]);
                racc = M::add_min(e4[e], win[q * 4 + e], racc);
            }
        }
        racc = warp_min(racc);
        if (lane == 0 && M::finite(racc)) atomicMin(&d.vin_k[row], M::key(racc));
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

// Theorem 3 sweep: D[i][j] = min(D[i][j], in[i] + out[j]).  One warp per
// row; out[] is staged once per CTA in shared memory.  Each lane streams 8
// vectors at a time and only builds a 32-bit mask of the entries that
// improve; those few entries are then written one by one (the new value is
// in[i] + out[j]; the row data is no longer needed).  A dead row and p
// itself have in[] = missing, so one load decides whether a row is swept.
// Row p and column p are never improved by the sweep (their candidates are
// missing), so they are written afterwards by k_insert_finish.
template <typename T>
__global__ void __launch_bounds__(256, 4) k_insert_relax(Dev<T> d, int p) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int span = d.span;
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
    for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < span; row += nwarps) {
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

// Row p = out (Corollary 1), column p = in (Corollary 2), D[p][p] = 0, the
// weights of p, and p becomes live.
template <typename T>
__global__ void k_insert_finish(Dev<T> d, int p) {
    using M = MinPlus<T>;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.span) return;
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

// --------------------------------------------------------------------------
// Edge decrease u -> v to weight w (exact direct relaxation)
//   D'[i][j] = min(D[i][j], D[i][u] + w + D[v][j])   (+ (v,u) if undirected)
// A row can change only if D[i][u] + w < D[i][v], which the prepass tests.
// --------------------------------------------------------------------------

template <typename T>
__global__ void k_dec_prepass(Dev<T> d, int u, int v, T w) {
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
__global__ void k_rm_gather(Dev<T> d, int k) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.span) return;
    d.x[i] = col_src(d, k, i);                 // D[i][k]
    d.y[i] = d.D[(int64_t)k * d.ld + i];       // D[k][i]
    clear_repair_scratch(d, i);
}

template <typename T>
__global__ void k_inc_prepass(Dev<T> d, int u, int v, T w_old, T w_new) {
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

constexpr int DETECT_HB = 256;  // per-warp buffer of a row's affected columns

// Second scan of a row with more affected pairs than the warp buffer holds:
// the same test, writing each pair at the row's reserved offsets with the
// direct-edge weights of the batch fetched together.  Out of line so the hot
// scan keeps its registers.
template <typename T, bool TWO>
__device__ __noinline__ void det_wide_write(const Dev<T> &d, int kind, int i, int a, long long base, T s1, T s2,
                                            bool use1, bool use2, T wn_x, T wn_x2, const T *ys, const T *y2s) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    const int lane = threadIdx.x & 31;
    const int nv4 = d.span / 4;
    const V4 *Dr4 = reinterpret_cast<const V4 *>(d.D + (int64_t)i * d.ld);
    const V4 *Wr4 = reinterpret_cast<const V4 *>(d.W + (int64_t)i * d.ld);
    const V4 *ys4 = reinterpret_cast<const V4 *>(ys);
    const V4 *y2s4 = reinterpret_cast<const V4 *>(y2s);
    const int ci = i >> 2, cia = i & 3;
    const int ca = kind == 0 ? (a >> 2) : -1, caa = a & 3;
    constexpr int B = 4;
    int n = 0;
    for (int c0 = 0; c0 < nv4; c0 += 32 * B) {
        V4 v[B], wv[B];
#pragma unroll
        for (int bb = 0; bb < B; ++bb) {
            const int c4 = c0 + bb * 32 + lane;
            if (c4 < nv4) {
                v[bb] = Dr4[c4];
                wv[bb] = __ldg(Wr4 + c4);
            }
        }
        unsigned mask = 0;
#pragma unroll
        for (int bb = 0; bb < B; ++bb) {
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
                if (c4 == ci) m &= ~(1u << cia);
                if (c4 == ca) m &= ~(1u << caa);
                mask |= m << (4 * bb);
            }
        }
        int tot;
        int off = n + warp_exclusive_scan(__popc(mask), &tot);
#pragma unroll
        for (int bb = 0; bb < B; ++bb) {
            const T wv4[4] = {wv[bb].x, wv[bb].y, wv[bb].z, wv[bb].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (!(mask >> (4 * bb + e) & 1u)) continue;
                const int j = 4 * (c0 + bb * 32 + lane) + e;
                T init = wv4[e];
                if (kind == 1)
                    init = M::mn(init, M::mn(M::add(wn_x, M::mn(ys[j], M::inf())),
                                             M::add(wn_x2, TWO ? M::mn(y2s[j], M::inf()) : M::inf())));
                d.pairs[base + off] = j;
                d.pmin[base + off] = M::key(init);
                d.pstamp[base + off] = 0;
                d.D[(int64_t)i * d.ld + j] = init;
                if (d.DT) d.DT[(int64_t)j * d.ld + i] = init;
                ++off;
            }
        }
        n += tot;
    }
}

// kind 0: removal of node a (rows: every live row != a).  Affected pairs are
//   exactly the need_update_list of Section 3.2: (i, j), i != j, both != a,
//   listed unless D[i][j] < D[i][a] + D[a][j] (Corollary 3).
// kind 1: increase of edge a -> b from w_old to w_new (rows: prepass list):
//   the same test with the path through the old edge.
// One warp per row, 8 vectors per lane in flight.  Each lane turns its 8
// vectors into a 32-bit mask of tight entries (for an exact APSP matrix a
// path through the removed node / old edge is never shorter than the stored
// distance, so tight means equal, or equal within the fp32 slack); batches
// where some lane has a bit set append those columns, in order, to a
// per-warp buffer (one prefix sum).  One packed atomic reserves the row's
// slots; a row with more than DETECT_HB pairs is scanned a second time the
// same way, writing at the reserved offsets.
template <typename T, bool TWO>
__global__ void __launch_bounds__(256, 3) k_detect(Dev<T> d, int kind, int a, int b, T w_old, T w_new) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int32_t hbuf[8][DETECT_HB];
    const int span = d.span;
    T *ys = reinterpret_cast<T *>(smem_raw);
    T *y2s = ys + span;
    stage_vec<T>(ys, d.y, span);
    if (TWO) stage_vec<T>(y2s, d.y2, span);
    __syncthreads();
    for (int c = threadIdx.x; c < span; c += blockDim.x) {
        ys[c] = M::leg(ys[c]);
        if (TWO) y2s[c] = M::leg(y2s[c]);
    }
    __syncthreads();
    const V4 *ys4 = reinterpret_cast<const V4 *>(ys);
    const V4 *y2s4 = reinterpret_cast<const V4 *>(y2s);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int32_t *hb = hbuf[wib];
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int nrows = kind == 0 ? span : *(volatile int32_t *)&d.ctl->r_count;
    const int nv4 = span / 4;
    int rows_hit = 0;
    for (int r = blockIdx.x * (blockDim.x >> 5) + wib; r < nrows; r += nwarps) {
        const int i = kind == 0 ? r : d.rlist[r];
        if (kind == 0 && i == a) continue;
        const T xi = d.x[i];  // missing for a dead row, so it is skipped below
        const T x2i = TWO ? d.x2[i] : M::inf();
        const T s1 = kind == 0 ? xi : M::add(xi, w_old);
        const T s2 = M::add(x2i, w_old);
        const bool use1 = M::finite(s1), use2 = TWO && M::finite(s2);
        if (!use1 && !use2) continue;
        const V4 *Dr4 = reinterpret_cast<const V4 *>(d.D + (int64_t)i * d.ld);
        const int ci = i >> 2, cia = i & 3;
        const int ca = kind == 0 ? (a >> 2) : -1, caa = a & 3;
        const T wn_x = kind == 1 ? M::add(xi, w_new) : M::inf();
        const T wn_x2 = kind == 1 ? M::add(x2i, w_new) : M::inf();
        int n = 0;
        for (int pass = 0; pass < 1; ++pass) {
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
                        if (c4 == ci) m &= ~(1u << cia);
                        if (c4 == ca) m &= ~(1u << caa);
                        mask |= m << (4 * bb);
                    }
                }
                if (__ballot_sync(0xffffffffu, mask != 0) == 0) continue;
                int tot;
                int off = n + warp_exclusive_scan(__popc(mask), &tot);
                for (unsigned m = mask; m; m &= m - 1) {
                    const int bit = __ffs(m) - 1;
                    if (off < DETECT_HB) hb[off] = 4 * (c0 + (bit >> 2) * 32 + lane) + (bit & 3);
                    ++off;
                }
                n += tot;
            }
            if (n == 0) break;
            // reserve the row's slots
            const int nit = (n + ITEM_PAIRS - 1) / ITEM_PAIRS;
            const int nseg = (n + YSEG - 1) / YSEG;
            const int nun = nit * nseg;
            unsigned long long old = 0;
            int ub = 0;
            if (lane == 0) {
                old = atomicAdd(&d.ctl->alloc, ((unsigned long long)n << 24) | (unsigned long long)nit);
                ub = atomicAdd(&d.ctl->unit_alloc, nun);
            }
            old = __shfl_sync(0xffffffffu, old, 0);
            ub = __shfl_sync(0xffffffffu, ub, 0);
            const long long rb = (long long)(old >> 24);
            const int ib = (int)(old & 0xFFFFFFull);
            if (rb + n > d.pair_cap || ib + nit > d.item_cap || (long long)ub + nun > d.unit_cap) {
                if (lane == 0) atomicOr(&d.ctl->overflow, 1);
                n = 0;
                break;
            }
            ++rows_hit;
            for (int t = lane; t < nit; t += 32)
                d.items[ib + t] = make_int4(i, (int)rb + t * ITEM_PAIRS, min(ITEM_PAIRS, n - t * ITEM_PAIRS) | (n << 8), (int)rb);
            for (int u = lane; u < nun; u += 32)
                d.units[ub + u] = (int32_t)((unsigned)(ib + u / nseg) | ((unsigned)(u % nseg) << 24));
            __syncwarp();
            if (n <= DETECT_HB) {
                // up to 8 pairs per lane; their gathers are issued together
                int jj[DETECT_HB / 32];
                T ww[DETECT_HB / 32];
#pragma unroll
                for (int q = 0; q < DETECT_HB / 32; ++q) {
                    const int t = lane + 32 * q;
                    jj[q] = t < n ? hb[t] : -1;
                    if (jj[q] >= 0) ww[q] = __ldg(d.W + (int64_t)i * d.ld + jj[q]);
                }
#pragma unroll
                for (int q = 0; q < DETECT_HB / 32; ++q) {
                    if (jj[q] < 0) continue;
                    const int j = jj[q];
                    T init = ww[q];
                    if (kind == 1)
                        init = M::mn(init, M::mn(M::add(wn_x, M::mn(ys[j], M::inf())),
                                                 M::add(wn_x2, TWO ? M::mn(y2s[j], M::inf()) : M::inf())));
                    d.pairs[rb + lane + 32 * q] = j;
                    d.pmin[rb + lane + 32 * q] = M::key(init);
                    d.pstamp[rb + lane + 32 * q] = 0;
                    d.D[(int64_t)i * d.ld + j] = init;
                    if (d.DT) d.DT[(int64_t)j * d.ld + i] = init;
                }
                __syncwarp();  // the buffer is reused by the next row
                break;
            }
            det_wide_write<T, TWO>(d, kind, i, a, rb, s1, s2, use1, use2, wn_x, wn_x2, ys, y2s);
        }
    }
    if (lane == 0 && rows_hit) atomicAdd(&d.ctl->n_rows, rows_hit);
}

// Removal: node k's row and column become missing, slot k dead.
template <typename T>
__global__ void k_tombstone(Dev<T> d, int k) {
    using M = MinPlus<T>;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= d.span) return;
    const T inf = M::inf();
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
};

// Minimum of four per-lane values over the warp with 6 shuffles: returns, in
// every lane of each group of 8 lanes g = lane / 8, the minimum of value g.
template <typename T> __device__ __forceinline__ T warp_min4(T a0, T a1, T a2, T a3, int lane) {
    using M = MinPlus<T>;
    const bool hi = lane & 16;
    const T s0 = hi ? a0 : a2, s1 = hi ? a1 : a3;
    T k0 = hi ? a2 : a0, k1 = hi ? a3 : a1;
    k0 = M::mn(k0, __shfl_xor_sync(0xffffffffu, s0, 16));
    k1 = M::mn(k1, __shfl_xor_sync(0xffffffffu, s1, 16));
    const bool b3 = lane & 8;
    const T s = b3 ? k0 : k1;
    T k = b3 ? k1 : k0;
    k = M::mn(k, __shfl_xor_sync(0xffffffffu, s, 8));
    k = M::mn(k, __shfl_xor_sync(0xffffffffu, k, 4));
    k = M::mn(k, __shfl_xor_sync(0xffffffffu, k, 2));
    k = M::mn(k, __shfl_xor_sync(0xffffffffu, k, 1));
    return k;
}

template <typename T>
__device__ void repair_warm(Dev<T> &d, int n_items) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    Ctl *ctl = d.ctl;
    const int lane = threadIdx.x & 31;
    const int span = d.span;
    const int64_t ld = d.ld;
    const T *cols = d.DT ? d.DT : d.D;   // row j of `cols` is column j of D
    const int nchunk = (span + PASS1_CHUNK - 1) / PASS1_CHUNK;
    constexpr int CV = PASS1_CHUNK / 128;  // 16-byte vectors per lane per chunk
    const long long n_units = *(volatile const int32_t *)&ctl->unit_alloc;

    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->t_start = globaltimer_ns();

    const int wq = (int)((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % QUEUES) * 32;

    // Pass 1: one warp per unit = (work item, group of PASS1_GROUP chunks of
    // x), units ordered group-major so all warps sweep the same window of
    // columns.  Per chunk the row's slice stays in registers and four pairs'
    // column slices are loaded at a time; lane t keeps pair t's running
    // minimum, stored once per unit with a fire-and-forget atomic min.
    {
        const int ngroups = (nchunk + PASS1_GROUP - 1) / PASS1_GROUP;
        const int n1 = n_items * ngroups;   // items < 2^19 and groups <= 18 at the largest capacity
        int t = 0;
        if (lane == 0) t = atomicAdd(&ctl->q1[wq], 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        while (true) {
            const int u = (wq >> 5) + QUEUES * t;
            if (u >= n1 || u < 0) break;
            const int g = u / n_items, it = u - g * n_items;
            if (lane == 0) t = atomicAdd(&ctl->q1[wq], 1);   // next unit, in flight meanwhile
            const int4 item = __ldcg(d.items + it);
            const int cnt = item.z & 0xff;
            const int jl = lane < cnt ? __ldcg(d.pairs + item.y + lane) : 0;
            const T *Dr = d.D + (int64_t)item.x * ld;
            T pacc = M::inf();
            for (int sc = 0; sc < PASS1_GROUP; ++sc) {
                const int x0 = (g * PASS1_GROUP + sc) * PASS1_CHUNK;
                if (x0 >= span) break;
                const int nv = (min(span, x0 + PASS1_CHUNK) - x0) / 4;
                const V4 *r4 = reinterpret_cast<const V4 *>(Dr + x0);
                V4 rv[CV];
#pragma unroll
                for (int k = 0; k < CV; ++k)
                    if (lane + 32 * k < nv) rv[k] = __ldcg(r4 + lane + 32 * k);
                for (int q = 0; q < cnt; q += 4) {
                    int jq[4];
                    jq[0] = __shfl_sync(0xffffffffu, jl, q);
#pragma unroll
                    for (int u4 = 1; u4 < 4; ++u4) {
                        const int jj = __shfl_sync(0xffffffffu, jl, (q + u4) & 31);
                        jq[u4] = q + u4 < cnt ? jj : jq[0];
                    }
                    V4 a[4][CV];
#pragma unroll
                    for (int u4 = 0; u4 < 4; ++u4) {
                        const V4 *c4 = reinterpret_cast<const V4 *>(cols + (int64_t)jq[u4] * ld + x0);
#pragma unroll
                        for (int k = 0; k < CV; ++k)
                            if (lane + 32 * k < nv) a[u4][k] = __ldcg(c4 + lane + 32 * k);
                    }
                    T acc[4];
#pragma unroll
                    for (int u4 = 0; u4 < 4; ++u4) {
                        acc[u4] = M::inf();
#pragma unroll
                        for (int k = 0; k < CV; ++k) {
                            if (lane + 32 * k < nv) {
                                acc[u4] = M::add_min(rv[k].x, a[u4][k].x, acc[u4]);
                                acc[u4] = M::add_min(rv[k].y, a[u4][k].y, acc[u4]);
                                acc[u4] = M::add_min(rv[k].z, a[u4][k].z, acc[u4]);
                                acc[u4] = M::add_min(rv[k].w, a[u4][k].w, acc[u4]);
                            }
                        }
                    }
                    const T r = warp_min4(acc[0], acc[1], acc[2], acc[3], lane);
                    // pair q + g' sits in lanes 8g'..8g'+7; hand it to lane q + g'
                    const T got = __shfl_sync(0xffffffffu, r, ((lane - q) * 8) & 31);
                    if (lane >= q && lane < q + 4) pacc = M::mn(pacc, got);
                }
            }
            if (lane < cnt) atomicMin(d.pmin + item.y + lane, M::key(pacc));
            t = __shfl_sync(0xffffffffu, t, 0);
        }
    }
    int pass = 1;
    auto leader = [&]() {
        volatile Ctl *cv = ctl;
        const int par = pass & 1;
        cv->stop = pass >= 2 && cv->changed[par] == 0;
        cv->changed[par ^ 1] = 0;
        for (int q = 0; q < QUEUES; ++q) cv->qn[par ^ 1][32 * q] = 0;
        cv->passes = pass;
        const unsigned long long now = globaltimer_ns();
        if (pass == 1) cv->t_pass1 = now;
        cv->t_end = now;
    };
    if (!grid_barrier(ctl, leader)) return;

    // Passes >= 2: one warp per unit = (work item, segment of YSEG of the
    // row's listed targets y); lane t owns pair t of the item and gathers
    // D[y][j_t] for up to 8 y at a time.  Pass 2 reads D[i][.] of listed
    // pairs from pmin and stores every pair; later passes store only pairs
    // they lower.  Stores are atomic minima (several units share a pair).
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
            T cur = M::inf();
            if (mine) {
                j = __ldcg(d.pairs + item.y + lane);
                cur = pass == 2 ? M::unkey(__ldcg(d.pmin + item.y + lane)) : __ldcg(Di + j);
            }
            const int y1 = min(nrow, (seg + 1) * YSEG);
            T acc = M::inf();
            for (int s = seg * YSEG; s < y1; s += 32) {
                const int yi = s + lane;
                int y = 0;
                T dy = M::inf();
                bool ok = false;
                if (yi < y1) {
                    y = __ldcg(d.pairs + item.w + yi);
                    if (pass == 2) {
                        dy = M::unkey(__ldcg(d.pmin + item.w + yi));
                        ok = true;
                    } else if ((int)__ldcg(d.pstamp + item.w + yi) >= pass - 1) {
                        dy = __ldcg(Di + y);
                        ok = true;
                    }
                }
                unsigned m = __ballot_sync(0xffffffffu, ok);
                while (m) {
                    int ys[8];
                    T dys[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int src = m ? __ffs(m) - 1 : 0;
                        const bool has = m != 0;
                        m &= m - 1;
                        ys[e] = __shfl_sync(0xffffffffu, y, src);
                        const T dd = __shfl_sync(0xffffffffu, dy, src);
                        dys[e] = has ? dd : M::inf();
                    }
                    T v[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        v[e] = (mine && dys[e] < cur) ? __ldcg(d.D + (int64_t)ys[e] * ld + j) : M::inf();
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc = M::add_min(dys[e], v[e], acc);
                }
            }
            if (seg == 0 && lane == 0) evals += cnt;
            const bool lower = mine && acc < cur;
            if (mine && (pass == 2 || lower)) {
                const int32_t key = M::key(M::mn(acc, cur));
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

// Warm repair (cooperative launch): restricted re-relaxation.
template <typename T>
__global__ void __launch_bounds__(256, 3) k_repair_warm(Dev<T> d, RepairCfg cfg) {
    float cost, pw, pc;
    int n_items;
    const int reason = repair_decide(d.ctl, cfg, &cost, &pw, &pc, &n_items);
    if (reason != 0) {
        if (reason < 0) repair_record(d.ctl, reason, cost, pw, pc);
        return;
    }
    repair_record(d.ctl, reason, cost, pw, pc);
    repair_warm<T>(d, n_items);
}

// Cold repair (cooperative launch): persistent blocked Floyd-Warshall,
// running only when the decision says cold.
template <typename T>
__global__ void __launch_bounds__(256, 2) k_repair_cold(Dev<T> d, RepairCfg cfg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float cost, pw, pc;
    int n_items;
    const int reason = repair_decide(d.ctl, cfg, &cost, &pw, &pc, &n_items);
    if (reason <= 0) return;
    repair_record(d.ctl, reason, cost, pw, pc);
    repair_cold<T>(d, smem_raw);
}

}  // namespace apsp
