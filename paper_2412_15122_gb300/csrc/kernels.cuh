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
    int4 *items;              // (row, first pair, pair count, 0)
    int32_t *pairs;           // affected column per pair, grouped by row
    Ctl *ctl;
    int64_t pair_cap;
    int32_t item_cap;
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
// Tile: 256 rows x 512 columns per CTA; each lane owns 16 columns; partial
// results meet in global memory through atomicMin on ordered keys.
constexpr int INS_RB = 256, INS_CB = 512;

template <typename T>
__global__ void __launch_bounds__(256) k_insert_reduce(Dev<T> d) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    __shared__ T red[8][INS_CB];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c0 = blockIdx.x * INS_CB, r0 = blockIdx.y * INS_RB;
    T win[16], col[16];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            int c = c0 + q * 128 + lane * 4 + e;
            win[q * 4 + e] = c < d.span ? d.w_in[c] : M::inf();
            col[q * 4 + e] = M::inf();
        }
#pragma unroll 2
    for (int t = 0; t < INS_RB / 8; ++t) {
        int row = r0 + w + 8 * t;
        if (row >= d.span) break;
        if (!d.alive[row]) continue;
        T wo = d.w_out[row];
        T racc = M::inf();
        const T *Dr = d.D + (int64_t)row * d.ld;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int c = c0 + q * 128 + lane * 4;
            if (c < d.span) {
                V4 v = *reinterpret_cast<const V4 *>(Dr + c);
                T e4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    col[q * 4 + e] = M::add_min(wo, e4[e], col[q * 4 + e]);
                    racc = M::add_min(e4[e], win[q * 4 + e], racc);
                }
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

// Theorem 3 sweep: D[i][j] = min(D[i][j], in[i] + out[j]), then row p = out,
// column p = in, D[p][p] = 0, and the weights of p.  Rows are visited in the
// reverse of the reduction's order so its last rows are still in L2.
template <typename T>
__global__ void __launch_bounds__(256) k_insert_relax(Dev<T> d, int p) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *so = reinterpret_cast<T *>(smem_raw);
    const int span = d.span;
    for (int c = threadIdx.x; c < span; c += blockDim.x) so[c] = M::unkey(d.vout_k[c]);
    __syncthreads();
    const V4 *so4 = reinterpret_cast<const V4 *>(so);
    for (int r = blockIdx.x; r < span; r += gridDim.x) {
        const int row = span - 1 - r;
        if (row == p) {
            for (int c = threadIdx.x; c < span; c += blockDim.x) {
                T o = c == p ? (T)0 : so[c];
                d.D[(int64_t)p * d.ld + c] = o;
                d.W[(int64_t)p * d.ld + c] = c == p ? (T)0 : d.w_out[c];
                if (d.DT) d.DT[(int64_t)c * d.ld + p] = o;
            }
            if (threadIdx.x == 0) d.alive[p] = 1;
            continue;
        }
        if (!d.alive[row]) continue;
        const T vi = M::unkey(d.vin_k[row]);
        if (!M::finite(vi)) continue;
        T *Dr = d.D + (int64_t)row * d.ld;
        for (int c4 = threadIdx.x; c4 < span / 4; c4 += blockDim.x) {
            V4 v = *reinterpret_cast<const V4 *>(Dr + 4 * c4);
            V4 o = so4[c4];
            T dv[4] = {v.x, v.y, v.z, v.w};
            T ov[4] = {o.x, o.y, o.z, o.w};
            bool any = false;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                T cand = vi + ov[e];
                if (cand < dv[e]) {
                    dv[e] = cand;
                    any = true;
                    if (d.DT) d.DT[(int64_t)(4 * c4 + e) * d.ld + row] = cand;
                }
            }
            if (any) {
                V4 nv; nv.x = dv[0]; nv.y = dv[1]; nv.z = dv[2]; nv.w = dv[3];
                *reinterpret_cast<V4 *>(Dr + 4 * c4) = nv;
            }
        }
        __syncthreads();  // the vector holding column p is written above
        if (threadIdx.x == 0) {
            Dr[p] = vi;
            d.W[(int64_t)row * d.ld + p] = d.w_in[row];
            if (d.DT) d.DT[(int64_t)p * d.ld + row] = vi;
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
__global__ void __launch_bounds__(256) k_dec_sweep(Dev<T> d, T w) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    const int nrows = *(volatile int32_t *)&d.ctl->r_count;
    const V4 *y4 = reinterpret_cast<const V4 *>(d.y);
    const V4 *y24 = reinterpret_cast<const V4 *>(d.y2);
    for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int i = d.rlist[r];
        const T a1 = M::add(d.x[i], w);
        const T a2 = d.undirected ? M::add(d.x2[i], w) : M::inf();
        T *Dr = d.D + (int64_t)i * d.ld;
        for (int c4 = threadIdx.x; c4 < d.span / 4; c4 += blockDim.x) {
            V4 v = *reinterpret_cast<const V4 *>(Dr + 4 * c4);
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
                *reinterpret_cast<V4 *>(Dr + 4 * c4) = nv;
            }
        }
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

template <typename T>
__global__ void k_rm_gather(Dev<T> d, int k) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.span) return;
    d.x[i] = col_src(d, k, i);                 // D[i][k]
    d.y[i] = d.D[(int64_t)k * d.ld + i];       // D[k][i]
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

// kind 0: removal of node a (rows: every live row != a)
// kind 1: increase of edge a -> b from w_old to w_new (rows: prepass list)
template <typename T>
__global__ void __launch_bounds__(256) k_detect(Dev<T> d, int kind, int a, int b, T w_old, T w_new) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int span = d.span;
    T *ys = reinterpret_cast<T *>(smem_raw);
    T *y2s = ys + span;
    int32_t *hits = reinterpret_cast<int32_t *>(y2s + (d.undirected ? span : 0));
    __shared__ int cnt_s, base_s, item_s, ovf_s;
    for (int c = threadIdx.x; c < span; c += blockDim.x) {
        ys[c] = d.y[c];
        if (d.undirected) y2s[c] = d.y2[c];
    }
    if (threadIdx.x == 0) cnt_s = 0;
    __syncthreads();
    const int nrows = kind == 0 ? span : *(volatile int32_t *)&d.ctl->r_count;
    for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int i = kind == 0 ? r : d.rlist[r];
        if (kind == 0 && (i == a || !d.alive[i])) continue;
        const T xi = d.x[i];
        const T x2i = (kind == 1 && d.undirected) ? d.x2[i] : M::inf();
        const T s1 = kind == 0 ? xi : M::add(xi, w_old);
        const T s2 = M::add(x2i, w_old);
        if (!M::finite(s1) && !M::finite(s2)) continue;
        const T *Dr = d.D + (int64_t)i * d.ld;
        const T *Wr = d.W + (int64_t)i * d.ld;
        for (int c4 = threadIdx.x; c4 < span / 4; c4 += blockDim.x) {
            V4 v = *reinterpret_cast<const V4 *>(Dr + 4 * c4);
            T dv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = 4 * c4 + e;
                const T dd = dv[e];
                if (j == i || !M::finite(dd)) continue;
                bool hit;
                if (kind == 0) {
                    hit = j != a && M::tight(M::add(s1, ys[j]), dd);
                } else {
                    hit = M::tight(M::add(s1, ys[j]), dd) ||
                          (d.undirected && M::tight(M::add(s2, y2s[j]), dd));
                }
                if (hit) {
                    const bool changed_edge = kind == 1 && ((i == a && j == b) || (d.undirected && i == b && j == a));
                    if (!changed_edge && Wr[j] == dd) hit = false;  // direct edge is a shortest path
                }
                if (hit) hits[atomicAdd(&cnt_s, 1)] = j;
            }
        }
        __syncthreads();
        const int n = cnt_s;
        __syncthreads();  // every thread has read n before cnt_s is reset
        if (n > 0) {
            if (threadIdx.x == 0) {
                cnt_s = 0;
                const int nit = (n + ITEM_PAIRS - 1) / ITEM_PAIRS;
                unsigned long long base = atomicAdd(&d.ctl->n_pairs, (unsigned long long)n);
                int ib = atomicAdd(&d.ctl->n_items, nit);
                atomicAdd(&d.ctl->n_rows, 1);
                int ovf = (base + n > (unsigned long long)d.pair_cap) || (ib + nit > d.item_cap);
                if (ovf) atomicOr(&d.ctl->overflow, 1);
                base_s = (int)(ovf ? 0 : base);
                item_s = ib;
                ovf_s = ovf;
            }
            __syncthreads();
            if (!ovf_s) {
                const int base = base_s;
                const T wn_x = kind == 1 ? M::add(xi, w_new) : M::inf();
                const T wn_x2 = kind == 1 ? M::add(x2i, w_new) : M::inf();
                for (int t = threadIdx.x; t < n; t += blockDim.x) {
                    const int j = hits[t];
                    d.pairs[base + t] = j;
                    T init = Wr[j];  // direct edge (new weight if it is the changed edge)
                    if (kind == 1) init = M::mn(init, M::mn(M::add(wn_x, ys[j]), M::add(wn_x2, d.undirected ? y2s[j] : M::inf())));
                    d.D[(int64_t)i * d.ld + j] = init;
                    if (d.DT) d.DT[(int64_t)j * d.ld + i] = init;
                }
                const int nit = (n + ITEM_PAIRS - 1) / ITEM_PAIRS;
                for (int t = threadIdx.x; t < nit; t += blockDim.x)
                    d.items[item_s + t] = make_int4(i, base + t * ITEM_PAIRS, min(ITEM_PAIRS, n - t * ITEM_PAIRS), 0);
            }
            __syncthreads();  // hits[] is reused by the next row
        }
    }
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
// Warm (restricted re-relaxation, replacing Algorithm 5's per-row Dijkstra):
// every listed pair starts at an achievable upper bound; each pass sets
//     D[i][j] = min(D[i][j], min_x D[i][x] + D[x][j])
// for the listed pairs only (row i staged in shared memory, column j read as
// row j of DT).  Unlisted pairs are exact and values only decrease, so a pass
// that changes nothing leaves the exact APSP matrix; path doubling bounds the
// passes by about log2(hops) + 2.
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

template <typename T>
__device__ void repair_warm(Dev<T> &d, int n_items, T *row_s) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    Ctl *ctl = d.ctl;
    __shared__ int item_sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int span = d.span;
    const T *cols = d.DT ? d.DT : d.D;
    int pass = 0;
    for (; pass < MAX_PASSES; ++pass) {
        const int par = pass & 1;
        while (true) {
            if (threadIdx.x == 0) item_sh = atomicAdd(&ctl->item_next[par], 1);
            __syncthreads();
            const int it = item_sh;
            if (it >= n_items) break;
            const int4 item = d.items[it];
            const int i = item.x;
            T *Dr = d.D + (int64_t)i * d.ld;
            V4 *row4 = reinterpret_cast<V4 *>(row_s);
            for (int c4 = threadIdx.x; c4 < span / 4; c4 += blockDim.x)
                row4[c4] = __ldcg(reinterpret_cast<const V4 *>(Dr) + c4);
            __syncthreads();
            bool changed = false;
            for (int q = warp; q < item.z; q += nwarps) {
                const int j = d.pairs[item.y + q];
                const V4 *cj = reinterpret_cast<const V4 *>(cols + (int64_t)j * d.ld);
                T acc0 = M::inf(), acc1 = M::inf();
#pragma unroll 4
                for (int c4 = lane; c4 < span / 4; c4 += 32) {
                    V4 av = row4[c4];
                    V4 bv = __ldcg(cj + c4);
                    acc0 = M::add_min(av.x, bv.x, acc0);
                    acc1 = M::add_min(av.y, bv.y, acc1);
                    acc0 = M::add_min(av.z, bv.z, acc0);
                    acc1 = M::add_min(av.w, bv.w, acc1);
                }
                T acc = warp_min(M::mn(acc0, acc1));
                if (lane == 0) {
                    T cur = __ldcg(Dr + j);
                    if (acc < cur) {
                        Dr[j] = acc;
                        if (d.DT) d.DT[(int64_t)j * d.ld + i] = acc;
                        changed = true;
                    }
                }
            }
            if (changed) *(volatile int32_t *)&ctl->changed[par] = 1;
            __syncthreads();
        }
        const bool ok = grid_barrier(ctl, [&]() {
            volatile Ctl *c = ctl;
            int ch = c->changed[par];
            c->stop = ch == 0;
            c->changed[par ^ 1] = 0;
            c->item_next[par ^ 1] = 0;
            c->passes = pass + 1;
        });
        if (!ok) return;
        if (*(volatile int32_t *)&ctl->stop) break;
    }
    if (pass == MAX_PASSES && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ctl->err, ERR_PASSES);
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


template <typename T>
__global__ void __launch_bounds__(256) k_repair(Dev<T> d, RepairCfg cfg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Ctl *ctl = d.ctl;
    const int trivial = *(volatile int32_t *)&ctl->trivial;
    const int n_items = *(volatile int32_t *)&ctl->n_items;
    const int ovf = *(volatile int32_t *)&ctl->overflow;
    const int rows = *(volatile int32_t *)&ctl->n_rows;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    if (trivial || (n_items == 0 && !ovf)) {
        if (lead) ctl->path = PATH_TRIVIAL;
        return;
    }
    const float cost = (float)rows / (float)max(1, cfg.n_live_before - 1);
    int cold_reason = 0;
    float pw = 0.f, pc = 0.f;
    if (ovf) cold_reason = 4;
    else if (cfg.mode == 2) cold_reason = 3;
    else if (cfg.mode == 3 && cfg.has_model) {
        const float n = (float)max(2, cfg.n_live_before);
        const unsigned long long np = *(volatile unsigned long long *)&ctl->n_pairs;
        float feat[MLP_IN] = {cfg.feat_type, log2f(n), cfg.feat_dw, (float)np / (n * n), cost,
                              (float)rows / n};
        __shared__ float out[MLP_OUT];
        mlp_predict_cta(cfg.model, feat, out);
        pw = out[0];
        pc = out[1];
        if (pc < pw) cold_reason = 2;
    } else if (cfg.mode != 1 && cost > cfg.delta) cold_reason = 1;
    if (lead) {
        ctl->cost = cost;
        ctl->cold_reason = cold_reason;
        ctl->model_warm = pw;
        ctl->model_cold = pc;
        ctl->path = cold_reason ? PATH_COLD : PATH_WARM;
    }
    if (cold_reason) repair_cold<T>(d, smem_raw);
    else repair_warm<T>(d, n_items, reinterpret_cast<T *>(smem_raw));
}

}  // namespace apsp
