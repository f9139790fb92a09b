// Minimax (bottleneck) distances: the variant named in the paper's
// Discussion, where a path's value is its largest edge weight and the
// distance is the least such value over all paths.  The warm-start steps of
// Sections 3.1-3.3 carry over with max in place of +:
//   - adding p: out[c] = min_t max(w(p, t), D[t][c]) (Corollary 1),
//     in[r] = min_t max(D[r][t], w(t, p)) (Corollary 2), then
//     D[i][j] = min(D[i][j], max(in[i], out[j])) (Theorem 3);
//   - removing k: Corollary 3's test becomes max(D[i][k], D[k][j]) <= D[i][j]
//     (ties are the rule under max, so the test is "not strictly below");
//     listed pairs restart from their direct edge and are re-relaxed,
//     D[i][j] = min(D[i][j], min over x of max(D[i][x], D[x][j])), until a
//     pass lowers nothing (or the update goes cold: Floyd-Warshall in the
//     (min, max) semiring);
//   - a decreased edge (u, v): D[i][j] = min(D[i][j], max(D[i][u], w,
//     D[v][j])), exact because a best path to u or from v never uses (u, v);
//   - an increased edge: the removal's test with max(D[i][u], w_old, D[v][j])
//     as the path through the edge, starting bounds min(W'[i][j],
//     max(D[i][u], w_new, D[v][j])).
// max and min are exact in int32 and fp32, so every test is exact and no
// slack is needed.  Listed pairs are kept as a bitmask of one bit per (i, j).
#pragma once

#include "kernels.cuh"

namespace apsp {

constexpr int MM_CB = 512;   // columns per CTA of the insertion reduce

// Corollaries 1 and 2 with max: one pass over D.  Dead rows and columns hold
// missing in D and the masked weights, so no liveness test is needed.
template <typename T>
__global__ void __launch_bounds__(256) k_mm_insert_reduce(Dev<T> d, int rows_per_cta) {
    using M = MinMax<T>;
    using V4 = typename M::V4;
    __shared__ T red[8][MM_CB];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c0 = blockIdx.x * MM_CB;
    const int r0 = blockIdx.y * rows_per_cta;
    const int r1 = min(d.span, r0 + rows_per_cta);
    T win[16], col[16];
    bool cin[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        cin[q] = c0 + q * 128 + lane * 4 < d.span;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = c0 + q * 128 + lane * 4 + e;
            win[q * 4 + e] = c < d.span ? d.w_in[c] : M::inf();
            col[q * 4 + e] = M::inf();
        }
    }
    for (int row = r0 + w; row < r1; row += 8) {
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
            const T e4[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
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
    for (int c = threadIdx.x; c < MM_CB; c += blockDim.x) {
        T m = red[0][c];
#pragma unroll
        for (int k = 1; k < 8; ++k) m = M::mn(m, red[k][c]);
        if (c0 + c < d.span && M::finite(m)) atomicMin(&d.vout_k[c0 + c], M::key(m));
    }
}

// Theorem 3 with max, one CTA per row: D[i][j] = min(D[i][j], max(in[i],
// out[j])) on live rows (with DT kept in step), row p = out, column p = in.
template <typename T>
__global__ void __launch_bounds__(256) k_mm_insert_relax(Dev<T> d, int p) {
    using M = MinMax<T>;
    for (int r = blockIdx.x; r < d.span; r += gridDim.x) {
        T *Dr = d.D + (int64_t)r * d.ld;
        if (r == p) {
            for (int c = threadIdx.x; c < d.span; c += blockDim.x) {
                const T o = c == p ? (T)0 : M::unkey(d.vout_k[c]);
                Dr[c] = o;
                if (d.DT) d.DT[(int64_t)c * d.ld + p] = o;
            }
            continue;
        }
        if (!d.alive[r]) continue;
        const T vi = M::unkey(d.vin_k[r]);
        if (M::finite(vi)) {
            for (int c = threadIdx.x; c < d.span; c += blockDim.x) {
                const T cand = M::add(vi, M::unkey(d.vout_k[c]));
                if (cand < Dr[c]) {
                    Dr[c] = cand;
                    if (d.DT) d.DT[(int64_t)c * d.ld + r] = cand;
                }
            }
        }
        __syncthreads();   // column p may have been written above
        if (threadIdx.x == 0) {
            Dr[p] = vi;
            if (d.DT) d.DT[(int64_t)p * d.ld + r] = vi;
        }
    }
}

// The new node's weights into W (row / column p), and p becomes live.
template <typename T> __global__ void k_mm_insert_finish(Dev<T> d, int p) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.span) return;
    d.W[(int64_t)p * d.ld + c] = c == p ? (T)0 : d.w_out[c];
    d.W[(int64_t)c * d.ld + p] = c == p ? (T)0 : d.w_in[c];
    if (c == p) d.alive[p] = 1;
}

// Path legs: x[i] = D[i][a], y[i] = D[b][i] (and, for an undirected edge,
// x2[i] = D[i][b], y2[i] = D[a][i]).  For an edge update thread 0 also
// writes the new weight into W (both orientations when undirected).
template <typename T> __global__ void k_mm_legs(Dev<T> d, int a, int b, int two, int set_w, T w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && set_w) {
        d.W[(int64_t)a * d.ld + b] = w;
        if (d.undirected) d.W[(int64_t)b * d.ld + a] = w;
    }
    if (i >= d.span) return;
    d.x[i] = col_src(d, a, i);
    d.y[i] = d.D[(int64_t)b * d.ld + i];
    if (two) {
        d.x2[i] = col_src(d, b, i);
        d.y2[i] = d.D[(int64_t)a * d.ld + i];
    }
}

// Removal of k: row and column k of D, DT and W become missing, k dead.
template <typename T> __global__ void k_mm_tomb(Dev<T> d, int k) {
    using M = MinMax<T>;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.span) return;
    const T inf = M::inf();
    d.D[(int64_t)k * d.ld + c] = inf;
    d.D[(int64_t)c * d.ld + k] = inf;
    d.W[(int64_t)k * d.ld + c] = inf;
    d.W[(int64_t)c * d.ld + k] = inf;
    if (d.DT) {
        d.DT[(int64_t)k * d.ld + c] = inf;
        d.DT[(int64_t)c * d.ld + k] = inf;
    }
    if (c == k) d.alive[k] = 0;
}

// Affected pairs (one warp per row, 32 columns per step, a ballot per mask
// word).  kind 0, removal of node a: the path through it is
// max(x[i], y[j]); kind 1, increase of edge (a, b) from w_old: the path
// through the edge is max(x[i], w_old, y[j]) (and max(x2[i], w_old, y2[j])
// for an undirected edge).  (i, j) is listed iff i != j are live (and not
// the removed node), D[i][j] is finite and the path through is not above it.
// A listed pair gets its starting bound in D (and DT): the direct edge W[i][j]
// (W already holds an increased edge's new weight), for an increase also the
// path through the edge at its new weight.  Rows holding a pair are listed in
// rlist; counts go to the control block.
template <typename T, bool TWO>
__global__ void __launch_bounds__(256) k_mm_detect(Dev<T> d, uint32_t *mask, int words, int kind, int a, T w_old,
                                                   T w_new) {
    using M = MinMax<T>;
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < d.span; i += nw) {
        uint32_t *mrow = mask + (int64_t)i * words;
        const bool row_ok = d.alive[i] && !(kind == 0 && i == a);
        const T xi = d.x[i];
        const T xi2 = TWO ? d.x2[i] : M::inf();
        int cnt = 0;
        for (int c0 = 0; c0 < d.span; c0 += 32) {
            const int c = c0 + lane;
            bool hit = false;
            T sb = M::inf();
            if (row_ok && c != i && !(kind == 0 && c == a) && d.alive[c]) {
                const T dij = d.D[(int64_t)i * d.ld + c];
                if (M::finite(dij)) {
                    T via = kind == 0 ? M::add(xi, d.y[c]) : M::add(M::add(xi, w_old), d.y[c]);
                    hit = M::tight(via, dij);
                    if (TWO) hit = hit || M::tight(M::add(M::add(xi2, w_old), d.y2[c]), dij);
                    if (hit) {
                        sb = d.W[(int64_t)i * d.ld + c];
                        if (kind == 1) {
                            sb = M::mn(sb, M::add(M::add(xi, w_new), d.y[c]));
                            if (TWO) sb = M::mn(sb, M::add(M::add(xi2, w_new), d.y2[c]));
                        }
                        d.D[(int64_t)i * d.ld + c] = sb;
                        if (d.DT) d.DT[(int64_t)c * d.ld + i] = sb;
                    }
                }
            }
            const uint32_t word = __ballot_sync(0xffffffffu, hit);
            if (lane == 0) mrow[c0 >> 5] = word;
            cnt += __popc(word);
        }
        for (int wd = (d.span >> 5) + lane; wd < words; wd += 32) mrow[wd] = 0u;
        if (lane == 0 && cnt) {
            atomicAdd(&d.ctl->n_pairs, (unsigned long long)cnt);
            const int r = atomicAdd(&d.ctl->r_count, 1);
            d.rlist[r] = i;
            atomicAdd(&d.ctl->n_rows, 1);
        }
    }
}

// One re-relaxation pass over the listed pairs (one warp per listed row):
//     D[i][j] = min(D[i][j], min over x of max(D[i][x], D[x][j]))
// reading row i and row j of DT (column j of D) in 16-byte vectors.  Values
// are written as they are found; readers see either value, and both are
// achievable path values.  Pass p runs only if pass p - 1 lowered a pair,
// and records in mm_changed[p] whether it lowered one: a pass that lowers
// nothing leaves the fixed point, which is exact.
template <typename T>
__global__ void __launch_bounds__(256) k_mm_pass(Dev<T> d, const uint32_t *mask, int words, int pass) {
    using M = MinMax<T>;
    using V4 = typename M::V4;
    Ctl *ctl = d.ctl;
    if (pass > 1 && *(volatile int32_t *)&ctl->mm_changed[pass - 1] == 0) return;
    const int lane = threadIdx.x & 31;
    const int nrows = *(volatile int32_t *)&ctl->r_count;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const T *cols = d.DT ? d.DT : d.D;
    const int nv = d.span / 4;
    bool changed = false;
    for (int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < nrows; r += nw) {
        const int i = d.rlist[r];
        T *Di = d.D + (int64_t)i * d.ld;
        const V4 *ri = reinterpret_cast<const V4 *>(Di);
        for (int w0 = 0; w0 < words; w0 += 32) {
            const uint32_t my = w0 + lane < words ? mask[(int64_t)i * words + w0 + lane] : 0u;
            for (unsigned nz = __ballot_sync(0xffffffffu, my != 0u); nz; nz &= nz - 1) {
                const int src = __ffs(nz) - 1;
                uint32_t m = __shfl_sync(0xffffffffu, my, src);
                while (m) {
                    const int j = (w0 + src) * 32 + __ffs(m) - 1;
                    m &= m - 1;
                    const V4 *cj = reinterpret_cast<const V4 *>(cols + (int64_t)j * d.ld);
                    T a0 = M::inf(), a1 = M::inf();
                    for (int v4 = lane; v4 < nv; v4 += 32) {
                        const V4 x = __ldcg(ri + v4), y = __ldcg(cj + v4);
                        a0 = M::add_min(x.x, y.x, a0);
                        a1 = M::add_min(x.y, y.y, a1);
                        a0 = M::add_min(x.z, y.z, a0);
                        a1 = M::add_min(x.w, y.w, a1);
                    }
                    const T best = warp_min(M::mn(a0, a1));
                    if (lane == 0 && M::lowers(best, __ldcg(Di + j))) {
                        Di[j] = best;
                        if (d.DT) d.DT[(int64_t)j * d.ld + i] = best;
                        changed = true;
                    }
                }
            }
        }
    }
    if (changed) *(volatile int32_t *)&ctl->mm_changed[pass] = 1;
}

// A decreased edge (a, b) with new weight w: rows with max(x[i], w) below
// D[i][b] (or, undirected, max(x2[i], w) below D[i][a]) can change; those
// rows take D[i][j] = min(D[i][j], max(x[i], w, y[j])) (and the reverse
// orientation), with DT in step.  One warp per row.
template <typename T, bool TWO>
__global__ void __launch_bounds__(256) k_mm_decrease(Dev<T> d, int a, int b, T w) {
    using M = MinMax<T>;
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < d.span; i += nw) {
        if (!d.alive[i]) continue;
        T *Di = d.D + (int64_t)i * d.ld;
        const T a1 = M::add(d.x[i], w);
        const T a2 = TWO ? M::add(d.x2[i], w) : M::inf();
        if (!(a1 < Di[b] || (TWO && a2 < Di[a]))) continue;   // uniform across the warp
        if (lane == 0) atomicAdd(&d.ctl->r_count, 1);
        for (int c = lane; c < d.span; c += 32) {
            if (c == i) continue;
            T cand = M::add(a1, d.y[c]);
            if (TWO) cand = M::mn(cand, M::add(a2, d.y2[c]));
            if (cand < Di[c]) {
                Di[c] = cand;
                if (d.DT) d.DT[(int64_t)c * d.ld + i] = cand;
            }
        }
    }
}

}  // namespace apsp
