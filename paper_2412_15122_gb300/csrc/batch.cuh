// Batched execution: one persistent kernel applies a batch of updates to many
// independent graphs.  CTAs take graphs from a device queue; a CTA applies its
// graph's updates in order (each graph's sequence is causal, different graphs
// are independent), with the same steps as the single-graph path:
//   add       Corollary 1 / Corollary 2 as row reductions over D and D^T,
//             then the Theorem 3 sweep, then row / column p;
//   decrease  D = min(D, D[:,u] + w + D[v,:]) on rows with D[i][u] + w < D[i][v];
//   increase  tightness of the old edge, Corollary 3's test through it, and
//   removal   Corollary 3's test through the removed node (the
//             need_update_list of Section 3.2): listed pairs restart from an
//             achievable upper bound and are re-relaxed,
//                 D[i][j] = min over x of D[i][x] + D[x][j],
//             in full passes until a pass lowers nothing (the fixed point of
//             D = min(D, D (x) D) over the listed pairs is exact).
// Graphs are directed (D and D^T kept, row-major, ld = the graph's leading
// dimension); the host has already chosen new nodes' slots, read old edge
// weights from its mirror and masked new-node weight vectors.
#pragma once

#include "kernels.cuh"

namespace apsp {

enum : int32_t { BOP_ADD = 0, BOP_REMOVE = 1, BOP_DECREASE = 2, BOP_INCREASE = 3 };

struct BatchGraph {
    void *D, *DT, *W;         // T* (device)
    int32_t *alive;
    int64_t ld;
    uint32_t *mask;           // listed-pair bitmask scratch: mask_words words per row
    int32_t mask_words;
    int32_t first, count;     // this graph's updates in the batch's op array
    int32_t status;           // written by the kernel: 0, or ERR_* bits
};

struct BatchOp {
    int32_t op;
    int32_t a, b;             // add: slot p; remove: k; edges: (u, v)
    int32_t span;             // slots covered by the graph's sweeps during this update
    int64_t vec;              // add: element offset of in_w then out_w (span each) in the vector arena
    int32_t w_bits, w_old_bits;   // edges: new and old weight (bit patterns of T)
};

struct BatchHeader {
    BatchGraph *graphs;
    const BatchOp *ops;
    const void *vecs;
    int32_t n_graphs;
    int32_t max_span;         // largest span of any update (sizes the shared arrays)
    int32_t queue;            // next graph to take
    int32_t pad_;
    volatile int32_t *done;   // optional (mapped host memory): 1 + status per graph when it is finished
};

template <typename T> __device__ __forceinline__ T bits_as(int32_t b) {
    if constexpr (std::is_same<T, float>::value) return __int_as_float(b);
    else return (T)b;
}

template <typename T> struct BG {
    T *D, *DT, *W;
    int32_t *alive;
    int64_t ld;
    __device__ T &d(int i, int j) const { return D[(int64_t)i * ld + j]; }
    __device__ T &dt(int i, int j) const { return DT[(int64_t)i * ld + j]; }
    __device__ T &w(int i, int j) const { return W[(int64_t)i * ld + j]; }
    __device__ void set(int i, int j, T v) const {
        D[(int64_t)i * ld + j] = v;
        DT[(int64_t)j * ld + i] = v;
    }
};

// A warp walks vectors [0, span/4) of a row, 4 vectors per lane in flight,
// calling f(c4, v) for each.
template <typename V4, typename F> __device__ __forceinline__ void b_row(const V4 *row, int nv4, F &&f) {
    const int lane = threadIdx.x & 31;
    for (int c0 = lane; c0 < nv4; c0 += 128) {
        V4 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (c0 + 32 * k < nv4) v[k] = __ldcg(row + c0 + 32 * k);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (c0 + 32 * k < nv4) f(c0 + 32 * k, v[k]);
    }
}

// Warp-wide min over x < span of D[i][x] + D[x][j] (D[x][j] read as D^T row j).
template <typename T> __device__ __forceinline__ T b_dot_min(const BG<T> &g, int i, int j, int span) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    const int lane = threadIdx.x & 31;
    const V4 *r4 = reinterpret_cast<const V4 *>(g.D + (int64_t)i * g.ld);
    const V4 *c4 = reinterpret_cast<const V4 *>(g.DT + (int64_t)j * g.ld);
    const int nv4 = span / 4;
    T acc = M::inf();
    for (int v0 = lane; v0 < nv4; v0 += 128) {
        V4 a[4], b[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (v0 + 32 * k < nv4) {
                a[k] = __ldcg(r4 + v0 + 32 * k);
                b[k] = __ldcg(c4 + v0 + 32 * k);
            }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (v0 + 32 * k < nv4) {
                acc = M::add_min(a[k].x, b[k].x, acc);
                acc = M::add_min(a[k].y, b[k].y, acc);
                acc = M::add_min(a[k].z, b[k].z, acc);
                acc = M::add_min(a[k].w, b[k].w, acc);
            }
    }
    return warp_min(acc);
}

// Re-relaxes the listed pairs (bitmask rows of `words` words; the rows
// holding any are rows[0, nrows)) in full passes until a pass lowers
// nothing; returns false when the pass cap is reached.
template <typename T>
__device__ bool b_relax(const BG<T> &g, const uint32_t *mask, int words, int span, const int32_t *rows, int nrows) {
    using M = MinPlus<T>;
    __shared__ int changed_s;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int pass = 0; pass < MAX_PASSES; ++pass) {
        if (threadIdx.x == 0) changed_s = 0;
        __syncthreads();
        bool changed = false;
        for (int r = wid; r < nrows; r += nw) {
            const int i = rows[r];
            for (int w0 = 0; w0 < words; w0 += 32) {
                const uint32_t my = w0 + lane < words ? __ldcg(mask + (int64_t)i * words + w0 + lane) : 0u;
                for (unsigned nz = __ballot_sync(0xffffffffu, my != 0u); nz; nz &= nz - 1) {
                    const int src = __ffs(nz) - 1;
                    uint32_t m = __shfl_sync(0xffffffffu, my, src);
                    while (m) {
                        const int j = (w0 + src) * 32 + __ffs(m) - 1;
                        m &= m - 1;
                        const T cand = b_dot_min(g, i, j, span);
                        if (lane == 0 && M::lowers(cand, __ldcg(&g.d(i, j)))) {
                            g.set(i, j, cand);
                            changed = true;
                        }
                    }
                }
            }
        }
        if (changed) changed_s = 1;
        __syncthreads();
        const int any = changed_s;
        __syncthreads();
        if (!any) return true;
    }
    return false;
}

// Clears rows [0, span) of the bitmask and the listed-row count.
__device__ __forceinline__ void b_clear_mask(uint32_t *mask, int words, int span, int *nrows_s) {
    for (int64_t t = threadIdx.x; t < (int64_t)span * words; t += blockDim.x) mask[t] = 0u;
    if (threadIdx.x == 0) *nrows_s = 0;
    __syncthreads();
}

// Node insertion at slot p with masked weights wi (t -> p) and wo (p -> t).
template <typename T>
__device__ __noinline__ void b_add(const BG<T> &g, int p, int span, const T *wi, const T *wo, T *s_in, T *s_out, T *s_wi,
                      T *s_wo) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nv4 = span / 4;
    for (int t = threadIdx.x; t < span; t += blockDim.x) {
        s_wi[t] = wi[t];
        s_wo[t] = wo[t];
    }
    __syncthreads();
    const V4 *wi4 = reinterpret_cast<const V4 *>(s_wi), *wo4 = reinterpret_cast<const V4 *>(s_wo);
    // Corollary 2: D[i][p] = min_t D[i][t] + w(t -> p); Corollary 1:
    // D[p][j] = min_t w(p -> t) + D[t][j], a row reduction over D^T row j
    for (int r = wid; r < span; r += nw) {
        T a = M::inf(), b = M::inf();
        if (g.alive[r] && r != p) {
            b_row(reinterpret_cast<const V4 *>(g.D + (int64_t)r * g.ld), nv4, [&](int c4, const V4 &v) {
                const V4 w = wi4[c4];
                a = M::mn(a, M::mn(M::mn(M::add(v.x, w.x), M::add(v.y, w.y)), M::mn(M::add(v.z, w.z), M::add(v.w, w.w))));
            });
            b_row(reinterpret_cast<const V4 *>(g.DT + (int64_t)r * g.ld), nv4, [&](int c4, const V4 &v) {
                const V4 w = wo4[c4];
                b = M::mn(b, M::mn(M::mn(M::add(v.x, w.x), M::add(v.y, w.y)), M::mn(M::add(v.z, w.z), M::add(v.w, w.w))));
            });
        }
        a = warp_min(a);
        b = warp_min(b);
        if (lane == 0) {
            s_in[r] = a;
            s_out[r] = b;
        }
    }
    __syncthreads();
    // Theorem 3: D[i][j] = min(D[i][j], D[i][p] + D[p][j]) (s_out[p] and the
    // dead columns are missing, so those entries never improve)
    if (threadIdx.x == 0) s_out[p] = M::inf();
    __syncthreads();
    for (int i = wid; i < span; i += nw) {
        const T vi = s_in[i];
        if (i == p || !M::finite(vi)) continue;
        T *Di = g.D + (int64_t)i * g.ld;
        b_row(reinterpret_cast<const V4 *>(Di), nv4, [&](int c4, const V4 &v) {
            const T dv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const T o = s_out[4 * c4 + e];
                if (M::finite(o) && vi + o < dv[e]) g.set(i, 4 * c4 + e, vi + o);
            }
        });
    }
    __syncthreads();
    for (int t = threadIdx.x; t < span; t += blockDim.x) {
        const T out_t = t == p ? (T)0 : s_out[t];
        const T in_t = t == p ? (T)0 : s_in[t];
        g.set(p, t, out_t);
        g.set(t, p, in_t);
        g.w(p, t) = t == p ? (T)0 : s_wo[t];
        g.w(t, p) = t == p ? (T)0 : s_wi[t];
    }
    __syncthreads();
    if (threadIdx.x == 0) g.alive[p] = 1;
    __syncthreads();
}

// Marks the entries j != i of row i with s + y[j] tight against D[i][j] in
// the row's bitmask words (bit j % 32 of word j / 32); returns whether any.
// Lane l holds 4 consecutive entries of each 128-entry block, so the bits of
// a 32-entry word come from 8 lanes and are combined with shuffles.
template <typename T>
__device__ __forceinline__ bool b_detect_row(const BG<T> &g, int i, T s, const T *sy, int span, uint32_t *mrow) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    const int lane = threadIdx.x & 31;
    bool any = false;
    b_row(reinterpret_cast<const V4 *>(g.D + (int64_t)i * g.ld), span / 4, [&](int c4, const V4 &v) {
        const T dv[4] = {v.x, v.y, v.z, v.w};
        uint32_t m = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = 4 * c4 + e;
            if (j != i && M::slack_tight(M::slack(s + sy[j], dv[e]))) m |= 1u << e;
        }
        // entries 4 c4 .. 4 c4 + 3 sit at bits 4 (c4 % 8) .. of word c4 / 8;
        // the row length is a multiple of 32 entries, so a word's 8 lanes
        // are active together (the last batch of a row may leave whole
        // groups out)
        const unsigned am = __activemask();
        m <<= 4 * (c4 & 7);
        m |= __shfl_xor_sync(am, m, 1);
        m |= __shfl_xor_sync(am, m, 2);
        m |= __shfl_xor_sync(am, m, 4);
        if ((lane & 7) == 0 && m) mrow[c4 >> 3] = m;
        any |= m != 0u;
    });
    return __any_sync(0xffffffffu, any);
}

// Edge decrease (u, v) -> w.
template <typename T> __device__ __noinline__ void b_decrease(const BG<T> &g, int u, int v, T w, int span, T *sx, T *sy) {
    using M = MinPlus<T>;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = threadIdx.x; t < span; t += blockDim.x) {
        sx[t] = __ldcg(&g.dt(u, t));   // D[t][u]
        sy[t] = __ldcg(&g.d(v, t));    // D[v][t]
    }
    __syncthreads();
    if (threadIdx.x == 0) g.w(u, v) = w;
    for (int i = wid; i < span; i += nw) {
        const T xi = sx[i];
        if (!M::finite(xi) || !(M::add(xi, w) < __ldcg(&g.dt(v, i)))) continue;   // row filter
        const T s = xi + w;
        b_row(reinterpret_cast<const typename M::V4 *>(g.D + (int64_t)i * g.ld), span / 4,
              [&](int c4, const typename M::V4 &dv4) {
                  const T dv[4] = {dv4.x, dv4.y, dv4.z, dv4.w};
#pragma unroll
                  for (int e = 0; e < 4; ++e) {
                      const T y = sy[4 * c4 + e];
                      if (M::finite(y) && s + y < dv[e]) g.set(i, 4 * c4 + e, s + y);
                  }
              });
    }
    __syncthreads();
}

// Edge increase (u, v): w_old -> w (w may be missing: a deletion).  Returns
// false on the pass cap.
template <typename T>
__device__ __noinline__ bool b_increase(const BG<T> &g, int u, int v, T w_old, T w, int span, uint32_t *mask, int words, T *sx,
                           T *sy, int32_t *rows, int *nrows_s) {
    using M = MinPlus<T>;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bool tight_edge = M::tight(w_old, __ldcg(&g.d(u, v)));
    __syncthreads();
    if (threadIdx.x == 0) g.w(u, v) = w;
    if (!tight_edge) {
        __syncthreads();
        return true;
    }
    for (int t = threadIdx.x; t < span; t += blockDim.x) {
        sx[t] = __ldcg(&g.dt(u, t));   // D[t][u]
        sy[t] = M::leg(__ldcg(&g.d(v, t)));
    }
    b_clear_mask(mask, words, span, nrows_s);
    // pairs whose distance is a path through the old edge (Corollary 3 for an edge)
    for (int i = wid; i < span; i += nw) {
        const T xi = sx[i];
        if (!M::finite(xi) || !g.alive[i]) continue;
        const T s = M::add(xi, w_old);
        if (!M::tight(s, __ldcg(&g.dt(v, i)))) continue;
        const bool any = b_detect_row(g, i, s, sy, span, mask + (int64_t)i * words);
        if (lane == 0 && any) rows[atomicAdd(nrows_s, 1)] = i;
    }
    __syncthreads();
    // starting upper bounds: the direct edge, or the path through the edge at its new weight
    const int nrows = *nrows_s;
    for (int r = wid; r < nrows; r += nw) {
        const int i = rows[r];
        for (int wd = 0; wd < words; ++wd) {
            const uint32_t m = mask[(int64_t)i * words + wd];
            const int j = wd * 32 + lane;
            if ((m >> lane) & 1u) {
                const T via = M::add(M::add(sx[i], w), M::mn(sy[j], M::inf()));
                g.set(i, j, M::mn(__ldcg(&g.w(i, j)), via));
            }
        }
    }
    __syncthreads();
    return b_relax(g, mask, words, span, rows, nrows);
}

// Removal of node k.  Returns false on the pass cap.
template <typename T>
__device__ __noinline__ bool b_remove(const BG<T> &g, int k, int span, uint32_t *mask, int words, T *sx, T *sy, int32_t *rows,
                         int *nrows_s) {
    using M = MinPlus<T>;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = threadIdx.x; t < span; t += blockDim.x) {
        sx[t] = __ldcg(&g.dt(k, t));                         // D[t][k]
        sy[t] = t == k ? unreachable_leg<T>() : M::leg(__ldcg(&g.d(k, t)));   // D[k][t]
    }
    b_clear_mask(mask, words, span, nrows_s);
    // need_update_list: D[i][k] + D[k][j] == D[i][j], i != j, both != k
    for (int i = wid; i < span; i += nw) {
        const T xi = sx[i];
        if (i == k || !M::finite(xi) || !g.alive[i]) continue;
        const bool any = b_detect_row(g, i, xi, sy, span, mask + (int64_t)i * words);
        if (lane == 0 && any) rows[atomicAdd(nrows_s, 1)] = i;
    }
    __syncthreads();
    // tombstone k (Section 3.2: its distances become infinite), then the
    // listed pairs restart from their direct edges
    const T inf = M::inf();
    for (int t = threadIdx.x; t < span; t += blockDim.x) {
        g.set(k, t, inf);
        g.set(t, k, inf);
        g.w(k, t) = inf;
        g.w(t, k) = inf;
    }
    if (threadIdx.x == 0) g.alive[k] = 0;
    __syncthreads();
    const int nrows = *nrows_s;
    for (int r = wid; r < nrows; r += nw) {
        const int i = rows[r];
        for (int wd = 0; wd < words; ++wd) {
            const uint32_t m = mask[(int64_t)i * words + wd];
            const int j = wd * 32 + lane;
            if ((m >> lane) & 1u) g.set(i, j, __ldcg(&g.w(i, j)));
        }
    }
    __syncthreads();
    return b_relax(g, mask, words, span, rows, nrows);
}

// Widths (threads per CTA) the executor's autotuner chooses from.
constexpr int BATCH_WIDTHS[3] = {128, 256, 512};

template <typename T, int NT> __global__ void __launch_bounds__(NT, 768 / NT) k_batch(BatchHeader *hdr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int gi_s, nrows_s;
    const T *vecs = reinterpret_cast<const T *>(hdr->vecs);
    while (true) {
        if (threadIdx.x == 0) gi_s = atomicAdd(&hdr->queue, 1);
        __syncthreads();
        const int gi = gi_s;
        __syncthreads();
        if (gi >= hdr->n_graphs) break;
        BatchGraph &bg = hdr->graphs[gi];
        BG<T> g{reinterpret_cast<T *>(bg.D), reinterpret_cast<T *>(bg.DT), reinterpret_cast<T *>(bg.W), bg.alive, bg.ld};
        T *s0 = reinterpret_cast<T *>(smem_raw);
        T *s1 = s0 + hdr->max_span;
        T *s2 = s1 + hdr->max_span;
        T *s3 = s2 + hdr->max_span;
        int32_t *srows = reinterpret_cast<int32_t *>(s3 + hdr->max_span);
        int err = 0;
        for (int q = bg.first; q < bg.first + bg.count; ++q) {
            const BatchOp op = hdr->ops[q];
            bool ok = true;
            if (op.op == BOP_ADD) {
                b_add<T>(g, op.a, op.span, vecs + op.vec, vecs + op.vec + op.span, s0, s1, s2, s3);
            } else if (op.op == BOP_DECREASE) {
                b_decrease<T>(g, op.a, op.b, bits_as<T>(op.w_bits), op.span, s0, s1);
            } else if (op.op == BOP_INCREASE) {
                ok = b_increase<T>(g, op.a, op.b, bits_as<T>(op.w_old_bits), bits_as<T>(op.w_bits), op.span, bg.mask,
                                   bg.mask_words, s0, s1, srows, &nrows_s);
            } else {
                ok = b_remove<T>(g, op.a, op.span, bg.mask, bg.mask_words, s0, s1, srows, &nrows_s);
            }
            if (!ok) err |= ERR_PASSES;
        }
        if (threadIdx.x == 0) {
            bg.status = err;
            if (hdr->done) {
                __threadfence_system();   // the graph's results are written before its flag
                hdr->done[gi] = 1 + err;
            }
        }
        __syncthreads();
    }
}

}  // namespace apsp
