// Batched execution: one persistent kernel applies a batch of updates to many
// independent graphs.  Each graph's updates are applied in order (a graph's
// sequence is causal, different graphs are independent), with the same steps
// as the single-graph path:
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
// Who works on a graph: large graphs (the first n_team of `order`) go to
// teams of team_size co-resident CTAs, team t taking large graphs t,
// t + n_teams, ...; the team splits each step's rows over all its warps and
// meets at a bounded team barrier between steps, with its scratch vectors in
// global memory.  Every other graph goes to a single CTA (scratch in shared
// memory, __syncthreads between steps) from a device queue, which the teams'
// CTAs also join once their large graphs are done.  The grid is never larger
// than the CTAs that fit on the device at once, so every team's CTAs run
// together.  Graphs are directed (D and D^T kept, row-major, ld = the graph's
// leading dimension); the host has already chosen new nodes' slots, read old
// edge weights from its mirror and masked new-node weight vectors.
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

// Per team, in global memory: 4 vectors of max_span elements, the listed rows
// (max_span), then the team's counters.
constexpr int TEAM_INTS = 8;   // nrows, changed, barrier count, barrier generation, spare
constexpr int TEAM_MAX = 8;    // largest team

struct BatchHeader {
    BatchGraph *graphs;
    const BatchOp *ops;
    const void *vecs;
    int32_t n_graphs;
    int32_t max_span;         // largest span of any update (sizes the scratch arrays)
    int32_t queue;            // next single-CTA graph to take
    int32_t n_team;           // order[0, n_team) go to teams
    int32_t team_size;        // CTAs per team (1: no teams)
    int32_t n_teams;
    const int32_t *order;     // graph indices: large ones first
    void *team_scratch;       // n_teams * team_stride bytes
    int64_t team_stride;
    volatile int32_t *done;   // optional (mapped host memory): 1 + status per graph when it is finished
};

// Who works on the current graph.  SOLO: this CTA alone.  Team: CTA `rank`
// of `size`; warps and threads are numbered across the team.
struct Team {
    int rank, size;
    int32_t *ints;            // team mode: nrows, changed, barrier count, generation
    __device__ int gw() const { return rank * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5); }
    __device__ int nw() const { return size * (int)(blockDim.x >> 5); }
    __device__ int gt() const { return rank * (int)blockDim.x + (int)threadIdx.x; }
    __device__ int nt() const { return size * (int)blockDim.x; }
    __device__ bool leader() const { return rank == 0 && threadIdx.x == 0; }
};

// Scratch shared by the team: shared memory for one CTA (plain loads), global
// memory for a team (loads bypass L1, where another CTA's writes are not seen).
template <bool TEAM, typename V> __device__ __forceinline__ V tld(const V *p) {
    if constexpr (TEAM) return __ldcg(p);
    else return *p;
}

// Barrier between the steps of an update.  A team's wait is bounded: after
// BARRIER_TIMEOUT_NS the CTA records ERR_TIMEOUT in *err and returns false.
template <bool TEAM> __device__ __forceinline__ bool team_sync(const Team &tm, int32_t *err) {
    if constexpr (!TEAM) {
        __syncthreads();
        return true;
    } else {
        __shared__ int ok_s;
        __syncthreads();
        if (threadIdx.x == 0) {
            volatile int32_t *gen = tm.ints + 3;
            const int32_t g0 = *gen;
            __threadfence();
            int ok = 1;
            if (atomicAdd(tm.ints + 2, 1) == tm.size - 1) {
                tm.ints[2] = 0;
                __threadfence();
                atomicAdd(tm.ints + 3, 1);
            } else {
                const unsigned long long t0 = globaltimer_ns();
                unsigned spins = 0;
                while (*gen == g0) {
                    __nanosleep(64);
                    if ((++spins & 1023u) == 0 && globaltimer_ns() - t0 > BARRIER_TIMEOUT_NS) {
                        atomicOr(err, (int32_t)ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
            __threadfence();
            ok_s = ok;
        }
        __syncthreads();
        return ok_s != 0;
    }
}

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
// nothing; returns false when the pass cap is reached or a team wait gave up.
template <typename T, bool TEAM>
__device__ bool b_relax(const BG<T> &g, const Team &tm, int32_t *err, const uint32_t *mask, int words, int span,
                        const int32_t *rows, int nrows, int32_t *changed_p) {
    using M = MinPlus<T>;
    const int lane = threadIdx.x & 31, wid = tm.gw(), nw = tm.nw();
    for (int pass = 0; pass < MAX_PASSES; ++pass) {
        if (tm.leader()) *changed_p = 0;
        if (!team_sync<TEAM>(tm, err)) return false;
        bool changed = false;
        for (int r = wid; r < nrows; r += nw) {
            const int i = tld<TEAM>(rows + r);
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
        if (changed) atomicExch(changed_p, 1);
        if (!team_sync<TEAM>(tm, err)) return false;
        const int any = tld<TEAM>(changed_p);
        if (!team_sync<TEAM>(tm, err)) return false;
        if (!any) return true;
    }
    return false;
}

// Clears rows [0, span) of the bitmask and the listed-row count.
template <bool TEAM>
__device__ __forceinline__ bool b_clear_mask(const Team &tm, int32_t *err, uint32_t *mask, int words, int span,
                                             int32_t *nrows_p) {
    for (int64_t t = tm.gt(); t < (int64_t)span * words; t += tm.nt()) mask[t] = 0u;
    if (tm.leader()) *nrows_p = 0;
    return team_sync<TEAM>(tm, err);
}

// Node insertion at slot p with masked weights wi (t -> p) and wo (p -> t).
template <typename T, bool TEAM>
__device__ __noinline__ bool b_add(const BG<T> &g, const Team &tm, int32_t *err, int p, int span, const T *wi,
                                   const T *wo, T *s_in, T *s_out, T *s_wi, T *s_wo) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    const int lane = threadIdx.x & 31, wid = tm.gw(), nw = tm.nw();
    const int nv4 = span / 4;
    if constexpr (TEAM) {   // the host-written vectors are read where they are
        s_wi = const_cast<T *>(wi);
        s_wo = const_cast<T *>(wo);
    } else {
        for (int t = threadIdx.x; t < span; t += blockDim.x) {
            s_wi[t] = wi[t];
            s_wo[t] = wo[t];
        }
        __syncthreads();
    }
    const V4 *wi4 = reinterpret_cast<const V4 *>(s_wi), *wo4 = reinterpret_cast<const V4 *>(s_wo);
    // Corollary 2: D[i][p] = min_t D[i][t] + w(t -> p); Corollary 1:
    // D[p][j] = min_t w(p -> t) + D[t][j], a row reduction over D^T row j
    for (int r = wid; r < span; r += nw) {
        T a = M::inf(), b = M::inf();
        if (__ldcg(g.alive + r) && r != p) {
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
            s_out[r] = r == p ? M::inf() : b;   // s_out[p] stays missing: those entries never improve
        }
    }
    if (!team_sync<TEAM>(tm, err)) return false;
    // Theorem 3: D[i][j] = min(D[i][j], D[i][p] + D[p][j]) (s_out[p] and the
    // dead columns are missing, so those entries never improve)
    for (int i = wid; i < span; i += nw) {
        const T vi = tld<TEAM>(s_in + i);
        if (i == p || !M::finite(vi)) continue;
        T *Di = g.D + (int64_t)i * g.ld;
        b_row(reinterpret_cast<const V4 *>(Di), nv4, [&](int c4, const V4 &v) {
            const T dv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const T o = tld<TEAM>(s_out + 4 * c4 + e);
                if (M::finite(o) && vi + o < dv[e]) g.set(i, 4 * c4 + e, vi + o);
            }
        });
    }
    if (!team_sync<TEAM>(tm, err)) return false;
    for (int t = tm.gt(); t < span; t += tm.nt()) {
        const T out_t = t == p ? (T)0 : tld<TEAM>(s_out + t);
        const T in_t = t == p ? (T)0 : tld<TEAM>(s_in + t);
        g.set(p, t, out_t);
        g.set(t, p, in_t);
        g.w(p, t) = t == p ? (T)0 : s_wo[t];
        g.w(t, p) = t == p ? (T)0 : s_wi[t];
    }
    if (tm.leader()) g.alive[p] = 1;
    return team_sync<TEAM>(tm, err);
}

// Marks the entries j != i of row i with s + y[j] tight against D[i][j] in
// the row's bitmask words (bit j % 32 of word j / 32); returns whether any.
// Lane l holds 4 consecutive entries of each 128-entry block, so the bits of
// a 32-entry word come from 8 lanes and are combined with shuffles.
template <typename T, bool TEAM>
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
            if (j != i && M::slack_tight(M::slack(s + tld<TEAM>(sy + j), dv[e]))) m |= 1u << e;
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
template <typename T, bool TEAM>
__device__ __noinline__ bool b_decrease(const BG<T> &g, const Team &tm, int32_t *err, int u, int v, T w, int span, T *sx,
                                        T *sy) {
    using M = MinPlus<T>;
    const int wid = tm.gw(), nw = tm.nw();
    for (int t = tm.gt(); t < span; t += tm.nt()) {
        sx[t] = __ldcg(&g.dt(u, t));   // D[t][u]
        sy[t] = __ldcg(&g.d(v, t));    // D[v][t]
    }
    if (!team_sync<TEAM>(tm, err)) return false;
    if (tm.leader()) g.w(u, v) = w;
    for (int i = wid; i < span; i += nw) {
        const T xi = tld<TEAM>(sx + i);
        if (!M::finite(xi) || !(M::add(xi, w) < __ldcg(&g.dt(v, i)))) continue;   // row filter
        const T s = xi + w;
        b_row(reinterpret_cast<const typename M::V4 *>(g.D + (int64_t)i * g.ld), span / 4,
              [&](int c4, const typename M::V4 &dv4) {
                  const T dv[4] = {dv4.x, dv4.y, dv4.z, dv4.w};
#pragma unroll
                  for (int e = 0; e < 4; ++e) {
                      const T y = tld<TEAM>(sy + 4 * c4 + e);
                      if (M::finite(y) && s + y < dv[e]) g.set(i, 4 * c4 + e, s + y);
                  }
              });
    }
    return team_sync<TEAM>(tm, err);
}

// Edge increase (u, v): w_old -> w (w may be missing: a deletion).  Returns
// false on the pass cap or a team wait that gave up.
template <typename T, bool TEAM>
__device__ __noinline__ bool b_increase(const BG<T> &g, const Team &tm, int32_t *err, int u, int v, T w_old, T w,
                                        int span, uint32_t *mask, int words, T *sx, T *sy, int32_t *rows,
                                        int32_t *nrows_p, int32_t *changed_p) {
    using M = MinPlus<T>;
    const int lane = threadIdx.x & 31, wid = tm.gw(), nw = tm.nw();
    const bool tight_edge = M::tight(w_old, __ldcg(&g.d(u, v)));
    if (!team_sync<TEAM>(tm, err)) return false;   // every CTA has read D[u][v] before it changes
    if (tm.leader()) g.w(u, v) = w;
    if (!tight_edge) return team_sync<TEAM>(tm, err);
    for (int t = tm.gt(); t < span; t += tm.nt()) {
        sx[t] = __ldcg(&g.dt(u, t));   // D[t][u]
        sy[t] = M::leg(__ldcg(&g.d(v, t)));
    }
    if (!b_clear_mask<TEAM>(tm, err, mask, words, span, nrows_p)) return false;
    // pairs whose distance is a path through the old edge (Corollary 3 for an edge)
    for (int i = wid; i < span; i += nw) {
        const T xi = tld<TEAM>(sx + i);
        if (!M::finite(xi) || !__ldcg(g.alive + i)) continue;
        const T s = M::add(xi, w_old);
        if (!M::tight(s, __ldcg(&g.dt(v, i)))) continue;
        const bool any = b_detect_row<T, TEAM>(g, i, s, sy, span, mask + (int64_t)i * words);
        if (lane == 0 && any) rows[atomicAdd(nrows_p, 1)] = i;
    }
    if (!team_sync<TEAM>(tm, err)) return false;
    // starting upper bounds: the direct edge, or the path through the edge at its new weight
    const int nrows = tld<TEAM>(nrows_p);
    for (int r = wid; r < nrows; r += nw) {
        const int i = tld<TEAM>(rows + r);
        for (int wd = 0; wd < words; ++wd) {
            const uint32_t m = __ldcg(mask + (int64_t)i * words + wd);
            const int j = wd * 32 + lane;
            if ((m >> lane) & 1u) {
                const T via = M::add(M::add(tld<TEAM>(sx + i), w), M::mn(tld<TEAM>(sy + j), M::inf()));
                g.set(i, j, M::mn(__ldcg(&g.w(i, j)), via));
            }
        }
    }
    if (!team_sync<TEAM>(tm, err)) return false;
    return b_relax<T, TEAM>(g, tm, err, mask, words, span, rows, nrows, changed_p);
}

// Removal of node k.  Returns false on the pass cap or a team wait that gave up.
template <typename T, bool TEAM>
__device__ __noinline__ bool b_remove(const BG<T> &g, const Team &tm, int32_t *err, int k, int span, uint32_t *mask,
                                      int words, T *sx, T *sy, int32_t *rows, int32_t *nrows_p, int32_t *changed_p) {
    using M = MinPlus<T>;
    const int lane = threadIdx.x & 31, wid = tm.gw(), nw = tm.nw();
    for (int t = tm.gt(); t < span; t += tm.nt()) {
        sx[t] = __ldcg(&g.dt(k, t));                         // D[t][k]
        sy[t] = t == k ? unreachable_leg<T>() : M::leg(__ldcg(&g.d(k, t)));   // D[k][t]
    }
    if (!b_clear_mask<TEAM>(tm, err, mask, words, span, nrows_p)) return false;
    // need_update_list: D[i][k] + D[k][j] == D[i][j], i != j, both != k
    for (int i = wid; i < span; i += nw) {
        const T xi = tld<TEAM>(sx + i);
        if (i == k || !M::finite(xi) || !__ldcg(g.alive + i)) continue;
        const bool any = b_detect_row<T, TEAM>(g, i, xi, sy, span, mask + (int64_t)i * words);
        if (lane == 0 && any) rows[atomicAdd(nrows_p, 1)] = i;
    }
    if (!team_sync<TEAM>(tm, err)) return false;
    // tombstone k (Section 3.2: its distances become infinite), then the
    // listed pairs restart from their direct edges
    const T inf = M::inf();
    for (int t = tm.gt(); t < span; t += tm.nt()) {
        g.set(k, t, inf);
        g.set(t, k, inf);
        g.w(k, t) = inf;
        g.w(t, k) = inf;
    }
    if (tm.leader()) g.alive[k] = 0;
    if (!team_sync<TEAM>(tm, err)) return false;
    const int nrows = tld<TEAM>(nrows_p);
    for (int r = wid; r < nrows; r += nw) {
        const int i = tld<TEAM>(rows + r);
        for (int wd = 0; wd < words; ++wd) {
            const uint32_t m = __ldcg(mask + (int64_t)i * words + wd);
            const int j = wd * 32 + lane;
            if ((m >> lane) & 1u) g.set(i, j, __ldcg(&g.w(i, j)));
        }
    }
    if (!team_sync<TEAM>(tm, err)) return false;
    return b_relax<T, TEAM>(g, tm, err, mask, words, span, rows, nrows, changed_p);
}

// Widths (threads per CTA) the executor's autotuner chooses from.
constexpr int BATCH_WIDTHS[3] = {128, 256, 512};

// All updates of graph gi by a team (or one CTA); then the graph's status and
// completion flag.  A pass cap reached is recorded and the next update goes
// on; a team wait that gave up ends the graph (the team is out of step).
template <typename T, bool TEAM>
__device__ void b_graph(BatchHeader *hdr, int gi, const Team &tm, T *s0, T *s1, T *s2, T *s3, int32_t *srows,
                        int32_t *nrows_p, int32_t *changed_p) {
    BatchGraph &bg = hdr->graphs[gi];
    BG<T> g{reinterpret_cast<T *>(bg.D), reinterpret_cast<T *>(bg.DT), reinterpret_cast<T *>(bg.W), bg.alive, bg.ld};
    const T *vecs = reinterpret_cast<const T *>(hdr->vecs);
    int32_t *err = &bg.status;
    for (int q = bg.first; q < bg.first + bg.count; ++q) {
        const BatchOp op = hdr->ops[q];
        bool ok;
        if (op.op == BOP_ADD) {
            ok = b_add<T, TEAM>(g, tm, err, op.a, op.span, vecs + op.vec, vecs + op.vec + op.span, s0, s1, s2, s3);
        } else if (op.op == BOP_DECREASE) {
            ok = b_decrease<T, TEAM>(g, tm, err, op.a, op.b, bits_as<T>(op.w_bits), op.span, s0, s1);
        } else if (op.op == BOP_INCREASE) {
            ok = b_increase<T, TEAM>(g, tm, err, op.a, op.b, bits_as<T>(op.w_old_bits), bits_as<T>(op.w_bits),
                                     op.span, bg.mask, bg.mask_words, s0, s1, srows, nrows_p, changed_p);
        } else {
            ok = b_remove<T, TEAM>(g, tm, err, op.a, op.span, bg.mask, bg.mask_words, s0, s1, srows, nrows_p,
                                   changed_p);
        }
        if (!ok) {
            if (__ldcg(err) & (int32_t)ERR_TIMEOUT) break;
            if (tm.leader()) atomicOr(err, (int32_t)ERR_PASSES);
        }
    }
    const bool synced = team_sync<TEAM>(tm, err);   // every CTA of the team is done with the graph
    if (tm.leader()) {
        const int32_t st = __ldcg(err) | (synced ? 0 : (int32_t)ERR_TIMEOUT);
        bg.status = st;
        if (hdr->done) {
            __threadfence_system();   // the graph's results are written before its flag
            hdr->done[gi] = 1 + st;
        }
    }
    __syncthreads();
}

template <typename T, int NT> __global__ void __launch_bounds__(NT, 768 / NT) k_batch(BatchHeader *hdr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int32_t gi_s, nrows_s, changed_s;
    const int G = hdr->team_size;
    const int max_span = hdr->max_span;
    // large graphs: team t = blockIdx / G takes order[t], order[t + n_teams], ...
    if (G > 1 && (int)blockIdx.x < hdr->n_teams * G) {
        const int t = (int)blockIdx.x / G;
        unsigned char *base = reinterpret_cast<unsigned char *>(hdr->team_scratch) + (int64_t)t * hdr->team_stride;
        T *t0 = reinterpret_cast<T *>(base);
        int32_t *trows = reinterpret_cast<int32_t *>(t0 + 4 * (int64_t)max_span);
        int32_t *ints = trows + max_span;
        const Team tm{(int)blockIdx.x % G, G, ints};
        for (int k = t; k < hdr->n_team; k += hdr->n_teams)
            b_graph<T, true>(hdr, hdr->order[k], tm, t0, t0 + max_span, t0 + 2 * max_span, t0 + 3 * max_span, trows,
                             ints + 0, ints + 1);
    }
    // every other graph: one CTA each, from the queue
    T *s0 = reinterpret_cast<T *>(smem_raw);
    int32_t *srows = reinterpret_cast<int32_t *>(s0 + 4 * (int64_t)max_span);
    const Team solo{0, 1, nullptr};
    const int n_solo = hdr->n_graphs - hdr->n_team;
    while (true) {
        if (threadIdx.x == 0) gi_s = atomicAdd(&hdr->queue, 1);
        __syncthreads();
        const int q = gi_s;
        __syncthreads();
        if (q >= n_solo) break;
        b_graph<T, false>(hdr, hdr->order[hdr->n_team + q], solo, s0, s0 + max_span, s0 + 2 * max_span,
                          s0 + 3 * max_span, srows, &nrows_s, &changed_s);
    }
}

}  // namespace apsp
