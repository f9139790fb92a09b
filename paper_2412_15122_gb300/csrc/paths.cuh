// Warm-start path queries (Section 4): Algorithm 7 and the trees behind
// Algorithm 8, on the device.
//
// Three tiers, by the number K of candidates a query turns out to have:
//   warp tier   (K <= PW_K, nearly every query): one warp per query, no
//               CTA-wide barrier anywhere, per-warp arrays in shared memory;
//   block tier  (K <= PQ_KS): one CTA per query, as below;
//   wide tier   (any K): PQ_WIDE_GRID CTAs, arrays in global scratch.
// A tier that meets a larger K marks the query deferred and the next tier
// (a later launch) redoes it.  Batches smaller than the SM count start at the
// block tier, whose 512 threads read a query's rows with more loads in flight
// than one warp.  The block tier, per query:
//   1. candidate scan: the live nodes t other than i and j that are not
//      excluded by the test SPD(i, j) < SPD(i, t) + SPD(t, j) (Algorithm 7;
//      Theorem al_correct: every shortest i -> j path uses only them).  Row i
//      of D and row j of D^T (column j of D) are read with 16-byte vectors,
//      each thread owning a contiguous run of slots, so a block-wide
//      exclusive scan gives the candidates in increasing slot order:
//      cand = [i, t..., j], K entries.
//   2. Dijkstra on the small graph (adjacency among the candidates: gathered
//      into shared memory by the whole CTA when K <= PQ_SK, else read from W
//      as it goes): one warp, lanes owning candidates a = lane (mod 32);
//      the next node is the unvisited one of least distance, the lowest small
//      index on a tie, and a predecessor changes only on a strict
//      improvement.  Forward from small node 0 (stops when K - 1 settles for
//      a single path); for Algorithm 8 a second warp runs it backward from
//      K - 1 on the reversed small graph.
//   3. output: the path i -> j (Algorithm 7's translation back to slot ids),
//      or the candidate list and both predecessor arrays (Algorithm 8's
//      joins are assembled by the host library).
// Small graphs of up to PQ_KS candidates live in shared memory.  A query with
// more candidates (only possible with many equal-length routes, e.g. zero
// weights) is marked deferred and redone by a second launch of PQ_WIDE_GRID
// CTAs whose per-CTA arrays sit in a library-owned global scratch area.
//
// The end of the file holds Algorithm 12's test before a repair
// (alg12_keep, k_det_alg12), which reuses the warp tier's scan and small
// Dijkstra with the removed node left out.
#pragma once

#include "kernels.cuh"

namespace apsp {

constexpr int PQ_THREADS = 512;
constexpr int PQ_KS = 1024;
constexpr int PQ_SK = 64;           // small graphs of up to PQ_SK nodes have their matrix staged in shared memory
constexpr int PQ_WIDE_GRID = 4;
constexpr int PW_K = 128;           // warp tier: candidates per query
constexpr int PW_SK = 32;           // warp tier: small matrix staged when K <= PW_SK
constexpr int PW_WARPS = 8;         // warp tier: warps per CTA
constexpr int32_t PQ_BROKEN = -1;   // the small graph does not reach j: D is not the APSP matrix of W
constexpr int32_t PQ_DEFERRED = -2; // for the block tier
constexpr int32_t PQ_DEFERRED_WIDE = -3;   // for the wide tier

struct PathQuery {
    const int32_t *uv;     // count (i, j) pairs, device
    int count;
    int32_t *out;          // count rows of `row` int32, device
    int64_t row;
    int stride;            // mode 0: path entries kept per query (row = 1 + stride)
    int mode;              // 0: Algorithm 7 path; 1: Algorithm 8 trees (row = 1 + 3 * wide_slots)
    int32_t *wide;         // PQ_WIDE_GRID * wide_stride int32
    int64_t wide_stride;
    int wide_slots;        // candidates a wide CTA can hold (>= span + 2)
    int all;               // block tier: answer every query (small batches start there), not only deferred ones
};

// Per-CTA arrays of one query.
template <typename T> struct PqArrays {
    int32_t *cand;
    T *fdist, *bdist;
    int32_t *fpred, *bpred;
    uint8_t *fdone, *bdone;
};

template <typename T> __device__ __forceinline__ uint32_t pq_okey(T v) { return (uint32_t)MinPlus<T>::key(v); }

// Candidate test of Algorithm 7 for one slot: kept unless D[i][j] < D[i][t] +
// D[t][j].  Float: within the same relative slack as the tightness test (an
// extra candidate only enlarges the small graph).
template <typename T> __device__ __forceinline__ bool pq_keep(T a, T b, T dij) {
    return MinPlus<T>::tight(a + b, dij);
}

// Step 1.  Writes the interior candidates to cand[1 ..] in slot order (only
// those that fit in kcap - 2 entries) and returns their number.  All threads.
template <typename T>
__device__ int pq_scan(const Dev<T> &d, int i, int j, T dij, int32_t *cand, int kcap, int *wtot) {
    using V4 = typename MinPlus<T>::V4;
    const int nv = d.span >> 2;
    const int per = (nv + (int)blockDim.x - 1) / (int)blockDim.x;   // <= 16: span <= 32768
    const int v0 = threadIdx.x * per;
    const int v1 = min(v0 + per, nv);
    const V4 *ri = reinterpret_cast<const V4 *>(d.D + (int64_t)i * d.ld);
    const V4 *rj = reinterpret_cast<const V4 *>((d.DT ? d.DT : d.D) + (int64_t)j * d.ld);
    const int4 *al = reinterpret_cast<const int4 *>(d.alive);
    unsigned long long mask = 0ull;
#pragma unroll 4
    for (int v = v0; v < v1; ++v) {
        const V4 a = ri[v], b = rj[v];
        const int4 l = al[v];
        const int t = v << 2;
        const unsigned bit = (unsigned)(v - v0) << 2;
        if (l.x && t != i && t != j && pq_keep<T>(a.x, b.x, dij)) mask |= 1ull << bit;
        if (l.y && t + 1 != i && t + 1 != j && pq_keep<T>(a.y, b.y, dij)) mask |= 1ull << (bit + 1);
        if (l.z && t + 2 != i && t + 2 != j && pq_keep<T>(a.z, b.z, dij)) mask |= 1ull << (bit + 2);
        if (l.w && t + 3 != i && t + 3 != j && pq_keep<T>(a.w, b.w, dij)) mask |= 1ull << (bit + 3);
    }
    const int mine = __popcll(mask);
    int wsum;
    const int wex = warp_exclusive_scan(mine, &wsum);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) wtot[warp] = wsum;
    __syncthreads();
    if (warp == 0) {
        const int nw = (int)blockDim.x >> 5;
        int x = lane < nw ? wtot[lane] : 0, tot;
        const int ex = warp_exclusive_scan(x, &tot);
        __syncwarp();
        if (lane < nw) wtot[lane] = ex;
        if (lane == 0) wtot[32] = tot;
    }
    __syncthreads();
    int pos = 1 + wtot[warp] + wex;
    const int total = wtot[32];
    while (mask) {
        const int b = __ffsll((long long)mask) - 1;
        mask &= mask - 1;
        if (pos < kcap - 1) cand[pos] = (v0 << 2) + b;
        ++pos;
    }
    return total;
}

// Step 2, one warp.  Dijkstra over the K candidates from small node `src`;
// `reverse` relaxes a -> b with the weight of edge cand[b] -> cand[a].
template <typename T>
__device__ void pq_dijkstra(const Dev<T> &d, const int32_t *cand, int K, int src, bool reverse, bool stop_at_last,
                            const T *small, T *dist, int32_t *pred, uint8_t *done) {
    using M = MinPlus<T>;
    const int lane = threadIdx.x & 31;
    for (int a = lane; a < K; a += 32) {
        dist[a] = a == src ? (T)0 : M::inf();
        pred[a] = -1;
        done[a] = 0;
    }
    __syncwarp();
    for (int it = 0; it < K; ++it) {
        unsigned long long best = ~0ull;
        for (int a = lane; a < K; a += 32)
            if (!done[a]) {
                const unsigned long long key = ((unsigned long long)pq_okey<T>(dist[a]) << 32) | (unsigned)a;
                best = key < best ? key : best;
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
            best = y < best ? y : best;
        }
        if (best == ~0ull) break;
        const int a = (int)(best & 0xffffffffu);
        const T da = M::unkey((int32_t)(best >> 32));
        if (!M::finite(da)) break;
        if ((a & 31) == lane) done[a] = 1;
        if (stop_at_last && a == K - 1) break;
        const int ca = cand[a];
        for (int b = lane; b < K; b += 32) {
            if (done[b]) continue;
            T w;
            if (small) {
                w = reverse ? small[b * K + a] : small[a * K + b];
            } else {
                const int cb = cand[b];
                w = reverse ? d.W[(int64_t)cb * d.ld + ca] : d.W[(int64_t)ca * d.ld + cb];
            }
            if (!M::finite(w)) continue;
            const T nd = M::add(da, w);
            if (nd < dist[b]) {
                dist[b] = nd;
                pred[b] = a;
            }
        }
        __syncwarp();
    }
}

template <typename T, bool WIDE>
__global__ void __launch_bounds__(PQ_THREADS) k_path_query(Dev<T> d, PathQuery q) {
    using M = MinPlus<T>;
    extern __shared__ __align__(16) unsigned char pq_smem[];
    __shared__ int wtot[33];
    __shared__ int32_t o0_s;
    PqArrays<T> A;
    int kcap;
    if (!WIDE) {
        kcap = PQ_KS;
        A.cand = reinterpret_cast<int32_t *>(pq_smem);
        A.fdist = reinterpret_cast<T *>(A.cand + PQ_KS);
        A.bdist = A.fdist + PQ_KS;
        A.fpred = reinterpret_cast<int32_t *>(A.bdist + PQ_KS);
        A.bpred = A.fpred + PQ_KS;
        A.fdone = reinterpret_cast<uint8_t *>(A.bpred + PQ_KS);
        A.bdone = A.fdone + PQ_KS;
    } else {
        kcap = q.wide_slots;
        int32_t *base = q.wide + (int64_t)blockIdx.x * q.wide_stride;
        A.cand = base;
        A.fdist = reinterpret_cast<T *>(base + kcap);
        A.bdist = A.fdist + kcap;
        A.fpred = reinterpret_cast<int32_t *>(A.bdist + kcap);
        A.bpred = A.fpred + kcap;
        A.fdone = reinterpret_cast<uint8_t *>(A.bpred + kcap);
        A.bdone = A.fdone + kcap;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int qi = blockIdx.x; qi < q.count; qi += gridDim.x) {
        int32_t *o = q.out + (int64_t)qi * q.row;
        {   // only the queries the previous tier deferred
            if (threadIdx.x == 0) o0_s = o[0];
            __syncthreads();
            const int32_t o0 = o0_s;
            __syncthreads();
            if (!(WIDE ? o0 == PQ_DEFERRED_WIDE : (q.all || o0 == PQ_DEFERRED))) continue;
        }
        const int i = q.uv[2 * qi], j = q.uv[2 * qi + 1];
        if (i == j) {   // Algorithm 7: the path of a node to itself is [i]
            if (threadIdx.x == 0) {
                o[0] = 1;
                if (q.mode == 0) {
                    if (q.stride > 0) o[1] = i;
                } else {
                    o[1] = i;
                    o[2] = -1;
                    o[3] = -1;
                }
            }
            continue;
        }
        const T dij = d.D[(int64_t)i * d.ld + j];
        if (!M::finite(dij)) {   // unreachable: no path
            if (threadIdx.x == 0) o[0] = 0;
            continue;
        }
        const int K = pq_scan<T>(d, i, j, dij, A.cand, kcap, wtot) + 2;
        if (K > kcap) {
            if (threadIdx.x == 0) o[0] = WIDE ? PQ_BROKEN : PQ_DEFERRED_WIDE;
            __syncthreads();
            continue;
        }
        if (threadIdx.x == 0) {
            A.cand[0] = i;
            A.cand[K - 1] = j;
        }
        __syncthreads();
        // Algorithm 7's small_matrix: gathered at once by the whole CTA when
        // it fits, else read from W by the Dijkstra warp as it goes
        const T *small = nullptr;
        if (!WIDE && K <= PQ_SK) {
            T *sm = reinterpret_cast<T *>(A.bdone + PQ_KS);
            for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
                const int a = e / K, b = e - a * K;
                sm[e] = d.W[(int64_t)A.cand[a] * d.ld + A.cand[b]];
            }
            __syncthreads();
            small = sm;
        }
        if (warp == 0) pq_dijkstra<T>(d, A.cand, K, 0, false, q.mode == 0, small, A.fdist, A.fpred, A.fdone);
        else if (warp == 1 && q.mode == 1)
            pq_dijkstra<T>(d, A.cand, K, K - 1, true, false, small, A.bdist, A.bpred, A.bdone);
        __syncthreads();
        if (q.mode == 0) {
            if (threadIdx.x == 0) {
                int L = 1, b = K - 1;
                while (b != 0 && L <= K) {
                    b = A.fpred[b];
                    if (b < 0) break;
                    ++L;
                }
                if (b != 0) {
                    o[0] = PQ_BROKEN;
                } else {
                    o[0] = L;
                    b = K - 1;
                    for (int p = L - 1; p >= 0; --p) {
                        if (p < q.stride) o[1 + p] = A.cand[b];
                        b = A.fpred[b];
                    }
                }
            }
        } else if (warp == 0) {
            for (int a = lane; a < K; a += 32) {
                o[1 + a] = A.cand[a];
                o[1 + K + a] = A.fpred[a];
                o[1 + 2 * K + a] = A.bpred[a];
            }
            if (lane == 0) o[0] = K;
        }
        __syncthreads();
    }
}

// Warp tier: one warp per query.
template <typename T> struct PwWarpSmem {
    int32_t cand[PW_K];
    T fdist[PW_K], bdist[PW_K];
    int32_t fpred[PW_K], bpred[PW_K];
    uint8_t fdone[PW_K], bdone[PW_K];
    T small[PW_SK * PW_SK];
};

template <typename T> __global__ void __launch_bounds__(PW_WARPS * 32) k_path_warp(Dev<T> d, PathQuery q) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    constexpr int B = 4;   // vectors of each row in flight per lane
    extern __shared__ __align__(16) unsigned char pw_smem[];
    PwWarpSmem<T> &S = reinterpret_cast<PwWarpSmem<T> *>(pw_smem)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * PW_WARPS;
    const int nv = d.span >> 2;
    for (int qi = blockIdx.x * PW_WARPS + (threadIdx.x >> 5); qi < q.count; qi += nwarps) {
        int32_t *o = q.out + (int64_t)qi * q.row;
        const int i = q.uv[2 * qi], j = q.uv[2 * qi + 1];
        if (i == j) {   // Algorithm 7: the path of a node to itself is [i]
            if (lane == 0) {
                o[0] = 1;
                if (q.mode == 0) {
                    if (q.stride > 0) o[1] = i;
                } else {
                    o[1] = i;
                    o[2] = -1;
                    o[3] = -1;
                }
            }
            continue;
        }
        const T dij = d.D[(int64_t)i * d.ld + j];
        if (!M::finite(dij)) {   // unreachable: no path
            if (lane == 0) o[0] = 0;
            continue;
        }
        // Step 1, candidate scan in slot order.  Dead and never-used slots hold
        // missing distances, so the test itself rejects them.
        const V4 *ri = reinterpret_cast<const V4 *>(d.D + (int64_t)i * d.ld);
        const V4 *rj = reinterpret_cast<const V4 *>((d.DT ? d.DT : d.D) + (int64_t)j * d.ld);
        int total = 0;
        for (int base = 0; base < nv && total <= PW_K - 2; base += 32 * B) {
            V4 a[B], c[B];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int v = base + 32 * b + lane;
                if (v < nv) {
                    a[b] = ri[v];
                    c[b] = rj[v];
                }
            }
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int v = base + 32 * b + lane;
                unsigned m4 = 0;
                if (v < nv) {
                    const int t = v << 2;
                    if (t != i && t != j && pq_keep<T>(a[b].x, c[b].x, dij)) m4 |= 1u;
                    if (t + 1 != i && t + 1 != j && pq_keep<T>(a[b].y, c[b].y, dij)) m4 |= 2u;
                    if (t + 2 != i && t + 2 != j && pq_keep<T>(a[b].z, c[b].z, dij)) m4 |= 4u;
                    if (t + 3 != i && t + 3 != j && pq_keep<T>(a[b].w, c[b].w, dij)) m4 |= 8u;
                }
                int wsum;
                int pos = 1 + total + warp_exclusive_scan(__popc(m4), &wsum);
                while (m4) {
                    const int e = __ffs(m4) - 1;
                    m4 &= m4 - 1;
                    if (pos < PW_K - 1) S.cand[pos] = (v << 2) + e;
                    ++pos;
                }
                total += wsum;
            }
        }
        const int K = total + 2;
        if (K > PW_K) {
            if (lane == 0) o[0] = PQ_DEFERRED;
            __syncwarp();
            continue;
        }
        if (lane == 0) {
            S.cand[0] = i;
            S.cand[K - 1] = j;
        }
        __syncwarp();
        // Algorithm 7's small_matrix, staged when it fits
        const T *small = nullptr;
        if (K <= PW_SK) {
            for (int e = lane; e < K * K; e += 32) {
                const int a = e / K, b = e - a * K;
                S.small[e] = d.W[(int64_t)S.cand[a] * d.ld + S.cand[b]];
            }
            __syncwarp();
            small = S.small;
        }
        // Step 2
        pq_dijkstra<T>(d, S.cand, K, 0, false, q.mode == 0, small, S.fdist, S.fpred, S.fdone);
        if (q.mode == 1) pq_dijkstra<T>(d, S.cand, K, K - 1, true, false, small, S.bdist, S.bpred, S.bdone);
        __syncwarp();
        // Step 3
        if (q.mode == 0) {
            if (lane == 0) {
                int L = 1, b = K - 1;
                while (b != 0 && L <= K) {
                    b = S.fpred[b];
                    if (b < 0) break;
                    ++L;
                }
                if (b != 0) {
                    o[0] = PQ_BROKEN;
                } else {
                    o[0] = L;
                    b = K - 1;
                    for (int p = L - 1; p >= 0; --p) {
                        if (p < q.stride) o[1 + p] = S.cand[b];
                        b = S.fpred[b];
                    }
                }
            }
        } else {
            for (int a = lane; a < K; a += 32) {
                o[1 + a] = S.cand[a];
                o[1 + K + a] = S.fpred[a];
                o[1 + 2 * K + a] = S.bpred[a];
            }
            if (lane == 0) o[0] = K;
        }
        __syncwarp();
    }
}

template <typename T> constexpr size_t pw_smem_bytes() { return PW_WARPS * sizeof(PwWarpSmem<T>); }

// ---------------------------------------------------------------------------
// Algorithm 12 before the repair (list mode APSP_LIST_ALGORITHM12).  For a
// pair (i, j) that Corollary 3 lists, with old distance dold: the candidates
// t (not i, j or the removed node `excl`) with D[i][t] + D[t][j] <= dold,
// Algorithm 7's small graph over them, and Dijkstra from i to j on it.  If it
// reaches j within dold, a shortest path avoids the removed node (for an
// increase, W already holds the edge's new, larger weight, so a path through
// the edge cannot be that short) and the pair keeps its distance: it leaves
// the list.  Returns true when the pair stays (also when the candidates
// exceed PW_K: staying is always safe).  One warp; D must still hold the old
// distances.
template <typename T>
__device__ bool alg12_keep(const Dev<T> &d, int i, int j, int excl, T dold, PwWarpSmem<T> &S) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    constexpr int B = 4;
    const int lane = threadIdx.x & 31;
    const int nv = d.span >> 2;
    const V4 *ri = reinterpret_cast<const V4 *>(d.D + (int64_t)i * d.ld);
    const V4 *rj = reinterpret_cast<const V4 *>((d.DT ? d.DT : d.D) + (int64_t)j * d.ld);
    int total = 0;
    for (int base = 0; base < nv && total <= PW_K - 2; base += 32 * B) {
        V4 a[B], c[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int v = base + 32 * b + lane;
            if (v < nv) {
                a[b] = __ldcg(ri + v);
                c[b] = __ldcg(rj + v);
            }
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int v = base + 32 * b + lane;
            unsigned m4 = 0;
            if (v < nv) {
                const int t = v << 2;
                if (t != i && t != j && t != excl && pq_keep<T>(a[b].x, c[b].x, dold)) m4 |= 1u;
                if (t + 1 != i && t + 1 != j && t + 1 != excl && pq_keep<T>(a[b].y, c[b].y, dold)) m4 |= 2u;
                if (t + 2 != i && t + 2 != j && t + 2 != excl && pq_keep<T>(a[b].z, c[b].z, dold)) m4 |= 4u;
                if (t + 3 != i && t + 3 != j && t + 3 != excl && pq_keep<T>(a[b].w, c[b].w, dold)) m4 |= 8u;
            }
            int wsum;
            int pos = 1 + total + warp_exclusive_scan(__popc(m4), &wsum);
            while (m4) {
                const int e = __ffs(m4) - 1;
                m4 &= m4 - 1;
                if (pos < PW_K - 1) S.cand[pos] = (v << 2) + e;
                ++pos;
            }
            total += wsum;
        }
    }
    const int K = total + 2;
    if (K > PW_K) return true;
    __syncwarp();
    if (lane == 0) {
        S.cand[0] = i;
        S.cand[K - 1] = j;
    }
    __syncwarp();
    const T *small = nullptr;
    if (K <= PW_SK) {
        for (int e = lane; e < K * K; e += 32) {
            const int a = e / K, b = e - a * K;
            S.small[e] = __ldcg(d.W + (int64_t)S.cand[a] * d.ld + S.cand[b]);
        }
        __syncwarp();
        small = S.small;
    }
    pq_dijkstra<T>(d, S.cand, K, 0, false, true, small, S.fdist, S.fpred, S.fdone);
    __syncwarp();
    const T dj = S.fdist[K - 1];
    __syncwarp();   // every lane has read it before the next pair reuses the arrays
    return !(dj <= dold);
}

// One warp per flagged (row, batch) of the detection scan, before the
// reservation: the exact mask, then Algorithm 12's test for each of its pairs
// (one after another, the whole warp on each).  The surviving mask is kept
// for k_det_write and the batch's count replaced, so the reservation and the
// writes see Algorithm 12's list.
template <typename T, bool TWO>
__global__ void __launch_bounds__(PW_WARPS * 32) k_det_alg12(Dev<T> d, int kind, int a, T w_old, uint32_t *umask) {
    pdl_enter();
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    extern __shared__ __align__(16) unsigned char pw_smem[];
    PwWarpSmem<T> &S = reinterpret_cast<PwWarpSmem<T> *>(pw_smem)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int n_units = *(volatile const int32_t *)&d.ctl->hit_units;
    const int nwarps = gridDim.x * PW_WARPS;
    const int nv4 = d.span / 4;
    for (int u = blockIdx.x * PW_WARPS + (threadIdx.x >> 5); u < n_units; u += nwarps) {
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
        const unsigned mask = det_exact_mask<T, TWO>(d, v, c0, s1, s2, use1, use2, i, a, kind);
        unsigned keep = mask, rem = mask;
        while (true) {
            const unsigned who = __ballot_sync(0xffffffffu, rem != 0u);
            if (!who) break;
            const int src = __ffs(who) - 1;
            int bit = 0;
            if (lane == src) {
                bit = __ffs(rem) - 1;
                rem &= rem - 1;
            }
            bit = __shfl_sync(0xffffffffu, bit, src);
            const int j = 4 * (c0 + (bit >> 2) * 32 + src) + (bit & 3);
            const T dold = __ldcg(d.D + (int64_t)i * d.ld + j);
            const bool stays = alg12_keep<T>(d, i, j, kind == 0 ? a : -1, dold, S);
            if (!stays && lane == src) keep &= ~(1u << bit);
        }
        umask[(int64_t)u * 32 + lane] = keep;
        const int c = warp_sum(__popc(keep));
        if (lane == 0) d.rowcnt[(int64_t)i * DET_MAXB + ue.y] = c;
    }
}

template <typename T> constexpr size_t pq_smem_bytes() {
    return (size_t)PQ_KS * (3 * sizeof(int32_t) + 2 * sizeof(T) + 2) + (size_t)PQ_SK * PQ_SK * sizeof(T);
}

}  // namespace apsp
