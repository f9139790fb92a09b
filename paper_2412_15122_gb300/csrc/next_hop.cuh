// Next hops, the optional next-hop output of the hot-path plan, derived from
// the resident D and W when asked for instead of being carried through every
// update (which would double the bytes of every sweep).
//
// For a live row i and every j:
//     NH[i][j] = the lowest live t != i with W[i][t] + D[t][j] == D[i][j]
// (fp32: within the tightness slack), i for j == i, -1 when j is dead or
// unreachable.  Only an edge that is itself a shortest path can start such a
// walk: W[i][t] + D[t][j] == D[i][j] <= D[i][t] + D[t][j] forces
// W[i][t] == D[i][t].  So a CTA first lists row i's tight out-edges in slot
// order (ballots and a CTA prefix sum), then each thread takes columns j and
// tries them in that order, reading D[t][j] coalesced across the threads.
#pragma once

#include "kernels.cuh"

namespace apsp {

template <typename T>
__global__ void __launch_bounds__(256) k_next_hop(Dev<T> d, const int32_t *rows, int nrows, int32_t *out,
                                                  int64_t ld_out) {
    using M = MinPlus<T>;
    extern __shared__ int32_t nh_tl[];   // the row's tight out-edges, span entries at most
    __shared__ int s_cnt;
    __shared__ int w_cnt[8];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int i = rows[r];
        const T *Di = d.D + (int64_t)i * d.ld;
        const T *Wi = d.W + (int64_t)i * d.ld;
        if (tid == 0) s_cnt = 0;
        __syncthreads();
        for (int t0 = 0; t0 < d.span; t0 += 256) {
            const int t = t0 + tid;
            const bool ok = t < d.span && t != i && d.alive[t] && M::finite(Wi[t]) && M::tight(Wi[t], Di[t]);
            const unsigned b = __ballot_sync(0xffffffffu, ok);
            if (lane == 0) w_cnt[w] = __popc(b);
            __syncthreads();
            int off = s_cnt;
            for (int k = 0; k < w; ++k) off += w_cnt[k];
            if (ok) nh_tl[off + __popc(b & ((1u << lane) - 1u))] = t;
            __syncthreads();
            if (tid == 0) {
                int tot = 0;
                for (int k = 0; k < 8; ++k) tot += w_cnt[k];
                s_cnt += tot;
            }
            __syncthreads();
        }
        const int nt = s_cnt;
        int32_t *o = out + (int64_t)r * ld_out;
        for (int j = tid; j < d.span; j += blockDim.x) {
            int nh = -1;
            if (j == i) {
                nh = i;
            } else if (d.alive[j]) {
                const T dij = Di[j];
                if (M::finite(dij)) {
                    for (int q = 0; q < nt; ++q) {
                        const int t = nh_tl[q];
                        const T dtj = __ldcg(d.D + (int64_t)t * d.ld + j);
                        if (M::finite(dtj) && M::tight(M::add(__ldg(Wi + t), dtj), dij)) {
                            nh = t;
                            break;
                        }
                    }
                }
            }
            o[j] = nh;
        }
        __syncthreads();   // the list is rebuilt for the next row
    }
}

}  // namespace apsp
