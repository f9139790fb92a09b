// First pass of the restricted re-relaxation, as its own kernel.
//
// For every listed pair (i, j) of the current removal / edge increase:
//     pmin[pair] = min over all x of D[i][x] + D[x][j]
// with the starting values (D is only read; the later passes run in
// k_repair_main).  One warp per unit = (row i and up to P1_PAIRS of its
// listed columns j, from the list detection writes; window of PASS1_COLS
// values of x).  Units of 16 pairs rather than the later passes' 32 halve
// the longest unit, which ends the pass on lists with a few long rows
// (measured: the 10th-percentile benchmark removal's pass 47 -> 31 us),
// units ordered window-major so that all warps sweep the same window at a
// time and the rows and columns it touches stay in L2 (about 35 MB at
// n = 8192).  The row's slice of the window is staged in the warp's shared
// buffer with cp.async; per pair the whole column slice DT[j][x0 ..] is
// loaded into registers (8 vectors a lane), two pairs at a time so both
// slices are in flight before either is used, reduced over the warp and
// kept by lane t for pair t; one atomic min per pair and unit stores it.
//
// A plain (not cooperative) launch: no grid-wide wait, so its occupancy is
// its own.  Measured on GB300 against a variant that streamed the column
// slices through a five-stage shared-memory ring filled by cp.async.bulk:
// the ring's shared memory left room for 8 warps per SM, too few to issue
// the add-min work and the reductions, and the pass took 285 us per removal
// of the n = 8192 benchmark against 158 us for this register version.
#pragma once

#include "kernels.cuh"

namespace apsp {

template <typename T>
__device__ __forceinline__ void k_repair_p1_body(Dev<T> d, RepairCfg cfg) {
    using M = MinPlus<T>;
    using V4 = typename M::V4;
    constexpr int CW = PASS1_COLS / 128;   // 16-byte vectors per lane per window
    __shared__ V4 rowbuf[8][PASS1_COLS / 4];
    Ctl *ctl = d.ctl;
    float cost, pw, pc;
    int n_items;
    if (repair_decide(ctl, cfg, &cost, &pw, &pc, &n_items) != 0) return;   // not warm: nothing to do

    const int lane = threadIdx.x & 31;
    const int span = d.span;
    const int64_t ld = d.ld;
    const T *cols = d.DT ? d.DT : d.D;   // row j of `cols` is column j of D
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->t_start = globaltimer_ns();
    const int wq = (int)((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % QUEUES) * 32;
    V4 *rb = rowbuf[threadIdx.x >> 5];
    const int nwin = (span + PASS1_COLS - 1) / PASS1_COLS;
    const int nh = *(volatile const int32_t *)&ctl->p1_alloc;   // units of up to P1_PAIRS pairs
    const int n1 = nh * nwin;   // units < 2^20 and windows <= 18 at the largest capacity
    int t = 0;
    if (lane == 0) t = atomicAdd(&ctl->q1[wq], 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    while (true) {
        const int u = (wq >> 5) + QUEUES * t;
        if (u >= n1 || u < 0) break;
        const int g = u / nh, h = u - g * nh;
        if (lane == 0) t = atomicAdd(&ctl->q1[wq], 1);   // next unit, in flight meanwhile
        const int4 item = __ldcg(d.p1u + h);   // (row, first pair, pairs, 0)
        const int cnt = item.z;
        const int jl = lane < cnt ? __ldcg(d.pairs + item.y + lane) : 0;
        const int x0 = g * PASS1_COLS;
        const int nv = (min(span, x0 + PASS1_COLS) - x0) / 4;
        const V4 *r4 = reinterpret_cast<const V4 *>(d.D + (int64_t)item.x * ld + x0);
        __syncwarp();   // the previous unit's reads of the buffer are done
#pragma unroll
        for (int k = 0; k < CW; ++k)
            if (lane + 32 * k < nv) cp_async16(rb + lane + 32 * k, r4 + lane + 32 * k);
        T pacc = M::inf();
        for (int q = 0; q < cnt; q += 2) {
            const bool two = q + 1 < cnt;
            const int ja = __shfl_sync(0xffffffffu, jl, q);
            const int jb = __shfl_sync(0xffffffffu, jl, two ? q + 1 : q);
            const V4 *ca = reinterpret_cast<const V4 *>(cols + (int64_t)ja * ld + x0);
            const V4 *cb = reinterpret_cast<const V4 *>(cols + (int64_t)jb * ld + x0);
            V4 a[CW], b[CW];
#pragma unroll
            for (int k = 0; k < CW; ++k)
                if (lane + 32 * k < nv) {
                    a[k] = __ldcg(ca + lane + 32 * k);
                    if (two) b[k] = __ldcg(cb + lane + 32 * k);
                }
            cp_async_wait_all();   // the row slice (in flight with the first columns)
            __syncwarp();
            // two independent minima per pair halve the add-min chains
            T a0 = M::inf(), a1 = M::inf(), b0 = M::inf(), b1 = M::inf();
#pragma unroll
            for (int k = 0; k < CW; ++k) {
                if (lane + 32 * k < nv) {
                    const V4 r = rb[lane + 32 * k];
                    a0 = M::add_min(r.x, a[k].x, a0);
                    a1 = M::add_min(r.y, a[k].y, a1);
                    a0 = M::add_min(r.z, a[k].z, a0);
                    a1 = M::add_min(r.w, a[k].w, a1);
                    if (two) {
                        b0 = M::add_min(r.x, b[k].x, b0);
                        b1 = M::add_min(r.y, b[k].y, b1);
                        b0 = M::add_min(r.z, b[k].z, b0);
                        b1 = M::add_min(r.w, b[k].w, b1);
                    }
                }
            }
            T acc = M::mn(a0, a1), acc2 = M::mn(b0, b1);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc = M::mn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
                acc2 = M::mn(acc2, __shfl_xor_sync(0xffffffffu, acc2, o));
            }
            if (lane == q) pacc = acc;
            if (two && lane == q + 1) pacc = acc2;
        }
        if (lane < cnt) atomicMin(d.pmin + item.y + lane, M::key(pacc));
        t = __shfl_sync(0xffffffffu, t, 0);
    }
    // the last CTA to finish stamps the end of the pass
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&ctl->p1_done, 1) == (int)gridDim.x - 1) ctl->t_pass1 = globaltimer_ns();
    }
}

template <typename T>
__global__ void __launch_bounds__(256, 2) k_repair_p1(Dev<T> d, RepairCfg cfg) {
    pdl_enter();
    k_repair_p1_body<T>(d, cfg);
}

}  // namespace apsp
