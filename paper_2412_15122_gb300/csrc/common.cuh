// Shared device-side definitions for the warm-start APSP kernels (sm_103a).
//
// Min-plus arithmetic for the two element types, the per-graph control
// block that kernels use to pass counts and decisions along a stream without
// host round trips, and a grid-wide barrier with a bounded wait for the
// cooperative repair kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "apsp.h"

namespace apsp {

constexpr int32_t INF_I32 = 0x3FFFFFFF;

// Relative slack of the fp32 tightness test.  A pair whose stored distance
// equals a path through the removed node / changed edge up to this relative
// rounding error is treated as affected: a missed pair would keep a stale,
// too-small distance, while an extra one only costs a recomputation.
//
// Every stored fp32 distance is a rounded sum over the h edges of one path,
// formed as a binary tree of additions of non-negative terms, so it lies
// within a relative (h - 1) * 2^-24 of that path's exact length, whatever the
// order in which updates built it.  If every stored path of the pair (i, j)
// runs through k, then D[i][k] + D[k][j] (one more rounding) exceeds the
// stored D[i][j] by at most about (2 (h - 1) + 1) * 2^-24 relative.  With
// h <= APSP_MAX_CAPACITY - 1 that is below 2^-8, so this slack catches every
// affected pair on every graph the library accepts; on lognormal complete
// graphs it lists about 4 % more pairs than an exact test.
constexpr float F32_TIGHT_REL = 1.0f / 256.0f;

// Re-relaxation in fp32 stops counting a pair as lowered when the new value
// is within this relative amount of the current one.  Sums of the same long
// path taken in different orders differ in their last bits, so an exact
// "lower" test can keep finding ulp-sized improvements for many passes; with
// this threshold every stored value stays within 2^-18 relative (3.8e-6) of
// the exact fixed point of the relaxation.
constexpr float F32_SETTLE_REL = 1.0f / 262144.0f;
static_assert(2 * APSP_MAX_CAPACITY + 1 < 65536, "2^-8 = 65536 * 2^-24 must cover 2 (h - 1) + 1 roundings");

template <typename T> struct MinPlus;

template <> struct MinPlus<int32_t> {
    using V4 = int4;
    __host__ __device__ static constexpr int32_t inf() { return INF_I32; }
    __device__ static bool finite(int32_t a) { return a < INF_I32; }
    // a, b <= INF: a + b <= 2*INF fits in int32; saturate to INF.
    __device__ static int32_t add(int32_t a, int32_t b) { return min(a + b, INF_I32); }
    // min(a + b, c) for a, b, c <= INF.  Stays <= c <= INF.
    __device__ static int32_t add_min(int32_t a, int32_t b, int32_t c) { return __viaddmin_s32(a, b, c); }
    __device__ static int32_t mn(int32_t a, int32_t b) { return min(a, b); }
    // re-relaxation: does candidate a lower the current value c (exact)
    __device__ static bool lowers(int32_t a, int32_t c) { return a < c; }
    // `via` is the length of a path through the removed node / changed edge,
    // `d` the stored distance (via >= d for an exact D): tight iff equal.
    __device__ static bool tight(int32_t via, int32_t d) { return via <= d; }
    // via - d for the batch screen (>= 0 for an exact APSP matrix; 0 = tight)
    __device__ static int32_t slack(int32_t via, int32_t d) { return via - d; }
    __device__ static bool slack_tight(int32_t s) { return s <= 0; }
    // batch screen: some entry is tight iff s <= max over entries of
    // screen_bound(d, y) (exact for int32: s + y <= d  <=>  s <= d - y)
    __device__ static int32_t screen_bound(int32_t d, int32_t y) { return d - y; }
    __device__ static int32_t screen_floor() { return -INF_I32 - 2; }
    // staged path-leg values: an unreachable leg becomes INF + 1 so that no
    // sum through it can equal a stored distance
    __device__ static int32_t leg(int32_t y) { return y >= INF_I32 ? INF_I32 + 1 : y; }
    // ordered bit pattern for atomicMin
    __device__ static int32_t key(int32_t a) { return a; }
    __device__ static int32_t unkey(int32_t a) { return a; }
};

template <> struct MinPlus<float> {
    using V4 = float4;
    __host__ __device__ static constexpr float inf() { return __builtin_huge_valf(); }
    __device__ static bool finite(float a) { return a < inf(); }
    __device__ static float add(float a, float b) { return a + b; }
    __device__ static float add_min(float a, float b, float c) { return fminf(a + b, c); }
    __device__ static float mn(float a, float b) { return fminf(a, b); }
    // re-relaxation: a lowers c only by more than F32_SETTLE_REL relative
    // (any finite a lowers a missing c)
    __device__ static bool lowers(float a, float c) { return c < inf() ? a < c - c * F32_SETTLE_REL : a < c; }
    __device__ static bool tight(float via, float d) { return via <= d + d * F32_TIGHT_REL; }
    // <= 0 when tight within the relative slack (NaN, from inf - inf, is not)
    __device__ static float slack(float via, float d) { return via - fmaf(d, F32_TIGHT_REL, d); }
    __device__ static bool slack_tight(float s) { return s <= 0.f; }
    // batch screen with twice the slack, so rounding in the rearranged test
    // can only let extra batches through to the exact test (inf - inf gives
    // NaN, which fmaxf ignores)
    __device__ static float screen_bound(float d, float y) { return fmaf(d, 2.f * F32_TIGHT_REL, d) - y; }
    __device__ static float screen_floor() { return -inf(); }
    __device__ static float leg(float y) { return y; }
    // non-negative floats (and +inf) order like their bit patterns as int32
    __device__ static int32_t key(float a) { return __float_as_int(a); }
    __device__ static float unkey(int32_t a) { return __int_as_float(a); }
};

// The (min, max) semiring of minimax (bottleneck) paths, the variant the
// paper's Discussion names: a path's value is its largest edge weight and the
// distance is the least such value.  "+" becomes max; max and min are exact in
// both element types, so the tightness test needs no slack.  Same interface
// as MinPlus for the kernels that are shared (the blocked Floyd-Warshall).
template <typename T> struct MinMax;

template <> struct MinMax<int32_t> {
    using V4 = int4;
    __host__ __device__ static constexpr int32_t inf() { return INF_I32; }
    __device__ static bool finite(int32_t a) { return a < INF_I32; }
    __device__ static int32_t add(int32_t a, int32_t b) { return max(a, b); }
    __device__ static int32_t add_min(int32_t a, int32_t b, int32_t c) { return min(max(a, b), c); }
    __device__ static int32_t mn(int32_t a, int32_t b) { return min(a, b); }
    __device__ static bool lowers(int32_t a, int32_t c) { return a < c; }
    __device__ static bool tight(int32_t via, int32_t d) { return via <= d; }
    __device__ static int32_t key(int32_t a) { return a; }
    __device__ static int32_t unkey(int32_t a) { return a; }
};

template <> struct MinMax<float> {
    using V4 = float4;
    __host__ __device__ static constexpr float inf() { return __builtin_huge_valf(); }
    __device__ static bool finite(float a) { return a < inf(); }
    __device__ static float add(float a, float b) { return fmaxf(a, b); }
    __device__ static float add_min(float a, float b, float c) { return fminf(fmaxf(a, b), c); }
    __device__ static float mn(float a, float b) { return fminf(a, b); }
    __device__ static bool lowers(float a, float c) { return a < c; }
    __device__ static bool tight(float via, float d) { return via <= d; }
    __device__ static int32_t key(float a) { return __float_as_int(a); }
    __device__ static float unkey(int32_t a) { return __int_as_float(a); }
};

template <typename V> __device__ __forceinline__ V ldcg4(const V *p) { return __ldcg(p); }

// Error bits, OR-ed into Ctl::err by kernels and turned into an
// apsp_status by the host at the next point where it waits for the stream.
enum : uint32_t {
    ERR_TIMEOUT = 1u,     // a bounded wait gave up
    ERR_NEGATIVE = 2u,    // negative weight in device-side input
    ERR_NAN = 4u,         // NaN in device-side input
    ERR_NOT_SYMMETRIC = 8u,
    ERR_PASSES = 16u      // re-relaxation did not settle within the pass cap
};

// Decision codes written by the repair kernel.
enum : int32_t { PATH_NONE = 0, PATH_SWEEP = 1, PATH_TRIVIAL = 2, PATH_WARM = 3, PATH_COLD = 4 };

constexpr int QUEUES = 16;

// Per-graph control block in device memory.  Cleared (except `err`) before
// each update; read back by the host only for statistics.
// Passes of the minimax re-relaxation the control block can record.
constexpr int MM_PASS_SLOTS = 64;

struct Ctl {
    // produced by the prepass / detection of the current update
    int32_t r_count;          // rows in the prepass row list
    int32_t n_rows;           // distinct affected rows (need_update_list items)
    int32_t n_items;          // work items (row, up to ITEM_PAIRS pairs)
    int32_t overflow;         // affected set did not fit the scratch
    unsigned long long n_pairs;
    int32_t n_live_before;    // N of Eq. (equ:cost_defi)
    int32_t trivial;          // 1 when the edge was not tight (increase)
    // produced by the repair kernel
    int32_t path;
    int32_t passes;
    int32_t cold_reason;
    float cost;
    float model_warm, model_cold;
    // grid barrier and pass bookkeeping of the repair kernel
    unsigned int bar_count;
    unsigned int bar_gen;
    int32_t changed[2];
    int32_t stop;
    int32_t unit_alloc;       // re-relaxation units reserved by detection
    // work queues of the re-relaxation: QUEUES counters, each on its own
    // 128-byte line (warp w takes units from queue w % QUEUES), for pass 1
    // and for passes >= 2 by parity
    int32_t q1[QUEUES * 32];
    int32_t qn[2][QUEUES * 32];
    int32_t qd[QUEUES * 32];  // detection's row queues
    int32_t hit_rows;         // rows flagged by the detection scan
    int32_t hit_units;        // (row, batch) units flagged by the detection scan
    unsigned long long alloc; // detection reservations: (pairs << 24) | work items
    unsigned long long pairs_evaluated;  // semi-naive pair evaluations (passes >= 2)
    unsigned long long t_start, t_pass1, t_end;  // device timestamps (ns) of the warm repair
    unsigned long long grown_pairs;  // listed pairs whose distance grew (Algorithm 12's list), when measured
    int32_t grown_rows;              // rows holding one of them
    int32_t p1_done;                 // CTAs of the first re-relaxation pass that finished
    int32_t p1_alloc;                // first-pass units reserved by detection
    // node insertion: argmin of each weight vector as the complement of
    // (ordered key << 32 | slot) (0: none), and the candidate rows / columns
    // of the reduction
    unsigned long long ins_amin_out, ins_amin_in;
    int32_t ins_nout, ins_nin;
    int32_t ins_narrow;              // 1: the reduction reads only the candidates
    int32_t mm_changed[MM_PASS_SLOTS];  // minimax re-relaxation: pass p lowered a pair
    uint32_t err;             // sticky until the host reads it
};

constexpr int ITEM_PAIRS = 32;          // affected pairs per re-relaxation work item
constexpr int P1_PAIRS = 16;            // affected pairs per first-pass work unit (shorter units end the pass sooner)
constexpr int PASS1_COLS = 1024;        // columns of x per pass-1 work unit (the swept window stays in L2)
constexpr int YSEG = 256;               // intermediates per work unit in passes >= 2
constexpr int MAX_PASSES = 48;          // path doubling needs <= log2(hops) + 1 passes
constexpr unsigned long long BARRIER_TIMEOUT_NS = 2000000000ull;  // 2 s

// 16-byte asynchronous global -> shared copy (no registers held while in
// flight) and the wait for all of this thread's copies.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Programmatic dependent launch.  The kernels of an update's launch
// sequence are launched with programmatic stream serialization, so a
// kernel's CTAs may be scheduled while its predecessor in the stream is
// still draining.  Every such kernel calls pdl_enter() first: it waits
// until the predecessor grid has completed and its writes are visible
// (griddepcontrol.wait; a no-op for an ordinary launch), then allows its
// own successor to begin launching.  Nothing is read or written before the
// wait, so the order of the updates' effects is that of the stream.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Grid-wide barrier for a cooperatively launched grid (all CTAs resident).
// The last CTA to arrive runs `leader()` before releasing the others, so the
// leader can publish decisions that every CTA reads after the barrier.  The
// wait is bounded: after BARRIER_TIMEOUT_NS the CTA records ERR_TIMEOUT and
// returns false; callers then leave the kernel.
template <typename Leader>
__device__ bool grid_barrier(Ctl *ctl, Leader leader) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *genp = &ctl->bar_gen;
        unsigned int gen = *genp;
        __threadfence();
        unsigned int arrived = atomicAdd(&ctl->bar_count, 1u);
        int ok = 1;
        if (arrived == gridDim.x - 1) {
            leader();
            ctl->bar_count = 0;
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            unsigned long long t0 = globaltimer_ns();
            unsigned int spins = 0;
            while (*genp == gen) {
                __nanosleep(64);
                if ((++spins & 1023u) == 0 && globaltimer_ns() - t0 > BARRIER_TIMEOUT_NS) {
                    atomicOr(&ctl->err, ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        if (ok && (*(volatile uint32_t *)&ctl->err & ERR_TIMEOUT)) ok = 0;
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

struct NoLeader { __device__ void operator()() const {} };

}  // namespace apsp
