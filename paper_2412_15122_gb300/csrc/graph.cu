// C ABI of the warm-start APSP library (declared in include/apsp.h).
//
// Owns the per-graph device state, the slot allocator, a host mirror of the
// weight matrix (so an edge update knows its old weight without a device
// round trip), pinned staging for host inputs, deferred device errors and
// launch instrumentation.  All compute runs in the kernels of kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <thread>
#include <limits>
#include <new>
#include <map>
#include <mutex>
#include <set>
#include <type_traits>
#include <string>
#include <vector>

#include "apsp.h"
#include "launch.h"

using apsp::Ctl;
using apsp::Dev;
using apsp::LaunchCtx;
using apsp::RepairCfg;

namespace {

apsp_alloc_fn g_alloc = nullptr;
apsp_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;

struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
};

}  // namespace

struct apsp_graph {
    int dtype = APSP_I32;
    uint32_t flags = 0;
    bool undirected = false;
    int n_live = 0, hwm = 0, cap = 0;
    int64_t ld = 0;
    size_t esz = 4;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 1;

    // device state
    void *W = nullptr, *D = nullptr, *DT = nullptr;
    int32_t *alive = nullptr;
    void *w_in = nullptr, *w_out = nullptr, *x = nullptr, *x2 = nullptr, *y = nullptr, *y2 = nullptr;
    int32_t *vin_k = nullptr, *vout_k = nullptr, *rlist = nullptr, *pairs = nullptr;
    int32_t *pmin = nullptr, *units = nullptr;
    int4 *hrows = nullptr;
    int4 *hunits = nullptr, *hralloc = nullptr;
    int32_t *rowcnt = nullptr;
    uint32_t *bmask = nullptr;   // detection: exact masks of flagged batches
    int32_t bmask_nb = 0;
    long long *hbase = nullptr;
    uint8_t *pstamp = nullptr, *rstamp = nullptr;
    int4 *items = nullptr;
    int32_t *icand = nullptr;   // node insertion: candidate rows / columns of the reduction
    int4 *p1u = nullptr;        // first-pass units
    int32_t p1u_cap = 0;
    Ctl *ctl = nullptr;
    // path queries (Section 4): per-call buffers, grown on demand
    void *pq_uv = nullptr, *pq_out = nullptr, *pq_wide = nullptr;
    int64_t pq_uv_bytes = 0, pq_out_bytes = 0, pq_wide_bytes = 0;
    // next hops: requested rows and their output, grown on demand
    void *nh_rows = nullptr, *nh_out = nullptr;
    int64_t nh_rows_bytes = 0, nh_out_bytes = 0;
    float *model = nullptr;
    int64_t pair_cap = 0;
    int32_t item_cap = 0;
    int32_t unit_cap = 0;
    apsp_alloc_fn alloc_fn = nullptr;
    apsp_free_fn free_fn = nullptr;
    void *alloc_ctx = nullptr;
    std::vector<std::pair<void *, size_t>> allocs;
    int64_t dev_bytes = 0;

    // host side
    std::vector<uint8_t> alive_h;
    // Mirror of W in two cap x cap copies, so that no update writes a column:
    // row i of Wh holds W[i][.] and row j of WhT holds W[.][j], each as set
    // by the latest add of that slot; an edge update writes both.  W[i][j] of
    // live i != j is in the copy of whichever of i and j was added later
    // (mirror_get); a removal writes nothing (its slot's next add rewrites
    // both rows).
    std::vector<char> Wh, WhT;
    std::vector<uint64_t> add_seq;   // per slot: order of its latest add (0: the initial graph)
    uint64_t seq = 0;
    static constexpr int RING = 8;   // host-input adds staged, device-input adds awaiting their weights
    void *pin = nullptr;             // pinned: RING x 2 * cap elements (add_node staging ring)
    cudaEvent_t pin_ev[RING] = {};
    bool pin_used[RING] = {};
    int pin_next = 0;
    void *pin_fetch = nullptr;       // mapped pinned: RING x 2 * cap elements (device-input adds' weights)
    void *pin_fetch_dev = nullptr;   // its device view (written by the prep kernel)
    cudaEvent_t fetch_ev[RING] = {};
    struct Fetch {
        int p;                       // slot added
        uint64_t seq;                // its add_seq at the add
        int ring;                    // pinned buffer / event
    };
    std::deque<Fetch> fetches;       // device-input adds not yet in the mirror, oldest first
    int fetch_next = 0;
    apsp::IncGraph incg;             // edge increase as one CUDA graph (built on first use)
    void *pin_small = nullptr;   // pinned scratch for queries / control block
    int64_t pin_small_bytes = 0;

    // dispatch
    int mode = APSP_DISPATCH_DELTA;
    float delta = 1.0f;
    bool has_model = false;
    int32_t *grown_flag = nullptr;   // set when Algorithm 12's list is measured (apsp_set_exact_list)
    int list_mode = APSP_LIST_COROLLARY3;   // apsp_set_list_mode
    uint32_t *umask = nullptr;              // list mode APSP_LIST_ALGORITHM12: per-unit surviving masks
    // minimax (bottleneck) distances: one bit per listed pair (i, j)
    bool minimax = false;
    uint32_t *mm_mask = nullptr;
    int32_t mm_words = 0;

    apsp_stats last{};
    LaunchCtx lc;

    // instrumentation
    int64_t launches = 0;
    bool prof = false;
    std::vector<ProfRec> pending;
    std::vector<cudaEvent_t> ev_pool;
    cudaEvent_t cur_a = nullptr;
    std::map<std::string, std::pair<int64_t, double>> prof_acc;
};

namespace {

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int span_of(const apsp_graph *g) { return (int)std::min<int64_t>(round_up(std::max(g->hwm, 1), 32), g->ld); }

cudaEvent_t take_event(apsp_graph *g) {
    if (!g->ev_pool.empty()) {
        cudaEvent_t e = g->ev_pool.back();
        g->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void flush_profile(apsp_graph *g) {
    if (g->pending.empty()) return;
    cudaStreamSynchronize(g->stream);
    for (auto &r : g->pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto &acc = g->prof_acc[r.name];
        acc.first += 1;
        acc.second += ms;
        g->ev_pool.push_back(r.a);
        g->ev_pool.push_back(r.b);
    }
    g->pending.clear();
}

void hook_pre(void *ctx, const char *) {
    apsp_graph *g = (apsp_graph *)ctx;
    g->launches++;
    if (g->prof) {
        if (g->pending.size() > 8192) flush_profile(g);
        g->cur_a = take_event(g);
        cudaEventRecord(g->cur_a, g->stream);
    }
}

void hook_post(void *ctx, const char *name) {
    apsp_graph *g = (apsp_graph *)ctx;
    if (g->prof) {
        cudaEvent_t b = take_event(g);
        cudaEventRecord(b, g->stream);
        g->pending.push_back({name, g->cur_a, b});
    }
}

// The CUDA error behind the last APSP_E_CUDA / APSP_E_NOMEM of this thread.
thread_local int g_last_cuda_error = 0;

apsp_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return APSP_OK;
    g_last_cuda_error = (int)e;
    if (e == cudaErrorMemoryAllocation) return APSP_E_NOMEM;
    return APSP_E_CUDA;
}

void *dalloc(apsp_graph *g, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (g->alloc_fn) {
        p = g->alloc_fn(bytes, (void *)g->stream, g->alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        p = nullptr;
    }
    if (p) {
        g->allocs.push_back({p, bytes});
        g->dev_bytes += (int64_t)bytes;
    }
    return p;
}

// Frees one buffer from dalloc before the handle is destroyed.
void dfree(apsp_graph *g, void *p) {
    if (!p) return;
    for (size_t k = 0; k < g->allocs.size(); ++k) {
        if (g->allocs[k].first != p) continue;
        if (g->free_fn) {
            g->free_fn(p, g->allocs[k].second, (void *)g->stream, g->alloc_ctx);
        } else {
            cudaStreamSynchronize(g->stream);
            cudaFree(p);
        }
        g->dev_bytes -= (int64_t)g->allocs[k].second;
        g->allocs.erase(g->allocs.begin() + (std::ptrdiff_t)k);
        return;
    }
}

// Grows a library-owned device buffer to at least `bytes` (contents are not kept).
bool ensure_buf(apsp_graph *g, void **p, int64_t *have, int64_t bytes) {
    if (*p && *have >= bytes) return true;
    dfree(g, *p);
    *p = dalloc(g, (size_t)bytes);
    *have = *p ? bytes : 0;
    return *p != nullptr;
}

void release(apsp_graph *g) {
    cudaStreamSynchronize(g->stream);
    apsp::destroy_increase_graph(&g->incg);
    for (auto &a : g->allocs) {
        if (g->free_fn) g->free_fn(a.first, a.second, (void *)g->stream, g->alloc_ctx);
        else cudaFree(a.first);
    }
    g->allocs.clear();
    if (g->pin) cudaFreeHost(g->pin);
    if (g->pin_fetch) cudaFreeHost(g->pin_fetch);
    if (g->pin_small) cudaFreeHost(g->pin_small);
    for (int r = 0; r < apsp_graph::RING; ++r) {
        if (g->pin_ev[r]) cudaEventDestroy(g->pin_ev[r]);
        if (g->fetch_ev[r]) cudaEventDestroy(g->fetch_ev[r]);
    }
    for (auto &r : g->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : g->ev_pool) cudaEventDestroy(e);
}

// Reads the control block (waiting for the stream) and turns a sticky device
// error into a status; clears it.
apsp_status sync_ctl(apsp_graph *g, Ctl *out) {
    Ctl *h = (Ctl *)g->pin_small;
    cudaError_t e = cudaMemcpyAsync(h, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (out) *out = *h;
    uint32_t err = h->err;
    if (err) {
        cudaMemsetAsync(&g->ctl->err, 0, sizeof(uint32_t), g->stream);
        cudaStreamSynchronize(g->stream);
        if (err & apsp::ERR_TIMEOUT) return APSP_E_TIMEOUT;
        if (err & apsp::ERR_PASSES) return APSP_E_TIMEOUT;
        if (err & apsp::ERR_NEGATIVE) return APSP_E_NEGATIVE;
        return APSP_E_ARG;
    }
    return APSP_OK;
}

template <typename T> Dev<T> dev_of(apsp_graph *g) {
    Dev<T> d;
    d.W = (T *)g->W;
    d.D = (T *)g->D;
    d.DT = (T *)g->DT;
    d.ld = g->ld;
    d.span = span_of(g);
    d.undirected = g->undirected ? 1 : 0;
    d.alive = g->alive;
    d.w_in = (T *)g->w_in;
    d.w_out = (T *)g->w_out;
    d.vin_k = g->vin_k;
    d.vout_k = g->vout_k;
    d.x = (T *)g->x;
    d.x2 = (T *)g->x2;
    d.y = (T *)g->y;
    d.y2 = (T *)g->y2;
    d.rlist = g->rlist;
    d.hrows = g->hrows;
    d.hunits = g->hunits;
    d.hralloc = g->hralloc;
    d.rowcnt = g->rowcnt;
    d.bmask = g->bmask;
    d.bmask_nb = g->bmask_nb;
    d.hbase = g->hbase;
    d.items = g->items;
    d.icand = g->icand;
    d.p1u = g->p1u;
    d.p1u_cap = g->p1u_cap;
    d.pairs = g->pairs;
    d.pmin = g->pmin;
    d.pstamp = g->pstamp;
    d.rstamp = g->rstamp;
    d.units = g->units;
    d.ctl = g->ctl;
    d.pair_cap = g->pair_cap;
    d.item_cap = g->item_cap;
    d.unit_cap = g->unit_cap;
    return d;
}

cudaError_t reset_ctl(apsp_graph *g) {
    return cudaMemsetAsync(g->ctl, 0, offsetof(Ctl, err), g->stream);
}

template <typename T> T inf_of() { return (T)apsp::MinPlus<T>::inf(); }

// Host-side check of a weight; returns 0 ok, else a status.  Int32 values
// above INF are clamped to INF (missing).
template <typename T> apsp_status check_weight(T &w) {
    if constexpr (std::is_same<T, float>::value) {
        if (std::isnan(w)) return APSP_E_ARG;
        if (w < 0.f) return APSP_E_NEGATIVE;
        if (w == 0.f) w = 0.f;
    } else {
        if (w < 0) return APSP_E_NEGATIVE;
        if (w > apsp::INF_I32) w = apsp::INF_I32;
    }
    return APSP_OK;
}

template <typename T> T *mirror_row(apsp_graph *g, int i) { return (T *)g->Wh.data() + (int64_t)i * g->cap; }
template <typename T> T *mirror_col(apsp_graph *g, int j) { return (T *)g->WhT.data() + (int64_t)j * g->cap; }

// W[i][j] of live i, j (see the mirror's layout in apsp_graph).
template <typename T> T mirror_get(apsp_graph *g, int i, int j) {
    if (i == j) return (T)0;
    return g->add_seq[j] > g->add_seq[i] ? mirror_col<T>(g, j)[i] : mirror_row<T>(g, i)[j];
}

template <typename T> void mirror_edge(apsp_graph *g, int u, int v, T w) {
    mirror_row<T>(g, u)[v] = w;
    mirror_col<T>(g, v)[u] = w;
    if (g->undirected) {
        mirror_row<T>(g, v)[u] = w;
        mirror_col<T>(g, u)[v] = w;
    }
}

// Row and column of the node added at slot p from its raw weight vectors
// (an invalid entry is read as missing; entries of slots that were not live
// at the add are never read: a slot added later defines its own row and
// column).
template <typename T> void mirror_node(apsp_graph *g, int p, const T *in, const T *out) {
    T *r = mirror_row<T>(g, p), *c = mirror_col<T>(g, p);
    for (int t = 0; t < g->cap; ++t) {
        T a = in[t], b = out[t];
        if (check_weight<T>(a) != APSP_OK || check_weight<T>(b) != APSP_OK) a = b = inf_of<T>();
        c[t] = a;
        r[t] = b;
    }
    r[p] = c[p] = (T)0;
}

// Applies a device-input add_node to the mirror once its weight vectors have
// reached the host (waits for that small D2H copy only).  Skipped when the
// slot was added again since.
template <typename T> void settle_one(apsp_graph *g, const apsp_graph::Fetch &f) {
    cudaEventSynchronize(g->fetch_ev[f.ring]);
    if (g->add_seq[f.p] != f.seq) return;
    const T *in = (const T *)g->pin_fetch + (size_t)f.ring * 2 * g->cap;
    mirror_node<T>(g, f.p, in, in + g->cap);
}

// All pending device-input adds (for callers that read the whole mirror).
template <typename T> void settle_fetch(apsp_graph *g) {
    while (!g->fetches.empty()) {
        settle_one<T>(g, g->fetches.front());
        g->fetches.pop_front();
    }
}

// Only the pending adds of slots u and v, whose weights W[u][v] may need:
// other updates read no mirror entry, so a device-input add does not stall
// the host until an edge update touches the added node.
template <typename T> void settle_for(apsp_graph *g, int u, int v) {
    for (auto it = g->fetches.begin(); it != g->fetches.end();) {
        if (it->p == u || it->p == v) {
            settle_one<T>(g, *it);
            it = g->fetches.erase(it);
        } else {
            ++it;
        }
    }
}

template <typename T> RepairCfg repair_cfg(apsp_graph *g, int n_before, float type_feat, float dw) {
    RepairCfg c;
    c.mode = g->mode;
    c.delta = g->delta;
    c.n_live_before = n_before;
    c.has_model = g->has_model ? 1 : 0;
    c.model = g->model;
    c.feat_type = type_feat;
    c.feat_dw = dw;
    c.grown_flag = g->grown_flag;
    c.list_mode = g->list_mode;
    c.umask = g->umask;
    return c;
}

int pick_slot(apsp_graph *g) {
    for (int s = 0; s < g->hwm; ++s)
        if (!g->alive_h[s]) return s;
    return g->hwm < g->cap ? g->hwm : -1;
}

// ---------------------------------------------------------------------------
// typed implementations
// ---------------------------------------------------------------------------

template <typename T>
apsp_status init_impl(apsp_graph *g, const void *W, int n, const void *Dgiven) {
    cudaError_t e;
    const size_t esz = sizeof(T);
    const int64_t ld = g->ld;
    const size_t mat = (size_t)ld * ld * esz;
    g->W = dalloc(g, mat);
    g->D = dalloc(g, mat);
    if (!g->undirected) g->DT = dalloc(g, mat);
    g->alive = (int32_t *)dalloc(g, ld * 4);
    g->w_in = dalloc(g, ld * esz);
    g->w_out = dalloc(g, ld * esz);
    g->x = dalloc(g, ld * esz);
    g->x2 = dalloc(g, ld * esz);
    g->y = dalloc(g, ld * esz);
    g->y2 = dalloc(g, ld * esz);
    g->vin_k = (int32_t *)dalloc(g, ld * 4);
    g->vout_k = (int32_t *)dalloc(g, ld * 4);
    g->rlist = (int32_t *)dalloc(g, ld * 4);
    const int64_t hunit_cap = ld * ((ld + 1023) / 1024);   // every batch of every row
    g->hrows = (int4 *)dalloc(g, ld * sizeof(int4));
    g->hunits = (int4 *)dalloc(g, hunit_cap * sizeof(int4));
    g->hralloc = (int4 *)dalloc(g, ld * sizeof(int4));
    g->rowcnt = (int32_t *)dalloc(g, ld * apsp::DET_MAXB * sizeof(int32_t));
    g->bmask_nb = (int32_t)((ld + 1023) / 1024);
    g->bmask = (uint32_t *)dalloc(g, (size_t)ld * g->bmask_nb * 32 * sizeof(uint32_t));
    g->hbase = (long long *)dalloc(g, hunit_cap * sizeof(long long));
    g->pair_cap = std::min<int64_t>((int64_t)ld * 512, (int64_t)1 << 30);
    g->item_cap = (int32_t)(g->pair_cap / apsp::ITEM_PAIRS + ld);
    g->pairs = (int32_t *)dalloc(g, g->pair_cap * 4);
    g->items = (int4 *)dalloc(g, (size_t)g->item_cap * sizeof(int4));
    g->icand = (int32_t *)dalloc(g, (size_t)2 * ld * sizeof(int32_t));
    g->p1u_cap = (int32_t)(g->pair_cap / apsp::P1_PAIRS + ld);
    g->p1u = (int4 *)dalloc(g, (size_t)g->p1u_cap * sizeof(int4));
    g->incg.args = dalloc(g, 256);
    if (g->incg.args) cudaMemsetAsync(g->incg.args, 0, 256, g->stream);
    static_assert(sizeof(apsp::UpdArgs<float>) <= 256 && sizeof(apsp::UpdArgs<int32_t>) <= 256, "update argument block");
    g->unit_cap = (int32_t)std::min<int64_t>(g->pair_cap, (int64_t)1 << 30);
    g->pmin = (int32_t *)dalloc(g, g->pair_cap * 4);
    g->pstamp = (uint8_t *)dalloc(g, g->pair_cap);
    g->rstamp = (uint8_t *)dalloc(g, ld);
    g->units = (int32_t *)dalloc(g, (size_t)g->unit_cap * 4);
    g->ctl = (Ctl *)dalloc(g, sizeof(Ctl));
    g->model = (float *)dalloc(g, apsp::MLP_NPARAM * sizeof(float));
    if (g->minimax) {
        g->mm_words = (int32_t)(ld / 32);
        g->mm_mask = (uint32_t *)dalloc(g, (size_t)ld * g->mm_words * sizeof(uint32_t));
        if (!g->mm_mask) return APSP_E_NOMEM;
    }
    if (!g->W || !g->D || (!g->undirected && !g->DT) || !g->alive || !g->w_in || !g->w_out || !g->x || !g->x2 ||
        !g->y || !g->y2 || !g->vin_k || !g->vout_k || !g->rlist || !g->pairs || !g->items || !g->icand || !g->p1u || !g->incg.args || !g->ctl || !g->model ||
        !g->pmin || !g->pstamp || !g->rstamp || !g->units || !g->hrows || !g->hunits || !g->hralloc || !g->rowcnt ||
        !g->hbase || !g->bmask)
        return APSP_E_NOMEM;
    if (cudaMallocHost(&g->pin, (size_t)apsp_graph::RING * 2 * g->cap * esz) != cudaSuccess) return APSP_E_NOMEM;
    if (cudaHostAlloc(&g->pin_fetch, (size_t)apsp_graph::RING * 2 * g->cap * esz, cudaHostAllocMapped) != cudaSuccess)
        return APSP_E_NOMEM;
    if (cudaHostGetDevicePointer(&g->pin_fetch_dev, g->pin_fetch, 0) != cudaSuccess) return APSP_E_NOMEM;
    g->pin_small_bytes = std::max<int64_t>(sizeof(Ctl), 1 << 16);
    if (cudaMallocHost(&g->pin_small, g->pin_small_bytes) != cudaSuccess) return APSP_E_NOMEM;
    for (int r = 0; r < apsp_graph::RING; ++r) {
        cudaEventCreateWithFlags(&g->pin_ev[r], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&g->fetch_ev[r], cudaEventDisableTiming);
    }

    if ((e = apsp::setup_shapes<T>(g->lc, ld, g->undirected ? 1 : 0)) != cudaSuccess) return cuda_status(e);
    const LaunchCtx &c = g->lc;
    const T inf = inf_of<T>();
    if ((e = apsp::run_fill<T>(c, (T *)g->W, inf, ld * ld)) != cudaSuccess) return cuda_status(e);
    if ((e = apsp::run_fill<T>(c, (T *)g->D, inf, ld * ld)) != cudaSuccess) return cuda_status(e);
    if (g->DT && (e = apsp::run_fill<T>(c, (T *)g->DT, inf, ld * ld)) != cudaSuccess) return cuda_status(e);
    cudaMemsetAsync(g->alive, 0, ld * 4, g->stream);
    cudaMemsetAsync(g->ctl, 0, sizeof(Ctl), g->stream);
    if (n > 0) apsp::run_fill<int32_t>(c, g->alive, 1, n);
    const cudaMemcpyKind kind = (g->flags & APSP_DEVICE_INPUT) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (n > 0) {
        e = cudaMemcpy2DAsync(g->W, ld * esz, W, (size_t)n * esz, (size_t)n * esz, n, kind, g->stream);
        if (e != cudaSuccess) return cuda_status(e);
        apsp::run_sanitize<T>(c, (T *)g->W, ld, n, g->undirected ? 1 : 0, g->ctl);
    }
    g->hwm = n;
    g->n_live = n;
    Dev<T> d = dev_of<T>(g);
    if ((g->flags & APSP_D_GIVEN) && n > 0) {
        e = cudaMemcpy2DAsync(g->D, ld * esz, Dgiven, (size_t)n * esz, (size_t)n * esz, n, kind, g->stream);
        if (e != cudaSuccess) return cuda_status(e);
        apsp::run_sanitize<T>(c, (T *)g->D, ld, n, 0, g->ctl);
        if ((e = apsp::run_transpose<T>(c, d)) != cudaSuccess) return cuda_status(e);
    } else if (n > 0) {
        e = g->minimax ? apsp::run_mm_fw<T>(c, d) : apsp::run_fw<T>(c, d);
        if (e != cudaSuccess) return cuda_status(e);
    }
    // host mirror of W
    g->alive_h.assign(g->cap, 0);
    for (int i = 0; i < n; ++i) g->alive_h[i] = 1;
    g->Wh.assign((size_t)g->cap * g->cap * esz, 0);
    g->WhT.assign((size_t)g->cap * g->cap * esz, 0);   // read only for slots added later
    g->add_seq.assign(g->cap, 0);
    {
        T *wh = (T *)g->Wh.data();
        std::fill(wh, wh + (size_t)g->cap * g->cap, inf);
        if (n > 0) {
            e = cudaMemcpy2DAsync(wh, (size_t)g->cap * esz, g->W, ld * esz, (size_t)n * esz, n, cudaMemcpyDeviceToHost, g->stream);
            if (e != cudaSuccess) return cuda_status(e);
        }
    }
    apsp_status st = sync_ctl(g, nullptr);
    if (st != APSP_OK) return st;
    g->last = apsp_stats{};
    g->last.op = APSP_OP_INIT;
    g->last.path = APSP_PATH_COLD;
    g->last.node = g->last.node2 = -1;
    g->last.n_live = n;
    return APSP_OK;
}

template <typename T>
apsp_status add_impl(apsp_graph *g, const void *in_w, const void *out_w, int32_t *new_id, bool device_input) {
    if (!out_w || !new_id) return APSP_E_ARG;
    if (!in_w) {
        if (!g->undirected) return APSP_E_ARG;
        in_w = out_w;
    }
    const int p = pick_slot(g);
    if (p < 0) return APSP_E_CAPACITY;
    const int cap = g->cap;
    const T *din, *dout;
    T *fetch = nullptr;   // device-input adds: where the prep kernel copies the raw weights
    int fetch_ring = 0;
    if (!device_input) {
        const T *hi = (const T *)in_w, *ho = (const T *)out_w;
        for (int t = 0; t < cap; ++t) {
            if (t == p || !g->alive_h[t]) continue;
            T a = hi[t], b = ho[t];
            apsp_status s1 = check_weight<T>(a), s2 = check_weight<T>(b);
            if (s1 != APSP_OK) return s1;
            if (s2 != APSP_OK) return s2;
            if (g->undirected && !(a == b)) return APSP_E_ARG;
        }
        // a ring of pinned staging buffers: this waits only for the copy
        // issued RING host-input adds ago
        const int r = g->pin_next;
        g->pin_next = (r + 1) % apsp_graph::RING;
        if (g->pin_used[r]) cudaEventSynchronize(g->pin_ev[r]);
        T *pin_in = (T *)g->pin + (size_t)r * 2 * cap, *pin_out = pin_in + cap;
        std::memcpy(pin_in, hi, cap * sizeof(T));
        std::memcpy(pin_out, ho, cap * sizeof(T));
        cudaMemcpyAsync(g->x, pin_in, cap * sizeof(T), cudaMemcpyHostToDevice, g->stream);
        cudaMemcpyAsync(g->y, pin_out, cap * sizeof(T), cudaMemcpyHostToDevice, g->stream);
        cudaEventRecord(g->pin_ev[r], g->stream);
        g->pin_used[r] = true;
        din = (const T *)g->x;
        dout = (const T *)g->y;
        g->add_seq[p] = ++g->seq;
        mirror_node<T>(g, p, hi, ho);
    } else {
        din = (const T *)in_w;
        dout = (const T *)out_w;
        // the weights reach the mirror later (settle_one), without a wait here
        if ((int)g->fetches.size() == apsp_graph::RING) {
            settle_one<T>(g, g->fetches.front());
            g->fetches.pop_front();
        }
        fetch_ring = g->fetch_next;
        g->fetch_next = (fetch_ring + 1) % apsp_graph::RING;
        fetch = (T *)g->pin_fetch_dev + (size_t)fetch_ring * 2 * cap;   // written by the prep kernel
        g->add_seq[p] = ++g->seq;
        g->fetches.push_back(apsp_graph::Fetch{p, g->add_seq[p], fetch_ring});
    }
    g->hwm = std::max(g->hwm, p + 1);
    reset_ctl(g);
    Dev<T> d = dev_of<T>(g);
    cudaError_t e = g->minimax ? apsp::run_mm_insert<T>(g->lc, d, din, dout, cap, p, fetch)
                               : apsp::run_insert<T>(g->lc, d, din, dout, cap, p, fetch);
    if (e != cudaSuccess) return cuda_status(e);
    if (fetch) cudaEventRecord(g->fetch_ev[fetch_ring], g->stream);
    g->alive_h[p] = 1;
    g->n_live++;
    *new_id = p;
    g->last = apsp_stats{};
    g->last.op = APSP_OP_ADD;
    g->last.path = APSP_PATH_SWEEP;
    g->last.node = p;
    g->last.node2 = -1;
    g->last.n_live = g->n_live;
    return APSP_OK;
}

// Minimax removal / increase after detection (minimax.cuh): reads the list's
// counts (waits), chooses warm or cold by the dispatch mode (delta rule on
// Cost; the cost model is not used here), then re-relaxes the listed pairs
// pass by pass until one lowers nothing, or runs the (min, max)
// Floyd-Warshall.  Fills the statistics of the update.
template <typename T> apsp_status mm_repair(apsp_graph *g, int n_before) {
    Ctl c;
    apsp_status st = sync_ctl(g, &c);
    if (st != APSP_OK) return st;
    g->last.affected_pairs = (int64_t)c.n_pairs;
    g->last.affected_rows = c.n_rows;
    g->last.cost = n_before > 1 ? (float)c.n_rows / (float)(n_before - 1) : 0.f;
    if (c.n_pairs == 0) {
        g->last.path = APSP_PATH_TRIVIAL;
        return APSP_OK;
    }
    const bool cold = g->mode == APSP_DISPATCH_ALWAYS_COLD ||
                      (g->mode != APSP_DISPATCH_ALWAYS_WARM && g->last.cost > g->delta);
    Dev<T> d = dev_of<T>(g);
    cudaError_t e;
    if (cold) {
        if ((e = apsp::run_mm_fw<T>(g->lc, d)) != cudaSuccess) return cuda_status(e);
        g->last.path = APSP_PATH_COLD;
        g->last.cold_reason = g->mode == APSP_DISPATCH_ALWAYS_COLD ? 3 : 1;
        return sync_ctl(g, nullptr);
    }
    g->last.path = APSP_PATH_WARM;
    for (int p = 1; p < apsp::MM_PASS_SLOTS - 1; ++p) {
        if ((e = apsp::run_mm_pass<T>(g->lc, d, g->mm_mask, g->mm_words, p)) != cudaSuccess) return cuda_status(e);
        if (p >= 2 && (p % 2 == 0 || p == apsp::MM_PASS_SLOTS - 2)) {
            if ((st = sync_ctl(g, &c)) != APSP_OK) return st;
            int q = 1;
            while (q <= p && c.mm_changed[q]) ++q;
            if (q <= p) {   // pass q lowered nothing: the fixed point
                g->last.passes = q;
                return APSP_OK;
            }
        }
    }
    return APSP_E_TIMEOUT;   // no fixed point within the pass slots
}

template <typename T> apsp_status remove_impl(apsp_graph *g, int v) {
    if (v < 0 || v >= g->cap || !g->alive_h[v]) return APSP_E_NODE;
    reset_ctl(g);
    if (g->minimax) {
        const int n_before = g->n_live;
        Dev<T> d = dev_of<T>(g);
        cudaError_t e = apsp::run_mm_detect<T>(g->lc, d, g->mm_mask, g->mm_words, 0, v, v, (T)0, (T)0);
        if (e != cudaSuccess) return cuda_status(e);
        g->alive_h[v] = 0;   // the mirror keeps the slot's rows until its next add
        g->n_live--;
        g->last = apsp_stats{};
        g->last.op = APSP_OP_REMOVE;
        g->last.node = v;
        g->last.node2 = -1;
        g->last.n_live = g->n_live;
        return mm_repair<T>(g, n_before);
    }
    Dev<T> d = dev_of<T>(g);
    RepairCfg cfg = repair_cfg<T>(g, g->n_live, 1.0f / 3.0f, 0.0f);
    cudaError_t e = apsp::run_remove<T>(g->lc, d, v, cfg);
    if (e != cudaSuccess) return cuda_status(e);
    g->alive_h[v] = 0;   // the mirror keeps the slot's rows until its next add
    g->n_live--;
    g->last = apsp_stats{};
    g->last.op = APSP_OP_REMOVE;
    g->last.path = -1;  // decided on the device
    g->last.node = v;
    g->last.node2 = -1;
    g->last.n_live = g->n_live;
    return APSP_OK;
}

template <typename T> apsp_status edge_impl(apsp_graph *g, int u, int v, const void *wp) {
    if (!wp) return APSP_E_ARG;
    if (u < 0 || v < 0 || u >= g->cap || v >= g->cap || !g->alive_h[u] || !g->alive_h[v]) return APSP_E_NODE;
    settle_for<T>(g, u, v);
    if (u == v) return APSP_E_ARG;
    T w = *(const T *)wp;
    apsp_status s = check_weight<T>(w);
    if (s != APSP_OK) return s;
    const T w_old = mirror_get<T>(g, u, v);
    g->last = apsp_stats{};
    g->last.node = u;
    g->last.node2 = v;
    g->last.n_live = g->n_live;
    if (w == w_old) {
        g->last.op = APSP_OP_SAME;
        g->last.path = APSP_PATH_NONE;
        return APSP_OK;
    }
    Dev<T> d = dev_of<T>(g);
    cudaError_t e;
    if (g->minimax) {
        reset_ctl(g);
        if (w < w_old) {
            e = apsp::run_mm_decrease<T>(g->lc, d, u, v, w);
            g->last.op = APSP_OP_DECREASE;
            g->last.path = APSP_PATH_SWEEP;
        } else {
            e = apsp::run_mm_detect<T>(g->lc, d, g->mm_mask, g->mm_words, 1, u, v, w_old, w);
            g->last.op = APSP_OP_INCREASE;
        }
        if (e != cudaSuccess) return cuda_status(e);
        mirror_edge<T>(g, u, v, w);
        if (w < w_old) {
            Ctl c;
            apsp_status st = sync_ctl(g, &c);
            g->last.sweep_rows = c.r_count;
            return st;
        }
        return mm_repair<T>(g, g->n_live);
    }
    if (w < w_old) {
        reset_ctl(g);
        e = apsp::run_decrease<T>(g->lc, d, u, v, w);
        g->last.op = APSP_OP_DECREASE;
        g->last.path = APSP_PATH_SWEEP;
    } else {
        float dw = (std::isfinite((double)w) && (double)w < apsp::INF_I32 && (double)w_old > 0)
                       ? (float)(((double)w - (double)w_old) / (double)w_old) : 1.0f;
        RepairCfg cfg = repair_cfg<T>(g, g->n_live, 1.0f, dw);
        // the graph form (inc_graph.cuh) covers the default list mode without
        // per-kernel profiling or the measured Algorithm 12 list
        if (cfg.list_mode == 0 && !cfg.grown_flag && !g->prof) {
            e = apsp::launch_increase_graph<T>(g->lc, d, &g->incg, offsetof(Ctl, err), u, v, w_old, w, cfg);
        } else {
            reset_ctl(g);
            e = apsp::run_increase<T>(g->lc, d, u, v, w_old, w, cfg);
        }
        g->last.op = APSP_OP_INCREASE;
        g->last.path = -1;
    }
    if (e != cudaSuccess) return cuda_status(e);
    mirror_edge<T>(g, u, v, w);
    return APSP_OK;
}

template <typename T> apsp_status recompute_impl(apsp_graph *g) {
    settle_fetch<T>(g);
    Dev<T> d = dev_of<T>(g);
    cudaError_t e = g->minimax ? apsp::run_mm_fw<T>(g->lc, d) : apsp::run_fw<T>(g->lc, d);
    if (e != cudaSuccess) return cuda_status(e);
    g->last = apsp_stats{};
    g->last.op = APSP_OP_RECOMPUTE;
    g->last.path = APSP_PATH_COLD;
    g->last.node = g->last.node2 = -1;
    g->last.n_live = g->n_live;
    return APSP_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Path queries (Section 4): Algorithm 7 for batches of pairs, Algorithm 8 for
// one pair (its joins assembled here from the device's trees).
// ---------------------------------------------------------------------------

namespace {

constexpr int PQ_CHUNK = 65536;

inline int pq_slots(const apsp_graph *g) { return (int)round_up(g->ld + 2, 4); }

bool pq_nodes_ok(const apsp_graph *g, int u, int v) {
    return u >= 0 && v >= 0 && u < g->cap && v < g->cap && g->alive_h[u] && g->alive_h[v];
}

// Runs the path kernel over nb queries (uv host) and copies the rows of
// `row` int32 back into out_h; redoes deferred queries with the wide pass.
template <typename T>
apsp_status pq_run(apsp_graph *g, const int32_t *uv, int nb, int mode, int stride, int64_t row,
                   std::vector<int32_t> &out_h) {
    const int S = pq_slots(g);
    const int64_t wide_stride = 5 * (int64_t)S + (2 * (int64_t)S + 3) / 4;
    if (!ensure_buf(g, &g->pq_uv, &g->pq_uv_bytes, (int64_t)nb * 8) ||
        !ensure_buf(g, &g->pq_out, &g->pq_out_bytes, (int64_t)nb * row * 4) ||
        !ensure_buf(g, &g->pq_wide, &g->pq_wide_bytes, apsp::PQ_WIDE_GRID * wide_stride * 4))
        return APSP_E_NOMEM;
    cudaError_t e = cudaMemcpyAsync(g->pq_uv, uv, (size_t)nb * 8, cudaMemcpyHostToDevice, g->stream);
    if (e != cudaSuccess) return cuda_status(e);
    apsp::PathQuery q;
    q.uv = (const int32_t *)g->pq_uv;
    q.count = nb;
    q.out = (int32_t *)g->pq_out;
    q.row = row;
    q.stride = stride;
    q.mode = mode;
    q.wide = (int32_t *)g->pq_wide;
    q.wide_stride = wide_stride;
    q.wide_slots = S;
    const Dev<T> d = dev_of<T>(g);
    out_h.resize((size_t)nb * row);
    q.all = nb < g->lc.num_sms ? 1 : 0;
    for (int tier = q.all ? 1 : 0; tier < 3; ++tier) {
        if ((e = apsp::run_path_query<T>(g->lc, d, q, tier)) != cudaSuccess) return cuda_status(e);
        e = cudaMemcpyAsync(out_h.data(), g->pq_out, (size_t)nb * row * 4, cudaMemcpyDeviceToHost, g->stream);
        if (e != cudaSuccess) return cuda_status(e);
        apsp_status st = sync_ctl(g, nullptr);
        if (st != APSP_OK) return st;
        const int32_t marker = tier == 0 ? apsp::PQ_DEFERRED : apsp::PQ_DEFERRED_WIDE;
        bool deferred = false;
        for (int k = 0; k < nb && !deferred; ++k) deferred = out_h[(size_t)k * row] == marker;
        if (!deferred || tier == 2) break;   // the next tier reads the markers from the device copy
    }
    for (int k = 0; k < nb; ++k)
        if (out_h[(size_t)k * row] < 0) return APSP_E_ARG;   // D is not the APSP matrix of W
    return APSP_OK;
}

template <typename T>
apsp_status paths_impl(apsp_graph *g, const int32_t *uv, int32_t count, int32_t *paths, int32_t stride,
                       int32_t *lens) {
    if (count < 0 || stride < 0 || (count > 0 && (!uv || !lens)) || (count > 0 && stride > 0 && !paths))
        return APSP_E_ARG;
    for (int32_t k = 0; k < count; ++k)
        if (!pq_nodes_ok(g, uv[2 * k], uv[2 * k + 1])) return APSP_E_NODE;
    settle_fetch<T>(g);
    const int64_t row = 1 + (int64_t)stride;
    std::vector<int32_t> out_h;
    for (int32_t b0 = 0; b0 < count; b0 += PQ_CHUNK) {
        const int nb = std::min(PQ_CHUNK, count - b0);
        apsp_status st = pq_run<T>(g, uv + 2 * (int64_t)b0, nb, 0, stride, row, out_h);
        if (st != APSP_OK) return st;
        for (int k = 0; k < nb; ++k) {
            const int32_t *o = out_h.data() + (size_t)k * row;
            lens[b0 + k] = o[0];
            const int keep = std::min<int32_t>(o[0], stride);
            if (keep > 0) std::memcpy(paths + (int64_t)(b0 + k) * stride, o + 1, (size_t)keep * 4);
        }
    }
    return APSP_OK;
}

// Walks a predecessor array from small node `from` until `to`; empty if it
// does not get there within K steps.
std::vector<int32_t> pq_walk(const int32_t *pred, int K, int from, int to) {
    std::vector<int32_t> w{from};
    while (w.back() != to) {
        const int32_t p = pred[w.back()];
        if (p < 0 || (int)w.size() > K) return {};
        w.push_back(p);
    }
    return w;
}

// Next hops of the requested rows, in chunks that bound the device buffer.
template <typename T>
apsp_status next_hops_impl(apsp_graph *g, const int32_t *rows, int32_t count, int32_t *out, int64_t ld_out) {
    settle_fetch<T>(g);
    const int64_t S = g->hwm;
    const Dev<T> d = dev_of<T>(g);
    const int64_t P = std::max<int64_t>(d.span, 1);   // device pitch: the kernel writes span columns a row
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(count, ((int64_t)1 << 26) / P));
    if (!ensure_buf(g, &g->nh_rows, &g->nh_rows_bytes, chunk * 4) ||
        !ensure_buf(g, &g->nh_out, &g->nh_out_bytes, chunk * P * 4))
        return APSP_E_NOMEM;
    for (int64_t r0 = 0; r0 < count; r0 += chunk) {
        const int nr = (int)std::min<int64_t>(chunk, count - r0);
        cudaError_t e = cudaMemcpyAsync(g->nh_rows, rows + r0, (size_t)nr * 4, cudaMemcpyHostToDevice, g->stream);
        if (e == cudaSuccess)
            e = apsp::run_next_hop<T>(g->lc, d, (const int32_t *)g->nh_rows, nr, (int32_t *)g->nh_out, P);
        if (e == cudaSuccess && S > 0)
            e = cudaMemcpy2DAsync(out + r0 * ld_out, (size_t)ld_out * 4, g->nh_out, (size_t)P * 4, (size_t)S * 4, nr,
                                  cudaMemcpyDeviceToHost, g->stream);
        if (e != cudaSuccess) return cuda_status(e);
        apsp_status st = sync_ctl(g, nullptr);
        if (st != APSP_OK) return st;
    }
    return APSP_OK;
}

template <typename T>
apsp_status all_paths_impl(apsp_graph *g, int32_t u, int32_t v, int32_t *nodes, int64_t nodes_cap,
                           int64_t *offsets, int32_t paths_cap, int32_t *n_paths, int64_t *n_nodes) {
    if (!n_paths || !n_nodes || nodes_cap < 0 || paths_cap < 0) return APSP_E_ARG;
    if (!pq_nodes_ok(g, u, v)) return APSP_E_NODE;
    settle_fetch<T>(g);
    std::vector<std::vector<int32_t>> out;
    if (u == v) {
        out.push_back({u});
    } else {
        const int S = pq_slots(g);
        const int64_t row = 1 + 3 * (int64_t)S;
        const int32_t uv[2] = {u, v};
        std::vector<int32_t> o;
        apsp_status st = pq_run<T>(g, uv, 1, 1, 0, row, o);
        if (st != APSP_OK) return st;
        const int K = o[0];
        if (K >= 2) {
            const int32_t *cand = o.data() + 1, *pf = cand + K, *pb = pf + K;
            // Psi(i, j): the forward tree path to small node K - 1
            std::vector<int32_t> psi = pq_walk(pf, K, K - 1, 0);
            if (psi.empty()) return APSP_E_ARG;
            std::reverse(psi.begin(), psi.end());
            std::set<std::vector<int32_t>> seen;
            // Float weights: a candidate may lie within the candidate test's
            // slack of a shortest path without being on one, so a join is
            // kept only if its length (summed in double from the weights)
            // is within the small Dijkstra's rounding, (2 K + 2) * 2^-24
            // relative, of the length of Algorithm 7's path.  Int32
            // candidates are exact and every join is a shortest path.
            const bool fp = std::is_same<T, float>::value;
            auto length = [&](const std::vector<int32_t> &small) {
                double L = 0.0;
                for (size_t k = 0; k + 1 < small.size(); ++k) L += (double)mirror_get<T>(g, cand[small[k]], cand[small[k + 1]]);
                return L;
            };
            const double lim = fp ? length(psi) * (1.0 + (2.0 * K + 2.0) * 0x1p-24) : 0.0;
            auto emit = [&](const std::vector<int32_t> &small) {
                if (fp && !out.empty() && length(small) > lim) return;
                std::vector<int32_t> p(small.size());
                for (size_t k = 0; k < small.size(); ++k) p[k] = cand[small[k]];
                if (seen.insert(p).second) out.push_back(std::move(p));
            };
            emit(psi);
            std::vector<int32_t> stamp(K, -1);
            for (int t = 1; t < K - 1; ++t) {
                std::vector<int32_t> first = pq_walk(pf, K, t, 0);       // t .. 0
                std::vector<int32_t> second = pq_walk(pb, K, t, K - 1);  // t .. K - 1
                if (first.empty() || second.empty()) continue;
                std::reverse(first.begin(), first.end());
                first.insert(first.end(), second.begin() + 1, second.end());
                bool simple = true;   // a join through a zero-weight cycle is a walk, not a path
                for (int32_t a : first) {
                    if (stamp[a] == t) {
                        simple = false;
                        break;
                    }
                    stamp[a] = t;
                }
                if (simple) emit(first);
            }
        }
    }
    int64_t total = 0;
    for (auto &p : out) total += (int64_t)p.size();
    *n_paths = (int32_t)out.size();
    *n_nodes = total;
    if (!nodes || !offsets) return APSP_OK;   // size query
    if ((int64_t)out.size() > paths_cap || total > nodes_cap) return APSP_E_ARG;
    int64_t at = 0;
    for (size_t k = 0; k < out.size(); ++k) {
        offsets[k] = at;
        std::memcpy(nodes + at, out[k].data(), out[k].size() * 4);
        at += (int64_t)out[k].size();
    }
    offsets[out.size()] = at;
    return APSP_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

const char *apsp_version(void) { return "0.1.0"; }

int32_t apsp_last_cuda_error(const char **name) {
    if (name) *name = cudaGetErrorName((cudaError_t)g_last_cuda_error);
    return g_last_cuda_error;
}

const char *apsp_status_string(apsp_status s) {
    switch (s) {
    case APSP_OK: return "ok";
    case APSP_E_ARG: return "invalid argument";
    case APSP_E_NODE: return "node id out of range or not live";
    case APSP_E_NEGATIVE: return "negative weight";
    case APSP_E_CAPACITY: return "no free slot";
    case APSP_E_NOMEM: return "out of memory";
    case APSP_E_CUDA: return "CUDA error";
    case APSP_E_TIMEOUT: return "bounded device wait timed out";
    case APSP_E_BUSY: return "busy";
    case APSP_E_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

apsp_status apsp_set_allocator(apsp_alloc_fn alloc, apsp_free_fn free_fn, void *ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) return APSP_E_ARG;
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_ctx = ctx;
    return APSP_OK;
}

apsp_status apsp_init(apsp_graph **out, const void *W, int32_t n, int32_t capacity, apsp_dtype dtype,
                      uint32_t flags, const void *D_or_null, void *cuda_stream) {
    if (!out) return APSP_E_ARG;
    *out = nullptr;
    if (n < 0 || capacity < 1 || n > capacity || capacity > APSP_MAX_CAPACITY) return APSP_E_ARG;
    if (dtype != APSP_I32 && dtype != APSP_F32) return APSP_E_ARG;
    if (flags & ~(uint32_t)(APSP_UNDIRECTED | APSP_D_GIVEN | APSP_DEVICE_INPUT | APSP_MINIMAX)) return APSP_E_ARG;
    if (n > 0 && !W) return APSP_E_ARG;
    if ((flags & APSP_D_GIVEN) && !D_or_null) return APSP_E_ARG;
    int dev = 0, ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1 || cudaGetDevice(&dev) != cudaSuccess) return APSP_E_CUDA;
    apsp_graph *g = new apsp_graph();
    g->dtype = dtype;
    g->flags = flags;
    g->undirected = (flags & APSP_UNDIRECTED) != 0;
    g->minimax = (flags & APSP_MINIMAX) != 0;
    g->cap = capacity;
    g->ld = round_up(capacity, 128);
    g->esz = 4;
    g->stream = (cudaStream_t)cuda_stream;
    g->alloc_fn = g_alloc;
    g->free_fn = g_free;
    g->alloc_ctx = g_alloc_ctx;
    cudaGetDevice(&g->device);
    cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    g->lc.stream = g->stream;
    g->lc.num_sms = g->num_sms;
    g->lc.hook = apsp::Hook{hook_pre, hook_post, g};
    apsp_status st = dtype == APSP_F32 ? init_impl<float>(g, W, n, D_or_null) : init_impl<int32_t>(g, W, n, D_or_null);
    if (st != APSP_OK) {
        release(g);
        delete g;
        return st;
    }
    *out = g;
    return APSP_OK;
}

apsp_status apsp_destroy(apsp_graph *g) {
    if (!g) return APSP_E_ARG;
    release(g);
    delete g;
    return APSP_OK;
}

apsp_status apsp_add_node(apsp_graph *g, const void *in_w, const void *out_w, int32_t *new_id) {
    if (!g) return APSP_E_ARG;
    return g->dtype == APSP_F32 ? add_impl<float>(g, in_w, out_w, new_id, false) : add_impl<int32_t>(g, in_w, out_w, new_id, false);
}

apsp_status apsp_add_node_device(apsp_graph *g, const void *in_w, const void *out_w, int32_t *new_id) {
    if (!g) return APSP_E_ARG;
    return g->dtype == APSP_F32 ? add_impl<float>(g, in_w, out_w, new_id, true) : add_impl<int32_t>(g, in_w, out_w, new_id, true);
}

apsp_status apsp_remove_node(apsp_graph *g, int32_t v) {
    if (!g) return APSP_E_ARG;
    return g->dtype == APSP_F32 ? remove_impl<float>(g, v) : remove_impl<int32_t>(g, v);
}

apsp_status apsp_update_edge(apsp_graph *g, int32_t u, int32_t v, const void *w) {
    if (!g) return APSP_E_ARG;
    return g->dtype == APSP_F32 ? edge_impl<float>(g, u, v, w) : edge_impl<int32_t>(g, u, v, w);
}

apsp_status apsp_recompute(apsp_graph *g) {
    if (!g) return APSP_E_ARG;
    return g->dtype == APSP_F32 ? recompute_impl<float>(g) : recompute_impl<int32_t>(g);
}

apsp_status apsp_query(apsp_graph *g, int32_t u, int32_t v, void *dist_out) {
    if (!g || !dist_out) return APSP_E_ARG;
    if (u < 0 || v < 0 || u >= g->cap || v >= g->cap || !g->alive_h[u] || !g->alive_h[v]) return APSP_E_NODE;
    char *h = (char *)g->pin_small + sizeof(Ctl);
    cudaError_t e = cudaMemcpyAsync(h, (const char *)g->D + ((int64_t)u * g->ld + v) * g->esz, g->esz,
                                    cudaMemcpyDeviceToHost, g->stream);
    if (e != cudaSuccess) return cuda_status(e);
    apsp_status st = sync_ctl(g, nullptr);
    std::memcpy(dist_out, h, g->esz);
    return st;
}

apsp_status apsp_query_batch(apsp_graph *g, const int32_t *uv, int32_t count, void *out) {
    if (!g || (count > 0 && (!uv || !out)) || count < 0) return APSP_E_ARG;
    for (int32_t i = 0; i < count; ++i) {
        int u = uv[2 * i], v = uv[2 * i + 1];
        if (u < 0 || v < 0 || u >= g->cap || v >= g->cap || !g->alive_h[u] || !g->alive_h[v]) return APSP_E_NODE;
    }
    const int64_t room = (g->pin_small_bytes - (int64_t)sizeof(Ctl)) / (int64_t)g->esz;
    char *h = (char *)g->pin_small + sizeof(Ctl);
    for (int32_t b0 = 0; b0 < count; b0 += (int32_t)room) {
        int32_t nb = (int32_t)std::min<int64_t>(room, count - b0);
        for (int32_t i = 0; i < nb; ++i) {
            int u = uv[2 * (b0 + i)], v = uv[2 * (b0 + i) + 1];
            cudaMemcpyAsync(h + i * g->esz, (const char *)g->D + ((int64_t)u * g->ld + v) * g->esz, g->esz,
                            cudaMemcpyDeviceToHost, g->stream);
        }
        apsp_status st = sync_ctl(g, nullptr);
        if (st != APSP_OK) return st;
        std::memcpy((char *)out + (size_t)b0 * g->esz, h, (size_t)nb * g->esz);
    }
    return APSP_OK;
}

// Path queries (Section 4): Algorithm 7 and Algorithm 8.
apsp_status apsp_query_paths(apsp_graph *g, const int32_t *uv, int32_t count, int32_t *paths, int32_t stride,
                             int32_t *lens) {
    if (!g) return APSP_E_ARG;
    if (g->minimax) return APSP_E_UNSUPPORTED;
    return g->dtype == APSP_F32 ? paths_impl<float>(g, uv, count, paths, stride, lens)
                                : paths_impl<int32_t>(g, uv, count, paths, stride, lens);
}

apsp_status apsp_query_path(apsp_graph *g, int32_t u, int32_t v, int32_t *path, int32_t cap, int32_t *len) {
    const int32_t uv[2] = {u, v};
    return apsp_query_paths(g, uv, 1, path, cap, len);
}

apsp_status apsp_query_all_paths(apsp_graph *g, int32_t u, int32_t v, int32_t *nodes, int64_t nodes_cap,
                                 int64_t *offsets, int32_t paths_cap, int32_t *n_paths, int64_t *n_nodes) {
    if (!g) return APSP_E_ARG;
    if (g->minimax) return APSP_E_UNSUPPORTED;
    return g->dtype == APSP_F32 ? all_paths_impl<float>(g, u, v, nodes, nodes_cap, offsets, paths_cap, n_paths, n_nodes)
                                : all_paths_impl<int32_t>(g, u, v, nodes, nodes_cap, offsets, paths_cap, n_paths, n_nodes);
}

apsp_status apsp_next_hops(apsp_graph *g, const int32_t *rows, int32_t count, int32_t *out, int64_t ld_out) {
    if (!g || count < 0 || (count > 0 && (!rows || !out)) || ld_out < g->hwm) return APSP_E_ARG;
    if (g->minimax) return APSP_E_UNSUPPORTED;
    for (int32_t r = 0; r < count; ++r)
        if (rows[r] < 0 || rows[r] >= g->cap || !g->alive_h[rows[r]]) return APSP_E_NODE;
    if (count == 0) return APSP_OK;
    return g->dtype == APSP_F32 ? next_hops_impl<float>(g, rows, count, out, ld_out)
                                : next_hops_impl<int32_t>(g, rows, count, out, ld_out);
}

static apsp_status copy_mat(apsp_graph *g, const void *src, void *dst, int64_t ld_dst, int32_t on_dev) {
    if (!g || !dst || ld_dst < g->hwm) return APSP_E_ARG;
    if (g->hwm > 0) {
        cudaError_t e = cudaMemcpy2DAsync(dst, ld_dst * g->esz, src, g->ld * g->esz, (size_t)g->hwm * g->esz, g->hwm,
                                          on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return sync_ctl(g, nullptr);
}

apsp_status apsp_copy_D(apsp_graph *g, void *dst, int64_t ld_dst, int32_t on_dev) { return g ? copy_mat(g, g->D, dst, ld_dst, on_dev) : APSP_E_ARG; }
apsp_status apsp_copy_W(apsp_graph *g, void *dst, int64_t ld_dst, int32_t on_dev) { return g ? copy_mat(g, g->W, dst, ld_dst, on_dev) : APSP_E_ARG; }

apsp_status apsp_copy_alive(apsp_graph *g, uint8_t *alive) {
    if (!g || !alive) return APSP_E_ARG;
    std::memcpy(alive, g->alive_h.data(), g->cap);
    return APSP_OK;
}

apsp_status apsp_info_get(apsp_graph *g, apsp_info *info) {
    if (!g || !info) return APSP_E_ARG;
    info->n_live = g->n_live;
    info->n_slots = g->hwm;
    info->capacity = g->cap;
    info->ld = (int32_t)g->ld;
    info->dtype = g->dtype;
    info->flags = g->flags;
    info->device_bytes = g->dev_bytes;
    return APSP_OK;
}

apsp_status apsp_sync(apsp_graph *g) {
    if (!g) return APSP_E_ARG;
    return sync_ctl(g, nullptr);
}

apsp_status apsp_last_stats(apsp_graph *g, apsp_stats *s) {
    if (!g || !s) return APSP_E_ARG;
    Ctl c;
    apsp_status st = sync_ctl(g, &c);
    *s = g->last;
    s->grown_pairs = -1;
    s->grown_rows = -1;
    s->grown_cost = -1.f;
    if (g->minimax) return st;   // filled by the update itself
    const int op = g->last.op;
    if (op == APSP_OP_REMOVE || op == APSP_OP_INCREASE) {
        s->affected_rows = c.n_rows;
        s->affected_pairs = (int64_t)c.n_pairs;
        s->overflow = c.overflow;
        s->passes = c.passes;
        s->cold_reason = c.cold_reason;
        s->cost = c.cost;
        s->model_warm = c.model_warm;
        s->model_cold = c.model_cold;
        s->sweep_rows = c.r_count;
        s->pairs_rechecked = (int64_t)c.pairs_evaluated;
        if (g->grown_flag && !c.overflow) {
            s->grown_pairs = (int64_t)c.grown_pairs;
            s->grown_rows = c.grown_rows;
            const int N = op == APSP_OP_REMOVE ? s->n_live + 1 : s->n_live;
            s->grown_cost = N > 1 ? (float)c.grown_rows / (float)(N - 1) : 0.f;
        }
        if (c.path == apsp::PATH_WARM && c.t_end > c.t_start) {
            s->warm_pass1_us = (float)((double)(c.t_pass1 - c.t_start) * 1e-3);
            s->warm_total_us = (float)((double)(c.t_end - c.t_start) * 1e-3);
        }
        s->path = c.path == apsp::PATH_COLD ? APSP_PATH_COLD
                : c.path == apsp::PATH_WARM ? APSP_PATH_WARM : APSP_PATH_TRIVIAL;
        if (op == APSP_OP_REMOVE && c.path == 0) s->path = APSP_PATH_TRIVIAL;
    } else if (op == APSP_OP_DECREASE) {
        s->sweep_rows = c.r_count;
        s->path = c.r_count > 0 ? APSP_PATH_SWEEP : APSP_PATH_TRIVIAL;
    } else if (op == APSP_OP_ADD) {
        s->reduce_rows = c.ins_narrow ? c.ins_nout + c.ins_nin : -1;
    }
    return st;
}

apsp_status apsp_copy_last_list(apsp_graph *g, int32_t *ij, int64_t cap, int64_t *count) {
    if (!g || !count) return APSP_E_ARG;
    *count = 0;
    Ctl c;
    apsp_status st = sync_ctl(g, &c);
    if (st != APSP_OK) return st;
    const int op = g->last.op;
    if (op != APSP_OP_REMOVE && op != APSP_OP_INCREASE) return APSP_OK;
    if (g->minimax) {
        const int64_t words = g->mm_words, rows = g->hwm;
        std::vector<uint32_t> m((size_t)(rows * words));
        if (rows > 0) {
            cudaError_t e = cudaMemcpyAsync(m.data(), g->mm_mask, m.size() * 4, cudaMemcpyDeviceToHost, g->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
            if (e != cudaSuccess) return cuda_status(e);
        }
        int64_t n = 0;
        for (uint32_t x : m) n += __builtin_popcount(x);
        *count = n;
        if (!ij) return APSP_OK;
        if (cap < n) return APSP_E_ARG;
        int64_t q = 0;
        for (int64_t i = 0; i < rows; ++i)
            for (int64_t wd = 0; wd < words; ++wd)
                for (uint32_t x = m[(size_t)(i * words + wd)]; x; x &= x - 1) {
                    ij[2 * q] = (int32_t)i;
                    ij[2 * q + 1] = (int32_t)(wd * 32 + __builtin_ctz(x));
                    ++q;
                }
        return APSP_OK;
    }
    if (c.overflow) return APSP_E_CAPACITY;
    const int n_items = (int)(c.alloc & 0xFFFFFFull);
    const int64_t n_pairs = (int64_t)(c.alloc >> 24);
    if (c.trivial || n_items == 0) return APSP_OK;
    *count = n_pairs;
    if (!ij) return APSP_OK;
    if (cap < n_pairs) return APSP_E_ARG;
    std::vector<int4> items((size_t)n_items);
    std::vector<int32_t> cols((size_t)n_pairs);
    cudaError_t e = cudaMemcpyAsync(items.data(), g->items, sizeof(int4) * (size_t)n_items, cudaMemcpyDeviceToHost,
                                    g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cols.data(), g->pairs, sizeof(int32_t) * (size_t)n_pairs, cudaMemcpyDeviceToHost,
                            g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_status(e);
    int64_t q = 0;
    for (const int4 &it : items) {
        const int cnt = it.z & 0xFF;
        if (it.y < 0 || (int64_t)it.y + cnt > n_pairs || q + cnt > n_pairs) return APSP_E_CUDA;
        for (int k = 0; k < cnt; ++k, ++q) {
            ij[2 * q] = it.x;
            ij[2 * q + 1] = cols[(size_t)it.y + k];
        }
    }
    if (q != n_pairs) return APSP_E_CUDA;
    return APSP_OK;
}

apsp_status apsp_set_dispatch(apsp_graph *g, apsp_dispatch mode, double delta) {
    if (!g || mode < APSP_DISPATCH_DELTA || mode > APSP_DISPATCH_MODEL || !(delta >= 0.0)) return APSP_E_ARG;
    g->mode = mode;
    g->delta = (float)delta;
    return APSP_OK;
}

apsp_status apsp_set_list_mode(apsp_graph *g, apsp_list_mode mode) {
    if (!g || mode < APSP_LIST_COROLLARY3 || mode > APSP_LIST_ALGORITHM12) return APSP_E_ARG;
    if (g->minimax && mode != APSP_LIST_COROLLARY3) return APSP_E_UNSUPPORTED;
    if (mode == APSP_LIST_ALGORITHM12 && !g->umask) {
        const int64_t hunit_cap = g->ld * ((g->ld + 1023) / 1024);
        g->umask = (uint32_t *)dalloc(g, (size_t)hunit_cap * 32 * sizeof(uint32_t));
        if (!g->umask) return APSP_E_NOMEM;
    }
    g->list_mode = mode;
    return APSP_OK;
}

apsp_status apsp_set_exact_list(apsp_graph *g, int32_t on) {
    if (!g) return APSP_E_ARG;
    if (g->minimax && on) return APSP_E_UNSUPPORTED;
    if (on && !g->grown_flag) {
        g->grown_flag = (int32_t *)dalloc(g, (size_t)g->ld * sizeof(int32_t));
        if (!g->grown_flag) return APSP_E_NOMEM;
    } else if (!on && g->grown_flag) {
        dfree(g, g->grown_flag);
        g->grown_flag = nullptr;
    }
    return APSP_OK;
}

apsp_status apsp_set_model(apsp_graph *g, const float *params) {
    if (!g) return APSP_E_ARG;
    if (!params) {
        g->has_model = false;
        return APSP_OK;
    }
    for (int i = 0; i < apsp::MLP_IN; ++i)   // standardisation divides by sd
        if (!(params[apsp::MLP_OFF_SD + i] > 0.f)) return APSP_E_ARG;
    // the copy is staged before the call returns (pageable source)
    cudaError_t e = cudaMemcpyAsync(g->model, params, apsp::MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice, g->stream);
    if (e != cudaSuccess) return cuda_status(e);
    g->has_model = true;
    return APSP_OK;
}

int64_t apsp_launch_count(apsp_graph *g) {
    if (!g) return -1;
    // kernels of increase graphs whose IF body ran (a device counter; waits for the stream)
    unsigned long long bodies = 0;
    if (g->incg.args) {
        const size_t off = g->dtype == APSP_F32 ? offsetof(apsp::UpdArgs<float>, bodies) : offsetof(apsp::UpdArgs<int32_t>, bodies);
        cudaMemcpyAsync(&bodies, (const char *)g->incg.args + off, sizeof(bodies), cudaMemcpyDeviceToHost, g->stream);
        cudaStreamSynchronize(g->stream);
    }
    return g->launches + (int64_t)apsp::INC_GRAPH_BODY_KERNELS * (int64_t)bodies;
}

apsp_status apsp_profile_enable(apsp_graph *g, int32_t on) {
    if (!g) return APSP_E_ARG;
    g->prof = on != 0;
    return APSP_OK;
}

apsp_status apsp_profile_read(apsp_graph *g, apsp_profile_entry *out, int32_t cap, int32_t *count) {
    if (!g || !count || (cap > 0 && !out)) return APSP_E_ARG;
    flush_profile(g);
    int32_t i = 0;
    for (auto &kv : g->prof_acc) {
        if (i < cap) {
            std::memset(&out[i], 0, sizeof(apsp_profile_entry));
            std::strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
            out[i].launches = kv.second.first;
            out[i].total_ms = kv.second.second;
        }
        ++i;
    }
    *count = i;
    return APSP_OK;
}

apsp_status apsp_profile_reset(apsp_graph *g) {
    if (!g) return APSP_E_ARG;
    flush_profile(g);
    g->prof_acc.clear();
    return APSP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched execution (apsp_batch_*): the host validates every item, resolves
// slots / old weights / spans in order on each graph's mirrors, packs one
// upload (header, graph table, updates, masked new-node vectors) and launches
// one persistent kernel (k_batch) over all graphs.
// ---------------------------------------------------------------------------

struct apsp_batch {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int32_t *h_done = nullptr;    // mapped completion flags, one per graph of the last launch
    int32_t *d_done = nullptr;
    int done_cap = 0;
    size_t o_tab = 0;             // where the graph table sits in the last upload
    int n_graphs = 0;
    char *h_blob = nullptr;   // pinned staging of the upload
    size_t h_cap = 0;
    char *d_blob = nullptr;
    size_t d_cap = 0;
    uint32_t *d_mask = nullptr;   // listed-pair bitmasks
    size_t mask_cap = 0;          // words
    void *d_team = nullptr;       // team scratch (vectors, listed rows, counters) for large graphs
    size_t team_cap = 0;
    bool team_dirty = false;      // counters must be zeroed before the next launch
    // One CUDA graph per (dtype, CTA width) holding a whole launch: the
    // upload, the persistent kernel and the status read-back.  Later launches
    // of the same kind only update the three nodes' parameters (sizes,
    // pointers, grid, shared memory) and replay it.
    struct Captured {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphNode_t h2d = nullptr, kern = nullptr, d2h = nullptr;
        void *func = nullptr;
    };
    Captured cap[2][3];
    int nt_fixed = 0;             // 0: the autotuner picks the CTA width
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int pend_dtype = -1, pend_bucket = -1, pend_k = -1;   // launch awaiting its time for the autotuner
    double pend_work = 0.0;
    int64_t launches = 0, captures = 0, replays = 0;
    int last_nt = 0;
};

namespace {

size_t align256(size_t a) { return (a + 255) & ~size_t(255); }

// Graphs whose sweeps span at least this many slots go to teams of CTAs.
constexpr int TEAM_MIN_SPAN = 384;

template <typename T> apsp_status batch_weight(double w, T *out) {
    if (std::isnan(w)) return APSP_E_ARG;
    if (w < 0) return APSP_E_NEGATIVE;
    if constexpr (std::is_same<T, float>::value) {
        *out = w >= (double)std::numeric_limits<float>::max() ? inf_of<float>() : (float)w;
        if (*out == 0.f) *out = 0.f;
    } else {
        if (w >= (double)apsp::INF_I32) {
            *out = apsp::INF_I32;
        } else {
            if (w != std::floor(w)) return APSP_E_ARG;
            *out = (int32_t)w;
        }
    }
    return APSP_OK;
}

template <typename T> int32_t bits_of(T v) {
    int32_t b;
    std::memcpy(&b, &v, sizeof(b));
    return b;
}

// ---- autotuner of the batched kernel's CTA width -------------------------
// Process-wide table per (dtype, log2 of the batch's widest span).  Results
// never depend on the width, so tuning runs on live batches: each width is
// used for TUNE_SAMPLES batches of enough work, the cost of a batch being its
// device time per span^2 summed over its updates, and the cheapest mean wins
// and is kept for the rest of the process.
constexpr int TUNE_SAMPLES = 2;
constexpr double TUNE_MIN_WORK = 1 << 20;
struct TuneCell {
    double cost[3] = {0, 0, 0};
    int n[3] = {0, 0, 0};
    int chosen = -1;
};
std::mutex g_tune_mu;
TuneCell g_tune[2][32];

int tune_bucket(int max_span) {
    int b = 0;
    while ((1 << b) < max_span && b < 31) ++b;
    return b;
}

int tune_pick(int dtype, int bucket) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneCell &c = g_tune[dtype][bucket];
    if (c.chosen >= 0) return c.chosen;
    for (int k = 0; k < 3; ++k)
        if (c.n[k] < TUNE_SAMPLES) return k;
    int best = 0;
    for (int k = 1; k < 3; ++k)
        if (c.cost[k] / c.n[k] < c.cost[best] / c.n[best]) best = k;
    c.chosen = best;
    return best;
}

void tune_record(int dtype, int bucket, int k, double cost) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneCell &c = g_tune[dtype][bucket];
    if (c.chosen >= 0 || c.n[k] >= TUNE_SAMPLES) return;
    c.cost[k] += cost;
    c.n[k]++;
}

// Captures one launch (upload, kernel, read-back) as a CUDA graph.
template <typename T>
cudaError_t batch_capture(apsp_batch *b, apsp_batch::Captured &cp, size_t total, size_t o_tab, size_t tab_bytes,
                          int grid, size_t smem, int nt) {
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaMemcpyAsync(b->d_blob, b->h_blob, total, cudaMemcpyHostToDevice, b->stream);
    apsp::run_batch<T>(b->stream, reinterpret_cast<apsp::BatchHeader *>(b->d_blob), grid, smem, nt);
    cudaMemcpyAsync(b->h_blob + o_tab, b->d_blob + o_tab, tab_bytes, cudaMemcpyDeviceToHost, b->stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->stream, &graph);
    if (e != cudaSuccess) return e;
    cudaGraphNode_t nodes[8];
    size_t num = 8;
    if ((e = cudaGraphGetNodes(graph, nodes, &num)) != cudaSuccess || num != 3) {
        cudaGraphDestroy(graph);
        return e != cudaSuccess ? e : cudaErrorStreamCaptureInvalidated;
    }
    for (size_t k = 0; k < num; ++k) {
        cudaGraphNodeType t;
        cudaGraphNodeGetType(nodes[k], &t);
        if (t == cudaGraphNodeTypeKernel) {
            cudaKernelNodeParams kp{};
            cudaGraphKernelNodeGetParams(nodes[k], &kp);
            cp.kern = nodes[k];
            cp.func = kp.func;
        } else if (t == cudaGraphNodeTypeMemcpy) {
            cudaMemcpy3DParms mp{};
            cudaGraphMemcpyNodeGetParams(nodes[k], &mp);
            if (mp.srcPtr.ptr == b->h_blob) cp.h2d = nodes[k];
            else cp.d2h = nodes[k];
        }
    }
    cudaGraphExec_t exec = nullptr;
    if (!cp.kern || !cp.h2d || !cp.d2h || (e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return e != cudaSuccess ? e : cudaErrorStreamCaptureInvalidated;
    }
    cp.graph = graph;
    cp.exec = exec;
    b->captures++;
    return cudaSuccess;
}

// Enqueues one launch: replays the captured graph of this (dtype, width)
// with updated parameters, capturing it first if needed.
template <typename T>
cudaError_t batch_enqueue(apsp_batch *b, size_t total, size_t o_tab, size_t tab_bytes, int grid, size_t smem, int nt,
                          int k) {
    const int dt = std::is_same<T, float>::value ? 1 : 0;
    apsp_batch::Captured &cp = b->cap[dt][k];
    cudaError_t e;
    if (!cp.exec) {
        if ((e = batch_capture<T>(b, cp, total, o_tab, tab_bytes, grid, smem, nt)) != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
    }
    if ((e = cudaGraphExecMemcpyNodeSetParams1D(cp.exec, cp.h2d, b->d_blob, b->h_blob, total,
                                                cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    apsp::BatchHeader *dh = reinterpret_cast<apsp::BatchHeader *>(b->d_blob);
    void *args[] = {&dh};
    cudaKernelNodeParams kp{};
    kp.func = cp.func;
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(nt);
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    if ((e = cudaGraphExecKernelNodeSetParams(cp.exec, cp.kern, &kp)) != cudaSuccess) return e;
    if ((e = cudaGraphExecMemcpyNodeSetParams1D(cp.exec, cp.d2h, b->h_blob + o_tab, b->d_blob + o_tab, tab_bytes,
                                                cudaMemcpyDeviceToHost)) != cudaSuccess)
        return e;
    if ((e = cudaGraphLaunch(cp.exec, b->stream)) != cudaSuccess) return e;
    b->replays++;
    return cudaSuccess;
}

// Validates, resolves and launches the batch on b->stream without waiting;
// per-graph completion flags go to b->h_done when `flags` is set.
template <typename T>
apsp_status batch_launch(apsp_batch *b, apsp_graph *const *graphs, int n_graphs, const apsp_batch_item *items,
                         int count, int32_t *new_ids, bool flags) {
    using apsp::BatchGraph;
    using apsp::BatchHeader;
    using apsp::BatchOp;
    std::vector<std::vector<int>> per(n_graphs);
    for (int q = 0; q < count; ++q) per[items[q].graph].push_back(q);
    // ---- validation on simulated liveness (nothing changes on an error)
    for (int gi = 0; gi < n_graphs; ++gi) {
        apsp_graph *g = graphs[gi];
        std::vector<uint8_t> alive = g->alive_h;
        int hwm = g->hwm;
        for (int q : per[gi]) {
            const apsp_batch_item &it = items[q];
            if (it.op == APSP_BATCH_ADD) {
                int p = -1;
                for (int s = 0; s < hwm && p < 0; ++s)
                    if (!alive[s]) p = s;
                if (p < 0) p = hwm < g->cap ? hwm : -1;
                if (p < 0) return APSP_E_CAPACITY;
                if (!it.in_w || !it.out_w) return APSP_E_ARG;
                const T *hi = (const T *)it.in_w, *ho = (const T *)it.out_w;
                for (int t = 0; t < g->cap; ++t) {
                    if (t == p || !alive[t]) continue;
                    T a = hi[t], c = ho[t];
                    apsp_status s1 = check_weight<T>(a), s2 = check_weight<T>(c);
                    if (s1 != APSP_OK) return s1;
                    if (s2 != APSP_OK) return s2;
                }
                alive[p] = 1;
                hwm = std::max(hwm, p + 1);
            } else if (it.op == APSP_BATCH_REMOVE) {
                if (it.u < 0 || it.u >= g->cap || !alive[it.u]) return APSP_E_NODE;
                alive[it.u] = 0;
            } else if (it.op == APSP_BATCH_EDGE) {
                if (it.u < 0 || it.v < 0 || it.u >= g->cap || it.v >= g->cap || !alive[it.u] || !alive[it.v])
                    return APSP_E_NODE;
                if (it.u == it.v) return APSP_E_ARG;
                T w;
                apsp_status s = batch_weight<T>(it.w, &w);
                if (s != APSP_OK) return s;
            } else {
                return APSP_E_ARG;
            }
        }
    }
    // ---- wait for each graph's own pending work
    for (int gi = 0; gi < n_graphs; ++gi) {
        settle_fetch<T>(graphs[gi]);
        if (cudaStreamSynchronize(graphs[gi]->stream) != cudaSuccess) return APSP_E_CUDA;
    }
    // ---- resolve the updates in order on the mirrors
    std::vector<BatchGraph> table;
    std::vector<BatchOp> ops;
    std::vector<T> vecs;
    std::vector<int> spans;
    int max_span = 32;
    for (int gi = 0; gi < n_graphs; ++gi) {
        apsp_graph *g = graphs[gi];
        BatchGraph bg{};
        bg.D = g->D;
        bg.DT = g->DT;
        bg.W = g->W;
        bg.alive = g->alive;
        bg.ld = g->ld;
        bg.first = (int)ops.size();
        int gspan = span_of(g);
        for (int q : per[gi]) {
            const apsp_batch_item &it = items[q];
            if (new_ids) new_ids[q] = -1;
            BatchOp op{};
            if (it.op == APSP_BATCH_ADD) {
                const int p = pick_slot(g);
                g->hwm = std::max(g->hwm, p + 1);
                const int span = span_of(g);
                const T *hi = (const T *)it.in_w, *ho = (const T *)it.out_w;
                op.op = apsp::BOP_ADD;
                op.a = p;
                op.span = span;
                op.vec = (int64_t)vecs.size();
                vecs.resize(vecs.size() + 2 * (size_t)span, inf_of<T>());
                T *wi = vecs.data() + op.vec, *wo = wi + span;
                T *mr = mirror_row<T>(g, p), *mc = mirror_col<T>(g, p);
                for (int t = 0; t < g->cap; ++t) {
                    T a = inf_of<T>(), c = inf_of<T>();
                    if (t != p && g->alive_h[t]) {
                        a = hi[t];
                        c = ho[t];
                        check_weight<T>(a);
                        check_weight<T>(c);
                    }
                    if (t < span) {
                        wi[t] = a;
                        wo[t] = c;
                    }
                    mc[t] = a;
                    mr[t] = c;
                }
                mr[p] = mc[p] = (T)0;
                g->add_seq[p] = ++g->seq;
                g->alive_h[p] = 1;
                g->n_live++;
                if (new_ids) new_ids[q] = p;
            } else if (it.op == APSP_BATCH_REMOVE) {
                op.op = apsp::BOP_REMOVE;
                op.a = it.u;
                op.span = span_of(g);
                g->alive_h[it.u] = 0;
                g->n_live--;
            } else {
                T w;
                batch_weight<T>(it.w, &w);
                const T w_old = mirror_get<T>(g, it.u, it.v);
                if (w == w_old) continue;
                op.op = w < w_old ? apsp::BOP_DECREASE : apsp::BOP_INCREASE;
                op.a = it.u;
                op.b = it.v;
                op.span = span_of(g);
                op.w_bits = bits_of<T>(w);
                op.w_old_bits = bits_of<T>(w_old);
                mirror_edge<T>(g, it.u, it.v, w);
            }
            gspan = std::max(gspan, op.span);
            ops.push_back(op);
        }
        bg.count = (int)ops.size() - bg.first;
        bg.mask_words = (gspan + 31) / 32;
        spans.push_back(gspan);
        max_span = std::max(max_span, gspan);
        table.push_back(bg);
    }
    // ---- device buffers
    size_t mask_words = 0;
    for (int gi = 0; gi < n_graphs; ++gi) mask_words += (size_t)spans[gi] * table[gi].mask_words;
    if (mask_words > b->mask_cap) {
        if (b->d_mask) cudaFree(b->d_mask);
        b->d_mask = nullptr;
        b->mask_cap = 0;
        if (cudaMalloc(&b->d_mask, mask_words * 4) != cudaSuccess) return APSP_E_NOMEM;
        b->mask_cap = mask_words;
    }
    size_t off = 0;
    for (int gi = 0; gi < n_graphs; ++gi) {
        table[gi].mask = b->d_mask + off;
        off += (size_t)spans[gi] * table[gi].mask_words;
    }
    const size_t o_hdr = 0, o_tab = align256(sizeof(BatchHeader));
    const size_t o_ops = o_tab + align256(table.size() * sizeof(BatchGraph));
    const size_t o_vec = o_ops + align256(std::max<size_t>(1, ops.size()) * sizeof(BatchOp));
    const size_t o_ord = o_vec + align256(std::max<size_t>(1, vecs.size()) * sizeof(T));
    const size_t total = o_ord + align256((size_t)n_graphs * sizeof(int32_t));
    if (total > b->h_cap) {
        if (b->h_blob) cudaFreeHost(b->h_blob);
        b->h_blob = nullptr;
        b->h_cap = 0;
        if (cudaMallocHost(&b->h_blob, total) != cudaSuccess) return APSP_E_NOMEM;
        b->h_cap = total;
    }
    if (total > b->d_cap) {
        if (b->d_blob) cudaFree(b->d_blob);
        b->d_blob = nullptr;
        b->d_cap = 0;
        if (cudaMalloc(&b->d_blob, total) != cudaSuccess) return APSP_E_NOMEM;
        b->d_cap = total;
    }
    BatchHeader hdr{};
    hdr.graphs = reinterpret_cast<BatchGraph *>(b->d_blob + o_tab);
    hdr.ops = reinterpret_cast<const BatchOp *>(b->d_blob + o_ops);
    hdr.vecs = b->d_blob + o_vec;
    hdr.n_graphs = n_graphs;
    hdr.max_span = max_span;
    hdr.queue = 0;
    hdr.done = nullptr;
    if (flags) {
        if (n_graphs > b->done_cap) {
            if (b->h_done) cudaFreeHost(b->h_done);
            b->h_done = nullptr;
            b->done_cap = 0;
            if (cudaHostAlloc(&b->h_done, (size_t)n_graphs * sizeof(int32_t), cudaHostAllocMapped) != cudaSuccess)
                return APSP_E_NOMEM;
            if (cudaHostGetDevicePointer((void **)&b->d_done, b->h_done, 0) != cudaSuccess) return APSP_E_CUDA;
            b->done_cap = n_graphs;
        }
        std::memset(b->h_done, 0, (size_t)n_graphs * sizeof(int32_t));
        hdr.done = b->d_done;
    }
    std::memcpy(b->h_blob + o_hdr, &hdr, sizeof(hdr));
    std::memcpy(b->h_blob + o_tab, table.data(), table.size() * sizeof(BatchGraph));
    if (!ops.empty()) std::memcpy(b->h_blob + o_ops, ops.data(), ops.size() * sizeof(BatchOp));
    if (!vecs.empty()) std::memcpy(b->h_blob + o_vec, vecs.data(), vecs.size() * sizeof(T));
    // CTA width: fixed by the caller, else the autotuner's choice for this size
    const int dt = std::is_same<T, float>::value ? 1 : 0;
    const int bucket = tune_bucket(max_span);
    int k = 1;
    if (b->nt_fixed) k = b->nt_fixed == 128 ? 0 : b->nt_fixed == 512 ? 2 : 1;
    else k = tune_pick(dt, bucket);
    const int nt = apsp::BATCH_WIDTHS[k];
    const size_t smem = (size_t)max_span * (4 * sizeof(T) + sizeof(int32_t));
    cudaError_t e;
    int per_sm = 0, dev = 0, sms = 1;
    if ((e = apsp::batch_occupancy<T>(smem, nt, &per_sm)) != cudaSuccess) return cuda_status(e);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // Teams for the large graphs when the batch has fewer graphs than CTAs
    // that fit on the device at once (otherwise single CTAs already keep
    // every SM busy; measured: teams cost 8 % on 512 graphs): teams of G (at
    // most TEAM_MAX) CTAs.  The large graphs go first in the order, largest
    // first, then the others, largest first (the longest jobs start earliest).
    const int C = std::max(1, per_sm) * sms;
    std::vector<int32_t> order((size_t)n_graphs);
    for (int gi = 0; gi < n_graphs; ++gi) order[gi] = gi;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t c) { return spans[a] > spans[c]; });
    int n_large = 0;
    while (n_large < n_graphs && spans[order[n_large]] >= TEAM_MIN_SPAN) ++n_large;
    int team = 1, n_teams = 0;
    if (n_large > 0 && n_graphs < C) {   // with a graph for every CTA, single CTAs already fill the device
        team = std::min(apsp::TEAM_MAX, std::max(2, C / n_large));
        n_teams = std::min(n_large, C / team);
    }
    if (n_teams < 1) {
        team = 1;
        n_teams = 0;
        n_large = 0;
    }
    const int grid = std::max(1, std::min(C, std::max(n_teams * team + (n_graphs - n_large), n_teams * team)));
    const int64_t team_stride = (int64_t)align256(4 * (size_t)max_span * sizeof(T) + (size_t)max_span * 4 +
                                                  apsp::TEAM_INTS * 4);
    if (n_teams > 0) {
        const size_t need = (size_t)n_teams * (size_t)team_stride;
        if (need > b->team_cap) {
            if (b->d_team) cudaFree(b->d_team);
            b->d_team = nullptr;
            b->team_cap = 0;
            if (cudaMalloc(&b->d_team, need) != cudaSuccess) return APSP_E_NOMEM;
            b->team_cap = need;
            b->team_dirty = true;
        }
        if (b->team_dirty) {   // barrier counters start at zero
            if (cudaMemsetAsync(b->d_team, 0, b->team_cap, b->stream) != cudaSuccess) return APSP_E_CUDA;
            b->team_dirty = false;
        }
    }
    hdr.n_team = n_large;
    hdr.team_size = team;
    hdr.n_teams = n_teams;
    hdr.order = reinterpret_cast<const int32_t *>(b->d_blob + o_ord);
    hdr.team_scratch = b->d_team;
    hdr.team_stride = team_stride;
    std::memcpy(b->h_blob + o_hdr, &hdr, sizeof(hdr));
    std::memcpy(b->h_blob + o_ord, order.data(), (size_t)n_graphs * sizeof(int32_t));
    const size_t tab_bytes = table.size() * sizeof(BatchGraph);
    double work = 0.0;
    for (const BatchOp &op : ops) work += (double)op.span * op.span;
    if (!b->ev0) {
        cudaEventCreate(&b->ev0);
        cudaEventCreate(&b->ev1);
    }
    cudaEventRecord(b->ev0, b->stream);
    if (batch_enqueue<T>(b, total, o_tab, tab_bytes, grid, smem, nt, k) != cudaSuccess) {
        // no graph (for example a stream that cannot be captured): plain launches
        if ((e = cudaMemcpyAsync(b->d_blob, b->h_blob, total, cudaMemcpyHostToDevice, b->stream)) != cudaSuccess)
            return cuda_status(e);
        if ((e = apsp::run_batch<T>(b->stream, reinterpret_cast<BatchHeader *>(b->d_blob), grid, smem, nt)) !=
            cudaSuccess)
            return cuda_status(e);
        // statuses back (the graph table is re-read after the kernel)
        e = cudaMemcpyAsync(b->h_blob + o_tab, b->d_blob + o_tab, tab_bytes, cudaMemcpyDeviceToHost, b->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    cudaEventRecord(b->ev1, b->stream);
    b->launches++;
    b->last_nt = nt;
    b->pend_dtype = (!b->nt_fixed && work >= TUNE_MIN_WORK) ? dt : -1;
    b->pend_bucket = bucket;
    b->pend_k = k;
    b->pend_work = work;
    b->o_tab = o_tab;
    b->n_graphs = n_graphs;
    return APSP_OK;
}

// Waits for the last launch and returns its status.
apsp_status batch_finish(apsp_batch *b) {
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (b->pend_dtype >= 0) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, b->ev0, b->ev1) == cudaSuccess && ms > 0.f)
            tune_record(b->pend_dtype, b->pend_bucket, b->pend_k, ms / b->pend_work);
        b->pend_dtype = -1;
    }
    const apsp::BatchGraph *done = reinterpret_cast<const apsp::BatchGraph *>(b->h_blob + b->o_tab);
    for (int gi = 0; gi < b->n_graphs; ++gi)
        if (done[gi].status) {
            if (done[gi].status & apsp::ERR_TIMEOUT) b->team_dirty = true;   // a team barrier may be mid-count
            return APSP_E_TIMEOUT;
        }
    return APSP_OK;
}

template <typename T>
apsp_status batch_impl(apsp_batch *b, apsp_graph *const *graphs, int n_graphs, const apsp_batch_item *items, int count,
                       int32_t *new_ids) {
    apsp_status s = batch_launch<T>(b, graphs, n_graphs, items, count, new_ids, false);
    return s != APSP_OK ? s : batch_finish(b);
}

}  // namespace

extern "C" {

apsp_status apsp_batch_create(apsp_batch **out, void *cuda_stream) {
    if (!out) return APSP_E_ARG;
    apsp_batch *b = new (std::nothrow) apsp_batch();
    if (!b) return APSP_E_NOMEM;
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return APSP_E_CUDA;
        }
        b->own_stream = true;
    }
    *out = b;
    return APSP_OK;
}

apsp_status apsp_batch_destroy(apsp_batch *b) {
    if (!b) return APSP_E_ARG;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->h_blob) cudaFreeHost(b->h_blob);
    if (b->d_blob) cudaFree(b->d_blob);
    if (b->d_mask) cudaFree(b->d_mask);
    if (b->d_team) cudaFree(b->d_team);
    if (b->h_done) cudaFreeHost(b->h_done);
    for (auto &row : b->cap)
        for (auto &cp : row) {
            if (cp.exec) cudaGraphExecDestroy(cp.exec);
            if (cp.graph) cudaGraphDestroy(cp.graph);
        }
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return APSP_OK;
}

apsp_status apsp_batch_set_width(apsp_batch *b, int32_t threads) {
    if (!b || (threads != 0 && threads != 128 && threads != 256 && threads != 512)) return APSP_E_ARG;
    b->nt_fixed = threads;
    return APSP_OK;
}

apsp_status apsp_batch_info_get(apsp_batch *b, apsp_batch_info *info) {
    if (!b || !info) return APSP_E_ARG;
    info->launches = b->launches;
    info->graph_captures = b->captures;
    info->graph_replays = b->replays;
    info->last_width = b->last_nt;
    info->fixed_width = b->nt_fixed;
    return APSP_OK;
}

apsp_status apsp_batch_tuned_width(apsp_dtype dtype, int32_t max_span, int32_t *threads) {
    if (!threads || (dtype != APSP_I32 && dtype != APSP_F32) || max_span < 1) return APSP_E_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const TuneCell &c = g_tune[dtype == APSP_F32 ? 1 : 0][tune_bucket(max_span)];
    *threads = c.chosen >= 0 ? apsp::BATCH_WIDTHS[c.chosen] : 0;
    return APSP_OK;
}

apsp_status apsp_batch_run(apsp_batch *b, apsp_graph *const *graphs, int32_t n_graphs, const apsp_batch_item *items,
                           int32_t count, int32_t *new_ids) {
    if (!b || !graphs || n_graphs <= 0 || count < 0 || (count > 0 && !items)) return APSP_E_ARG;
    const int dtype = graphs[0] ? graphs[0]->dtype : -1;
    for (int gi = 0; gi < n_graphs; ++gi) {
        apsp_graph *g = graphs[gi];
        if (!g || g->dtype != dtype) return APSP_E_ARG;
        if (g->undirected || !g->DT || g->minimax || g->cap > APSP_BATCH_MAX_SLOTS) return APSP_E_UNSUPPORTED;
        for (int gj = 0; gj < gi; ++gj)
            if (graphs[gj] == g) return APSP_E_ARG;
    }
    for (int q = 0; q < count; ++q)
        if (items[q].graph < 0 || items[q].graph >= n_graphs) return APSP_E_ARG;
    if (dtype == APSP_F32) return batch_impl<float>(b, graphs, n_graphs, items, count, new_ids);
    return batch_impl<int32_t>(b, graphs, n_graphs, items, count, new_ids);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Serving loop (apsp_serve): real-time replay of a request trace with
// wave-level continuous batching.
// ---------------------------------------------------------------------------

namespace {

struct Clock {
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

}  // namespace

struct apsp_server {
    struct Req {
        apsp_batch_item item{};
        std::vector<char> iw, ow;   // copies of an ADD's weight vectors
        apsp_request_result res{};
        bool done = false;
    };
    std::vector<apsp_graph *> graphs;
    apsp_serve_config cfg{};
    int dtype = APSP_I32, device = 0;
    std::vector<char> small;
    std::vector<double> bytes;
    apsp_batch *b = nullptr;
    void *qbuf = nullptr;           // pinned: the query result in flight, one element per graph
    Clock clk;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req> reqs;           // by ticket; deque: elements never move
    std::deque<int64_t> inbox;      // submitted, not yet taken by the worker
    bool stop = false;
    std::thread worker;
};

namespace {

// The worker: intake, completions, then one dispatch round over the graphs
// that have no work on the GPU.
template <typename T> void server_loop(apsp_server *s) {
    cudaSetDevice(s->device);
    const int G = (int)s->graphs.size();
    struct GraphState {
        std::deque<int64_t> pend;
        bool busy = false, in_batch = false, bdone = false;
        std::vector<int64_t> seg;
        int64_t query = -1;
        int bidx = -1;
        cudaEvent_t ev = nullptr;
    };
    std::vector<GraphState> gs(G);
    for (auto &g : gs) cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming);
    cudaEvent_t small_q_ev = nullptr;
    cudaEventCreateWithFlags(&small_q_ev, cudaEventDisableTiming);
    T *qbuf = (T *)s->qbuf;
    bool batch_busy = false, batch_q = false;
    apsp_status bst = APSP_OK;
    std::vector<int> bg;
    double used = 0;
    int wave = 0;

    auto finish = [&](int gi, apsp_status override_st) {
        GraphState &g = gs[gi];
        const double t = s->clk.now();
        std::lock_guard<std::mutex> lock(s->mu);
        for (int64_t q : g.seg) {
            apsp_server::Req &r = s->reqs[(size_t)q];
            r.res.done_s = t;
            if (override_st != APSP_OK && r.res.status == APSP_OK) r.res.status = override_st;
            if (r.item.op == APSP_BATCH_QUERY && r.res.status == APSP_OK) r.res.dist = (double)qbuf[gi];
            r.done = true;
        }
        g.seg.clear();
        g.busy = g.in_batch = false;
        g.query = -1;
        used -= s->bytes[gi];
        s->cv_done.notify_all();
    };
    // the graph's requests up to and including its first query
    auto take = [&](int gi, int &budget_left) {
        GraphState &g = gs[gi];
        while (!g.pend.empty() && budget_left != 0) {
            const int64_t q = g.pend.front();
            g.pend.pop_front();
            g.seg.push_back(q);
            if (budget_left > 0) --budget_left;
            if (s->reqs[(size_t)q].item.op == APSP_BATCH_QUERY) {
                g.query = q;
                break;
            }
        }
    };
    // one call per update on the graph's own stream
    auto issue_calls = [&](int gi) {
        GraphState &g = gs[gi];
        apsp_graph *gr = s->graphs[gi];
        for (int64_t q : g.seg) {
            apsp_server::Req &r = s->reqs[(size_t)q];
            const apsp_batch_item &it = r.item;
            apsp_status st = APSP_OK;
            if (it.op == APSP_BATCH_ADD) {
                int32_t id = -1;
                st = apsp_add_node(gr, it.in_w, it.out_w, &id);
                r.res.new_id = id;
            } else if (it.op == APSP_BATCH_REMOVE) {
                st = apsp_remove_node(gr, it.u);
            } else if (it.op == APSP_BATCH_EDGE) {
                T w;
                st = batch_weight<T>(it.w, &w);
                if (st == APSP_OK) st = apsp_update_edge(gr, it.u, it.v, &w);
            } else if (it.u < 0 || it.v < 0 || it.u >= gr->cap || it.v >= gr->cap) {
                st = APSP_E_NODE;
            } else {
                cudaMemcpyAsync(qbuf + gi, (T *)gr->D + (int64_t)it.u * gr->ld + it.v, sizeof(T),
                                cudaMemcpyDeviceToHost, gr->stream);
            }
            r.res.status = st;
        }
        cudaEventRecord(g.ev, gr->stream);
        g.busy = true;
    };

    while (true) {
        // ---- intake
        {
            std::unique_lock<std::mutex> lock(s->mu);
            while (!s->inbox.empty()) {
                const int64_t q = s->inbox.front();
                s->inbox.pop_front();
                gs[s->reqs[(size_t)q].item.graph].pend.push_back(q);
            }
            if (s->stop) {
                bool idle = !batch_busy;
                for (auto &g : gs) idle = idle && !g.busy && g.pend.empty();
                if (idle) break;
            }
        }
        bool progress = false;
        // ---- completions: graphs on their own streams
        for (int gi = 0; gi < G; ++gi)
            if (gs[gi].busy && !gs[gi].in_batch && cudaEventQuery(gs[gi].ev) == cudaSuccess) {
                finish(gi, APSP_OK);
                progress = true;
            }
        // ---- completions: the batched launch (per-graph flags in mapped memory)
        if (batch_busy) {
            bool all = true, q_ready = !batch_q;
            for (int gi : bg) {
                GraphState &g = gs[gi];
                if (g.bdone) continue;
                const int flag = ((volatile int32_t *)s->b->h_done)[g.bidx];
                if (flag > 1) bst = APSP_E_TIMEOUT;
                if (flag != 0 && g.query >= 0 && !q_ready) q_ready = cudaEventQuery(small_q_ev) == cudaSuccess;
                if (flag != 0 && (g.query < 0 || q_ready)) {
                    g.bdone = true;
                    finish(gi, bst);
                    progress = true;
                } else {
                    all = false;
                }
            }
            if (all) {
                batch_finish(s->b);
                batch_busy = false;
                bg.clear();
            }
        }
        // ---- dispatch round
        int budget_left = s->cfg.max_wave_requests > 0 ? s->cfg.max_wave_requests : -1;
        std::vector<int> round;
        auto fits = [&](int gi) {
            return s->cfg.hbm_budget_bytes <= 0 || used <= 0 || used + s->bytes[gi] <= s->cfg.hbm_budget_bytes;
        };
        if (!batch_busy) {
            std::vector<apsp_graph *> bgraphs;
            std::vector<apsp_batch_item> bitems;
            std::vector<int64_t> bmap;
            for (int gi = 0; gi < G && budget_left != 0; ++gi) {
                GraphState &g = gs[gi];
                if (!s->small[gi] || g.busy || g.pend.empty() || !fits(gi)) continue;
                take(gi, budget_left);
                g.busy = g.in_batch = true;
                g.bdone = false;
                g.bidx = (int)bgraphs.size();
                used += s->bytes[gi];
                bgraphs.push_back(s->graphs[gi]);
                bg.push_back(gi);
                round.push_back(gi);
                for (int64_t q : g.seg) {
                    const apsp_batch_item &it = s->reqs[(size_t)q].item;
                    if (it.op == APSP_BATCH_QUERY) continue;
                    apsp_batch_item bi = it;
                    bi.graph = g.bidx;
                    bitems.push_back(bi);
                    bmap.push_back(q);
                }
            }
            if (!bgraphs.empty()) {
                std::vector<int32_t> ids(bitems.size(), -1);
                bst = batch_launch<T>(s->b, bgraphs.data(), (int)bgraphs.size(), bitems.data(), (int)bitems.size(),
                                      ids.data(), true);
                if (bst == APSP_OK) {
                    batch_busy = true;
                    batch_q = false;
                    for (size_t k = 0; k < bmap.size(); ++k) s->reqs[(size_t)bmap[k]].res.new_id = ids[k];
                    for (int gi : bg)
                        if (gs[gi].query >= 0) {
                            const apsp_batch_item &it = s->reqs[(size_t)gs[gi].query].item;
                            apsp_graph *gr = s->graphs[gi];
                            if (it.u < 0 || it.v < 0 || it.u >= gr->cap || it.v >= gr->cap) {
                                s->reqs[(size_t)gs[gi].query].res.status = APSP_E_NODE;
                                continue;
                            }
                            cudaMemcpyAsync(qbuf + gi, (T *)gr->D + (int64_t)it.u * gr->ld + it.v, sizeof(T),
                                            cudaMemcpyDeviceToHost, s->b->stream);
                            batch_q = true;
                        }
                    if (batch_q) cudaEventRecord(small_q_ev, s->b->stream);
                } else {
                    // a request the batch rejects: these graphs go one call per
                    // update instead, so each request gets its own status
                    for (int gi : bg) {
                        gs[gi].in_batch = false;
                        issue_calls(gi);
                    }
                    bg.clear();
                    bst = APSP_OK;
                }
            }
        }
        for (int gi = 0; gi < G && budget_left != 0; ++gi) {
            GraphState &g = gs[gi];
            if (s->small[gi] || g.busy || g.pend.empty() || !fits(gi)) continue;
            take(gi, budget_left);
            used += s->bytes[gi];
            issue_calls(gi);
            round.push_back(gi);
        }
        if (!round.empty()) {
            const double t = s->clk.now();
            std::lock_guard<std::mutex> lock(s->mu);
            for (int gi : round)
                for (int64_t q : gs[gi].seg) {
                    s->reqs[(size_t)q].res.admit_s = t;
                    s->reqs[(size_t)q].res.wave = wave;
                }
            ++wave;
            progress = true;
        }
        if (!progress) {
            std::unique_lock<std::mutex> lock(s->mu);
            bool anything_busy = batch_busy;
            for (auto &g : gs) anything_busy = anything_busy || g.busy;
            if (s->inbox.empty() && !s->stop)
                s->cv_work.wait_for(lock, std::chrono::microseconds(anything_busy ? 20 : 2000));
        }
    }
    for (auto &g : gs) cudaEventDestroy(g.ev);
    cudaEventDestroy(small_q_ev);
}

}  // namespace

extern "C" {

apsp_status apsp_server_create(apsp_server **out, apsp_graph *const *graphs, int32_t n_graphs,
                               const apsp_serve_config *cfg) {
    if (!out || !graphs || n_graphs <= 0 || !cfg) return APSP_E_ARG;
    *out = nullptr;
    const int dtype = graphs[0] ? graphs[0]->dtype : -1;
    for (int gi = 0; gi < n_graphs; ++gi) {
        if (!graphs[gi] || graphs[gi]->dtype != dtype) return APSP_E_ARG;
        if (graphs[gi]->minimax) return APSP_E_UNSUPPORTED;
        for (int gj = 0; gj < gi; ++gj)
            if (graphs[gj] == graphs[gi]) return APSP_E_ARG;
    }
    apsp_server *s = new (std::nothrow) apsp_server();
    if (!s) return APSP_E_NOMEM;
    s->graphs.assign(graphs, graphs + n_graphs);
    s->cfg = *cfg;
    s->dtype = dtype;
    s->device = graphs[0]->device;
    for (int gi = 0; gi < n_graphs; ++gi) {
        apsp_graph *g = graphs[gi];
        s->small.push_back(cfg->small_max_slots > 0 && g->cap <= cfg->small_max_slots && !g->undirected && g->DT &&
                           g->cap <= APSP_BATCH_MAX_SLOTS);
        s->bytes.push_back((double)g->ld * g->ld * g->esz * (g->undirected ? 2 : 3));
    }
    apsp_status st = apsp_batch_create(&s->b, nullptr);
    if (st != APSP_OK) {
        delete s;
        return st;
    }
    if (cudaMallocHost(&s->qbuf, (size_t)n_graphs * 4) != cudaSuccess) {
        apsp_batch_destroy(s->b);
        delete s;
        return APSP_E_NOMEM;
    }
    s->worker = dtype == APSP_F32 ? std::thread(server_loop<float>, s) : std::thread(server_loop<int32_t>, s);
    *out = s;
    return APSP_OK;
}

apsp_status apsp_server_submit(apsp_server *s, const apsp_batch_item *item, int64_t *ticket) {
    if (!s || !item || !ticket) return APSP_E_ARG;
    if (item->graph < 0 || item->graph >= (int)s->graphs.size() || item->op < 0 || item->op > APSP_BATCH_QUERY)
        return APSP_E_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return APSP_E_BUSY;
    s->reqs.emplace_back();
    apsp_server::Req &r = s->reqs.back();
    r.item = *item;
    r.res.new_id = -1;
    r.res.wave = -1;
    r.res.status = APSP_OK;
    if (item->op == APSP_BATCH_ADD) {
        const size_t n = (size_t)s->graphs[item->graph]->cap * 4;
        if (item->in_w) r.iw.assign((const char *)item->in_w, (const char *)item->in_w + n);
        if (item->out_w) r.ow.assign((const char *)item->out_w, (const char *)item->out_w + n);
        r.item.in_w = item->in_w ? r.iw.data() : nullptr;
        r.item.out_w = item->out_w ? r.ow.data() : nullptr;
    }
    *ticket = (int64_t)s->reqs.size() - 1;
    s->inbox.push_back(*ticket);
    s->cv_work.notify_one();
    return APSP_OK;
}

apsp_status apsp_server_poll(apsp_server *s, int64_t ticket, apsp_request_result *res, int32_t *done) {
    if (!s || !res || !done) return APSP_E_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    if (ticket < 0 || ticket >= (int64_t)s->reqs.size()) return APSP_E_ARG;
    const apsp_server::Req &r = s->reqs[(size_t)ticket];
    *done = r.done ? 1 : 0;
    if (r.done) *res = r.res;
    return APSP_OK;
}

apsp_status apsp_server_wait(apsp_server *s, int64_t ticket, double timeout_s, apsp_request_result *res) {
    if (!s || !res) return APSP_E_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    if (ticket < 0 || ticket >= (int64_t)s->reqs.size()) return APSP_E_ARG;
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(std::max(0.0, timeout_s));
    while (!s->reqs[(size_t)ticket].done)
        if (s->cv_done.wait_until(lock, until) == std::cv_status::timeout && !s->reqs[(size_t)ticket].done)
            return APSP_E_BUSY;
    *res = s->reqs[(size_t)ticket].res;
    return APSP_OK;
}

double apsp_server_clock(apsp_server *s) { return s ? s->clk.now() : -1.0; }

apsp_status apsp_server_destroy(apsp_server *s) {
    if (!s) return APSP_E_ARG;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    apsp_batch_destroy(s->b);
    cudaFreeHost(s->qbuf);
    delete s;
    return APSP_OK;
}

apsp_status apsp_serve(apsp_graph *const *graphs, int32_t n_graphs, const apsp_request *reqs, int32_t count,
                       const apsp_serve_config *cfg, apsp_request_result *results) {
    if (!graphs || n_graphs <= 0 || count < 0 || (count > 0 && (!reqs || !results)) || !cfg) return APSP_E_ARG;
    for (int q = 0; q < count; ++q) {
        const apsp_request &r = reqs[q];
        if (r.item.graph < 0 || r.item.graph >= n_graphs || r.item.op < 0 || r.item.op > APSP_BATCH_QUERY) return APSP_E_ARG;
        if (!(r.arrival_s >= 0) || (q > 0 && r.arrival_s < reqs[q - 1].arrival_s)) return APSP_E_ARG;
    }
    apsp_server *s = nullptr;
    apsp_status st = apsp_server_create(&s, graphs, n_graphs, cfg);
    if (st != APSP_OK) return st;
    std::vector<int64_t> tickets((size_t)count, -1);
    for (int q = 0; q < count; ++q) {
        // submit at the arrival time (sleep through long gaps, then spin)
        while (true) {
            const double gap = reqs[q].arrival_s - s->clk.now();
            if (gap <= 0) break;
            if (gap > 2e-4) std::this_thread::sleep_for(std::chrono::duration<double>(gap - 1e-4));
        }
        if ((st = apsp_server_submit(s, &reqs[q].item, &tickets[(size_t)q])) != APSP_OK) break;
    }
    for (int q = 0; q < count && st == APSP_OK; ++q) {
        while (apsp_server_wait(s, tickets[(size_t)q], 3600.0, &results[q]) == APSP_E_BUSY) {
        }
    }
    apsp_server_destroy(s);
    return st;
}

}  // extern "C"
