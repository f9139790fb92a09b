// Host-side launch sequences for each update type.  Instantiated for int32
// and float in kern_i32.cu / kern_f32.cu; graph.cu calls them through the
// declarations in launch.h.
#pragma once

#include <mutex>

#include "kernels.cuh"
#include "launch.h"

namespace apsp {

template <typename F> static inline cudaError_t launch(const LaunchCtx &c, const char *name, F &&f) {
    c.hook.begin(name);
    f();
    c.hook.end(name);
    return cudaGetLastError();
}

// Launch with programmatic stream serialization (the kernel begins with
// pdl_enter()): its CTAs may be scheduled while the previous kernel in the
// stream drains, which hides most of the launch gap between the short
// kernels of an update.  Returns the launch's own status.
template <typename... KArgs, typename... Args>
static inline cudaError_t pdl(cudaStream_t s, dim3 grid, dim3 block, size_t smem, void (*k)(KArgs...), Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// As launch(), for a callable that returns the launch status.
template <typename F> static inline cudaError_t launch_s(const LaunchCtx &c, const char *name, F &&f) {
    c.hook.begin(name);
    const cudaError_t e = f();
    c.hook.end(name);
    const cudaError_t last = cudaGetLastError();
    return e != cudaSuccess ? e : last;
}

static inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

template <typename T> cudaError_t run_fill(const LaunchCtx &c, T *p, T v, int64_t n) {
    int g = (int)std::min<int64_t>(cdiv(n, 256), (int64_t)c.num_sms * 8);
    if (g < 1) g = 1;
    return launch(c, "fill", [&] { k_fill<T><<<g, 256, 0, c.stream>>>(p, v, n); });
}

template <typename T> cudaError_t run_sanitize(const LaunchCtx &c, T *M, int64_t ld, int n, int check_sym, Ctl *ctl) {
    int g = std::max(1, (int)std::min<int64_t>(cdiv((int64_t)n * n, 256), (int64_t)c.num_sms * 8));
    return launch(c, "sanitize", [&] { k_sanitize<T><<<g, 256, 0, c.stream>>>(M, ld, n, check_sym, ctl); });
}

template <typename T> cudaError_t run_transpose(const LaunchCtx &c, const Dev<T> &d) {
    if (!d.DT) return cudaSuccess;
    int tiles = d.span / 32;
    int g = std::max(1, std::min(tiles * tiles, c.num_sms * 16));
    return launch(c, "transpose", [&] { k_transpose<T><<<g, dim3(32, 8), 0, c.stream>>>(d.D, d.DT, d.ld, d.span); });
}

// Cold solver: D = W, then nb rounds of the three phases, then DT = D^T.
template <typename T> cudaError_t run_fw(const LaunchCtx &c, const Dev<T> &d) {
    const int nb = cdiv(d.span, FW_B);
    cudaError_t e = cudaMemcpyAsync(d.D, d.W, (size_t)nb * FW_B * d.ld * sizeof(T), cudaMemcpyDeviceToDevice, c.stream);
    if (e != cudaSuccess) return e;
    for (int kb = 0; kb < nb; ++kb) {
        if ((e = launch(c, "fw_phase1", [&] { k_fw_p1<T><<<1, FW_THREADS, 0, c.stream>>>(d.D, d.ld, kb); })) != cudaSuccess) return e;
        if (nb == 1) break;
        if ((e = launch(c, "fw_phase2", [&] { k_fw_p2<T><<<2 * (nb - 1), FW_THREADS, 0, c.stream>>>(d.D, d.ld, kb, nb); })) != cudaSuccess) return e;
        if ((e = launch(c, "fw_phase3", [&] { k_fw_p3<T><<<(nb - 1) * (nb - 1), FW_THREADS, 0, c.stream>>>(d.D, d.ld, kb, nb); })) != cudaSuccess) return e;
    }
    return run_transpose<T>(c, d);
}

template <typename T>
cudaError_t run_insert(const LaunchCtx &c, const Dev<T> &d, const T *in_raw, const T *out_raw, int cap, int p, T *fetch) {
    cudaError_t e;
    if ((e = launch_s(c, "insert_prep", [&] { return pdl(c.stream, cdiv(d.span, 256), 256, 0, k_insert_prep<T>, d, in_raw, out_raw, cap, p, 1, fetch); })) != cudaSuccess) return e;
    if ((e = launch_s(c, "insert_cand", [&] { return pdl(c.stream, 1, INS_CAND_THREADS, 0, k_insert_cand<T>, d, p); })) != cudaSuccess) return e;
    // exactly one wave (never a partial second one): the resident CTAs split
    // into column bands x row ranges
    const int bands = cdiv(d.span, INS_CB);
    const int ranges = std::max(1, std::min(cdiv(d.span, 16), c.insred_per_sm * c.num_sms / bands));
    const int rows_per = cdiv(d.span, ranges);
    dim3 g(bands, cdiv(d.span, rows_per));
    if ((e = launch_s(c, "insert_reduce", [&] { return pdl(c.stream, g, 256, 0, k_insert_reduce<T>, d, rows_per); })) != cudaSuccess) return e;
    int gr = c.relax_grid;
    size_t sm = (size_t)d.span * sizeof(int32_t);
    const int nranges = cdiv(d.span, rows_per);
    return launch_s(c, "insert_relax", [&] { return pdl(c.stream, gr, 256, sm, k_insert_relax<T>, d, p, nranges, rows_per); });
}

template <typename T> cudaError_t run_decrease(const LaunchCtx &c, const Dev<T> &d, int u, int v, T w) {
    cudaError_t e;
    if ((e = launch_s(c, "decrease_prepass", [&] { return pdl(c.stream, cdiv(d.span, 256), 256, 0, k_dec_prepass<T>, d, u, v, w); })) != cudaSuccess) return e;
    return launch_s(c, "decrease_sweep", [&] { return pdl(c.stream, c.num_sms * 2, 256, 0, k_dec_sweep<T>, d, w); });
}

template <typename T> static size_t detect_smem(const Dev<T> &d, bool two) {
    return (size_t)d.span * sizeof(T) * (two ? 2 : 1);
}

// Detection: the streaming scan over the candidate rows (with exact counts of
// the batches it flags), then the reservation and the writes of those units.
template <typename T, bool TWO>
static cudaError_t run_detect_t(const LaunchCtx &c, const Dev<T> &d, int kind, int a, T w_old, T w_new,
                                const RepairCfg &cfg, const char *name) {
    cudaError_t e;
    const int scan_grid = TWO ? c.detect2_grid : c.detect_grid;
    const int mode = cfg.list_mode;
    if ((e = launch_s(c, name, [&] { return pdl(c.stream, scan_grid, 256, detect_smem(d, TWO), k_det_scan<T, TWO>, d, kind, a, w_old); })) != cudaSuccess) return e;
    if (mode == 1 &&
        (e = launch_s(c, "detect_recount", [&] { return pdl(c.stream, c.detunit_grid, 256, 0, k_det_recount<T, TWO>, d, kind, a, w_old); })) != cudaSuccess)
        return e;
    if (mode == 2 &&
        (e = launch_s(c, "detect_alg12", [&] {
             return pdl(c.stream, c.pw_grid, PW_WARPS * 32, pw_smem_bytes<T>(), k_det_alg12<T, TWO>, d, kind, a, w_old, cfg.umask);
         })) != cudaSuccess)
        return e;
    if ((e = launch_s(c, "detect_alloc", [&] { return pdl(c.stream, c.detalloc_grid, 256, 0, k_det_alloc<T>, d); })) != cudaSuccess) return e;
    if (mode == 1)
        return launch_s(c, "detect_write", [&] { return pdl(c.stream, c.detunit_grid, 256, 0, k_det_write<T, TWO, 1>, d, kind, a, w_old, w_new, (const uint32_t *)nullptr); });
    if (mode == 2)
        return launch_s(c, "detect_write", [&] { return pdl(c.stream, c.detunit_grid, 256, 0, k_det_write<T, TWO, 2>, d, kind, a, w_old, w_new, (const uint32_t *)cfg.umask); });
    return launch_s(c, "detect_write", [&] { return pdl(c.stream, c.detunit_grid, 256, 0, k_det_write<T, TWO, 0>, d, kind, a, w_old, w_new, (const uint32_t *)nullptr); });
}

template <typename T>
static cudaError_t run_detect(const LaunchCtx &c, const Dev<T> &d, int kind, int a, T w_old, T w_new,
                              const RepairCfg &cfg, const char *name) {
    if (d.undirected && kind == 1) return run_detect_t<T, true>(c, d, kind, a, w_old, w_new, cfg, name);
    return run_detect_t<T, false>(c, d, kind, a, w_old, w_new, cfg, name);
}

// Cooperative grids of different graphs (streams) must not be resident at
// the same time: each needs all its CTAs on the device at once, so two of
// them sharing the SMs could each wait for the other's.  Every cooperative
// launch of the process waits for the previous one (an event chain on the
// device; other kernels stay concurrent).
struct CoopChain {
    std::mutex mu;
    cudaEvent_t last[64] = {};
    cudaStream_t last_stream[64] = {};   // stream order already serialises work on the same stream
};
inline CoopChain &coop_chain() {
    static CoopChain c;
    return c;
}

template <typename F> static cudaError_t coop_launch(cudaStream_t stream, F &&launch_fn) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    CoopChain &cc = coop_chain();
    std::lock_guard<std::mutex> lock(cc.mu);
    if (!cc.last[dev]) {
        if ((e = cudaEventCreateWithFlags(&cc.last[dev], cudaEventDisableTiming)) != cudaSuccess) return e;
    } else if (cc.last_stream[dev] != stream && (e = cudaStreamWaitEvent(stream, cc.last[dev], 0)) != cudaSuccess) {
        return e;
    }
    if ((e = launch_fn()) != cudaSuccess) return e;
    cc.last_stream[dev] = stream;
    return cudaEventRecord(cc.last[dev], stream);
}

// The repair: the first re-relaxation pass (k_repair_p1, a plain launch that
// returns at once unless the device-side decision is warm), then the cooperative
// k_repair_main, which makes the same decision and runs either the later
// passes or the cold Floyd-Warshall.
template <typename T> cudaError_t run_repair(const LaunchCtx &c, const Dev<T> &d, const RepairCfg &cfg) {
    cudaError_t e = launch_s(c, "repair_p1", [&] { return pdl(c.stream, c.p1_grid, 256, 0, k_repair_p1<T>, d, cfg); });
    if (e != cudaSuccess) return e;
    Dev<T> dd = d;
    RepairCfg cc = cfg;
    void *args[] = {(void *)&dd, (void *)&cc};
    cudaError_t le = cudaSuccess;
    e = launch(c, "repair_main", [&] {
        le = coop_launch(c.stream, [&] {
            return cudaLaunchCooperativeKernel((void *)k_repair_main<T>, dim3(c.repair_grid), dim3(256), args,
                                               c.repair_smem, c.stream);
        });
    });
    return le != cudaSuccess ? le : e;
}

// Optional: Algorithm 12's need_update_list measured after the repair.
template <typename T> static cudaError_t run_grown(const LaunchCtx &c, const Dev<T> &d, int kind, T w_old, const RepairCfg &cfg) {
    if (!cfg.grown_flag) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(cfg.grown_flag, 0, (size_t)d.ld * sizeof(int32_t), c.stream);
    if (e != cudaSuccess) return e;
    const int grid = 2 * c.num_sms;
    if (d.undirected && kind == 1)
        return launch_s(c, "grown_count", [&] { return pdl(c.stream, grid, 256, 0, k_grown_count<T, true>, d, kind, w_old, cfg.grown_flag); });
    return launch_s(c, "grown_count", [&] { return pdl(c.stream, grid, 256, 0, k_grown_count<T, false>, d, kind, w_old, cfg.grown_flag); });
}

template <typename T> cudaError_t run_remove(const LaunchCtx &c, const Dev<T> &d, int k, const RepairCfg &cfg) {
    cudaError_t e;
    // the detection scan also stages the removed node's row and column (x, y)
    if ((e = run_detect<T>(c, d, 0, k, (T)0, (T)0, cfg, "detect_remove")) != cudaSuccess) return e;
    if ((e = run_repair<T>(c, d, cfg)) != cudaSuccess) return e;
    return run_grown<T>(c, d, 0, (T)0, cfg);
}

template <typename T>
cudaError_t run_increase(const LaunchCtx &c, const Dev<T> &d, int u, int v, T w_old, T w_new, const RepairCfg &cfg) {
    cudaError_t e;
    if ((e = launch_s(c, "increase_prepass", [&] { return pdl(c.stream, cdiv(d.span, 256), 256, 0, k_inc_prepass<T>, d, u, v, w_old, w_new); })) != cudaSuccess) return e;
    if ((e = run_detect<T>(c, d, 1, u, w_old, w_new, cfg, "detect_increase")) != cudaSuccess) return e;
    if ((e = run_repair<T>(c, d, cfg)) != cudaSuccess) return e;
    return run_grown<T>(c, d, 1, w_old, cfg);
}

template <typename F> static cudaError_t allow_max_smem(F *kernel);

// Graph: clear the control block -> prepass (sets the branch) -> IF tight:
// scan -> reservation -> writes -> first pass -> cooperative repair.
template <typename T, bool TWO>
static cudaError_t build_increase_graph(const LaunchCtx &c, const Dev<T> &d, IncGraph *ig, size_t ctl_bytes) {
    cudaError_t e;
    if ((e = allow_max_smem(k_det_scan_g<T, TWO>)) != cudaSuccess) return e;
    if ((e = allow_max_smem(k_repair_main_g<T>)) != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_repair_main_g<T>, 256, c.repair_smem)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid_main = std::min(c.repair_grid, per_sm * c.num_sms);
    cudaGraph_t g = nullptr;
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return e;
    auto fail = [&](cudaError_t x) {
        cudaGraphDestroy(g);
        return x;
    };
    cudaGraphNode_t clear = nullptr, pre = nullptr, cond = nullptr;
    cudaMemsetParams mp = {};
    mp.dst = (void *)d.ctl;
    mp.value = 0;
    mp.elementSize = 1;
    mp.width = ctl_bytes;
    mp.height = 1;
    if ((e = cudaGraphAddMemsetNode(&clear, g, nullptr, 0, &mp)) != cudaSuccess) return fail(e);
    cudaGraphConditionalHandle branch = 0;
    if ((e = cudaGraphConditionalHandleCreate(&branch, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess) return fail(e);
    Dev<T> dd = d;
    UpdArgs<T> *ua = (UpdArgs<T> *)ig->args;
    int u = 0, v = 0;
    T wo = (T)0, wn = (T)0;
    RepairCfg cf{};
    void *pp[] = {&dd, &u, &v, &wo, &wn, &cf, &ua, &branch};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)k_inc_prepass_g<T>;
    kp.gridDim = dim3(cdiv(d.span, 256));
    kp.blockDim = dim3(256);
    kp.kernelParams = pp;
    if ((e = cudaGraphAddKernelNode(&pre, g, &clear, 1, &kp)) != cudaSuccess) return fail(e);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = branch;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    if ((e = cudaGraphAddNode(&cond, g, &pre, nullptr, 1, &cp)) != cudaSuccess) return fail(e);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaGraphNode_t prev = nullptr, node = nullptr;
    void *pa[] = {&dd};
    void *pb[] = {&dd, &ua};
    auto add = [&](void *func, int grid, size_t smem, void **params) {
        cudaKernelNodeParams q = {};
        q.func = func;
        q.gridDim = dim3(grid);
        q.blockDim = dim3(256);
        q.sharedMemBytes = (unsigned)smem;
        q.kernelParams = params;
        cudaError_t x = cudaGraphAddKernelNode(&node, body, prev ? &prev : nullptr, prev ? 1 : 0, &q);
        if (x == cudaSuccess) prev = node;
        return x;
    };
    if ((e = add((void *)k_det_scan_g<T, TWO>, TWO ? c.detect2_grid : c.detect_grid, detect_smem(d, TWO), pb)) != cudaSuccess)
        return fail(e);
    if ((e = add((void *)k_det_alloc<T>, c.detalloc_grid, 0, pa)) != cudaSuccess) return fail(e);
    if ((e = add((void *)k_det_write_g<T, TWO>, c.detunit_grid, 0, pb)) != cudaSuccess) return fail(e);
    if ((e = add((void *)k_repair_p1_g<T>, c.p1_grid, 0, pb)) != cudaSuccess) return fail(e);
    if ((e = add((void *)k_repair_main_g<T>, grid_main, c.repair_smem, pb)) != cudaSuccess) return fail(e);
    cudaLaunchAttributeValue coop = {};
    coop.cooperative = 1;
    if ((e = cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributeCooperative, &coop)) != cudaSuccess) return fail(e);
    cudaGraphExec_t ex = nullptr;
    if ((e = cudaGraphInstantiate(&ex, g, 0)) != cudaSuccess) return fail(e);
    ig->graph = g;
    ig->exec = ex;
    ig->pre = pre;
    ig->branch = branch;
    ig->span = d.span;
    ig->grid_main = grid_main;
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_increase_graph(const LaunchCtx &c, const Dev<T> &d, IncGraph *ig, size_t ctl_bytes, int u, int v,
                                  T w_old, T w_new, const RepairCfg &cfg) {
    cudaError_t e;
    if (!ig->exec || ig->span != d.span) {
        destroy_increase_graph(ig);
        e = d.undirected ? build_increase_graph<T, true>(c, d, ig, ctl_bytes) : build_increase_graph<T, false>(c, d, ig, ctl_bytes);
        if (e != cudaSuccess) return e;
    }
    Dev<T> dd = d;
    UpdArgs<T> *ua = (UpdArgs<T> *)ig->args;
    RepairCfg cf = cfg;
    cudaGraphConditionalHandle branch = ig->branch;
    void *pp[] = {&dd, &u, &v, &w_old, &w_new, &cf, &ua, &branch};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)k_inc_prepass_g<T>;
    kp.gridDim = dim3(cdiv(d.span, 256));
    kp.blockDim = dim3(256);
    kp.kernelParams = pp;
    if ((e = cudaGraphExecKernelNodeSetParams(ig->exec, ig->pre, &kp)) != cudaSuccess) return e;
    // the graph holds a cooperative kernel: ordered against other streams'
    // cooperative work like a cooperative launch
    // counted as one launch here (the prepass); the body's kernels are added
    // from the device counter when the count is read
    return launch_s(c, "increase_graph", [&] { return coop_launch(c.stream, [&] { return cudaGraphLaunch(ig->exec, c.stream); }); });
}

// The dynamic shared memory limit is a per-function setting shared by every
// graph of the process, so it is raised once to the device's maximum (graphs
// of different sizes then never lower it under each other); occupancy is
// computed from each launch's actual bytes.
template <typename F> static cudaError_t allow_max_smem(F *kernel) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess)   // the opt-in limit covers static and dynamic shared memory together
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
}

// Occupancy-derived launch shapes for a graph of leading dimension ld.
template <typename T> cudaError_t setup_shapes(LaunchCtx &c, int64_t ld, int undirected) {
    cudaError_t e;
    size_t row = (size_t)ld * sizeof(T);
    size_t fw = sizeof(FwSmem<T>) > sizeof(FwDiagSmem<T>) ? sizeof(FwSmem<T>) : sizeof(FwDiagSmem<T>);
    c.repair_smem = std::max<size_t>(fw, 32 * 33 * sizeof(T));
    if ((e = allow_max_smem(k_repair_main<T>)) != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_repair_main<T>, 256, c.repair_smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    c.repair_grid = per_sm * c.num_sms;
    int p1_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p1_sm, k_repair_p1<T>, 256, 0)) != cudaSuccess) return e;
    if (p1_sm < 1) return cudaErrorInvalidConfiguration;
    c.p1_grid = p1_sm * c.num_sms;
    if ((e = allow_max_smem(k_det_scan<T, false>)) != cudaSuccess) return e;
    int det_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&det_sm, k_det_scan<T, false>, 256, row)) != cudaSuccess) return e;
    c.detect_grid = std::max(1, det_sm) * c.num_sms;
    if ((e = allow_max_smem(k_det_scan<T, true>)) != cudaSuccess) return e;
    int det2_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&det2_sm, k_det_scan<T, true>, 256, 2 * row)) != cudaSuccess) return e;
    c.detect2_grid = std::max(1, det2_sm) * c.num_sms;
    c.detunit_grid = 4 * c.num_sms;
    c.detalloc_grid = (int)((ld + 255) / 256);   // a lane per row: 256 rows a CTA
    if ((e = allow_max_smem(k_path_warp<T>)) != cudaSuccess) return e;
    if ((e = allow_max_smem(k_next_hop<T>)) != cudaSuccess) return e;
    if ((e = allow_max_smem(k_det_alg12<T, false>)) != cudaSuccess) return e;
    if ((e = allow_max_smem(k_det_alg12<T, true>)) != cudaSuccess) return e;
    int pw_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pw_sm, k_path_warp<T>, PW_WARPS * 32, pw_smem_bytes<T>())) !=
        cudaSuccess)
        return e;
    c.pw_grid = std::max(1, pw_sm) * c.num_sms;
    int ir_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ir_sm, k_insert_reduce<T>, 256, 0)) != cudaSuccess) return e;
    c.insred_per_sm = std::max(1, ir_sm);
    size_t rel = (size_t)ld * sizeof(int32_t);
    if ((e = allow_max_smem(k_insert_relax<T>)) != cudaSuccess) return e;
    int rel_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rel_sm, k_insert_relax<T>, 256, rel)) != cudaSuccess) return e;
    c.relax_grid = std::max(1, rel_sm) * c.num_sms;
    return cudaSuccess;
}

// Path queries (paths.cuh), tier 0: a warp per query over every query;
// tier 1: a CTA per query over those tier 0 deferred; tier 2: PQ_WIDE_GRID
// CTAs over those tier 1 deferred.
template <typename T> cudaError_t run_path_query(const LaunchCtx &c, const Dev<T> &d, const PathQuery &q, int tier) {
    if (q.count <= 0) return cudaSuccess;
    if (tier == 2)
        return launch(c, "path_query_wide",
                      [&] { k_path_query<T, true><<<PQ_WIDE_GRID, PQ_THREADS, 0, c.stream>>>(d, q); });
    if (tier == 1) {
        const int grid = std::min(q.count, 4 * c.num_sms);
        return launch(c, "path_query_block",
                      [&] { k_path_query<T, false><<<grid, PQ_THREADS, pq_smem_bytes<T>(), c.stream>>>(d, q); });
    }
    const int grid = std::max(1, std::min(cdiv(q.count, PW_WARPS), c.pw_grid));
    return launch(c, "path_query",
                  [&] { k_path_warp<T><<<grid, PW_WARPS * 32, pw_smem_bytes<T>(), c.stream>>>(d, q); });
}

// One persistent launch for a whole batch of graphs (batch.cuh).
template <typename T> cudaError_t run_batch(cudaStream_t s, BatchHeader *hdr, int grid, size_t smem, int nt) {
    if (nt == 128) k_batch<T, 128><<<grid, 128, smem, s>>>(hdr);
    else if (nt == 512) k_batch<T, 512><<<grid, 512, smem, s>>>(hdr);
    else k_batch<T, 256><<<grid, 256, smem, s>>>(hdr);
    return cudaGetLastError();
}

template <typename T> cudaError_t batch_occupancy(size_t smem, int nt, int *per_sm) {
    cudaError_t e;
    if (nt == 128) {
        if ((e = allow_max_smem(k_batch<T, 128>)) != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch<T, 128>, 128, smem);
    }
    if (nt == 512) {
        if ((e = allow_max_smem(k_batch<T, 512>)) != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch<T, 512>, 512, smem);
    }
    if ((e = allow_max_smem(k_batch<T, 256>)) != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch<T, 256>, 256, smem);
}

// ---- minimax (bottleneck) distances: minimax.cuh --------------------------

template <typename T> cudaError_t run_mm_fw(const LaunchCtx &c, const Dev<T> &d) {
    using M = MinMax<T>;
    const int nb = cdiv(d.span, FW_B);
    cudaError_t e = cudaMemcpyAsync(d.D, d.W, (size_t)nb * FW_B * d.ld * sizeof(T), cudaMemcpyDeviceToDevice, c.stream);
    if (e != cudaSuccess) return e;
    for (int kb = 0; kb < nb; ++kb) {
        if ((e = launch(c, "mm_fw_phase1", [&] { k_fw_p1<T, M><<<1, FW_THREADS, 0, c.stream>>>(d.D, d.ld, kb); })) != cudaSuccess) return e;
        if (nb == 1) break;
        if ((e = launch(c, "mm_fw_phase2", [&] { k_fw_p2<T, M><<<2 * (nb - 1), FW_THREADS, 0, c.stream>>>(d.D, d.ld, kb, nb); })) != cudaSuccess) return e;
        if ((e = launch(c, "mm_fw_phase3", [&] { k_fw_p3<T, M><<<(nb - 1) * (nb - 1), FW_THREADS, 0, c.stream>>>(d.D, d.ld, kb, nb); })) != cudaSuccess) return e;
    }
    return run_transpose<T>(c, d);
}

template <typename T>
cudaError_t run_mm_insert(const LaunchCtx &c, const Dev<T> &d, const T *in_raw, const T *out_raw, int cap, int p, T *fetch) {
    cudaError_t e;
    if ((e = launch(c, "insert_prep", [&] { k_insert_prep<T><<<cdiv(d.span, 256), 256, 0, c.stream>>>(d, in_raw, out_raw, cap, p, 0, fetch); })) != cudaSuccess) return e;
    const int bands = cdiv(d.span, MM_CB);
    int ranges = std::max(1, (3 * c.num_sms + bands - 1) / bands);
    ranges = std::min(ranges, std::max(1, cdiv(d.span, 8)));
    const int rows_per = cdiv(d.span, ranges);
    const dim3 g(bands, cdiv(d.span, rows_per));
    if ((e = launch(c, "mm_insert_reduce", [&] { k_mm_insert_reduce<T><<<g, 256, 0, c.stream>>>(d, rows_per); })) != cudaSuccess) return e;
    if ((e = launch(c, "mm_insert_relax", [&] { k_mm_insert_relax<T><<<std::min(d.span, 4 * c.num_sms), 256, 0, c.stream>>>(d, p); })) != cudaSuccess) return e;
    return launch(c, "mm_insert_finish", [&] { k_mm_insert_finish<T><<<cdiv(d.span, 256), 256, 0, c.stream>>>(d, p); });
}

template <typename T> cudaError_t run_mm_decrease(const LaunchCtx &c, const Dev<T> &d, int u, int v, T w) {
    cudaError_t e;
    const int two = d.undirected ? 1 : 0;
    if ((e = launch(c, "mm_legs", [&] { k_mm_legs<T><<<cdiv(d.span, 256), 256, 0, c.stream>>>(d, u, v, two, 1, w); })) != cudaSuccess) return e;
    const int g = std::max(1, std::min(cdiv(d.span, 8), 4 * c.num_sms));
    if (two) return launch(c, "mm_decrease", [&] { k_mm_decrease<T, true><<<g, 256, 0, c.stream>>>(d, u, v, w); });
    return launch(c, "mm_decrease", [&] { k_mm_decrease<T, false><<<g, 256, 0, c.stream>>>(d, u, v, w); });
}

// kind 0: removal of node a (legs through a, list, then the tombstone);
// kind 1: increase of edge (a, b) from w_old to w_new (W updated first).
template <typename T>
cudaError_t run_mm_detect(const LaunchCtx &c, const Dev<T> &d, uint32_t *mask, int words, int kind, int a, int b,
                          T w_old, T w_new) {
    cudaError_t e;
    const bool two = kind == 1 && d.undirected;
    const int lb = kind == 0 ? a : b;
    if ((e = launch(c, "mm_legs", [&] {
             k_mm_legs<T><<<cdiv(d.span, 256), 256, 0, c.stream>>>(d, a, lb, two ? 1 : 0, kind == 1 ? 1 : 0, w_new);
         })) != cudaSuccess)
        return e;
    const int g = std::max(1, std::min(cdiv(d.span, 8), 4 * c.num_sms));
    if (two)
        e = launch(c, "mm_detect", [&] { k_mm_detect<T, true><<<g, 256, 0, c.stream>>>(d, mask, words, kind, a, w_old, w_new); });
    else
        e = launch(c, "mm_detect", [&] { k_mm_detect<T, false><<<g, 256, 0, c.stream>>>(d, mask, words, kind, a, w_old, w_new); });
    if (e != cudaSuccess || kind != 0) return e;
    return launch(c, "mm_tomb", [&] { k_mm_tomb<T><<<cdiv(d.span, 256), 256, 0, c.stream>>>(d, a); });
}

template <typename T>
cudaError_t run_mm_pass(const LaunchCtx &c, const Dev<T> &d, const uint32_t *mask, int words, int pass) {
    const int g = 4 * c.num_sms;
    return launch(c, "mm_pass", [&] { k_mm_pass<T><<<g, 256, 0, c.stream>>>(d, mask, words, pass); });
}

template <typename T>
cudaError_t run_next_hop(const LaunchCtx &c, const Dev<T> &d, const int32_t *rows, int nrows, int32_t *out,
                         int64_t ld_out) {
    const int g = std::max(1, std::min(nrows, 4 * c.num_sms));
    return launch(c, "next_hop", [&] {
        k_next_hop<T><<<g, 256, (size_t)d.span * sizeof(int32_t), c.stream>>>(d, rows, nrows, out, ld_out);
    });
}

#define APSP_INSTANTIATE(T)                                                                                   \
    template cudaError_t run_fill<T>(const LaunchCtx &, T *, T, int64_t);                                     \
    template cudaError_t run_sanitize<T>(const LaunchCtx &, T *, int64_t, int, int, Ctl *);                   \
    template cudaError_t run_transpose<T>(const LaunchCtx &, const Dev<T> &);                                 \
    template cudaError_t run_fw<T>(const LaunchCtx &, const Dev<T> &);                                        \
    template cudaError_t run_insert<T>(const LaunchCtx &, const Dev<T> &, const T *, const T *, int, int, T *); \
    template cudaError_t run_decrease<T>(const LaunchCtx &, const Dev<T> &, int, int, T);                     \
    template cudaError_t run_remove<T>(const LaunchCtx &, const Dev<T> &, int, const RepairCfg &);            \
    template cudaError_t run_increase<T>(const LaunchCtx &, const Dev<T> &, int, int, T, T, const RepairCfg &); \
    template cudaError_t run_repair<T>(const LaunchCtx &, const Dev<T> &, const RepairCfg &);                 \
    template cudaError_t run_path_query<T>(const LaunchCtx &, const Dev<T> &, const PathQuery &, int);        \
    template cudaError_t setup_shapes<T>(LaunchCtx &, int64_t, int);                                          \
    template cudaError_t run_batch<T>(cudaStream_t, BatchHeader *, int, size_t, int);                         \
    template cudaError_t batch_occupancy<T>(size_t, int, int *);                                             \
    template cudaError_t run_mm_fw<T>(const LaunchCtx &, const Dev<T> &);                                     \
    template cudaError_t run_mm_insert<T>(const LaunchCtx &, const Dev<T> &, const T *, const T *, int, int, T *); \
    template cudaError_t run_mm_decrease<T>(const LaunchCtx &, const Dev<T> &, int, int, T);                  \
    template cudaError_t run_mm_detect<T>(const LaunchCtx &, const Dev<T> &, uint32_t *, int, int, int, int, T, T); \
    template cudaError_t run_mm_pass<T>(const LaunchCtx &, const Dev<T> &, const uint32_t *, int, int);          \
    template cudaError_t run_next_hop<T>(const LaunchCtx &, const Dev<T> &, const int32_t *, int, int32_t *, int64_t); \
    template cudaError_t launch_increase_graph<T>(const LaunchCtx &, const Dev<T> &, IncGraph *, size_t, int, int, T, T, \
                                                  const RepairCfg &);

}  // namespace apsp
