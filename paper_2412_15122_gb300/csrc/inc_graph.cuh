// An edge increase as one CUDA graph with a device-side branch.
//
// Most increases in a random stream hit an edge that lies on no shortest path
// (w_old > D[u][v]); D then stays as it is and only W changes.  The stream
// form still launches detection and both repair kernels, each returning at
// once.  In the graph form the prepass sets a conditional handle
// (cudaGraphSetConditional) to whether the edge is tight, and the detection
// and repair kernels sit in the body of an IF node, so a non-tight increase
// runs the control-block clear and the prepass only.  The body's kernels read
// the update's arguments from a small device block the prepass writes, so the
// instantiated graph is reused: only the prepass node's parameters change per
// update.
#pragma once

#include "kernels.cuh"
#include "repair_p1.cuh"

namespace apsp {

template <typename T> struct UpdArgs {
    int32_t kind, a;
    T w_old, w_new;
    RepairCfg cfg;
    unsigned long long bodies;   // launches whose IF body ran (zeroed at allocation), for the launch count
};

constexpr int INC_GRAPH_BODY_KERNELS = 5;   // kernels in the IF body

template <typename T>
__global__ void k_inc_prepass_g(Dev<T> d, int u, int v, T w_old, T w_new, RepairCfg cfg, UpdArgs<T> *ua,
                                cudaGraphConditionalHandle branch) {
    pdl_enter();
    k_inc_prepass_body<T>(d, u, v, w_old, w_new);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ua->kind = 1;
        ua->a = u;
        ua->w_old = w_old;
        ua->w_new = w_new;
        ua->cfg = cfg;
        const bool tight_edge = MinPlus<T>::tight(w_old, d.D[(int64_t)u * d.ld + v]);
        if (tight_edge) ua->bodies += 1;   // graph launches on one stream run one after another
        cudaGraphSetConditional(branch, tight_edge ? 1u : 0u);
    }
}

template <typename T, bool TWO>
__global__ void __launch_bounds__(256, 4) k_det_scan_g(Dev<T> d, const UpdArgs<T> *ua) {
    pdl_enter();
    k_det_scan_body<T, TWO>(d, ua->kind, ua->a, ua->w_old);
}

template <typename T, bool TWO>
__global__ void __launch_bounds__(256, 4) k_det_write_g(Dev<T> d, const UpdArgs<T> *ua) {
    pdl_enter();
    k_det_write_body<T, TWO, 0>(d, ua->kind, ua->a, ua->w_old, ua->w_new, nullptr);
}

template <typename T>
__global__ void __launch_bounds__(256, 2) k_repair_p1_g(Dev<T> d, const UpdArgs<T> *ua) {
    pdl_enter();
    k_repair_p1_body<T>(d, ua->cfg);
}

template <typename T>
__global__ void __launch_bounds__(256, 2) k_repair_main_g(Dev<T> d, const UpdArgs<T> *ua) {
    const RepairCfg cfg = ua->cfg;
    repair_main_body<T>(d, cfg);
}

}  // namespace apsp
