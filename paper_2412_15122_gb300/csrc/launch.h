// Declarations of the per-update launch sequences (defined in launch.cuh,
// instantiated for int32 and float in kern_i32.cu / kern_f32.cu).
#pragma once

#include <algorithm>
#include <cuda_runtime.h>

#include "batch.cuh"
#include "kernels.cuh"
#include "paths.cuh"
#include "repair_p1.cuh"
#include "minimax.cuh"
#include "next_hop.cuh"
#include "inc_graph.cuh"

namespace apsp {

struct LaunchCtx {
    cudaStream_t stream = nullptr;
    Hook hook{nullptr, nullptr, nullptr};
    int num_sms = 1;
    int repair_grid = 1;
    size_t repair_smem = 0;
    int detect_grid = 1;
    int relax_grid = 1;
    int p1_grid = 1;
    int detect2_grid = 1;
    int detunit_grid = 1;
    int detalloc_grid = 1;
    int insred_per_sm = 1;
    int pw_grid = 1;
};

template <typename T> cudaError_t run_fill(const LaunchCtx &, T *, T, int64_t);
template <typename T> cudaError_t run_sanitize(const LaunchCtx &, T *, int64_t, int, int, Ctl *);
template <typename T> cudaError_t run_transpose(const LaunchCtx &, const Dev<T> &);
template <typename T> cudaError_t run_fw(const LaunchCtx &, const Dev<T> &);
template <typename T> cudaError_t run_insert(const LaunchCtx &, const Dev<T> &, const T *, const T *, int, int, T *);
template <typename T> cudaError_t run_decrease(const LaunchCtx &, const Dev<T> &, int, int, T);
template <typename T> cudaError_t run_remove(const LaunchCtx &, const Dev<T> &, int, const RepairCfg &);
template <typename T> cudaError_t run_increase(const LaunchCtx &, const Dev<T> &, int, int, T, T, const RepairCfg &);
template <typename T> cudaError_t run_repair(const LaunchCtx &, const Dev<T> &, const RepairCfg &);
template <typename T> cudaError_t run_path_query(const LaunchCtx &, const Dev<T> &, const PathQuery &, int);
template <typename T> cudaError_t setup_shapes(LaunchCtx &, int64_t, int);
template <typename T> cudaError_t run_batch(cudaStream_t, BatchHeader *, int, size_t, int);
template <typename T> cudaError_t batch_occupancy(size_t, int, int *);
// minimax (bottleneck) distances
template <typename T> cudaError_t run_mm_fw(const LaunchCtx &, const Dev<T> &);
template <typename T> cudaError_t run_mm_insert(const LaunchCtx &, const Dev<T> &, const T *, const T *, int, int, T *);
template <typename T> cudaError_t run_mm_decrease(const LaunchCtx &, const Dev<T> &, int, int, T);
template <typename T>
cudaError_t run_mm_detect(const LaunchCtx &, const Dev<T> &, uint32_t *, int, int, int, int, T, T);
template <typename T> cudaError_t run_mm_pass(const LaunchCtx &, const Dev<T> &, const uint32_t *, int, int);
template <typename T> cudaError_t run_next_hop(const LaunchCtx &, const Dev<T> &, const int32_t *, int, int32_t *, int64_t);

// An edge increase as one instantiated CUDA graph (inc_graph.cuh): built on
// first use and again when the graph's span changes; `args` is the device
// block (sizeof(UpdArgs<T>) bytes, owned by the caller) that the prepass fills.
struct IncGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t pre = nullptr;               // the prepass node: its parameters change per update
    cudaGraphConditionalHandle branch = 0;
    int span = -1;
    int grid_main = 0;                           // cooperative grid of the repair kernel in the graph
    void *args = nullptr;
};
inline void destroy_increase_graph(IncGraph *ig) {
    if (ig->exec) cudaGraphExecDestroy(ig->exec);
    if (ig->graph) cudaGraphDestroy(ig->graph);
    ig->exec = nullptr;
    ig->graph = nullptr;
    ig->pre = nullptr;
    ig->span = -1;
}

template <typename T>
cudaError_t launch_increase_graph(const LaunchCtx &, const Dev<T> &, IncGraph *, size_t ctl_bytes, int, int, T, T,
                                  const RepairCfg &);

}  // namespace apsp
