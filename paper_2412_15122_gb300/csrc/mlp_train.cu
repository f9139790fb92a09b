// Training and batched inference of the warm/cold cost model (network and
// parameter layout in mlp.cuh).  Stateless C entry points on host buffers:
// loss + gradient over a sample set, prediction, and mini-batch Adam
// training.
//
// Gradient kernel: one warp per sample; lane l owns hidden units l and l+32
// of both layers (their W1 rows, biases and W3 weights stay in registers).
// W2 is staged in shared memory with a padded row stride (65) so that both
// the forward (row access) and the backward (column access) reads are free
// of bank conflicts.  The CTA accumulates its samples' gradients in a shared
// copy of the trainable block (dW2 with column-per-lane atomics, the rest
// from per-lane registers at the end) and adds it once to the global
// gradient.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "apsp.h"
#include "mlp.cuh"

namespace {

using namespace apsp;
static_assert(MLP_NPARAM == APSP_MODEL_NPARAM, "parameter block size");
static_assert(MLP_NTRAIN == APSP_MODEL_NTRAIN, "trainable block size");

constexpr int GW = 8;            // warps per CTA of the gradient kernel
constexpr int W2S = MLP_H + 1;   // padded row stride of W2 in shared memory
// offsets inside the trainable block (gradient layout)
constexpr int T_W1 = MLP_OFF_W1 - MLP_OFF_TRAIN, T_B1 = MLP_OFF_B1 - MLP_OFF_TRAIN;
constexpr int T_W2 = MLP_OFF_W2 - MLP_OFF_TRAIN, T_B2 = MLP_OFF_B2 - MLP_OFF_TRAIN;
constexpr int T_W3 = MLP_OFF_W3 - MLP_OFF_TRAIN, T_B3 = MLP_OFF_B3 - MLP_OFF_TRAIN;

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Loss (sum of squared errors over present labels, times inv_n) and its
// gradient for samples idx[0..count) (idx == nullptr: samples 0..count).
__global__ void __launch_bounds__(GW * 32) k_mlp_grad(const float *__restrict__ P, const float *__restrict__ X,
                                                      const float *__restrict__ Y, const int *__restrict__ idx,
                                                      int count, float inv_n, float *__restrict__ G,
                                                      float *__restrict__ loss_acc) {
    __shared__ float sW2[MLP_H * W2S];
    __shared__ float sG[MLP_NTRAIN];
    __shared__ float sh1[GW][MLP_H], sdh2[GW][MLP_H];
    for (int t = threadIdx.x; t < MLP_H * MLP_H; t += blockDim.x) sW2[(t / MLP_H) * W2S + t % MLP_H] = P[MLP_OFF_W2 + t];
    for (int t = threadIdx.x; t < MLP_NTRAIN; t += blockDim.x) sG[t] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int ua = lane, ub = lane + 32;
    float mu[MLP_IN], isd[MLP_IN], w1a[MLP_IN], w1b[MLP_IN];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) {
        mu[i] = P[MLP_OFF_MU + i];
        isd[i] = 1.f / P[MLP_OFF_SD + i];
        w1a[i] = P[MLP_OFF_W1 + ua * MLP_IN + i];
        w1b[i] = P[MLP_OFF_W1 + ub * MLP_IN + i];
    }
    const float b1a = P[MLP_OFF_B1 + ua], b1b = P[MLP_OFF_B1 + ub];
    const float b2a = P[MLP_OFF_B2 + ua], b2b = P[MLP_OFF_B2 + ub];
    const float w3a0 = P[MLP_OFF_W3 + ua], w3b0 = P[MLP_OFF_W3 + ub];
    const float w3a1 = P[MLP_OFF_W3 + MLP_H + ua], w3b1 = P[MLP_OFF_W3 + MLP_H + ub];
    const float b30 = P[MLP_OFF_B3], b31 = P[MLP_OFF_B3 + 1];
    float gw1a[MLP_IN] = {}, gw1b[MLP_IN] = {};
    float gb1a = 0.f, gb1b = 0.f, gb2a = 0.f, gb2b = 0.f;
    float gw3a0 = 0.f, gw3b0 = 0.f, gw3a1 = 0.f, gw3b1 = 0.f, gb30 = 0.f, gb31 = 0.f, lacc = 0.f;
    for (int s = blockIdx.x * GW + w; s < count; s += gridDim.x * GW) {
        const int r = idx ? idx[s] : s;
        float x[MLP_IN];
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) x[i] = (X[(size_t)r * MLP_IN + i] - mu[i]) * isd[i];
        const float y0 = Y[(size_t)r * 2], y1 = Y[(size_t)r * 2 + 1];
        // forward
        float za = b1a, zb = b1b;
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) {
            za = fmaf(w1a[i], x[i], za);
            zb = fmaf(w1b[i], x[i], zb);
        }
        const float h1a = fmaxf(za, 0.f), h1b = fmaxf(zb, 0.f);
        sh1[w][ua] = h1a;
        sh1[w][ub] = h1b;
        __syncwarp();
        float z2a = b2a, z2b = b2b;
#pragma unroll 8
        for (int k = 0; k < MLP_H; ++k) {
            const float hk = sh1[w][k];
            z2a = fmaf(sW2[ua * W2S + k], hk, z2a);
            z2b = fmaf(sW2[ub * W2S + k], hk, z2b);
        }
        const float h2a = fmaxf(z2a, 0.f), h2b = fmaxf(z2b, 0.f);
        const float o0 = wsum(w3a0 * h2a + w3b0 * h2b) + b30;
        const float o1 = wsum(w3a1 * h2a + w3b1 * h2b) + b31;
        // loss and output gradient (a NaN label is missing)
        const float d0 = isnan(y0) ? 0.f : o0 - y0, d1 = isnan(y1) ? 0.f : o1 - y1;
        lacc += d0 * d0 + d1 * d1;
        const float g0 = 2.f * d0 * inv_n, g1 = 2.f * d1 * inv_n;
        gw3a0 = fmaf(g0, h2a, gw3a0);
        gw3b0 = fmaf(g0, h2b, gw3b0);
        gw3a1 = fmaf(g1, h2a, gw3a1);
        gw3b1 = fmaf(g1, h2b, gw3b1);
        gb30 += g0;
        gb31 += g1;
        // second hidden layer
        const float dh2a = z2a > 0.f ? fmaf(w3a0, g0, w3a1 * g1) : 0.f;
        const float dh2b = z2b > 0.f ? fmaf(w3b0, g0, w3b1 * g1) : 0.f;
        gb2a += dh2a;
        gb2b += dh2b;
        sdh2[w][ua] = dh2a;
        sdh2[w][ub] = dh2b;
        __syncwarp();
        // dW2[u][k] += dh2[u] h1[k]: lane takes columns k = lane, lane + 32
        float dh1a = 0.f, dh1b = 0.f;
        for (int u = 0; u < MLP_H; ++u) {
            const float du = sdh2[w][u];
            if (du == 0.f) continue;   // warp-uniform: inactive unit
            atomicAdd(&sG[T_W2 + u * MLP_H + ua], du * h1a);
            atomicAdd(&sG[T_W2 + u * MLP_H + ub], du * h1b);
            dh1a = fmaf(sW2[u * W2S + ua], du, dh1a);
            dh1b = fmaf(sW2[u * W2S + ub], du, dh1b);
        }
        // first hidden layer
        dh1a = za > 0.f ? dh1a : 0.f;
        dh1b = zb > 0.f ? dh1b : 0.f;
        gb1a += dh1a;
        gb1b += dh1b;
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) {
            gw1a[i] = fmaf(dh1a, x[i], gw1a[i]);
            gw1b[i] = fmaf(dh1b, x[i], gw1b[i]);
        }
        __syncwarp();   // sh1 / sdh2 are rewritten by the next sample
    }
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) {
        atomicAdd(&sG[T_W1 + ua * MLP_IN + i], gw1a[i]);
        atomicAdd(&sG[T_W1 + ub * MLP_IN + i], gw1b[i]);
    }
    atomicAdd(&sG[T_B1 + ua], gb1a);
    atomicAdd(&sG[T_B1 + ub], gb1b);
    atomicAdd(&sG[T_B2 + ua], gb2a);
    atomicAdd(&sG[T_B2 + ub], gb2b);
    atomicAdd(&sG[T_W3 + ua], gw3a0);
    atomicAdd(&sG[T_W3 + ub], gw3b0);
    atomicAdd(&sG[T_W3 + MLP_H + ua], gw3a1);
    atomicAdd(&sG[T_W3 + MLP_H + ub], gw3b1);
    if (lane == 0) {
        atomicAdd(&sG[T_B3], gb30);
        atomicAdd(&sG[T_B3 + 1], gb31);
        atomicAdd(loss_acc, lacc * inv_n);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < MLP_NTRAIN; t += blockDim.x)
        if (sG[t] != 0.f) atomicAdd(&G[t], sG[t]);
}

// Adam step on the trainable block; clears the gradient for the next batch.
__global__ void k_mlp_adam(float *P, float *G, float *M, float *V, float lr, float c1, float c2) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= MLP_NTRAIN) return;
    const float g = G[t];
    const float m = 0.9f * M[t] + 0.1f * g;
    const float v = 0.999f * V[t] + 0.001f * g * g;
    M[t] = m;
    V[t] = v;
    P[MLP_OFF_TRAIN + t] -= lr * (m * c1) / (sqrtf(v * c2) + 1e-8f);
    G[t] = 0.f;
}

// Outputs of n samples, one warp each.
__global__ void k_mlp_predict(const float *__restrict__ P, const float *__restrict__ X, int n, float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int ua = lane, ub = lane + 32;
    __shared__ float sh1[8][MLP_H];
    const int w = threadIdx.x >> 5;
    for (int s = blockIdx.x * 8 + w; s < n; s += gridDim.x * 8) {
        float za = P[MLP_OFF_B1 + ua], zb = P[MLP_OFF_B1 + ub];
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) {
            const float x = (X[(size_t)s * MLP_IN + i] - P[MLP_OFF_MU + i]) / P[MLP_OFF_SD + i];
            za = fmaf(P[MLP_OFF_W1 + ua * MLP_IN + i], x, za);
            zb = fmaf(P[MLP_OFF_W1 + ub * MLP_IN + i], x, zb);
        }
        sh1[w][ua] = fmaxf(za, 0.f);
        sh1[w][ub] = fmaxf(zb, 0.f);
        __syncwarp();
        float z2a = P[MLP_OFF_B2 + ua], z2b = P[MLP_OFF_B2 + ub];
        for (int k = 0; k < MLP_H; ++k) {
            z2a = fmaf(P[MLP_OFF_W2 + ua * MLP_H + k], sh1[w][k], z2a);
            z2b = fmaf(P[MLP_OFF_W2 + ub * MLP_H + k], sh1[w][k], z2b);
        }
        const float h2a = fmaxf(z2a, 0.f), h2b = fmaxf(z2b, 0.f);
        const float o0 = wsum(P[MLP_OFF_W3 + ua] * h2a + P[MLP_OFF_W3 + ub] * h2b) + P[MLP_OFF_B3];
        const float o1 = wsum(P[MLP_OFF_W3 + MLP_H + ua] * h2a + P[MLP_OFF_W3 + MLP_H + ub] * h2b) + P[MLP_OFF_B3 + 1];
        if (lane == 0) {
            out[(size_t)s * 2] = o0;
            out[(size_t)s * 2 + 1] = o1;
        }
        __syncwarp();
    }
}

// Device buffers of one call; freed on every exit path.
struct Bufs {
    std::vector<void *> ptrs;
    cudaStream_t stream = nullptr;
    ~Bufs() {
        if (stream) cudaStreamSynchronize(stream);
        for (void *p : ptrs) cudaFree(p);
        if (stream) cudaStreamDestroy(stream);
    }
    template <typename T> T *alloc(size_t count) {
        void *p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return static_cast<T *>(p);
    }
};

int grad_grid(int count) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, std::min(2 * sms, (count + GW - 1) / GW));
}

apsp_status to_status(cudaError_t e) {
    if (e == cudaSuccess) return APSP_OK;
    if (e == cudaErrorMemoryAllocation) return APSP_E_NOMEM;
    return APSP_E_CUDA;
}

// SplitMix64 (Steele, Lea, Flood 2014) for initialisation and shuffles.
struct SplitMix64 {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }   // (0, 1)
    double normal() {   // Box-Muller
        const double u = uniform(), v = uniform();
        return std::sqrt(-2.0 * std::log(u)) * std::cos(6.283185307179586 * v);
    }
    uint64_t below(uint64_t n) { return n ? next() % n : 0; }
};

}  // namespace

extern "C" apsp_status apsp_model_loss_grad(const float *params, const float *X, const float *Y, int32_t n,
                                            float *loss, float *grad) {
    if (!params || !X || !Y || n <= 0 || !loss || !grad) return APSP_E_ARG;
    Bufs b;
    if (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess) return APSP_E_CUDA;
    float *dP = b.alloc<float>(MLP_NPARAM), *dX = b.alloc<float>((size_t)n * MLP_IN), *dY = b.alloc<float>((size_t)n * 2);
    float *dG = b.alloc<float>(MLP_NTRAIN), *dL = b.alloc<float>(1);
    if (!dP || !dX || !dY || !dG || !dL) return APSP_E_NOMEM;
    cudaMemcpyAsync(dP, params, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice, b.stream);
    cudaMemcpyAsync(dX, X, (size_t)n * MLP_IN * sizeof(float), cudaMemcpyHostToDevice, b.stream);
    cudaMemcpyAsync(dY, Y, (size_t)n * 2 * sizeof(float), cudaMemcpyHostToDevice, b.stream);
    cudaMemsetAsync(dG, 0, MLP_NTRAIN * sizeof(float), b.stream);
    cudaMemsetAsync(dL, 0, sizeof(float), b.stream);
    k_mlp_grad<<<grad_grid(n), GW * 32, 0, b.stream>>>(dP, dX, dY, nullptr, n, 1.f / (float)n, dG, dL);
    cudaMemcpyAsync(grad, dG, MLP_NTRAIN * sizeof(float), cudaMemcpyDeviceToHost, b.stream);
    cudaMemcpyAsync(loss, dL, sizeof(float), cudaMemcpyDeviceToHost, b.stream);
    return to_status(cudaStreamSynchronize(b.stream) != cudaSuccess ? cudaErrorUnknown : cudaGetLastError());
}

extern "C" apsp_status apsp_model_predict(const float *params, const float *X, int32_t n, float *out) {
    if (!params || !X || n <= 0 || !out) return APSP_E_ARG;
    Bufs b;
    if (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess) return APSP_E_CUDA;
    float *dP = b.alloc<float>(MLP_NPARAM), *dX = b.alloc<float>((size_t)n * MLP_IN), *dO = b.alloc<float>((size_t)n * 2);
    if (!dP || !dX || !dO) return APSP_E_NOMEM;
    cudaMemcpyAsync(dP, params, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice, b.stream);
    cudaMemcpyAsync(dX, X, (size_t)n * MLP_IN * sizeof(float), cudaMemcpyHostToDevice, b.stream);
    k_mlp_predict<<<grad_grid(n), 256, 0, b.stream>>>(dP, dX, n, dO);
    cudaMemcpyAsync(out, dO, (size_t)n * 2 * sizeof(float), cudaMemcpyDeviceToHost, b.stream);
    return to_status(cudaStreamSynchronize(b.stream) != cudaSuccess ? cudaErrorUnknown : cudaGetLastError());
}

extern "C" apsp_status apsp_model_train(const float *X, const float *Y, int32_t n, int32_t epochs, int32_t batch,
                                        float lr, uint64_t seed, float *params_out, float *final_loss) {
    if (!X || !Y || n <= 0 || epochs < 0 || batch <= 0 || !(lr > 0.f) || !params_out) return APSP_E_ARG;
    // standardisation and initialisation on the host
    std::vector<float> P(MLP_NPARAM, 0.f);
    for (int i = 0; i < MLP_IN; ++i) {
        double s = 0, s2 = 0;
        for (int r = 0; r < n; ++r) {
            const double v = X[(size_t)r * MLP_IN + i];
            s += v;
            s2 += v * v;
        }
        const double m = s / n, var = std::max(0.0, s2 / n - m * m);
        P[MLP_OFF_MU + i] = (float)m;
        P[MLP_OFF_SD + i] = var > 1e-12 ? (float)std::sqrt(var) : 1.f;
    }
    SplitMix64 rng{seed};
    for (int t = 0; t < MLP_H * MLP_IN; ++t) P[MLP_OFF_W1 + t] = (float)(rng.normal() * std::sqrt(2.0 / MLP_IN));
    for (int t = 0; t < MLP_H * MLP_H; ++t) P[MLP_OFF_W2 + t] = (float)(rng.normal() * std::sqrt(2.0 / MLP_H));
    for (int t = 0; t < MLP_OUT * MLP_H; ++t) P[MLP_OFF_W3 + t] = (float)(rng.normal() * std::sqrt(1.0 / MLP_H));
    for (int o = 0; o < MLP_OUT; ++o) {   // start the output biases at the label means
        double s = 0;
        int c = 0;
        for (int r = 0; r < n; ++r) {
            const float y = Y[(size_t)r * 2 + o];
            if (!std::isnan(y)) {
                s += y;
                ++c;
            }
        }
        P[MLP_OFF_B3 + o] = c ? (float)(s / c) : 0.f;
    }
    Bufs b;
    if (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess) return APSP_E_CUDA;
    float *dP = b.alloc<float>(MLP_NPARAM), *dX = b.alloc<float>((size_t)n * MLP_IN), *dY = b.alloc<float>((size_t)n * 2);
    float *dG = b.alloc<float>(MLP_NTRAIN), *dM = b.alloc<float>(MLP_NTRAIN), *dV = b.alloc<float>(MLP_NTRAIN);
    float *dL = b.alloc<float>(1);
    int *dI = b.alloc<int>(n);
    if (!dP || !dX || !dY || !dG || !dM || !dV || !dL || !dI) return APSP_E_NOMEM;
    cudaMemcpyAsync(dP, P.data(), MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice, b.stream);
    cudaMemcpyAsync(dX, X, (size_t)n * MLP_IN * sizeof(float), cudaMemcpyHostToDevice, b.stream);
    cudaMemcpyAsync(dY, Y, (size_t)n * 2 * sizeof(float), cudaMemcpyHostToDevice, b.stream);
    cudaMemsetAsync(dG, 0, MLP_NTRAIN * sizeof(float), b.stream);
    cudaMemsetAsync(dM, 0, MLP_NTRAIN * sizeof(float), b.stream);
    cudaMemsetAsync(dV, 0, MLP_NTRAIN * sizeof(float), b.stream);
    std::vector<int> perm(n);
    for (int r = 0; r < n; ++r) perm[r] = r;
    std::vector<int> pinned_copy;   // the permutation must outlive its async copy
    int step = 0;
    double p1 = 1.0, p2 = 1.0;
    for (int e = 0; e < epochs; ++e) {
        for (int r = n - 1; r > 0; --r) std::swap(perm[r], perm[(size_t)rng.below((uint64_t)r + 1)]);
        pinned_copy = perm;
        cudaMemcpyAsync(dI, pinned_copy.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, b.stream);
        for (int s0 = 0; s0 < n; s0 += batch) {
            const int cnt = std::min(batch, n - s0);
            k_mlp_grad<<<grad_grid(cnt), GW * 32, 0, b.stream>>>(dP, dX, dY, dI + s0, cnt, 1.f / (float)cnt, dG, dL);
            ++step;
            p1 *= 0.9;
            p2 *= 0.999;
            k_mlp_adam<<<(MLP_NTRAIN + 255) / 256, 256, 0, b.stream>>>(dP, dG, dM, dV, lr, (float)(1.0 / (1.0 - p1)),
                                                                     (float)(1.0 / (1.0 - p2)));
        }
        // the host permutation buffer is reused next epoch
        if (cudaStreamSynchronize(b.stream) != cudaSuccess) return APSP_E_CUDA;
    }
    cudaMemsetAsync(dL, 0, sizeof(float), b.stream);
    cudaMemsetAsync(dG, 0, MLP_NTRAIN * sizeof(float), b.stream);
    k_mlp_grad<<<grad_grid(n), GW * 32, 0, b.stream>>>(dP, dX, dY, nullptr, n, 1.f / (float)n, dG, dL);
    cudaMemcpyAsync(params_out, dP, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, b.stream);
    float l = 0.f;
    cudaMemcpyAsync(&l, dL, sizeof(float), cudaMemcpyDeviceToHost, b.stream);
    if (cudaStreamSynchronize(b.stream) != cudaSuccess) return APSP_E_CUDA;
    if (final_loss) *final_loss = l;
    return to_status(cudaGetLastError());
}
