// Learned warm/cold cost model: a 6 -> 64 -> 64 -> 2 multilayer perceptron
// with ReLU hidden layers, fp32.  Input features of one update:
//   0 update type (0 add, 1/3 removal, 2/3 decrease, 1 increase)
//   1 log2(n)
//   2 relative weight change (0 for node updates)
//   3 affected pairs / n^2
//   4 Cost of Eq. (equ:cost_defi): affected rows / (N - 1)
//   5 affected rows / n
// Outputs: predicted log2(microseconds) of the warm path and of the cold path.
// Features are standardised with the mean / std stored in the parameters.
//
// Parameter block (floats, this order): mu[6], sd[6], W1[64][6], b1[64],
// W2[64][64], b2[64], W3[2][64], b3[2].
#pragma once

namespace apsp {

constexpr int MLP_IN = 6, MLP_H = 64, MLP_OUT = 2;
constexpr int MLP_OFF_MU = 0;
constexpr int MLP_OFF_SD = MLP_OFF_MU + MLP_IN;
constexpr int MLP_OFF_W1 = MLP_OFF_SD + MLP_IN;
constexpr int MLP_OFF_B1 = MLP_OFF_W1 + MLP_H * MLP_IN;
constexpr int MLP_OFF_W2 = MLP_OFF_B1 + MLP_H;
constexpr int MLP_OFF_B2 = MLP_OFF_W2 + MLP_H * MLP_H;
constexpr int MLP_OFF_W3 = MLP_OFF_B2 + MLP_H;
constexpr int MLP_OFF_B3 = MLP_OFF_W3 + MLP_OUT * MLP_H;
constexpr int MLP_NPARAM = MLP_OFF_B3 + MLP_OUT;
// trainable part (everything after the standardisation constants)
constexpr int MLP_OFF_TRAIN = MLP_OFF_W1;
constexpr int MLP_NTRAIN = MLP_NPARAM - MLP_OFF_TRAIN;

// Forward pass of one feature vector by a whole CTA (>= 64 threads).  Every
// thread passes the same `feat`; out2 (shared) receives the two outputs.
// The arithmetic order is fixed, so every CTA computes bit-identical outputs.
__device__ __forceinline__ void mlp_predict_cta(const float *P, const float *feat, float *out2) {
    __shared__ float xin[MLP_IN], h1[MLP_H], h2[MLP_H];
    const int t = threadIdx.x;
    if (t < MLP_IN) xin[t] = (feat[t] - P[MLP_OFF_MU + t]) / P[MLP_OFF_SD + t];
    __syncthreads();
    if (t < MLP_H) {
        float s = P[MLP_OFF_B1 + t];
        for (int k = 0; k < MLP_IN; ++k) s = fmaf(P[MLP_OFF_W1 + t * MLP_IN + k], xin[k], s);
        h1[t] = fmaxf(s, 0.f);
    }
    __syncthreads();
    if (t < MLP_H) {
        float s = P[MLP_OFF_B2 + t];
        for (int k = 0; k < MLP_H; ++k) s = fmaf(P[MLP_OFF_W2 + t * MLP_H + k], h1[k], s);
        h2[t] = fmaxf(s, 0.f);
    }
    __syncthreads();
    if (t < MLP_OUT) {
        float s = P[MLP_OFF_B3 + t];
        for (int k = 0; k < MLP_H; ++k) s = fmaf(P[MLP_OFF_W3 + t * MLP_H + k], h2[k], s);
        out2[t] = s;
    }
    __syncthreads();
}

}  // namespace apsp
