// Blocked min-plus Floyd-Warshall building blocks (cold path, Section 2 /
// Algorithm 5's Floyd_Warshall call): one CTA of 256 threads works on one
// 128 x 128 tile.
//
// Round kb of the blocked algorithm, with K the kb-th block of 128 nodes:
//   phase 1  D[K][K] <- its own closure (sequential over k inside the tile);
//   phase 2  D[K][J] <- min(D[K][J], D[K][K] (x) D[K][J])   for every J != K
//            D[I][K] <- min(D[I][K], D[I][K] (x) D[K][K])   for every I != K
//            (with the closed diagonal tile this is a plain product: a path
//            from r in K to c splits at its last node m in K);
//   phase 3  D[I][J] <- min(D[I][J], D[I][K] (x) D[K][J])   for I, J != K,
// where (x) is the min-plus product.  Phases 2 and 3 use minplus_tile: the
// C tile lives in registers (8 x 8 per thread), A and B are staged through
// shared memory in chunks of 32 along k.  All global loads bypass L1 (ld.cg)
// so the routines are also correct inside a persistent kernel where other
// CTAs wrote the tiles earlier in the same launch.
#pragma once

#include "common.cuh"

namespace apsp {

constexpr int FW_B = 128;
constexpr int FW_KC = 32;
constexpr int FW_THREADS = 256;

template <typename T> struct FwSmem {
    T As[FW_KC][FW_B];   // As[k][i] = A[i][kc + k]
    T Bs[FW_KC][FW_B];   // Bs[k][j] = B[kc + k][j]
};

template <typename T> struct FwDiagSmem {
    T rowb[2][FW_B];
    T colb[2][FW_B];
};

// C = min(C, A (x) B) on 128 x 128 tiles with leading dimension ld, in the
// semiring M (min-plus by default; min-max for bottleneck paths).
// B may alias C (phase 2): C is only stored after the last read of B.
template <typename T, typename M = MinPlus<T>>
__device__ void minplus_tile(T *c, const T *a, const T *b, int64_t ld, FwSmem<T> &sm) {
    using V4 = typename M::V4;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    T acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const T *crow = c + (int64_t)(ty * 8 + r) * ld;
        V4 c0 = __ldcg(reinterpret_cast<const V4 *>(crow + tx * 4));
        V4 c1 = __ldcg(reinterpret_cast<const V4 *>(crow + 64 + tx * 4));
        acc[r][0] = c0.x; acc[r][1] = c0.y; acc[r][2] = c0.z; acc[r][3] = c0.w;
        acc[r][4] = c1.x; acc[r][5] = c1.y; acc[r][6] = c1.z; acc[r][7] = c1.w;
    }
    for (int kc = 0; kc < FW_B; kc += FW_KC) {
        __syncthreads();
        // A chunk (128 rows x 32 cols), stored transposed: thread -> row i, quad q.
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            int idx = tid + t * FW_THREADS;
            int i = idx & (FW_B - 1), q = idx >> 7;  // q in [0, 8)
            V4 v = __ldcg(reinterpret_cast<const V4 *>(a + (int64_t)i * ld + kc + q * 4));
            sm.As[q * 4 + 0][i] = v.x;
            sm.As[q * 4 + 1][i] = v.y;
            sm.As[q * 4 + 2][i] = v.z;
            sm.As[q * 4 + 3][i] = v.w;
        }
        // B chunk (32 rows x 128 cols).
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            int idx = tid + t * FW_THREADS;
            int k = idx >> 5, q = idx & 31;
            V4 v = __ldcg(reinterpret_cast<const V4 *>(b + (int64_t)(kc + k) * ld + q * 4));
            *reinterpret_cast<V4 *>(&sm.Bs[k][q * 4]) = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < FW_KC; ++k) {
            V4 a0 = *reinterpret_cast<const V4 *>(&sm.As[k][ty * 8]);
            V4 a1 = *reinterpret_cast<const V4 *>(&sm.As[k][ty * 8 + 4]);
            V4 b0 = *reinterpret_cast<const V4 *>(&sm.Bs[k][tx * 4]);
            V4 b1 = *reinterpret_cast<const V4 *>(&sm.Bs[k][64 + tx * 4]);
            T av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            T bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[r][q] = M::add_min(av[r], bv[q], acc[r][q]);
        }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        T *crow = c + (int64_t)(ty * 8 + r) * ld;
        V4 c0, c1;
        c0.x = acc[r][0]; c0.y = acc[r][1]; c0.z = acc[r][2]; c0.w = acc[r][3];
        c1.x = acc[r][4]; c1.y = acc[r][5]; c1.z = acc[r][6]; c1.w = acc[r][7];
        *reinterpret_cast<V4 *>(crow + tx * 4) = c0;
        *reinterpret_cast<V4 *>(crow + 64 + tx * 4) = c1;
    }
}

// Phase 1: in-place closure of a 128 x 128 diagonal tile.  Thread (ty, tx)
// keeps rows ty*8.. and columns tx*8.. in registers; at step k the owners of
// row k and column k publish them to shared memory (double-buffered by the
// parity of k, so one barrier per step suffices).
template <typename T, typename M = MinPlus<T>>
__device__ void fw_close_diag(T *t, int64_t ld, FwDiagSmem<T> &sm) {
    using V4 = typename M::V4;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    T acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const T *row = t + (int64_t)(ty * 8 + r) * ld + tx * 8;
        V4 c0 = __ldcg(reinterpret_cast<const V4 *>(row));
        V4 c1 = __ldcg(reinterpret_cast<const V4 *>(row + 4));
        acc[r][0] = c0.x; acc[r][1] = c0.y; acc[r][2] = c0.z; acc[r][3] = c0.w;
        acc[r][4] = c1.x; acc[r][5] = c1.y; acc[r][6] = c1.z; acc[r][7] = c1.w;
    }
    __syncthreads();
    for (int kb = 0; kb < 16; ++kb) {
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const int k = kb * 8 + kk;
            const int buf = k & 1;
            if (ty == kb) {
#pragma unroll
                for (int q = 0; q < 8; ++q) sm.rowb[buf][tx * 8 + q] = acc[kk][q];
            }
            if (tx == kb) {
#pragma unroll
                for (int r = 0; r < 8; ++r) sm.colb[buf][ty * 8 + r] = acc[r][kk];
            }
            __syncthreads();
            T av[8], bv[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) av[r] = sm.colb[buf][ty * 8 + r];
#pragma unroll
            for (int q = 0; q < 8; ++q) bv[q] = sm.rowb[buf][tx * 8 + q];
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[r][q] = M::add_min(av[r], bv[q], acc[r][q]);
        }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        T *row = t + (int64_t)(ty * 8 + r) * ld + tx * 8;
        V4 c0, c1;
        c0.x = acc[r][0]; c0.y = acc[r][1]; c0.z = acc[r][2]; c0.w = acc[r][3];
        c1.x = acc[r][4]; c1.y = acc[r][5]; c1.z = acc[r][6]; c1.w = acc[r][7];
        *reinterpret_cast<V4 *>(row) = c0;
        *reinterpret_cast<V4 *>(row + 4) = c1;
    }
    __syncthreads();
}

// Tile t of phase 2 in round kb (nb blocks): t < nb-1 -> pivot-row tile,
// else pivot-column tile.  The diagonal block is skipped.
template <typename T, typename M = MinPlus<T>>
__device__ void fw_phase2_tile(T *D, int64_t ld, int kb, int nb, int t, FwSmem<T> &sm) {
    const int64_t B = FW_B;
    T *diag = D + kb * B * ld + kb * B;
    if (t < nb - 1) {
        int J = t < kb ? t : t + 1;
        T *c = D + kb * B * ld + J * B;
        minplus_tile<T, M>(c, diag, c, ld, sm);
    } else {
        int s = t - (nb - 1);
        int I = s < kb ? s : s + 1;
        T *c = D + I * B * ld + kb * B;
        minplus_tile<T, M>(c, c, diag, ld, sm);
    }
}

// Tile t of phase 3 in round kb: (I, J) over the (nb-1)^2 off-pivot tiles.
template <typename T, typename M = MinPlus<T>>
__device__ void fw_phase3_tile(T *D, int64_t ld, int kb, int nb, int t, FwSmem<T> &sm) {
    const int64_t B = FW_B;
    int I = t / (nb - 1), J = t % (nb - 1);
    I += (I >= kb);
    J += (J >= kb);
    minplus_tile<T, M>(D + I * B * ld + J * B, D + I * B * ld + kb * B, D + kb * B * ld + J * B, ld, sm);
}

}  // namespace apsp
