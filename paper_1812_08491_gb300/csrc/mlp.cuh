// mlp.cuh -- the candidate-scoring network used to order conditioning subsets.
//
// A candidate k of row i at level l (a neighbour of i in A'_G) is described by
//   x = (|C_ik|, mean_j |C_jk|, mean_j |C_ij|, l / 8, mean_j |rho_ij.k|),
// the means over the row's other neighbours j (rho_ij.k the first-order partial
// correlation). At level 1 the two terms that need every C_jk of the row -- as
// many reads as the level's own tests -- are 0. One score per (row, candidate)
// gives one order per row, so the tests of a row still share each subset S
// across its j. The network is
//   h1 = relu(W1 x + b1) (64), h2 = relu(W2 h1 + b2) (64), y = w3 . h2 + b3.
// Parameters are packed W1 (64x5), b1, W2 (64x64), b2, w3, b3 (row-major).
// Training keeps FP32 master weights; scoring reads their bf16 rounding with
// FP32 accumulation. The paper has no learned component.
#pragma once

#include <cuda_bf16.h>

namespace cupc {

constexpr int MLP_IN = 5, MLP_H = 64;
constexpr int MLP_OFF_W1 = 0;
constexpr int MLP_OFF_B1 = MLP_OFF_W1 + MLP_H * MLP_IN;
constexpr int MLP_OFF_W2 = MLP_OFF_B1 + MLP_H;
constexpr int MLP_OFF_B2 = MLP_OFF_W2 + MLP_H * MLP_H;
constexpr int MLP_OFF_W3 = MLP_OFF_B2 + MLP_H;
constexpr int MLP_OFF_B3 = MLP_OFF_W3 + MLP_H;
constexpr int MLP_NP = MLP_OFF_B3 + 1;  // 4609

// |rho_ij.k| from cij = C_ij, cik = C_ik, cjk = C_jk (FP32); 1 when a
// conditional variance vanishes.
__device__ __forceinline__ float mlp_rho1(float cij, float cik, float cjk)
{
    const float den = (1.f - cik * cik) * (1.f - cjk * cjk);
    return den > 1e-12f ? fabsf((cij - cik * cjk) * rsqrtf(den)) : 1.f;
}

// Features of candidate k of row i at level l: cik = C_ik; mjk, mij, mrho the
// means over the row's other neighbours j of |C_jk|, |C_ij| and |rho_ij.k|
// (0 for mjk and mrho at level 1).
__device__ __forceinline__ void mlp_features(float cik, float mjk, float mij, int l, float mrho, float (&x)[MLP_IN])
{
    x[0] = fabsf(cik);
    x[1] = mjk;
    x[2] = mij;
    x[3] = (float)l * 0.125f;
    x[4] = mrho;
}

// Features of candidate c (position in the row's neighbour list nb[0..d)) of
// row i at level l, from the FP32 correlation row accessor C(a, b): the means
// run over the row's other neighbours.
template <typename CF>
__device__ __forceinline__ void mlp_row_features(CF C, int i, const int* nb, int d, int c, int l, float sum_abs_cij,
                                                 float (&x)[MLP_IN])
{
    const int k = nb[c];
    const float cik = C(i, k);
    const float mij = d > 1 ? (sum_abs_cij - fabsf(cik)) / (float)(d - 1) : 0.f;
    float mjk = 0.f, mrho = 0.f;
    if (l >= 2 && d > 1) {
        for (int u = 0; u < d; ++u) {
            if (u == c) continue;
            const int j = nb[u];
            const float cjk = C(j, k);
            mjk += fabsf(cjk);
            mrho += mlp_rho1(C(i, j), cik, cjk);
        }
        mjk /= (float)(d - 1);
        mrho /= (float)(d - 1);
    }
    mlp_features(cik, mjk, mij, l, mrho, x);
}

__device__ __forceinline__ float mlp_wval(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float mlp_wval(float v) { return v; }

// Score of one candidate with weights W (packed as above; bf16, or their FP32
// copy, which gives the same score) in shared or global memory; FP32
// accumulation.
template <typename WT>
__device__ __forceinline__ float mlp_score(const WT* __restrict__ W, const float (&x)[MLP_IN])
{
    float h1[MLP_H];
#pragma unroll
    for (int o = 0; o < MLP_H; ++o) {
        float a = mlp_wval(W[MLP_OFF_B1 + o]);
#pragma unroll
        for (int c = 0; c < MLP_IN; ++c) a = fmaf(mlp_wval(W[MLP_OFF_W1 + o * MLP_IN + c]), x[c], a);
        h1[o] = fmaxf(a, 0.f);
    }
    float y = mlp_wval(W[MLP_OFF_B3]);
#pragma unroll 4
    for (int o = 0; o < MLP_H; ++o) {
        float a = mlp_wval(W[MLP_OFF_B2 + o]);
        const WT* row = W + MLP_OFF_W2 + o * MLP_H;
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) a = fmaf(mlp_wval(row[k]), h1[k], a);
        y = fmaf(mlp_wval(W[MLP_OFF_W3 + o]), fmaxf(a, 0.f), y);
    }
    return y;
}

}  // namespace cupc
