// mlp.cuh -- the candidate-scoring network used to order conditioning subsets.
//
// A candidate k for edge side (i, j) at level l is described by
//   x = (|C_ik|, |C_jk|, |C_ij|, l / 8, |rho_ij.k|),
// rho_ij.k the first-order partial correlation; the network is
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

// Features of candidate k for side (i, j) from correlations cij = C_ij,
// cik = C_ik, cjk = C_jk (FP32).
__device__ __forceinline__ void mlp_features(float cij, float cik, float cjk, int l, float (&x)[MLP_IN])
{
    x[0] = fabsf(cik);
    x[1] = fabsf(cjk);
    x[2] = fabsf(cij);
    x[3] = (float)l * 0.125f;
    const float den = (1.f - cik * cik) * (1.f - cjk * cjk);
    x[4] = den > 1e-12f ? fabsf((cij - cik * cjk) * rsqrtf(den)) : 1.f;
}

// Score of one candidate with weights W (bf16, packed as above) in shared or
// global memory; FP32 accumulation.
__device__ __forceinline__ float mlp_score(const __nv_bfloat16* __restrict__ W, const float (&x)[MLP_IN])
{
    float h1[MLP_H];
#pragma unroll
    for (int o = 0; o < MLP_H; ++o) {
        float a = __bfloat162float(W[MLP_OFF_B1 + o]);
#pragma unroll
        for (int c = 0; c < MLP_IN; ++c) a = fmaf(__bfloat162float(W[MLP_OFF_W1 + o * MLP_IN + c]), x[c], a);
        h1[o] = fmaxf(a, 0.f);
    }
    float y = __bfloat162float(W[MLP_OFF_B3]);
#pragma unroll 4
    for (int o = 0; o < MLP_H; ++o) {
        float a = __bfloat162float(W[MLP_OFF_B2 + o]);
        const __nv_bfloat16* row = W + MLP_OFF_W2 + o * MLP_H;
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) a = fmaf(__bfloat162float(row[k]), h1[k], a);
        y = fmaf(__bfloat162float(W[MLP_OFF_W3 + o]), fmaxf(a, 0.f), y);
    }
    return y;
}

}  // namespace cupc
