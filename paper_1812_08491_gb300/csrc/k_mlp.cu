// k_mlp.cu -- training and scoring kernels of the candidate-scoring network.
//
// Loss: mean binary cross-entropy with logits over a batch,
//   L = mean( log(1 + e^y) - t y ),  dL/dy = (sigmoid(y) - t) / B.
// Gradients are formed per block over chunks of 128 samples staged in shared
// memory (forward pre-activations, then the backward deltas), each parameter's
// gradient being one thread's ordered sum over the samples -- so the result
// is deterministic. A second kernel adds the block partials in block order and
// applies Adam (Kingma and Ba, 2015) to the FP32 master weights, refreshing
// their bf16 copy used for scoring.
#include <algorithm>

#include "kernels.cuh"
#include "mlp.cuh"

namespace cupc {
namespace {

constexpr int NT = 256;
constexpr int CH = 128;                                   // samples per chunk
constexpr int PER_THREAD = (MLP_NP + NT - 1) / NT;         // parameters owned per thread

struct MlpSmem {
    float W[MLP_NP];
    float x[CH][MLP_IN];
    float a1[CH][MLP_H];     // pre-activation of layer 1
    float a2[CH][MLP_H];     // pre-activation of layer 2
    float d2[CH][MLP_H];     // dL/da2
    float d1[CH][MLP_H];     // dL/da1
    float dy[CH];
    float y[CH];
};

__device__ __forceinline__ float softplus(float y) { return y > 0.f ? y + log1pf(__expf(-y)) : log1pf(__expf(y)); }

// Gradient of the mean loss over samples [s0, s1) (inv_batch = 1/(s1 - s0)),
// per block: gpart[block][p], lpart[block] = summed loss.
__global__ void __launch_bounds__(NT) k_mlp_grad(const float* __restrict__ P, const float* __restrict__ X,
                                                 const float* __restrict__ T, long long s0, long long s1,
                                                 float inv_batch, float* __restrict__ gpart,
                                                 float* __restrict__ lpart)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
    const int tid = threadIdx.x;
    for (int q = tid; q < MLP_NP; q += NT) S.W[q] = P[q];
    float g[PER_THREAD];
#pragma unroll
    for (int u = 0; u < PER_THREAD; ++u) g[u] = 0.f;
    float loss = 0.f;
    __syncthreads();
    for (long long c0 = s0 + (long long)blockIdx.x * CH; c0 < s1; c0 += (long long)gridDim.x * CH) {
        const int m = (int)min((long long)CH, s1 - c0);
        for (int e = tid; e < CH * MLP_IN; e += NT) {
            const int b = e / MLP_IN, c = e % MLP_IN;
            S.x[b][c] = (b < m) ? X[(c0 + b) * MLP_IN + c] : 0.f;
        }
        __syncthreads();
        for (int e = tid; e < CH * MLP_H; e += NT) {
            const int b = e / MLP_H, o = e % MLP_H;
            float a = S.W[MLP_OFF_B1 + o];
#pragma unroll
            for (int c = 0; c < MLP_IN; ++c) a = fmaf(S.W[MLP_OFF_W1 + o * MLP_IN + c], S.x[b][c], a);
            S.a1[b][o] = a;
        }
        __syncthreads();
        for (int e = tid; e < CH * MLP_H; e += NT) {
            const int b = e / MLP_H, o = e % MLP_H;
            float a = S.W[MLP_OFF_B2 + o];
            for (int k = 0; k < MLP_H; ++k) a = fmaf(S.W[MLP_OFF_W2 + o * MLP_H + k], fmaxf(S.a1[b][k], 0.f), a);
            S.a2[b][o] = a;
        }
        __syncthreads();
        if (tid < CH) {
            const int b = tid;
            float y = S.W[MLP_OFF_B3];
            for (int o = 0; o < MLP_H; ++o) y = fmaf(S.W[MLP_OFF_W3 + o], fmaxf(S.a2[b][o], 0.f), y);
            S.y[b] = y;
            if (b < m) {
                const float t = T[c0 + b];
                S.dy[b] = (1.f / (1.f + __expf(-y)) - t) * inv_batch;
            } else {
                S.dy[b] = 0.f;
            }
        }
        __syncthreads();
        if (tid == 0)
            for (int b = 0; b < m; ++b) loss += softplus(S.y[b]) - T[c0 + b] * S.y[b];
        for (int e = tid; e < CH * MLP_H; e += NT) {
            const int b = e / MLP_H, o = e % MLP_H;
            S.d2[b][o] = S.a2[b][o] > 0.f ? S.dy[b] * S.W[MLP_OFF_W3 + o] : 0.f;
        }
        __syncthreads();
        for (int e = tid; e < CH * MLP_H; e += NT) {
            const int b = e / MLP_H, k = e % MLP_H;
            float a = 0.f;
            if (S.a1[b][k] > 0.f)
                for (int o = 0; o < MLP_H; ++o) a = fmaf(S.W[MLP_OFF_W2 + o * MLP_H + k], S.d2[b][o], a);
            S.d1[b][k] = a;
        }
        __syncthreads();
        // each owned parameter: an ordered sum over the chunk's samples
#pragma unroll
        for (int u = 0; u < PER_THREAD; ++u) {
            const int q = tid + u * NT;
            if (q >= MLP_NP) continue;
            float a = 0.f;
            if (q < MLP_OFF_B1) {
                const int o = q / MLP_IN, c = q % MLP_IN;
                for (int b = 0; b < m; ++b) a = fmaf(S.d1[b][o], S.x[b][c], a);
            } else if (q < MLP_OFF_W2) {
                const int o = q - MLP_OFF_B1;
                for (int b = 0; b < m; ++b) a += S.d1[b][o];
            } else if (q < MLP_OFF_B2) {
                const int o = (q - MLP_OFF_W2) / MLP_H, k = (q - MLP_OFF_W2) % MLP_H;
                for (int b = 0; b < m; ++b) a = fmaf(S.d2[b][o], fmaxf(S.a1[b][k], 0.f), a);
            } else if (q < MLP_OFF_W3) {
                const int o = q - MLP_OFF_B2;
                for (int b = 0; b < m; ++b) a += S.d2[b][o];
            } else if (q < MLP_OFF_B3) {
                const int o = q - MLP_OFF_W3;
                for (int b = 0; b < m; ++b) a = fmaf(S.dy[b], fmaxf(S.a2[b][o], 0.f), a);
            } else {
                for (int b = 0; b < m; ++b) a += S.dy[b];
            }
            g[u] += a;
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < PER_THREAD; ++u) {
        const int q = tid + u * NT;
        if (q < MLP_NP) gpart[(size_t)blockIdx.x * MLP_NP + q] = g[u];
    }
    if (tid == 0) lpart[blockIdx.x] = loss;
}

// Adds the block partials in block order; with lr > 0 applies one Adam step
// (bias-corrected, step counted from 1) and refreshes the bf16 copy.
__global__ void k_mlp_apply(float* __restrict__ P, float* __restrict__ M, float* __restrict__ V,
                            const float* __restrict__ gpart, int nblocks, float* __restrict__ gsum, int step,
                            float lr, float beta1, float beta2, float eps, __nv_bfloat16* __restrict__ Pb)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= MLP_NP) return;
    float gq = 0.f;
    for (int b = 0; b < nblocks; ++b) gq += gpart[(size_t)b * MLP_NP + q];
    if (gsum) gsum[q] = gq;
    if (lr > 0.f) {
        const float m = beta1 * M[q] + (1.f - beta1) * gq;
        const float v = beta2 * V[q] + (1.f - beta2) * gq * gq;
        M[q] = m;
        V[q] = v;
        const float mh = m / (1.f - powf(beta1, (float)step));
        const float vh = v / (1.f - powf(beta2, (float)step));
        const float w = P[q] - lr * mh / (sqrtf(vh) + eps);
        P[q] = w;
        if (Pb) Pb[q] = __float2bfloat16_rn(w);
    }
}

__global__ void k_mlp_to_bf16(const float* __restrict__ P, __nv_bfloat16* __restrict__ Pb)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < MLP_NP) Pb[q] = __float2bfloat16_rn(P[q]);
}

// Scores of N feature rows with the bf16 weights (one thread per row).
__global__ void k_mlp_forward(const __nv_bfloat16* __restrict__ Pb, const float* __restrict__ X, long long N,
                              float* __restrict__ y)
{
    __shared__ __nv_bfloat16 W[MLP_NP];
    for (int q = threadIdx.x; q < MLP_NP; q += blockDim.x) W[q] = Pb[q];
    __syncthreads();
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    float x[MLP_IN];
#pragma unroll
    for (int c = 0; c < MLP_IN; ++c) x[c] = X[r * MLP_IN + c];
    y[r] = mlp_score(W, x);
}

}  // namespace

size_t mlp_grad_smem() { return sizeof(MlpSmem); }

cudaError_t launch_mlp_grad(const float* P, const float* X, const float* T, long long s0, long long s1, float* gpart,
                            float* lpart, int blocks, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(MlpSmem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_mlp_grad<<<blocks, NT, sizeof(MlpSmem), st>>>(P, X, T, s0, s1, 1.f / (float)(s1 - s0), gpart, lpart);
    return cudaGetLastError();
}

cudaError_t launch_mlp_apply(float* P, float* M, float* V, const float* gpart, int nblocks, float* gsum, int step,
                             float lr, void* Pb, cudaStream_t st)
{
    k_mlp_apply<<<(MLP_NP + 255) / 256, 256, 0, st>>>(P, M, V, gpart, nblocks, gsum, step, lr, 0.9f, 0.999f, 1e-8f,
                                                      (__nv_bfloat16*)Pb);
    return cudaGetLastError();
}

cudaError_t launch_mlp_to_bf16(const float* P, void* Pb, cudaStream_t st)
{
    k_mlp_to_bf16<<<(MLP_NP + 255) / 256, 256, 0, st>>>(P, (__nv_bfloat16*)Pb);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const void* Pb, const float* X, long long N, float* y, cudaStream_t st)
{
    if (N == 0) return cudaSuccess;
    k_mlp_forward<<<(unsigned)((N + 127) / 128), 128, 0, st>>>((const __nv_bfloat16*)Pb, X, N, y);
    return cudaGetLastError();
}


// Training examples: q[6e .. 6e + 6) = (row i, candidate position c, first
// entry of the row's frozen neighbour list in nbs, its length d, level l,
// label); the feature row is the one the level kernel scores candidate c of
// row i with (mlp_row_features over the list, from the FP32 correlation C,
// p x p).
__global__ void k_mlp_examples(const float* __restrict__ C, long long p, const int* __restrict__ nbs,
                               const int* __restrict__ q, long long n, float* __restrict__ X, float* __restrict__ t)
{
    auto Cf = [&](int a, int b) { return __ldg(C + (size_t)a * p + b); };
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int* r = q + 6 * e;
        const int i = r[0], c = r[1], d = r[3], l = r[4];
        const int* nb = nbs + r[2];
        float sum = 0.f;
        for (int u = 0; u < d; ++u) sum += fabsf(Cf(i, nb[u]));
        float x[MLP_IN];
        mlp_row_features(Cf, i, nb, d, c, l, sum, x);
#pragma unroll
        for (int k = 0; k < MLP_IN; ++k) X[e * MLP_IN + k] = x[k];
        t[e] = (float)r[5];
    }
}

cudaError_t launch_mlp_examples(const float* C, long long p, const int* nbs, const int* q, long long n, float* X,
                                float* t, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int block = 256;
    const unsigned grid = (unsigned)std::min<long long>((n + block - 1) / block, 4096);
    k_mlp_examples<<<grid, block, 0, st>>>(C, p, nbs, q, n, X, t);
    return cudaGetLastError();
}
}  // namespace cupc
