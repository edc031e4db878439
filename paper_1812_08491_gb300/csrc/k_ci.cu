// k_ci.cu -- partial correlations for a batch of (i, j, S) queries with the CI
// kernels' device arithmetic (Sec. 4.3), for verification.
#include "kernels.cuh"

namespace cupc {

// ---------------------------------------------------------------------------
// rho(V_i, V_j | S) for a batch of queries with the same device arithmetic.
// ---------------------------------------------------------------------------
template <typename T, int LB>
__global__ void k_pcor(const T* __restrict__ C, int p, const int* __restrict__ q, long long nq, int l,
                       double* __restrict__ rho)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nq) return;
    const int* row = q + t * (2 + l);
    const int i = row[0], j = row[1];
    int Sx[LB];
#pragma unroll
    for (int c = 0; c < LB; ++c) Sx[c] = (c < l) ? row[2 + c] : 0;
    Factor<T, LB> F;
    const T tol = sizeof(T) == 8 ? T(1e-12) : T(1e-6);
    factor_build<T, LB>(F, l, tol, [&](int a, int b) { return C[(size_t)Sx[a] * p + Sx[b]]; },
                        [&](int a) { return C[(size_t)i * p + Sx[a]]; });
    T H12, H22;
    factor_apply<T, LB>(F, l, C[(size_t)i * p + j], [&](int a) { return C[(size_t)j * p + Sx[a]]; }, H12, H22);
    const T H11 = T(1) - F.uu;
    rho[t] = (H11 > T(kVarZero) && H22 > T(kVarZero)) ? (double)(H12 / t_sqrt<T>(H11 * H22)) : nan("");
}

template <typename T>
static cudaError_t launch_pcor_t(const T* C, int p, const int* q, long long nq, int l, double* rho, cudaStream_t st)
{
    const int block = 128;
    const unsigned grid = (unsigned)((nq + block - 1) / block);
    if (l <= 1) k_pcor<T, 1><<<grid, block, 0, st>>>(C, p, q, nq, l, rho);
    else if (l <= 2) k_pcor<T, 2><<<grid, block, 0, st>>>(C, p, q, nq, l, rho);
    else if (l <= 4) k_pcor<T, 4><<<grid, block, 0, st>>>(C, p, q, nq, l, rho);
    else if (l <= 8) k_pcor<T, 8><<<grid, block, 0, st>>>(C, p, q, nq, l, rho);
    else k_pcor<T, 16><<<grid, block, 0, st>>>(C, p, q, nq, l, rho);
    return cudaGetLastError();
}

cudaError_t launch_pcor(int fp32, const void* C, int p, const int* q, long long nq, int l, double* rho,
                        cudaStream_t st)
{
    if (nq == 0) return cudaSuccess;
    return fp32 ? launch_pcor_t<float>((const float*)C, p, q, nq, l, rho, st)
                : launch_pcor_t<double>((const double*)C, p, q, nq, l, rho, st);
}

}  // namespace cupc
