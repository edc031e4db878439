// k_prep.cu -- standardisation of the data and the FP64 correlation product.
//
// C = Z^T Z / n with Z the standardised data (Sec. 4.3 defines C as the
// correlation matrix; the paper does not say where it is formed). Moments are
// FP64 and two-pass (mean, then centred sum of squares), divisor n.
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace cupc {

// ---------------------------------------------------------------------------
// Sample-major X (X[s*ld + v]) to variable-major (Xt[v*n + s]), 32x32 tiles.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_transpose(const T* __restrict__ X, long long ld, int n, int p, T* __restrict__ Xt)
{
    __shared__ T tile[32][33];
    const int v0 = blockIdx.x * 32, s0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int s = s0 + r, v = v0 + threadIdx.x;
        if (s < n && v < p) tile[r][threadIdx.x] = X[(size_t)s * ld + v];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int v = v0 + r, s = s0 + threadIdx.x;
        if (s < n && v < p) Xt[(size_t)v * n + s] = tile[threadIdx.x][r];
    }
}

// Batch form: block z transposes problem z's n x p sample-major block at
// x_off into its p x n variable-major block at the same offset of Xt.
template <typename T>
__global__ void k_transpose_batch(const T* __restrict__ X, const ProbDesc* __restrict__ probs, T* __restrict__ Xt)
{
    __shared__ T tile[32][33];
    const ProbDesc& D = probs[blockIdx.z];
    const int n = D.n, p = D.p;
    const int v0 = blockIdx.x * 32, s0 = blockIdx.y * 32;
    if (v0 >= p || s0 >= n) return;
    const T* src = X + D.x_off;
    T* dst = Xt + D.x_off;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int s = s0 + r, v = v0 + threadIdx.x;
        if (s < n && v < p) tile[r][threadIdx.x] = src[(size_t)s * p + v];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int v = v0 + r, s = s0 + threadIdx.x;
        if (s < n && v < p) dst[(size_t)v * n + s] = tile[threadIdx.x][r];
    }
}

// One block per variable. Moments in FP64 in one pass over shifted values
// (shift K = the variable's first sample, so the centred sums do not cancel):
// S1 = sum (x - K), S2 = sum (x - K)^2, mean = K + S1/n,
// var = (S2 - S1^2/n) / n (population variance, divisor n). A second pass
// writes z = (x - mean)/sd in FP64 and, in FP32 mode, its bf16 split.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_standardize(const T* __restrict__ Xv, long long ld, int n, int p,
                                                    double* __restrict__ mu, double* __restrict__ isd,
                                                    double* __restrict__ z64, long long ldz,
                                                    __nv_bfloat16* __restrict__ zhi, __nv_bfloat16* __restrict__ zlo,
                                                    long long ldb, Meta* meta, const int* __restrict__ vprob,
                                                    const ProbDesc* __restrict__ probs)
{
    __shared__ double red[2][NT / 32];
    const int v = blockIdx.x;
    if (v >= p) return;
    const T* row = Xv + (size_t)v * ld;
    double* zrow = z64 ? z64 + (size_t)v * ldz : nullptr;
    if (vprob) {
        // batch: global vertex v of problem D, whose variable-major rows (ld = its
        // n) start at x_off and whose FP64 rows start at z_off; a padding vertex
        // gets zero bf16 rows
        const ProbDesc& D = probs[vprob[v]];
        const int loc = v - D.off;
        if (loc >= D.p) {
            if (threadIdx.x == 0) {
                mu[v] = 0.0;
                isd[v] = 0.0;
            }
            if (zhi)
                for (int k = threadIdx.x; k < ldb; k += NT) {
                    zhi[(size_t)v * ldb + k] = __float2bfloat16(0.f);
                    zlo[(size_t)v * ldb + k] = __float2bfloat16(0.f);
                }
            return;
        }
        n = D.n;
        row = Xv + D.x_off + (size_t)loc * n;
        if (z64) zrow = z64 + D.z_off + (long long)loc * n;
    }
    const double K = (double)row[0];
    double s1 = 0.0, s2 = 0.0;
    for (int k = threadIdx.x; k < n; k += NT) {
        const double d = (double)row[k] - K;
        s1 += d;
        s2 = fma(d, d, s2);
    }
    // deterministic block reduction: warp trees, then the warp partials in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][w] = s1;
        red[1][w] = s2;
    }
    __syncthreads();
    double S1 = 0.0, S2 = 0.0;
#pragma unroll
    for (int k = 0; k < NT / 32; ++k) {
        S1 += red[0][k];
        S2 += red[1][k];
    }
    const double mean = K + S1 / (double)n;
    const double var = (S2 - S1 * S1 / (double)n) / (double)n;
    const bool ok = (var > 0.0) && isfinite(var) && isfinite(mean);
    const double inv = ok ? 1.0 / sqrt(var) : 0.0;
    if (threadIdx.x == 0) {
        mu[v] = mean;
        isd[v] = inv;
        if (!ok) atomicOr(&meta->error, 1);
    }
    // z = (x - mean) / sd in FP64; the bf16 split z = hi + lo (|z - hi - lo| <
    // 2^-18 |z|) takes the FP64 centring and an FP32 scaling (2^-24, far below
    // the split's 2^-18)
    const float fi = (float)inv;
    for (int k = threadIdx.x; k < n; k += NT) {
        const double d = (double)row[k] - mean;
        if (zrow) zrow[k] = d * inv;
        if (zhi) {
            const float z = (float)d * fi;
            const __nv_bfloat16 h = __float2bfloat16_rn(z);
            zhi[(size_t)v * ldb + k] = h;
            zlo[(size_t)v * ldb + k] = __float2bfloat16_rn(z - __bfloat162float(h));
        }
    }
    // zero the K padding so the tensor-core product can read whole 64-wide slabs
    if (zhi)
        for (int k = n + threadIdx.x; k < ldb; k += NT) {
            zhi[(size_t)v * ldb + k] = __float2bfloat16(0.f);
            zlo[(size_t)v * ldb + k] = __float2bfloat16(0.f);
        }
}

// ---------------------------------------------------------------------------
// SIMT symmetric product C = Z Z^T * (1/n) over the upper-triangle tiles,
// mirrored into the lower triangle (so C is exactly symmetric), unit diagonal.
// BM x BM tile, BK-deep slabs through shared memory, TM x TM per thread.
// ---------------------------------------------------------------------------
template <typename T, int BM, int BK, int TM>
__global__ void __launch_bounds__((BM / TM) * (BM / TM))
k_syrk(const T* __restrict__ Z, long long ldz, int n, int p, T* __restrict__ C, double inv_n)
{
    constexpr int TD = BM / TM;          // threads per tile dimension
    constexpr int NT = TD * TD;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BM + 1];
    // triangular tile index -> (bi <= bj)
    const long long t = blockIdx.x;
    int bj = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long long)(bj + 1) * (bj + 2) / 2 <= t) ++bj;
    while ((long long)bj * (bj + 1) / 2 > t) --bj;
    const int bi = (int)(t - (long long)bj * (bj + 1) / 2);
    const int i0 = bi * BM, j0 = bj * BM;
    const int tx = threadIdx.x % TD, ty = threadIdx.x / TD;
    T acc[TM][TM];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) acc[a][b] = T(0);

    for (int k0 = 0; k0 < n; k0 += BK) {
        for (int e = threadIdx.x; e < BM * BK; e += NT) {
            const int r = e / BK, k = e % BK;
            const int gi = i0 + r, gj = j0 + r, gk = k0 + k;
            As[k][r] = (gi < p && gk < n) ? Z[(size_t)gi * ldz + gk] : T(0);
            Bs[k][r] = (gj < p && gk < n) ? Z[(size_t)gj * ldz + gk] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            T a[TM], b[TM];
#pragma unroll
            for (int m = 0; m < TM; ++m) {
                a[m] = As[k][ty + TD * m];
                b[m] = Bs[k][tx + TD * m];
            }
#pragma unroll
            for (int m = 0; m < TM; ++m)
#pragma unroll
                for (int q = 0; q < TM; ++q) acc[m][q] = fma(a[m], b[q], acc[m][q]);
        }
        __syncthreads();
    }
    const T sc = (T)inv_n;
#pragma unroll
    for (int m = 0; m < TM; ++m) {
        const int gi = i0 + ty + TD * m;
#pragma unroll
        for (int q = 0; q < TM; ++q) {
            const int gj = j0 + tx + TD * q;
            if (gi >= p || gj >= p) continue;
            if (bi == bj) {
                // diagonal tile: (gi,gj) and (gj,gi) are the same dot product in the
                // same order, so each is written by its own thread
                C[(size_t)gi * p + gj] = (gi == gj) ? T(1) : acc[m][q] * sc;
            } else {
                const T val = acc[m][q] * sc;
                C[(size_t)gi * p + gj] = val;
                C[(size_t)gj * p + gi] = val;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
cudaError_t launch_transpose(int dtype, const void* X, long long ld, int n, int p, void* Xt, cudaStream_t st)
{
    dim3 grid((p + 31) / 32, (n + 31) / 32), block(32, 8);
    if (dtype == CUPC_F64)
        k_transpose<double><<<grid, block, 0, st>>>((const double*)X, ld, n, p, (double*)Xt);
    else
        k_transpose<float><<<grid, block, 0, st>>>((const float*)X, ld, n, p, (float*)Xt);
    return cudaGetLastError();
}

cudaError_t launch_standardize(int dtype, const void* Xv, long long ld, int n, int p, double* mu, double* isd,
                               double* z64, long long ldz, void* zhi, void* zlo, long long ldb, Meta* meta,
                               cudaStream_t st, const int* vprob, const ProbDesc* probs)
{
    constexpr int NT = 256;
    if (dtype == CUPC_F64)
        k_standardize<double, NT><<<p, NT, 0, st>>>((const double*)Xv, ld, n, p, mu, isd, z64, ldz,
                                                    (__nv_bfloat16*)zhi, (__nv_bfloat16*)zlo, ldb, meta, vprob,
                                                    probs);
    else
        k_standardize<float, NT><<<p, NT, 0, st>>>((const float*)Xv, ld, n, p, mu, isd, z64, ldz,
                                                   (__nv_bfloat16*)zhi, (__nv_bfloat16*)zlo, ldb, meta, vprob,
                                                   probs);
    return cudaGetLastError();
}

cudaError_t launch_transpose_batch(int dtype, const void* X, const ProbDesc* probs, int nprob, int pmax, int nmax,
                                   void* Xt, cudaStream_t st)
{
    dim3 grid((pmax + 31) / 32, (nmax + 31) / 32, nprob), block(32, 8);
    if (dtype == CUPC_F64)
        k_transpose_batch<double><<<grid, block, 0, st>>>((const double*)X, probs, (double*)Xt);
    else
        k_transpose_batch<float><<<grid, block, 0, st>>>((const float*)X, probs, (float*)Xt);
    return cudaGetLastError();
}

cudaError_t launch_syrk_f64(const double* Z, long long ldz, int n, int p, double* C, cudaStream_t st)
{
    constexpr int BM = 64, BK = 16, TM = 4;
    const long long nt = (p + BM - 1) / BM;
    const long long tiles = nt * (nt + 1) / 2;
    k_syrk<double, BM, BK, TM><<<(unsigned)tiles, (BM / TM) * (BM / TM), 0, st>>>(Z, ldz, n, p, C, 1.0 / n);
    return cudaGetLastError();
}

}  // namespace cupc
