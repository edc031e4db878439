// k_prep.cu -- standardisation of the data and the FP64 correlation product.
//
// C = Z^T Z / n with Z the standardised data (Sec. 4.3 defines C as the
// correlation matrix; the paper does not say where it is formed). Mean and
// variance are FP64 values, divisor n, from shifted sums.
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

// Batch form: block z transposes problem z's n x p sample-major data (xs)
// into its p x n variable-major block at offset x_off of Xt.
template <typename T>
__global__ void k_transpose_batch(const ProbDesc* __restrict__ probs, T* __restrict__ Xt)
{
    __shared__ T tile[32][33];
    const ProbDesc& D = probs[blockIdx.z];
    const int n = D.n, p = D.p;
    const int v0 = blockIdx.x * 32, s0 = blockIdx.y * 32;
    if (v0 >= p || s0 >= n) return;
    const T* src = (const T*)D.xs;
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

// ---------------------------------------------------------------------------
// FP32 data: moments in compensated FP32 pairs (two_sum, pair_add of the
// shared header); only the per-warp partial sums are widened to FP64.
// ---------------------------------------------------------------------------
// bf16 bit pattern of a finite float, rounded to nearest with ties to even,
// by integer arithmetic on the IEEE encoding (add half an ulp of the target
// minus one, plus the kept lowest bit, and truncate). Conversion instructions
// share GB300's narrow FP64 pipe; this keeps the split on the integer ALUs.
__device__ __forceinline__ unsigned short bf16_bits_rn(float x)
{
    const unsigned u = __float_as_uint(x);
    return (unsigned short)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}

__device__ __forceinline__ float bf16_bits_to_float(unsigned short h) { return __uint_as_float((unsigned)h << 16); }

// Row elements a thread loads before using them in the standardisation passes
// (the element order of its sums is unchanged).
constexpr int MU = 8;

// Shifted moments S1 = sum (x - K), S2 = sum (x - K)^2 of a row, by one block
// of NT threads, in a fixed order. FP64 data, or FP64 rows requested: FP64
// sums per thread, a warp tree and the warp partials in order. FP32 data
// otherwise: compensated pairs throughout -- x - K exactly as a pair
// (two_sum), its square exactly to 2^-48 (the product's error term by fma; the
// lo^2 term, below 2^-48 of the square, is dropped), sums by pair_add per
// thread and down the warp tree -- widened to FP64 only for the warp partials.
// The totals are valid in thread fin.
template <typename T, int NT>
__device__ __forceinline__ void shifted_moments(const T* __restrict__ row, int n, T K, bool pairs, int fin,
                                                double& S1, double& S2)
{
    __shared__ double red[2][NT / 32];
    __shared__ float redp[4][NT / 32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    S1 = 0.0;
    S2 = 0.0;
    if constexpr (sizeof(T) == 4) {
        if (pairs) {
            float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f;
            // a thread's elements k, k + NT, ... in order; eight loads in flight
            for (int k0 = threadIdx.x; k0 < n; k0 += NT * MU) {
                float x[MU];
#pragma unroll
                for (int u = 0; u < MU; ++u) x[u] = (k0 + u * NT < n) ? row[k0 + u * NT] : 0.f;
#pragma unroll
                for (int u = 0; u < MU; ++u) {
                    if (k0 + u * NT >= n) break;
                    float dh, dl;
                    two_sum(x[u], -K, dh, dl);
                    pair_add(ah, al, dh, dl);
                    const float p = __fmul_rn(dh, dh);
                    float q = fmaf(dh, dh, -p);
                    q = fmaf(2.f * dh, dl, q);
                    float ph, pl;
                    fast_two_sum(p, q, ph, pl);
                    pair_add(bh, bl, ph, pl);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float xh = __shfl_xor_sync(0xffffffffu, ah, o), xl = __shfl_xor_sync(0xffffffffu, al, o);
                const float yh = __shfl_xor_sync(0xffffffffu, bh, o), yl = __shfl_xor_sync(0xffffffffu, bl, o);
                pair_add(ah, al, xh, xl);
                pair_add(bh, bl, yh, yl);
            }
            if (lane == 0) {
                redp[0][w] = ah;
                redp[1][w] = al;
                redp[2][w] = bh;
                redp[3][w] = bl;
            }
            __syncthreads();
            // the warp partials in order, still in pairs; widened once (by the
            // block's finishing thread fin, which rotates over the warps)
            if (threadIdx.x == fin) {
                float sh = redp[0][0], sl = redp[1][0], th = redp[2][0], tl = redp[3][0];
                for (int k = 1; k < NT / 32; ++k) {
                    pair_add(sh, sl, redp[0][k], redp[1][k]);
                    pair_add(th, tl, redp[2][k], redp[3][k]);
                }
                S1 = (double)sh + (double)sl;
                S2 = (double)th + (double)tl;
            }
            return;
        }
    }
    const double Kd = (double)K;
    double s1 = 0.0, s2 = 0.0;
    for (int k0 = threadIdx.x; k0 < n; k0 += NT * MU) {
        T x[MU];
#pragma unroll
        for (int u = 0; u < MU; ++u) x[u] = (k0 + u * NT < n) ? row[k0 + u * NT] : T(0);
#pragma unroll
        for (int u = 0; u < MU; ++u) {
            if (k0 + u * NT >= n) break;
            const double d = (double)x[u] - Kd;
            s1 += d;
            s2 = fma(d, d, s2);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
        red[0][w] = s1;
        red[1][w] = s2;
    }
    __syncthreads();
    if (threadIdx.x == fin)
        for (int k = 0; k < NT / 32; ++k) {
            S1 += red[0][k];
            S2 += red[1][k];
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
                                                    float2* __restrict__ mup, double* __restrict__ z64, long long ldz,
                                                    __nv_bfloat16* __restrict__ zhi, __nv_bfloat16* __restrict__ zlo,
                                                    long long ldb, Meta* meta, const int* __restrict__ vprob,
                                                    const ProbDesc* __restrict__ probs, double inv_n)
{
    const int v = blockIdx.x;
    if (v >= p) return;
    const T* row = Xv + (size_t)v * ld;
    double* zrow = z64 ? z64 + (size_t)v * ldz : nullptr;
    long long kpad = ldb;  // bf16 columns written (the product reads whole 64-wide slabs)
    if (vprob) {
        // batch: global vertex v of problem D, whose variable-major rows (ld = its
        // n) start at xv and whose FP64 rows start at z_off; the product reads its
        // rows up to n rounded to 64; a padding vertex gets zero bf16 rows
        const ProbDesc& D = probs[vprob[v]];
        const int loc = v - D.off;
        kpad = ((long long)D.n + 63) / 64 * 64;
        if (loc >= D.p) {
            if (threadIdx.x == 0) {
                mu[v] = 0.0;
                isd[v] = 0.0;
                if (mup) mup[v] = make_float2(0.f, 0.f);
            }
            if (zhi)
                for (int k = threadIdx.x; k < kpad; k += NT) {
                    ((unsigned short*)zhi)[(size_t)v * ldb + k] = 0;
                    ((unsigned short*)zlo)[(size_t)v * ldb + k] = 0;
                }
            return;
        }
        n = D.n;
        inv_n = D.inv_n;
        row = (const T*)D.xv + (size_t)loc * n;
        if (z64) zrow = z64 + D.z_off + (long long)loc * n;
    }
    // FP32 mode (no FP64 rows requested): compensated FP32 pairs for FP32 data
    const bool fast = (zrow == nullptr);
    __shared__ double stat[2];
    __shared__ float fstat[3];
    {
        double S1, S2;
        // the thread finishing this block's FP64 work: a different warp per block,
        // so the FP64 work of consecutive blocks lands on different schedulers
        const int fin = (int)(blockIdx.x % (NT / 32)) * 32;
        shifted_moments<T, NT>(row, n, row[0], fast, fin, S1, S2);
        // mean, 1/sd and their FP32 forms, once per variable (1/n from the host:
        // a multiply instead of a divide on the FP64 pipe)
        if (threadIdx.x == fin) {
            const double K = (double)row[0];
            const double a = S1 * inv_n;
            const double mean = K + a;
            const double var = fma(-S1, a, S2) * inv_n;
            const bool ok = (var > 0.0) && isfinite(var) && isfinite(mean);
            const double inv = ok ? rsqrt(var) : 0.0;
            mu[v] = mean;
            isd[v] = inv;
            if (!ok) atomicOr(&meta->error, 1);
            stat[0] = mean;
            stat[1] = inv;
            const float mh = (float)mean;
            fstat[0] = mh;
            fstat[1] = (float)(mean - (double)mh);
            fstat[2] = (float)inv;
            if (mup) mup[v] = make_float2(fstat[0], fstat[1]);
        }
        __syncthreads();
    }
    const double mean = stat[0], inv = stat[1];
    // z = (x - mean) / sd in FP64 for the FP64 rows. The bf16 split z = hi + lo
    // (|z - hi - lo| < 2^-17 |z|) needs z to about 2^-20: for FP32 data it is
    // formed in FP32 as ((x - m_hi) - m_lo) * (1/sd) with mean = m_hi + m_lo
    // (x - m_hi exact when x is within a factor 2 of the mean, else rounded
    // relative to a result of the size of x), about 3 * 2^-24 in all; for FP64
    // data the centring is FP64.
    const float mh = fstat[0], ml = fstat[1], fi = fstat[2];
    unsigned short* hrow = zhi ? (unsigned short*)zhi + (size_t)v * ldb : nullptr;
    unsigned short* lrow = zlo ? (unsigned short*)zlo + (size_t)v * ldb : nullptr;
    // two loops, not one with a branch inside: the compiler would evaluate both
    // sides of a short branch, putting the FP64 side on every element
    // (eight loads in flight per thread, as in the moments)
    if (sizeof(T) == 4 && fast) {
        for (int k0 = threadIdx.x; k0 < n; k0 += NT * MU) {
            T x[MU];
#pragma unroll
            for (int u = 0; u < MU; ++u) x[u] = (k0 + u * NT < n) ? row[k0 + u * NT] : T(0);
#pragma unroll
            for (int u = 0; u < MU; ++u) {
                const int k = k0 + u * NT;
                if (k >= n) break;
                const float z = (((float)x[u] - mh) - ml) * fi;
                const unsigned short h = bf16_bits_rn(z);
                hrow[k] = h;
                lrow[k] = bf16_bits_rn(z - bf16_bits_to_float(h));
            }
        }
    } else {
        for (int k0 = threadIdx.x; k0 < n; k0 += NT * MU) {
            T x[MU];
#pragma unroll
            for (int u = 0; u < MU; ++u) x[u] = (k0 + u * NT < n) ? row[k0 + u * NT] : T(0);
#pragma unroll
            for (int u = 0; u < MU; ++u) {
                const int k = k0 + u * NT;
                if (k >= n) break;
                const double d = (double)x[u] - mean;
                if (zrow) zrow[k] = d * inv;
                if (hrow) {
                    const float z = (float)d * fi;
                    const unsigned short h = bf16_bits_rn(z);
                    hrow[k] = h;
                    lrow[k] = bf16_bits_rn(z - bf16_bits_to_float(h));
                }
            }
        }
    }
    // zero the K padding so the tensor-core product can read whole 64-wide slabs
    if (zhi)
        for (int k = n + threadIdx.x; k < kpad; k += NT) {
            ((unsigned short*)zhi)[(size_t)v * ldb + k] = 0;
            ((unsigned short*)zlo)[(size_t)v * ldb + k] = 0;
        }
}

// Standardisation of short rows (one problem, n <= kShortRow, at least 1024
// variables): a warp per variable. With a block per variable, a launch of many short rows waits on
// each block's reductions and its one finishing thread; a warp per variable
// keeps as many variables in flight as the GPU holds warps. Same arithmetic as
// k_standardize: shifted moments of x - K (K = the first sample) in FP64, or in
// compensated FP32 pairs for FP32 data when no FP64 rows are requested, each
// lane's elements in order and a fixed xor tree across the lanes; then the
// mean, 1/sd and the outputs as there.
constexpr int kShortRow = 4096;

template <typename T>
__global__ void __launch_bounds__(256) k_standardize_warp(const T* __restrict__ Xv, long long ld, int n, int p,
                                                          double* __restrict__ mu, double* __restrict__ isd,
                                                          float2* __restrict__ mup, double* __restrict__ z64,
                                                          long long ldz, __nv_bfloat16* __restrict__ zhi,
                                                          __nv_bfloat16* __restrict__ zlo, long long ldb, Meta* meta,
                                                          double inv_n)
{
    const int lane = threadIdx.x & 31;
    const int v = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (v >= p) return;
    const T* row = Xv + (size_t)v * ld;
    double* zrow = z64 ? z64 + (size_t)v * ldz : nullptr;
    const bool fast = (zrow == nullptr);
    const T Kt = row[0];
    double S1 = 0.0, S2 = 0.0;
    bool done = false;
    if constexpr (sizeof(T) == 4) {
        if (fast) {
            const float K = (float)Kt;
            float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f;
            for (int k0 = lane; k0 < n; k0 += 32 * MU) {
                float x[MU];
#pragma unroll
                for (int u = 0; u < MU; ++u) x[u] = (k0 + u * 32 < n) ? (float)row[k0 + u * 32] : 0.f;
#pragma unroll
                for (int u = 0; u < MU; ++u) {
                    if (k0 + u * 32 >= n) break;
                    float dh, dl;
                    two_sum(x[u], -K, dh, dl);
                    pair_add(ah, al, dh, dl);
                    const float pp = __fmul_rn(dh, dh);
                    float q = fmaf(dh, dh, -pp);
                    q = fmaf(2.f * dh, dl, q);
                    float ph, pl;
                    fast_two_sum(pp, q, ph, pl);
                    pair_add(bh, bl, ph, pl);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float xh = __shfl_xor_sync(0xffffffffu, ah, o), xl = __shfl_xor_sync(0xffffffffu, al, o);
                const float yh = __shfl_xor_sync(0xffffffffu, bh, o), yl = __shfl_xor_sync(0xffffffffu, bl, o);
                pair_add(ah, al, xh, xl);
                pair_add(bh, bl, yh, yl);
            }
            S1 = (double)ah + (double)al;
            S2 = (double)bh + (double)bl;
            done = true;
        }
    }
    if (!done) {
        const double Kd = (double)Kt;
        double s1 = 0.0, s2 = 0.0;
        for (int k0 = lane; k0 < n; k0 += 32 * MU) {
            T x[MU];
#pragma unroll
            for (int u = 0; u < MU; ++u) x[u] = (k0 + u * 32 < n) ? row[k0 + u * 32] : T(0);
#pragma unroll
            for (int u = 0; u < MU; ++u) {
                if (k0 + u * 32 >= n) break;
                const double d = (double)x[u] - Kd;
                s1 += d;
                s2 = fma(d, d, s2);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        S1 = s1;
        S2 = s2;
    }
    // mean and 1/sd by lane 0, broadcast (the FP64 pipe is narrow)
    double mean = 0.0, inv = 0.0;
    float mh = 0.f, ml = 0.f, fi = 0.f;
    if (lane == 0) {
        const double K = (double)Kt;
        const double a = S1 * inv_n;
        mean = K + a;
        const double var = fma(-S1, a, S2) * inv_n;
        const bool ok = (var > 0.0) && isfinite(var) && isfinite(mean);
        inv = ok ? rsqrt(var) : 0.0;
        mu[v] = mean;
        isd[v] = inv;
        if (!ok) atomicOr(&meta->error, 1);
        mh = (float)mean;
        ml = (float)(mean - (double)mh);
        fi = (float)inv;
        if (mup) mup[v] = make_float2(mh, ml);
    }
    mean = __shfl_sync(0xffffffffu, mean, 0);
    inv = __shfl_sync(0xffffffffu, inv, 0);
    mh = __shfl_sync(0xffffffffu, mh, 0);
    ml = __shfl_sync(0xffffffffu, ml, 0);
    fi = __shfl_sync(0xffffffffu, fi, 0);
    unsigned short* hrow = zhi ? (unsigned short*)zhi + (size_t)v * ldb : nullptr;
    unsigned short* lrow = zlo ? (unsigned short*)zlo + (size_t)v * ldb : nullptr;
    if (sizeof(T) == 4 && fast) {
        for (int k0 = lane; k0 < n; k0 += 32 * MU) {
            T x[MU];
#pragma unroll
            for (int u = 0; u < MU; ++u) x[u] = (k0 + u * 32 < n) ? row[k0 + u * 32] : T(0);
#pragma unroll
            for (int u = 0; u < MU; ++u) {
                const int k = k0 + u * 32;
                if (k >= n) break;
                const float z = (((float)x[u] - mh) - ml) * fi;
                const unsigned short h = bf16_bits_rn(z);
                hrow[k] = h;
                lrow[k] = bf16_bits_rn(z - bf16_bits_to_float(h));
            }
        }
    } else {
        for (int k0 = lane; k0 < n; k0 += 32 * MU) {
            T x[MU];
#pragma unroll
            for (int u = 0; u < MU; ++u) x[u] = (k0 + u * 32 < n) ? row[k0 + u * 32] : T(0);
#pragma unroll
            for (int u = 0; u < MU; ++u) {
                const int k = k0 + u * 32;
                if (k >= n) break;
                const double d = (double)x[u] - mean;
                if (zrow) zrow[k] = d * inv;
                if (hrow) {
                    const float z = (float)d * fi;
                    const unsigned short h = bf16_bits_rn(z);
                    hrow[k] = h;
                    lrow[k] = bf16_bits_rn(z - bf16_bits_to_float(h));
                }
            }
        }
    }
    if (zhi)
        for (int k = n + lane; k < ldb; k += 32) {
            hrow[k] = 0;
            lrow[k] = 0;
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
                               float2* mup, double* z64, long long ldz, void* zhi, void* zlo, long long ldb,
                               Meta* meta, cudaStream_t st, const int* vprob, const ProbDesc* probs)
{
    constexpr int NT = 256;
    if (!vprob && n <= kShortRow && p >= 1024) {   // (few variables: a block each is quicker)
        const unsigned grid = (unsigned)(((long long)p * 32 + NT - 1) / NT);
        const double inv_n = 1.0 / (double)(n > 0 ? n : 1);
        if (dtype == CUPC_F64)
            k_standardize_warp<double><<<grid, NT, 0, st>>>((const double*)Xv, ld, n, p, mu, isd, mup, z64, ldz,
                                                            (__nv_bfloat16*)zhi, (__nv_bfloat16*)zlo, ldb, meta,
                                                            inv_n);
        else
            k_standardize_warp<float><<<grid, NT, 0, st>>>((const float*)Xv, ld, n, p, mu, isd, mup, z64, ldz,
                                                           (__nv_bfloat16*)zhi, (__nv_bfloat16*)zlo, ldb, meta,
                                                           inv_n);
        return cudaGetLastError();
    }
    if (dtype == CUPC_F64)
        k_standardize<double, NT><<<p, NT, 0, st>>>((const double*)Xv, ld, n, p, mu, isd, mup, z64, ldz,
                                                    (__nv_bfloat16*)zhi, (__nv_bfloat16*)zlo, ldb, meta, vprob,
                                                    probs, 1.0 / (double)(n > 0 ? n : 1));
    else
        k_standardize<float, NT><<<p, NT, 0, st>>>((const float*)Xv, ld, n, p, mu, isd, mup, z64, ldz,
                                                   (__nv_bfloat16*)zhi, (__nv_bfloat16*)zlo, ldb, meta, vprob,
                                                   probs, 1.0 / (double)(n > 0 ? n : 1));
    return cudaGetLastError();
}

cudaError_t launch_transpose_batch(int dtype, const ProbDesc* probs, int nprob, int pmax, int nmax, void* Xt,
                                   cudaStream_t st)
{
    dim3 grid((pmax + 31) / 32, (nmax + 31) / 32, nprob), block(32, 8);
    if (dtype == CUPC_F64)
        k_transpose_batch<double><<<grid, block, 0, st>>>(probs, (double*)Xt);
    else
        k_transpose_batch<float><<<grid, block, 0, st>>>(probs, (float*)Xt);
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
