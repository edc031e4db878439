// cupc_internal.cuh -- device-side building blocks shared by the sm_103a kernels.
//
// Notation follows the paper (Zarebavani et al., TPDS 2019): A_G is the live
// adjacency (a bitset here), A'_G its frozen compaction at the start of a level
// (CSR here), n'_i the degree of row i, l the level (|S|).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cupc.h"

namespace cupc {

constexpr unsigned long long RANK_NONE = ~0ull;
// A conditional variance H11 or H22 at or below this is zero: the variable is a
// linear function of S (C has a unit diagonal, so the scale is absolute).
constexpr double kVarZero = 1e-10;
constexpr int WARP = 32;

// Device counters of one call, read back once per level.
struct Meta {
    unsigned long long tests;          // CI tests executed (this level)
    unsigned long long rechecks;       // FP64 rechecks performed (this level)
    unsigned long long removed;        // edges removed (this level)
    unsigned long long serial_tests;   // serial-order test count (canonical lex runs)
    unsigned long long edges;          // undirected edges at level start
    unsigned long long nnz;            // CSR slots (2 * edges)
    unsigned long long n_items;        // CI work items
    unsigned long long queue_len;      // recheck entries pushed (may exceed capacity)
    unsigned long long rec_ints;       // SepSet record ints appended (may exceed capacity)
    unsigned long long next_item;      // persistent work counter
    unsigned long long block_entries;  // sum over rows with work of (n'_i + 1)^2
    int maxdeg;                        // max n'_i at level start
    int range_error;                   // a subset count saturated 64 bits
    int error;                         // device-side error flags
    int pad;
};

// ---------------------------------------------------------------------------
// Binomial table: binom[k * mstride + m] = C(m, k), saturating at 2^64-1,
// for 0 <= k <= CUPC_MAX_LEVEL + 1 and 0 <= m < mstride.
// ---------------------------------------------------------------------------
struct Binom {
    const unsigned long long* tab;
    int mstride;
    __device__ __forceinline__ unsigned long long operator()(int m, int k) const {
        return (m < 0 || k < 0) ? 0ull : __ldg(tab + (size_t)k * mstride + m);
    }
};

// C(m, k) for m < kBinomS from a copy in shared memory (a level's subset
// unranking does a few dependent lookups per member).
constexpr int kBinomS = 64;
struct BinomS {
    const unsigned long long* tab;   // shared: [k][m], m < kBinomS
    __device__ __forceinline__ unsigned long long operator()(int m, int k) const {
        return (m < 0 || k < 0) ? 0ull : tab[k * kBinomS + m];
    }
};

// The t-th l-subset of the positions {0, .., d-1} in lexicographic order
// (Sec. 4.2, Eq. comb). With k = l - 1 - c members still to place after place
// c, the subsets whose place-c member is >= v number N(v) = C(d - v, k + 1)
// (hockey-stick sum of the counts in Eq. comb); those with a smaller member
// come first. So the member is the largest v with N(prev) - N(v) <= t, found by
// binary search since N falls with v, and t drops by N(prev) - N(v).
// Positions come out increasing; a rank beyond C(d, l) cannot leave the row.
// BT: the table in global memory (Binom) or its small-m part in shared
// memory (BinomS).
template <int LB, typename BT>
__device__ __forceinline__ void unrank_lex(unsigned long long t, int d, int l, const BT& B, int (&P)[LB])
{
    int prev = 0;
#pragma unroll
    for (int c = 0; c < LB; ++c) {
        if (c < l) {
            const int k = l - 1 - c;
            const unsigned long long total = B(d - prev, k + 1);
            const unsigned long long target = total > t ? total - t : 1ull;  // need N(v) >= target
            int lo = prev, hi = max(prev, d - 1 - k);
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (B(d - mid, k + 1) >= target) lo = mid; else hi = mid - 1;
            }
            t -= total - B(d - lo, k + 1);
            P[c] = min(lo, d - 1);
            prev = lo + 1;
        }
    }
}

// Rank of the increasing positions Q[0..l) among the l-subsets of {0..d-1}
// in lexicographic order (inverse of unrank_lex): the subsets skipped at place
// c are N(prev) - N(Q[c]) with N as above.
template <int LB>
__device__ __forceinline__ unsigned long long rank_lex(const int (&Q)[LB], int d, int l, const Binom& B)
{
    unsigned long long r = 0;
    int prev = 0;
#pragma unroll
    for (int c = 0; c < LB; ++c) {
        if (c < l) {
            const int k = l - 1 - c;
            r += B(d - prev, k + 1) - B(d - Q[c], k + 1);
            prev = Q[c] + 1;
        }
    }
    return r;
}

// ---------------------------------------------------------------------------
// Sec. 4.3 arithmetic: with M2 = C[S,S] = L L^T (Cholesky), u = L^-1 C[S,i],
// v = L^-1 C[S,j]:  H11 = 1 - u.u, H22 = 1 - v.v, H12 = C[i,j] - u.v, which
// is H = M0 - M1 M2^-1 M1^T written through the factor (C has a unit
// diagonal). A pivot whose square is <= rank_tol marks that member of S as
// linearly dependent on the earlier ones; it is left out of the projection,
// which gives the same H as the Moore-Penrose route of Algorithm 7.
// ---------------------------------------------------------------------------
template <typename T, int LB>
struct Factor {
    T L[LB * (LB + 1) / 2];   // packed lower triangle, row a at a*(a+1)/2
    T inv[LB];                // 1 / L[a][a] (0 for a dependent member)
    T u[LB];
    T uu;
    T minpiv2;                // smallest pivot^2 (of the kept members)
    unsigned dropped;         // bitmask of dependent members
};

template <typename T> __device__ __forceinline__ T t_sqrt(T x);
template <> __device__ __forceinline__ float t_sqrt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double t_sqrt<double>(double x) { return sqrt(x); }

// Factor M2 given an accessor m2(a, b) for a > b (the diagonal is 1) and
// ci(a) = C[i, S_a].
template <typename T, int LB, typename M2F, typename CIF>
__device__ __forceinline__ void factor_build(Factor<T, LB>& F, int l, T rank_tol, M2F m2, CIF ci)
{
    F.dropped = 0u;
    F.minpiv2 = T(1);
#pragma unroll
    for (int a = 0; a < LB; ++a) {
        if (a < l) {
#pragma unroll
            for (int b = 0; b < LB; ++b) {
                if (b < a) {
                    T s = m2(a, b);
#pragma unroll
                    for (int k = 0; k < LB; ++k)
                        if (k < b) s -= F.L[a * (a + 1) / 2 + k] * F.L[b * (b + 1) / 2 + k];
                    F.L[a * (a + 1) / 2 + b] = s * F.inv[b];
                }
            }
            T s = T(1);
#pragma unroll
            for (int k = 0; k < LB; ++k)
                if (k < a) s -= F.L[a * (a + 1) / 2 + k] * F.L[a * (a + 1) / 2 + k];
            if (s <= rank_tol) {
                F.dropped |= 1u << a;
                F.L[a * (a + 1) / 2 + a] = T(0);
                F.inv[a] = T(0);
            } else {
                const T d = t_sqrt<T>(s);
                F.L[a * (a + 1) / 2 + a] = d;
                F.inv[a] = T(1) / d;
                F.minpiv2 = s < F.minpiv2 ? s : F.minpiv2;
            }
        }
    }
    // u = L^-1 c_i (forward substitution; dependent members get 0)
    T uu = T(0);
#pragma unroll
    for (int a = 0; a < LB; ++a) {
        if (a < l) {
            T s = ci(a);
#pragma unroll
            for (int k = 0; k < LB; ++k)
                if (k < a) s -= F.L[a * (a + 1) / 2 + k] * F.u[k];
            F.u[a] = s * F.inv[a];
            uu += F.u[a] * F.u[a];
        }
    }
    F.uu = uu;
}

// For one j: H12 and H22 given cj(a) = C[j, S_a] and cij = C[i, j].
template <typename T, int LB, typename CJF>
__device__ __forceinline__ void factor_apply(const Factor<T, LB>& F, int l, T cij, CJF cj, T& H12, T& H22)
{
    T v[LB];
    T vv = T(0), uv = T(0);
#pragma unroll
    for (int a = 0; a < LB; ++a) {
        if (a < l) {
            T s = cj(a);
#pragma unroll
            for (int k = 0; k < LB; ++k)
                if (k < a) s -= F.L[a * (a + 1) / 2 + k] * v[k];
            v[a] = s * F.inv[a];
            vv += v[a] * v[a];
            uv += F.u[a] * v[a];
        }
    }
    H12 = cij - uv;
    H22 = T(1) - vv;
}

// ---------------------------------------------------------------------------
// Bitset adjacency: row i has W = ceil(p/32) words; bit b of word w is j=32w+b.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bitset_clear_pair(unsigned* bits, int W, int i, int j)
{
    atomicAnd(bits + (size_t)i * W + (j >> 5), ~(1u << (j & 31)));
    atomicAnd(bits + (size_t)j * W + (i >> 5), ~(1u << (i & 31)));
}

// Same with the row starts given (rb_i: word of column 0 in row i).
__device__ __forceinline__ void bitset_clear_pair_at(unsigned* bits, long long rb_i, long long rb_j, int i, int j)
{
    atomicAnd(bits + rb_i + (j >> 5), ~(1u << (j & 31)));
    atomicAnd(bits + rb_j + (i >> 5), ~(1u << (i & 31)));
}

__device__ __forceinline__ bool bitset_test(const unsigned* bits, int W, int i, int j)
{
    return (bits[(size_t)i * W + (j >> 5)] >> (j & 31)) & 1u;
}

// ---------------------------------------------------------------------------
// Standardised value z = ((double)x - mu) * isd of one variable, recomputed
// in FP64 from its variable-major data row (FP32 or FP64) and the moments of
// the standardisation: the centring rounds once, the scaling once.
// ---------------------------------------------------------------------------
// FP32 -> FP64 widening (exact) by integer operations on the IEEE encodings:
// normal numbers get the exponent rebiased from 127 to 1023 and the mantissa
// shifted left by 29; zeros keep the sign; subnormals (m 2^-149) are
// normalised at their leading one; infinities and NaNs keep the all-ones
// exponent. GB300 issues the conversion instruction on its narrow FP64 pipe.
__device__ __forceinline__ double widen_f32(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned m = u & 0x7fffffu;
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    unsigned long long ex, man;
    if (e != 0u) {
        ex = (e == 0xffu) ? 2047ull : (unsigned long long)(e + 896u);
        man = (unsigned long long)m << 29;
    } else if (m != 0u) {
        const int lead = 31 - __clz((int)m);                 // bit of the leading one, 0..22
        ex = (unsigned long long)(lead + 874);               // 2^(lead - 149)
        man = ((unsigned long long)m << (52 - lead)) & ((1ull << 52) - 1ull);
    } else {
        ex = 0ull;
        man = 0ull;
    }
    return __longlong_as_double((long long)(sign | (ex << 52) | man));
}

// ---------------------------------------------------------------------------
// Compensated FP32 pairs ("double-word" numbers hi + lo): Knuth's two-sum,
// Dekker's fast two-sum (|a| >= |b|) and the accurate pair addition of
// Joldes, Muller and Popescu (2017), relative error below 3 * 2^-48. GB300
// runs FP32 at many times its FP64 rate. The roundings are spelled out
// (__fadd_rn, __fmul_rn), so no contraction into a fused multiply-add can
// change an error-free transformation.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void pair_add(float& xh, float& xl, float yh, float yl)
{
    float sh, sl, th, tl, vh, vl;
    two_sum(xh, yh, sh, sl);
    two_sum(xl, yl, th, tl);
    sl = __fadd_rn(sl, th);
    fast_two_sum(sh, sl, vh, vl);
    vl = __fadd_rn(vl, tl);
    fast_two_sum(vh, vl, xh, xl);
}

// S += (ah + al)(bh + bl) for a pair accumulator (Sh, Sl) kept in the
// compensated-dot form of Ogita, Rump and Oishi (2005): the product's leading
// float, its exact rounding error (fma) and the cross terms, the leading sum's
// error by two-sum, all errors gathered in Sl. Sl is folded back into Sh
// (two_sum) every few terms by the caller.
__device__ __forceinline__ void pair_dot_acc(float& Sh, float& Sl, float ah, float al, float bh, float bl)
{
    const float ph = __fmul_rn(ah, bh);
    float pe = fmaf(ah, bh, -ph);
    pe = fmaf(ah, bl, pe);
    pe = fmaf(al, bh, pe);
    pe = fmaf(al, bl, pe);
    float s, e;
    two_sum(Sh, ph, s, e);
    Sh = s;
    Sl = __fadd_rn(Sl, __fadd_rn(e, pe));
}

// One FP32 variable's row for the compensated rechecks: x - mu as a pair
// (dh, dl), the FP64 mean given as the pair mh + ml (2^-48 relative):
// x - mh exactly by two-sum, then minus ml.
struct XRowP {
    const float* p;
    float mh, ml;
    __device__ __forceinline__ void centred(int k, float& dh, float& dl) const
    {
        float e;
        two_sum(__ldg(p + k), -mh, dh, e);
        dl = __fsub_rn(e, ml);
    }
};

// One variable's row for the rechecks: its variable-major data (FP32 or FP64)
// and the moments of the standardisation, z = (x - mu) * isd. The Gram sums
// below accumulate the centred values x - mu and apply isd_a isd_b once.
struct XRow {
    const void* p;
    int f64;
    double mu, isd;
    __device__ __forceinline__ double centred(int k) const
    {
        const double x = f64 ? __ldg((const double*)p + k) : widen_f32(__ldg((const float*)p + k));
        return x - mu;
    }
};

// ---------------------------------------------------------------------------
// FP64 block of C for the rechecks: for the m variables with rows R, the
// strictly lower packed entries G[b(b-1)/2 + a] = C[V_a, V_b] (a < b) by the
// definition C_ab = sum_s z_as z_bs / n = isd_a isd_b sum_s (x_as - mu_a)
// (x_bs - mu_b) / n, every pair in one pass (threads of the block stride the
// samples), then a fixed-order block reduction -- an entry's value does not
// depend on the test it serves. Must be called by all NT threads of the
// block; red holds (NT/32) * M(M-1)/2 doubles.
// ---------------------------------------------------------------------------
template <int M, int NT>
__device__ __forceinline__ void c_block(const XRow (&R)[M], int n, int m, double (&G)[M * (M - 1) / 2], double* red)
{
    constexpr int D = M * (M - 1) / 2;
#pragma unroll
    for (int q = 0; q < D; ++q) G[q] = 0.0;
#pragma unroll 4
    for (int k = threadIdx.x; k < n; k += NT) {
        double x[M];
#pragma unroll
        for (int a = 0; a < M; ++a) x[a] = (a < m) ? R[a].centred(k) : 0.0;
#pragma unroll
        for (int b = 1; b < M; ++b)
#pragma unroll
            for (int a = 0; a < b; ++a) G[b * (b - 1) / 2 + a] = fma(x[a], x[b], G[b * (b - 1) / 2 + a]);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < D; ++q) {
        double g = G[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        if (lane == 0) red[w * D + q] = g;
    }
    __syncthreads();
    const double inv_n = 1.0 / (double)n;
#pragma unroll
    for (int b = 1; b < M; ++b)
#pragma unroll
        for (int a = 0; a < b; ++a) {
            const int q = b * (b - 1) / 2 + a;
            double g = 0.0;
#pragma unroll
            for (int k = 0; k < NT / 32; ++k) g += red[k * D + q];
            G[q] = g * (R[a].isd * R[b].isd) * inv_n;
        }
    __syncthreads();
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Recheck queue entry of a level >= 1 test (slot e of row i, subset rank s
// over the row and the members of S), or of a level-0 pair (i, j).
struct QEntry {
    int a;                      // slot e (level >= 1) or i (level 0)
    int b;                      // unused (level >= 1) or j (level 0)
    unsigned long long s;       // subset rank
    int S[CUPC_MAX_LEVEL];      // members of S (level >= 1)
};

}  // namespace cupc
