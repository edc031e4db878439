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

// The t-th l-subset of the positions {0, .., d-1} in lexicographic order
// (Sec. 4.2, Eq. comb): for each place c, step the value forward while the
// number of subsets that start with the current prefix is <= the remaining
// rank, subtracting those counts. Positions come out increasing.
template <int LB>
__device__ __forceinline__ void unrank_lex(unsigned long long t, int d, int l, const Binom& B,
                                           int (&P)[LB])
{
    int v = 0;
#pragma unroll
    for (int c = 0; c < LB; ++c) {
        if (c < l) {
            const int k = l - 1 - c;
            // bounded by d: a rank beyond C(d, l) cannot run past the row
            for (; v < d - 1; ++v) {
                const unsigned long long cnt = B(d - 1 - v, k);
                if (t < cnt) break;
                t -= cnt;
            }
            P[c] = v < d ? v : d - 1;
            ++v;
        }
    }
}

// Rank of the increasing positions Q[0..l) among the l-subsets of {0..d-1}
// in lexicographic order (inverse of unrank_lex).
template <int LB>
__device__ __forceinline__ unsigned long long rank_lex(const int (&Q)[LB], int d, int l, const Binom& B)
{
    unsigned long long r = 0;
    int prev = -1;
#pragma unroll
    for (int c = 0; c < LB; ++c) {
        if (c < l) {
            const int k = l - 1 - c;
            for (int v = prev + 1; v < Q[c]; ++v) r += B(d - 1 - v, k);
            prev = Q[c];
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

__device__ __forceinline__ bool bitset_test(const unsigned* bits, int W, int i, int j)
{
    return (bits[(size_t)i * W + (j >> 5)] >> (j & 31)) & 1u;
}

// Recheck queue entry of a level >= 1 test (slot e of row i; subset rank s over
// the row), or of a level-0 pair (i, j) with rank unused.
struct QEntry {
    int a;                      // slot e (level >= 1) or i (level 0)
    int b;                      // unused (level >= 1) or j (level 0)
    unsigned long long s;       // subset rank
};

}  // namespace cupc
