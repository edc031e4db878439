// k_ci.cu -- the persistent per-level CI-test kernel (levels l >= 1).
//
// Work decomposition (cf. cuPC-S, Sec. 3.4, Algorithm 5, used here as prior
// art): a row i of the frozen compaction A'_G has n'_i neighbours and
// C(n'_i, l) candidate sets S. Work items are (row, range of subset ranks);
// warps pull items from a device counter until none are left. Each lane owns
// one S per round: it unranks S (Sec. 4.2), factors M2 = C[S,S] once and then
// tests every j of the row not in S against it (S shared within the row), so
// one factorisation serves up to n'_i - l tests.
//
// Early termination (Sec. 4.1): a test (S, j) is skipped when the slot (i, j)
// already holds a separating set of smaller rank (canonical mode: the
// lexicographically first S must still be found) or any separating set (free
// mode), and on the larger endpoint's side when the smaller side has one.
//
// FP32 mode: tests whose |rho| lies within a band of tanh(tau) -- widened for
// ill-conditioned M2 and small conditional variances -- are not decided in
// FP32; they go to the FP64 recheck queue.
#include "kernels.cuh"

namespace cupc {

template <typename T, bool FP32>
__device__ __forceinline__ int ci_decide(T H11, T H12, T H22, T minpiv2, const CIParams& P)
{
    if (!FP32) {
        // zero conditional variance (rounding level of the unit diagonal): V_i or
        // V_j is a linear function of S -> independent
        if (!(H11 > T(kVarZero)) || !(H22 > T(kVarZero))) return 1;
        return (H12 * H12 <= (T)P.r2 * H11 * H22) ? 1 : 0;
    } else {
        if (!(minpiv2 >= (T)P.piv_floor) || !(H11 > T(1e-4)) || !(H22 > T(1e-4))) return 2;
        const float rho = fabsf((float)H12) * rsqrtf((float)(H11 * H22));
        const float band = (float)P.band_abs + (float)P.band_rel / ((float)minpiv2 * fminf((float)H11, (float)H22));
        const float r = (float)P.r;
        if (rho > r + band) return 0;
        if (rho < r - band) return 1;
        return 2;
    }
}

template <typename T, int LB, bool FP32>
__global__ void __launch_bounds__(256) k_ci(CIParams P)
{
    const int lane = threadIdx.x & 31;
    const T* __restrict__ C = (const T*)P.C;
    const int p = P.p, l = P.l;
    unsigned long long ntests = 0;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(&P.meta->next_item, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= P.n_items) break;
        const int i = P.item_row[item];
        const long long k = (long long)item - P.item_off[i];
        const long long off = P.row_off[i];
        const int d = (int)(P.row_off[i + 1] - off);
        const unsigned long long nsets = P.B(d, l);
        const unsigned long long s0 = (unsigned long long)k * (unsigned long long)P.chunk;
        const unsigned long long s1 = min(s0 + (unsigned long long)P.chunk, nsets);
        const T* __restrict__ Ci = C + (size_t)i * p;
        for (unsigned long long base = s0; base < s1; base += 32) {
            const unsigned long long s = base + lane;
            const bool active = s < s1;
            int Pos[LB], Sx[LB];
            Factor<T, LB> F;
#pragma unroll
            for (int c = 0; c < LB; ++c) { Pos[c] = -1; Sx[c] = 0; }
            if (active) {
                unrank_lex<LB>(s, d, l, P.B, Pos);
#pragma unroll
                for (int c = 0; c < LB; ++c)
                    if (c < l) Sx[c] = __ldg(P.cols + off + Pos[c]);
                factor_build<T, LB>(
                    F, l, (T)P.rank_tol,
                    [&](int a, int b) { return __ldg(C + (size_t)Sx[a] * p + Sx[b]); },
                    [&](int a) { return __ldg(Ci + Sx[a]); });
            }
            for (int jp = 0; jp < d; ++jp) {
                const long long e = off + jp;
                bool t = active;
#pragma unroll
                for (int c = 0; c < LB; ++c)
                    if (c < l && Pos[c] == jp) t = false;
                if (!__any_sync(0xffffffffu, t)) continue;
                const int j = __ldg(P.cols + e);
                if (t) {
                    const unsigned long long be = P.best[e];
                    if (P.canonical ? (be < s) : (be != RANK_NONE)) t = false;
                }
                if (t && (!P.canonical || i > j)) {
                    if (P.best[__ldg(P.partner + e)] != RANK_NONE) t = false;
                }
                if (t) {
                    T H12, H22;
                    const T* __restrict__ Cj = C + (size_t)j * p;
                    factor_apply<T, LB>(F, l, __ldg(Ci + j), [&](int a) { return __ldg(Cj + Sx[a]); }, H12, H22);
                    const T H11 = T(1) - F.uu;
                    ++ntests;
                    const int dec = ci_decide<T, FP32>(H11, H12, H22, F.minpiv2, P);
                    if (dec == 1) {
                        atomicMin(P.best + e, s);
                    } else if (FP32 && dec == 2) {
                        const unsigned long long q = atomicAdd(&P.meta->queue_len, 1ull);
                        if (q < P.qcap) P.queue[q] = QEntry{(int)e, 0, s};
                    }
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ntests += __shfl_xor_sync(0xffffffffu, ntests, o);
    if (lane == 0 && ntests) atomicAdd(&P.meta->tests, ntests);
}

template <typename T, bool FP32>
static cudaError_t launch_ci_t(const CIParams& P, int grid, int block, cudaStream_t st)
{
    if (P.l <= 1) k_ci<T, 1, FP32><<<grid, block, 0, st>>>(P);
    else if (P.l <= 2) k_ci<T, 2, FP32><<<grid, block, 0, st>>>(P);
    else if (P.l <= 4) k_ci<T, 4, FP32><<<grid, block, 0, st>>>(P);
    else if (P.l <= 8) k_ci<T, 8, FP32><<<grid, block, 0, st>>>(P);
    else k_ci<T, 16, FP32><<<grid, block, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_ci(int fp32, const CIParams& P, int grid, int block, cudaStream_t st)
{
    return fp32 ? launch_ci_t<float, true>(P, grid, block, st) : launch_ci_t<double, false>(P, grid, block, st);
}

int ci_max_level_supported() { return 16; }

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
