// k_graph.cu -- level 0 (Algorithm 3) with its FP64 rechecks, the degree and
// offset scan used to size the level buffers, and small utilities.
#include "kernels.cuh"

namespace cupc {

// ---------------------------------------------------------------------------
// Level 0 (Algorithm 3, Sec. 4.3: rho = C[i,j] for S empty). One warp per row
// i; lane b decides j = 32w + b and the warp ballot forms adjacency word w.
// Independent iff |C_ij| <= tanh(tau_0) (the Fisher-z rule with atanh
// monotone). In FP32 mode |C_ij| within band0 of the threshold keeps the
// edge for now and queues the pair (once, from the i < j side) for FP64.
// ---------------------------------------------------------------------------
// In a batch (descriptors given) row i reads its problem's block of C, its
// threshold, and writes only its problem's words; padding rows stay empty.
template <typename T, bool FP32>
__global__ void k_level0(const T* __restrict__ C, int p, int W, double r0, double band0, unsigned* __restrict__ bits,
                         QEntry* __restrict__ q, unsigned long long qcap, Meta* meta, const int* __restrict__ vprob,
                         const ProbDesc* __restrict__ probs, int nrows)
{
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= nrows) return;
    const ProbDesc* D = prob_of(vprob, probs, i);
    const int off = D ? D->off : 0, pp = D ? D->p : p;
    const int wlo = D ? D->wlo : 0, whi = D ? D->whi : W;
    const long long rb = rowbase(D, W, i);
    const bool live = i - off < pp;
    const T* row = C + (D ? D->c_off : 0) + (long long)(i - off) * pp - off;
    if (D) r0 = D->r[0];
    const T hi = (T)(r0 + band0), lo = (T)(r0 - band0);  // FP32 band edges
    // eight words at a time: their loads are issued before any is used
    constexpr int U = 8;
    for (int w0 = wlo; w0 < whi; w0 += U) {
        T cv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = ((w0 + u) << 5) + lane;
            cv[u] = (w0 + u < whi && live && j - off < pp && j != i) ? row[j] : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
        const int w = w0 + u;
        if (w >= whi) break;
        const int j = (w << 5) + lane;
        bool keep = false;
        if (live && j - off < pp && j != i) {
            const T c = cv[u] < T(0) ? -cv[u] : cv[u];
            if (!FP32) {
                keep = !(c <= (T)r0);
            } else {
                if (c > hi) keep = true;
                else if (c < lo) keep = false;
                else {
                    keep = true;
                    if (i < j) {
                        const unsigned long long k = atomicAdd(&meta->queue_len, 1ull);
                        if (k < qcap) {
                            q[k].a = i;
                            q[k].b = j;
                            q[k].s = 0ull;
                        }
                    }
                }
            }
        }
        const unsigned word = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) bits[rb + w] = word;
        }
    }
}

// Level 0 of one problem on the upper triangle of C only (C is exactly
// symmetric): a warp owns the 32 x 32 tile of rows 32 bi.. and columns 32 bj..,
// bi <= bj, reads it row by row (one coalesced 128-byte line per row), and
// writes word bj of its rows (a ballot per row) and, for bi < bj, word bi of its
// columns' rows (each lane collects its column's 32 bits). Every bitset word is
// written by exactly one tile, so no atomics; half of C is read.
template <typename T, bool FP32>
__global__ void k_level0_tri(const T* __restrict__ C, int p, int W, double r0, double band0,
                             unsigned* __restrict__ bits, QEntry* __restrict__ q, unsigned long long qcap,
                             Meta* meta, long long ntiles)
{
    const int lane = threadIdx.x & 31;
    const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= ntiles) return;
    // tile t of the upper triangle in row-major order: bi, then bj >= bi
    int bi = 0;
    {
        // rows bi hold W - bi tiles; invert t = bi W - bi (bi - 1) / 2 + (bj - bi)
        long long lo = 0, hi = W - 1;
        while (lo < hi) {
            const long long mid = (lo + hi + 1) >> 1;
            const long long first = mid * W - mid * (mid - 1) / 2;
            if (first <= t) lo = mid; else hi = mid - 1;
        }
        bi = (int)lo;
    }
    const int bj = bi + (int)(t - ((long long)bi * W - (long long)bi * (bi - 1) / 2));
    const int j = (bj << 5) + lane;
    const bool jin = j < p;
    const T hi = (T)(r0 + band0), lo = (T)(r0 - band0);  // FP32 band edges
    T cv[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const int i = (bi << 5) + r;
        cv[r] = (i < p && jin) ? C[(long long)i * p + j] : T(0);
    }
    unsigned colmask = 0u;   // bit r: pair (32 bi + r, j) kept
    unsigned myrow = 0u;     // diagonal tile: row 32 bi + lane's bits towards j > i
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const int i = (bi << 5) + r;
        // each pair is decided once, from its i < j side
        bool keep = false;
        if (i < p && jin && j > i) {
            const T c = cv[r] < T(0) ? -cv[r] : cv[r];
            if (!FP32) {
                keep = !(c <= (T)r0);
            } else if (c > hi) {
                keep = true;
            } else if (c >= lo) {
                keep = true;                   // within the band: kept for now, queued
                const unsigned long long k = atomicAdd(&meta->queue_len, 1ull);
                if (k < qcap) {
                    q[k].a = i;
                    q[k].b = j;
                    q[k].s = 0ull;
                }
            }
        }
        const unsigned word = __ballot_sync(0xffffffffu, keep);
        if (keep) colmask |= 1u << r;
        if (bi != bj) {
            if (lane == 0 && i < p) bits[(long long)i * W + bj] = word;
        } else if (lane == r) {
            myrow = word;
        }
    }
    if (bi != bj) {
        // the transposed words: row j's bits towards rows 32 bi ..
        if (jin) bits[(long long)j * W + bi] = colmask;
    } else {
        // diagonal tile: row 32 bi + lane keeps its j > i bits (its ballot) and
        // its j < i bits (the pairs decided in the earlier rows, collected in
        // this lane's column mask)
        const int i = (bi << 5) + lane;
        if (i < p) bits[(long long)i * W + bi] = myrow | colmask;
    }
}

cudaError_t launch_level0(int fp32, const void* C, int p, int W, double r0, double band0, unsigned* bits,
                          QEntry* q, unsigned long long qcap, Meta* meta, cudaStream_t st, const int* vprob,
                          const ProbDesc* probs, int nrows)
{
    if (!vprob) {
        // one problem: the upper-triangle form
        const long long ntiles = (long long)W * (W + 1) / 2;
        const int block = 256;
        const long long grid = (ntiles * 32 + block - 1) / block;
        if (fp32)
            k_level0_tri<float, true><<<(unsigned)grid, block, 0, st>>>((const float*)C, p, W, r0, band0, bits, q,
                                                                         qcap, meta, ntiles);
        else
            k_level0_tri<double, false><<<(unsigned)grid, block, 0, st>>>((const double*)C, p, W, r0, band0, bits,
                                                                           q, qcap, meta, ntiles);
        return cudaGetLastError();
    }
    const int block = 256, grid = (int)(((long long)nrows * 32 + block - 1) / block);
    if (fp32)
        k_level0<float, true><<<grid, block, 0, st>>>((const float*)C, p, W, r0, band0, bits, q, qcap, meta, vprob,
                                                      probs, nrows);
    else
        k_level0<double, false><<<grid, block, 0, st>>>((const double*)C, p, W, r0, band0, bits, q, qcap, meta,
                                                        vprob, probs, nrows);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Compaction (Sec. 3.3 "Compact"): degrees, one block scan for the CSR offsets
// and the work-item offsets, then each row's sorted neighbour list.
// ---------------------------------------------------------------------------
__global__ void k_degree(const unsigned* __restrict__ bits, int p, int W, int* __restrict__ deg, Meta* meta,
                         const int* __restrict__ vprob, const ProbDesc* __restrict__ probs)
{
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= p) return;
    const ProbDesc* D = prob_of(vprob, probs, i);
    const int wlo = D ? D->wlo : 0, whi = D ? D->whi : W;
    const long long rb = rowbase(D, W, i);
    int c = 0;
    for (int w = wlo + lane; w < whi; w += 32) c += __popc(bits[rb + w]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) {
        deg[i] = c;
        atomicMax(&meta->maxdeg, c);
        if (c) atomicAdd(&meta->nnz, (unsigned long long)c);
    }
}

cudaError_t launch_degree(const unsigned* bits, int p, int W, int* deg, Meta* meta, cudaStream_t st,
                          const int* vprob, const ProbDesc* probs)
{
    const int block = 256, grid = (int)(((long long)p * 32 + block - 1) / block);
    k_degree<<<grid, block, 0, st>>>(bits, p, W, deg, meta, vprob, probs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Level-0 FP64 rechecks: one block per queued pair (S empty: rho = C_ij).
// FP32 data: the centred sum in compensated FP32 pairs (every thread strides
// the samples in the compensated-dot form, folded every 8 samples; a fixed
// xor tree per warp, the warps in order), widened to FP64 once; FP64 data:
// the FP64 block sum.
// ---------------------------------------------------------------------------
constexpr int RC_THREADS = 256;

__device__ __forceinline__ double pair_centred_dot(const XRowP& A, const XRowP& B, int n, float2* red)
{
    float sh = 0.f, sl = 0.f;
    for (int kb = threadIdx.x; kb < n; kb += RC_THREADS * 8) {
        const int ke = min(n, kb + RC_THREADS * 8);
#pragma unroll 8
        for (int k = kb; k < ke; k += RC_THREADS) {
            float ah, al, bh, bl;
            A.centred(k, ah, al);
            B.centred(k, bh, bl);
            pair_dot_acc(sh, sl, ah, al, bh, bl);
        }
        two_sum(sh, sl, sh, sl);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl, o);
        pair_add(sh, sl, oh, ol);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = make_float2(sh, sl);
    __syncthreads();
    double g = 0.0;
    if (threadIdx.x == 0) {
        float h = red[0].x, l = red[0].y;
        for (int k = 1; k < RC_THREADS / 32; ++k) pair_add(h, l, red[k].x, red[k].y);
        g = widen_f32(h) + widen_f32(l);
    }
    __syncthreads();
    return g;  // valid in thread 0
}

__global__ void __launch_bounds__(RC_THREADS) k_recheck0(Recheck0Params P)
{
    __shared__ double red[RC_THREADS / 32];
    __shared__ float2 redp[RC_THREADS / 32];
    unsigned long long nq = P.meta->queue_len;
    if (nq > P.qcap) nq = P.qcap;
    unsigned long long done = 0;
    for (long long qi = blockIdx.x; qi < (long long)nq; qi += gridDim.x) {
        const QEntry E = P.queue[qi];
        const ProbDesc* D = prob_of(P.vprob, P.probs, E.a);
        double G[1];
        if (P.c64) {
            G[0] = P.c64[(size_t)E.a * P.p + E.b];
        } else if (!P.xf64) {
            // FP32 data rows of the pair (a batch problem's own rows, its sample count)
            const int n = D ? D->n : P.n;
            XRowP R[2];
            const int V[2] = {E.a, E.b};
            for (int a = 0; a < 2; ++a) {
                const float2 m = P.mup[V[a]];
                R[a].mh = m.x;
                R[a].ml = m.y;
                R[a].p = D ? (const float*)D->xv + (size_t)(V[a] - D->off) * D->n
                           : (const float*)P.xv + (size_t)V[a] * P.ldx;
            }
            const double g = pair_centred_dot(R[0], R[1], n, redp);
            G[0] = g * (P.isd[E.a] * P.isd[E.b]) * (D ? D->inv_n : P.inv_n);
        } else {
            // the pair's FP64 data rows
            const int V[2] = {E.a, E.b};
            XRow R[2];
            for (int a = 0; a < 2; ++a) {
                R[a].f64 = 1;
                R[a].mu = P.mu[V[a]];
                R[a].isd = P.isd[V[a]];
                R[a].p = D ? (const char*)D->xv + (size_t)(V[a] - D->off) * D->n * 8
                           : (const char*)P.xv + (size_t)V[a] * P.ldx * 8;
            }
            c_block<2, RC_THREADS>(R, D ? D->n : P.n, 2, G, red);
        }
        // independent iff rho^2 <= tanh(tau_0)^2
        const double r2 = D ? D->r2[0] : P.r2;
        if (threadIdx.x == 0 && G[0] * G[0] <= r2)
            bitset_clear_pair_at(P.bits, rowbase(D, P.W, E.a), rowbase(D, P.W, E.b), E.a, E.b);
        ++done;
    }
    if (threadIdx.x == 0 && done) atomicAdd(&P.meta->rechecks, done);
}

cudaError_t launch_recheck0(const Recheck0Params& P, int grid, cudaStream_t st)
{
    k_recheck0<<<grid, RC_THREADS, 0, st>>>(P);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Utilities
// ---------------------------------------------------------------------------
template <typename Tin>
__global__ void k_symmetrize(const Tin* __restrict__ Cin, long long ld, int p, double* __restrict__ C64,
                             float* __restrict__ C32)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)p * p) return;
    const int i = (int)(k / p), j = (int)(k % p);
    const int a = min(i, j), b = max(i, j);
    const double v = (i == j) ? 1.0 : (double)Cin[(size_t)a * ld + b];
    if (C64) C64[k] = v;
    if (C32) C32[k] = (float)v;
}

cudaError_t launch_symmetrize(int dtype, const void* Cin, long long ld, int p, double* C64, float* C32,
                              cudaStream_t st)
{
    const long long tot = (long long)p * p;
    const int block = 256;
    const unsigned grid = (unsigned)((tot + block - 1) / block);
    if (dtype == CUPC_F64) k_symmetrize<double><<<grid, block, 0, st>>>((const double*)Cin, ld, p, C64, C32);
    else k_symmetrize<float><<<grid, block, 0, st>>>((const float*)Cin, ld, p, C64, C32);
    return cudaGetLastError();
}

__global__ void k_bits_to_u8(const unsigned* __restrict__ bits, int p, int W, unsigned char* __restrict__ out)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)p * p) return;
    const int i = (int)(k / p), j = (int)(k % p);
    out[k] = (unsigned char)((bits[(size_t)i * W + (j >> 5)] >> (j & 31)) & 1u);
}

cudaError_t launch_bits_to_u8(const unsigned* bits, int p, int W, unsigned char* out, cudaStream_t st)
{
    const long long tot = (long long)p * p;
    const int block = 256;
    k_bits_to_u8<<<(unsigned)((tot + block - 1) / block), block, 0, st>>>(bits, p, W, out);
    return cudaGetLastError();
}

}  // namespace cupc
