// k_graph.cu -- level 0, compaction of A_G into A'_G, FP64 rechecks and the
// per-level finalisation (edge removal from G, SepSet records).
#include "kernels.cuh"

namespace cupc {

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// ---------------------------------------------------------------------------
// Level 0 (Algorithm 3, Sec. 4.3: rho = C[i,j] for S empty). One warp per row
// i; lane b decides j = 32w + b and the warp ballot forms adjacency word w.
// Independent iff |C_ij| <= tanh(tau_0) (the Fisher-z rule with atanh
// monotone). In FP32 mode |C_ij| within band0 of the threshold keeps the
// edge for now and queues the pair (once, from the i < j side) for FP64.
// ---------------------------------------------------------------------------
template <typename T, bool FP32>
__global__ void k_level0(const T* __restrict__ C, int p, int W, double r0, double band0, unsigned* __restrict__ bits,
                         QEntry* __restrict__ q, unsigned long long qcap, Meta* meta)
{
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= p) return;
    const T* row = C + (size_t)i * p;
    for (int w = 0; w < W; ++w) {
        const int j = (w << 5) + lane;
        bool keep = false;
        if (j < p && j != i) {
            const double c = fabs((double)row[j]);
            if (!FP32) {
                keep = !(c <= r0);
            } else {
                if (c > r0 + band0) keep = true;
                else if (c < r0 - band0) keep = false;
                else {
                    keep = true;
                    if (i < j) {
                        const unsigned long long k = atomicAdd(&meta->queue_len, 1ull);
                        if (k < qcap) q[k] = QEntry{i, j, 0ull};
                    }
                }
            }
        }
        const unsigned word = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) bits[(size_t)i * W + w] = word;
    }
}

cudaError_t launch_level0(int fp32, const void* C, int p, int W, double r0, double band0, unsigned* bits,
                          QEntry* q, unsigned long long qcap, Meta* meta, cudaStream_t st)
{
    const int block = 256, grid = (p * 32 + block - 1) / block;
    if (fp32)
        k_level0<float, true><<<grid, block, 0, st>>>((const float*)C, p, W, r0, band0, bits, q, qcap, meta);
    else
        k_level0<double, false><<<grid, block, 0, st>>>((const double*)C, p, W, r0, band0, bits, q, qcap, meta);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Compaction (Sec. 3.3 "Compact"): degrees, one block scan for the CSR offsets
// and the work-item offsets, then each row's sorted neighbour list.
// ---------------------------------------------------------------------------
__global__ void k_degree(const unsigned* __restrict__ bits, int p, int W, int* __restrict__ deg, Meta* meta)
{
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= p) return;
    int c = 0;
    for (int w = lane; w < W; w += 32) c += __popc(bits[(size_t)i * W + w]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) {
        deg[i] = c;
        atomicMax(&meta->maxdeg, c);
    }
}

cudaError_t launch_degree(const unsigned* bits, int p, int W, int* deg, Meta* meta, cudaStream_t st)
{
    const int block = 256, grid = (p * 32 + block - 1) / block;
    k_degree<<<grid, block, 0, st>>>(bits, p, W, deg, meta);
    return cudaGetLastError();
}

// Single-block exclusive scans of deg (CSR offsets) and of the per-row work
// items (rows with n'_i >= l + 1 get ceil(C(n'_i, l) / chunk) items).
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ deg, int p, int l, int chunk, Binom B,
                                               long long* __restrict__ row_off, long long* __restrict__ item_off,
                                               Meta* meta)
{
    __shared__ long long sa[32], sb[32];
    const int t = threadIdx.x, NT = blockDim.x;
    const int per = (p + NT - 1) / NT;
    const int lo = min(p, t * per), hi = min(p, lo + per);
    long long a = 0, b = 0;
    unsigned long long sq = 0;
    int rng = 0;
    for (int i = lo; i < hi; ++i) {
        const int d = deg[i];
        a += d;
        if (d >= l + 1) {
            const unsigned long long ns = B(d, l);
            if (ns == ~0ull) rng = 1;
            b += (long long)((ns + chunk - 1) / chunk);
            sq += (unsigned long long)(d + 1) * (unsigned long long)(d + 1);
        }
    }
    {
        unsigned long long t2 = sq;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t2 += __shfl_xor_sync(0xffffffffu, t2, o);
        if ((threadIdx.x & 31) == 0 && t2) atomicAdd(&meta->block_entries, t2);
    }
    // block exclusive scan of (a, b)
    const int lane = t & 31, w = t >> 5;
    long long ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long xa = __shfl_up_sync(0xffffffffu, ia, o);
        const long long xb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) { ia += xa; ib += xb; }
    }
    if (lane == 31) { sa[w] = ia; sb[w] = ib; }
    __syncthreads();
    if (w == 0) {
        long long va = (lane < NT / 32) ? sa[lane] : 0, vb = (lane < NT / 32) ? sb[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long xa = __shfl_up_sync(0xffffffffu, va, o);
            const long long xb = __shfl_up_sync(0xffffffffu, vb, o);
            if (lane >= o) { va += xa; vb += xb; }
        }
        sa[lane] = va;
        sb[lane] = vb;
    }
    __syncthreads();
    long long ea = ia - a + (w > 0 ? sa[w - 1] : 0);
    long long eb = ib - b + (w > 0 ? sb[w - 1] : 0);
    for (int i = lo; i < hi; ++i) {
        const int d = deg[i];
        row_off[i] = ea;
        item_off[i] = eb;
        ea += d;
        if (d >= l + 1) {
            const unsigned long long ns = B(d, l);
            eb += (long long)((ns + chunk - 1) / chunk);
        }
    }
    if (rng) atomicOr(&meta->range_error, 1);
    if (t == NT - 1) {
        row_off[p] = ea;
        item_off[p] = eb;
        meta->nnz = (unsigned long long)ea;
        meta->edges = (unsigned long long)ea / 2;
        meta->n_items = (unsigned long long)eb;
    }
}

cudaError_t launch_scan(const int* deg, int p, int l, int chunk, Binom B, long long* row_off,
                        long long* item_off, Meta* meta, cudaStream_t st)
{
    k_scan<<<1, 1024, 0, st>>>(deg, p, l, chunk, B, row_off, item_off, meta);
    return cudaGetLastError();
}

// Row i's neighbours in increasing order: each lane owns words lane, lane+32,
// ...; a warp prefix of the word popcounts gives each word's output position.
__global__ void k_fill(const unsigned* __restrict__ bits, int p, int W, const long long* __restrict__ row_off,
                       int* __restrict__ cols, int* __restrict__ srow)
{
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= p) return;
    long long base = row_off[i];
    for (int w0 = 0; w0 < W; w0 += 32) {
        const int w = w0 + lane;
        unsigned word = (w < W) ? bits[(size_t)i * W + w] : 0u;
        const int c = __popc(word);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += x;
        }
        long long pos = base + incl - c;
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            cols[pos] = (w << 5) + b;
            srow[pos] = i;
            ++pos;
        }
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
}

cudaError_t launch_fill(const unsigned* bits, int p, int W, const long long* row_off, int* cols, int* srow,
                        cudaStream_t st)
{
    const int block = 256, grid = (p * 32 + block - 1) / block;
    k_fill<<<grid, block, 0, st>>>(bits, p, W, row_off, cols, srow);
    return cudaGetLastError();
}

__global__ void k_items(const long long* __restrict__ item_off, int p, int* __restrict__ item_row)
{
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= p) return;
    for (long long k = item_off[i] + lane; k < item_off[i + 1]; k += 32) item_row[k] = i;
}

cudaError_t launch_items(const long long* item_off, int p, int* item_row, cudaStream_t st)
{
    const int block = 256, grid = (p * 32 + block - 1) / block;
    k_items<<<grid, block, 0, st>>>(item_off, p, item_row);
    return cudaGetLastError();
}

// partner[e] = slot of (j, i) for slot e = (i, j), by binary search in row j.
__global__ void k_partner(const long long* __restrict__ row_off, const int* __restrict__ cols,
                          const int* __restrict__ srow, long long nnz, int* __restrict__ partner)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const int i = srow[e], j = cols[e];
    long long lo = row_off[j], hi = row_off[j + 1];
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (cols[mid] < i) lo = mid + 1; else hi = mid;
    }
    partner[e] = (int)lo;
}

cudaError_t launch_partner(const long long* row_off, const int* cols, const int* srow, long long nnz,
                           int* partner, cudaStream_t st)
{
    if (nnz == 0) return cudaSuccess;
    const int block = 256;
    k_partner<<<(unsigned)((nnz + block - 1) / block), block, 0, st>>>(row_off, cols, srow, nnz, partner);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Finalisation of level l: an edge (x < y) is removed when either side found
// a separating set; the SepSet is the smaller side's when it has one (the
// serial order of the oracle). Records (x, y, l, S) are appended to the pool.
// With count_serial the number of tests the serial order performs is summed:
// side x up to and including its first separating set (or all of them), and
// side y only when side x found none.
// ---------------------------------------------------------------------------
template <int LB>
__device__ __forceinline__ void side_set(const FinalizeParams& P, int a, unsigned long long rank, int (&Pos)[LB])
{
    const long long off = P.row_off[a];
    const int d = (int)(P.row_off[a + 1] - off);
    unrank_lex<LB>(rank, d, P.l, P.B, Pos);
}

template <int LB>
__device__ __forceinline__ unsigned long long side_serial(const FinalizeParams& P, int a, long long slot_b,
                                                          unsigned long long rank)
{
    const long long off = P.row_off[a];
    const int d = (int)(P.row_off[a + 1] - off);
    if (rank == RANK_NONE) return P.B(d - 1, P.l);
    int Pos[LB];
    unrank_lex<LB>(rank, d, P.l, P.B, Pos);
    const int pb = (int)(slot_b - off);
#pragma unroll
    for (int c = 0; c < LB; ++c)
        if (c < P.l && Pos[c] > pb) Pos[c] -= 1;
    return rank_lex<LB>(Pos, d - 1, P.l, P.B) + 1;
}

template <int LB>
__global__ void k_finalize(FinalizeParams P)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool removed = false;
    unsigned long long serial = 0;
    if (e < (long long)P.nnz) {
        const int x = P.srow[e], y = P.cols[e];
        if (x < y) {
            const long long f = P.partner[e];
            const unsigned long long bx = P.best[e], by = P.best[f];
            int side = -1;
            unsigned long long rank = 0;
            if (bx != RANK_NONE) { side = x; rank = bx; }
            else if (by != RANK_NONE) { side = y; rank = by; }
            if (side >= 0) {
                removed = true;
                bitset_clear_pair(P.bits, P.W, x, y);
                int Pos[LB];
                side_set<LB>(P, side, rank, Pos);
                const int ints = 3 + P.l;
                const unsigned long long at = atomicAdd(&P.meta->rec_ints, (unsigned long long)ints);
                if (at + ints <= P.rec_cap) {
                    int* r = P.rec + at;
                    r[0] = x; r[1] = y; r[2] = P.l;
                    const long long off = P.row_off[side];
#pragma unroll
                    for (int c = 0; c < LB; ++c)
                        if (c < P.l) r[3 + c] = P.cols[off + Pos[c]];
                }
            }
            if (P.count_serial) {
                serial = side_serial<LB>(P, x, e, bx);
                if (bx == RANK_NONE) serial += side_serial<LB>(P, y, f, by);
            }
        }
    }
    const unsigned long long nrem = warp_sum_u64(removed ? 1ull : 0ull);
    const unsigned long long ns = warp_sum_u64(serial);
    if ((threadIdx.x & 31) == 0) {
        if (nrem) atomicAdd(&P.meta->removed, nrem);
        if (ns) atomicAdd(&P.meta->serial_tests, ns);
    }
}

cudaError_t launch_finalize(const FinalizeParams& P, cudaStream_t st)
{
    if (P.nnz == 0) return cudaSuccess;
    const int block = 256;
    const unsigned grid = (unsigned)((P.nnz + block - 1) / block);
    if (P.l <= 2) k_finalize<2><<<grid, block, 0, st>>>(P);
    else if (P.l <= 4) k_finalize<4><<<grid, block, 0, st>>>(P);
    else if (P.l <= 8) k_finalize<8><<<grid, block, 0, st>>>(P);
    else k_finalize<16><<<grid, block, 0, st>>>(P);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 rechecks. One block per queued test. C entries come from the resident
// FP64 correlation when there is one; otherwise they are formed from the FP64
// standardised rows by the definition C_ab = sum_s z_as z_bs / n: every pair of
// the test's m = l + 2 variables in one pass over the samples (threads stride
// the samples, four samples in flight each), then a fixed-order block
// reduction, so the value of an entry does not depend on the test it serves.
// ---------------------------------------------------------------------------
constexpr int RC_THREADS = 256;

template <int M>
__device__ __forceinline__ void c_block(const RecheckParams& P, const int (&V)[M], int m,
                                        double (&G)[M * (M - 1) / 2], double* red)
{
    constexpr int D = M * (M - 1) / 2;
    if (P.c64) {
#pragma unroll
        for (int b = 1; b < M; ++b)
#pragma unroll
            for (int a = 0; a < b; ++a)
                G[b * (b - 1) / 2 + a] = (b < m) ? P.c64[(size_t)V[a] * P.p + V[b]] : 0.0;
        return;
    }
    const double* rows[M];
#pragma unroll
    for (int a = 0; a < M; ++a) rows[a] = P.z64 + (size_t)(a < m ? V[a] : V[0]) * P.ldz;
#pragma unroll
    for (int q = 0; q < D; ++q) G[q] = 0.0;
#pragma unroll 4
    for (int k = threadIdx.x; k < P.n; k += RC_THREADS) {
        double x[M];
#pragma unroll
        for (int a = 0; a < M; ++a) x[a] = (a < m) ? __ldg(rows[a] + k) : 0.0;
#pragma unroll
        for (int b = 1; b < M; ++b)
#pragma unroll
            for (int a = 0; a < b; ++a) G[b * (b - 1) / 2 + a] = fma(x[a], x[b], G[b * (b - 1) / 2 + a]);
    }
    // block reduction: warp trees, then the 8 warp partials in order
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < D; ++q) {
        double g = G[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        if (lane == 0) red[w * D + q] = g;
    }
    __syncthreads();
    const double inv_n = 1.0 / (double)P.n;
#pragma unroll
    for (int q = 0; q < D; ++q) {
        double g = 0.0;
#pragma unroll
        for (int k = 0; k < RC_THREADS / 32; ++k) g += red[k * D + q];
        G[q] = g * inv_n;
    }
    __syncthreads();
}

template <int LB>
__global__ void __launch_bounds__(RC_THREADS) k_recheck(RecheckParams P)
{
    constexpr int M = LB + 2;
    constexpr int D = M * (M - 1) / 2;
    __shared__ double red[(RC_THREADS / 32) * D];
    unsigned long long nq = P.meta->queue_len;
    if (nq > P.qcap) nq = P.qcap;
    unsigned long long done = 0;
    for (long long qi = blockIdx.x; qi < (long long)nq; qi += gridDim.x) {
        const QEntry E = P.queue[qi];
        const long long e = E.a;
        const int i = P.srow[e], j = P.cols[e];
        const long long off = P.row_off[i];
        const int d = (int)(P.row_off[i + 1] - off);
        int Pos[LB];
        unrank_lex<LB>(E.s, d, P.l, P.B, Pos);
        int V[M];
        V[0] = i;
        V[1] = j;
#pragma unroll
        for (int c = 0; c < LB; ++c) V[2 + c] = (c < P.l) ? P.cols[off + Pos[c]] : i;
        const int m = P.l + 2;
        double G[D];
        c_block<M>(P, V, m, G, red);
        if (threadIdx.x == 0) {
            // V index 0 = i, 1 = j, 2 + a = S_a; G[b(b-1)/2 + a] holds C[V_a, V_b], a < b
            Factor<double, LB> F;
            factor_build<double, LB>(
                F, P.l, P.rank_tol, [&](int a, int b) { return G[(a + 2) * (a + 1) / 2 + (b + 2)]; },
                [&](int a) { return G[(a + 2) * (a + 1) / 2 + 0]; });
            double H12, H22;
            factor_apply<double, LB>(F, P.l, G[0], [&](int a) { return G[(a + 2) * (a + 1) / 2 + 1]; }, H12, H22);
            const double H11 = 1.0 - F.uu;
            const bool indep =
                (!(H11 > kVarZero) || !(H22 > kVarZero)) ? true : (H12 * H12 <= P.r2 * H11 * H22);
            if (indep) atomicMin(P.best + e, E.s);
        }
        ++done;
    }
    if (threadIdx.x == 0 && done) atomicAdd(&P.meta->rechecks, done);
}

__global__ void __launch_bounds__(RC_THREADS) k_recheck0(RecheckParams P)
{
    __shared__ double red[RC_THREADS / 32];
    unsigned long long nq = P.meta->queue_len;
    if (nq > P.qcap) nq = P.qcap;
    unsigned long long done = 0;
    for (long long qi = blockIdx.x; qi < (long long)nq; qi += gridDim.x) {
        const QEntry E = P.queue[qi];
        const int V[2] = {E.a, E.b};
        double G[1];
        c_block<2>(P, V, 2, G, red);
        // S empty: rho = C_ij; independent iff rho^2 <= tanh(tau_0)^2
        if (threadIdx.x == 0 && G[0] * G[0] <= P.r2) bitset_clear_pair(P.bits, P.W, E.a, E.b);
        ++done;
    }
    if (threadIdx.x == 0 && done) atomicAdd(&P.meta->rechecks, done);
}

cudaError_t launch_recheck(const RecheckParams& P, int grid, cudaStream_t st)
{
    const int block = RC_THREADS;
    if (P.l <= 2) k_recheck<2><<<grid, block, 0, st>>>(P);
    else if (P.l <= 4) k_recheck<4><<<grid, block, 0, st>>>(P);
    else if (P.l <= 8) k_recheck<8><<<grid, block, 0, st>>>(P);
    else k_recheck<16><<<grid, block, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_recheck0(const RecheckParams& P, int grid, cudaStream_t st)
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
