// k_level.cu -- one level l >= 1 of Algorithm 2 in a single cooperative
// (persistent) kernel: all CTAs are resident and pass bounded grid barriers
// between the phases, so a level costs one launch and no host round trip.
//
//   P1  one block scans the degrees (kept current by the previous level's
//       removals) into the CSR offsets of A'_G, the CI work items
//       (ceil(C(n'_i, l) / chunk) per row) and the max degree; the other blocks
//       take per-row prefix popcounts of A_G's words and, in FP32 mode, a copy
//       of A_G; then termination (Algorithm 1: level l runs only while some node
//       has degree - 1 >= l)
//   P2  A'_G: each row's neighbours in increasing order with, for each slot
//       (i, j), the slot of (j, i) from the prefix popcounts (warp per row); the
//       rows of the work items; best ranks reset
//   P4  CI tests (Sec. 4.3), persistent item pulling, early termination
//   P5  FP32 mode: FP64 rechecks of the near-threshold tests
//   P6  edge removal from G (bitset and degrees) and SepSet records
//
// CI work decomposition (cf. cuPC-S, Sec. 3.4, Algorithm 5, prior art): an
// item is a row i of A'_G and a range of subset ranks. Each lane owns one S per
// round: it unranks S (Sec. 4.2), factors M2 = C[S,S] once and tests every j of
// the row not in S against it, so one factorisation serves up to n'_i - l
// tests. A test (S, j) is skipped once slot (i, j) holds a separating set of
// smaller rank (canonical mode, which must find the lexicographically first S)
// or any separating set (free mode), and on the larger endpoint's side once
// the smaller side has one (Sec. 4.1).
//
// Data written by other CTAs' atomics (best ranks, counters) is read through
// L2 (ld.cg); everything else written in one phase is first loaded after the
// barrier that ends that phase.
#include <cstdio>

#include "kernels.cuh"
#include "mlp.cuh"

namespace cupc {
namespace {

constexpr int NT = 512;                              // threads per CTA
constexpr int NW = NT / 32;
constexpr unsigned long long kBarrierNs = 2000000000ull;

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_cg(const unsigned long long* p) { return __ldcg(p); }

// One of the two CSR buffers of A'_G.
struct Csr {
    long long* row_off;
    int* cols;
    int* srow;
    int* partner;
};

__device__ __forceinline__ Csr csr_view(const LevelParams& P, int b)
{
    return b ? Csr{P.row_off2, P.cols2, P.srow2, P.partner2} : Csr{P.row_off, P.cols, P.srow, P.partner};
}

// View of the correlation block of vertex v's problem, indexed by global ids.
template <typename T>
struct CView {
    const T* base;
    int off, p;
    __device__ __forceinline__ const T* row(int a) const { return base + (long long)(a - off) * p - off; }
};

template <typename T>
__device__ __forceinline__ CView<T> cview(const LevelParams& P, int v)
{
    CView<T> c;
    const ProbDesc* D = prob_of(P.vprob, P.probs, v);
    c.base = (const T*)P.C + (D ? D->c_off : 0);
    c.off = D ? D->off : 0;
    c.p = D ? D->p : P.p;
    return c;
}

// Bitset words of row v that can hold neighbours, and the row's base.
__device__ __forceinline__ void word_range(const LevelParams& P, int v, int& lo, int& hi, long long& rb)
{
    const ProbDesc* D = prob_of(P.vprob, P.probs, v);
    lo = D ? D->wlo : 0;
    hi = D ? D->whi : P.W;
    rb = rowbase(D, P.W, v);
}


// tanh(tau_l) of vertex v's problem and its square.
__device__ __forceinline__ void thresholds(const LevelParams& P, int v, double& r, double& r2)
{
    if (P.vprob) {
        const ProbDesc& D = P.probs[P.vprob[v]];
        r = D.r[P.l];
        r2 = D.r2[P.l];
    } else {
        r = P.r;
        r2 = P.r2;
    }
}

// Grid-wide barrier for a cooperative launch. Returns false (uniformly in the
// CTA) when the kernel must stop: a wait expired or an error was raised. One
// 64-bit word holds the arrivals and the generation: a CTA arrives with one
// atomic add; the last one adds 2^32 - N, which returns the arrivals to 0 and
// advances the generation in the same operation, and the others poll the
// generation (the error flag and the clock every 64th poll).
// The wait is limited to kBarrierNs, or to P.barrier_ns when that is set (a
// test of the expiry path).
__device__ bool grid_sync(const LevelParams& P)
{
    __shared__ int ok;
    LevelMeta* lm = P.lm;
    const unsigned long long lim = P.barrier_ns ? (unsigned long long)P.barrier_ns : kBarrierNs;
    const unsigned every = 63u;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned long long old = atomicAdd(&lm->bar, 1ull);
        const unsigned g = (unsigned)(old >> 32);
        if ((unsigned)old + 1u == gridDim.x) {
            atomicAdd(&lm->bar, (1ull << 32) - (unsigned long long)gridDim.x);
        } else {
            volatile unsigned long long* vb = &lm->bar;
            const unsigned long long t0 = gtimer();
            for (unsigned it = 1; (unsigned)(*vb >> 32) == g; ++it) {
                if ((it & every) == 0) {
                    if (*(volatile int*)&lm->error) break;
                    if (gtimer() - t0 > lim) {
                        atomicOr(&lm->error, 8);
                        break;
                    }
                }
            }
        }
        __threadfence();
        ok = (*(volatile int*)&lm->error == 0);
    }
    __syncthreads();
    return ok != 0;
}

// ---------------------------------------------------------------------------
// P1 (blocks other than 0): exclusive prefix popcounts of each row's words,
// wpre[i*W + w] = number of neighbours of i below 32 w; FP32 mode: A_G copy
// ---------------------------------------------------------------------------
__device__ void phase_prefix(const LevelParams& P, int skip)
{
    const int lane = threadIdx.x & 31;
    // (skip = 1: block 0 is scanning; with a single block it does this part too)
    const int nb = (skip && gridDim.x > 1) ? gridDim.x - 1 : gridDim.x;
    const int bid = (skip && gridDim.x > 1) ? blockIdx.x - 1 : blockIdx.x;
    const int gw = (bid * NT + threadIdx.x) >> 5;
    const int nwarps = (nb * NT) >> 5;
    for (int i = gw; i < P.p; i += nwarps) {
        int wlo, whi;
        long long rb;
        word_range(P, i, wlo, whi, rb);
        int base = 0;
        for (int w0 = wlo; w0 < whi; w0 += 32) {
            const int q = w0 + lane;
            const int c = (q < whi) ? __popc(P.bits[rb + q]) : 0;
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int x = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += x;
            }
            if (q < whi) P.wpre[rb + q] = base + incl - c;
            base += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

// ---------------------------------------------------------------------------
// Learned ordering (FP32 mode, levels >= 1). When a level builds A'_G from the
// bitset A_G (level 1, and a level run again), every row's candidates are
// scored by the network (features of mlp.cuh: the candidate's correlation with
// the row variable and means over the row's other neighbours) and the row is
// enumerated in descending score (ties: increasing position), so the
// S-shared tests of a row keep sharing each subset across j. A level that
// builds A'_G from the previous level's keeps the survivors' relative order,
// and a reused A'_G keeps its order. The order is a permutation of the row:
// every subset is still reached, so the skeleton cannot change; the ranks the
// tests record (and the SepSet the serial order stores) are those of the
// permuted order. A row with more than kLrnMaxDeg neighbours keeps its
// increasing order.
// ---------------------------------------------------------------------------
constexpr int kLrnMaxDeg = 512;
// dynamic shared memory of the scoring phase: the weights as FP32
constexpr size_t kLrnBytes = ((size_t)MLP_NP * sizeof(float) + 15) & ~(size_t)15;

// The score of every slot (i, k) of A'_G (candidate k of row i), one thread per
// slot; the weights are staged in shared memory as FP32 (each weight read by
// the warp's lanes at once, a broadcast), the row sums of |C_ij| come from the
// fill phase. The score is mlp_score's, as the forward kernel computes it.
__device__ void phase_lrn_score(const LevelParams& P, const Csr& A, unsigned char* dyn)
{
    float* Ws = (float*)dyn;
    const __nv_bfloat16* Wg = (const __nv_bfloat16*)P.mlp_w;
    for (int q = threadIdx.x; q < MLP_NP; q += NT) Ws[q] = __bfloat162float(Wg[q]);
    __syncthreads();
    const long long nnz = A.row_off[P.p];
    for (long long e = (long long)blockIdx.x * NT + threadIdx.x; e < nnz; e += (long long)gridDim.x * NT) {
        const int i = A.srow[e];
        const long long off = A.row_off[i];
        const int d = (int)(A.row_off[i + 1] - off);
        if (d > kLrnMaxDeg) continue;
        const CView<float> CV = cview<float>(P, i);
        auto C = [&](int a, int b) { return __ldg(CV.row(a) + b); };
        float x[MLP_IN];
        mlp_row_features(C, i, A.cols + off, d, (int)(e - off), P.l, P.lrsum[i], x);
        const float y = mlp_score(Ws, x);
        P.lscore[e] = (y == y) ? y : -INFINITY;
    }
}

// Each slot's position in its row's order: iperm, and perm as its inverse.
__device__ void phase_lrn_rank(const LevelParams& P, const Csr& A)
{
    const long long nnz = A.row_off[P.p];
    for (long long e = (long long)blockIdx.x * NT + threadIdx.x; e < nnz; e += (long long)gridDim.x * NT) {
        const int i = A.srow[e];
        const long long off = A.row_off[i];
        const int d = (int)(A.row_off[i + 1] - off);
        const int c = (int)(e - off);
        int v = c;
        if (d <= kLrnMaxDeg) {
            // (plain loads: the scores were written before the grid barrier and
            // this SM has not read them in this launch)
            const float* sc = P.lscore + off;
            const float y = sc[c];
            v = 0;
#pragma unroll 8
            for (int u = 0; u < d; ++u) {
                const float y2 = sc[u];
                v += (y2 > y) || (y2 == y && u < c);
            }
        }
        P.iperm[e] = v;
        P.perm[off + v] = c;
    }
}

// P1 of a level whose A'_G is built from the previous level's (old buffer O):
// per old row, the position of each surviving slot among the row's survivors
// (-1 for a removed edge), from the alive flags the previous level's removal
// phase wrote. Same CTA split as phase_prefix. LRN: also each survivor's
// position among the survivors in the old row's learned order (vrank).
template <bool LRN>
__device__ void phase_rank(const LevelParams& P, const Csr& O, int skip)
{
    const int lane = threadIdx.x & 31;
    const int nb = (skip && gridDim.x > 1) ? gridDim.x - 1 : gridDim.x;
    const int bid = (skip && gridDim.x > 1) ? blockIdx.x - 1 : blockIdx.x;
    const int gw = (bid * NT + threadIdx.x) >> 5;
    const int nwarps = (nb * NT) >> 5;
    for (int i = gw; i < P.p; i += nwarps) {
        const long long off = O.row_off[i], end = O.row_off[i + 1];
        int base = 0;
        for (long long e0 = off; e0 < end; e0 += 32) {
            const long long e = e0 + lane;
            const bool a = e < end && P.alive[e] != 0;
            const unsigned m = __ballot_sync(0xffffffffu, a);
            if (e < end) P.nrank[e] = a ? base + __popc(m & ((1u << lane) - 1u)) : -1;
            base += __popc(m);
        }
        if (LRN) {
            base = 0;
            for (long long v0 = off; v0 < end; v0 += 32) {
                const long long v = v0 + lane;
                const long long e = v < end ? off + P.perm[v] : 0;
                const bool a = v < end && P.alive[e] != 0;
                const unsigned m = __ballot_sync(0xffffffffu, a);
                if (a) P.vrank[e] = base + __popc(m & ((1u << lane) - 1u));
                base += __popc(m);
            }
        }
    }
}

// P2 of such a level: the surviving slots of the old A'_G, in order, into the
// new buffer A (row offsets from the degree scan); a slot's partner is found
// through the old partner's position. LRN: the new rows' order from vrank.
template <bool LRN>
__device__ void phase_fill_incr(const LevelParams& P, const Csr& O, const Csr& A)
{
    const long long nnz_old = O.row_off[P.p];
    for (long long e = (long long)blockIdx.x * NT + threadIdx.x; e < nnz_old; e += (long long)gridDim.x * NT) {
        const int r = P.nrank[e];
        if (r < 0) continue;
        const int i = O.srow[e], j = O.cols[e];
        const long long ne = A.row_off[i] + r;
        A.cols[ne] = j;
        A.srow[ne] = i;
        A.partner[ne] = (int)(A.row_off[j] + P.nrank[O.partner[e]]);
        if (LRN) {
            const int v = P.vrank[e];
            P.perm[A.row_off[i] + v] = r;
            P.iperm[ne] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// P1: block 0 scans degrees into CSR offsets and work-item offsets. The chunk
// (subset ranks per item) doubles until the items fit the item array.
// ---------------------------------------------------------------------------
// Work items of a row with degree d at level l: the subset ranks of the row
// (S shared across j).
// With the j split (level 1), each subset chunk is further cut into the row's
// j positions in ranges of 32: item k of the row is subset chunk k / J and
// j range k % J, J = ceil(d / 32).
__device__ __forceinline__ int j_ranges(int d, int l, bool js) { return (js && l == 1) ? (d + 31) >> 5 : 1; }

__device__ __forceinline__ unsigned long long row_items(const Binom& B, int d, int l, int chunk, bool js)
{
    if (d < l + 1) return 0;
    return (B(d, l) + chunk - 1) / chunk * (unsigned long long)j_ranges(d, l, js);
}

// Adds a row with K items to the round histogram (bin min(K, RND - 1); rows
// without items are not counted). Lanes with the same bin are combined first:
// most rows fall in a handful of bins, and shared atomics on one address
// serialise.
__device__ __forceinline__ void hist_add(unsigned long long* hist, unsigned long long K)
{
    const int bin = K == 0 ? -1 : (int)(K < RND - 1 ? K : RND - 1);
    const unsigned peers = __match_any_sync(__activemask(), bin);
    const int lane = threadIdx.x & 31;
    if (bin >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (unsigned long long)__popc(peers));
}

// Degrees of rows [i0, i0 + 8) (0 past hi): all loads issued before use, so a
// thread walking its range pays one memory latency per 8 rows.
__device__ __forceinline__ void load8(const LevelParams& P, int i0, int hi, int (&d)[8], int (&di)[8])
{
#pragma unroll
    for (int u = 0; u < 8; ++u) d[u] = (i0 + u < hi) ? P.deg[i0 + u] : 0;
    if (P.vlmax) {
        int m[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) m[u] = (i0 + u < hi) ? P.vlmax[i0 + u] : 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) di[u] = (P.l > m[u]) ? 0 : d[u];
    } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) di[u] = d[u];
    }
}

// Rows up to which one CTA scans the degrees (phase_scan_one): beyond it a scan
// by every CTA (phase_scan_a/b) costs an extra grid barrier but no longer
// walks all rows in one CTA.
constexpr int kScanOne = 4096;

// P1 for graphs of at most kScanOne rows: block 0 scans every row while the
// other CTAs build the word prefixes (no second barrier).
__device__ void phase_scan_one(const LevelParams& P, const Csr& A)
{
    __shared__ long long sa[32], sb[32];
    __shared__ unsigned long long stot;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int per = (P.p + NT - 1) / NT;
    const int lo = min(P.p, t * per), hi = min(P.p, lo + per);
    const int l = P.l;
    int rng = 0;
    int d8[8], di8[8];
    // one pass for the sums at the default chunk; the chunk doubles (items
    // recounted) only while the items would not fit the item array
    int chunk = P.chunk0;
    long long a = 0, b = 0;
    unsigned long long sq = 0;
    int dmax = 0;
    for (int i0 = lo; i0 < hi; i0 += 8) {
        load8(P, i0, hi, d8, di8);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int d = di8[u];
            dmax = max(dmax, d);
            a += d8[u];
            b += (long long)row_items(P.B, d, l, chunk, P.jsplit);
            if (d >= l + 1) {
                if (P.B(d, l) == ~0ull) rng = 1;
                sq += (unsigned long long)(d + 1) * (unsigned long long)(d + 1);
            }
        }
    }
    for (int it = 0; it < 48; ++it) {
        const unsigned long long bw = warp_sum_u64((unsigned long long)b);
        if (lane == 0) sb[w] = (long long)bw;
        __syncthreads();
        if (t == 0) {
            unsigned long long tot = 0;
            for (int k = 0; k < NW; ++k) tot += (unsigned long long)sb[k];
            stot = tot;
        }
        __syncthreads();
        const bool fits = stot <= P.item_cap;
        __syncthreads();
        if (fits || chunk > (1 << 29)) break;
        chunk *= 2;
        b = 0;
        for (int i0 = lo; i0 < hi; i0 += 8) {
            load8(P, i0, hi, d8, di8);
#pragma unroll
            for (int u = 0; u < 8; ++u) b += (long long)row_items(P.B, di8[u], l, chunk, P.jsplit);
        }
    }
    sq = warp_sum_u64(sq);
    if (lane == 0 && sq) atomicAdd(&P.lm->block_entries[l], sq);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if (lane == 0) atomicMax(&P.lm->maxdeg[l], dmax);
    long long ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long xa = __shfl_up_sync(0xffffffffu, ia, o);
        const long long xb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) { ia += xa; ib += xb; }
    }
    __syncthreads();
    if (lane == 31) { sa[w] = ia; sb[w] = ib; }
    __syncthreads();
    if (w == 0) {
        long long va = (lane < NW) ? sa[lane] : 0, vb = (lane < NW) ? sb[lane] : 0;
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
    // rows by their item count (capped at RND - 1) and the items past the cap
    __shared__ unsigned long long hist[RND];
    for (int q = t; q < RND; q += NT) hist[q] = 0;
    __syncthreads();
    unsigned long long ovf = 0;
    for (int i0 = lo; i0 < hi; i0 += 8) {
        load8(P, i0, hi, d8, di8);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u;
            if (i >= hi) break;
            const int d = di8[u];
            A.row_off[i] = ea;
            P.item_off[i] = eb;
            ea += d8[u];
            const unsigned long long K = row_items(P.B, d, l, chunk, P.jsplit);
            eb += (long long)K;
            hist_add(hist, K);
            if (K > RND - 1) ovf += K - (RND - 1);
        }
    }
    ovf = warp_sum_u64(ovf);
    if (lane == 0 && ovf) atomicAdd(&hist[0], ovf);   // bin 0 (no row has 0 items counted) carries the overflow
    __syncthreads();
    for (int q = t; q < RND; q += NT)
        if (hist[q]) P.lm->round_hist[l][q] = hist[q];
    if (rng) atomicOr(&P.lm->range_error, 1);
    if (t == NT - 1) {
        A.row_off[P.p] = ea;
        P.item_off[P.p] = eb;
        P.lm->edges[l] = (unsigned long long)ea / 2;
        P.lm->items[l] = (unsigned long long)eb;
        P.lm->chunk[l] = chunk;
        if ((unsigned long long)ea > P.nnz_cap || (unsigned long long)eb > P.item_cap) atomicOr(&P.lm->error, 16);
    }
}

// Contiguous rows of this CTA (the scan's order).
__device__ __forceinline__ void cta_rows(const LevelParams& P, int& r0, int& r1)
{
    r0 = (int)((long long)P.p * blockIdx.x / gridDim.x);
    r1 = (int)((long long)P.p * (blockIdx.x + 1) / gridDim.x);
}

// Block-wide sum of two u64 values (fixed order); the result is valid in thread 0.
__device__ __forceinline__ void block_sum2(unsigned long long (&v)[2], unsigned long long (*red)[2])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 2; ++k) v[k] = warp_sum_u64(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 2; ++k) red[w][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 1; q < NW; ++q)
#pragma unroll
            for (int k = 0; k < 2; ++k) v[k] += red[q][k];
    __syncthreads();
}

// P1a (every CTA, its contiguous rows): CSR slots and work items at the
// default chunk; max degree, C sub-block entries and the 64-bit range check go
// to the level counters.
__device__ void phase_scan_a(const LevelParams& P)
{
    __shared__ unsigned long long red[NW][2];
    const int l = P.l;
    int r0, r1;
    cta_rows(P, r0, r1);
    unsigned long long v[2] = {0, 0};   // slots, items
    unsigned long long sq = 0;
    int dmax = 0, rng = 0;
    for (int i = r0 + (int)threadIdx.x; i < r1; i += NT) {
        const int d = P.deg[i];
        const int di = (P.vlmax && l > P.vlmax[i]) ? 0 : d;
        v[0] += (unsigned long long)d;
        v[1] += row_items(P.B, di, l, P.chunk0, P.jsplit);
        dmax = max(dmax, di);
        if (di >= l + 1) {
            if (P.B(di, l) == ~0ull) rng = 1;
            sq += (unsigned long long)(di + 1) * (unsigned long long)(di + 1);
        }
    }
    sq = warp_sum_u64(sq);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        if (sq) atomicAdd(&P.lm->block_entries[l], sq);
        if (dmax) atomicMax(&P.lm->maxdeg[l], dmax);
    }
    if (__any_sync(0xffffffffu, rng) && lane == 0) atomicOr(&P.lm->range_error, 1);
    block_sum2(v, red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 2; ++k) P.scan_part[(size_t)blockIdx.x * 2 + k] = v[k];
}

// P1b (every CTA, after a grid barrier): the chunk from the totals (it doubles
// while the items would not fit; each doubling recounts and takes another
// barrier), then this CTA's rows' CSR offsets, item offsets and its part of
// the round histogram. Returns false when a barrier failed.
__device__ bool phase_scan_b(const LevelParams& P, const Csr& A)
{
    __shared__ unsigned long long sbase[2], stot[2];
    __shared__ unsigned long long rsum[NW][2];
    __shared__ unsigned long long wsum[NW][2];
    __shared__ unsigned long long hist[RND];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int l = P.l;
    int r0, r1;
    cta_rows(P, r0, r1);
    // totals of the CTAs, and the exclusive prefix for this CTA (fixed order)
    // (thread c loads CTA c's partials; two block sums in a fixed order)
    auto totals = [&]() {
        unsigned long long v[2] = {0, 0}, u[2] = {0, 0};
        if (t < (int)gridDim.x)
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                v[k] = __ldcg(P.scan_part + (size_t)t * 2 + k);
                u[k] = t < (int)blockIdx.x ? v[k] : 0ull;
            }
        block_sum2(v, rsum);
        block_sum2(u, rsum);
        if (t == 0)
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                stot[k] = v[k];
                sbase[k] = u[k];
            }
        __syncthreads();
    };
    totals();
    int chunk = P.chunk0;
    for (int it = 0; it < 40 && stot[1] > P.item_cap && chunk <= (1 << 29); ++it) {
        // recount this CTA's items at twice the chunk
        chunk *= 2;
        unsigned long long b = 0;
        for (int i = r0 + t; i < r1; i += NT) {
            const int di = (P.vlmax && l > P.vlmax[i]) ? 0 : P.deg[i];
            b += row_items(P.B, di, l, chunk, P.jsplit);
        }
        b = warp_sum_u64(b);
        if (lane == 0) wsum[w][0] = b;
        __syncthreads();
        if (t == 0) {
            unsigned long long x = 0;
            for (int q = 0; q < NW; ++q) x += wsum[q][0];
            P.scan_part[(size_t)blockIdx.x * 2 + 1] = x;
        }
        if (!grid_sync(P)) return false;
        totals();
    }
    // this CTA's rows: exclusive scans of (slots, items), in tiles of NT rows
    for (int q = t; q < RND; q += NT) hist[q] = 0;
    __syncthreads();
    unsigned long long ca = sbase[0], cb = sbase[1];
    unsigned long long ovf = 0;
    for (int base = r0; base < r1; base += NT) {
        const int i = base + t;
        unsigned long long a = 0, b = 0;
        if (i < r1) {
            const int d = P.deg[i];
            const int di = (P.vlmax && l > P.vlmax[i]) ? 0 : d;
            a = (unsigned long long)d;
            b = row_items(P.B, di, l, chunk, P.jsplit);
            if (b > RND - 1) ovf += b - (RND - 1);
        }
        hist_add(hist, b);
        // inclusive warp scans, then the warp totals in order
        unsigned long long ia = a, ib = b;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long xa = __shfl_up_sync(0xffffffffu, ia, o);
            const unsigned long long xb = __shfl_up_sync(0xffffffffu, ib, o);
            if (lane >= o) { ia += xa; ib += xb; }
        }
        if (lane == 31) { wsum[w][0] = ia; wsum[w][1] = ib; }
        __syncthreads();
        unsigned long long pa = 0, pb = 0, ta = 0, tb = 0;
        for (int q = 0; q < NW; ++q) {
            if (q < w) { pa += wsum[q][0]; pb += wsum[q][1]; }
            ta += wsum[q][0]; tb += wsum[q][1];
        }
        if (i < r1) {
            A.row_off[i] = (long long)(ca + pa + ia - a);
            P.item_off[i] = (long long)(cb + pb + ib - b);
        }
        ca += ta;
        cb += tb;
        __syncthreads();
    }
    ovf = warp_sum_u64(ovf);
    if (lane == 0 && ovf) atomicAdd(&hist[0], ovf);   // bin 0 carries the items past the first RND - 1
    __syncthreads();
    for (int q = t; q < RND; q += NT)
        if (hist[q]) atomicAdd(&P.lm->round_hist[l][q], hist[q]);
    if (blockIdx.x == gridDim.x - 1 && t == 0) {
        const unsigned long long ea = stot[0], eb = stot[1];
        A.row_off[P.p] = (long long)ea;
        P.item_off[P.p] = (long long)eb;
        P.lm->edges[l] = ea / 2;
        P.lm->items[l] = eb;
        P.lm->chunk[l] = chunk;
        if (ea > P.nnz_cap || eb > P.item_cap) atomicOr(&P.lm->error, 16);
    }
    return true;
}

// ---------------------------------------------------------------------------
// P2: A'_G rows, item rows, best reset
// ---------------------------------------------------------------------------
// Work items in dispatch order: each CTA takes a contiguous range of rows,
// reserves slots in every round for them (one global atomic per round), then
// each row's warp writes its items (row, index within the row) into them. The
// order within a round is unspecified; results do not depend on it.
__device__ void phase_items(const LevelParams& P, const Csr& A)
{
    __shared__ unsigned cnt[RND];
    __shared__ unsigned long long base[RND], cur[RND];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int l = P.l;
    int r0, r1;
    cta_rows(P, r0, r1);
    for (int q = threadIdx.x; q < RND; q += NT) {
        cnt[q] = 0;
        cur[q] = 0;
    }
    __syncthreads();
    unsigned long long ovf = 0;
    for (int i = r0 + (int)threadIdx.x; i < r1; i += NT) {
        const long long K = P.item_off[i + 1] - P.item_off[i];
        const int bin = K == 0 ? -1 : (int)(K < RND - 1 ? K : RND - 1);
        const unsigned peers = __match_any_sync(__activemask(), bin);
        if (bin >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[bin], (unsigned)__popc(peers));
        if (K > RND - 1) ovf += (unsigned long long)(K - (RND - 1));
    }
    ovf = warp_sum_u64(ovf);
    __shared__ unsigned long long sovf;
    if (threadIdx.x == 0) sovf = 0;
    __syncthreads();
    if (lane == 0 && ovf) atomicAdd(&sovf, ovf);
    __syncthreads();
    // first slot of each round, from the level's histogram of rows by item count
    // (round c < RND - 1 holds the rows with more than c items, the last round
    // the items past the first RND - 1 of every row)
    __shared__ unsigned long long roff[RND], rh[RND];
    for (int q = threadIdx.x; q < RND; q += NT) rh[q] = __ldcg(&P.lm->round_hist[l][q]);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long n_round[RND], above = 0, off = 0;
        for (int v = RND - 1; v >= 1; --v) {
            above += rh[v];
            n_round[v - 1] = above;
        }
        n_round[RND - 1] = rh[0];
        for (int q = 0; q < RND; ++q) {
            roff[q] = off;
            off += n_round[q];
        }
    }
    __syncthreads();
    if (threadIdx.x < RND) {
        const int q = threadIdx.x;
        unsigned long long nq = 0;
        if (q < RND - 1) {
            for (int v = q + 1; v < RND; ++v) nq += cnt[v];
        } else {
            nq = sovf;
        }
        base[q] = nq ? roff[q] + atomicAdd(&P.lm->round_cur[l][q], nq) : 0;
    }
    __syncthreads();
    for (int i = r0 + w; i < r1; i += NW) {
        const long long K = P.item_off[i + 1] - P.item_off[i];
        const int kc = (int)(K < RND - 1 ? K : RND - 1);
        for (int c = lane; c < kc; c += 32) {
            const unsigned long long slot = base[c] + atomicAdd(&cur[c], 1ull);
            P.item_row[slot] = i;
            P.item_c[slot] = c;
        }
        if (K > RND - 1) {
            unsigned long long k0 = 0;
            if (lane == 0) k0 = atomicAdd(&cur[RND - 1], (unsigned long long)(K - (RND - 1)));
            k0 = __shfl_sync(0xffffffffu, k0, 0);
            for (long long q = lane; q < K - (RND - 1); q += 32) {
                const unsigned long long slot = base[RND - 1] + k0 + (unsigned long long)q;
                P.item_row[slot] = i;
                P.item_c[slot] = (int)(RND - 1 + q);
            }
        }
    }
}

template <typename T, bool LRN>
__device__ void phase_fill(const LevelParams& P, const Csr& A, const Csr& O, bool reuse, bool incr, bool pivot)
{
    const int lane = threadIdx.x & 31;
    if (incr) {
        phase_fill_incr<LRN>(P, O, A);
        reuse = true;                              // (the bitset walk below is skipped)
    }
    const int gw = (blockIdx.x * NT + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * NT) >> 5;
    for (int i = reuse ? P.p : gw; i < P.p; i += nwarps) {
        long long base = A.row_off[i];
        int wlo, whi;
        long long rb;
        word_range(P, i, wlo, whi, rb);
        const ProbDesc* Di = prob_of(P.vprob, P.probs, i);   // every neighbour is in i's problem
        const T* Crow = (pivot || LRN) ? cview<T>(P, i).row(i) : nullptr;
        float rs = 0.f;                            // LRN: sum of |C_ij| over the row
        for (int w0 = wlo; w0 < whi; w0 += 32) {
            const int q = w0 + lane;
            unsigned word = (q < whi) ? P.bits[rb + q] : 0u;
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
                const int j = (q << 5) + b;
                A.cols[pos] = j;
                A.srow[pos] = i;
                // slot of (j, i): row j's offset + neighbours of j below i
                const long long rbj = rowbase(Di, P.W, j);
                const unsigned wj = P.bits[rbj + (i >> 5)];
                A.partner[pos] = (int)(A.row_off[j] + P.wpre[rbj + (i >> 5)] +
                                       __popc(wj & ((1u << (i & 31)) - 1u)));
                if (pivot) ((T*)P.cval)[pos] = Crow[j];
                if (LRN) rs += fabsf((float)Crow[j]);
                ++pos;
            }
            base += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (LRN) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
            if (lane == 0) P.lrsum[i] = rs;
        }
    }
    if (!pivot) phase_items(P, A);
    const long long nnz = A.row_off[P.p];
    for (long long e = (long long)blockIdx.x * NT + threadIdx.x; e < nnz; e += (long long)gridDim.x * NT)
        P.best[e] = RANK_NONE;
}

// ---------------------------------------------------------------------------
// P4: CI tests
// ---------------------------------------------------------------------------
// 0 dependent, 1 independent, 2 undecided in FP32 (sent to the FP64 recheck)
// Decision constants of one work item, converted once (conversions run on
// GB300's narrow FP64 pipe): tanh(tau_l) and its square, the FP32 band.
struct Decide {
    float r, band_abs, band_rel, piv_floor;
    double r2;
};

__device__ __forceinline__ Decide decide_consts(const LevelParams& P, double r, double r2)
{
    Decide d;
    d.r = (float)r;
    d.band_abs = (float)P.band_abs;
    d.band_rel = (float)P.band_rel;
    d.piv_floor = (float)P.piv_floor;
    d.r2 = r2;
    return d;
}

template <typename T, bool FP32>
__device__ __forceinline__ int ci_decide(T H11, T H12, T H22, T minpiv2, const Decide& dc)
{
    if (!FP32) {
        // zero conditional variance (rounding level of the unit diagonal): V_i or
        // V_j is a linear function of S -> independent
        if (!(H11 > T(kVarZero)) || !(H22 > T(kVarZero))) return 1;
        return (H12 * H12 <= (T)dc.r2 * H11 * H22) ? 1 : 0;
    } else {
        if (!(minpiv2 >= dc.piv_floor) || !(H11 > 1e-4f) || !(H22 > 1e-4f)) return 2;
        const float rho = fabsf((float)H12) * rsqrtf((float)(H11 * H22));
        const float band = dc.band_abs + dc.band_rel / ((float)minpiv2 * fminf((float)H11, (float)H22));
        if (rho > dc.r + band) return 0;
        if (rho < dc.r - band) return 1;
        return 2;
    }
}

// LRN: the row's candidates are enumerated in the network's order: position v
// of the enumeration is slot off + P.perm[off + v] (ranks and the per-slot
// best ranks are then over these virtual positions).
template <typename T, int LB, bool FP32, bool LRN = false>
__device__ void phase_ci(const LevelParams& P, const Csr& A)
{
    const int lane = threadIdx.x & 31;
    const int l = P.l;
    // C(m, k) for small m, k <= LB + 1, in shared memory for the unranking
    __shared__ unsigned long long sbin[(LB + 2) * kBinomS];
    for (int q = threadIdx.x; q < (LB + 2) * kBinomS; q += NT) sbin[q] = P.B(q % kBinomS, q / kBinomS);
    __syncthreads();
    const BinomS BS{sbin};
    const unsigned long long n_items = P.lm->items[l];
    const int chunk = P.lm->chunk[l];
    // at most one item per warp: warp g takes item g (the shared counter would
    // only make every warp queue on one atomic to learn that nothing is left)
    const unsigned long long nwarps = ((unsigned long long)gridDim.x * NT) >> 5;
    const bool fixed = n_items <= nwarps;
    const unsigned long long gwarp = ((unsigned long long)blockIdx.x * NT + threadIdx.x) >> 5;
    bool taken = false;
    unsigned long long ntests = 0;
    for (;;) {
        unsigned long long item = 0;
        if (fixed) {
            if (taken) break;
            taken = true;
            item = gwarp;
        } else {
            if (lane == 0) item = atomicAdd(&P.lm->next_item[l], 1ull);
            item = __shfl_sync(0xffffffffu, item, 0);
        }
        if (item >= n_items) break;
        const int i = P.item_row[item];
        const long long kr = P.item_c[item];
        const long long off = A.row_off[i];
        const int d = (int)(A.row_off[i + 1] - off);
        // subset chunk k and j positions [jlo, jhi) of this item
        const int nj = j_ranges(d, l, P.jsplit);
        const long long k = kr / nj;
        const int jlo = (int)(kr % nj) * 32, jhi = nj > 1 ? min(d, jlo + 32) : d;
        const unsigned long long nsets = P.B(d, l);
        const unsigned long long s0 = (unsigned long long)k * (unsigned long long)chunk;
        const unsigned long long s1 = min(s0 + (unsigned long long)chunk, nsets);
        const CView<T> CV = cview<T>(P, i);
        double thr, thr2;
        thresholds(P, i, thr, thr2);
        const Decide dc = decide_consts(P, thr, thr2);
        const T* __restrict__ Ci = CV.row(i);
        // complement mode when most of the row is in S (high levels): a broadcast j
        // is then valid for few lanes' subsets, so each lane walks its own d - l
        // non-members instead and all lanes test at once
        const bool comp = 4 * (d - l) <= 3 * d;
        auto vmap = [&](int v) -> int { return LRN ? P.perm[off + v] : v; };
        for (unsigned long long base = s0; base < s1; base += 32) {
            const unsigned long long s = base + lane;
            const bool active = s < s1;
            int Pos[LB], Sx[LB];
            Factor<T, LB> F;
#pragma unroll
            for (int c = 0; c < LB; ++c) { Pos[c] = -1; Sx[c] = 0; }
            if (active) {
                if (d < kBinomS) unrank_lex<LB>(s, d, l, BS, Pos);
                else unrank_lex<LB>(s, d, l, P.B, Pos);
#pragma unroll
                for (int c = 0; c < LB; ++c)
                    if (c < l) Sx[c] = A.cols[off + vmap(Pos[c])];
                factor_build<T, LB>(
                    F, l, (T)P.rank_tol, [&](int a, int b) { return __ldg(CV.row(Sx[a]) + Sx[b]); },
                    [&](int a) { return __ldg(Ci + Sx[a]); });
            }
            // one test of this lane's subset against the neighbour j of slot e
            auto test = [&](long long e, int j, T cij) {
                T H12, H22;
                const T* __restrict__ Cj = CV.row(j);
                factor_apply<T, LB>(F, l, cij, [&](int a) { return __ldg(Cj + Sx[a]); }, H12, H22);
                const T H11 = T(1) - F.uu;
                ++ntests;
                const int dec = ci_decide<T, FP32>(H11, H12, H22, F.minpiv2, dc);
                if (dec == 1) {
                    atomicMin(P.best + e, s);
                } else if (FP32 && dec == 2) {
                    const unsigned long long qq = atomicAdd(&P.lm->queue_len[l], 1ull);
                    if (qq < P.qcap) {
                        QEntry* Q = P.queue + qq;
                        Q->a = (int)e;
                        Q->b = 0;
                        Q->s = s;
#pragma unroll
                        for (int c = 0; c < LB; ++c)
                            if (c < l) Q->S[c] = Sx[c];
                    }
                }
            };
            if (comp) {
                for (int v = 0; v < d - l; ++v) {
                    // the v-th position outside S (Pos increasing)
                    int jp = v;
#pragma unroll
                    for (int c = 0; c < LB; ++c)
                        if (c < l && Pos[c] <= jp) ++jp;
                    if (!active) continue;
                    const long long e = off + vmap(jp);
                    const int j = A.cols[e];
                    const unsigned long long be = ld_cg(P.best + e);
                    const unsigned long long pb = (!P.canonical || i > j) ? ld_cg(P.best + A.partner[e]) : RANK_NONE;
                    if (pb == RANK_NONE && (P.canonical ? (be >= s) : (be == RANK_NONE))) test(e, j, __ldg(Ci + j));
                }
                continue;
            }
            // the row's per-j data in chunks of 32: lane q loads j-position jc + q
            // (coalesced), then the chunk is broadcast one j at a time by shuffles
            for (int jc = jlo; jc < jhi; jc += 32) {
                int j_l = 0, e_l = 0;
                unsigned long long b_l = RANK_NONE, pb_l = RANK_NONE;
                T cij_l = T(0);
                if (jc + lane < jhi) {
                    const long long e = off + vmap(jc + lane);
                    e_l = (int)e;
                    j_l = A.cols[e];
                    b_l = ld_cg(P.best + e);
                    // the larger endpoint's side stops once the smaller side separates
                    // (free mode: either side stops the other)
                    if (!P.canonical || i > j_l) pb_l = ld_cg(P.best + A.partner[e]);
                    cij_l = __ldg(Ci + j_l);
                }
                const int jn = min(32, jhi - jc);
#pragma unroll 4
                for (int q = 0; q < jn; ++q) {
                    const int jp = jc + q;
                    const int j = __shfl_sync(0xffffffffu, j_l, q);
                    const int e = __shfl_sync(0xffffffffu, e_l, q);
                    const unsigned long long be = __shfl_sync(0xffffffffu, b_l, q);
                    const unsigned long long pb = __shfl_sync(0xffffffffu, pb_l, q);
                    const T cij = __shfl_sync(0xffffffffu, cij_l, q);
                    bool t = active && pb == RANK_NONE && (P.canonical ? (be >= s) : (be == RANK_NONE));
#pragma unroll
                    for (int c = 0; c < LB; ++c)
                        if (c < l && Pos[c] == jp) t = false;
                    if (t) test(e, j, cij);
                }
            }
        }
    }
    ntests = warp_sum_u64(ntests);
    if (lane == 0 && ntests) atomicAdd(&P.lm->tests[l], ntests);
}

// ---------------------------------------------------------------------------
// P4 at level 1, by conditioning variable. A test (i, j | k) with k in
// adj(i) \ {j} (side i, S = {k}) reads C_ik, C_jk and C_ij only (Sec. 4.3 with
// |S| = 1: H11 = 1 - C_ik^2, H22 = 1 - C_jk^2, H12 = C_ij - C_ik C_jk). Since k in
// adj(i) iff i in adj(k), the tests sharing k are the slots (i, j) of the rows
// i in adj(k): a CTA stages row k of C in shared memory with coalesced 16-byte
// loads, then its warps walk those rows (lane q takes slot q of row i, reading
// the row's neighbour list and its C_ij values contiguously), so C_ik and C_jk
// come from shared memory and every row of C is read from memory once per
// level instead of once per common neighbour. The rank of {k} on side i is k's
// position in row i (the slot partner of (k, i)); the smallest separating rank
// per slot is kept by atomicMin, which is the rank the serial order finds
// first. Pivots are claimed in increasing order, so k's position in each of its
// rows grows as the level proceeds: a test whose slot already holds a smaller
// separating rank is skipped (read with the slot's other data), which cannot
// change that minimum.
// ---------------------------------------------------------------------------
// Staging of pivot rows by the bulk-copy engine: one thread starts a
// cp.async.bulk of the row's 16-byte-aligned middle into a shared buffer,
// completing on an mbarrier; the few entries before and after it are loaded
// by threads after the wait. The buffer holds the row from entry `mis` on, so
// source and destination share their 16-byte alignment.
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init1(unsigned long long* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase of parity `parity`, at most kBarrierNs; false on expiry
// (error flag 8 raised) or, with stop_on_error, when another CTA raised an
// error. Without it the wait only ends on completion or expiry (used to drain
// a copy in flight before the CTA leaves).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity, LevelMeta* lm,
                                                  bool stop_on_error = true)
{
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (unsigned it = 1;; ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 15u) == 0) {
            if (stop_on_error && *(volatile int*)&lm->error) return false;
            if (gtimer() - t0 > kBarrierNs) {
                atomicOr(&lm->error, 8);
                return false;
            }
        }
    }
}

struct PivotRow {
    int k;          // pivot (-1: none left)
    int mis;        // entry of the buffer holding the row's first entry
    int head;       // entries before the bulk-copied middle
    int body;       // entries bulk-copied
    int n;          // entries of the row
};

// Claims the next pivot with neighbours and starts copying its C row into buf
// (thread 0 only).
template <typename T>
__device__ void pivot_issue(const LevelParams& P, const Csr& A, T* buf, unsigned long long* bar, PivotRow& R)
{
    constexpr int V = 16 / sizeof(T);
    for (;;) {
        const unsigned long long kk = atomicAdd(&P.lm->next_item[1], 1ull);
        if (kk >= (unsigned long long)P.p) {
            R.k = -1;
            return;
        }
        const int k = (int)kk;
        if (A.row_off[k + 1] == A.row_off[k] || (P.vlmax && P.vlmax[k] < 1)) continue;
        const CView<T> CV = cview<T>(P, k);
        const T* src = CV.row(k) + CV.off;
        R.k = k;
        R.n = CV.p;
        R.mis = (int)(((uintptr_t)src & 15) / sizeof(T));
        R.head = min(CV.p, (V - R.mis) % V);
        R.body = ((CV.p - R.head) / V) * V;
        const uint32_t bytes = (uint32_t)(R.body * sizeof(T));
        if (bytes) {
            // the buffer's previous contents were read through the generic proxy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_addr(buf + R.mis + R.head)),
                "l"((unsigned long long)(src + R.head)), "r"(bytes), "r"(smem_addr(bar))
                : "memory");
        } else {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
        }
        return;
    }
}

// Decision of a level-1 test (minpiv2 = 1) as ci_decide, with the band's
// division by the smaller conditional variance done by the fast reciprocal
// (the band is a safety margin; its few-ulp rounding only moves its edge).
template <typename T, bool FP32>
__device__ __forceinline__ int l1_decide(T H11, T H12, T H22, const Decide& dc)
{
    if (!FP32) return ci_decide<T, false>(H11, H12, H22, T(1), dc);
    if (!(H22 > 1e-4f)) return 2;                  // (H11 is checked once per row)
    const float rho = fabsf((float)H12) * rsqrtf((float)(H11 * H22));
    const float band = dc.band_abs + __fdividef(dc.band_rel, fminf((float)H11, (float)H22));
    if (rho > dc.r + band) return 0;
    if (rho < dc.r - band) return 1;
    return 2;
}

constexpr int kL1Nb = 256;   // neighbours of the pivot staged per round
constexpr int kL1U = 4;      // slot loads in flight per lane

// LRN: the rank of {k} on side i is k's position in row i's learned order.
template <typename T, bool FP32, bool LRN>
__device__ void phase_l1_pivot(const LevelParams& P, const Csr& A, unsigned char* dyn)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __shared__ __align__(8) unsigned long long pbar[2];
    __shared__ PivotRow prow[2];
    __shared__ int sabort;
    // the rows i in adj(k) of one round: slot offset, degree, position of k
    __shared__ int nb_off[kL1Nb], nb_d[kL1Nb], nb_pos[kL1Nb], nb_i[kL1Nb];
    __shared__ int nb_rk[LRN ? kL1Nb : 1];
    const int nbuf = P.l1_pivot;
    const size_t bbytes = l1_buf_bytes(P.pstage, sizeof(T));
    T* buf[2] = {(T*)dyn, (T*)(dyn + (nbuf > 1 ? bbytes : 0))};
    unsigned ntests = 0;
    const T* __restrict__ cval = (const T*)P.cval;
    if (threadIdx.x == 0) {
        mbar_init1(&pbar[0]);
        mbar_init1(&pbar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sabort = 0;
        pivot_issue<T>(P, A, buf[0], &pbar[0], prow[0]);
    }
    __syncthreads();
    uint32_t par[2] = {0u, 0u};
    int b = 0;
    for (;;) {
        const PivotRow R = prow[b];
        if (R.k < 0) break;
        if (threadIdx.x == 0) {
            // the next pivot's row streams into the other buffer meanwhile
            if (nbuf > 1) pivot_issue<T>(P, A, buf[b ^ 1], &pbar[b ^ 1], prow[b ^ 1]);
            if (!mbar_wait_bounded(&pbar[b], par[b], P.lm)) {
                sabort = 1;
                mbar_wait_bounded(&pbar[b], par[b], P.lm, false);   // this buffer's copy, drained
            }
        }
        par[b] ^= 1u;
        T* row = buf[b] + R.mis;
        {
            const T* src = cview<T>(P, R.k).row(R.k) + cview<T>(P, R.k).off;
            const int tail0 = R.head + R.body;
            for (int c = threadIdx.x; c < R.head; c += NT) row[c] = __ldg(src + c);
            for (int c = tail0 + threadIdx.x; c < R.n; c += NT) row[c] = __ldg(src + c);
        }
        const int k = R.k;
        const long long offk = A.row_off[k];
        const int dk = (int)(A.row_off[k + 1] - offk);
        double thr, thr2;
        thresholds(P, k, thr, thr2);
        const Decide dc = decide_consts(P, thr, thr2);
        const T* __restrict__ sk_row = row - cview<T>(P, k).off;   // indexed by global column ids
        for (int t0 = 0; t0 < dk; t0 += kL1Nb) {
            const int nt = min(kL1Nb, dk - t0);
            __syncthreads();                       // the previous round's metadata is no longer read
            for (int t = threadIdx.x; t < nt; t += NT) {
                const int i = A.cols[offk + t0 + t];
                const long long offi = A.row_off[i];
                nb_i[t] = i;
                nb_off[t] = (int)offi;
                nb_d[t] = (int)(A.row_off[i + 1] - offi);
                const int sk = A.partner[offk + t0 + t];            // slot (i, k)
                nb_pos[t] = sk - (int)offi;
                if (LRN) nb_rk[t] = P.iperm[sk];
            }
            __syncthreads();                       // (the first one also publishes the staged row)
            if (sabort) break;
            for (int t = w; t < nt; t += NW) {
                const int di = nb_d[t];
                if (di < 2) continue;
                const int offi = nb_off[t], posk = nb_pos[t];
                const unsigned long long rk = (unsigned long long)(LRN ? nb_rk[t] : posk);
                const T cik = sk_row[nb_i[t]];
                const T H11 = T(1) - cik * cik;
                // (FP32: a tiny conditional variance sends every test of the row to FP64)
                const bool h11_ok = !FP32 || (float)H11 > 1e-4f;
                for (int q0 = 0; q0 < di; q0 += 32 * kL1U) {
                    int jj[kL1U];
                    T cv[kL1U];
                    unsigned long long be[kL1U];
#pragma unroll
                    for (int u = 0; u < kL1U; ++u) {
                        const int q = q0 + 32 * u + lane;
                        const bool in = q < di && q != posk;
                        jj[u] = in ? A.cols[offi + q] : 0;
                        cv[u] = in ? cval[offi + q] : T(0);
                        // the slot's smallest separating rank so far: a test of a
                        // larger rank cannot change the result (canonical mode), nor
                        // can any test once the slot has one (free mode)
                        be[u] = in ? __ldcg(P.best + offi + q) : 0ull;
                    }
#pragma unroll
                    for (int u = 0; u < kL1U; ++u) {
                        const bool go = P.canonical ? (be[u] > rk) : (be[u] == RANK_NONE);
                        if (go) {
                            const int e = offi + q0 + 32 * u + lane;
                            const T cjk = sk_row[jj[u]];
                            const T H12 = cv[u] - cik * cjk;
                            const T H22 = T(1) - cjk * cjk;
                            ++ntests;
                            const int dec = h11_ok ? l1_decide<T, FP32>(H11, H12, H22, dc) : 2;
                            if (dec == 1) {
                                atomicMin(P.best + e, rk);
                            } else if (FP32 && dec == 2) {
                                const unsigned long long qq = atomicAdd(&P.lm->queue_len[1], 1ull);
                                if (qq < P.qcap) {
                                    QEntry* Q = P.queue + qq;
                                    Q->a = e;
                                    Q->b = 0;
                                    Q->s = rk;
                                    Q->S[0] = k;
                                }
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();                           // buffer b and the metadata are no longer read
        if (sabort) break;
        if (nbuf > 1) {
            b ^= 1;
        } else if (threadIdx.x == 0) {
            pivot_issue<T>(P, A, buf[0], &pbar[0], prow[0]);
        }
        __syncthreads();                           // the next pivot's descriptor is visible
    }
    if (sabort && threadIdx.x == 0 && nbuf > 1 && prow[b ^ 1].k >= 0) {
        // a copy may still be in flight into the other buffer: wait for it
        // (bounded) before the CTA leaves
        mbar_wait_bounded(&pbar[b ^ 1], par[b ^ 1], P.lm, false);
    }
    const unsigned long long nt64 = warp_sum_u64((unsigned long long)ntests);
    if (lane == 0 && nt64) atomicAdd(&P.lm->tests[1], nt64);
}

// ---------------------------------------------------------------------------
// P5: FP64 rechecks. The samples of each queued test are cut into S slices
// (S depends on n only, so the summation order is fixed); CTAs take (test,
// slice) units and write partial Gram sums of the test's l + 2 standardised
// rows, then after a barrier one CTA per test adds its slices in order, forms
// H in FP64 and decides. A single SM's FP64 rate is low on this part, so
// spreading each test over several SMs shortens the phase when few tests
// are queued. The queue is processed in batches that fit the partial buffer.
// ---------------------------------------------------------------------------

// Data row of vertex v for the rechecks (its problem's rows in a batch) and
// its problem's sample count.
__device__ __forceinline__ XRow xrow(const LevelParams& P, int v, int& n)
{
    const int es = P.xf64 ? 8 : 4;
    const ProbDesc* D = prob_of(P.vprob, P.probs, v);
    XRow r;
    r.f64 = P.xf64;
    r.mu = P.mu[v];
    r.isd = P.isd[v];
    if (D) {
        r.p = (const char*)D->xv + (size_t)(v - D->off) * D->n * es;
        n = D->n;
    } else {
        r.p = (const char*)P.xv + (size_t)v * P.ldx * es;
        n = P.n;
    }
    return r;
}

// FP32 data: the row as read by the compensated rechecks, and 1/n of v's problem.
__device__ __forceinline__ XRowP xrowp(const LevelParams& P, int v, int& n)
{
    const ProbDesc* D = prob_of(P.vprob, P.probs, v);
    XRowP r;
    const float2 m = P.mup[v];
    r.mh = m.x;
    r.ml = m.y;
    if (D) {
        r.p = (const float*)D->xv + (size_t)(v - D->off) * D->n;
        n = D->n;
    } else {
        r.p = (const float*)P.xv + (size_t)v * P.ldx;
        n = P.n;
    }
    return r;
}

__device__ __forceinline__ double inv_n_of(const LevelParams& P, int v)
{
    const ProbDesc* D = prob_of(P.vprob, P.probs, v);
    return D ? D->inv_n : P.inv_n;
}

__device__ __forceinline__ int n_of(const LevelParams& P, int v)
{
    const ProbDesc* D = prob_of(P.vprob, P.probs, v);
    return D ? D->n : P.n;
}

// Lanes of a recheck warp: entry x of the Gram block (x = lane mod DP, DP = D
// rounded up to a power of two, at most 32) and sample (or slice) group
// g = lane / DP of G = 32 / DP; the rolled loops below keep the code small,
// since a level runs this phase once, from a cold instruction cache.
template <int LB>
struct RecheckLanes {
    static constexpr int M = LB + 2;
    static constexpr int D = M * (M - 1) / 2;
    static constexpr int DP = D <= 4 ? 4 : D <= 8 ? 8 : D <= 16 ? 16 : 32;
    static constexpr int G = 32 / DP;
};

// Packed Gram index x -> (a, b2), a < b2: x = b2 (b2 - 1) / 2 + a.
__device__ __forceinline__ void gram_pair(int x, int& a, int& b2)
{
    b2 = 1;
    while ((b2 + 1) * b2 / 2 <= x) ++b2;
    a = x - b2 * (b2 - 1) / 2;
}

// Asks L2 for the 128-byte lines of bytes [b0, b1) of a row, lines g, g + G,
// ... of them, so that a lane's sequential walk through its slice does not
// wait on one line at a time.
__device__ __forceinline__ void prefetch_lines(const char* base, long long b0, long long b1, int g, int G)
{
    for (long long c = (b0 >> 7) + g; c <= ((b1 - 1) >> 7); c += G)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(base + (c << 7)));
}

// Member g of the test's (i, j, S) list (0 = i, 1 = j, 2 + c = S_c).
__device__ __forceinline__ int gram_var(const QEntry* E, int i, int j, int g)
{
    return g == 0 ? i : g == 1 ? j : E->S[g - 2];
}

// Gram entries sum_s (x_as - mu_a)(x_bs - mu_b) over sample slice k of S of
// one queued test, by one warp: the lanes of entry x stride the slice by G and
// a fixed xor tree adds the G groups. FP32 data: compensated FP32 pairs
// (pair_dot_acc, folded every 8 samples; about 2^-48 relative per term like an
// FP64 sum), out as the pair (hi, lo) per entry; FP64 data: FP64 fma, out as
// a double.
template <int LB, bool PAIRS>
__device__ __forceinline__ void recheck_unit(const LevelParams& P, const QEntry* E, int i, int j, int k, int S,
                                             double* out)
{
    using L = RecheckLanes<LB>;
    const int lane = threadIdx.x & 31, g = lane / L::DP;
    const int m = P.l + 2;
    const int zn = n_of(P, i);
    const int k0 = (int)((long long)zn * k / S), k1 = (int)((long long)zn * (k + 1) / S);
    for (int x0 = 0; x0 < L::D; x0 += L::DP) {
        const int x = x0 + lane % L::DP;
        int a, b2;
        gram_pair(x, a, b2);
        const bool act = x < L::D && b2 < m;
        int dummy;
        if constexpr (PAIRS) {
            float h = 0.f, lo = 0.f;
            if (act) {
                const XRowP A = xrowp(P, gram_var(E, i, j, a), dummy), B = xrowp(P, gram_var(E, i, j, b2), dummy);
                if (k1 > k0) {
                    prefetch_lines((const char*)A.p, 4ll * k0, 4ll * k1, g, L::G);
                    prefetch_lines((const char*)B.p, 4ll * k0, 4ll * k1, g, L::G);
                }
                for (int kb = k0 + g; kb < k1; kb += L::G * 8) {
                    const int ke = min(k1, kb + L::G * 8);
#pragma unroll 2
                    for (int kk = kb; kk < ke; kk += L::G) {
                        float ah, al, bh, bl;
                        A.centred(kk, ah, al);
                        B.centred(kk, bh, bl);
                        pair_dot_acc(h, lo, ah, al, bh, bl);
                    }
                    two_sum(h, lo, h, lo);
                }
            }
#pragma unroll
            for (int o = 16; o >= L::DP; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
                pair_add(h, lo, oh, ol);
            }
            if (x < L::D && g == 0) ((float2*)out)[x] = make_float2(h, lo);
        } else {
            double acc = 0.0;
            if (act) {
                const XRow A = xrow(P, gram_var(E, i, j, a), dummy), B = xrow(P, gram_var(E, i, j, b2), dummy);
                const double* pa = (const double*)A.p;
                const double* pb = (const double*)B.p;
                if (k1 > k0) {
                    prefetch_lines((const char*)pa, 8ll * k0, 8ll * k1, g, L::G);
                    prefetch_lines((const char*)pb, 8ll * k0, 8ll * k1, g, L::G);
                }
#pragma unroll 4
                for (int kk = k0 + g; kk < k1; kk += L::G) acc = fma(__ldg(pa + kk) - A.mu, __ldg(pb + kk) - B.mu, acc);
            }
#pragma unroll
            for (int o = 16; o >= L::DP; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (x < L::D && g == 0) out[x] = acc;
        }
    }
}

// A queued test whose outcome cannot change the level's result: the edge's
// removal is already decided by a definitive FP32 independence at a smaller
// rank on the side that wins (canonical: the smaller endpoint's side first,
// then the smaller rank), or by any definitive independence (non-canonical).
// best[] does not change while this is evaluated (it is written only after the
// grid barrier that follows), so every slice of a test agrees.
__device__ __forceinline__ bool recheck_moot(const LevelParams& P, const Csr& A, long long e, int i, int j, unsigned long long s)
{
    const unsigned long long be = ld_cg(P.best + e);
    const unsigned long long bf = ld_cg(P.best + A.partner[e]);
    if (!P.canonical) return be != RANK_NONE || bf != RANK_NONE;
    if (i < j) return be < s;                      // this side is the first one
    return bf != RANK_NONE || be < s;              // the first side already removes it
}

// Gram entries of one slice of a queued test, summed over the NW warps of the
// CTA in warp order by warp 0: out[x] (x < D) as an FP32 pair (pairs) or a
// double. Must be called by the whole CTA.
template <int LB>
__device__ __forceinline__ void recheck_slice(const LevelParams& P, const Csr& A, const QEntry* E, int i, int j, int s, int S,
                                              bool pairs, double (*sred)[(LB + 2) * (LB + 1) / 2], double* out)
{
    constexpr int D = (LB + 2) * (LB + 1) / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (pairs)
        recheck_unit<LB, true>(P, E, i, j, s * NW + warp, S * NW, &sred[warp][0]);
    else
        recheck_unit<LB, false>(P, E, i, j, s * NW + warp, S * NW, &sred[warp][0]);
    __syncthreads();
    if (warp == 0) {
        for (int x = lane; x < D; x += 32) {
            if (pairs) {
                float h = 0.f, lo = 0.f;
                for (int w2 = 0; w2 < NW; ++w2) {
                    const float2 t2 = ((const float2*)&sred[w2][0])[x];
                    pair_add(h, lo, t2.x, t2.y);
                }
                ((float2*)out)[x] = make_float2(h, lo);
            } else {
                double v = 0.0;
                for (int w2 = 0; w2 < NW; ++w2) v += sred[w2][x];
                out[x] = v;
            }
        }
    }
}

// Decision of a recheck by warp 0 from its Gram entries (slices already
// added: g[x] as a pair or a double, or C64 when given): eliminates the
// members of S from the (l + 2) x (l + 2) correlation block of (S, i, j); the
// trailing 2 x 2 Schur complement is the conditional covariance of (V_i, V_j)
// given S (Eq. PartialCorMat). A member whose remaining pivot is at or below
// the rank tolerance is linearly dependent on the members before it and is
// dropped (the pseudo-inverse's treatment). Returns independence (lane 0).
template <int LB>
__device__ __forceinline__ void recheck_eliminate(const LevelParams& P, const QEntry* E, int i, int j, bool pairs,
                                                  const double* g, double (*sA)[LB + 2], double& H11, double& H12,
                                                  double& H22)
{
    constexpr int M = LB + 2;
    constexpr int D = M * (M - 1) / 2;
    const int lane = threadIdx.x & 31;
    const int l = P.l, m = l + 2;
    int V[M];
    V[0] = i;
    V[1] = j;
#pragma unroll
    for (int q = 0; q < LB; ++q) V[2 + q] = (q < l) ? E->S[q] : i;
    // elimination position of Gram index x (0 = i, 1 = j, 2 + a = S_a)
    auto pos = [&](int x) { return x >= 2 ? x - 2 : l + x; };
    const double inv_n = inv_n_of(P, i);
    for (int x = lane; x < D; x += 32) {
        int a, b2;
        gram_pair(x, a, b2);
        if (b2 < m) {
            const int pa = pos(a), pb = pos(b2);
            double v;
            if (P.c64) {
                v = P.c64[(size_t)V[a] * P.p + V[b2]];
            } else {
                const double raw = pairs ? widen_f32(((const float2*)g)[x].x) + widen_f32(((const float2*)g)[x].y)
                                         : g[x];
                v = raw * (P.isd[V[a]] * P.isd[V[b2]]) * inv_n;
            }
            sA[max(pa, pb)][min(pa, pb)] = v;
        }
    }
    if (lane < m) sA[lane][lane] = 1.0;
    __syncwarp();
    // lower triangle only: step k updates A[a][b], k < b <= a < m
    for (int k = 0; k < l; ++k) {
        const double piv = sA[k][k];
        if (piv > P.rank_tol) {
            const double rp = 1.0 / piv;
            const int r = m - k - 1;
            for (int q = lane; q < r * (r + 1) / 2; q += 32) {
                int aa = 0;
                while ((aa + 1) * (aa + 2) / 2 <= q) ++aa;
                const int bb = q - aa * (aa + 1) / 2;
                const int a = k + 1 + aa, b = k + 1 + bb;
                sA[a][b] = fma(-sA[a][k] * rp, sA[b][k], sA[a][b]);
            }
        }
        __syncwarp();
    }
    H11 = sA[l][l];
    H12 = sA[l + 1][l];
    H22 = sA[l + 1][l + 1];
    __syncwarp();
}

template <int LB>
__device__ __forceinline__ bool recheck_decide(const LevelParams& P, const Csr& A, const QEntry* E, int i, int j,
                                               bool pairs, const double* g, double (*sA)[LB + 2])
{
    double H11, H12, H22;
    recheck_eliminate<LB>(P, E, i, j, pairs, g, sA, H11, H12, H22);
    double thr, thr2;
    thresholds(P, i, thr, thr2);
    return (!(H11 > kVarZero) || !(H22 > kVarZero)) ? true : (H12 * H12 <= thr2 * H11 * H22);
}

// rho(V_i, V_j | S) of a batch of queries with the recheck arithmetic (for
// verification): a warp per query, all samples in one slice.
constexpr int kPcW = 4;
template <int LB>
__global__ void __launch_bounds__(32 * kPcW) k_pcor_recheck(LevelParams P, const int* __restrict__ q, long long nq,
                                                             double* __restrict__ rho)
{
    constexpr int M = LB + 2;
    constexpr int D = M * (M - 1) / 2;
    __shared__ double sA[kPcW][M][M];
    __shared__ double sred[kPcW][D];
    __shared__ QEntry sE[kPcW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long t = (long long)blockIdx.x * kPcW + warp;
    if (t >= nq) return;
    const int* row = q + t * (2 + P.l);
    const int i = row[0], j = row[1];
    if (lane < CUPC_MAX_LEVEL) sE[warp].S[lane] = (lane < P.l) ? row[2 + lane] : i;
    __syncwarp();
    const bool pairs = !P.xf64;
    if (pairs)
        recheck_unit<LB, true>(P, &sE[warp], i, j, 0, 1, &sred[warp][0]);
    else
        recheck_unit<LB, false>(P, &sE[warp], i, j, 0, 1, &sred[warp][0]);
    __syncwarp();
    double H11, H12, H22;
    recheck_eliminate<LB>(P, &sE[warp], i, j, pairs, &sred[warp][0], sA[warp], H11, H12, H22);
    if (lane == 0) rho[t] = (H11 > kVarZero && H22 > kVarZero) ? H12 / sqrt(H11 * H22) : nan("");
}

// FP64 rechecks of the queued tests. (1) The tests whose outcome can still
// matter are listed (one grid barrier). (2) Each listed test is cut into S
// sample slices, S = 1 when the tests outnumber the CTAs, else up to 16 so
// that few tests still spread over many SMs; a CTA takes one (test, slice)
// unit, its NW warps form the slice's Gram entries of the m = l + 2 variables
// over NW sub-slices (FP64, or compensated FP32 pairs for FP32 data) and add
// them in warp order. With S > 1 each CTA stores its slice's sums and the CTA
// that completes a test (a counter per test) adds the S slices in slice order
// and decides; no further grid barrier is needed. The slices depend on n and
// S only, and S on the number of listed tests, so a test's FP64 value does not
// depend on which CTAs compute it.
template <int LB>
__device__ bool phase_recheck(const LevelParams& P, const Csr& A, unsigned long long nq)
{
    constexpr int M = LB + 2;
    constexpr int D = M * (M - 1) / 2;
    constexpr int NA = LB <= 8 ? NW : 1;           // elimination blocks (one per warp in warp mode)
    __shared__ double sA[NA][M][M];
    __shared__ double sred[NW][D];                 // per warp: its sub-slice's Gram entries
    __shared__ double sg[D];                       // the slice (or test) sums
    __shared__ unsigned long long su;
    __shared__ int slast;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool timer = (blockIdx.x == 0 && threadIdx.x == 0);
    // FP32 data: Gram sums in compensated FP32 pairs (GB300's FP64 pipe is narrow)
    const bool pairs = !P.c64 && !P.xf64;
    const unsigned long long tp = timer ? gtimer() : 0;
    // (1) the queued tests whose outcome can still matter, in queue order
    for (long long t = (long long)blockIdx.x * NT + threadIdx.x; t < (long long)nq; t += (long long)gridDim.x * NT) {
        const QEntry* E = P.queue + t;
        const long long e = E->a;
        if (!recheck_moot(P, A, e, A.srow[e], A.cols[e], E->s)) {
            const unsigned long long w = atomicAdd(&P.lm->live[P.l], 1ull);
            P.live[w] = (int)t;
            if (w < (unsigned long long)kRcCnt) P.rc_cnt[w] = 0;
        }
    }
    if (!grid_sync(P)) return false;
    const unsigned long long nl = ld_cg(&P.lm->live[P.l]);
    unsigned long long done = 0;
    if (LB <= 8 && nl >= (unsigned long long)gridDim.x) {
        // (2') at least as many tests as CTAs: a warp takes a whole test (all
        // samples in one slice) and decides it
        const long long gw = (long long)warp * gridDim.x + blockIdx.x;
        for (long long ti = gw; ti < (long long)nl; ti += (long long)gridDim.x * NW) {
            const QEntry* E = P.queue + P.live[ti];
            const long long e = E->a;
            const int i = A.srow[e], j = A.cols[e];
            if (!P.c64) {
                if (pairs)
                    recheck_unit<LB, true>(P, E, i, j, 0, 1, &sred[warp][0]);
                else
                    recheck_unit<LB, false>(P, E, i, j, 0, 1, &sred[warp][0]);
            }
            __syncwarp();
            const bool indep = recheck_decide<LB>(P, A, E, i, j, pairs, &sred[warp][0], sA[warp % NA]);
            if (lane == 0) {
                ++done;
                if (indep) atomicMin(P.best + e, E->s);
            }
            __syncwarp();
        }
        if (timer) P.lm->recheck_ns[P.l][0] += gtimer() - tp;
        done = warp_sum_u64(done);
        if (lane == 0 && done) atomicAdd(&P.lm->rechecks[P.l], done);
        return true;
    }
    // (2) units (test, slice)
    int S = 1;
    if (!P.c64 && nl < (unsigned long long)gridDim.x && nl < (unsigned long long)kRcCnt) {
        S = (int)min(16ull, (unsigned long long)gridDim.x / max(nl, 1ull));
        // slice sums of every test must fit the partial buffer (pairs: one double each)
        while (S > 1 && (unsigned long long)S * nl * D > P.part_cap) --S;
    }
    const unsigned long long units = nl * (unsigned long long)S;
    for (;;) {
        __syncthreads();                           // sg / sA of the previous unit are no longer read
        if (threadIdx.x == 0) su = atomicAdd(&P.lm->rc_next[P.l], 1ull);
        __syncthreads();
        const unsigned long long u = su;
        if (u >= units) break;
        const unsigned long long ti = u / S;
        const int sl = (int)(u % S);
        const QEntry* E = P.queue + P.live[ti];
        const long long e = E->a;
        const int i = A.srow[e], j = A.cols[e];
        if (!P.c64) recheck_slice<LB>(P, A, E, i, j, sl, S, pairs, sred, (S == 1) ? sg : P.part + (ti * S + sl) * D);
        bool last = (S == 1);
        if (S > 1) {
            // publish this slice; the CTA that brings the test's count to S decides
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) slast = (atomicAdd(&P.rc_cnt[ti], 1) == S - 1) ? 1 : 0;
            __syncthreads();
            last = slast != 0;
            if (last && warp == 0 && !P.c64) {
                __threadfence();
                for (int x = lane; x < D; x += 32) {
                    if (pairs) {
                        float h = 0.f, lo = 0.f;
                        for (int s2 = 0; s2 < S; ++s2) {
                            const float2 t2 = __ldcg((const float2*)(P.part + (ti * S + s2) * D) + x);
                            pair_add(h, lo, t2.x, t2.y);
                        }
                        ((float2*)sg)[x] = make_float2(h, lo);
                    } else {
                        double v = 0.0;
                        for (int s2 = 0; s2 < S; ++s2) v += __ldcg(P.part + (ti * S + s2) * D + x);
                        sg[x] = v;
                    }
                }
            }
        }
        __syncthreads();
        if (last && warp == 0) {
            const bool indep = recheck_decide<LB>(P, A, E, i, j, pairs, sg, sA[0]);
            if (lane == 0) {
                ++done;
                if (indep) atomicMin(P.best + e, E->s);
            }
        }
    }
    if (timer) P.lm->recheck_ns[P.l][0] += gtimer() - tp;
    if (threadIdx.x == 0 && done) atomicAdd(&P.lm->rechecks[P.l], done);
    return true;
}

// ---------------------------------------------------------------------------
// P6: an edge (x < y) is removed when either side found a separating set; the
// SepSet is the smaller side's when it has one (the serial order). With
// canonical SepSets the tests the serial order performs are counted: side x
// up to and including its first separating set (or all), side y only when
// side x found none.
// ---------------------------------------------------------------------------
template <int LB>
__device__ __forceinline__ unsigned long long side_serial(const LevelParams& P, const Csr& A, int a, long long slot_b,
                                                          unsigned long long rank, bool lrn)
{
    const long long off = A.row_off[a];
    const int d = (int)(A.row_off[a + 1] - off);
    if (rank == RANK_NONE) return P.B(d - 1, P.l);
    int Pos[LB];
    unrank_lex<LB>(rank, d, P.l, P.B, Pos);
    const int pb = lrn ? P.iperm[slot_b] : (int)(slot_b - off);   // b's position in the row's order
#pragma unroll
    for (int c = 0; c < LB; ++c)
        if (c < P.l && Pos[c] > pb) Pos[c] -= 1;
    return rank_lex<LB>(Pos, d - 1, P.l, P.B) + 1;
}

// Members of the separating set of rank `rank` found on side a, in increasing order.
template <int LB>
__device__ __forceinline__ void side_members(const LevelParams& P, const Csr& A, int a, unsigned long long rank,
                                             bool lrn, int (&S)[LB])
{
    const long long off = A.row_off[a];
    const int d = (int)(A.row_off[a + 1] - off);
    int Pos[LB];
    unrank_lex<LB>(rank, d, P.l, P.B, Pos);
#pragma unroll
    for (int c = 0; c < LB; ++c) S[c] = (c < P.l) ? A.cols[off + (lrn ? P.perm[off + Pos[c]] : Pos[c])] : 0x7fffffff;
    if (lrn) {
#pragma unroll
        for (int x = 1; x < LB; ++x)
#pragma unroll
            for (int y = LB - 1; y >= x; --y)
                if (S[y - 1] > S[y]) { const int tmp = S[y - 1]; S[y - 1] = S[y]; S[y] = tmp; }
    }
}

template <int LB>
__device__ void phase_finalize(const LevelParams& P, const Csr& A, bool lrn)
{
    const long long nnz = A.row_off[P.p];
    const int l = P.l;
    for (long long e0 = (long long)blockIdx.x * NT; e0 < nnz; e0 += (long long)gridDim.x * NT) {
        const long long e = e0 + threadIdx.x;
        bool removed = false;
        unsigned long long serial = 0;
        if (e < nnz) {
            const int x = A.srow[e], y = A.cols[e];
            if (x < y) {
                const long long f = A.partner[e];
                const unsigned long long bx = ld_cg(P.best + e), by = ld_cg(P.best + f);
                int side = -1;
                unsigned long long rank = 0;
                if (bx != RANK_NONE) { side = x; rank = bx; }
                else if (by != RANK_NONE) { side = y; rank = by; }
                if (side >= 0) {
                    removed = true;
                    const ProbDesc* Dx = prob_of(P.vprob, P.probs, x);
                    bitset_clear_pair_at(P.bits, rowbase(Dx, P.W, x), rowbase(Dx, P.W, y), x, y);
                    atomicSub(P.deg + x, 1);
                    atomicSub(P.deg + y, 1);
                    int S[LB];
                    side_members<LB>(P, A, side, rank, lrn, S);
                    const int ints = 3 + l;
                    const unsigned long long at = atomicAdd(&P.lm->rec_ints, (unsigned long long)ints);
                    if (at + ints <= P.rec_cap) {
                        int* r = P.rec + at;
                        r[0] = x;
                        r[1] = y;
                        r[2] = l;
#pragma unroll
                        for (int c = 0; c < LB; ++c)
                            if (c < l) r[3 + c] = S[c];
                    }
                }
                P.alive[e] = removed ? 0 : 1;
                P.alive[f] = removed ? 0 : 1;
                if (P.canonical) {
                    serial = side_serial<LB>(P, A, x, e, bx, lrn);
                    if (bx == RANK_NONE) serial += side_serial<LB>(P, A, y, f, by, lrn);
                    if (P.prob_serial && serial) atomicAdd(P.prob_serial + (size_t)P.vprob[x] * LV + l, serial);
                }
            }
        }
        const unsigned long long nrem = warp_sum_u64(removed ? 1ull : 0ull);
        const unsigned long long ns = warp_sum_u64(serial);
        if ((threadIdx.x & 31) == 0) {
            if (nrem) atomicAdd(&P.lm->removed[l], nrem);
            if (ns) atomicAdd(&P.lm->serial[l], ns);
        }
    }
}

// ---------------------------------------------------------------------------
// The level kernel
// ---------------------------------------------------------------------------
// Tells the host whether this level runs (1, with the level's starting max
// degree in bits 4 and up) or the loop has ended (2), through pinned host
// memory the host polls to decide on further launches.
// The store is not fenced: the host only waits a little longer when it lands
// late (at the latest when the kernel ends), while a system-scope fence would
// hold this thread, and the barrier after it, for microseconds.
__device__ __forceinline__ void signal_host(const LevelParams& P, int v)
{
    if (P.host_flags) *(volatile int*)(P.host_flags + P.l) = v;
}

template <typename T, int LB, bool FP32, bool LEARNED>
// (two CTAs per SM at level 1, except with the learned order, whose scoring
// keeps a candidate's 64 hidden units in registers)
__global__ void __launch_bounds__(NT, (LB == 1 && !LEARNED) ? 2 : 1) k_level(LevelParams P)
{
    LevelMeta* lm = P.lm;
    const int l = P.l;
    // a previous level ended the loop (termination, overflow or error), or level 0
    // failed (an error, or its recheck queue overflowed: its decisions are incomplete)
    const bool level0_bad =
        P.meta0 && (*(volatile const int*)&P.meta0->error != 0 || ld_cg(&P.meta0->queue_len) > P.qcap0);
    if (level0_bad || *(volatile int*)&lm->done_level || *(volatile int*)&lm->overflow_level ||
        *(volatile int*)&lm->error) {
        if (blockIdx.x == 0 && threadIdx.x == 0) signal_host(P, 2);
        return;
    }
    if (P.barrier_ns && blockIdx.x == 0) {
        // test of the barrier-expiry path: this CTA never arrives at the first
        // grid barrier (a generation that nothing advances), so every other CTA
        // waits out P.barrier_ns there, raises the error and ends; no CTA passes
        // that barrier
        if (threadIdx.x == 0) signal_host(P, 2);
        return;
    }
    unsigned long long t0 = 0, t1;
    const bool timer = (blockIdx.x == 0 && threadIdx.x == 0);
    if (timer) t0 = gtimer();

    // A'_G of the previous level is still valid when that level removed no edge:
    // the neighbour lists, partner slots and word prefixes are reused (the work
    // items, which depend on l, are rebuilt)
    // A level after one that removed edges builds its A'_G from that level's
    // (incr) into the other buffer; the first level and a rerun build it from the
    // bitset A_G
    const int cur = *(volatile int*)&lm->csr_cur;
    const bool prev = l >= 2 && *(volatile int*)&lm->csr_level == l - 1;
    const bool reuse = prev && ld_cg(&lm->removed[l - 1]) == 0ull;
    const bool incr = prev && !reuse;
    const int nbuf = reuse ? cur : 1 - cur;
    const Csr A = csr_view(P, nbuf);
    const Csr O = csr_view(P, cur);
    // learned order: every level's rows are ordered when their A'_G is built
    // (a reused A'_G keeps its order)
    const bool lrn = LEARNED && P.learned;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    // one CTA scans graphs up to kScanOne rows (no second barrier); larger ones
    // are scanned by every CTA over its own rows, then offset by the others'
    // totals after a grid barrier
    const bool one = P.p <= kScanOne;
    if (one) {
        if (blockIdx.x == 0) phase_scan_one(P, A);
        if (!reuse && (blockIdx.x != 0 || gridDim.x == 1)) {
            if (incr) {
                if (lrn) phase_rank<LEARNED>(P, O, 1);
                else phase_rank<false>(P, O, 1);
            } else {
                phase_prefix(P, 1);
            }
        }
    } else {
        phase_scan_a(P);
        if (incr) {
            if (lrn) phase_rank<LEARNED>(P, O, 0);
            else phase_rank<false>(P, O, 0);
        } else if (!reuse) {
            phase_prefix(P, 0);
        }
    }
    if (!grid_sync(P)) {
        if (timer) signal_host(P, 2);
        return;
    }
    if (timer) lm->csr_cur = nbuf;                 // every CTA read the old value before the barrier
    if (*(volatile int*)&lm->maxdeg[l] - 1 < l || *(volatile int*)&lm->range_error) {
        if (timer) {
            lm->done_level = l;
            signal_host(P, 2);
        }
        return;
    }
    if (timer) signal_host(P, 1 | (min(*(volatile int*)&lm->maxdeg[l], 1 << 26) << 4));
    if (!one) {
        if (!phase_scan_b(P, A)) return;
        if (!grid_sync(P)) return;
    }
    const bool pivot = (LB == 1) && l == 1 && P.l1_pivot;
    if (lrn) phase_fill<T, LEARNED>(P, A, O, reuse, incr, pivot);
    else phase_fill<T, false>(P, A, O, reuse, incr, pivot);
    if (!grid_sync(P)) return;
    if (LEARNED && lrn && !reuse && !incr) {
        // an A'_G built from the bitset: score and order its rows
        unsigned long long s0 = 0, s1 = 0;
        if (timer) s0 = gtimer();
        phase_lrn_score(P, A, dyn_smem);
        if (!grid_sync(P)) return;
        if (timer) s1 = gtimer();
        phase_lrn_rank(P, A);
        if (!grid_sync(P)) return;
        if (timer) {
            lm->order_ns[l][0] += s1 - s0;
            lm->order_ns[l][1] += gtimer() - s1;
        }
    }
    if (timer) {
        lm->csr_level = l;
        lm->learned_on[l] = lrn ? 1 : 0;
        t1 = gtimer();
        lm->phase_ns[l][0] += t1 - t0;
        t0 = t1;
    }

    if (pivot) {
        if (lrn) phase_l1_pivot<T, FP32, LEARNED>(P, A, dyn_smem);
        else phase_l1_pivot<T, FP32, false>(P, A, dyn_smem);
    } else {
        if (lrn) phase_ci<T, LB, FP32, LEARNED>(P, A);
        else phase_ci<T, LB, FP32, false>(P, A);
    }
    if (!grid_sync(P)) return;
    if (timer) { t1 = gtimer(); lm->phase_ns[l][1] += t1 - t0; t0 = t1; }

    if (FP32) {
        const unsigned long long nq = ld_cg(&lm->queue_len[l]);
        if (nq > P.qcap) {
            // the queue overflowed: stop; the host enlarges it and reruns this level
            if (timer) lm->overflow_level = l;
            return;
        }
        if (nq > 0) {
            if (!phase_recheck<LB>(P, A, nq)) return;
            if (!grid_sync(P)) return;            // every recheck decided before the removals
        }
        if (timer) { t1 = gtimer(); lm->phase_ns[l][2] += t1 - t0; t0 = t1; }
    }
    phase_finalize<LB>(P, A, lrn);
    if (timer) {
        t1 = gtimer();
        lm->phase_ns[l][3] += t1 - t0;
    }
}

template <typename T, int LB, bool FP32, bool LEARNED>
cudaError_t launch_level_t(const LevelParams& P, int num_sms, cudaStream_t st)
{
    // level-1 instances reserve shared memory for the pivot form's staged row
    // (the largest problem's p entries), learned-order instances the warps'
    // scoring scratch (the same memory at level 1: the phases do not overlap);
    // one occupancy per reserved size
    size_t dyn = (LB == 1 && P.l1_pivot) ? (size_t)P.l1_pivot * l1_buf_bytes(P.pstage, sizeof(T)) : 0;
    if (LEARNED && P.learned) dyn = dyn > kLrnBytes ? dyn : kLrnBytes;
    static int per_sm = 0;
    static size_t per_sm_dyn = 0;
    if (per_sm == 0 || per_sm_dyn != dyn) {
        if (LB == 1 || LEARNED) {
            cudaError_t e = cudaFuncSetAttribute(k_level<T, LB, FP32, LEARNED>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kL1StageBytes);
            if (e != cudaSuccess) return e;
        }
        cudaError_t e =
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_level<T, LB, FP32, LEARNED>, NT, dyn);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        per_sm = per_sm > 2 ? 2 : per_sm;
        per_sm_dyn = dyn;
    }
    // CTAs per SM: as many as fit, at most 2, or fewer when asked
    const int k = (P.ctas_per_sm > 0 && P.ctas_per_sm < per_sm) ? P.ctas_per_sm : per_sm;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(num_sms * k);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs resident: the grid barrier relies on it
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_level<T, LB, FP32, LEARNED>, P);
}

template <typename T, bool FP32, bool LEARNED>
cudaError_t launch_level_b(const LevelParams& P, int num_sms, cudaStream_t st)
{
    if (P.l <= 1) return launch_level_t<T, 1, FP32, LEARNED>(P, num_sms, st);
    if (P.l <= 2) return launch_level_t<T, 2, FP32, LEARNED>(P, num_sms, st);
    if (P.l <= 4) return launch_level_t<T, 4, FP32, LEARNED>(P, num_sms, st);
    if (P.l <= 8) return launch_level_t<T, 8, FP32, LEARNED>(P, num_sms, st);
    if (P.l <= 12) return launch_level_t<T, 12, FP32, LEARNED>(P, num_sms, st);
    return launch_level_t<T, 16, FP32, LEARNED>(P, num_sms, st);
}

}  // namespace

cudaError_t launch_pcor_recheck(const LevelParams& P, const int* q, long long nq, double* rho, cudaStream_t st)
{
    if (nq <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((nq + kPcW - 1) / kPcW);
    if (P.l <= 1) k_pcor_recheck<1><<<grid, 32 * kPcW, 0, st>>>(P, q, nq, rho);
    else if (P.l <= 2) k_pcor_recheck<2><<<grid, 32 * kPcW, 0, st>>>(P, q, nq, rho);
    else if (P.l <= 4) k_pcor_recheck<4><<<grid, 32 * kPcW, 0, st>>>(P, q, nq, rho);
    else if (P.l <= 8) k_pcor_recheck<8><<<grid, 32 * kPcW, 0, st>>>(P, q, nq, rho);
    else k_pcor_recheck<16><<<grid, 32 * kPcW, 0, st>>>(P, q, nq, rho);
    return cudaGetLastError();
}

cudaError_t launch_level(int fp32, const LevelParams& P, int num_sms, cudaStream_t st)
{
    if (fp32 && P.learned) return launch_level_b<float, true, true>(P, num_sms, st);
    return fp32 ? launch_level_b<float, true, false>(P, num_sms, st)
                : launch_level_b<double, false, false>(P, num_sms, st);
}

}  // namespace cupc
