// k_records.cu -- the host-facing lists of one skeleton, built on the device so
// that the host downloads them ready to use: the SepSet records of the
// removals at levels >= 1 (Algorithm 1's SepSet output) in (i, j) order, and
// the skeleton's edge list (its output graph G) in (i, j) order.
//
// Records. A call appends its level-l records (i, j, l, S_1 .. S_l), i < j,
// level by level, in the order the removals happened. The pairs removed at
// levels >= 1 are exactly the set bits of R = A0 & ~A in columns j > i, with
// A0 the adjacency after level 0 and A the final one, so a record's place in
// (i, j) order is the number of bits of R before (i, j) in row-major order:
// per-row counts and per-word prefix counts of R, an exclusive scan over the
// rows, and per record its rank. The records' lengths (3 + l ints) are summed
// per row, scanned over the rows, and a warp per row adds its records' lengths
// in rank order and copies each record to its offset. Every step checks what
// it relies on (a record's level and pair, its bit in R, one record per rank)
// and raises an error flag instead of writing out of place; the host compares
// the totals and falls back to its own sort when they disagree. The first
// kernel also clears the scratch the later ones accumulate into, and the
// totals land in a status block the host downloads with the list.
//
// Batches: the rows are those of the block-diagonal union graph (problem
// vprob[g] holds global row g; its bitset block stores local columns), the
// sort runs over the global (i, j) order, which is problem by problem, the
// records are written with local ids, and the per-problem, per-level record
// counts are gathered on the way.
#include "kernels.cuh"
#include "records.cuh"

namespace cupc {
namespace {

constexpr int RT = 256;   // threads per block of the per-row and per-record kernels

// Row g of one problem or of a batch's union: its first word, local index,
// words, columns and the id offset of its problem.
struct Row {
    long long base, i;
    int W, p, off;
};

__device__ __forceinline__ Row row_at(const RowView& V, long long g)
{
    Row r;
    if (V.probs) {
        const ProbDesc& D = V.probs[V.vprob[g]];
        r.off = D.off;
        r.i = g - D.off;
        r.W = D.whi - D.wlo;
        r.p = D.p;
    } else {
        r.off = 0;
        r.i = g;
        r.W = V.W;
        r.p = V.p;
    }
    r.base = (V.probs ? V.probs[V.vprob[g]].bw : 0) + r.i * r.W;
    return r;
}

// Word w of row R of A (a0 == nullptr) or of A0 & ~A, restricted to columns
// i < j < p.
__device__ __forceinline__ unsigned upper_word(const unsigned* __restrict__ a, const unsigned* __restrict__ a0,
                                               const Row& R, int w)
{
    const long long at = R.base + w;
    unsigned m = a0 ? (a0[at] & ~a[at]) : a[at];
    const int w0 = (int)((R.i + 1) >> 5);
    if (w < w0) return 0u;
    if (w == w0) m &= ~0u << ((R.i + 1) & 31);
    const long long c0 = (long long)w * 32;
    if (c0 + 32 > R.p) m &= (c0 >= R.p) ? 0u : ((1u << (R.p - c0)) - 1u);
    return m;
}

// A warp per row: cnt[g] = bits of the row's upper part; wpre[base + w] (when
// given) = those bits in the row's words before w. With the records' scratch
// given: rowints and status[0] cleared, slot[0 .. nslot) set to -1.
__global__ void __launch_bounds__(RT) k_row_bits(const unsigned* __restrict__ a, const unsigned* __restrict__ a0,
                                                 RowView V, long long nrows, unsigned* __restrict__ wpre,
                                                 long long* __restrict__ cnt, unsigned long long* __restrict__ rowints,
                                                 long long* __restrict__ slot, long long nslot,
                                                 long long* __restrict__ status)
{
    const int lane = threadIdx.x & 31;
    const long long t = (long long)blockIdx.x * RT + threadIdx.x;
    if (slot)
        for (long long k = t; k < nslot; k += (long long)gridDim.x * RT) slot[k] = -1;
    if (status && t == 0) status[0] = 0;
    const long long g = t >> 5;
    if (g >= nrows) return;
    if (rowints && lane == 0) rowints[g] = 0;
    const Row R = row_at(V, g);
    unsigned carry = 0;
    for (int b = 0; b < R.W; b += 32) {
        const int w = b + lane;
        const unsigned m = (w < R.W) ? upper_word(a, a0, R, w) : 0u;
        const unsigned c = __popc(m);
        unsigned inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned x = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += x;
        }
        if (wpre && w < R.W) wpre[R.base + w] = carry + inc - c;
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) cnt[g] = (long long)carry;
}

// Exclusive prefix sums: out[k] = v[0] + ... + v[k-1] for k <= n (out[n] the
// total). One block of 1024 threads walks v in chunks.
__global__ void __launch_bounds__(1024) k_scan_ll(const long long* __restrict__ v, long long n,
                                                  long long* __restrict__ out)
{
    __shared__ long long ws[32];
    __shared__ long long base;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) base = 0;
    __syncthreads();
    for (long long c0 = 0; c0 < n; c0 += 1024) {
        const long long k = c0 + t;
        const long long x = (k < n) ? v[k] : 0;
        long long inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) ws[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            long long s = ws[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            ws[lane] = s;
        }
        __syncthreads();
        const long long b = base;
        if (k < n) out[k] = b + (warp ? ws[warp - 1] : 0) + inc - x;
        __syncthreads();
        if (t == 0) base = b + ws[31];
        __syncthreads();
    }
    if (t == 0) out[n] = base;
}

// A thread per record: its rank in (i, j) order (slot[rank] = its int offset)
// and its length added to its row's; batches also count it for its problem
// and level (plc[problem * plc_stride + l]).
__global__ void __launch_bounds__(RT) k_rec_rank(const int* __restrict__ rec, RecGroups G,
                                                 const unsigned* __restrict__ a, const unsigned* __restrict__ a0,
                                                 RowView V, long long nrows, const unsigned* __restrict__ wpre,
                                                 const long long* __restrict__ rowstart, long long* __restrict__ slot,
                                                 unsigned long long* __restrict__ rowints,
                                                 unsigned long long* __restrict__ err,
                                                 unsigned long long* __restrict__ plc, int plc_stride)
{
    const long long r = (long long)blockIdx.x * RT + threadIdx.x;
    if (r >= G.total) return;
    int q = 0;
    while (q + 1 < G.groups && r >= G.first[q + 1]) ++q;
    const int l = G.lev[q];
    const long long src = G.start[q] + (r - G.first[q]) * (long long)(3 + l);
    const int gi = rec[src], gj = rec[src + 1];
    if (rec[src + 2] != l || gi < 0 || gi >= nrows || gj < 0 || gj >= nrows) {
        atomicOr(err, 1ull);
        return;
    }
    const Row R = row_at(V, gi);
    const long long j = (long long)gj - R.off;
    if (R.i >= R.p || j <= R.i || j >= R.p) {
        atomicOr(err, 1ull);
        return;
    }
    const int w = (int)(j >> 5);
    const unsigned m = upper_word(a, a0, R, w);
    if (((m >> (j & 31)) & 1u) == 0u) {
        atomicOr(err, 2ull);                         // not a pair removed at a level >= 1
        return;
    }
    const long long pos = rowstart[gi] + wpre[R.base + w] + __popc(m & ((1u << (j & 31)) - 1u));
    if (pos >= G.total) {
        atomicOr(err, 4ull);                         // more removed pairs than records
        return;
    }
    if (atomicCAS((unsigned long long*)(slot + pos), ~0ull, (unsigned long long)src) != ~0ull) {
        atomicOr(err, 8ull);                         // two records of one pair
        return;
    }
    atomicAdd(rowints + gi, (unsigned long long)(3 + l));
    if (plc) atomicAdd(plc + (long long)V.vprob[gi] * plc_stride + l, 1ull);
}

// A warp per row: the row's records in rank order, each copied (ids made
// local to its problem) to the row's int offset plus the lengths of the
// records before it; status[1], status[2] = the removed pairs and the ints
// placed.
__global__ void __launch_bounds__(RT) k_rec_place(const int* __restrict__ rec, RowView V, long long nrows,
                                                  const long long* __restrict__ rowstart,
                                                  const long long* __restrict__ rowoff,
                                                  const long long* __restrict__ slot, long long total,
                                                  int* __restrict__ out, long long* __restrict__ status)
{
    const int lane = threadIdx.x & 31;
    const long long t = (long long)blockIdx.x * RT + threadIdx.x;
    if (t == 0) {
        status[1] = rowstart[nrows];
        status[2] = rowoff[nrows];
    }
    const long long g = t >> 5;
    if (g >= nrows) return;
    const int off = V.probs ? V.probs[V.vprob[g]].off : 0;
    const long long q1 = min(rowstart[g + 1], total);
    long long at = rowoff[g];
    for (long long qb = rowstart[g]; qb < q1; qb += 32) {
        const long long q = qb + lane;
        long long src = -1;
        int len = 0;
        if (q < q1) {
            src = slot[q];
            if (src >= 0) len = 3 + rec[src + 2];
        }
        int inc = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += x;
        }
        const long long o = at + inc - len;
        for (int c = 0; c < len; ++c) out[o + c] = (c == 2) ? rec[src + c] : rec[src + c] - off;
        at += __shfl_sync(0xffffffffu, inc, 31);
    }
}

// A warp per row of one problem: the row's edges (i, j), j > i, in column
// order at pair off[i] + (edges of the row before j); pairs at or past cap are
// not written; status[0] = the number of edges.
__global__ void __launch_bounds__(RT) k_edge_fill(const unsigned* __restrict__ a, RowView V,
                                                  const long long* __restrict__ off, long long cap,
                                                  int* __restrict__ out, long long* __restrict__ status)
{
    const int lane = threadIdx.x & 31;
    const long long t = (long long)blockIdx.x * RT + threadIdx.x;
    if (t == 0) status[0] = off[V.p];
    const long long g = t >> 5;
    if (g >= V.p) return;
    const Row R = row_at(V, g);
    long long carry = off[g];
    for (int b = 0; b < R.W; b += 32) {
        const int w = b + lane;
        unsigned m = (w < R.W) ? upper_word(a, nullptr, R, w) : 0u;
        const int c = __popc(m);
        int inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += x;
        }
        long long e = carry + inc - c;
        while (m) {
            const int bit = __ffs(m) - 1;
            m &= m - 1;
            if (e < cap) {
                out[2 * e] = (int)g;
                out[2 * e + 1] = w * 32 + bit;
            }
            ++e;
        }
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
}

inline unsigned row_blocks(long long rows) { return (unsigned)((rows * 32 + RT - 1) / RT); }

}  // namespace

cudaError_t launch_records_sort(const int* rec, const RecGroups& G, const unsigned* bits, const unsigned* bits0,
                                const RowView& V, long long nrows, unsigned* wpre, long long* rowcnt,
                                long long* rowstart, unsigned long long* rowints, long long* rowoff, long long* slot,
                                int* out, long long* status, unsigned long long* plc, int plc_stride, cudaStream_t st)
{
    if (nrows <= 0) return cudaSuccess;
    k_row_bits<<<row_blocks(nrows), RT, 0, st>>>(bits, bits0, V, nrows, wpre, rowcnt, rowints, slot, G.total, status);
    k_scan_ll<<<1, 1024, 0, st>>>(rowcnt, nrows, rowstart);
    if (G.total > 0)
        k_rec_rank<<<(unsigned)((G.total + RT - 1) / RT), RT, 0, st>>>(
            rec, G, bits, bits0, V, nrows, wpre, rowstart, slot, rowints, (unsigned long long*)status, plc, plc_stride);
    k_scan_ll<<<1, 1024, 0, st>>>((const long long*)rowints, nrows, rowoff);
    k_rec_place<<<row_blocks(nrows), RT, 0, st>>>(rec, V, nrows, rowstart, rowoff, slot, G.total, out, status);
    return cudaGetLastError();
}

cudaError_t launch_edge_list(const unsigned* bits, int p, int W, long long* rowcnt, long long* off, long long cap,
                             int* out, long long* status, cudaStream_t st)
{
    if (p <= 0) return cudaSuccess;
    const RowView V{nullptr, nullptr, W, p};
    k_row_bits<<<row_blocks(p), RT, 0, st>>>(bits, nullptr, V, p, nullptr, rowcnt, nullptr, nullptr, 0, nullptr);
    k_scan_ll<<<1, 1024, 0, st>>>(rowcnt, p, off);
    k_edge_fill<<<row_blocks(p), RT, 0, st>>>(bits, V, off, cap, out, status);
    return cudaGetLastError();
}

}  // namespace cupc
