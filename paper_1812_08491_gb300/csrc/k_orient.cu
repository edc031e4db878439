// k_orient.cu -- the second step of PC-stable (Sec. 2.4): v-structures read off
// the SepSets, then Meek's rules R1-R3, giving the CPDAG of Sec. 2.2.
//
// State: two p x W bitsets over the skeleton's edges.
//   head[x]  bit y: the edge x - y has an arrowhead at x
//   headT[x] bit y: the edge x - y has an arrowhead at y   (= head[y] bit x)
// so x -> y is (headT[x] bit y, head[x] bit y) = (1, 0), x - y is (0, 0) and
// an edge two v-structures disagree on has both (1, 1).
//
// Readings (the paper names the step only): every unshielded triple i - k - j
// with k outside SepSet(i, j) is a v-structure, all applied together (atomic
// ORs, so the order does not matter); the rules run in rounds that decide from
// the marks at the start of the round (propose kernel) and then apply every
// orientation together (apply kernel), until a round changes nothing; an edge
// proposed both ways in one round stays undirected; only undirected edges are
// oriented and only directed edges count as arrows in the premises:
//   R1  c -> a, a - b, c and b not adjacent                  =>  a -> b
//   R2  a -> c -> b, a - b                                   =>  a -> b
//   R3  a - c1 -> b, a - c2 -> b, c1, c2 not adjacent, a - b  =>  a -> b
#include "orient.cuh"

namespace cupc {
namespace {

__device__ __forceinline__ bool bit_of(const unsigned* B, int W, int x, int y)
{
    return (__ldg(B + (size_t)x * W + (y >> 5)) >> (y & 31)) & 1u;
}

// Reads of head/headT that a kernel of the same round may have written (the
// v-structure and apply kernels) go through L2.
__device__ __forceinline__ bool bit_cg(const unsigned* B, int W, int x, int y)
{
    return (__ldcg(B + (size_t)x * W + (y >> 5)) >> (y & 31)) & 1u;
}

__device__ __forceinline__ void set_bit(unsigned* B, int W, int x, int y)
{
    atomicOr(B + (size_t)x * W + (y >> 5), 1u << (y & 31));
}

// arrowhead at k on the edge i - k
__device__ __forceinline__ void arrow_at(unsigned* head, unsigned* headT, int W, int i, int k)
{
    set_bit(head, W, k, i);
    set_bit(headT, W, i, k);
}

// ---------------------------------------------------------------------------
// neighbour lists of the skeleton
// ---------------------------------------------------------------------------
__global__ void k_or_degree(const unsigned* __restrict__ bits, int p, int W, int* __restrict__ deg)
{
    const int lane = threadIdx.x & 31;
    const int v = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (v >= p) return;
    int c = 0;
    for (int w = lane; w < W; w += 32) c += __popc(bits[(size_t)v * W + w]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) deg[v] = c;
}

// One CTA: each thread scans a contiguous run of rows, then a block scan.
constexpr int SCAN_T = 1024;
__global__ void __launch_bounds__(SCAN_T) k_or_scan(const int* __restrict__ deg, int p, long long* __restrict__ off)
{
    __shared__ long long part[SCAN_T / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int per = (p + SCAN_T - 1) / SCAN_T;
    const int lo = min(p, t * per), hi = min(p, lo + per);
    long long s = 0;
    for (int i = lo; i < hi; ++i) s += deg[i];
    long long incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) part[w] = incl;
    __syncthreads();
    if (w == 0) {
        long long v = part[lane];
        long long iv = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long x = __shfl_up_sync(0xffffffffu, iv, o);
            if (lane >= o) iv += x;
        }
        part[lane] = iv - v;   // exclusive
    }
    __syncthreads();
    long long e = part[w] + incl - s;
    for (int i = lo; i < hi; ++i) {
        off[i] = e;
        e += deg[i];
    }
    if (t == SCAN_T - 1) off[p] = e;
}

// Warp per row: its neighbours in increasing order.
__global__ void k_or_fill(const unsigned* __restrict__ bits, int p, int W, const long long* __restrict__ off,
                          int* __restrict__ cols)
{
    const int lane = threadIdx.x & 31;
    const int v = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (v >= p) return;
    long long base = off[v];
    for (int w0 = 0; w0 < W; w0 += 32) {
        const int q = w0 + lane;
        unsigned word = q < W ? bits[(size_t)v * W + q] : 0u;
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
            cols[pos++] = (q << 5) + b;
        }
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// ---------------------------------------------------------------------------
// v-structures
// ---------------------------------------------------------------------------
// CTA per vertex k, threads over the pairs (x < y) of its neighbour list: the
// pair (i, j) is a v-structure at k when i and j are not adjacent and were
// removed at level 0 (S empty, so k is not in it).
__global__ void k_or_vstruct0(const unsigned* __restrict__ bits, const unsigned* __restrict__ bits0, int p, int W,
                              const long long* __restrict__ off, const int* __restrict__ cols, unsigned* head,
                              unsigned* headT)
{
    const int k = blockIdx.x;
    const long long o = off[k];
    const long long d = off[k + 1] - o;
    const long long npairs = d * (d - 1) / 2;
    for (long long q = threadIdx.x; q < npairs; q += blockDim.x) {
        // q = y (y - 1) / 2 + x, 0 <= x < y < d
        long long y = (long long)((1.0 + sqrt(1.0 + 8.0 * (double)q)) * 0.5);
        while (y * (y - 1) / 2 > q) --y;
        while ((y + 1) * y / 2 <= q) ++y;
        const long long x = q - y * (y - 1) / 2;
        const int i = cols[o + x], j = cols[o + y];
        if (!bit_of(bits, W, i, j) && !bit_of(bits0, W, i, j)) {
            arrow_at(head, headT, W, i, k);
            arrow_at(head, headT, W, j, k);
        }
    }
}

// Warp per SepSet record (i, j, l, S): every common neighbour k of i and j
// outside S is a v-structure i -> k <- j.
__global__ void k_or_vstructS(const unsigned* __restrict__ bits, int p, int W, const long long* __restrict__ off,
                              const int* __restrict__ cols, const int* __restrict__ rec, OrRecords R, unsigned* head,
                              unsigned* headT)
{
    const int lane = threadIdx.x & 31;
    const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= R.total) return;
    int q = 0;
    while (q + 1 < R.groups && r >= R.first[q + 1]) ++q;
    const int l = R.lev[q];
    const int* g = rec + R.start[q] + (r - R.first[q]) * (long long)(3 + l);
    const int i = g[0], j = g[1];
    int S[CUPC_MAX_LEVEL];
#pragma unroll
    for (int c = 0; c < CUPC_MAX_LEVEL; ++c) S[c] = c < l ? g[3 + c] : -1;
    const long long o = off[i], d = off[i + 1] - o;
    for (long long x = lane; x < d; x += 32) {
        const int k = cols[o + x];
        if (k == j || !bit_of(bits, W, j, k)) continue;
        bool in = false;
#pragma unroll
        for (int c = 0; c < CUPC_MAX_LEVEL; ++c) in |= (S[c] == k);
        if (!in) {
            arrow_at(head, headT, W, i, k);
            arrow_at(head, headT, W, j, k);
        }
    }
}

// ---------------------------------------------------------------------------
// Meek's rules, one round
// ---------------------------------------------------------------------------
constexpr int PROP_T = 256;
constexpr int TCAP = 128;   // R3 candidates kept per warp in shared memory

// x -> y: arrowhead at y, none at x
__device__ __forceinline__ bool dir_of(const unsigned* head, const unsigned* headT, int W, int x, int y)
{
    return bit_cg(headT, W, x, y) && !bit_cg(head, W, x, y);
}

// Warp per row a: for every undirected a - b, R1 and R2 over the neighbours c
// of a (lanes), then R3 over the pairs of candidates c (a - c -> b).
__global__ void __launch_bounds__(PROP_T) k_or_propose(const unsigned* __restrict__ bits, int p, int W,
                                                       const long long* __restrict__ off, const int* __restrict__ cols,
                                                       const unsigned* head, const unsigned* headT, unsigned* prop,
                                                       const unsigned long long* gate)
{
    __shared__ int cand[PROP_T / 32][TCAP];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int a = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (a >= p) return;
    if (gate && *(volatile const unsigned long long*)gate == 0ull) return;   // the rounds have ended
    const long long o = off[a], d = off[a + 1] - o;
    int* T = cand[wid];
    for (long long bi = 0; bi < d; ++bi) {
        const int b = cols[o + bi];
        if (bit_cg(head, W, a, b) || bit_cg(headT, W, a, b)) continue;   // not undirected
        bool hit = false;
        int nT = 0;
        bool overflow = false;
        for (long long c0 = 0; c0 < d && !hit; c0 += 32) {
            const long long x = c0 + lane;
            bool r12 = false, c3 = false;
            int c = -1;
            if (x < d && x != bi) {
                c = cols[o + x];
                const bool hc = bit_cg(head, W, a, c), tc = bit_cg(headT, W, a, c);
                if (hc && !tc && !bit_of(bits, W, c, b)) r12 = true;                  // R1: c -> a
                if (!r12 && tc && !hc && dir_of(head, headT, W, c, b)) r12 = true;    // R2: a -> c -> b
                if (!hc && !tc && dir_of(head, headT, W, c, b)) c3 = true;           // R3 candidate
            }
            hit = __any_sync(0xffffffffu, r12);
            const unsigned m = __ballot_sync(0xffffffffu, c3);
            if (c3) {
                const int at = nT + __popc(m & ((1u << lane) - 1u));
                if (at < TCAP) T[at] = c;
            }
            nT += __popc(m);
            if (nT > TCAP) overflow = true;
        }
        __syncwarp();
        if (!hit && nT >= 2) {
            if (!overflow) {
                // lanes over c1, a loop over c2 > c1 in the list
                bool h3 = false;
                for (int u = lane; u < nT && !h3; u += 32)
                    for (int v = u + 1; v < nT; ++v)
                        if (!bit_of(bits, W, T[u], T[v])) {
                            h3 = true;
                            break;
                        }
                hit = __any_sync(0xffffffffu, h3);
            } else {
                // more candidates than the list holds: both loops over the row
                bool h3 = false;
                for (long long x = lane; x < d && !h3; x += 32) {
                    if (x == bi) continue;
                    const int c1 = cols[o + x];
                    if (bit_cg(head, W, a, c1) || bit_cg(headT, W, a, c1) || !dir_of(head, headT, W, c1, b)) continue;
                    for (long long y = x + 1; y < d; ++y) {
                        if (y == bi) continue;
                        const int c2 = cols[o + y];
                        if (bit_cg(head, W, a, c2) || bit_cg(headT, W, a, c2) || !dir_of(head, headT, W, c2, b))
                            continue;
                        if (!bit_of(bits, W, c1, c2)) {
                            h3 = true;
                            break;
                        }
                    }
                }
                hit = __any_sync(0xffffffffu, h3);
            }
        }
        if (hit && lane == 0) set_bit(prop, W, a, b);
        __syncwarp();
    }
}

// Thread per word (a, w) of the proposals: a -> b is applied unless b -> a was
// proposed too.
__global__ void k_or_apply(const unsigned* __restrict__ prop, int p, int W, unsigned* head, unsigned* headT,
                           unsigned long long* flags, const unsigned long long* gate)
{
    if (gate && *(volatile const unsigned long long*)gate == 0ull) return;   // the rounds have ended
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long applied = 0, both = 0;
    if (t < (long long)p * W) {
        const int a = (int)(t / W), w = (int)(t % W);
        unsigned m = prop[t];
        while (m) {
            const int bb = __ffs(m) - 1;
            m &= m - 1;
            const int b = (w << 5) + bb;
            if (bit_of(prop, W, b, a)) {
                ++both;
            } else {
                arrow_at(head, headT, W, a, b);
                ++applied;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        applied += __shfl_xor_sync(0xffffffffu, applied, o);
        both += __shfl_xor_sync(0xffffffffu, both, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (applied) atomicAdd(flags + 0, applied);
        if (both) atomicAdd(flags + 1, both);
    }
}

// Warp per row a, lanes over columns b: the marks and the edge counts (a < b).
__global__ void k_or_marks(const unsigned* __restrict__ bits, const unsigned* __restrict__ headT, int p, int W,
                           unsigned char* __restrict__ marks, unsigned long long* flags)
{
    const int lane = threadIdx.x & 31;
    const int a = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (a >= p) return;
    unsigned long long nd = 0, nu = 0, nb = 0;
    for (int b = lane; b < p; b += 32) {
        unsigned char v = 0;
        if (bit_of(bits, W, a, b)) {
            const bool hb = bit_of(headT, W, a, b);   // arrowhead at b
            v = hb ? 1 : 2;
            if (a < b) {
                const bool ha = bit_of(headT, W, b, a);   // arrowhead at a
                if (ha && hb) ++nb;
                else if (ha || hb) ++nd;
                else ++nu;
            }
        }
        marks[(size_t)a * p + b] = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nd += __shfl_xor_sync(0xffffffffu, nd, o);
        nu += __shfl_xor_sync(0xffffffffu, nu, o);
        nb += __shfl_xor_sync(0xffffffffu, nb, o);
    }
    if (lane == 0) {
        if (nd) atomicAdd(flags + 2, nd);
        if (nu) atomicAdd(flags + 3, nu);
        if (nb) atomicAdd(flags + 4, nb);
    }
}

unsigned warp_blocks(long long rows, int threads) { return (unsigned)((rows * 32 + threads - 1) / threads); }

}  // namespace

cudaError_t launch_or_degree(const unsigned* bits, int p, int W, int* deg, cudaStream_t st)
{
    k_or_degree<<<warp_blocks(p, 256), 256, 0, st>>>(bits, p, W, deg);
    return cudaGetLastError();
}

cudaError_t launch_or_scan(const int* deg, int p, long long* off, cudaStream_t st)
{
    k_or_scan<<<1, SCAN_T, 0, st>>>(deg, p, off);
    return cudaGetLastError();
}

cudaError_t launch_or_fill(const unsigned* bits, int p, int W, const long long* off, int* cols, cudaStream_t st)
{
    k_or_fill<<<warp_blocks(p, 256), 256, 0, st>>>(bits, p, W, off, cols);
    return cudaGetLastError();
}

cudaError_t launch_or_vstruct0(const unsigned* bits, const unsigned* bits0, int p, int W, const long long* off,
                               const int* cols, unsigned* head, unsigned* headT, cudaStream_t st)
{
    k_or_vstruct0<<<p, 256, 0, st>>>(bits, bits0, p, W, off, cols, head, headT);
    return cudaGetLastError();
}

cudaError_t launch_or_vstructS(const unsigned* bits, int p, int W, const long long* off, const int* cols,
                               const int* rec, const OrRecords& R, unsigned* head, unsigned* headT, cudaStream_t st)
{
    if (R.total <= 0) return cudaSuccess;
    k_or_vstructS<<<warp_blocks(R.total, 256), 256, 0, st>>>(bits, p, W, off, cols, rec, R, head, headT);
    return cudaGetLastError();
}

cudaError_t launch_or_propose(const unsigned* bits, int p, int W, const long long* off, const int* cols,
                              const unsigned* head, const unsigned* headT, unsigned* prop,
                              const unsigned long long* gate, cudaStream_t st)
{
    k_or_propose<<<warp_blocks(p, PROP_T), PROP_T, 0, st>>>(bits, p, W, off, cols, head, headT, prop, gate);
    return cudaGetLastError();
}

cudaError_t launch_or_apply(const unsigned* prop, int p, int W, unsigned* head, unsigned* headT,
                            unsigned long long* flags, const unsigned long long* gate, cudaStream_t st)
{
    const long long words = (long long)p * W;
    k_or_apply<<<(unsigned)((words + 255) / 256), 256, 0, st>>>(prop, p, W, head, headT, flags, gate);
    return cudaGetLastError();
}

cudaError_t launch_or_marks(const unsigned* bits, const unsigned* headT, int p, int W, unsigned char* marks,
                            unsigned long long* flags, cudaStream_t st)
{
    k_or_marks<<<warp_blocks(p, 256), 256, 0, st>>>(bits, headT, p, W, marks, flags);
    return cudaGetLastError();
}

}  // namespace cupc
