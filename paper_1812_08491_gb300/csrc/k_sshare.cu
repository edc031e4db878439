// k_sshare.cu -- global sharing of conditioning sets at one level (Sec. 5.5,
// Fig. 9): every l-subset S of adj(i) in each row i of A'_G that runs tests at
// the level is counted once per row, in a device hash table keyed by S, then
// the per-set row counts are binned. This is the "global search" the paper
// weighs against row-local sharing; its device time is the search's cost.
#include <algorithm>

#include "kernels.cuh"

namespace cupc {
namespace {

constexpr unsigned long long kEmpty = ~0ull;

// S packed into 64 bits: members increasing, `bits` bits each (16 for l <= 4,
// 32 for l <= 2).
__device__ __forceinline__ unsigned long long mix64(unsigned long long x)
{
    // splitmix64 finaliser (Steele, Lea, Flood 2014)
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

template <int LB>
__global__ void k_sshare_insert(const long long* __restrict__ off, const int* __restrict__ cols,
                                const long long* __restrict__ pre, int nrows, int l, int bits, Binom B,
                                unsigned long long total, unsigned long long* __restrict__ keys,
                                unsigned* __restrict__ cnt, unsigned long long mask, int* err)
{
    for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (unsigned long long)gridDim.x * blockDim.x) {
        // row of pair t: the last row whose first pair is <= t
        int lo = 0, hi = nrows - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((unsigned long long)pre[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const long long o = off[lo];
        const int d = (int)(off[lo + 1] - o);
        int Pos[LB];
        unrank_lex<LB>(t - (unsigned long long)pre[lo], d, l, B, Pos);
        unsigned long long key = 0;
#pragma unroll
        for (int c = 0; c < LB; ++c)
            if (c < l) key = (key << bits) | (unsigned long long)cols[o + Pos[c]];
        unsigned long long h = mix64(key) & mask;
        for (unsigned long long probe = 0;; ++probe) {
            if (probe > mask) {                      // table full: cannot happen at its size
                atomicOr(err, 1);
                break;
            }
            const unsigned long long prev = atomicCAS(keys + h, kEmpty, key);
            if (prev == kEmpty || prev == key) {
                atomicAdd(cnt + h, 1u);
                break;
            }
            h = (h + 1) & mask;
        }
    }
}

// out[0..nbins): sets per bin; out[nbins]: distinct sets, [nbins + 1]: sets in
// two rows or more, [nbins + 2]: largest row count.
__global__ void k_sshare_hist(const unsigned long long* __restrict__ keys, const unsigned* __restrict__ cnt,
                              unsigned long long slots, const long long* __restrict__ bins, int nbins,
                              unsigned long long* __restrict__ out)
{
    for (unsigned long long h = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; h < slots;
         h += (unsigned long long)gridDim.x * blockDim.x) {
        if (keys[h] == kEmpty) continue;
        const long long c = cnt[h];
        int k = 0;
        while (k + 1 < nbins && bins[k + 1] <= c) ++k;
        if (bins[k] <= c) atomicAdd(out + k, 1ull);
        atomicAdd(out + nbins, 1ull);
        if (c >= 2) atomicAdd(out + nbins + 1, 1ull);
        atomicMax(out + nbins + 2, (unsigned long long)c);
    }
}

}  // namespace

cudaError_t launch_sshare(const long long* off, const int* cols, const long long* pre, int nrows, int l, int bits,
                          const Binom& B, unsigned long long total, unsigned long long* keys, unsigned* cnt,
                          unsigned long long slots, const long long* bins, int nbins, unsigned long long* out,
                          int* err, int num_sms, cudaStream_t st)
{
    const int block = 256;
    const unsigned grid = (unsigned)std::max(1, num_sms * 8);
    if (total) {
        if (l <= 2)
            k_sshare_insert<2><<<grid, block, 0, st>>>(off, cols, pre, nrows, l, bits, B, total, keys, cnt,
                                                       slots - 1, err);
        else
            k_sshare_insert<4><<<grid, block, 0, st>>>(off, cols, pre, nrows, l, bits, B, total, keys, cnt,
                                                       slots - 1, err);
    }
    k_sshare_hist<<<grid, block, 0, st>>>(keys, cnt, slots, bins, nbins, out);
    return cudaGetLastError();
}

}  // namespace cupc
