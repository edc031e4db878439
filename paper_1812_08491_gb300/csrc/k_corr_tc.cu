// k_corr_tc.cu -- the correlation product C = Z Z^T / n on the 5th-generation
// tensor cores (tcgen05), split precision.
//
// Each standardised value z (FP64) is split into two bf16 numbers,
// hi = bf16(z) and lo = bf16(z - hi), so z = hi + lo to about 2^-18 relative.
// C_ij is accumulated in FP32 (in TMEM) over three bf16 products,
//     sum_s hi_i hi_j + hi_i lo_j + lo_i hi_j,
// i.e. one GEMM over K = 3 n' whose A operand walks (hi, hi, lo) and whose B
// operand walks (hi, lo, hi); the dropped lo*lo term is below 2^-18.
//
// Kernel shape: persistent CTAs, one per SM, each walking a list of work units
// (a 128 x 256 output tile of the upper triangle and a range of K steps).
// Warp 0 issues TMA loads (128B-swizzled, K-major) into a 4-stage ring of
// 16 KiB A and 32 KiB B slabs, one thread of warp 1 issues tcgen05.mma
// (M=128, N=256, K=16, bf16 -> f32) and returns stages with tcgen05.commit.
// The N=256 shape halves the shared-memory operand traffic per flop of the
// square 128 x 128 tile, whose operand reads plus TMA writes exceed what the
// SM's shared memory delivers. The tensor core's FP32 accumulation error grows
// with the number of products summed into one accumulator, so the MMA thread
// restarts accumulation every GROUP K slabs, alternating between two TMEM
// accumulators of 256 columns (all 512 columns of the SM); warps 2-17 drain each
// finished group (tcgen05.ld 32x32b; four warps per lane quadrant, one per
// 64-column quarter) into FP32 registers with round-to-nearest adds while the
// next group -- of the same unit or of the next one -- runs. A unit that covers
// the whole K range writes its tile of C directly: times 1/n, the i <= j
// entries row by row and their mirror images (j, i) column by column, so C is
// exactly symmetric; a unit that covers a K slice stores its partial tile, and
// a second kernel adds the slices in a fixed order as compensated FP32 pairs,
// scales by 1/n and writes both triangles the same way.
//
// Every mbarrier wait is bounded in time; on expiry the thread raises an error
// flag, the others stop at their next wait, TMEM is freed and the kernel ends.
#include <algorithm>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "kernels.cuh"

namespace cupc {
namespace {

constexpr int BM = 128, BN = 256, BK = 64;      // output tile and K slab (64 bf16 = 128 bytes)
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;            // 16 KiB A slab per stage
constexpr int B_BYTES = BN * BK * 2;            // 32 KiB B slab per stage
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int EPI_WARPS = 16;                   // four per TMEM lane quadrant
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int SEG = BN / 4;                     // columns drained by one epilogue thread
constexpr uint32_t TMEM_COLS = 512;             // two FP32 accumulators of 128 lanes x 256 columns
constexpr int GROUP = 8;                        // K slabs (512 products) per accumulator group
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 256 + 1024;
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s per wait


// Instruction descriptor of tcgen05.mma kind::f16: D f32 (bits 4-5 = 1), A and
// B bf16 (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase of parity `parity`; false if the time budget ran out or
// another thread of the kernel raised the error flag (both looked at every
// eighth unsuccessful try, so the spin stays off the memory system).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 7u) == 0) {
            if (*(volatile int*)err) return false;
            if (gtimer() - t0 > kWaitNs) {
                atomicOr(err, 4);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor for a K-major tile written by TMA with the
// 128-byte swizzle: start address >> 4 (bits 0-13), leading byte offset 16
// (unused for swizzled K-major), stride byte offset 1024 (8 rows of 128 bytes,
// bits 32-45), descriptor version 1 (bits 46-47), swizzle mode 2 = 128B (bits
// 61-63). Tile bases are 1024-byte aligned, so the base offset is 0.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}


// Upper-triangle tiles of 128 rows x 256 columns: row block bi meets column
// block bj when bi <= 2 bj + 1. Column blocks bj < b0 = nr / 2 hold 2 bj + 2
// tiles (bi = 0 .. 2 bj + 1), the later ones all nr row blocks; tiles are
// numbered column block by column block, so t < b0 (b0 + 1) lies in the first
// part. Count: b0 (b0 + 1) + (nc - b0) nr.
__device__ __forceinline__ void tile_rc(int t, int nr, int b0, int& bi, int& bj)
{
    const int first = b0 * (b0 + 1);
    if (t < first) {
        int j = (int)((sqrtf(4.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while ((j + 1) * (j + 2) <= t) ++j;
        while (j * (j + 1) > t) --j;
        bj = j;
        bi = t - j * (j + 1);
    } else {
        const int r = t - first;
        bj = b0 + r / nr;
        bi = r % nr;
    }
}

inline int tile_count(int nr, int nc) { const int b0 = nr / 2; return b0 * (b0 + 1) + (nc - b0) * nr; }

// Work unit of a batch (a list of independent products in one launch): the
// operand rows of the A and B tiles, the K steps [g0, g1) of its 3 kt, the
// workspace slot of its partial tile, or slot -1 and its problem when it
// covers the whole K range and writes C itself.
struct __align__(16) CorrWork {
    int ra, rb, g0, g1, kt, slot, prob, pad0;
};

// Split output tile of a batch: problem, tile coordinates, its partials' slots.
struct __align__(16) CorrTile {
    int prob, bi, bj, slot0, nsplit, pad0, pad1, pad2;
};

struct CorrArgs {
    int kt, kps, nsplit, tiles, nr, b0, n_units, p;  // single product: its plan
    float inv_n;
    float* ws;
    float* C;
    int* err;
    const CorrWork* work;                            // batch: the unit table
    const ProbDesc* probs;
};

// One unit as every role of the CTA sees it.
struct Unit {
    int ra, rb, g0, g1, kt;
    long long slot;  // partial tile slot, or -1: write C
    int p, row0, col0;
    float inv_n;
    float* C;
};

__device__ __forceinline__ Unit unit_of(const CorrArgs& a, int u)
{
    Unit U;
    if (a.work) {
        const CorrWork w = a.work[u];
        U.ra = w.ra;
        U.rb = w.rb;
        U.g0 = w.g0;
        U.g1 = w.g1;
        U.kt = w.kt;
        U.slot = w.slot;
        const ProbDesc& D = a.probs[w.prob];
        U.p = D.p;
        U.row0 = w.ra - D.off;
        U.col0 = w.rb - D.off;
        U.inv_n = (float)D.inv_n;
        U.C = a.C + D.c_off;
    } else {
        const int t = u % a.tiles, split = u / a.tiles;
        int bi, bj;
        tile_rc(t, a.nr, a.b0, bi, bj);
        U.ra = bi * BM;
        U.rb = bj * BN;
        U.g0 = split * a.kps;
        U.g1 = min(U.g0 + a.kps, 3 * a.kt);
        U.kt = a.kt;
        U.slot = a.nsplit == 1 ? -1 : (long long)split * a.tiles + t;
        U.p = a.p;
        U.row0 = U.ra;
        U.col0 = U.rb;
        U.inv_n = a.inv_n;
        U.C = a.C;
    }
    return U;
}

// Final values of one thread's row segment (row gi, 64 columns from cj of the
// tile) into C: the i <= j part along the row (unit diagonal), the i < j
// part mirrored to (j, i), where the lanes' consecutive rows make each
// column's 32 writes one segment.
__device__ __forceinline__ void store_c(float (&R)[SEG], const Unit& U, int row, int h)
{
    const int gi = U.row0 + row, cj = U.col0 + h * SEG, p = U.p;
    if (gi >= p) return;
    float* C = U.C;
    float* crow = C + (size_t)gi * p;
    const bool vec = ((p & 3) == 0) && (((uintptr_t)C & 15) == 0);
#pragma unroll
    for (int c = 0; c < SEG; ++c) R[c] *= U.inv_n;
#pragma unroll
    for (int c4 = 0; c4 < SEG / 4; ++c4) {
        const int gj = cj + 4 * c4;
        if (vec && gj > gi && gj + 3 < p) {
            *(float4*)(crow + gj) = make_float4(R[4 * c4], R[4 * c4 + 1], R[4 * c4 + 2], R[4 * c4 + 3]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = gj + e;
                if (j >= gi && j < p) crow[j] = (j == gi) ? 1.0f : R[4 * c4 + e];
            }
        }
    }
    // columns cj + c with gi < cj + c < p: c from c0 to c1 - 1
    const int c0 = max(0, gi + 1 - cj), c1 = min(SEG, p - cj);
    float* mp = C + (size_t)cj * p + gi;
#pragma unroll
    for (int c = 0; c < SEG; ++c) {
        if (c >= c0 && c < c1) *mp = R[c];
        mp += p;
    }
}

__global__ void __launch_bounds__(THREADS, 1)
k_corr_tc(const __grid_constant__ CUtensorMap tmAH, const __grid_constant__ CUtensorMap tmAL,
          const __grid_constant__ CUtensorMap tmBH, const __grid_constant__ CUtensorMap tmBL, const CorrArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = smem;                         // STAGES x 16 KiB
    unsigned char* sB = smem + STAGES * A_BYTES;      // STAGES x 32 KiB
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* acc_full = empty + STAGES;   // [2]: group accumulated (tcgen05.commit)
    uint64_t* acc_empty = acc_full + 2;    // [2]: group drained by the epilogue warps
    uint32_t* tmem_slot = (uint32_t*)(acc_empty + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], EPI_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // every role walks the same units (u = blockIdx.x, + gridDim.x, ...); ring
    // stages and accumulator buffers continue from one unit to the next
    if (warp == 0 && lane == 0) {
        // TMA producer
        int gs = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < a.n_units && ok; u += gridDim.x) {
            const Unit U = unit_of(a, u);
            for (int g = U.g0; g < U.g1; ++g, ++gs) {
                const int s = gs % STAGES;
                const uint32_t ph = (uint32_t)(gs / STAGES) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u, a.err)) {
                    ok = false;
                    break;
                }
                const int seg = g / U.kt, kk = g - seg * U.kt;
                mbar_expect_tx(&full[s], STAGE_BYTES);
                tma_load_2d(sA + s * A_BYTES, seg == 2 ? &tmAL : &tmAH, kk * BK, U.ra, &full[s]);
                tma_load_2d(sB + s * B_BYTES, seg == 1 ? &tmBL : &tmBH, kk * BK, U.rb, &full[s]);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: group gg accumulates into TMEM columns [256 (gg & 1), +256)
        int gs = 0, gg = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < a.n_units && ok; u += gridDim.x) {
            const Unit U = unit_of(a, u);
            const int nsteps = U.g1 - U.g0;
            for (int k = 0; k < nsteps; ++k, ++gs) {
                const int b = gg & 1;
                const bool first = (k % GROUP) == 0;
                if (first && gg >= 2) {
                    // the previous use of buffer b must have been drained
                    if (!mbar_wait(&acc_empty[b], (uint32_t)((gg >> 1) - 1) & 1u, a.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                }
                const int s = gs % STAGES;
                const uint32_t ph = (uint32_t)(gs / STAGES) & 1u;
                if (!mbar_wait(&full[s], ph, a.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint64_t ad = sdesc_sw128(smem_u32(sA + s * A_BYTES));
                const uint64_t bd = sdesc_sw128(smem_u32(sB + s * B_BYTES));
                const uint32_t dacc = tmem + (uint32_t)(b * BN);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)  // K = 16 per instruction: +32 bytes in the swizzled row
                    mma_bf16(dacc, ad + 2 * kk, bd + 2 * kk, (first && kk == 0) ? 0u : 1u);
                mma_commit(&empty[s]);
                if ((k % GROUP) == GROUP - 1 || k == nsteps - 1) {
                    mma_commit(&acc_full[b]);
                    ++gg;
                }
            }
        }
    } else if (warp >= 2) {
        // epilogue: warp w may read TMEM lanes 32 (w % 4) .. +31 (rows of the
        // tile); warps 2-5 take columns 0-63, warps 6-9 64-127, and so on
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int row = q * 32 + lane;
        int gg = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < a.n_units && ok; u += gridDim.x) {
            // (the unit is read again for the store: nothing of it stays live
            // across the accumulation)
            const int ngroups = [&] {
                const Unit U = unit_of(a, u);
                return (U.g1 - U.g0 + GROUP - 1) / GROUP;
            }();
            float R[SEG];
#pragma unroll
            for (int c = 0; c < SEG; ++c) R[c] = 0.f;
            for (int g = 0; g < ngroups; ++g, ++gg) {
                const int b = gg & 1;
                ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[b], (uint32_t)(gg >> 1) & 1u, a.err));
                if (!ok) break;
                tc_fence_after();
                const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + h * SEG);
#pragma unroll
                for (int c = 0; c < SEG; c += 16) {
                    uint32_t r[16];
                    tmem_ld16(base + (uint32_t)c, r);
#pragma unroll
                    for (int e = 0; e < 16; ++e) R[c + e] += __uint_as_float(r[e]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[b]);
            }
            if (!ok) break;
            const Unit U = unit_of(a, u);
            if (U.slot >= 0) {
                float4* out = (float4*)(a.ws + ((size_t)U.slot * BM + row) * BN + h * SEG);
#pragma unroll
                for (int c = 0; c < SEG / 4; ++c)
                    out[c] = make_float4(R[4 * c], R[4 * c + 1], R[4 * c + 2], R[4 * c + 3]);
            } else {
                store_c(R, U, row, h);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Sum of the K-slice partials in slice order, times 1/n; the i < j value is
// written to (i, j) and, through a shared-memory transpose, to (j, i); the
// diagonal is 1. The slices are added with Knuth's two-sum, the rounding error
// of each addition collected in a second FP32 word (the compensated sum Sum2 of
// Ogita, Rump and Oishi, 2005): the result is within 2^-24 |sum| +
// (k 2^-24)^2 sum|slice| of the exact sum of k slices. The second term is what
// separates it from an FP64 sum (within k 2^-53 sum|slice|); it stays below the
// output's own FP32 rounding while k^2 sum|slice| < 2^24 |sum|. GB300's FP64
// pipe is narrow, so the pair is used instead. Block (tile, 8-row band): 256
// threads, warp = row of the band; a lane
// owns columns 4 lane .. 4 lane + 3 and 128 + 4 lane .. 128 + 4 lane + 3 and
// reads them as two float4 per slice, eight slices' loads in flight at a time.
constexpr int RROWS = 8;
constexpr int RSL = 8;                               // slices loaded per batch
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float v)
{
    const float t = s + v, bb = t - s;
    e += (s - (t - bb)) + (v - bb);
    s = t;
}

__device__ __forceinline__ void reduce_band(const float* __restrict__ ws, long long slot0, long long stride,
                                            int nsplit, int bi, int bj, int p, float inv_n, float* __restrict__ C,
                                            float (*sm)[BN + 1])
{
    static_assert(BN == 256, "a lane covers two float4 groups of a 256-column row");
    const int r0 = blockIdx.y * RROWS;
    const int rr = threadIdx.x >> 5;            // row of the band (8 warps)
    const int lane = threadIdx.x & 31;
    const int r = r0 + rr, gi = bi * BM + r;
    const float4* src = (const float4*)(ws + ((size_t)slot0 * BM + r) * BN);
    const size_t step = (size_t)stride * BM * BN / 4;
    float hs[8], he[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) hs[u] = he[u] = 0.f;
    // the whole band row is summed (entries past p or below the diagonal are
    // finite partials of the tile and are discarded below)
    for (int k0 = 0; k0 < nsplit; k0 += RSL) {
        float4 a[RSL][2];
#pragma unroll
        for (int q = 0; q < RSL; ++q) {
            if (k0 + q < nsplit) {
                a[q][0] = __ldcs(src + (size_t)(k0 + q) * step + lane);
                a[q][1] = __ldcs(src + (size_t)(k0 + q) * step + 32 + lane);
            }
        }
#pragma unroll
        for (int q = 0; q < RSL; ++q) {
            if (k0 + q < nsplit) {
                two_sum_acc(hs[0], he[0], a[q][0].x);
                two_sum_acc(hs[1], he[1], a[q][0].y);
                two_sum_acc(hs[2], he[2], a[q][0].z);
                two_sum_acc(hs[3], he[3], a[q][0].w);
                two_sum_acc(hs[4], he[4], a[q][1].x);
                two_sum_acc(hs[5], he[5], a[q][1].y);
                two_sum_acc(hs[6], he[6], a[q][1].z);
                two_sum_acc(hs[7], he[7], a[q][1].w);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int c = (u < 4 ? 0 : 128) + 4 * lane + (u & 3);
        const int gj = bj * BN + c;
        const bool valid = gi < p && gj < p && gj >= gi;
        float v = 0.f;
        if (valid) {
            v = (gi == gj) ? 1.0f : fmaf(hs[u], inv_n, he[u] * inv_n);
            C[(size_t)gi * p + gj] = v;
        }
        sm[rr][c] = (valid && gj != gi) ? v : __int_as_float(0x7fc00001);
    }
    __syncthreads();
    // mirror: column gi of rows gj <- the band, 8 consecutive floats per row
    for (int e = threadIdx.x; e < BN * RROWS; e += 256) {
        const int c = e / RROWS, k = e % RROWS;
        const int gj = bj * BN + c, gi2 = bi * BM + r0 + k;
        const float v = sm[k][c];
        if (gj < p && gi2 < p && !(__float_as_int(v) == 0x7fc00001)) C[(size_t)gj * p + gi2] = v;
    }
}

__global__ void __launch_bounds__(256) k_corr_reduce(const float* __restrict__ ws, int tiles, int nr, int b0,
                                                     int nsplit, int p, float inv_n, float* __restrict__ C)
{
    __shared__ float sm[RROWS][BN + 1];
    const int t = blockIdx.x;
    int bi, bj;
    tile_rc(t, nr, b0, bi, bj);
    reduce_band(ws, t, tiles, nsplit, bi, bj, p, inv_n, C, sm);
}

// Batch form: block x = split tile of the table, written into its problem's
// p x p block of the packed C.
__global__ void __launch_bounds__(256) k_corr_reduce_batch(const float* __restrict__ ws,
                                                           const CorrTile* __restrict__ tt,
                                                           const ProbDesc* __restrict__ probs, float* __restrict__ C)
{
    __shared__ float sm[RROWS][BN + 1];
    const CorrTile T = tt[blockIdx.x];
    const ProbDesc& D = probs[T.prob];
    reduce_band(ws, T.slot0, 1, T.nsplit, T.bi, T.bj, D.p, (float)D.inv_n, C + D.c_off, sm);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    }
    return fn;
}

// Row-major bf16 panel of `rows` rows of ldk elements; boxes of 64 x box_rows.
bool make_map(CUtensorMap* m, const void* base, int rows, long long ldk, int box_rows)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)ldk, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ldk * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The four maps of a (hi, lo) operand pair; the last pair's maps are kept per
// host thread, since repeated calls reuse the same buffers and encoding is
// host work on the launch path.
bool make_maps(CUtensorMap (&m)[4], const void* hi, const void* lo, int rows, long long ldk)
{
    struct Last {
        const void *hi = nullptr, *lo = nullptr;
        int rows = -1;
        long long ldk = -1;
        CUtensorMap m[4];
    };
    static thread_local Last last;
    if (last.hi == hi && last.lo == lo && last.rows == rows && last.ldk == ldk) {
        for (int k = 0; k < 4; ++k) m[k] = last.m[k];
        return true;
    }
    if (!(make_map(&m[0], hi, rows, ldk, BM) && make_map(&m[1], lo, rows, ldk, BM) &&
          make_map(&m[2], hi, rows, ldk, BN) && make_map(&m[3], lo, rows, ldk, BN)))
        return false;
    last.hi = hi;
    last.lo = lo;
    last.rows = rows;
    last.ldk = ldk;
    for (int k = 0; k < 4; ++k) last.m[k] = m[k];
    return true;
}

cudaError_t set_smem_attr()
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_corr_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    return cudaSuccess;
}

}  // namespace

// Work split of a p x n product: K slices per tile so that the units fill the
// SMs in whole rounds (a persistent CTA per SM walks its units back to back,
// so a unit costs its K steps plus a little), slices adding a partial tile
// round trip and the reduction pass.
void corr_tc_plan(int p, long long ldk, int num_sms, int* tiles, int* nsplit, int* kps, size_t* ws_bytes)
{
    const int nr = (p + BM - 1) / BM, nc = (p + BN - 1) / BN;
    const int kt = (int)(ldk / BK);
    *tiles = tile_count(nr, nc);
    int best = 1;
    double best_cost = 1e300;
    for (int ns = 1; ns <= max(1, (3 * kt) / 8); ++ns) {
        const int k = (3 * kt + ns - 1) / ns;
        const long long units = (long long)(*tiles) * ns;
        const long long rounds = (units + num_sms - 1) / num_sms;
        const double cost = (double)rounds * (k + 1) + (ns > 1 ? 4.0 + 0.5 * (double)rounds : 0.0);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = ns;
        }
    }
    *kps = (3 * kt + best - 1) / best;
    *nsplit = (3 * kt + *kps - 1) / *kps;
    *ws_bytes = *nsplit > 1 ? (size_t)(*nsplit) * (*tiles) * BM * BN * sizeof(float) : 256;
}

cudaError_t launch_corr_tc(const void* hi, const void* lo, long long ldk, int p, int n, float* ws, float* C,
                           int num_sms, int* err, cudaStream_t st)
{
    if (ldk % BK != 0 || ((uintptr_t)hi & 15) || ((uintptr_t)lo & 15)) return cudaErrorInvalidValue;
    if (p <= 0) return cudaSuccess;
    CUtensorMap m[4];
    if (!make_maps(m, hi, lo, p, ldk)) return cudaErrorInvalidValue;
    int tiles, nsplit, kps;
    size_t wsb;
    corr_tc_plan(p, ldk, num_sms, &tiles, &nsplit, &kps, &wsb);
    cudaError_t e = set_smem_attr();
    if (e != cudaSuccess) return e;
    const int nr = (p + BM - 1) / BM;
    CorrArgs a{};
    a.kt = (int)(ldk / BK);
    a.kps = kps;
    a.nsplit = nsplit;
    a.tiles = tiles;
    a.nr = nr;
    a.b0 = nr / 2;
    a.n_units = tiles * nsplit;
    a.p = p;
    a.inv_n = (float)(1.0 / (double)n);
    a.ws = ws;
    a.C = C;
    a.err = err;
    const int grid = std::min(a.n_units, num_sms);
    k_corr_tc<<<grid, THREADS, SMEM_BYTES, st>>>(m[0], m[1], m[2], m[3], a);
    e = cudaGetLastError();
    if (e != cudaSuccess || nsplit == 1) return e;
    k_corr_reduce<<<dim3(tiles, BM / RROWS), 256, 0, st>>>(ws, tiles, nr, nr / 2, nsplit, p, a.inv_n, C);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batch: the products of many problems in one launch. The operands hold every
// problem's standardised rows at its vertex offset (ld = ldk for all); each
// problem's upper-triangle tiles are cut into K slices of at most kps steps
// (never past its own 3 kt_k steps), the work units ordered longest first.
// ---------------------------------------------------------------------------
void corr_tc_batch_plan(const std::vector<ProbDesc>& probs, int num_sms, int kps_req,
                        std::vector<CorrBatchUnit>& units, std::vector<CorrBatchTile>& tiles, size_t* ws_bytes,
                        int* kps_out)
{
    units.clear();
    tiles.clear();
    long long steps_total = 0;
    for (const ProbDesc& D : probs) {
        const int nr = (D.p + BM - 1) / BM, nc = (D.p + BN - 1) / BN;
        const int kt = (D.n + BK - 1) / BK;
        steps_total += (long long)tile_count(nr, nc) * 3 * kt;
    }
    // slice length: the makespan of one persistent CTA per SM, at least 8
    // steps a unit; a sliced tile adds its partials' round trip
    int best_kps = 8;
    double best_cost = 1e300;
    for (int kps = 8; kps <= 4096; kps *= 2) {
        long long n_units = 0, longest = 0, split_units = 0;
        for (const ProbDesc& D : probs) {
            const int nr = (D.p + BM - 1) / BM, nc = (D.p + BN - 1) / BN;
            const int kt = (D.n + BK - 1) / BK;
            const int ns = (3 * kt + kps - 1) / kps;
            const long long t = tile_count(nr, nc);
            n_units += t * ns;
            if (ns > 1) split_units += t * ns;
            longest = std::max<long long>(longest, std::min(kps, 3 * kt));
        }
        const double load = (double)(steps_total + n_units + split_units) / num_sms;
        const double cost = std::max(load, (double)(longest + 1)) + 0.02 * (double)n_units / num_sms;
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best_kps = kps;
        }
    }
    if (kps_req > 0) best_kps = kps_req;
    *kps_out = best_kps;
    int slot = 0;
    for (int k = 0; k < (int)probs.size(); ++k) {
        const ProbDesc& D = probs[k];
        const int nr = (D.p + BM - 1) / BM, nc = (D.p + BN - 1) / BN;
        const int kt = (D.n + BK - 1) / BK;
        const int ns = (3 * kt + best_kps - 1) / best_kps;
        for (int bj = 0; bj < nc; ++bj)
            for (int bi = 0; bi < nr && bi <= 2 * bj + 1; ++bi) {
                if (ns > 1) {
                    CorrBatchTile T{};
                    T.prob = k;
                    T.bi = bi;
                    T.bj = bj;
                    T.slot0 = slot;
                    T.nsplit = ns;
                    tiles.push_back(T);
                }
                for (int q = 0; q < ns; ++q) {
                    CorrBatchUnit U{};
                    U.ra = D.off + bi * BM;
                    U.rb = D.off + bj * BN;
                    U.g0 = q * best_kps;
                    U.g1 = std::min(3 * kt, (q + 1) * best_kps);
                    U.kt = kt;
                    U.slot = ns > 1 ? slot++ : -1;
                    U.prob = k;
                    units.push_back(U);
                }
            }
    }
    std::stable_sort(units.begin(), units.end(),
                     [](const CorrBatchUnit& a, const CorrBatchUnit& b) { return a.g1 - a.g0 > b.g1 - b.g0; });
    *ws_bytes = std::max<size_t>((size_t)slot * BM * BN * sizeof(float), 256);
}

cudaError_t launch_corr_tc_batch(const void* hi, const void* lo, long long ldk, int rows, const void* units,
                                 int n_units, const void* tiles, int n_tiles, const ProbDesc* probs, float* ws,
                                 float* C, int num_sms, int* err, cudaStream_t st)
{
    static_assert(sizeof(CorrBatchUnit) == sizeof(CorrWork), "work unit layout");
    static_assert(sizeof(CorrBatchTile) == sizeof(CorrTile), "tile layout");
    if (n_units == 0) return cudaSuccess;
    if (ldk % BK != 0 || ((uintptr_t)hi & 15) || ((uintptr_t)lo & 15)) return cudaErrorInvalidValue;
    CUtensorMap m[4];
    if (!make_maps(m, hi, lo, rows, ldk)) return cudaErrorInvalidValue;
    cudaError_t e = set_smem_attr();
    if (e != cudaSuccess) return e;
    CorrArgs a{};
    a.n_units = n_units;
    a.ws = ws;
    a.C = C;
    a.err = err;
    a.work = (const CorrWork*)units;
    a.probs = probs;
    k_corr_tc<<<std::min(n_units, num_sms), THREADS, SMEM_BYTES, st>>>(m[0], m[1], m[2], m[3], a);
    e = cudaGetLastError();
    if (e != cudaSuccess || n_tiles == 0) return e;
    k_corr_reduce_batch<<<dim3(n_tiles, BM / RROWS), 256, 0, st>>>(ws, (const CorrTile*)tiles, probs, C);
    return cudaGetLastError();
}

}  // namespace cupc
