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
// Kernel shape: one CTA per (128 x 128 upper-triangle output tile, K slice).
// Warp 0 issues TMA loads (128B-swizzled, K-major) into a 6-stage ring, one
// thread of warp 1 issues tcgen05.mma (M=128, N=128, K=16, bf16 -> f32) and
// returns stages with tcgen05.commit. The tensor core's FP32 accumulation
// error grows with the number of products summed into one accumulator, so the
// MMA thread restarts accumulation every GROUP K slabs, alternating between two
// TMEM accumulators; warps 2-5 drain each finished group (tcgen05.ld 32x32b)
// into FP32 registers with round-to-nearest adds while the next group runs,
// then store the partial tile. A second kernel adds the K-slice partials in a
// fixed order in FP64, scales by 1/n and writes both (i, j) and (j, i) from
// the i < j value, so C is exactly symmetric.
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

constexpr int BM = 128, BN = 128, BK = 64;      // output tile and K slab (64 bf16 = 128 bytes)
constexpr int STAGES = 6;
constexpr int TILE_BYTES = BM * BK * 2;         // 16 KiB per operand per stage
constexpr int STAGE_BYTES = 2 * TILE_BYTES;
constexpr int THREADS = 192;
constexpr uint32_t TMEM_COLS = 256;             // two FP32 accumulators of 128 lanes x 128 columns
constexpr int GROUP = 8;                        // K slabs (512 products) per accumulator group
constexpr size_t SMEM_BYTES = 2 * STAGES * TILE_BYTES + 256 + 1024;
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
// another thread of the kernel raised the error flag.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err)
{
    const unsigned long long t0 = gtimer();
    while (!mbar_try_wait(bar, parity)) {
        if (*(volatile int*)err) return false;
        if (gtimer() - t0 > kWaitNs) {
            atomicOr(err, 4);
            return false;
        }
    }
    return true;
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

__device__ __forceinline__ void tile_of(int t, int& bi, int& bj)
{
    int j = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((j + 1) * (j + 2) / 2 <= t) ++j;
    while (j * (j + 1) / 2 > t) --j;
    bj = j;
    bi = t - j * (j + 1) / 2;
}

// Work unit of a batch (a list of independent products in one launch): the
// operand rows of the A and B tiles, the K steps [g0, g1) of its 3 kt, and
// the workspace slot of its partial tile.
struct __align__(16) CorrWork {
    int ra, rb, g0, g1, kt, slot, pad0, pad1;
};

// Output tile of a batch: problem, tile coordinates, its partials' slots.
struct __align__(16) CorrTile {
    int prob, bi, bj, slot0, nsplit, pad0, pad1, pad2;
};

__global__ void __launch_bounds__(THREADS, 1)
k_corr_tc(const __grid_constant__ CUtensorMap tmH, const __grid_constant__ CUtensorMap tmL, int kt, int kps,
          int tiles, float* __restrict__ ws, int* err, const CorrWork* __restrict__ work)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = smem;
    unsigned char* sB = smem + STAGES * TILE_BYTES;
    uint64_t* full = (uint64_t*)(smem + 2 * STAGES * TILE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* acc_full = empty + STAGES;   // [2]: group accumulated (tcgen05.commit)
    uint64_t* acc_empty = acc_full + 2;    // [2]: group drained by the 4 epilogue warps
    uint32_t* tmem_slot = (uint32_t*)(acc_empty + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int ra, rb, g0, g1;
    long long slot;
    if (work) {
        const CorrWork w = work[blockIdx.x];
        ra = w.ra;
        rb = w.rb;
        g0 = w.g0;
        g1 = w.g1;
        kt = w.kt;
        slot = w.slot;
    } else {
        const int t = blockIdx.x, split = blockIdx.y;
        int bi, bj;
        tile_of(t, bi, bj);
        ra = bi * BM;
        rb = bj * BN;
        g0 = split * kps;
        g1 = min(g0 + kps, 3 * kt);
        slot = (long long)split * tiles + t;
    }
    const int nsteps = g1 - g0;
    const int ngroups = (nsteps + GROUP - 1) / GROUP;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);
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

    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int k = 0; k < nsteps; ++k) {
            const int s = k % STAGES;
            const uint32_t ph = (uint32_t)(k / STAGES) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u, err)) break;
            const int g = g0 + k, seg = g / kt, kk = g - seg * kt;
            mbar_expect_tx(&full[s], STAGE_BYTES);
            tma_load_2d(sA + s * TILE_BYTES, seg == 2 ? &tmL : &tmH, kk * BK, ra, &full[s]);
            tma_load_2d(sB + s * TILE_BYTES, seg == 1 ? &tmL : &tmH, kk * BK, rb, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: group g accumulates into TMEM columns [128 (g & 1), +128)
        for (int k = 0; k < nsteps; ++k) {
            const int g = k / GROUP, b = g & 1;
            const bool first = (k % GROUP) == 0;
            if (first && g >= 2) {
                // the previous use of buffer b must have been drained
                if (!mbar_wait(&acc_empty[b], (uint32_t)((g >> 1) - 1) & 1u, err)) break;
                tc_fence_after();
            }
            const int s = k % STAGES;
            const uint32_t ph = (uint32_t)(k / STAGES) & 1u;
            if (!mbar_wait(&full[s], ph, err)) break;
            tc_fence_after();
            const uint64_t ad = sdesc_sw128(smem_u32(sA + s * TILE_BYTES));
            const uint64_t bd = sdesc_sw128(smem_u32(sB + s * TILE_BYTES));
            const uint32_t dacc = tmem + (uint32_t)(b * BN);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)  // K = 16 per instruction: +32 bytes in the swizzled row
                mma_bf16(dacc, ad + 2 * kk, bd + 2 * kk, (first && kk == 0) ? 0u : 1u);
            mma_commit(&empty[s]);
            if ((k % GROUP) == GROUP - 1 || k == nsteps - 1) mma_commit(&acc_full[b]);
        }
    } else if (warp >= 2) {
        // epilogue: warp w may read TMEM lanes 32*(w%4) .. +31 (rows of the tile)
        const int q = warp & 3;
        const int row = q * 32 + lane;
        float R[BN];
#pragma unroll
        for (int c = 0; c < BN; ++c) R[c] = 0.f;
        bool ok = true;
        for (int g = 0; g < ngroups && ok; ++g) {
            const int b = g & 1;
            ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[b], (uint32_t)(g >> 1) & 1u, err));
            if (!ok) break;
            tc_fence_after();
            const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN);
#pragma unroll
            for (int c = 0; c < BN; c += 16) {
                uint32_t r[16];
                tmem_ld16(base + (uint32_t)c, r);
#pragma unroll
                for (int u = 0; u < 16; ++u) R[c + u] += __uint_as_float(r[u]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
        if (ok) {
            float4* out = (float4*)(ws + ((size_t)slot * BM + row) * BN);
#pragma unroll
            for (int c = 0; c < BN / 4; ++c) out[c] = make_float4(R[4 * c], R[4 * c + 1], R[4 * c + 2], R[4 * c + 3]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Sum of the K-slice partials in slice order in FP64, times 1/n; the i < j
// value is written to (i, j) and, through a shared-memory transpose, to
// (j, i); the diagonal is 1. Block (tile, 8-row band): 256 threads.
constexpr int RROWS = 8;
__device__ __forceinline__ void reduce_band(const float* __restrict__ ws, long long slot0, long long stride,
                                            int nsplit, int bi, int bj, int p, double inv_n, float* __restrict__ C,
                                            float (*sm)[BN + 1])
{
    const int r0 = blockIdx.y * RROWS;
    const int rr = threadIdx.x >> 5;            // row of the band (8 warps)
    const int lane = threadIdx.x & 31;
    const int r = r0 + rr, gi = bi * BM + r;
    for (int c = lane; c < BN; c += 32) {
        const int gj = bj * BN + c;
        float v = 0.f;
        bool valid = gi < p && gj < p && !(bi == bj && c < r);
        if (valid) {
            if (gi == gj) {
                v = 1.0f;
            } else {
                double acc = 0.0;
                for (int s = 0; s < nsplit; ++s) acc += (double)ws[((size_t)(slot0 + s * stride) * BM + r) * BN + c];
                v = (float)(acc * inv_n);
            }
            C[(size_t)gi * p + gj] = v;
        }
        sm[rr][c] = valid ? v : __int_as_float(0x7fc00001);
    }
    __syncthreads();
    // mirror: column gi of rows gj <- the band, 8 consecutive floats per row
    for (int e = threadIdx.x; e < BN * RROWS; e += 256) {
        const int c = e / RROWS, k = e % RROWS;
        const int gj = bj * BN + c, gi2 = bi * BM + r0 + k;
        const float v = sm[k][c];
        if (gj < p && gi2 < p && gj != gi2 && !(__float_as_int(v) == 0x7fc00001)) C[(size_t)gj * p + gi2] = v;
    }
}

__global__ void __launch_bounds__(256) k_corr_reduce(const float* __restrict__ ws, int tiles, int nsplit, int p,
                                                     double inv_n, float* __restrict__ C)
{
    __shared__ float sm[RROWS][BN + 1];
    const int t = blockIdx.x;
    int bi, bj;
    tile_of(t, bi, bj);
    reduce_band(ws, t, tiles, nsplit, bi, bj, p, inv_n, C, sm);
}

// Batch form: block x = output tile of the table, written into its problem's
// p x p block of the packed C.
__global__ void __launch_bounds__(256) k_corr_reduce_batch(const float* __restrict__ ws,
                                                           const CorrTile* __restrict__ tt,
                                                           const ProbDesc* __restrict__ probs, float* __restrict__ C)
{
    __shared__ float sm[RROWS][BN + 1];
    const CorrTile T = tt[blockIdx.x];
    const ProbDesc& D = probs[T.prob];
    reduce_band(ws, T.slot0, 1, T.nsplit, T.bi, T.bj, D.p, 1.0 / (double)D.n, C + D.c_off, sm);
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

bool make_map(CUtensorMap* m, const void* base, int rows, long long ldk)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)ldk, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ldk * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Workspace bytes and the split of the K loop for a p x n product.
void corr_tc_plan(int p, long long ldk, int num_sms, int* tiles, int* nsplit, int* kps, size_t* ws_bytes)
{
    const int nt = (p + BM - 1) / BM;
    const int kt = (int)(ldk / BK);
    *tiles = nt * (nt + 1) / 2;
    // K slices per tile: one CTA per SM at a time, so aim for whole waves
    // (tiles x slices close to a multiple of the SM count) with at least 16 K
    // slabs per CTA
    int best = 1;
    double best_cost = 1e300;
    for (int ns = 1; ns <= max(1, (3 * kt) / 16); ++ns) {
        const int k = (3 * kt + ns - 1) / ns;
        const long long ctas = (long long)(*tiles) * ns;
        const long long waves = (ctas + num_sms - 1) / num_sms;
        const double cost = (double)waves * (k + 4);  // +4: per-CTA fill and epilogue, in slabs
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = ns;
        }
    }
    *kps = (3 * kt + best - 1) / best;
    *nsplit = (3 * kt + *kps - 1) / *kps;
    *ws_bytes = (size_t)(*nsplit) * (*tiles) * BM * BN * sizeof(float);
}

cudaError_t launch_corr_tc(const void* hi, const void* lo, long long ldk, int p, int n, float* ws, float* C,
                           int num_sms, int* err, cudaStream_t st)
{
    if (ldk % BK != 0 || ((uintptr_t)hi & 15) || ((uintptr_t)lo & 15)) return cudaErrorInvalidValue;
    CUtensorMap mh, ml;
    if (!make_map(&mh, hi, p, ldk) || !make_map(&ml, lo, p, ldk)) return cudaErrorInvalidValue;
    int tiles, nsplit, kps;
    size_t wsb;
    corr_tc_plan(p, ldk, num_sms, &tiles, &nsplit, &kps, &wsb);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_corr_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int kt = (int)(ldk / BK);
    k_corr_tc<<<dim3(tiles, nsplit), THREADS, SMEM_BYTES, st>>>(mh, ml, kt, kps, tiles, ws, err, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_corr_reduce<<<dim3(tiles, BM / RROWS), 256, 0, st>>>(ws, tiles, nsplit, p, 1.0 / n, C);
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
        const int nt = (D.p + BM - 1) / BM;
        const int kt = (D.n + BK - 1) / BK;
        steps_total += (long long)nt * (nt + 1) / 2 * 3 * kt;
    }
    // slice length: whole waves of one CTA per SM, at least 16 steps a unit
    int best_kps = 16;
    double best_cost = 1e300;
    for (int kps = 16; kps <= 4096; kps *= 2) {
        long long n_units = 0, longest = 0;
        for (const ProbDesc& D : probs) {
            const int nt = (D.p + BM - 1) / BM;
            const int kt = (D.n + BK - 1) / BK;
            n_units += (long long)nt * (nt + 1) / 2 * ((3 * kt + kps - 1) / kps);
            longest = std::max<long long>(longest, std::min(kps, 3 * kt));
        }
        // a bound on the makespan: the average load per SM (+4 steps of fill per
        // unit) or the longest unit
        const double load = (double)(steps_total + 4 * n_units) / num_sms;
        const double cost = std::max(load, (double)(longest + 4)) + 0.02 * (double)n_units / num_sms;
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
        const int nt = (D.p + BM - 1) / BM;
        const int kt = (D.n + BK - 1) / BK;
        const int ns = (3 * kt + best_kps - 1) / best_kps;
        for (int bj = 0; bj < nt; ++bj)
            for (int bi = 0; bi <= bj; ++bi) {
                CorrBatchTile T{};
                T.prob = k;
                T.bi = bi;
                T.bj = bj;
                T.slot0 = slot;
                T.nsplit = ns;
                tiles.push_back(T);
                for (int q = 0; q < ns; ++q) {
                    CorrBatchUnit U{};
                    U.ra = D.off + bi * BM;
                    U.rb = D.off + bj * BN;
                    U.g0 = q * best_kps;
                    U.g1 = std::min(3 * kt, (q + 1) * best_kps);
                    U.kt = kt;
                    U.slot = slot++;
                    units.push_back(U);
                }
            }
    }
    std::stable_sort(units.begin(), units.end(),
                     [](const CorrBatchUnit& a, const CorrBatchUnit& b) { return a.g1 - a.g0 > b.g1 - b.g0; });
    *ws_bytes = (size_t)slot * BM * BN * sizeof(float);
}

cudaError_t launch_corr_tc_batch(const void* hi, const void* lo, long long ldk, int rows, const void* units,
                                 int n_units, const void* tiles, int n_tiles, const ProbDesc* probs, float* ws,
                                 float* C, int* err, cudaStream_t st)
{
    static_assert(sizeof(CorrBatchUnit) == sizeof(CorrWork), "work unit layout");
    static_assert(sizeof(CorrBatchTile) == sizeof(CorrTile), "tile layout");
    if (n_units == 0) return cudaSuccess;
    if (ldk % BK != 0 || ((uintptr_t)hi & 15) || ((uintptr_t)lo & 15)) return cudaErrorInvalidValue;
    CUtensorMap mh, ml;
    if (!make_map(&mh, hi, rows, ldk) || !make_map(&ml, lo, rows, ldk)) return cudaErrorInvalidValue;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_corr_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_corr_tc<<<n_units, THREADS, SMEM_BYTES, st>>>(mh, ml, 0, 0, 0, ws, err, (const CorrWork*)units);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_corr_reduce_batch<<<dim3(n_tiles, BM / RROWS), 256, 0, st>>>(ws, (const CorrTile*)tiles, probs, C);
    return cudaGetLastError();
}

}  // namespace cupc
