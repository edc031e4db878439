// api_batch.cu -- many independent problems in one pass, under a CUDA graph,
// and the autotuner for its launch configuration.
//
// The paper runs one problem per call; a problem with p of a few hundred
// leaves most of the GPU idle at every level. Here a batch of problems runs as
// one graph whose connected blocks are the problems (ProbDesc): one
// standardisation launch, one tensor-core launch over every problem's output
// tiles, one level-0 launch with its FP64 rechecks, and per level l >= 1 one
// fused level kernel whose work queue holds the (row, subset-rank chunk)
// items of all problems. PC-stable treats the blocks independently (no test
// crosses a block, Algorithm 1 only removes edges), so each problem's result
// is exactly the one of its own run.
//
// The device work of a call is recorded once into a CUDA graph and replayed
// by later calls with the same shapes: buffer sizes are fixed per plan. The
// CSR arrays are sized for the worst case (every pair an edge); the recheck
// queue and the SepSet pool start at generous sizes and, should a device-side
// capacity check trip, are enlarged, the graph re-recorded and the batch run
// again. All levels up to the plan's last possible one are in the graph; a
// level launched after the loop has ended returns at once.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "api_internal.h"
#include "records.cuh"

using namespace cupc;

namespace {

struct BatchKey {
    int nprob = 0, dtype = 0, layout = 0, on_device = 0;
    int canonical = 0, max_level = 0, chunk = 0, ctas = 0, kps = 0, direct = 0, l1form = 0;
    double margin = 0.0;
    std::vector<int64_t> n, p;
    std::vector<double> alpha;
    bool operator==(const BatchKey& o) const
    {
        return nprob == o.nprob && dtype == o.dtype && layout == o.layout && on_device == o.on_device &&
               canonical == o.canonical && max_level == o.max_level && chunk == o.chunk && ctas == o.ctas &&
               kps == o.kps && direct == o.direct && l1form == o.l1form && margin == o.margin && n == o.n && p == o.p &&
               alpha == o.alpha;
    }
};

struct BatchPlan {
    BatchKey key;
    std::vector<ProbDesc> probs;
    std::vector<int> vprob, vlmax;
    std::vector<CorrBatchUnit> units;
    std::vector<CorrBatchTile> tiles;
    int P = 0, pmax = 0, nmax = 0, lmax = 0, lmax_need = 0, kps = 0;
    long long words = 0, xelems = 0, zelems = 0, celems = 0, ldb = 0;
    size_t ws_bytes = 0;
    unsigned long long nnz_cap = 0, item_cap = 0, qcap = 0, rec_cap = 0;
    Buf d_probs, d_vprob, d_vlmax, d_units, d_tiles, x_in, xt, mu, isd, mup, zhi, zlo, ws, c32, bits, bits0;
    Buf deg, row_off, item_off, item_row, item_c, live, rc_cnt, scan_part, cols, srow, partner, row_off2, cols2, srow2, partner2, alive, nrank, wpre, best, cval, queue, part, rec, meta, lmeta, pserial;
    Binom binom{};
    // pinned host copies written at the end of each run
    unsigned* h_bits = nullptr;
    unsigned* h_bits0 = nullptr;
    LevelMeta* h_lm = nullptr;
    Meta* h_meta = nullptr;
    unsigned long long* h_ps = nullptr;
    ProbDesc* h_probs = nullptr;   // pinned: the descriptors uploaded before each run
    cudaStream_t gs = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr, ein = nullptr;
    cudaEvent_t ts[5] = {};  // stage boundaries: start, standardised, C formed, level 0 done, levels done
    int launches = 0;      // kernels one run launches
    bool graph_ok = false;
};

BatchPlan* plan_of(cupc_ctx* ctx) { return (BatchPlan*)ctx->batch; }

void plan_destroy(cupc_ctx* ctx, BatchPlan* B)
{
    if (!B) return;
    if (B->gs) cudaStreamSynchronize(B->gs);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    Buf* all[] = {&B->d_probs, &B->d_vprob, &B->d_vlmax, &B->d_units, &B->d_tiles, &B->x_in, &B->xt,      &B->mu,
                  &B->isd,     &B->mup,     &B->zhi,     &B->zlo,     &B->ws,   &B->c32,     &B->bits,
                  &B->bits0,   &B->deg,     &B->row_off, &B->item_off, &B->item_row, &B->item_c, &B->live, &B->rc_cnt, &B->scan_part, &B->cols,
                  &B->srow,    &B->partner, &B->row_off2, &B->cols2, &B->srow2, &B->partner2, &B->alive, &B->nrank, &B->wpre,    &B->best,    &B->cval,    &B->queue, &B->part,   &B->rec,
                  &B->meta,    &B->lmeta,   &B->pserial};
    for (Buf* b : all) ctx_free(ctx, b);
    if (B->h_bits) cudaFreeHost(B->h_bits);
    if (B->h_bits0) cudaFreeHost(B->h_bits0);
    if (B->h_lm) cudaFreeHost(B->h_lm);
    if (B->h_meta) cudaFreeHost(B->h_meta);
    if (B->h_ps) cudaFreeHost(B->h_ps);
    if (B->h_probs) cudaFreeHost(B->h_probs);
    if (B->e0) cudaEventDestroy(B->e0);
    if (B->e1) cudaEventDestroy(B->e1);
    if (B->ein) cudaEventDestroy(B->ein);
    for (cudaEvent_t e : B->ts)
        if (e) cudaEventDestroy(e);
    if (B->gs) cudaStreamDestroy(B->gs);
    delete B;
}

void batch_free_hook(cupc_ctx* ctx)
{
    plan_destroy(ctx, plan_of(ctx));
    ctx->batch = nullptr;
}

#define BCU(call)                                                                \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) return ctx_fail(ctx, CUPC_E_CUDA, #call, e_);     \
    } while (0)

size_t esize(int dtype) { return dtype == CUPC_F64 ? 8 : 4; }

// Layout of the problems in the packed buffers and the union graph.
void lay_out(cupc_ctx* ctx, BatchPlan& B)
{
    const BatchKey& K = B.key;
    B.probs.assign(K.nprob, ProbDesc{});
    long long off = 0, bw = 0, xo = 0, co = 0;
    B.pmax = B.nmax = 0;
    B.lmax_need = 0;
    for (int k = 0; k < K.nprob; ++k) {
        ProbDesc& D = B.probs[k];
        const int p = (int)K.p[k], n = (int)K.n[k];
        const int p32 = (p + 31) / 32 * 32;
        D.off = (int)off;
        D.p = p;
        D.n = n;
        D.inv_n = 1.0 / (double)n;
        D.wlo = (int)(off / 32);
        D.whi = (int)((off + p32) / 32);
        int lm = n - 4;
        if (K.max_level >= 0) lm = std::min(lm, K.max_level);
        D.lmax = lm;
        B.lmax_need = std::max(B.lmax_need, lm);
        D.bw = bw;
        D.c_off = co;
        D.z_off = xo;
        D.x_off = xo;
        for (int l = 0; l < LV; ++l) {
            const double r = (n - l - 3 > 0) ? std::tanh(ctx_fisher_tau(K.alpha[k], n, l)) : 0.0;
            D.r[l] = r;
            D.r2[l] = r * r;
        }
        bw += (long long)p32 * (p32 / 32);
        co += (long long)p * p;
        xo += (long long)p * n;
        off += p32;
        B.pmax = std::max(B.pmax, p);
        B.nmax = std::max(B.nmax, n);
    }
    B.P = (int)off;
    B.words = bw;
    B.celems = co;
    B.xelems = B.zelems = xo;
    B.ldb = ((long long)B.nmax + 63) / 64 * 64;
    B.vprob.assign(B.P, 0);
    B.vlmax.assign(B.P, 0);
    for (int k = 0; k < K.nprob; ++k) {
        const ProbDesc& D = B.probs[k];
        const int p32 = (D.whi - D.wlo) * 32;
        for (int v = 0; v < p32; ++v) {
            B.vprob[D.off + v] = k;
            B.vlmax[D.off + v] = D.lmax;
        }
    }
    B.lmax = std::min(B.lmax_need, CUPC_MAX_LEVEL);
}

// Device buffers of the plan (all sizes fixed by the layout and capacities).
cupc_status allocate(cupc_ctx* ctx, BatchPlan& B)
{
    const BatchKey& K = B.key;
    const size_t es = esize(K.dtype);
    struct Req {
        Buf* b;
        size_t bytes;
    };
    unsigned long long pairs2 = 0;
    for (const ProbDesc& D : B.probs) pairs2 += (unsigned long long)D.p * (D.p - 1);
    B.nnz_cap = std::max<unsigned long long>(pairs2, 1);
    B.item_cap = 1ull << 22;
    const Req reqs[] = {
        {&B.d_probs, B.probs.size() * sizeof(ProbDesc)},
        {&B.d_vprob, (size_t)B.P * 4},
        {&B.d_vlmax, (size_t)B.P * 4},
        {&B.d_units, std::max<size_t>(B.units.size(), 1) * sizeof(CorrBatchUnit)},
        {&B.d_tiles, std::max<size_t>(B.tiles.size(), 1) * sizeof(CorrBatchTile)},
        {&B.x_in, K.on_device ? 0 : (size_t)B.xelems * es},
        {&B.xt, K.layout == CUPC_LAYOUT_SAMPLE_MAJOR ? (size_t)B.xelems * es : 0},
        {&B.mu, (size_t)B.P * 8},
        {&B.isd, (size_t)B.P * 8},
        {&B.mup, (size_t)B.P * 8},
        {&B.zhi, (size_t)B.P * B.ldb * 2},
        {&B.zlo, (size_t)B.P * B.ldb * 2},
        {&B.ws, B.ws_bytes},
        {&B.c32, (size_t)B.celems * 4},
        {&B.bits, (size_t)B.words * 4},
        {&B.bits0, (size_t)B.words * 4},
        {&B.wpre, (size_t)B.words * 4},
        {&B.deg, (size_t)B.P * 4},
        {&B.row_off, (size_t)(B.P + 1) * 8},
        {&B.item_off, (size_t)(B.P + 1) * 8},
        {&B.item_row, (size_t)B.item_cap * 4},
        {&B.item_c, (size_t)B.item_cap * 4},
        {&B.scan_part, 4 * 1024 * sizeof(unsigned long long)},
        {&B.cols, (size_t)B.nnz_cap * 4},
        {&B.srow, (size_t)B.nnz_cap * 4},
        {&B.partner, (size_t)B.nnz_cap * 4},
        {&B.row_off2, (size_t)(B.P + 1) * 8},
        {&B.cols2, (size_t)B.nnz_cap * 4},
        {&B.srow2, (size_t)B.nnz_cap * 4},
        {&B.partner2, (size_t)B.nnz_cap * 4},
        {&B.alive, (size_t)B.nnz_cap},
        {&B.nrank, (size_t)B.nnz_cap * 4},
        {&B.best, (size_t)B.nnz_cap * 8},
        {&B.cval, (size_t)B.nnz_cap * 4},
        {&B.queue, (size_t)B.qcap * sizeof(QEntry)},
        {&B.live, (size_t)B.qcap * sizeof(int)},
        {&B.rc_cnt, (size_t)kRcCnt * sizeof(int)},
        {&B.part, kPartBytes},
        {&B.rec, (size_t)B.rec_cap * 4},
        {&B.meta, sizeof(Meta)},
        {&B.lmeta, sizeof(LevelMeta)},
        {&B.pserial, (size_t)K.nprob * LV * 8},
    };
    for (const Req& r : reqs) {
        cupc_status s = ctx_ensure(ctx, r.b, r.bytes);
        if (s != CUPC_OK) return s;
    }
    cupc_status s = ctx_binom(ctx, std::max(B.pmax + 2, 64), &B.binom);
    if (s != CUPC_OK) return s;
    if (!B.h_bits) {
        BCU(cudaHostAlloc((void**)&B.h_bits, (size_t)B.words * 4, cudaHostAllocDefault));
        BCU(cudaHostAlloc((void**)&B.h_bits0, (size_t)B.words * 4, cudaHostAllocDefault));
        BCU(cudaHostAlloc((void**)&B.h_lm, sizeof(LevelMeta), cudaHostAllocDefault));
        BCU(cudaHostAlloc((void**)&B.h_meta, sizeof(Meta), cudaHostAllocDefault));
        BCU(cudaHostAlloc((void**)&B.h_ps, (size_t)K.nprob * LV * 8, cudaHostAllocDefault));
        BCU(cudaHostAlloc((void**)&B.h_probs, B.probs.size() * sizeof(ProbDesc), cudaHostAllocDefault));
    }
    // descriptor tables (the pool allocations above are ordered on the context
    // stream; the problem descriptors are uploaded before each run)
    cudaStream_t st = ctx_stream(ctx);
    BCU(cudaMemcpyAsync(B.d_vprob.p, B.vprob.data(), (size_t)B.P * 4, cudaMemcpyHostToDevice, st));
    BCU(cudaMemcpyAsync(B.d_vlmax.p, B.vlmax.data(), (size_t)B.P * 4, cudaMemcpyHostToDevice, st));
    if (!B.units.empty())
        BCU(cudaMemcpyAsync(B.d_units.p, B.units.data(), B.units.size() * sizeof(CorrBatchUnit),
                            cudaMemcpyHostToDevice, st));
    if (!B.tiles.empty())
        BCU(cudaMemcpyAsync(B.d_tiles.p, B.tiles.data(), B.tiles.size() * sizeof(CorrBatchTile),
                            cudaMemcpyHostToDevice, st));
    BCU(cudaStreamSynchronize(st));  // host tables go out of scope later; the stream of the plan is another
    return CUPC_OK;
}

// The device work of one batch run, issued on stream st (recorded into the
// graph, or launched directly).
cupc_status issue(cupc_ctx* ctx, BatchPlan& B, cudaStream_t st, bool capturing)
{
    const BatchKey& K = B.key;
    const int* vprob = (const int*)B.d_vprob.p;
    const ProbDesc* probs = (const ProbDesc*)B.d_probs.p;
    Meta* meta = (Meta*)B.meta.p;
    LevelMeta* lm = (LevelMeta*)B.lmeta.p;
    int launches = 0;
    BCU(cudaMemsetAsync(meta, 0, sizeof(Meta), st));
    BCU(cudaMemsetAsync(lm, 0, sizeof(LevelMeta), st));
    BCU(cudaMemsetAsync(B.pserial.p, 0, (size_t)K.nprob * LV * 8, st));
    // stage boundaries (event nodes of the graph when recorded)
    auto stage = [&](int q) {
        return capturing ? cudaEventRecordWithFlags(B.ts[q], st, cudaEventRecordExternal) : cudaEventRecord(B.ts[q], st);
    };
    BCU(stage(0));
    // standardise every problem's variables (its variable-major rows: the data
    // itself, or its transpose)
    if (K.layout == CUPC_LAYOUT_SAMPLE_MAJOR) {
        BCU(launch_transpose_batch(K.dtype, probs, K.nprob, B.pmax, B.nmax, B.xt.p, st));
        ++launches;
    }
    BCU(launch_standardize(K.dtype, nullptr, 0, 0, B.P, (double*)B.mu.p, (double*)B.isd.p, (float2*)B.mup.p, nullptr,
                           0, B.zhi.p, B.zlo.p, B.ldb, meta, st, vprob, probs));
    ++launches;
    BCU(stage(1));
    // every problem's C on the tensor cores
    BCU(launch_corr_tc_batch(B.zhi.p, B.zlo.p, B.ldb, B.P, B.d_units.p, (int)B.units.size(), B.d_tiles.p,
                             (int)B.tiles.size(), probs, (float*)B.ws.p, (float*)B.c32.p, ctx_num_sms(ctx),
                             &meta->error, st));
    launches += (B.units.empty() ? 0 : 1) + (B.tiles.empty() ? 0 : 1);
    BCU(stage(2));
    // level 0 and its FP64 rechecks
    BCU(launch_level0(1, B.c32.p, B.P, 0, 0.0, kBand0, (unsigned*)B.bits.p, (QEntry*)B.queue.p, B.qcap, meta, st,
                      vprob, probs, B.P));
    ++launches;
    Recheck0Params rp{};
    rp.xf64 = K.dtype == CUPC_F64 ? 1 : 0;
    rp.mu = (const double*)B.mu.p;
    rp.isd = (const double*)B.isd.p;
    rp.mup = (const float2*)B.mup.p;
    rp.p = B.P;
    rp.queue = (const QEntry*)B.queue.p;
    rp.qcap = B.qcap;
    rp.meta = meta;
    rp.bits = (unsigned*)B.bits.p;
    rp.vprob = vprob;
    rp.probs = probs;
    BCU(launch_recheck0(rp, std::max(1, ctx_num_sms(ctx) * 8), st));
    ++launches;
    BCU(cudaMemcpyAsync(B.bits0.p, B.bits.p, (size_t)B.words * 4, cudaMemcpyDeviceToDevice, st));
    BCU(launch_degree((const unsigned*)B.bits.p, B.P, 0, (int*)B.deg.p, meta, st, vprob, probs));
    ++launches;
    BCU(stage(3));
    // levels 1 .. lmax of the union graph
    LevelParams LP{};
    LP.bits = (unsigned*)B.bits.p;
    LP.W = 0;
    LP.p = B.P;
    LP.nwords = B.words;
    LP.deg = (int*)B.deg.p;
    LP.row_off = (long long*)B.row_off.p;
    LP.item_off = (long long*)B.item_off.p;
    LP.item_row = (int*)B.item_row.p;
    LP.item_c = (int*)B.item_c.p;
    LP.item_cap = B.item_cap;
    LP.cols = (int*)B.cols.p;
    LP.srow = (int*)B.srow.p;
    LP.partner = (int*)B.partner.p;
    LP.row_off2 = (long long*)B.row_off2.p;
    LP.cols2 = (int*)B.cols2.p;
    LP.srow2 = (int*)B.srow2.p;
    LP.partner2 = (int*)B.partner2.p;
    LP.alive = (unsigned char*)B.alive.p;
    LP.nrank = (int*)B.nrank.p;
    LP.wpre = (int*)B.wpre.p;
    LP.best = (unsigned long long*)B.best.p;
    LP.nnz_cap = B.nnz_cap;
    LP.C = B.c32.p;
    // level 1 by conditioning variable when the largest problem's C row fits
    LP.l1_pivot = level1_by_pivot(K.l1form) ? l1_buffers(B.pmax, 4) : 0;
    LP.pstage = B.pmax;
    LP.cval = B.cval.p;
    LP.B = B.binom;
    LP.chunk0 = K.chunk ? K.chunk : 32;
    LP.canonical = K.canonical;
    LP.band_abs = (K.margin > 0) ? K.margin : kBandAbs;
    LP.band_rel = kBandRel;
    LP.rank_tol = kRankTol32;
    LP.piv_floor = kPivFloor;
    LP.queue = (QEntry*)B.queue.p;
    LP.live = (int*)B.live.p;
    LP.rc_cnt = (int*)B.rc_cnt.p;
    LP.qcap = B.qcap;
    LP.xf64 = K.dtype == CUPC_F64 ? 1 : 0;
    LP.mu = (const double*)B.mu.p;
    LP.isd = (const double*)B.isd.p;
    LP.mup = (const float2*)B.mup.p;
    LP.nmax = B.nmax;
    LP.part = (double*)B.part.p;
    LP.part_cap = kPartBytes / sizeof(double);
    LP.rec = (int*)B.rec.p;
    LP.rec_cap = B.rec_cap;
    LP.lm = lm;
    LP.scan_part = (unsigned long long*)B.scan_part.p;
    LP.vprob = vprob;
    LP.probs = probs;
    LP.vlmax = (const int*)B.d_vlmax.p;
    LP.prob_serial = (unsigned long long*)B.pserial.p;
    LP.ctas_per_sm = K.ctas;
    for (int l = 1; l <= B.lmax; ++l) {
        LP.l = l;
        BCU(launch_level(1, LP, ctx_num_sms(ctx), st));
        ++launches;
    }
    BCU(stage(4));
    // results to pinned host memory
    BCU(cudaMemcpyAsync(B.h_meta, meta, sizeof(Meta), cudaMemcpyDeviceToHost, st));
    BCU(cudaMemcpyAsync(B.h_lm, lm, sizeof(LevelMeta), cudaMemcpyDeviceToHost, st));
    BCU(cudaMemcpyAsync(B.h_bits, B.bits.p, (size_t)B.words * 4, cudaMemcpyDeviceToHost, st));
    BCU(cudaMemcpyAsync(B.h_bits0, B.bits0.p, (size_t)B.words * 4, cudaMemcpyDeviceToHost, st));
    BCU(cudaMemcpyAsync(B.h_ps, B.pserial.p, (size_t)K.nprob * LV * 8, cudaMemcpyDeviceToHost, st));
    B.launches = launches;
    return CUPC_OK;
}

// Records the run into a graph; on any capture failure the plan falls back to
// direct launches (B.graph_ok = false).
cupc_status capture(cupc_ctx* ctx, BatchPlan& B)
{
    if (B.exec) {
        cudaGraphExecDestroy(B.exec);
        B.exec = nullptr;
    }
    B.graph_ok = false;
    if (B.key.direct) return CUPC_OK;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(B.gs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();
        return CUPC_OK;
    }
    cupc_status s = issue(ctx, B, B.gs, true);
    cudaError_t e = cudaStreamEndCapture(B.gs, &g);
    if (s != CUPC_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        ctx->err.clear();
        return CUPC_OK;
    }
    e = cudaGraphInstantiate(&B.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        B.exec = nullptr;
        cudaGetLastError();
        return CUPC_OK;
    }
    B.graph_ok = true;
    return CUPC_OK;
}

cupc_status build_plan(cupc_ctx* ctx, const BatchKey& key, BatchPlan** out)
{
    BatchPlan* B = new BatchPlan();
    B->key = key;
    lay_out(ctx, *B);
    corr_tc_batch_plan(B->probs, ctx_num_sms(ctx), key.kps, B->units, B->tiles, &B->ws_bytes, &B->kps);
    B->qcap = std::max<unsigned long long>(1ull << 20, 4ull * B->P);
    B->rec_cap = (unsigned long long)(3 + B->lmax) * std::max<unsigned long long>(1ull << 20, 8ull * B->P);
    cupc_status s;
    if (cudaStreamCreateWithFlags(&B->gs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&B->e0) != cudaSuccess || cudaEventCreate(&B->e1) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ein, cudaEventDisableTiming) != cudaSuccess || cudaEventCreate(&B->ts[0]) ||
        cudaEventCreate(&B->ts[1]) || cudaEventCreate(&B->ts[2]) || cudaEventCreate(&B->ts[3]) ||
        cudaEventCreate(&B->ts[4])) {
        plan_destroy(ctx, B);
        return ctx_fail(ctx, CUPC_E_CUDA, "batch stream/events");
    }
    if ((s = allocate(ctx, *B)) != CUPC_OK || (s = capture(ctx, *B)) != CUPC_OK) {
        plan_destroy(ctx, B);
        return s;
    }
    *out = B;
    return CUPC_OK;
}

// Grows the buffer whose device-side capacity check tripped and re-records.
cupc_status grow(cupc_ctx* ctx, BatchPlan& B, unsigned long long qneed, unsigned long long rneed)
{
    if (qneed > B.qcap) {
        B.qcap = qneed + qneed / 2;
        ctx_free(ctx, &B.queue);
        ctx_free(ctx, &B.live);
    }
    if (rneed > B.rec_cap) {
        B.rec_cap = rneed + rneed / 2;
        ctx_free(ctx, &B.rec);
    }
    cupc_status s = allocate(ctx, B);
    if (s != CUPC_OK) return s;
    return capture(ctx, B);
}

cupc_status run_once(cupc_ctx* ctx, BatchPlan& B, const void* const* X, float* ms)
{
    const BatchKey& K = B.key;
    const size_t es = esize(K.dtype);
    // after the work already queued on the context stream
    BCU(cudaEventRecord(B.ein, ctx_stream(ctx)));
    BCU(cudaStreamWaitEvent(B.gs, B.ein, 0));
    BCU(cudaEventRecord(B.e0, B.gs));
    // inputs: host data is copied into the packed input buffer; device data is
    // read where it is. The descriptors carry this call's data pointers.
    for (int k = 0; k < K.nprob; ++k) {
        ProbDesc& D = B.probs[k];
        if (K.on_device) {
            D.xs = X[k];
        } else {
            D.xs = (const char*)B.x_in.p + (size_t)D.x_off * es;
            BCU(cudaMemcpyAsync((void*)D.xs, X[k], (size_t)D.p * D.n * es, cudaMemcpyHostToDevice, B.gs));
        }
        D.xv = (K.layout == CUPC_LAYOUT_SAMPLE_MAJOR) ? (const void*)((const char*)B.xt.p + (size_t)D.x_off * es)
                                                      : D.xs;
    }
    std::memcpy(B.h_probs, B.probs.data(), B.probs.size() * sizeof(ProbDesc));
    BCU(cudaMemcpyAsync(B.d_probs.p, B.h_probs, B.probs.size() * sizeof(ProbDesc), cudaMemcpyHostToDevice, B.gs));
    if (B.graph_ok) {
        BCU(cudaGraphLaunch(B.exec, B.gs));
    } else {
        cupc_status s = issue(ctx, B, B.gs, false);
        if (s != CUPC_OK) return s;
    }
    BCU(cudaEventRecord(B.e1, B.gs));
    BCU(cudaStreamWaitEvent(ctx_stream(ctx), B.e1, 0));  // later work on the context stream follows the batch
    BCU(cudaStreamSynchronize(B.gs));
    *ms = 0.f;
    cudaEventElapsedTime(ms, B.e0, B.e1);
    return CUPC_OK;
}

cupc_status check_args(cupc_ctx* ctx, int nprob, const void* const* X, int dtype, int layout,
                       const int64_t* n, const int64_t* p, const double* alpha, const cupc_options& o)
{
    if (nprob < 1 || nprob > 4096) return ctx_fail(ctx, CUPC_E_INVALID, "nprob must be in [1, 4096]");
    if (!X || !n || !p || !alpha) return ctx_fail(ctx, CUPC_E_INVALID, "NULL argument array");
    if (dtype != CUPC_F32 && dtype != CUPC_F64) return ctx_fail(ctx, CUPC_E_INVALID, "dtype");
    if (layout != CUPC_LAYOUT_SAMPLE_MAJOR && layout != CUPC_LAYOUT_VARIABLE_MAJOR)
        return ctx_fail(ctx, CUPC_E_INVALID, "layout");
    cupc_status s = ctx_validate(ctx, o);
    if (s != CUPC_OK) return s;
    if (o.mode != CUPC_MODE_FP32_RECHECK) return ctx_fail(ctx, CUPC_E_INVALID, "batches run in FP32_RECHECK mode");
    if (o.learned_order) return ctx_fail(ctx, CUPC_E_INVALID, "batches do not take learned_order");
    long long tot = 0;
    for (int k = 0; k < nprob; ++k) {
        if (!X[k]) return ctx_fail(ctx, CUPC_E_INVALID, "X[" + std::to_string(k) + "] is NULL");
        if (p[k] < 2 || p[k] > (1 << 20)) return ctx_fail(ctx, CUPC_E_INVALID, "p[k] must be in [2, 2^20]");
        if (n[k] < 4 || n[k] > (1ll << 31) - 1) return ctx_fail(ctx, CUPC_E_INVALID, "n_samples[k] out of range");
        if (!(alpha[k] > 0.0 && alpha[k] < 1.0)) return ctx_fail(ctx, CUPC_E_INVALID, "alpha[k] must be in (0, 1)");
        if ((double)n[k] * (double)p[k] > 4e9) return ctx_fail(ctx, CUPC_E_INVALID, "n * p too large");
        tot += (p[k] + 31) / 32 * 32;
    }
    if (tot > (1 << 20)) return ctx_fail(ctx, CUPC_E_INVALID, "sum of p (rounded up to 32) exceeds 2^20");
    return CUPC_OK;
}

BatchKey make_key(int nprob, int dtype, int layout, int on_device, const int64_t* n, const int64_t* p,
                  const double* alpha, const cupc_options& o)
{
    BatchKey k;
    k.nprob = nprob;
    k.dtype = dtype;
    k.layout = layout;
    k.on_device = on_device ? 1 : 0;
    k.canonical = o.canonical_sepset;
    k.max_level = o.max_level;
    k.chunk = o.chunk;
    k.ctas = o.ctas_per_sm;
    k.kps = o.corr_kps;
    k.direct = o.batch_direct;
    k.l1form = o.level1_form;
    k.margin = o.recheck_margin;
    k.n.assign(n, n + nprob);
    k.p.assign(p, p + nprob);
    k.alpha.assign(alpha, alpha + nprob);
    return k;
}

// Runs the batch on the context's plan (built or rebuilt as needed), growing
// capacities until the run fits. On success the pinned host copies hold the
// run's results.
cupc_status run_batch(cupc_ctx* ctx, const BatchKey& key, const void* const* X, float* ms)
{
    BatchPlan* B = plan_of(ctx);
    if (!B || !(B->key == key)) {
        if (B) batch_free_hook(ctx);
        cupc_status s = build_plan(ctx, key, &B);
        if (s != CUPC_OK) return s;
        ctx->batch = B;
        ctx->batch_free = batch_free_hook;
    }
    for (int attempt = 0;; ++attempt) {
        cupc_status s = run_once(ctx, *B, X, ms);
        if (s != CUPC_OK) return s;
        const Meta& M = *B->h_meta;
        const LevelMeta& H = *B->h_lm;
        if (M.error & 4) return ctx_fail(ctx, CUPC_E_TIMEOUT, "a bounded wait in the tensor-core product expired");
        if (M.error) return ctx_fail(ctx, CUPC_E_NUMERIC, "a variable has zero variance or non-finite data");
        if (H.error & 8) return ctx_fail(ctx, CUPC_E_TIMEOUT, "a grid barrier wait expired");
        if (H.error) return ctx_fail(ctx, CUPC_E_RANGE, "level buffers too small");
        if (H.range_error) return ctx_fail(ctx, CUPC_E_RANGE, "subset count exceeds 64 bits");
        unsigned long long qneed = M.queue_len;
        if (H.overflow_level) qneed = std::max(qneed, H.queue_len[H.overflow_level]);
        const unsigned long long rneed = H.rec_ints;
        if (qneed <= B->qcap && rneed <= B->rec_cap) break;
        if (attempt >= 4) return ctx_fail(ctx, CUPC_E_RANGE, "batch capacities keep overflowing");
        if ((s = grow(ctx, *B, qneed, rneed)) != CUPC_OK) return s;
    }
    const LevelMeta& H = *B->h_lm;
    if (B->lmax_need > CUPC_MAX_LEVEL && H.done_level == 0)
        return ctx_fail(ctx, CUPC_E_RANGE, "a level above CUPC_MAX_LEVEL would be needed");
    return CUPC_OK;
}

inline int popc32(unsigned w) { return __builtin_popcount(w); }

// Per-problem results (host-side bitsets and SepSet records) and batch stats.
cupc_status make_results(cupc_ctx* ctx, BatchPlan& B, float ms, cupc_result** out, cupc_stats* bst)
{
    const BatchKey& K = B.key;
    const LevelMeta& H = *B.h_lm;
    const Meta& M = *B.h_meta;
    const int last = H.done_level ? H.done_level - 1 : B.lmax;
    const int levels = last + 1;
    for (int k = 0; k < K.nprob; ++k) out[k] = nullptr;
    // records in (i, j) order with local ids, sorted on the device over the
    // union graph (problem by problem) and downloaded in one copy with each
    // row's int offset and the per-problem, per-level counts; the host sort
    // below is the fallback when the counts do not add up
    bool dev_sorted = false;
    const int32_t* srec = nullptr;          // the sorted records (pinned staging)
    const long long* roff = nullptr;        // int offset of each union row's records, P + 1
    const unsigned long long* plc = nullptr;  // records per problem and level
    size_t d2h_rec = 0;
    if (H.rec_ints > 0) {
        RecGroups G{};
        long long at = 0, idx = 0;
        for (int l = 1; l <= last && l <= CUPC_MAX_LEVEL; ++l) {
            const long long c = (long long)H.removed[l];
            if (c == 0) continue;
            G.lev[G.groups] = l;
            G.start[G.groups] = at;
            G.count[G.groups] = c;
            G.first[G.groups] = idx;
            ++G.groups;
            at += c * (3 + l);
            idx += c;
        }
        G.total = idx;
        if (at == (long long)H.rec_ints) {
            auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
            const size_t ints = (size_t)H.rec_ints, rows = (size_t)B.P;
            const size_t b_wpre = al((size_t)B.words * 4), b_r1 = al((rows + 1) * 8), b_slot = al((size_t)G.total * 8),
                         b_plc = al((size_t)K.nprob * kRecGroups * 8), b_out = al(64 + ints * 4);
            Buf* sb = ctx_buf(ctx, "rec_sort");
            cupc_status s = ctx_ensure(ctx, sb, b_wpre + 4 * b_r1 + b_slot + b_plc + b_out);
            if (s != CUPC_OK) return s;
            char* c = (char*)sb->p;
            unsigned* wpre = (unsigned*)c;
            c += b_wpre;
            long long* rowcnt = (long long*)c;
            c += b_r1;
            long long* rowstart = (long long*)c;
            c += b_r1;
            unsigned long long* rowints = (unsigned long long*)c;
            c += b_r1;
            long long* rowoff = (long long*)c;
            c += b_r1;
            long long* slot = (long long*)c;
            c += b_slot;
            unsigned long long* dplc = (unsigned long long*)c;
            c += b_plc;
            long long* status = (long long*)c;     // error flags, removed pairs, ints placed; the records follow
            char* h = nullptr;
            if ((s = ctx_host_stage(ctx, b_out + b_r1 + b_plc, &h)) != CUPC_OK) return s;
            const RowView V{(const int*)B.d_vprob.p, (const ProbDesc*)B.d_probs.p, 0, 0};
            BCU(cudaMemsetAsync(dplc, 0, b_plc, B.gs));
            BCU(launch_records_sort((const int*)B.rec.p, G, (const unsigned*)B.bits.p, (const unsigned*)B.bits0.p, V,
                                    (long long)rows, wpre, rowcnt, rowstart, rowints, rowoff, slot,
                                    (int*)((char*)status + 64), status, dplc, kRecGroups, B.gs));
            BCU(cudaMemcpyAsync(h, status, 64 + ints * 4, cudaMemcpyDeviceToHost, B.gs));
            BCU(cudaMemcpyAsync(h + b_out, rowoff, (rows + 1) * 8, cudaMemcpyDeviceToHost, B.gs));
            BCU(cudaMemcpyAsync(h + b_out + b_r1, dplc, (size_t)K.nprob * kRecGroups * 8, cudaMemcpyDeviceToHost,
                                B.gs));
            BCU(cudaStreamSynchronize(B.gs));
            d2h_rec = 64 + ints * 4 + (rows + 1) * 8 + (size_t)K.nprob * kRecGroups * 8;
            long long hs[3];
            std::memcpy(hs, h, sizeof(hs));
            if (hs[0] == 0 && hs[1] == G.total && hs[2] == (long long)ints) {
                dev_sorted = true;
                srec = (const int32_t*)(h + 64);
                roff = (const long long*)(h + b_out);
                plc = (const unsigned long long*)(h + b_out + b_r1);
            }
        }
    }
    std::vector<int32_t> raw;
    std::vector<std::vector<size_t>> idx(K.nprob);
    if (!dev_sorted && H.rec_ints > 0) {
        // records: (i, j, l, S) in global ids, split by problem into local ids
        raw.resize((size_t)H.rec_ints);
        BCU(cudaMemcpyAsync(raw.data(), B.rec.p, raw.size() * 4, cudaMemcpyDeviceToHost, B.gs));
        BCU(cudaStreamSynchronize(B.gs));
        d2h_rec = raw.size() * 4;
        // each problem's record offsets in (i, j) order: a least-significant-digit
        // radix sort, a stable counting sort on local j and then on local i
        for (size_t q = 0; q < raw.size();) {
            const int l = raw[q + 2];
            if (l < 1 || l > CUPC_MAX_LEVEL || q + 3 + l > raw.size())
                return ctx_fail(ctx, CUPC_E_STATE, "bad SepSet record");
            idx[B.vprob[raw[q]]].push_back(q);
            q += 3 + l;
        }
        std::vector<size_t> cnt, tmp;
        for (int k = 0; k < K.nprob; ++k) {
            std::vector<size_t>& v = idx[k];
            if (v.size() < 2) continue;
            const ProbDesc& D = B.probs[k];
            cnt.assign((size_t)D.p + 1, 0);
            tmp.resize(v.size());
            auto pass = [&](std::vector<size_t>& in, std::vector<size_t>& o, int field) {
                std::fill(cnt.begin(), cnt.end(), 0);
                for (const size_t q : in) ++cnt[(size_t)(raw[q + field] - D.off) + 1];
                for (int i = 0; i < D.p; ++i) cnt[(size_t)i + 1] += cnt[(size_t)i];
                for (const size_t q : in) o[cnt[(size_t)(raw[q + field] - D.off)]++] = q;
            };
            pass(v, tmp, 1);   // by local j
            pass(tmp, v, 0);   // by local i, stable
        }
    }
    cupc_stats S{};
    S.levels = levels;
    for (int k = 0; k < K.nprob; ++k) {
        const ProbDesc& D = B.probs[k];
        cupc_result* R = new cupc_result();
        R->ctx = ctx;
        ctx->refs++;
        R->p = D.p;
        R->W = D.whi - D.wlo;
        R->on_host = true;
        const size_t nw = (size_t)D.p * R->W;
        R->hbits.assign(B.h_bits + D.bw, B.h_bits + D.bw + nw);
        R->hbits0.assign(B.h_bits0 + D.bw, B.h_bits0 + D.bw + nw);
        std::vector<int64_t> rem(CUPC_STATS_LEVELS, 0);
        if (dev_sorted) {
            // its union rows D.off .. D.off + p32 hold its records, ids already local
            const long long a = roff[D.off], b = roff[D.off + (D.whi - D.wlo) * 32];
            R->hrec.assign(srec + a, srec + b);
            for (int l = 1; l < CUPC_STATS_LEVELS && l < kRecGroups; ++l) rem[l] = (int64_t)plc[(size_t)k * kRecGroups + l];
        } else {
            size_t ints = 0;
            for (const size_t q : idx[k]) ints += 3 + (size_t)raw[q + 2];
            R->hrec.resize(ints);
            R->index.resize(idx[k].size());
            size_t w = 0, r = 0;
            for (const size_t q : idx[k]) {
                const int l = raw[q + 2];
                const int i = raw[q] - D.off, j = raw[q + 1] - D.off;
                R->index[r++] = std::make_pair((uint64_t)i * (uint64_t)D.p + (uint64_t)j, (int64_t)w);
                int32_t* o = R->hrec.data() + w;
                o[0] = i;
                o[1] = j;
                o[2] = l;
                for (int c = 0; c < l; ++c) o[3 + c] = raw[q + 3 + c] - D.off;
                w += 3 + (size_t)l;
                if (l < CUPC_STATS_LEVELS) rem[l]++;
            }
        }
        R->host_ready = true;
        R->index_ready = !dev_sorted;
        R->rec_ints = (int64_t)R->hrec.size();
        // per-problem counters
        const int64_t pairs = (int64_t)D.p * (D.p - 1) / 2;
        int64_t e0 = 0;
        for (size_t w = 0; w < nw; ++w) e0 += popc32(R->hbits0[w]);
        e0 /= 2;
        cupc_stats& st = R->stats;
        st.levels = levels;
        st.tests[0] = pairs;
        st.serial_tests[0] = pairs;
        st.removed[0] = pairs - e0;
        st.edges_start[0] = pairs;
        st.rechecks[0] = -1;
        int64_t edges = e0;
        for (int l = 1; l < levels && l < CUPC_STATS_LEVELS; ++l) {
            st.tests[l] = -1;
            st.rechecks[l] = -1;
            st.edges_start[l] = edges;
            st.removed[l] = rem[l];
            st.serial_tests[l] = K.canonical ? (int64_t)B.h_ps[(size_t)k * LV + l] : -1;
            edges -= rem[l];
        }
        st.edges_final = edges;
        st.total_ms = ms;
        st.cuda_graph = B.graph_ok ? 1 : 0;
        out[k] = R;
        // batch totals
        S.tests[0] += pairs;
        S.serial_tests[0] += pairs;
        S.removed[0] += pairs - e0;
        S.edges_start[0] += pairs;
        S.edges_final += edges;
    }
    S.rechecks[0] = (int64_t)M.rechecks;
    S.max_degree[0] = B.pmax - 1;
    for (int l = 1; l < levels && l < CUPC_STATS_LEVELS; ++l) {
        S.tests[l] = (int64_t)H.tests[l];
        S.serial_tests[l] = K.canonical ? (int64_t)H.serial[l] : -1;
        S.removed[l] = (int64_t)H.removed[l];
        S.rechecks[l] = (int64_t)H.rechecks[l];
        S.edges_start[l] = (int64_t)H.edges[l];
        S.max_degree[l] = H.maxdeg[l];
        S.ci_block_entries[l] = (int64_t)H.block_entries[l];
        for (int c = 0; c < 4; ++c) S.phase_ms[l][c] = 1e-6f * (float)H.phase_ns[l][c];
        for (int c = 0; c < 3; ++c) S.recheck_ms[l][c] = 1e-6f * (float)H.recheck_ns[l][c];
        S.rechecks_queued[l] = (int64_t)H.queue_len[l];
    }
    for (int l = 1; l < LV; ++l) {
        S.kernel_ms[CUPC_K_COMPACT] += 1e-6f * (float)H.phase_ns[l][0];
        S.kernel_ms[CUPC_K_CI] += 1e-6f * (float)H.phase_ns[l][1];
        S.kernel_ms[CUPC_K_RECHECK] += 1e-6f * (float)H.phase_ns[l][2];
        S.kernel_ms[CUPC_K_FINALIZE] += 1e-6f * (float)H.phase_ns[l][3];
    }
    {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, B.e0, B.ts[0]) == cudaSuccess) S.kernel_ms[CUPC_K_UPLOAD] = t;
        if (cudaEventElapsedTime(&t, B.ts[0], B.ts[1]) == cudaSuccess) S.kernel_ms[CUPC_K_STANDARDIZE] = t;
        if (cudaEventElapsedTime(&t, B.ts[1], B.ts[2]) == cudaSuccess) S.kernel_ms[CUPC_K_CORRELATION] = t;
        if (cudaEventElapsedTime(&t, B.ts[2], B.ts[3]) == cudaSuccess) S.kernel_ms[CUPC_K_LEVEL0] = t;
        if (cudaEventElapsedTime(&t, B.ts[0], B.ts[2]) == cudaSuccess) S.prep_ms = t;
        if (cudaEventElapsedTime(&t, B.ts[3], B.ts[4]) == cudaSuccess) S.level_ms[1] = t;  // all levels >= 1
        cudaGetLastError();
    }
    S.kernel_count[CUPC_K_STANDARDIZE] = K.layout == CUPC_LAYOUT_SAMPLE_MAJOR ? 2 : 1;
    S.kernel_count[CUPC_K_CORRELATION] = 2;
    S.kernel_count[CUPC_K_LEVEL0] = 2;
    S.kernel_count[CUPC_K_COMPACT] = 1;
    S.kernel_count[CUPC_K_CI] = B.lmax;
    S.total_ms = ms;
    S.kernel_launches = B.launches;
    const size_t es = esize(K.dtype);
    S.h2d_bytes = K.on_device ? 0 : (int64_t)(B.xelems * es);
    S.d2h_bytes = (int64_t)(2 * B.words * 4 + sizeof(Meta) + sizeof(LevelMeta) + (size_t)K.nprob * LV * 8 + d2h_rec);
    S.cuda_graph = B.graph_ok ? 1 : 0;
    if (bst) *bst = S;
    return CUPC_OK;
}

}  // namespace

extern "C" {

cupc_status cupc_skeleton_batch(cupc_ctx* ctx, int nprob, const void* const* X, int dtype, int layout,
                                int on_device, const int64_t* n_samples, const int64_t* p, const double* alpha,
                                const cupc_options* opts, cupc_result** out, cupc_stats* batch_stats)
{
    if (!ctx) return CUPC_E_INVALID;
    if (!out) return ctx_fail(ctx, CUPC_E_INVALID, "out is NULL");
    const auto h0 = std::chrono::steady_clock::now();
    for (int k = 0; k < nprob && k < 4096; ++k) out[k] = nullptr;
    cupc_options o;
    cupc_options_default(&o);
    if (opts) o = *opts;
    cupc_status s = check_args(ctx, nprob, X, dtype, layout, n_samples, p, alpha, o);
    if (s != CUPC_OK) return s;
    BCU(cudaSetDevice(ctx->device));
    const BatchKey key = make_key(nprob, dtype, layout, on_device, n_samples, p, alpha, o);
    float ms = 0.f;
    if ((s = run_batch(ctx, key, X, &ms)) != CUPC_OK) return s;
    const auto h1 = std::chrono::steady_clock::now();
    s = make_results(ctx, *plan_of(ctx), ms, out, batch_stats);
    if (s != CUPC_OK) {
        for (int k = 0; k < nprob; ++k) {
            cupc_result_free(out[k]);
            out[k] = nullptr;
        }
        return s;
    }
    if (batch_stats) {
        batch_stats->host_ms[0] = std::chrono::duration<float, std::milli>(h1 - h0).count();
        batch_stats->host_ms[1] =
            std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - h1).count();
    }
    ctx->err.clear();
    return CUPC_OK;
}

cupc_status cupc_batch_autotune(cupc_ctx* ctx, int nprob, const void* const* X, int dtype, int layout,
                                int on_device, const int64_t* n_samples, const int64_t* p, const double* alpha,
                                const cupc_options* base, int reps, cupc_tune_entry* entries, int cap,
                                int* n_entries)
{
    if (!ctx) return CUPC_E_INVALID;
    if (!entries || !n_entries || cap < 1) return ctx_fail(ctx, CUPC_E_INVALID, "entries");
    if (reps < 1 || reps > 16) return ctx_fail(ctx, CUPC_E_INVALID, "reps must be in [1, 16]");
    *n_entries = 0;
    cupc_options o;
    cupc_options_default(&o);
    if (base) o = *base;
    cupc_status s = check_args(ctx, nprob, X, dtype, layout, n_samples, p, alpha, o);
    if (s != CUPC_OK) return s;
    BCU(cudaSetDevice(ctx->device));
    // the product's K steps: the cost model's choice, half and double of it
    int kps_model = 0;
    {
        cupc_options m = o;
        m.corr_kps = 0;
        const BatchKey key = make_key(nprob, dtype, layout, on_device, n_samples, p, alpha, m);
        BatchPlan probe;
        probe.key = key;
        lay_out(ctx, probe);
        size_t wsb;
        corr_tc_batch_plan(probe.probs, ctx_num_sms(ctx), 0, probe.units, probe.tiles, &wsb, &kps_model);
    }
    const int chunks[] = {8, 16, 32, 64, 128};
    const int ctas[] = {1, 2};
    const int kpss[] = {kps_model, std::max(16, kps_model / 2), kps_model * 2};
    std::vector<cupc_tune_entry> all;
    std::vector<unsigned> ref_bits;
    std::vector<int32_t> ref_rec;
    for (int kp : kpss)
        for (int c : ctas)
            for (int ch : chunks) {
                cupc_options t = o;
                t.chunk = ch;
                t.ctas_per_sm = c;
                t.corr_kps = kp;
                const BatchKey key = make_key(nprob, dtype, layout, on_device, n_samples, p, alpha, t);
                float best = 1e30f;
                for (int r = 0; r < reps + 1; ++r) {  // the first run may record the graph
                    float ms = 0.f;
                    if ((s = run_batch(ctx, key, X, &ms)) != CUPC_OK) return s;
                    if (r > 0) best = std::min(best, ms);
                }
                BatchPlan& B = *plan_of(ctx);
                // the configuration must not change the result
                std::vector<unsigned> bits(B.h_bits, B.h_bits + B.words);
                std::vector<int32_t> rec((size_t)B.h_lm->rec_ints);
                if (!rec.empty()) {
                    BCU(cudaMemcpy(rec.data(), B.rec.p, rec.size() * 4, cudaMemcpyDeviceToHost));
                }
                // records come in device order: compare them as a sorted multiset of records
                std::vector<std::vector<int32_t>> rs;
                for (size_t q = 0; q < rec.size();) {
                    const int l = rec[q + 2];
                    rs.emplace_back(rec.begin() + q, rec.begin() + q + 3 + l);
                    q += 3 + l;
                }
                std::sort(rs.begin(), rs.end());
                std::vector<int32_t> flat;
                for (auto& v : rs) flat.insert(flat.end(), v.begin(), v.end());
                if (all.empty()) {
                    ref_bits = bits;
                    ref_rec = flat;
                } else if (bits != ref_bits || (o.canonical_sepset && flat != ref_rec)) {
                    return ctx_fail(ctx, CUPC_E_STATE, "launch configurations disagree on the result");
                }
                cupc_tune_entry e{};
                e.chunk = ch;
                e.ctas_per_sm = c;
                e.corr_kps = B.kps;
                e.ms = best;
                all.push_back(e);
            }
    std::stable_sort(all.begin(), all.end(), [](const cupc_tune_entry& a, const cupc_tune_entry& b) {
        return a.ms < b.ms;
    });
    const int nw = std::min<int>(cap, (int)all.size());
    for (int q = 0; q < nw; ++q) entries[q] = all[q];
    *n_entries = nw;
    ctx->err.clear();
    return CUPC_OK;
}

}  // extern "C"
