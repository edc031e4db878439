// api.cu -- C ABI of the skeleton library: context, workspace, the level loop
// of Algorithm 2 (level 0, then per level: compact A_G into A'_G, CI tests,
// removal and SepSet records), results and their accessors.
#include <algorithm>
#include <cstddef>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "api_internal.h"
#include "records.cuh"

using namespace cupc;

namespace {

void ctx_release(cupc_ctx* c);

cupc_status fail(cupc_ctx* c, cupc_status s, const std::string& what, cudaError_t e = cudaSuccess)
{
    if (c) {
        c->err = what;
        if (e != cudaSuccess) {
            c->err += ": ";
            c->err += cudaGetErrorString(e);
            cudaGetLastError();
        }
    }
    return s;
}

#define CU(call)                                                                 \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) return fail(ctx, CUPC_E_CUDA, #call, e_);         \
    } while (0)

// Host-side fault injection (cupc_debug_fail): true when the armed failure of
// this kind is due now (the countdown reached the k-th event); it disarms.
bool injected(cupc_ctx* ctx, int kind)
{
    if (ctx->fail_kind != kind) return false;
    if (--ctx->fail_k > 0) return false;
    ctx->fail_kind = 0;
    return true;
}

#define LAUNCH(call)                                                             \
    do {                                                                         \
        if (injected(ctx, CUPC_FAIL_LAUNCH))                                     \
            return fail(ctx, CUPC_E_CUDA, "injected launch failure: " #call);    \
        cudaError_t e_ = (call);                                                 \
        ctx->launches++;                                                         \
        if (e_ != cudaSuccess) return fail(ctx, CUPC_E_CUDA, #call, e_);         \
    } while (0)

cupc_status dalloc(cupc_ctx* ctx, void** p, size_t bytes)
{
    *p = nullptr;
    if (injected(ctx, CUPC_FAIL_ALLOC))
        return fail(ctx, CUPC_E_NOMEM, "injected failure of a device allocation of " + std::to_string(bytes) + " bytes");
    if (bytes == 0) bytes = 256;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(ctx, CUPC_E_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes", e);
    }
    return CUPC_OK;
}

cupc_status ensure(cupc_ctx* ctx, Buf& b, size_t bytes, bool keep = false)
{
    if (b.p && b.cap >= bytes) return CUPC_OK;
    size_t cap = std::max(bytes, b.cap + b.cap / 2);
    cap = (cap + 255) & ~size_t(255);
    void* np = nullptr;
    cupc_status s = dalloc(ctx, &np, cap);
    if (s != CUPC_OK) return s;
    if (keep && b.p && b.cap) CU(cudaMemcpyAsync(np, b.p, b.cap, cudaMemcpyDeviceToDevice, ctx->stream));
    if (b.p) cudaFreeAsync(b.p, ctx->stream);
    b.p = np;
    b.cap = cap;
    return CUPC_OK;
}

void free_buf(cupc_ctx* ctx, Buf& b)
{
    if (b.p) cudaFreeAsync(b.p, ctx->stream);
    b.p = nullptr;
    b.cap = 0;
}

// --- threshold (Eq. threshold) -------------------------------------------------
// Lower-tail standard normal quantile: Newton steps on Phi(x) - q with
// Phi(x) = erfc(-x/sqrt 2)/2 and Phi'(x) = exp(-x^2/2)/sqrt(2 pi), started
// from the tail estimate x = -sqrt(-2 ln q) and kept inside a bisection bracket.
double normal_quantile_lower(double q)
{
    if (!(q > 0.0 && q < 0.5)) return q == 0.5 ? 0.0 : NAN;
    double lo = -40.0, hi = 0.0;
    double x = -std::sqrt(-2.0 * std::log(q));
    const double inv_sqrt_2pi = 0.3989422804014326779399461;
    for (int it = 0; it < 200; ++it) {
        const double f = 0.5 * std::erfc(-x / std::sqrt(2.0)) - q;
        if (f < 0.0) lo = x; else hi = x;
        const double fp = inv_sqrt_2pi * std::exp(-0.5 * x * x);
        double xn = (fp > 0.0) ? x - f / fp : 0.5 * (lo + hi);
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        if (std::fabs(xn - x) <= 1e-16 * std::fabs(x) || hi - lo <= 1e-16 * std::fabs(x)) { x = xn; break; }
        x = xn;
    }
    return x;
}

double fisher_tau(double alpha, int64_t n, int l)
{
    const double dof = (double)(n - l - 3);
    if (!(dof > 0.0)) return NAN;
    return -normal_quantile_lower(0.5 * alpha) / std::sqrt(dof);
}

// --- binomial table ------------------------------------------------------------
cupc_status ensure_binom(cupc_ctx* ctx, int m_needed)
{
    if (ctx->binom_mstride >= m_needed && ctx->binom.p) return CUPC_OK;
    const int ms = std::max(m_needed, 64);
    const int K = CUPC_MAX_LEVEL + 2;
    std::vector<unsigned long long> h((size_t)K * ms);
    for (int k = 0; k < K; ++k)
        for (int m = 0; m < ms; ++m) {
            unsigned long long v;
            if (k > m) v = 0;
            else if (k == 0) v = 1;
            else {
                // C(m, k) = C(m-1, k-1) + C(m-1, k), saturating
                const unsigned long long a = h[(size_t)(k - 1) * ms + (m - 1)];
                const unsigned long long b = h[(size_t)k * ms + (m - 1)];
                v = (a == ~0ull || b == ~0ull || a > ~0ull - b) ? ~0ull : a + b;
            }
            h[(size_t)k * ms + m] = v;
        }
    cupc_status s = ensure(ctx, ctx->binom, h.size() * sizeof(unsigned long long));
    if (s != CUPC_OK) return s;
    CU(cudaMemcpyAsync(ctx->binom.p, h.data(), h.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));  // h goes out of scope
    ctx->binom_mstride = ms;
    return CUPC_OK;
}

Binom binom_view(cupc_ctx* ctx)
{
    Binom b;
    b.tab = (const unsigned long long*)ctx->binom.p;
    b.mstride = ctx->binom_mstride;
    return b;
}

// Level-boundary checkpoint (host bytes): this header, then A_G after the last
// level run (p x W words), A_G after level 0 (p x W words) and the SepSet
// records (rec_ints int32, in the order the device appended them).
struct CkptHeader {
    char magic[8];              // "CUPCCKP1"
    int32_t version;            // 1
    int32_t level;              // last level run
    int64_t p, n;
    double alpha;
    int32_t mode, canonical, learned, W;
    int64_t rec_ints;
    cupc_stats stats;           // counters of levels 0 .. level
};
constexpr char kCkptMagic[8] = {'C', 'U', 'P', 'C', 'C', 'K', 'P', '1'};

struct Input {
    bool is_corr = false;
    const void* X = nullptr;
    int dtype = CUPC_F64;
    int layout = CUPC_LAYOUT_SAMPLE_MAJOR;
    int on_device = 0;
    int64_t n = 0, p = 0, ld = 0;
    // resume: the checkpoint's state (nullptr: a fresh run)
    const CkptHeader* ck = nullptr;
    const unsigned* ck_bits = nullptr;
    const unsigned* ck_bits0 = nullptr;
    const int32_t* ck_rec = nullptr;
};

size_t elem_size(int dtype) { return dtype == CUPC_F64 ? 8 : 4; }

// Opens a timed region of kernel class `cls`; returns its slot or -1 when the
// event pool is exhausted (the launch then goes untimed).
int tbegin(cupc_ctx* ctx, int cls)
{
    if (ctx->tused + 2 > (int)ctx->tev.size()) return -1;
    const int k = ctx->tused;
    ctx->tused += 2;
    ctx->tcls[k / 2] = cls;
    cudaEventRecord(ctx->tev[k], ctx->stream);
    return k;
}

void tend(cupc_ctx* ctx, int k)
{
    if (k >= 0) cudaEventRecord(ctx->tev[k + 1], ctx->stream);
}

// The copy stream of chunked uploads and its events, created on first use.
cupc_status ensure_copy_stream(cupc_ctx* ctx)
{
    if (ctx->cstream) return CUPC_OK;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return CUPC_E_CUDA;
    for (cudaEvent_t& e : ctx->cev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaStreamDestroy(st);
            return CUPC_E_CUDA;
        }
    ctx->cstream = st;
    return CUPC_OK;
}

void tcollect(cupc_ctx* ctx, cupc_stats& st)
{
    for (int k = 0; k + 1 < ctx->tused; k += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->tev[k], ctx->tev[k + 1]) == cudaSuccess) {
            const int c = ctx->tcls[k / 2];
            st.kernel_ms[c] += ms;
        }
    }
    cudaGetLastError();
    ctx->tused = 0;
}

#define TIMED(cls, call)                                                         \
    do {                                                                         \
        const int tk_ = tbegin(ctx, (cls));                                      \
        LAUNCH(call);                                                            \
        tend(ctx, tk_);                                                          \
        kcount[(cls)]++;                                                         \
    } while (0)

cupc_status readback(cupc_ctx* ctx)
{
    CU(cudaMemcpyAsync(ctx->hmeta, ctx->meta.p, sizeof(Meta), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->d2h += sizeof(Meta);
    return CUPC_OK;
}

// Standardise + correlation. On return *Cuse is the matrix the CI kernels
// read; c64 (correlation input) or the data view feeds the FP64 rechecks.
// Data the FP64 rechecks read: the variable-major data rows and the moments of
// the standardisation (z is recomputed from them bit for bit).
struct DataView {
    const void* xv = nullptr;
    long long ldx = 0;
    int xf64 = 0;
    const double* mu = nullptr;
    const double* isd = nullptr;
    const float2* mup = nullptr;   // the mean as an FP32 pair (FP32 mode)
};

cupc_status prepare(cupc_ctx* ctx, const Input& in, bool fp32, const void** Cuse, const double** c64_out,
                    DataView* dv, int* kcount)
{
    const int n = (int)in.n, p = (int)in.p;
    const size_t es = elem_size(in.dtype);
    Meta* meta = (Meta*)ctx->meta.p;
    *c64_out = nullptr;
    *dv = DataView();
    if (in.is_corr) {
        const void* src = in.X;
        const size_t extent = ((size_t)(p - 1) * in.ld + p) * es;
        if (!in.on_device) {
            cupc_status s = ensure(ctx, ctx->cin, extent);
            if (s != CUPC_OK) return s;
            const int tk = tbegin(ctx, CUPC_K_UPLOAD);
            CU(cudaMemcpyAsync(ctx->cin.p, in.X, extent, cudaMemcpyHostToDevice, ctx->stream));
            tend(ctx, tk);
            ctx->h2d += extent;
            src = ctx->cin.p;
        }
        cupc_status s = ensure(ctx, ctx->c64, (size_t)p * p * 8);
        if (s != CUPC_OK) return s;
        if (fp32) {
            s = ensure(ctx, ctx->c32, (size_t)p * p * 4);
            if (s != CUPC_OK) return s;
        }
        TIMED(CUPC_K_STANDARDIZE, launch_symmetrize(in.dtype, src, in.ld, p, (double*)ctx->c64.p,
                                                    fp32 ? (float*)ctx->c32.p : nullptr, ctx->stream));
        *c64_out = (const double*)ctx->c64.p;
        *Cuse = fp32 ? ctx->c32.p : ctx->c64.p;
        return CUPC_OK;
    }
    const void* src = in.X;
    const size_t extent = (in.layout == CUPC_LAYOUT_SAMPLE_MAJOR) ? ((size_t)(n - 1) * in.ld + p) * es
                                                                 : ((size_t)(p - 1) * in.ld + n) * es;
    const long long ldz = n;
    const long long ldb = ((long long)n + 63) / 64 * 64;  // K padded to whole 64-wide slabs
    {
        cupc_status s;
        if ((s = ensure(ctx, ctx->mu, (size_t)p * 8)) != CUPC_OK) return s;
        if ((s = ensure(ctx, ctx->isd, (size_t)p * 8)) != CUPC_OK) return s;
        if (fp32 && (s = ensure(ctx, ctx->mup, (size_t)p * 8)) != CUPC_OK) return s;
        // FP64 rows only for the FP64 product (plain mode); FP32 mode keeps the bf16 split
        if (!fp32 && (s = ensure(ctx, ctx->z64, (size_t)p * ldz * 8)) != CUPC_OK) return s;
        if (fp32) {
            if ((s = ensure(ctx, ctx->zhi, (size_t)p * ldb * 2)) != CUPC_OK) return s;
            if ((s = ensure(ctx, ctx->zlo, (size_t)p * ldb * 2)) != CUPC_OK) return s;
        }
    }
    auto standardize = [&](const void* rows, int v0, int v1) {
        return launch_standardize(in.dtype, rows, in.ld, n, v1 - v0, (double*)ctx->mu.p + v0,
                                  (double*)ctx->isd.p + v0, fp32 ? (float2*)ctx->mup.p + v0 : nullptr,
                                  fp32 ? nullptr : (double*)ctx->z64.p + (size_t)v0 * ldz, ldz,
                                  fp32 ? (void*)((unsigned short*)ctx->zhi.p + (size_t)v0 * ldb) : nullptr,
                                  fp32 ? (void*)((unsigned short*)ctx->zlo.p + (size_t)v0 * ldb) : nullptr, ldb,
                                  meta, ctx->stream);
    };
    // A variable-major host input of some size is uploaded in variable chunks on
    // a copy stream, and each chunk is standardised once it has arrived, so the
    // standardisation of one chunk runs while the next is on the host link. The
    // standardisation form a launch picks depends on its variable count, so the
    // chunks are used only where they pick the same form as the whole input.
    constexpr int kChunks = 4;
    constexpr size_t kChunkMinBytes = size_t(8) << 20;
    const bool same_form = n > 4096 || p < 1024 || p / kChunks >= 1024;
    const bool chunked = !in.on_device && in.layout == CUPC_LAYOUT_VARIABLE_MAJOR && extent >= kChunkMinBytes &&
                         p >= 4 * kChunks && same_form;
    bool standardized = false;
    if (!in.on_device) {
        cupc_status s = ensure(ctx, ctx->xin, extent);
        if (s != CUPC_OK) return s;
        if (chunked && ensure_copy_stream(ctx) == CUPC_OK) {
            // the copy stream starts after the context stream's earlier work (the
            // input buffer may still be read there)
            CU(cudaEventRecord(ctx->cev[7], ctx->stream));
            CU(cudaStreamWaitEvent(ctx->cstream, ctx->cev[7], 0));
            const int tk = (ctx->tused + 2 <= (int)ctx->tev.size()) ? ctx->tused : -1;
            if (tk >= 0) {
                ctx->tused += 2;
                ctx->tcls[tk / 2] = CUPC_K_UPLOAD;
                CU(cudaEventRecord(ctx->tev[tk], ctx->cstream));
            }
            for (int c = 0; c < kChunks; ++c) {
                const int v0 = (int)((long long)p * c / kChunks), v1 = (int)((long long)p * (c + 1) / kChunks);
                const size_t off = (size_t)v0 * in.ld * es;
                const size_t bytes = ((size_t)(v1 - 1 - v0) * in.ld + n) * es;
                CU(cudaMemcpyAsync((char*)ctx->xin.p + off, (const char*)in.X + off, bytes, cudaMemcpyHostToDevice,
                                   ctx->cstream));
                CU(cudaEventRecord(ctx->cev[c], ctx->cstream));
                CU(cudaStreamWaitEvent(ctx->stream, ctx->cev[c], 0));
                TIMED(CUPC_K_STANDARDIZE, standardize((const char*)ctx->xin.p + off, v0, v1));
            }
            if (tk >= 0) CU(cudaEventRecord(ctx->tev[tk + 1], ctx->cstream));
            standardized = true;
        } else {
            const int tk = tbegin(ctx, CUPC_K_UPLOAD);
            CU(cudaMemcpyAsync(ctx->xin.p, in.X, extent, cudaMemcpyHostToDevice, ctx->stream));
            tend(ctx, tk);
        }
        ctx->h2d += extent;
        src = ctx->xin.p;
    }
    const void* xv = src;
    long long ldv = in.ld;
    if (in.layout == CUPC_LAYOUT_SAMPLE_MAJOR) {
        cupc_status s = ensure(ctx, ctx->xt, (size_t)n * p * es);
        if (s != CUPC_OK) return s;
        TIMED(CUPC_K_STANDARDIZE, launch_transpose(in.dtype, src, in.ld, n, p, ctx->xt.p, ctx->stream));
        xv = ctx->xt.p;
        ldv = n;
    }
    cupc_status s;
    if (!standardized)
        TIMED(CUPC_K_STANDARDIZE,
              launch_standardize(in.dtype, xv, ldv, n, p, (double*)ctx->mu.p, (double*)ctx->isd.p,
                                 fp32 ? (float2*)ctx->mup.p : nullptr,
                                 fp32 ? nullptr : (double*)ctx->z64.p, ldz, fp32 ? ctx->zhi.p : nullptr,
                                 fp32 ? ctx->zlo.p : nullptr, ldb, meta, ctx->stream));
    dv->xv = xv;
    dv->ldx = ldv;
    dv->xf64 = in.dtype == CUPC_F64 ? 1 : 0;
    dv->mu = (const double*)ctx->mu.p;
    dv->isd = (const double*)ctx->isd.p;
    dv->mup = fp32 ? (const float2*)ctx->mup.p : nullptr;
    if (!fp32) {
        if ((s = ensure(ctx, ctx->c64, (size_t)p * p * 8)) != CUPC_OK) return s;
        TIMED(CUPC_K_CORRELATION,
              launch_syrk_f64((const double*)ctx->z64.p, ldz, n, p, (double*)ctx->c64.p, ctx->stream));
        *c64_out = (const double*)ctx->c64.p;
        *Cuse = ctx->c64.p;
    } else {
        if ((s = ensure(ctx, ctx->c32, (size_t)p * p * 4)) != CUPC_OK) return s;
        int tiles, nsplit, kps;
        size_t wsb;
        corr_tc_plan(p, ldb, ctx->num_sms, &tiles, &nsplit, &kps, &wsb);
        if ((s = ensure(ctx, ctx->cws, wsb)) != CUPC_OK) return s;
        TIMED(CUPC_K_CORRELATION, launch_corr_tc(ctx->zhi.p, ctx->zlo.p, ldb, p, n, (float*)ctx->cws.p,
                                                 (float*)ctx->c32.p, ctx->num_sms, &meta->error, ctx->stream));
        if (nsplit > 1) kcount[CUPC_K_CORRELATION]++;  // the K-slice reduction
        *Cuse = ctx->c32.p;
    }
    return CUPC_OK;
}

cupc_status validate_opts(cupc_ctx* ctx, const cupc_options& o)
{
    if (o.mode != CUPC_MODE_PLAIN_FP64 && o.mode != CUPC_MODE_FP32_RECHECK)
        return fail(ctx, CUPC_E_INVALID, "unknown mode");
    if (o.max_level < -1) return fail(ctx, CUPC_E_INVALID, "max_level must be >= -1");
    if (o.learned_order && !ctx->mlp_ready)
        return fail(ctx, CUPC_E_STATE, "learned ordering needs network weights (cupc_mlp_set_weights)");
    if (o.learned_order && o.mode != CUPC_MODE_FP32_RECHECK)
        return fail(ctx, CUPC_E_INVALID, "learned ordering runs in CUPC_MODE_FP32_RECHECK");
    if (o.threads_per_block != 0 && (o.threads_per_block % 32 != 0 || o.threads_per_block > 256))
        return fail(ctx, CUPC_E_INVALID, "threads_per_block must be a multiple of 32 up to 256");
    if (o.chunk < 0) return fail(ctx, CUPC_E_INVALID, "chunk must be >= 0");
    if (o.ctas_per_sm < 0 || o.corr_kps < 0) return fail(ctx, CUPC_E_INVALID, "ctas_per_sm, corr_kps must be >= 0");
    if (o.level1_form < CUPC_L1_AUTO || o.level1_form > CUPC_L1_BY_ROW)
        return fail(ctx, CUPC_E_INVALID, "level1_form must be CUPC_L1_AUTO, CUPC_L1_BY_PIVOT or CUPC_L1_BY_ROW");
    if (o.host_lists != 0 && o.host_lists != 1) return fail(ctx, CUPC_E_INVALID, "host_lists must be 0 or 1");
    return CUPC_OK;
}

void free_result(cupc_result* r)
{
    if (!r) return;
    cupc_ctx* ctx = r->ctx;
    if (ctx) {
        if (r->bits) cudaFreeAsync(r->bits, ctx->stream);
        if (r->bits0) cudaFreeAsync(r->bits0, ctx->stream);
        if (r->rec) cudaFreeAsync(r->rec, ctx->stream);
        ctx_release(ctx);
    }
    delete r;
}

// Pinned host memory of at least `bytes` for downloads of device-built result
// lists; the context keeps it for later calls.
cupc_status host_stage(cupc_ctx* ctx, size_t bytes, char** out)
{
    if (ctx->hstage_cap < bytes) {
        if (ctx->hstage) cudaFreeHost(ctx->hstage);
        ctx->hstage = nullptr;
        ctx->hstage_cap = 0;
        const size_t cap = std::max(bytes, (size_t)1 << 20);
        cudaError_t e = cudaMallocHost(&ctx->hstage, cap);
        if (e != cudaSuccess) {
            ctx->hstage = nullptr;
            return fail(ctx, CUPC_E_NOMEM, "pinned staging buffer of " + std::to_string(cap) + " bytes", e);
        }
        ctx->hstage_cap = cap;
    }
    *out = (char*)ctx->hstage;
    return CUPC_OK;
}

// Device scratch released on the context's stream when the scope ends.
struct ScratchGuard {
    cupc_ctx* ctx;
    void* p;
    ~ScratchGuard()
    {
        if (p) cudaFreeAsync(p, ctx->stream);
    }
};

// A single call's records grouped by level from its per-level removal counts
// (a call appends them level by level); false when the counts do not account
// for the pool exactly.
bool record_groups(const cupc_result* r, RecGroups& G)
{
    G = RecGroups{};
    long long at = 0, idx = 0;
    for (int l = 1; l < r->stats.levels && l < CUPC_STATS_LEVELS && l <= CUPC_MAX_LEVEL; ++l) {
        const long long c = r->stats.removed[l];
        if (c < 0) return false;
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
    return at == r->rec_ints;
}

// Edges of a single call's result from its per-level removal counts.
long long result_edge_count(const cupc_result* r)
{
    long long e = r->stats.edges_start[0] - r->stats.removed[0];
    for (int q = 1; q < r->stats.levels && q < CUPC_STATS_LEVELS; ++q) e -= r->stats.removed[q];
    return e;
}

// Device builds of a result's host lists in flight: where their downloads
// (a 64-byte status block, then the list) land in the pinned staging buffer.
struct ListsPending {
    bool recs = false, edges = false;
    char* h = nullptr;
    size_t rec_block = 0;          // bytes of the records' download (the edges' follows)
    long long n_recs = 0;
    long long n_edges = 0;
};

// Enqueues on the context's stream the device builds of the sorted records
// (recs) and of the edge list (edges) of a single call's result and their
// downloads; lists_finish takes them once the stream is synchronised. A list
// whose counts do not add up is left out (its first request then builds it
// on the host). Scratch is released in stream order.
cupc_status lists_enqueue(const cupc_result* r, bool recs, bool edges, ListsPending& L)
{
    cupc_ctx* ctx = r->ctx;
    L = ListsPending{};
    if (r->on_host) return CUPC_OK;
    RecGroups G;
    recs = recs && !r->host_ready && r->rec_ints > 0 && record_groups(r, G);
    const long long E = result_edge_count(r);
    edges = edges && !r->edges_ready && E >= 0;
    if (!recs && !edges) return CUPC_OK;
    const int p = (int)r->p, W = r->W;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t ints = recs ? (size_t)r->rec_ints : 0;
    const size_t b_rec = recs ? al(64 + ints * 4) : 0, b_edge = edges ? 64 + (size_t)E * 8 : 0;
    char* h = nullptr;
    cupc_status s = host_stage(ctx, b_rec + b_edge, &h);
    if (s != CUPC_OK) return s;
    cudaStream_t st = ctx->stream;
    const size_t b_p1 = al(((size_t)p + 1) * 8);
    if (recs) {
        const size_t m = (size_t)G.total;
        const size_t b_wpre = al((size_t)p * W * 4), b_slot = al(m * 8);
        void* scratch = nullptr;
        if ((s = dalloc(ctx, &scratch, b_wpre + 4 * b_p1 + b_slot + b_rec)) != CUPC_OK) return s;
        ScratchGuard guard{ctx, scratch};
        char* c = (char*)scratch;
        unsigned* wpre = (unsigned*)c;
        c += b_wpre;
        long long* rowcnt = (long long*)c;
        c += b_p1;
        long long* rowstart = (long long*)c;
        c += b_p1;
        unsigned long long* rowints = (unsigned long long*)c;
        c += b_p1;
        long long* rowoff = (long long*)c;
        c += b_p1;
        long long* slot = (long long*)c;
        c += b_slot;
        long long* status = (long long*)c;     // error flags, removed pairs, ints placed; the records follow
        const RowView V{nullptr, nullptr, W, p};
        LAUNCH(launch_records_sort(r->rec, G, r->bits, r->bits0, V, p, wpre, rowcnt, rowstart, rowints, rowoff, slot,
                                   (int*)(c + 64), status, nullptr, 0, st));
        CU(cudaMemcpyAsync(h, status, 64 + ints * 4, cudaMemcpyDeviceToHost, st));
        ctx->d2h += 64 + ints * 4;
        L.recs = true;
        L.n_recs = G.total;
    }
    if (edges) {
        void* scratch = nullptr;
        if ((s = dalloc(ctx, &scratch, 2 * b_p1 + b_edge)) != CUPC_OK) return s;
        ScratchGuard guard{ctx, scratch};
        long long* rowcnt = (long long*)scratch;
        long long* off = (long long*)((char*)scratch + b_p1);
        long long* status = (long long*)((char*)scratch + 2 * b_p1);   // the edge count; the pairs follow
        LAUNCH(launch_edge_list(r->bits, p, W, rowcnt, off, E, (int*)((char*)status + 64), status, st));
        CU(cudaMemcpyAsync(h + b_rec, status, b_edge, cudaMemcpyDeviceToHost, st));
        ctx->d2h += b_edge;
        L.edges = true;
        L.n_edges = E;
    }
    L.h = h;
    L.rec_block = b_rec;
    return CUPC_OK;
}

// Takes the downloads of lists_enqueue after the stream has been synchronised:
// each list whose checks pass becomes the result's host copy.
void lists_finish(const cupc_result* r, const ListsPending& L)
{
    if (L.recs) {
        long long hs[3];
        std::memcpy(hs, L.h, sizeof(hs));
        if (hs[0] == 0 && hs[1] == L.n_recs && hs[2] == r->rec_ints) {
            const int32_t* a = (const int32_t*)(L.h + 64);
            r->hrec.assign(a, a + r->rec_ints);
            r->host_ready = true;
            r->index_ready = false;
        }
    }
    if (L.edges) {
        const char* h = L.h + L.rec_block;
        long long total = 0;
        std::memcpy(&total, h, 8);
        if (total == L.n_edges) {
            const int32_t* a = (const int32_t*)(h + 64);
            r->hedges.assign(a, a + 2 * L.n_edges);
            r->edges_ready = true;
        }
    }
}

// Builds the requested lists on the device now (enqueue, synchronise, take).
cupc_status device_lists(const cupc_result* r, bool recs, bool edges)
{
    ListsPending L;
    cupc_status s = lists_enqueue(r, recs, edges, L);
    if (s != CUPC_OK || (!L.recs && !L.edges)) return s;
    cupc_ctx* ctx = r->ctx;
    CU(cudaStreamSynchronize(ctx->stream));
    lists_finish(r, L);
    return CUPC_OK;
}

// Event that marks the end of a call's device work (after the event slots of
// the prep step and the levels).
constexpr int kEvFin = CUPC_STATS_LEVELS + 2;

cupc_status run(cupc_ctx* ctx, const Input& in, double alpha, const cupc_options* popts, cupc_result** out)
{
    if (!out) return fail(ctx, CUPC_E_INVALID, "out is NULL");
    const auto h0 = std::chrono::steady_clock::now();
    *out = nullptr;
    cupc_options o;
    cupc_options_default(&o);
    if (popts) o = *popts;
    cupc_status s = validate_opts(ctx, o);
    if (s != CUPC_OK) return s;
    if (!in.X) return fail(ctx, CUPC_E_INVALID, "input pointer is NULL");
    if (in.dtype != CUPC_F32 && in.dtype != CUPC_F64) return fail(ctx, CUPC_E_INVALID, "dtype");
    if (in.p < 2 || in.p > (1 << 20)) return fail(ctx, CUPC_E_INVALID, "p must be in [2, 2^20]");
    if (!(alpha > 0.0 && alpha < 1.0)) return fail(ctx, CUPC_E_INVALID, "alpha must be in (0, 1)");
    if (in.n < 4 || in.n > (1ll << 31) - 1) return fail(ctx, CUPC_E_INVALID, "n_samples out of range");
    if (!in.is_corr) {
        if (in.layout != CUPC_LAYOUT_SAMPLE_MAJOR && in.layout != CUPC_LAYOUT_VARIABLE_MAJOR)
            return fail(ctx, CUPC_E_INVALID, "layout");
        if (in.ld < (in.layout == CUPC_LAYOUT_SAMPLE_MAJOR ? in.p : in.n))
            return fail(ctx, CUPC_E_INVALID, "ld smaller than the row length");
        if ((double)in.n * (double)in.p > 4e9) return fail(ctx, CUPC_E_INVALID, "n * p too large");
    } else if (in.ld < in.p) {
        return fail(ctx, CUPC_E_INVALID, "ld < p");
    }

    const CkptHeader* ck = in.ck;
    if (ck) {
        if (ck->p != in.p || ck->n != in.n || !(ck->alpha == alpha))
            return fail(ctx, CUPC_E_INVALID, "checkpoint of another problem (p, n or alpha differ)");
        if (ck->mode != o.mode || ck->canonical != o.canonical_sepset || ck->learned != o.learned_order)
            return fail(ctx, CUPC_E_INVALID, "checkpoint taken with other options (mode, canonical, learned)");
        if (o.max_level >= 0 && o.max_level < ck->level)
            return fail(ctx, CUPC_E_INVALID, "max_level below the checkpoint's level");
    }
    CU(cudaSetDevice(ctx->device));
    const bool fp32 = (o.mode == CUPC_MODE_FP32_RECHECK);
    const int p = (int)in.p;
    const int W = (p + 31) / 32;
    const int from = ck ? ck->level + 1 : 1;       // first level to run
    const unsigned barrier_ns = ctx->barrier_ns;   // a test's grid-barrier limit applies to one call
    ctx->barrier_ns = 0;
    // a cancellation request ends the call between levels (the work in flight is
    // waited for; the context stays usable)
    auto cancelled = [&]() -> bool {
        if (ctx->cancel.exchange(0) == 0) return false;
        cudaStreamSynchronize(ctx->stream);
        cudaGetLastError();
        return true;
    };
    const int64_t n = in.n;
    const unsigned long long launches0 = ctx->launches, h2d0 = ctx->h2d, d2h0 = ctx->d2h;
    int kcount[CUPC_KCLASSES] = {0};
    ctx->tused = 0;

    if ((s = ensure(ctx, ctx->meta, sizeof(Meta))) != CUPC_OK) return s;
    Meta* meta = (Meta*)ctx->meta.p;
    CU(cudaMemsetAsync(meta, 0, sizeof(Meta), ctx->stream));
    CU(cudaEventRecord(ctx->ev[0], ctx->stream));

    cupc_result* R = new cupc_result();
    R->ctx = ctx;
    ctx->refs++;
    R->p = p;
    R->W = W;
    R->n = n;
    R->alpha = alpha;
    R->mode = o.mode;
    R->canonical = o.canonical_sepset;
    R->learned = o.learned_order;
    struct Guard {
        cupc_result*& r;
        bool ok = false;
        ~Guard() { if (!ok) { free_result(r); r = nullptr; } }
    } guard{R};

    const void* Cuse = nullptr;
    const double* c64 = nullptr;
    DataView dv;
    if ((s = prepare(ctx, in, fp32, &Cuse, &c64, &dv, kcount)) != CUPC_OK) return s;
    CU(cudaEventRecord(ctx->ev[1], ctx->stream));

    const size_t bitbytes = (size_t)p * W * 4;
    if ((s = dalloc(ctx, (void**)&R->bits, bitbytes)) != CUPC_OK) return s;
    if ((s = dalloc(ctx, (void**)&R->bits0, bitbytes)) != CUPC_OK) return s;
    size_t qcap = o.test_qcap > 0 ? (size_t)o.test_qcap : std::max<size_t>(1u << 20, (size_t)4 * p);
    int reruns[4] = {0, 0, 0, 0};
    if (fp32 && (s = ensure(ctx, ctx->queue, qcap * sizeof(QEntry))) != CUPC_OK) return s;
    if ((s = ensure_binom(ctx, std::max(p + 1, 64))) != CUPC_OK) return s;

    const int grid_wide = std::max(1, ctx->num_sms * 8);
    auto recheck0_params = [&]() {
        Recheck0Params rp{};
        rp.xv = dv.xv;
        rp.ldx = dv.ldx;
        rp.xf64 = dv.xf64;
        rp.mu = dv.mu;
        rp.isd = dv.isd;
        rp.mup = dv.mup;
        rp.n = (int)n;
        rp.inv_n = 1.0 / (double)n;
        rp.c64 = c64;
        rp.p = p;
        const double r = std::tanh(fisher_tau(alpha, n, 0));
        rp.r2 = r * r;
        rp.queue = (const QEntry*)ctx->queue.p;
        rp.qcap = qcap;
        rp.meta = meta;
        rp.bits = R->bits;
        rp.W = W;
        return rp;
    };

    // ---------------- level 0 (Algorithm 3) and the levels (Algorithm 2 loop) ----------------
    const int64_t pairs = (int64_t)p * (p - 1) / 2;
    R->stats.tests[0] = pairs;
    R->stats.serial_tests[0] = pairs;
    R->stats.edges_start[0] = pairs;
    R->stats.max_degree[0] = p - 1;
    // last level that may run: Eq. (threshold) needs n - l - 3 > 0, and opts->max_level;
    // the loop ends earlier once max degree - 1 < l, decided on the device
    int lmax = (int)std::min<int64_t>(n - 4, CUPC_MAX_LEVEL + 1);
    if (o.max_level >= 0) lmax = std::min(lmax, o.max_level);
    bool range_stop = false;
    if (lmax > CUPC_MAX_LEVEL) {
        lmax = CUPC_MAX_LEVEL;
        range_stop = true;  // an error unless the loop terminates by itself before
    }
    const int chunk = o.chunk ? o.chunk : 32;
    // Level buffers are sized without waiting for level 0: the context keeps the
    // largest needs of its earlier calls (defaults on the first); a level that would
    // overflow one reports it and the levels run again with room.
    const unsigned long long all_slots = (unsigned long long)p * (unsigned long long)(p - 1);
    unsigned long long nnz_cap = std::min<unsigned long long>(
        all_slots, std::max<unsigned long long>({ctx->cap_nnz, 64ull * p, 1ull << 21}));
    if (o.test_nnz_cap > 0) nnz_cap = std::min<unsigned long long>(all_slots, (unsigned long long)o.test_nnz_cap);
    nnz_cap = std::max<unsigned long long>(nnz_cap, 1);
    const unsigned long long item_cap = 1ull << 22;
    size_t rec_len_cap =
        16 + (ctx->cap_rec ? std::max<size_t>(ctx->cap_rec, (size_t)1 << 16)
                           : std::min<size_t>((size_t)(3 + std::max(lmax, 0)) * (nnz_cap / 2), (size_t)1 << 22));
    const size_t base_rec = ck ? (size_t)ck->rec_ints : 0;   // records of the checkpoint's levels
    rec_len_cap += base_rec;
    if (o.test_rec_cap > 0) rec_len_cap = base_rec + (size_t)o.test_rec_cap;
    LevelMeta* lm = nullptr;
    LevelParams LP{};
    int levels_run = 1;
    int last_launched = 0;
    int host_stop = 0;   // first level the host saw could not run (not launched)
    Meta M{};
    for (int attempt = 0;; ++attempt) {
        if (attempt > 6) return fail(ctx, CUPC_E_RANGE, "level buffers keep overflowing");
        // level 0's counters (the error flags of the preparation stay)
        CU(cudaMemsetAsync(meta, 0, offsetof(Meta, error), ctx->stream));
        if (ck) {
            // resume: A_G after the checkpoint's last level and after level 0
            CU(cudaMemcpyAsync(R->bits, in.ck_bits, bitbytes, cudaMemcpyHostToDevice, ctx->stream));
            CU(cudaMemcpyAsync(R->bits0, in.ck_bits0, bitbytes, cudaMemcpyHostToDevice, ctx->stream));
            ctx->h2d += 2 * bitbytes;
        } else {
            const double r0 = std::tanh(fisher_tau(alpha, n, 0));
            TIMED(CUPC_K_LEVEL0, launch_level0(fp32, Cuse, p, W, r0, kBand0, R->bits, (QEntry*)ctx->queue.p, qcap,
                                               meta, ctx->stream));
            if (fp32) TIMED(CUPC_K_LEVEL0, launch_recheck0(recheck0_params(), grid_wide, ctx->stream));
            CU(cudaMemcpyAsync(R->bits0, R->bits, bitbytes, cudaMemcpyDeviceToDevice, ctx->stream));
        }
        if ((s = ensure(ctx, ctx->deg, (size_t)p * 4)) != CUPC_OK) return s;
        TIMED(CUPC_K_COMPACT, launch_degree(R->bits, p, W, (int*)ctx->deg.p, meta, ctx->stream));
        last_launched = 0;
        levels_run = from;
        if (lmax >= from) {
            if ((s = ensure(ctx, ctx->row_off, (size_t)(p + 1) * 8)) != CUPC_OK) return s;
            if ((s = ensure(ctx, ctx->item_off, (size_t)(p + 1) * 8)) != CUPC_OK) return s;
            if ((s = ensure(ctx, ctx->cols, (size_t)nnz_cap * 4)) != CUPC_OK) return s;
            if ((s = ensure(ctx, ctx->srow, (size_t)nnz_cap * 4)) != CUPC_OK) return s;
            if ((s = ensure(ctx, ctx->partner, (size_t)nnz_cap * 4)) != CUPC_OK) return s;
            if ((s = ensure(ctx, ctx->wpre, bitbytes)) != CUPC_OK) return s;
            if ((s = ensure(ctx, ctx->best, (size_t)nnz_cap * 8)) != CUPC_OK) return s;
            // the second A'_G buffer, the per-slot survival flags and positions
            if ((s = ensure(ctx, *ctx_buf(ctx, "row_off2"), (size_t)(p + 1) * 8)) != CUPC_OK) return s;
            if ((s = ensure(ctx, *ctx_buf(ctx, "cols2"), (size_t)nnz_cap * 4)) != CUPC_OK) return s;
            if ((s = ensure(ctx, *ctx_buf(ctx, "srow2"), (size_t)nnz_cap * 4)) != CUPC_OK) return s;
            if ((s = ensure(ctx, *ctx_buf(ctx, "partner2"), (size_t)nnz_cap * 4)) != CUPC_OK) return s;
            if ((s = ensure(ctx, *ctx_buf(ctx, "alive"), (size_t)nnz_cap)) != CUPC_OK) return s;
            if ((s = ensure(ctx, *ctx_buf(ctx, "nrank"), (size_t)nnz_cap * 4)) != CUPC_OK) return s;
            // level 1 by conditioning variable when a C row fits the staging buffer
            const size_t ce = fp32 ? 4 : 8;
            const int l1_pivot = level1_by_pivot(o.level1_form) ? l1_buffers(p, (int)ce) : 0;
            if (l1_pivot && (s = ensure(ctx, *ctx_buf(ctx, "cval"), (size_t)nnz_cap * ce)) != CUPC_OK) return s;
            if ((s = ensure(ctx, ctx->item_row, (size_t)item_cap * 4)) != CUPC_OK) return s;
            if ((s = ensure(ctx, *ctx_buf(ctx, "item_c"), (size_t)item_cap * 4)) != CUPC_OK) return s;
            if ((s = ensure_binom(ctx, p + 2)) != CUPC_OK) return s;
            if ((s = ensure(ctx, ctx->lmeta, sizeof(LevelMeta))) != CUPC_OK) return s;
            if ((s = ensure(ctx, *ctx_buf(ctx, "scan_part"), 4 * 1024 * sizeof(unsigned long long))) != CUPC_OK)
                return s;
            // recheck partials: batches of queued tests sized to this buffer per level
            if (fp32 && (s = ensure(ctx, ctx->part, kPartBytes)) != CUPC_OK) return s;
            if (R->rec) cudaFreeAsync(R->rec, ctx->stream);
            R->rec = nullptr;
            if ((s = dalloc(ctx, (void**)&R->rec, rec_len_cap * 4)) != CUPC_OK) return s;
            lm = (LevelMeta*)ctx->lmeta.p;
            CU(cudaMemsetAsync(lm, 0, sizeof(LevelMeta), ctx->stream));
            if (base_rec) {
                // the checkpoint's records come first; the levels append after them
                CU(cudaMemcpyAsync(R->rec, in.ck_rec, base_rec * 4, cudaMemcpyHostToDevice, ctx->stream));
                ctx->h2d += base_rec * 4;
                ctx->hlmeta->rec_ints = base_rec;
                CU(cudaMemcpyAsync(&lm->rec_ints, &ctx->hlmeta->rec_ints, sizeof(unsigned long long),
                                   cudaMemcpyHostToDevice, ctx->stream));
                CU(cudaStreamSynchronize(ctx->stream));   // (the pinned staging word is reused below)
            }

            LP = LevelParams{};
            LP.bits = R->bits;
            LP.W = W;
            LP.p = p;
            LP.nwords = (long long)p * W;
            LP.ctas_per_sm = o.ctas_per_sm;
            LP.deg = (int*)ctx->deg.p;
            LP.row_off = (long long*)ctx->row_off.p;
            LP.item_off = (long long*)ctx->item_off.p;
            LP.item_row = (int*)ctx->item_row.p;
            LP.item_c = (int*)ctx_buf(ctx, "item_c")->p;
            LP.item_cap = item_cap;
            LP.cols = (int*)ctx->cols.p;
            LP.srow = (int*)ctx->srow.p;
            LP.partner = (int*)ctx->partner.p;
            LP.row_off2 = (long long*)ctx_buf(ctx, "row_off2")->p;
            LP.cols2 = (int*)ctx_buf(ctx, "cols2")->p;
            LP.srow2 = (int*)ctx_buf(ctx, "srow2")->p;
            LP.partner2 = (int*)ctx_buf(ctx, "partner2")->p;
            LP.alive = (unsigned char*)ctx_buf(ctx, "alive")->p;
            LP.nrank = (int*)ctx_buf(ctx, "nrank")->p;
            LP.wpre = (int*)ctx->wpre.p;
            LP.best = (unsigned long long*)ctx->best.p;
            LP.nnz_cap = nnz_cap;
            LP.C = Cuse;
            LP.l1_pivot = l1_pivot;
            LP.pstage = p;
            LP.cval = l1_pivot ? ctx_buf(ctx, "cval")->p : nullptr;
            LP.B = binom_view(ctx);
            LP.chunk0 = chunk;
            // level 1 of a graph with few rows: split each row's j positions too, so
            // the work items outnumber the warps and a hub row is not one long item
            LP.jsplit = (p <= 4096) ? 1 : 0;
            LP.canonical = o.canonical_sepset;
            LP.band_abs = (o.recheck_margin > 0) ? o.recheck_margin : kBandAbs;
            LP.band_rel = kBandRel;
            LP.rank_tol = fp32 ? kRankTol32 : kRankTol64;
            LP.piv_floor = kPivFloor;
            LP.xv = dv.xv;
            LP.ldx = dv.ldx;
            LP.xf64 = dv.xf64;
            LP.mu = dv.mu;
            LP.isd = dv.isd;
            LP.mup = dv.mup;
            LP.n = (int)n;
            LP.inv_n = 1.0 / (double)n;
            LP.c64 = c64;
            LP.part = fp32 ? (double*)ctx->part.p : nullptr;
            LP.part_cap = kPartBytes / sizeof(double);
            LP.rec = R->rec;
            LP.rec_cap = rec_len_cap;
            LP.lm = lm;
            LP.scan_part = (unsigned long long*)ctx_buf(ctx, "scan_part")->p;
            LP.meta0 = meta;
            LP.qcap0 = fp32 ? qcap : ~0ull;
            LP.learned = o.learned_order ? 1 : 0;
            LP.barrier_ns = 0;
            if (o.learned_order) {
                // each A'_G row's order and its inverse, one entry per slot; the
                // order positions of an incremental A'_G's survivors; the scores
                if ((s = ensure(ctx, *ctx_buf(ctx, "perm"), (size_t)nnz_cap * 4)) != CUPC_OK) return s;
                if ((s = ensure(ctx, *ctx_buf(ctx, "iperm"), (size_t)nnz_cap * 4)) != CUPC_OK) return s;
                if ((s = ensure(ctx, *ctx_buf(ctx, "vrank"), (size_t)nnz_cap * 4)) != CUPC_OK) return s;
                if ((s = ensure(ctx, *ctx_buf(ctx, "lscore"), (size_t)nnz_cap * 4)) != CUPC_OK) return s;
                if ((s = ensure(ctx, *ctx_buf(ctx, "lrsum"), (size_t)p * 4)) != CUPC_OK) return s;
                LP.perm = (int*)ctx_buf(ctx, "perm")->p;
                LP.iperm = (int*)ctx_buf(ctx, "iperm")->p;
                LP.vrank = (int*)ctx_buf(ctx, "vrank")->p;
                LP.lscore = (float*)ctx_buf(ctx, "lscore")->p;
                LP.lrsum = (float*)ctx_buf(ctx, "lrsum")->p;
                LP.mlp_w = ctx_buf(ctx, "mlp_Pb")->p;
            }
        }

        // Levels are launched with at most two in flight: level l is launched only
        // once level l - 2 has reported (through pinned host memory, right after
        // its termination test) that it runs, so at most two launches follow the
        // last level and they return at once. The report carries level l - 2's
        // starting max degree: degrees only fall, so level l (which needs a node
        // of degree >= l + 1) is not launched when that is below l + 1.
        auto launch_levels = [&](int from) -> cupc_status {
            host_stop = 0;
            LP.queue = (QEntry*)ctx->queue.p;
            if (fp32) {
                cupc_status sl = ensure(ctx, *ctx_buf(ctx, "live"), qcap * sizeof(int));
                if (sl != CUPC_OK) return sl;
                LP.live = (int*)ctx_buf(ctx, "live")->p;
                sl = ensure(ctx, *ctx_buf(ctx, "rc_cnt"), (size_t)kRcCnt * sizeof(int));
                if (sl != CUPC_OK) return sl;
                LP.rc_cnt = (int*)ctx_buf(ctx, "rc_cnt")->p;
            }
            LP.qcap = qcap;
            LP.host_flags = ctx->dflags;
            for (int q = 0; q < LV; ++q) ((volatile int*)ctx->hflags)[q] = 0;
            for (int l = from; l <= lmax; ++l) {
                if (cancelled()) return fail(ctx, CUPC_E_CANCELLED, "cancelled before level " + std::to_string(l));
                if (l - 2 >= from) {
                    volatile int* fl = (volatile int*)ctx->hflags + (l - 2);
                    const auto t0 = std::chrono::steady_clock::now();
                    while (*fl == 0) {
                        if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(30)) {
                            CU(cudaStreamSynchronize(ctx->stream));
                            if (*fl == 0) return fail(ctx, CUPC_E_TIMEOUT, "level flag not written");
                        }
                    }
                    const int fv = *fl;
                    if ((fv & 3) == 2) break;
                    if ((fv >> 4) - 1 < l) {
                        host_stop = l;
                        break;
                    }
                }
                LP.l = l;
                LP.barrier_ns = (l == from) ? barrier_ns : 0;   // (the expiry test: first level only)
                const double r = std::tanh(fisher_tau(alpha, n, l));
                LP.r = r;
                LP.r2 = r * r;
                if (l < CUPC_STATS_LEVELS) CU(cudaEventRecord(ctx->ev[1 + l], ctx->stream));
                LAUNCH(launch_level(fp32, LP, ctx->num_sms, ctx->stream));
                kcount[CUPC_K_CI]++;
                last_launched = l;
            }
            return CUPC_OK;
        };
        if (cancelled()) return fail(ctx, CUPC_E_CANCELLED, "cancelled after level 0");
        if (lmax >= from && (s = launch_levels(from)) != CUPC_OK) return s;

        // one readback: level 0's counters and, when levels ran, theirs; the
        // device work of the call ends with it (unless a level runs again)
        CU(cudaMemcpyAsync(ctx->hmeta, meta, sizeof(Meta), cudaMemcpyDeviceToHost, ctx->stream));
        ctx->d2h += sizeof(Meta);
        if (lmax >= from) {
            CU(cudaMemcpyAsync(ctx->hlmeta, lm, sizeof(LevelMeta), cudaMemcpyDeviceToHost, ctx->stream));
            ctx->d2h += sizeof(LevelMeta);
        }
        CU(cudaEventRecord(ctx->ev[kEvFin], ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        M = *ctx->hmeta;
        if (M.error & 4) return fail(ctx, CUPC_E_TIMEOUT, "a bounded wait in the tensor-core product expired");
        if (M.error) return fail(ctx, CUPC_E_NUMERIC, "a variable has zero variance or non-finite data");
        if (fp32 && M.queue_len > qcap) {
            // the level-0 recheck queue overflowed (the levels stopped at entry):
            // enlarge it and run level 0 again
            qcap = (size_t)(M.queue_len * 2);
            if ((s = ensure(ctx, ctx->queue, qcap * sizeof(QEntry))) != CUPC_OK) return s;
            ++reruns[0];
            continue;
        }
        if (lmax < from) break;
        bool rerun = false;
        for (int ov = 0;; ++ov) {
            LevelMeta& H = *ctx->hlmeta;
            if (H.error & 8) return fail(ctx, CUPC_E_TIMEOUT, "a grid barrier wait expired");
            if (H.range_error) return fail(ctx, CUPC_E_RANGE, "subset count exceeds 64 bits");
            unsigned long long nnz_need = 0;
            for (int q = 1; q < LV; ++q) nnz_need = std::max(nnz_need, 2 * H.edges[q]);
            if ((H.error & 16) || nnz_need > nnz_cap) {
                // CSR arrays too small for some level: room for every slot seen, and again
                nnz_cap = std::min<unsigned long long>(all_slots, nnz_need + nnz_need / 2 + 1024);
                rerun = true;
                ++reruns[1];
                break;
            }
            if (H.error) return fail(ctx, CUPC_E_RANGE, "level buffers too small");
            if (H.rec_ints > rec_len_cap) {
                rec_len_cap = (size_t)(H.rec_ints + H.rec_ints / 4 + 16);
                rerun = true;
                ++reruns[2];
                break;
            }
            const int ol = H.overflow_level;
            if (ol == 0) break;
            // the recheck queue of level ol overflowed: that level stopped before its
            // removals and the later ones at entry, so A_G and the degrees are as at
            // its start; enlarge the queue, clear the counters of the levels from ol
            // and run them again (level ol rebuilds A'_G from A_G)
            if (ov >= 4) return fail(ctx, CUPC_E_RANGE, "recheck queue overflow persists");
            qcap = (size_t)(H.queue_len[ol] * 2);
            if ((s = ensure(ctx, ctx->queue, qcap * sizeof(QEntry))) != CUPC_OK) return s;
            ++reruns[3];
            unsigned long long keep = base_rec;
            for (int q = from; q < ol; ++q) keep += H.removed[q] * (unsigned long long)(3 + q);
            for (int q = ol; q < LV; ++q) {
                H.tests[q] = H.rechecks[q] = H.removed[q] = H.serial[q] = H.edges[q] = H.items[q] = 0;
                H.next_item[q] = H.queue_len[q] = H.block_entries[q] = 0;
                for (int c = 0; c < 4; ++c) H.phase_ns[q][c] = 0;
                for (int c = 0; c < RND; ++c) H.round_hist[q][c] = H.round_cur[q][c] = 0;
                H.recheck_ns[q][0] = H.recheck_ns[q][1] = H.recheck_ns[q][2] = 0;
                H.order_ns[q][0] = H.order_ns[q][1] = 0;
                H.live[q] = 0;
                H.rc_next[q] = 0;
                H.maxdeg[q] = 0;
                H.chunk[q] = 0;
            }
            H.rec_ints = keep;
            H.overflow_level = 0;
            H.done_level = 0;
            H.csr_level = 0;
            H.bar = 0;
            CU(cudaMemcpyAsync(lm, ctx->hlmeta, sizeof(LevelMeta), cudaMemcpyHostToDevice, ctx->stream));
            if ((s = launch_levels(ol)) != CUPC_OK) return s;
            CU(cudaMemcpyAsync(ctx->hlmeta, lm, sizeof(LevelMeta), cudaMemcpyDeviceToHost, ctx->stream));
            CU(cudaEventRecord(ctx->ev[kEvFin], ctx->stream));
            CU(cudaStreamSynchronize(ctx->stream));
            ctx->d2h += sizeof(LevelMeta);
        }
        if (!rerun) break;
    }
    R->stats.rechecks[0] = (int64_t)M.rechecks;
    R->stats.rechecks_queued[0] = (int64_t)M.queue_len;
    for (int k = 0; k < 4; ++k) R->stats.reruns[k] = reruns[k];
    R->stats.removed[0] = pairs - (int64_t)(M.nnz / 2);
    if (ck) {
        // the checkpoint's levels keep their counters
        const cupc_stats& c = ck->stats;
        for (int q = 0; q < from && q < CUPC_STATS_LEVELS; ++q) {
            R->stats.tests[q] = c.tests[q];
            R->stats.serial_tests[q] = c.serial_tests[q];
            R->stats.removed[q] = c.removed[q];
            R->stats.rechecks[q] = c.rechecks[q];
            R->stats.edges_start[q] = c.edges_start[q];
            R->stats.max_degree[q] = c.max_degree[q];
            R->stats.ci_block_entries[q] = c.ci_block_entries[q];
            R->stats.rechecks_queued[q] = c.rechecks_queued[q];
        }
        R->rec_ints = (int64_t)base_rec;
    }
    if (lmax >= from) {
        const LevelMeta& H = *ctx->hlmeta;
        // last level that ran: the one before the level whose termination test
        // ended the loop, or before the level the host did not launch
        const int last = std::max(from - 1, H.done_level ? H.done_level - 1 : host_stop ? host_stop - 1 : lmax);
        if (range_stop && H.done_level == 0 && host_stop == 0)
            return fail(ctx, CUPC_E_RANGE, "a level above CUPC_MAX_LEVEL would be needed");
        levels_run = last + 1;
        for (int l = from; l <= last && l < CUPC_STATS_LEVELS; ++l) {
            R->stats.tests[l] = (int64_t)H.tests[l];
            R->stats.removed[l] = (int64_t)H.removed[l];
            R->stats.serial_tests[l] = o.canonical_sepset ? (int64_t)H.serial[l] : -1;
            R->stats.rechecks[l] = (int64_t)H.rechecks[l];
            R->stats.edges_start[l] = (int64_t)H.edges[l];
            R->stats.max_degree[l] = H.maxdeg[l];
            R->stats.ci_block_entries[l] = (int64_t)H.block_entries[l];
            for (int c = 0; c < 4; ++c) R->stats.phase_ms[l][c] = 1e-6f * (float)H.phase_ns[l][c];
            for (int c = 0; c < 3; ++c) R->stats.recheck_ms[l][c] = 1e-6f * (float)H.recheck_ns[l][c];
            for (int c = 0; c < 2; ++c) R->stats.order_ms[l][c] = 1e-6f * (float)H.order_ns[l][c];
            R->stats.rechecks_queued[l] = (int64_t)H.queue_len[l];
        }
        for (int l = 1; l < LV; ++l) {
            R->stats.kernel_ms[CUPC_K_COMPACT] += 1e-6f * (float)H.phase_ns[l][0];
            R->stats.kernel_ms[CUPC_K_CI] += 1e-6f * (float)H.phase_ns[l][1];
            R->stats.kernel_ms[CUPC_K_RECHECK] += 1e-6f * (float)H.phase_ns[l][2];
            R->stats.kernel_ms[CUPC_K_FINALIZE] += 1e-6f * (float)H.phase_ns[l][3];
        }
        R->rec_ints = (int64_t)H.rec_ints;
        // the needs the next call on this context is sized for
        unsigned long long nnz_need = 0;
        for (int q = 1; q < LV; ++q) nnz_need = std::max(nnz_need, 2 * H.edges[q]);
        ctx->cap_nnz = std::max<unsigned long long>(ctx->cap_nnz, nnz_need + nnz_need / 4);
        ctx->cap_rec = std::max<size_t>(ctx->cap_rec, (size_t)(H.rec_ints + H.rec_ints / 4));
    } else if (range_stop) {
        return fail(ctx, CUPC_E_RANGE, "a level above CUPC_MAX_LEVEL would be needed");
    }
    // host lists asked for with the call: built after the device work's end
    // event, taken after one more synchronisation
    ListsPending lists;
    if (o.host_lists && (size_t)R->rec_ints <= rec_len_cap) {
        R->stats.levels = levels_run;
        R->rec_cap = rec_len_cap;
        if ((s = lists_enqueue(R, true, true, lists)) != CUPC_OK) return s;
        if (lists.recs || lists.edges) CU(cudaStreamSynchronize(ctx->stream));
    }
    const auto h1 = std::chrono::steady_clock::now();
    R->rec_cap = rec_len_cap;
    if ((size_t)R->rec_ints > rec_len_cap && R->rec_ints > 0)
        return fail(ctx, CUPC_E_RANGE, "SepSet record pool overflow");
    lists_finish(R, lists);

    // statistics
    R->stats.levels = levels_run;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
    R->stats.prep_ms = ms;
    if (ck)
        for (int q = 0; q < from && q < CUPC_STATS_LEVELS; ++q) R->stats.level_ms[q] = ck->stats.level_ms[q];
    for (int q = ck ? from : 0; q < levels_run && q < CUPC_STATS_LEVELS; ++q) {
        // level 0 spans the sizing step; level q >= 1 its level kernel launch (the
        // last one up to the end of the device work)
        if (q > 0 && q > last_launched) break;
        const int a = 1 + q, b = (q + 1 <= last_launched) ? 2 + q : kEvFin;
        if (cudaEventElapsedTime(&ms, ctx->ev[a], ctx->ev[b]) == cudaSuccess) R->stats.level_ms[q] = ms;
    }
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[kEvFin]);
    R->stats.total_ms = ms;
    cudaGetLastError();
    int64_t edges_final = R->stats.edges_start[0] - R->stats.removed[0];
    for (int q = 1; q < levels_run && q < CUPC_STATS_LEVELS; ++q) edges_final -= R->stats.removed[q];
    R->stats.edges_final = edges_final;
    for (int q = levels_run; q < CUPC_STATS_LEVELS; ++q) R->stats.serial_tests[q] = 0;
    R->stats.kernel_launches = (int64_t)(ctx->launches - launches0);
    tcollect(ctx, R->stats);
    for (int c = 0; c < CUPC_KCLASSES; ++c) R->stats.kernel_count[c] = kcount[c];
    R->stats.h2d_bytes = (int64_t)(ctx->h2d - h2d0);
    R->stats.d2h_bytes = (int64_t)(ctx->d2h - d2h0);
    R->stats.host_ms[0] = std::chrono::duration<float, std::milli>(h1 - h0).count();
    R->stats.host_ms[1] = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - h1).count();
    guard.ok = true;
    *out = R;
    ctx->err.clear();
    return CUPC_OK;
}

void ctx_release(cupc_ctx* c)
{
    if (--c->refs > 0) return;
    cudaSetDevice(c->device);
    cupc_ctx* ctx = c;
    Buf* all[] = {&c->xin, &c->xt, &c->mu, &c->isd, &c->mup, &c->z64, &c->zhi, &c->zlo, &c->cws, &c->c64, &c->c32, &c->cin,
                  &c->deg, &c->row_off, &c->item_off, &c->item_row, &c->cols, &c->srow, &c->partner, &c->wpre,
                  &c->best, &c->queue, &c->binom, &c->meta, &c->lmeta,
                  &c->part};
    for (Buf* b : all) free_buf(ctx, *b);
    for (auto& kv : c->named) free_buf(ctx, kv.second);
    if (c->batch_free) c->batch_free(c);
    cudaStreamSynchronize(c->stream);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    for (cudaEvent_t e : c->tev) cudaEventDestroy(e);
    if (c->hmeta) cudaFreeHost(c->hmeta);
    if (c->hlmeta) cudaFreeHost(c->hlmeta);
    if (c->hflags) cudaFreeHost(c->hflags);
    if (c->hstage) cudaFreeHost(c->hstage);
    for (cudaEvent_t e : c->cev)
        if (e) cudaEventDestroy(e);
    if (c->cstream) cudaStreamDestroy(c->cstream);
    if (c->pool) cudaMemPoolDestroy(c->pool);
    delete c;
}

// Index (i p + j) -> offset of the sorted host records, for single lookups.
void build_index(const cupc_result* r)
{
    if (r->index_ready) return;
    r->index.clear();
    for (size_t k = 0; k + 2 < r->hrec.size(); k += 3 + (size_t)r->hrec[k + 2])
        r->index.emplace_back((uint64_t)r->hrec[k] * (uint64_t)r->p + (uint64_t)r->hrec[k + 1], (int64_t)k);
    r->index_ready = true;
}

cupc_status build_host_records(const cupc_result* r)
{
    if (r->host_ready) return CUPC_OK;
    if (!r->on_host && r->rec_ints > 0) {
        const cupc_status s = device_lists(r, true, false);
        if (s != CUPC_OK) return s;
        if (r->host_ready) return CUPC_OK;
    }
    // host sort: results the device path does not cover (an empty pool, or
    // level counts that do not match the pool)
    std::vector<int32_t> raw((size_t)r->rec_ints);
    if (r->rec_ints) {
        cudaError_t e = cudaMemcpyAsync(raw.data(), r->rec, (size_t)r->rec_ints * 4, cudaMemcpyDeviceToHost,
                                        r->ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(r->ctx->stream);
        if (e != cudaSuccess) return CUPC_E_CUDA;
        r->ctx->d2h += (size_t)r->rec_ints * 4;
    }
    // records in (i, j) order: a least-significant-digit radix sort of the
    // record offsets, a stable counting sort on j and then on i
    const int64_t p = r->p;
    std::vector<int64_t> offs;
    offs.reserve((size_t)(r->rec_ints / 4 + 1));
    for (int64_t k = 0; k < r->rec_ints; k += 3 + raw[k + 2]) {
        if (k + 2 >= r->rec_ints || raw[k] < 0 || raw[k] >= p || raw[k + 1] < 0 || raw[k + 1] >= p ||
            raw[k + 2] < 1 || raw[k + 2] > CUPC_MAX_LEVEL || k + 3 + raw[k + 2] > r->rec_ints)
            return CUPC_E_STATE;
        offs.push_back(k);
    }
    const size_t m = offs.size();
    std::vector<int64_t> cnt((size_t)p + 1), tmp(m), ord(m);
    auto pass = [&](const std::vector<int64_t>& in, std::vector<int64_t>& out, int field) {
        std::fill(cnt.begin(), cnt.end(), 0);
        for (const int64_t k : in) ++cnt[(size_t)raw[k + field] + 1];
        for (int64_t i = 0; i < p; ++i) cnt[(size_t)i + 1] += cnt[(size_t)i];
        for (const int64_t k : in) out[(size_t)cnt[(size_t)raw[k + field]]++] = k;
    };
    pass(offs, tmp, 1);   // by j
    pass(tmp, ord, 0);    // by i, stable
    r->hrec.resize((size_t)r->rec_ints);
    r->index.resize(m);
    int64_t w = 0;
    for (size_t q = 0; q < m; ++q) {
        const int64_t k = ord[q];
        const int ints = 3 + raw[k + 2];
        r->index[q] = std::make_pair((uint64_t)raw[k] * (uint64_t)p + (uint64_t)raw[k + 1], w);
        std::memcpy(r->hrec.data() + w, raw.data() + k, (size_t)ints * 4);
        w += ints;
    }
    r->host_ready = true;
    r->index_ready = true;
    return CUPC_OK;
}

}  // namespace

// A'_G at the start of `level` >= 1 as neighbour lists (increasing): the
// result's skeleton plus the pairs its records remove at that level or later.
cupc_status result_frozen_lists(const cupc_result* r, int level, std::vector<long long>& off, std::vector<int>& cols)
{
    const size_t words = (size_t)r->p * r->W;
    std::vector<unsigned> hd;
    if (!r->on_host) {
        hd.resize(words);
        cudaError_t e = cudaMemcpyAsync(hd.data(), r->bits, words * 4, cudaMemcpyDeviceToHost, r->ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(r->ctx->stream);
        if (e != cudaSuccess) return fail(r->ctx, CUPC_E_CUDA, "skeleton download", e);
    }
    const std::vector<unsigned>& h = r->on_host ? r->hbits : hd;
    cupc_status s = build_host_records(r);
    if (s != CUPC_OK) return fail(r->ctx, s, "record download");
    const int64_t p = r->p;
    std::vector<std::vector<int>> nb((size_t)p);
    for (int64_t i = 0; i < p; ++i)
        for (int w = 0; w < r->W; ++w) {
            unsigned m = h[(size_t)i * r->W + w];
            while (m) {
                const int64_t j = (int64_t)w * 32 + __builtin_ctz(m);
                m &= m - 1;
                if (j < p && j != i) nb[(size_t)i].push_back((int)j);
            }
        }
    for (size_t k = 0; k < r->hrec.size();) {
        const int i = r->hrec[k], j = r->hrec[k + 1], l = r->hrec[k + 2];
        if (l >= level) {
            nb[(size_t)i].push_back(j);
            nb[(size_t)j].push_back(i);
        }
        k += 3 + (size_t)l;
    }
    off.assign((size_t)p + 1, 0);
    cols.clear();
    for (int64_t i = 0; i < p; ++i) {
        std::sort(nb[(size_t)i].begin(), nb[(size_t)i].end());
        off[(size_t)i + 1] = off[(size_t)i] + (long long)nb[(size_t)i].size();
        cols.insert(cols.end(), nb[(size_t)i].begin(), nb[(size_t)i].end());
    }
    return CUPC_OK;
}

cupc_status ctx_ensure(cupc_ctx* ctx, Buf* b, size_t bytes) { return ensure(ctx, *b, bytes); }
cupc_status ctx_host_stage(cupc_ctx* ctx, size_t bytes, char** out) { return host_stage(ctx, bytes, out); }
void ctx_free(cupc_ctx* ctx, Buf* b) { free_buf(ctx, *b); }
double ctx_fisher_tau(double alpha, int64_t n, int l) { return fisher_tau(alpha, n, l); }
cupc_status ctx_binom(cupc_ctx* ctx, int m_needed, Binom* out)
{
    cupc_status s = ensure_binom(ctx, m_needed);
    if (s == CUPC_OK) *out = binom_view(ctx);
    return s;
}
cupc_status ctx_validate(cupc_ctx* ctx, const cupc_options& o) { return validate_opts(ctx, o); }
Buf* ctx_buf(cupc_ctx* ctx, const char* name) { return &ctx->named[name]; }
int ctx_num_sms(cupc_ctx* ctx) { return ctx->num_sms; }
cudaStream_t ctx_stream(cupc_ctx* ctx) { return ctx->stream; }
cupc_status ctx_fail(cupc_ctx* ctx, cupc_status s, const std::string& what, cudaError_t e)
{
    return fail(ctx, s, what, e);
}
void ctx_count_launch(cupc_ctx* ctx) { ctx->launches++; }
void ctx_set_mlp(cupc_ctx* ctx, int ready, int step)
{
    ctx->mlp_ready = ready;
    ctx->mlp_step = step;
}
int ctx_mlp_ready(cupc_ctx* ctx) { return ctx->mlp_ready; }
int ctx_mlp_step(cupc_ctx* ctx) { return ctx->mlp_step; }

// =============================================================================
// C ABI
// =============================================================================
extern "C" {

void cupc_options_default(cupc_options* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->mode = CUPC_MODE_FP32_RECHECK;
    o->canonical_sepset = 1;
    o->learned_order = 0;
    o->max_level = -1;
    o->recheck_margin = 0.0;
}

cupc_status cupc_create(cupc_ctx** out, int device, void* stream)
{
    if (!out) return CUPC_E_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return CUPC_E_CUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return CUPC_E_CUDA;
    if (prop.major != 10 || prop.minor != 3) return CUPC_E_CUDA;  // built for sm_103a only
    if (cudaSetDevice(device) != cudaSuccess) return CUPC_E_CUDA;
    cupc_ctx* c = new cupc_ctx();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    c->num_sms = prop.multiProcessorCount;
    cudaMemPoolProps pp{};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = device;
    if (cudaMemPoolCreate(&c->pool, &pp) != cudaSuccess) {
        delete c;
        return CUPC_E_CUDA;
    }
    unsigned long long thr = ~0ull;
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    if (cudaHostAlloc((void**)&c->hmeta, sizeof(Meta), cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void**)&c->hlmeta, sizeof(LevelMeta), cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void**)&c->hflags, sizeof(int) * LV, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&c->dflags, c->hflags, 0) != cudaSuccess) {
        cudaMemPoolDestroy(c->pool);
        delete c;
        return CUPC_E_CUDA;
    }
    c->ev.resize(CUPC_STATS_LEVELS + 4);
    for (auto& e : c->ev) cudaEventCreate(&e);
    c->tev.resize(512);
    c->tcls.resize(256);
    for (auto& e : c->tev) cudaEventCreate(&e);
    *out = c;
    return CUPC_OK;
}

cupc_status cupc_cancel(cupc_ctx* ctx)
{
    if (!ctx) return CUPC_E_INVALID;
    ctx->cancel.store(1);
    return CUPC_OK;
}

cupc_status cupc_debug_fail(cupc_ctx* ctx, int kind, int64_t k)
{
    if (!ctx) return CUPC_E_INVALID;
    if (kind == CUPC_FAIL_NONE) {
        ctx->fail_kind = 0;
        ctx->barrier_ns = 0;
        return CUPC_OK;
    }
    if (kind == CUPC_FAIL_BARRIER) {
        if (k < 1000 || k > 1000000000) return fail(ctx, CUPC_E_INVALID, "barrier limit in ns must be in [1e3, 1e9]");
        ctx->barrier_ns = (unsigned)k;
        return CUPC_OK;
    }
    if ((kind != CUPC_FAIL_ALLOC && kind != CUPC_FAIL_LAUNCH) || k < 1)
        return fail(ctx, CUPC_E_INVALID, "unknown failure kind or k < 1");
    ctx->fail_kind = kind;
    ctx->fail_k = k;
    return CUPC_OK;
}

cupc_status cupc_set_stream(cupc_ctx* ctx, void* stream)
{
    if (!ctx) return CUPC_E_INVALID;
    ctx->stream = (cudaStream_t)stream;
    return CUPC_OK;
}

void cupc_destroy(cupc_ctx* ctx)
{
    if (ctx) ctx_release(ctx);
}

const char* cupc_last_error(const cupc_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : "null context";
}

cupc_status cupc_skeleton(cupc_ctx* ctx, const void* X, int dtype, int layout, int on_device, int64_t n_samples,
                          int64_t p, int64_t ld, double alpha, const cupc_options* opts, cupc_result** out)
{
    if (!ctx) return CUPC_E_INVALID;
    Input in;
    in.X = X;
    in.dtype = dtype;
    in.layout = layout;
    in.on_device = on_device;
    in.n = n_samples;
    in.p = p;
    in.ld = ld;
    return run(ctx, in, alpha, opts, out);
}

cupc_status cupc_skeleton_corr(cupc_ctx* ctx, const void* C, int dtype, int on_device, int64_t p, int64_t ld,
                               int64_t n_samples, double alpha, const cupc_options* opts, cupc_result** out)
{
    if (!ctx) return CUPC_E_INVALID;
    Input in;
    in.is_corr = true;
    in.X = C;
    in.dtype = dtype;
    in.on_device = on_device;
    in.n = n_samples;
    in.p = p;
    in.ld = ld;
    return run(ctx, in, alpha, opts, out);
}

cupc_status cupc_result_p(const cupc_result* r, int64_t* p)
{
    if (!r || !p) return CUPC_E_INVALID;
    *p = r->p;
    return CUPC_OK;
}

cupc_status cupc_result_adjacency(const cupc_result* r, uint8_t* out)
{
    if (!r || !out) return CUPC_E_INVALID;
    cupc_ctx* ctx = r->ctx;
    const size_t bytes = (size_t)r->p * r->W * 4;
    std::vector<unsigned> hd;
    if (!r->on_host) {
        hd.resize(bytes / 4);
        CU(cudaMemcpyAsync(hd.data(), r->bits, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        ctx->d2h += bytes;
    }
    const std::vector<unsigned>& h = r->on_host ? r->hbits : hd;
    const int64_t p = r->p;
    // eight columns at a time: byte b of a row's bits -> its eight 0/1 bytes
    static const auto table = [] {
        std::vector<uint8_t> t(256 * 8);
        for (int b = 0; b < 256; ++b)
            for (int k = 0; k < 8; ++k) t[(size_t)b * 8 + k] = (uint8_t)((b >> k) & 1);
        return t;
    }();
    for (int64_t i = 0; i < p; ++i) {
        const unsigned* row = h.data() + i * r->W;
        uint8_t* o = out + i * p;
        int64_t j = 0;
        for (; j + 8 <= p; j += 8) std::memcpy(o + j, &table[(size_t)((row[j >> 5] >> (j & 31)) & 0xffu) * 8], 8);
        if (j < p) std::memcpy(o + j, &table[(size_t)((row[j >> 5] >> (j & 31)) & 0xffu) * 8], (size_t)(p - j));
    }
    return CUPC_OK;
}

cupc_status cupc_result_edges(const cupc_result* r, int32_t* out, int64_t cap, int64_t* n_edges)
{
    if (!r || !n_edges) return CUPC_E_INVALID;
    cupc_ctx* ctx = r->ctx;
    if (!r->edges_ready && !r->on_host) {
        const cupc_status s = device_lists(r, false, true);
        if (s != CUPC_OK) return s;
    }
    if (!r->edges_ready) {
        const size_t bytes = (size_t)r->p * r->W * 4;
        std::vector<unsigned> hd;
        if (!r->on_host) {
            hd.resize(bytes / 4);
            CU(cudaMemcpyAsync(hd.data(), r->bits, bytes, cudaMemcpyDeviceToHost, ctx->stream));
            CU(cudaStreamSynchronize(ctx->stream));
            ctx->d2h += bytes;
        }
        const std::vector<unsigned>& h = r->on_host ? r->hbits : hd;
        const int64_t p = r->p;
        const int W = r->W;
        r->hedges.clear();
        for (int64_t i = 0; i < p; ++i) {
            const unsigned* row = h.data() + i * W;
            const int w0 = (int)((i + 1) >> 5);
            for (int w = w0; w < W; ++w) {
                unsigned m = row[w];
                if (w == w0) m &= ~0u << ((i + 1) & 31);   // columns j > i only
                while (m) {
                    const int64_t j = (int64_t)w * 32 + __builtin_ctz(m);
                    m &= m - 1;
                    if (j >= p) break;
                    r->hedges.push_back((int32_t)i);
                    r->hedges.push_back((int32_t)j);
                }
            }
        }
        r->edges_ready = true;
    }
    *n_edges = (int64_t)(r->hedges.size() / 2);
    if (out) std::memcpy(out, r->hedges.data(), (size_t)std::min<int64_t>(cap, *n_edges) * 2 * 4);
    return CUPC_OK;
}

cupc_status cupc_result_sep_levels(const cupc_result* r, int16_t* out)
{
    if (!r || !out) return CUPC_E_INVALID;
    cupc_ctx* ctx = r->ctx;
    const size_t bytes = (size_t)r->p * r->W * 4;
    std::vector<unsigned> hd;
    if (!r->on_host) {
        hd.resize(bytes / 4);
        CU(cudaMemcpyAsync(hd.data(), r->bits0, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        ctx->d2h += bytes;
    }
    const std::vector<unsigned>& h0 = r->on_host ? r->hbits0 : hd;
    cupc_status s = build_host_records(r);
    if (s != CUPC_OK) return fail(ctx, s, "record download");
    const int64_t p = r->p;
    for (int64_t i = 0; i < p; ++i)
        for (int64_t j = 0; j < p; ++j) {
            const bool after0 = (h0[i * r->W + (j >> 5)] >> (j & 31)) & 1u;
            out[i * p + j] = (i == j) ? -1 : (after0 ? -1 : 0);
        }
    for (size_t k = 0; k < r->hrec.size();) {
        const int i = r->hrec[k], j = r->hrec[k + 1], l = r->hrec[k + 2];
        out[(int64_t)i * p + j] = (int16_t)l;
        out[(int64_t)j * p + i] = (int16_t)l;
        k += 3 + l;
    }
    return CUPC_OK;
}

cupc_status cupc_result_sepset(const cupc_result* r, int64_t i, int64_t j, int32_t* out, int* len)
{
    if (!r || !out || !len) return CUPC_E_INVALID;
    if (i < 0 || j < 0 || i >= r->p || j >= r->p || i == j) return CUPC_E_INVALID;
    cupc_ctx* ctx = r->ctx;
    cupc_status s = build_host_records(r);
    if (s != CUPC_OK) return fail(ctx, s, "record download");
    build_index(r);
    const int64_t a = std::min(i, j), b = std::max(i, j);
    const uint64_t key = (uint64_t)a * (uint64_t)r->p + (uint64_t)b;
    auto it = std::lower_bound(r->index.begin(), r->index.end(), std::make_pair(key, (int64_t)-1));
    if (it != r->index.end() && it->first == key) {
        const int l = r->hrec[it->second + 2];
        for (int c = 0; c < l; ++c) out[c] = r->hrec[it->second + 3 + c];
        *len = l;
        return CUPC_OK;
    }
    // not a level >= 1 removal: present, or removed at level 0
    unsigned w0 = 0;
    if (r->on_host) w0 = r->hbits0[(size_t)a * r->W + (b >> 5)];
    else CU(cudaMemcpy(&w0, r->bits0 + a * r->W + (b >> 5), 4, cudaMemcpyDeviceToHost));
    *len = ((w0 >> (b & 31)) & 1u) ? -1 : 0;
    return CUPC_OK;
}

cupc_status cupc_result_sepset_records(const cupc_result* r, int32_t* out, int64_t cap, int64_t* n_ints)
{
    if (!r || !n_ints) return CUPC_E_INVALID;
    cupc_status s = build_host_records(r);
    if (s != CUPC_OK) return fail(r->ctx, s, "record download");
    *n_ints = (int64_t)r->hrec.size();
    if (out) std::memcpy(out, r->hrec.data(), (size_t)std::min<int64_t>(cap, *n_ints) * 4);
    return CUPC_OK;
}

cupc_status cupc_result_checkpoint(const cupc_result* r, void* buf, int64_t cap, int64_t* size)
{
    if (!r || !size) return CUPC_E_INVALID;
    if (r->on_host || !r->bits || !r->bits0) return fail(r->ctx, CUPC_E_STATE, "not a single-problem result");
    const size_t words = (size_t)r->p * r->W;
    const size_t total = sizeof(CkptHeader) + 2 * words * 4 + (size_t)r->rec_ints * 4;
    *size = (int64_t)total;
    if (!buf) return CUPC_OK;
    if (cap < (int64_t)total) return fail(r->ctx, CUPC_E_RANGE, "checkpoint buffer too small");
    cupc_ctx* ctx = r->ctx;
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = 1;
    h.level = r->stats.levels - 1;
    h.p = r->p;
    h.n = r->n;
    h.alpha = r->alpha;
    h.mode = r->mode;
    h.canonical = r->canonical;
    h.learned = r->learned;
    h.W = r->W;
    h.rec_ints = r->rec_ints;
    h.stats = r->stats;
    unsigned char* o = (unsigned char*)buf;
    std::memcpy(o, &h, sizeof(h));
    CU(cudaMemcpyAsync(o + sizeof(h), r->bits, words * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(o + sizeof(h) + words * 4, r->bits0, words * 4, cudaMemcpyDeviceToHost, ctx->stream));
    if (r->rec_ints)
        CU(cudaMemcpyAsync(o + sizeof(h) + 2 * words * 4, r->rec, (size_t)r->rec_ints * 4, cudaMemcpyDeviceToHost,
                           ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->d2h += total - sizeof(h);
    return CUPC_OK;
}

cupc_status cupc_skeleton_resume(cupc_ctx* ctx, const void* X, int dtype, int layout, int on_device, int64_t n_samples,
                                 int64_t p, int64_t ld, double alpha, const cupc_options* opts, const void* ckpt,
                                 int64_t ckpt_size, cupc_result** out)
{
    if (!ctx) return CUPC_E_INVALID;
    if (out) *out = nullptr;
    if (!ckpt || ckpt_size < (int64_t)sizeof(CkptHeader)) return fail(ctx, CUPC_E_INVALID, "checkpoint too short");
    CkptHeader h;
    std::memcpy(&h, ckpt, sizeof(h));
    if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 1)
        return fail(ctx, CUPC_E_INVALID, "not a checkpoint of this library");
    if (h.p < 2 || h.p > (1 << 20) || h.W != (int)((h.p + 31) / 32) || h.level < 0 ||
        h.level >= CUPC_STATS_LEVELS - 1 || h.level > CUPC_MAX_LEVEL || h.rec_ints < 0)
        return fail(ctx, CUPC_E_INVALID, "checkpoint header out of range");
    const size_t words = (size_t)h.p * h.W;
    if ((uint64_t)ckpt_size != sizeof(h) + 2 * words * 4 + (uint64_t)h.rec_ints * 4)
        return fail(ctx, CUPC_E_INVALID, "checkpoint size does not match its header");
    const unsigned char* b = (const unsigned char*)ckpt;
    Input in;
    in.X = X;
    in.dtype = dtype;
    in.layout = layout;
    in.on_device = on_device;
    in.n = n_samples;
    in.p = p;
    in.ld = ld;
    in.ck = &h;
    in.ck_bits = (const unsigned*)(b + sizeof(h));
    in.ck_bits0 = (const unsigned*)(b + sizeof(h) + words * 4);
    in.ck_rec = (const int32_t*)(b + sizeof(h) + 2 * words * 4);
    return run(ctx, in, alpha, opts, out);
}

cupc_status cupc_result_stats(const cupc_result* r, cupc_stats* out)
{
    if (!r || !out) return CUPC_E_INVALID;
    *out = r->stats;
    return CUPC_OK;
}

void cupc_result_free(cupc_result* r) { free_result(r); }

cupc_status cupc_correlation(cupc_ctx* ctx, const void* X, int dtype, int layout, int on_device, int64_t n_samples,
                             int64_t p, int64_t ld, int precision, void* C_out)
{
    if (!ctx || !X || !C_out) return CUPC_E_INVALID;
    if (p < 1 || n_samples < 2) return fail(ctx, CUPC_E_INVALID, "sizes");
    CU(cudaSetDevice(ctx->device));
    cupc_status s = ensure(ctx, ctx->meta, sizeof(Meta));
    if (s != CUPC_OK) return s;
    CU(cudaMemsetAsync(ctx->meta.p, 0, sizeof(Meta), ctx->stream));
    Input in;
    in.X = X;
    in.dtype = dtype;
    in.layout = layout;
    in.on_device = on_device;
    in.n = n_samples;
    in.p = p;
    in.ld = ld;
    const void* Cuse = nullptr;
    const double* c64 = nullptr;
    DataView dv;
    const bool fp32 = (precision == CUPC_F32);
    int kcount[CUPC_KCLASSES] = {0};
    ctx->tused = 0;
    if ((s = prepare(ctx, in, fp32, &Cuse, &c64, &dv, kcount)) != CUPC_OK) return s;
    CU(cudaMemcpyAsync(C_out, Cuse, (size_t)p * p * (fp32 ? 4 : 8), cudaMemcpyDeviceToDevice, ctx->stream));
    if ((s = readback(ctx)) != CUPC_OK) return s;
    if (ctx->hmeta->error & 4) return fail(ctx, CUPC_E_TIMEOUT, "a bounded wait in the tensor-core product expired");
    if (ctx->hmeta->error) return fail(ctx, CUPC_E_NUMERIC, "a variable has zero variance or non-finite data");
    return CUPC_OK;
}

cupc_status cupc_pcor_batch(cupc_ctx* ctx, const void* C, int dtype, int64_t p, const int32_t* queries, int64_t nq,
                            int l, double* rho_out)
{
    if (!ctx || !C || !queries || !rho_out) return CUPC_E_INVALID;
    if (l < 0 || l > CUPC_MAX_LEVEL) return fail(ctx, CUPC_E_RANGE, "l out of range");
    CU(cudaSetDevice(ctx->device));
    LAUNCH(launch_pcor(dtype == CUPC_F32, C, (int)p, queries, nq, l, rho_out, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return CUPC_OK;
}

cupc_status cupc_pcor_data(cupc_ctx* ctx, const void* X, int dtype, int layout, int on_device, int64_t n_samples,
                           int64_t p, int64_t ld, const int32_t* queries, int64_t nq, int l, double* rho_out)
{
    if (!ctx || !X || !queries || !rho_out) return CUPC_E_INVALID;
    if (l < 0 || l > CUPC_MAX_LEVEL) return fail(ctx, CUPC_E_RANGE, "l out of range");
    if (p < 2 || n_samples < 4 || nq < 0) return fail(ctx, CUPC_E_INVALID, "sizes");
    if (dtype != CUPC_F32 && dtype != CUPC_F64) return fail(ctx, CUPC_E_INVALID, "dtype");
    if (layout != CUPC_LAYOUT_SAMPLE_MAJOR && layout != CUPC_LAYOUT_VARIABLE_MAJOR)
        return fail(ctx, CUPC_E_INVALID, "layout");
    if (ld < (layout == CUPC_LAYOUT_SAMPLE_MAJOR ? p : n_samples)) return fail(ctx, CUPC_E_INVALID, "ld");
    CU(cudaSetDevice(ctx->device));
    cupc_status s = ensure(ctx, ctx->meta, sizeof(Meta));
    if (s != CUPC_OK) return s;
    CU(cudaMemsetAsync(ctx->meta.p, 0, sizeof(Meta), ctx->stream));
    Input in;
    in.X = X;
    in.dtype = dtype;
    in.layout = layout;
    in.on_device = on_device;
    in.n = n_samples;
    in.p = p;
    in.ld = ld;
    const void* Cuse = nullptr;
    const double* c64 = nullptr;
    DataView dv;
    int kcount[CUPC_KCLASSES] = {0};
    ctx->tused = 0;
    // the moments and data rows the FP32 form's rechecks read
    if ((s = prepare(ctx, in, true, &Cuse, &c64, &dv, kcount)) != CUPC_OK) return s;
    LevelParams P{};
    P.l = l;
    P.p = (int)p;
    P.xv = dv.xv;
    P.ldx = dv.ldx;
    P.xf64 = dv.xf64;
    P.mu = dv.mu;
    P.isd = dv.isd;
    P.mup = dv.mup;
    P.n = (int)n_samples;
    P.inv_n = 1.0 / (double)n_samples;
    P.rank_tol = kRankTol32;
    LAUNCH(launch_pcor_recheck(P, queries, nq, rho_out, ctx->stream));
    if ((s = readback(ctx)) != CUPC_OK) return s;
    if (ctx->hmeta->error) return fail(ctx, CUPC_E_NUMERIC, "a variable has zero variance or non-finite data");
    return CUPC_OK;
}

cupc_status cupc_fisher_threshold(double alpha, int64_t n_samples, int l, double* tau, double* r)
{
    if (!(alpha > 0.0 && alpha < 1.0) || n_samples - l - 3 <= 0) return CUPC_E_INVALID;
    const double t = fisher_tau(alpha, n_samples, l);
    if (tau) *tau = t;
    if (r) *r = std::tanh(t);
    return CUPC_OK;
}

}  // extern "C"
