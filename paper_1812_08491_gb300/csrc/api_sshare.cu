// api_sshare.cu -- cupc_result_sshare: the global-sharing diagnostic of
// Sec. 5.5 (Fig. 9) on a result's frozen A'_G at one level.
#include <algorithm>
#include <cstring>
#include <vector>

#include "api_internal.h"

using namespace cupc;

extern "C" cupc_status cupc_result_sshare(const cupc_result* r, int level, const int64_t* bins, int nbins,
                                          int64_t* counts, cupc_sshare_stats* stats)
{
    if (!r || !bins || nbins < 1 || nbins > 4096 || !counts) return CUPC_E_INVALID;
    cupc_ctx* ctx = r->ctx;
    if (level < 1 || level > 4) return ctx_fail(ctx, CUPC_E_RANGE, "level must be in [1, 4]");
    for (int k = 0; k < nbins; ++k)
        if (bins[k] < 1 || (k && bins[k] <= bins[k - 1])) return ctx_fail(ctx, CUPC_E_INVALID, "bins");
    const int bits = (r->p <= 65535) ? 16 : 32;
    if (level * bits > 64) return ctx_fail(ctx, CUPC_E_RANGE, "l-subsets of this p do not fit a 64-bit key");
    std::vector<long long> off;
    std::vector<int> cols;
    cupc_status s = result_frozen_lists(r, level, off, cols);
    if (s != CUPC_OK) return s;
    const int p = (int)r->p;
    // pairs (row, S) of the rows that run tests at the level
    int dmax = 0;
    for (int i = 0; i < p; ++i) dmax = std::max(dmax, (int)(off[i + 1] - off[i]));
    auto binom = [](long long m, int k) {
        long double v = 1;
        for (int q = 0; q < k; ++q) v = v * (long double)(m - q) / (long double)(q + 1);
        return (unsigned long long)(v + 0.5L);
    };
    std::vector<long long> pre((size_t)p + 1, 0);
    long long rows = 0;
    for (int i = 0; i < p; ++i) {
        const long long d = off[i + 1] - off[i];
        const unsigned long long c = (d >= level + 1) ? binom(d, level) : 0ull;
        rows += c ? 1 : 0;
        pre[i + 1] = pre[i] + (long long)c;
        if (pre[i + 1] > (1ll << 28)) return ctx_fail(ctx, CUPC_E_RANGE, "more than 2^28 (row, S) pairs");
    }
    const unsigned long long total = (unsigned long long)pre[p];
    unsigned long long slots = 1024;
    while (slots < 2 * total) slots <<= 1;
    Binom B;
    if ((s = ctx_binom(ctx, std::max(dmax + 2, 64), &B)) != CUPC_OK) return s;
    Buf* bo = ctx_buf(ctx, "ss_off");
    Buf* bc = ctx_buf(ctx, "ss_cols");
    Buf* bp = ctx_buf(ctx, "ss_pre");
    Buf* bk = ctx_buf(ctx, "ss_keys");
    Buf* bn = ctx_buf(ctx, "ss_cnt");
    Buf* bb = ctx_buf(ctx, "ss_bins");
    Buf* bq = ctx_buf(ctx, "ss_out");
    if ((s = ctx_ensure(ctx, bo, off.size() * 8)) != CUPC_OK || (s = ctx_ensure(ctx, bc, cols.size() * 4 + 4)) != CUPC_OK ||
        (s = ctx_ensure(ctx, bp, pre.size() * 8)) != CUPC_OK || (s = ctx_ensure(ctx, bk, slots * 8)) != CUPC_OK ||
        (s = ctx_ensure(ctx, bn, slots * 4)) != CUPC_OK || (s = ctx_ensure(ctx, bb, (size_t)nbins * 8)) != CUPC_OK ||
        (s = ctx_ensure(ctx, bq, ((size_t)nbins + 4) * 8)) != CUPC_OK)
        return s;
    cudaStream_t st = ctx_stream(ctx);
#define SC(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return ctx_fail(ctx, CUPC_E_CUDA, #call, e_);              \
    } while (0)
    SC(cudaMemcpyAsync(bo->p, off.data(), off.size() * 8, cudaMemcpyHostToDevice, st));
    if (!cols.empty()) SC(cudaMemcpyAsync(bc->p, cols.data(), cols.size() * 4, cudaMemcpyHostToDevice, st));
    SC(cudaMemcpyAsync(bp->p, pre.data(), pre.size() * 8, cudaMemcpyHostToDevice, st));
    SC(cudaMemcpyAsync(bb->p, bins, (size_t)nbins * 8, cudaMemcpyHostToDevice, st));
    SC(cudaMemsetAsync(bk->p, 0xff, slots * 8, st));
    SC(cudaMemsetAsync(bn->p, 0, slots * 4, st));
    SC(cudaMemsetAsync(bq->p, 0, ((size_t)nbins + 4) * 8, st));
    cudaEvent_t e0, e1;
    SC(cudaEventCreate(&e0));
    SC(cudaEventCreate(&e1));
    SC(cudaEventRecord(e0, st));
    unsigned long long* out = (unsigned long long*)bq->p;
    cudaError_t le = launch_sshare((const long long*)bo->p, (const int*)bc->p, (const long long*)bp->p, p, level, bits,
                                   B, total, (unsigned long long*)bk->p, (unsigned*)bn->p, slots,
                                   (const long long*)bb->p, nbins, out, (int*)(out + nbins + 3), ctx_num_sms(ctx), st);
    ctx_count_launch(ctx);
    ctx_count_launch(ctx);
    SC(le);
    SC(cudaEventRecord(e1, st));
    std::vector<unsigned long long> h((size_t)nbins + 4);
    SC(cudaMemcpyAsync(h.data(), out, h.size() * 8, cudaMemcpyDeviceToHost, st));
    SC(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (h[(size_t)nbins + 3]) return ctx_fail(ctx, CUPC_E_STATE, "hash table overflow");
    for (int k = 0; k < nbins; ++k) counts[k] = (int64_t)h[(size_t)k];
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->pairs = (int64_t)total;
        stats->distinct = (int64_t)h[(size_t)nbins];
        stats->redundant = (int64_t)h[(size_t)nbins + 1];
        stats->max_rows = (int64_t)h[(size_t)nbins + 2];
        stats->rows = rows;
        stats->search_ms = ms;
    }
    return CUPC_OK;
#undef SC
}
