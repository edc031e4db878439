// api_orient.cu -- C ABI of the orientation step (second step of PC-stable,
// Sec. 2.4): v-structures and Meek's rules on the device, kernels in
// k_orient.cu.
#include <algorithm>
#include <cstring>
#include <vector>

#include "api_internal.h"
#include "orient.cuh"

using namespace cupc;

namespace {

#define OCU(call)                                                                \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) return ctx_fail(ctx, CUPC_E_CUDA, #call, e_);     \
    } while (0)

#define OLAUNCH(call)                                                            \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        ctx_count_launch(ctx);                                                   \
        if (e_ != cudaSuccess) return ctx_fail(ctx, CUPC_E_CUDA, #call, e_);     \
    } while (0)

struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

template <typename T>
T* buf(cupc_ctx* ctx, const char* name) { return (T*)ctx_buf(ctx, name)->p; }

}  // namespace

extern "C" cupc_status cupc_result_orient(cupc_result* r, uint8_t* marks, cupc_orient_stats* stats)
{
    if (!r || !r->ctx) return CUPC_E_INVALID;
    cupc_ctx* ctx = r->ctx;
    OCU(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx_stream(ctx);
    const int p = (int)r->p, W = r->W;
    const size_t words = (size_t)p * W;
    cupc_status s;

    // the skeleton after the last level and after level 0 (device bitsets)
    const unsigned *bits = r->bits, *bits0 = r->bits0;
    if (r->on_host) {
        if (r->hbits.size() < words || r->hbits0.size() < words)
            return ctx_fail(ctx, CUPC_E_STATE, "result holds no skeleton");
        if ((s = ctx_ensure(ctx, ctx_buf(ctx, "or_bits"), words * 4)) != CUPC_OK) return s;
        if ((s = ctx_ensure(ctx, ctx_buf(ctx, "or_bits0"), words * 4)) != CUPC_OK) return s;
        OCU(cudaMemcpyAsync(buf<unsigned>(ctx, "or_bits"), r->hbits.data(), words * 4, cudaMemcpyHostToDevice, st));
        OCU(cudaMemcpyAsync(buf<unsigned>(ctx, "or_bits0"), r->hbits0.data(), words * 4, cudaMemcpyHostToDevice,
                            st));
        bits = buf<unsigned>(ctx, "or_bits");
        bits0 = buf<unsigned>(ctx, "or_bits0");
    }
    if (!bits || !bits0) return ctx_fail(ctx, CUPC_E_STATE, "result holds no skeleton");

    // SepSet records grouped by level: a single call's records are appended
    // level by level (3 + l ints each), so the per-level removal counts give
    // the groups; a batch result's host records are regrouped and uploaded
    OrRecords R{};
    const int* rec = r->rec;
    std::vector<int32_t> grouped;
    if (!r->on_host) {
        long long at = 0, idx = 0;
        for (int l = 1; l < r->stats.levels && l <= CUPC_MAX_LEVEL; ++l) {
            const long long c = r->stats.removed[l];
            if (c <= 0) continue;
            R.lev[R.groups] = l;
            R.start[R.groups] = at;
            R.count[R.groups] = c;
            R.first[R.groups] = idx;
            ++R.groups;
            at += c * (3 + l);
            idx += c;
        }
        R.total = idx;
        if (at != r->rec_ints) return ctx_fail(ctx, CUPC_E_STATE, "SepSet records do not match the level counts");
    } else {
        std::vector<std::vector<int32_t>> by(CUPC_MAX_LEVEL + 1);
        std::vector<long long> cnt(CUPC_MAX_LEVEL + 1, 0);
        for (size_t k = 0; k < r->hrec.size();) {
            const int l = r->hrec[k + 2];
            if (l < 1 || l > CUPC_MAX_LEVEL) return ctx_fail(ctx, CUPC_E_STATE, "bad SepSet record");
            by[l].insert(by[l].end(), r->hrec.begin() + k, r->hrec.begin() + k + 3 + l);
            ++cnt[l];
            k += 3 + l;
        }
        long long idx = 0;
        for (int l = 1; l <= CUPC_MAX_LEVEL; ++l) {
            if (!cnt[l]) continue;
            R.lev[R.groups] = l;
            R.start[R.groups] = (long long)grouped.size();
            R.count[R.groups] = cnt[l];
            R.first[R.groups] = idx;
            ++R.groups;
            idx += cnt[l];
            grouped.insert(grouped.end(), by[l].begin(), by[l].end());
        }
        R.total = idx;
        if (!grouped.empty()) {
            if ((s = ctx_ensure(ctx, ctx_buf(ctx, "or_rec"), grouped.size() * 4)) != CUPC_OK) return s;
            OCU(cudaMemcpyAsync(buf<int>(ctx, "or_rec"), grouped.data(), grouped.size() * 4, cudaMemcpyHostToDevice,
                                st));
            rec = buf<int>(ctx, "or_rec");
        }
    }
    if (R.total > 0 && !rec) return ctx_fail(ctx, CUPC_E_STATE, "result holds no SepSet records");

    Events ev;
    OCU(cudaEventCreate(&ev.a));
    OCU(cudaEventCreate(&ev.b));
    OCU(cudaEventRecord(ev.a, st));

    // neighbour lists of the skeleton
    if ((s = ctx_ensure(ctx, ctx_buf(ctx, "or_deg"), (size_t)p * 4)) != CUPC_OK) return s;
    if ((s = ctx_ensure(ctx, ctx_buf(ctx, "or_off"), (size_t)(p + 1) * 8)) != CUPC_OK) return s;
    if ((s = ctx_ensure(ctx, ctx_buf(ctx, "or_flags"), 8 * 8)) != CUPC_OK) return s;
    int* deg = buf<int>(ctx, "or_deg");
    long long* off = buf<long long>(ctx, "or_off");
    unsigned long long* flags = buf<unsigned long long>(ctx, "or_flags");
    OLAUNCH(launch_or_degree(bits, p, W, deg, st));
    OLAUNCH(launch_or_scan(deg, p, off, st));
    long long nnz = 0;
    OCU(cudaMemcpyAsync(&nnz, off + p, 8, cudaMemcpyDeviceToHost, st));
    OCU(cudaStreamSynchronize(st));
    if ((s = ctx_ensure(ctx, ctx_buf(ctx, "or_cols"), (size_t)std::max(nnz, 1ll) * 4)) != CUPC_OK) return s;
    int* cols = buf<int>(ctx, "or_cols");
    OLAUNCH(launch_or_fill(bits, p, W, off, cols, st));

    // arrowheads of the v-structures
    for (const char* nm : {"or_head", "or_headT", "or_prop"})
        if ((s = ctx_ensure(ctx, ctx_buf(ctx, nm), words * 4)) != CUPC_OK) return s;
    unsigned* head = buf<unsigned>(ctx, "or_head");
    unsigned* headT = buf<unsigned>(ctx, "or_headT");
    unsigned* prop = buf<unsigned>(ctx, "or_prop");
    OCU(cudaMemsetAsync(head, 0, words * 4, st));
    OCU(cudaMemsetAsync(headT, 0, words * 4, st));
    OCU(cudaMemsetAsync(flags, 0, 8 * 8, st));
    OLAUNCH(launch_or_vstruct0(bits, bits0, p, W, off, cols, head, headT, st));
    OLAUNCH(launch_or_vstructS(bits, p, W, off, cols, rec, R, head, headT, st));

    // Meek's rules in rounds until one changes nothing (each applied round
    // orients at least one of the nnz / 2 edges, so at most nnz / 2 + 2 rounds
    // run). Rounds are queued kBatch at a time with one readback: round k keeps
    // its counters in rflags[2k], rflags[2k + 1], and a round after one that
    // applied nothing does nothing.
    constexpr int kBatch = 4;
    const long long rmax = nnz / 2 + 2;
    if ((s = ctx_ensure(ctx, ctx_buf(ctx, "or_rflags"), (size_t)rmax * 2 * 8)) != CUPC_OK) return s;
    unsigned long long* rflags = buf<unsigned long long>(ctx, "or_rflags");
    OCU(cudaMemsetAsync(rflags, 0, (size_t)rmax * 2 * 8, st));
    long long rounds = 0, rule_conflicts = 0;
    unsigned long long hf[2 * kBatch];
    bool ended = false;
    for (long long k = 0; !ended;) {
        if (k >= rmax) return ctx_fail(ctx, CUPC_E_STATE, "orientation rounds do not end");
        const long long k0 = k;
        for (int q = 0; q < kBatch && k < rmax; ++q, ++k) {
            const unsigned long long* gate = k ? rflags + 2 * (k - 1) : nullptr;
            OCU(cudaMemsetAsync(prop, 0, words * 4, st));
            OLAUNCH(launch_or_propose(bits, p, W, off, cols, head, headT, prop, gate, st));
            OLAUNCH(launch_or_apply(prop, p, W, head, headT, rflags + 2 * k, gate, st));
        }
        OCU(cudaMemcpyAsync(hf, rflags + 2 * k0, (size_t)(k - k0) * 2 * 8, cudaMemcpyDeviceToHost, st));
        OCU(cudaStreamSynchronize(st));
        for (long long j = 0; j < k - k0; ++j) {
            ++rounds;
            rule_conflicts += (long long)(hf[2 * j + 1] / 2);
            if (hf[2 * j] == 0) {
                ended = true;
                break;
            }
        }
    }

    // edge marks and counts (the marks are copied out when asked for)
    if ((s = ctx_ensure(ctx, ctx_buf(ctx, "or_marks"), (size_t)p * p)) != CUPC_OK) return s;
    unsigned char* dmarks = buf<unsigned char>(ctx, "or_marks");
    OLAUNCH(launch_or_marks(bits, headT, p, W, dmarks, flags, st));
    OCU(cudaEventRecord(ev.b, st));
    if (marks) OCU(cudaMemcpyAsync(marks, dmarks, (size_t)p * p, cudaMemcpyDeviceToHost, st));
    unsigned long long cnt[3] = {0, 0, 0};
    OCU(cudaMemcpyAsync(cnt, flags + 2, 3 * 8, cudaMemcpyDeviceToHost, st));
    OCU(cudaStreamSynchronize(st));
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->rounds = rounds;
        stats->directed = (int64_t)cnt[0];
        stats->undirected = (int64_t)cnt[1];
        stats->bidirected = (int64_t)cnt[2];
        stats->rule_conflicts = rule_conflicts;
        float ms = 0.f;
        OCU(cudaEventElapsedTime(&ms, ev.a, ev.b));
        stats->ms = ms;
    }
    return CUPC_OK;
}
