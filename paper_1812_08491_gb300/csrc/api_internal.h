// api_internal.h -- context and result objects shared by the host files of
// the C ABI (api.cu, api_mlp.cu).
#pragma once

#include <atomic>
#include <map>
#include <string>
#include <vector>

#include "kernels.cuh"

namespace cupc {
constexpr double kBand0 = 2e-5;        // level 0 FP32 band on |C_ij|
constexpr double kBandAbs = 4e-6;      // levels >= 1 FP32 band on |rho|
constexpr double kBandRel = 4e-6;      // widening per 1/(pivot^2 * min conditional variance)
constexpr double kPivFloor = 1e-3;     // FP32: smaller pivot^2 goes to FP64
constexpr double kRankTol64 = 1e-12;   // FP64: pivot^2 at or below -> dependent member
constexpr double kRankTol32 = 1e-6;
constexpr size_t kPartBytes = size_t(32) << 20;  // FP64 recheck partial sums per batch of tests
}  // namespace cupc

struct Buf {
    void* p = nullptr;
    size_t cap = 0;
};

struct cupc_ctx {
    std::atomic<int> cancel{0};         // cupc_cancel: the running or next call stops between levels
    int fail_kind = 0;                  // cupc_debug_fail: armed failure (0 none)
    long long fail_k = 0;               // ... on the k-th next allocation / launch
    unsigned barrier_ns = 0;            // ... or the next call's grid-barrier wait limit
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaMemPool_t pool = nullptr;
    std::string err;
    int refs = 1;
    int num_sms = 0;
    Buf xin, xt, mu, isd, mup, z64, zhi, zlo, cws, c64, c32, cin;
    Buf deg, row_off, item_off, item_row, cols, srow, partner, wpre, best, queue, binom, meta, lmeta;
    Buf part;
    cupc::Meta* hmeta = nullptr;
    cupc::LevelMeta* hlmeta = nullptr;
    int* hflags = nullptr;         // pinned, mapped: per-level run / end flags written by the GPU
    int* dflags = nullptr;         // device view of hflags
    cudaStream_t cstream = nullptr;     // copy stream of chunked uploads (created on first use)
    cudaEvent_t cev[8] = {};            // chunk-arrival events (and [7]: the context stream's position)
    void* hstage = nullptr;        // pinned staging for device-built result lists (grown on demand)
    size_t hstage_cap = 0;
    int binom_mstride = 0;
    unsigned long long launches = 0;
    unsigned long long h2d = 0, d2h = 0;
    std::vector<cudaEvent_t> ev;
    // kernel-class timing: event pairs recorded around the timed launches
    std::vector<cudaEvent_t> tev;
    std::vector<int> tcls;
    int tused = 0;
    std::map<std::string, Buf> named;   // further device buffers (network state)
    int mlp_ready = 0;                  // network weights loaded
    int mlp_step = 0;                   // Adam steps taken
    // largest level-buffer needs seen by this context's calls (CSR slots, SepSet
    // ints, candidate-list entries): the next call is sized for them up front
    unsigned long long cap_nnz = 0;
    size_t cap_rec = 0;
    void* batch = nullptr;              // batch plan (api_batch.cu)
    void (*batch_free)(cupc_ctx*) = nullptr;
};

struct cupc_result {
    cupc_ctx* ctx = nullptr;
    int64_t p = 0;
    int64_t n = 0;                 // samples, alpha and the options the levels ran with
    double alpha = 0.0;
    int mode = 0, canonical = 0, learned = 0;
    int W = 0;
    unsigned* bits = nullptr;
    unsigned* bits0 = nullptr;
    int* rec = nullptr;
    int64_t rec_ints = 0;
    size_t rec_cap = 0;
    cupc_stats stats{};
    bool on_host = false;                                           // batch results: bitsets on the host
    std::vector<unsigned> hbits, hbits0;
    mutable bool host_ready = false;
    mutable std::vector<int32_t> hrec;                              // sorted records
    mutable std::vector<std::pair<uint64_t, int64_t>> index;        // (i*p+j) -> offset
    mutable bool index_ready = false;
    mutable bool edges_ready = false;
    mutable std::vector<int32_t> hedges;                            // edge list (i, j), i < j
};


// helpers with external linkage for the other host files
cupc_status result_frozen_lists(const cupc_result* r, int level, std::vector<long long>& off, std::vector<int>& cols);
cupc_status ctx_ensure(cupc_ctx* ctx, Buf* b, size_t bytes);
cupc_status ctx_host_stage(cupc_ctx* ctx, size_t bytes, char** out);   // pinned staging, grown on demand
void ctx_free(cupc_ctx* ctx, Buf* b);
double ctx_fisher_tau(double alpha, int64_t n, int l);
cupc_status ctx_binom(cupc_ctx* ctx, int m_needed, cupc::Binom* out);
cupc_status ctx_validate(cupc_ctx* ctx, const cupc_options& o);
Buf* ctx_buf(cupc_ctx* ctx, const char* name);
int ctx_num_sms(cupc_ctx* ctx);
cudaStream_t ctx_stream(cupc_ctx* ctx);
cupc_status ctx_fail(cupc_ctx* ctx, cupc_status s, const std::string& what, cudaError_t e = cudaSuccess);
void ctx_count_launch(cupc_ctx* ctx);
void ctx_set_mlp(cupc_ctx* ctx, int ready, int step);
int ctx_mlp_ready(cupc_ctx* ctx);
int ctx_mlp_step(cupc_ctx* ctx);
