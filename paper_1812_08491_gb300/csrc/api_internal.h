// api_internal.h -- context and result objects shared by the host files of
// the C ABI (api.cu, api_mlp.cu).
#pragma once

#include <map>
#include <string>
#include <vector>

#include "kernels.cuh"

struct Buf {
    void* p = nullptr;
    size_t cap = 0;
};

struct cupc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaMemPool_t pool = nullptr;
    std::string err;
    int refs = 1;
    int num_sms = 0;
    Buf xin, xt, mu, isd, z64, zhi, zlo, cws, c64, c32, cin;
    Buf deg, row_off, item_off, item_row, cols, srow, partner, wpre, best, queue, binom, meta, lmeta, backup[2];
    Buf part;
    cupc::Meta* hmeta = nullptr;
    cupc::LevelMeta* hlmeta = nullptr;
    int* hflags = nullptr;         // pinned, mapped: per-level run / end flags written by the GPU
    int* dflags = nullptr;         // device view of hflags
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
};

struct cupc_result {
    cupc_ctx* ctx = nullptr;
    int64_t p = 0;
    int W = 0;
    unsigned* bits = nullptr;
    unsigned* bits0 = nullptr;
    int* rec = nullptr;
    int64_t rec_ints = 0;
    size_t rec_cap = 0;
    cupc_stats stats{};
    mutable bool host_ready = false;
    mutable std::vector<int32_t> hrec;                              // sorted records
    mutable std::vector<std::pair<uint64_t, int64_t>> index;        // (i*p+j) -> offset
};


// helpers with external linkage for the other host files
cupc_status ctx_ensure(cupc_ctx* ctx, Buf* b, size_t bytes);
Buf* ctx_buf(cupc_ctx* ctx, const char* name);
int ctx_num_sms(cupc_ctx* ctx);
cudaStream_t ctx_stream(cupc_ctx* ctx);
cupc_status ctx_fail(cupc_ctx* ctx, cupc_status s, const std::string& what, cudaError_t e = cudaSuccess);
void ctx_count_launch(cupc_ctx* ctx);
void ctx_set_mlp(cupc_ctx* ctx, int ready, int step);
int ctx_mlp_ready(cupc_ctx* ctx);
int ctx_mlp_step(cupc_ctx* ctx);
