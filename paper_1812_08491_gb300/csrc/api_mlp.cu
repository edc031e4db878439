// api_mlp.cu -- C ABI of the candidate-scoring network: weights, gradient,
// scoring and training on the device (kernels in k_mlp.cu).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "api_internal.h"
#include "mlp.cuh"

using namespace cupc;

namespace {

cupc_status mlp_ensure(cupc_ctx* ctx)
{
    cupc_status s;
    if ((s = ctx_ensure(ctx, ctx_buf(ctx, "mlp_P"), MLP_NP * 4)) != CUPC_OK) return s;
    if ((s = ctx_ensure(ctx, ctx_buf(ctx, "mlp_M"), MLP_NP * 4)) != CUPC_OK) return s;
    if ((s = ctx_ensure(ctx, ctx_buf(ctx, "mlp_V"), MLP_NP * 4)) != CUPC_OK) return s;
    if ((s = ctx_ensure(ctx, ctx_buf(ctx, "mlp_Pb"), MLP_NP * 2)) != CUPC_OK) return s;
    if ((s = ctx_ensure(ctx, ctx_buf(ctx, "mlp_gsum"), MLP_NP * 4)) != CUPC_OK) return s;
    const int blocks = ctx_num_sms(ctx);
    if ((s = ctx_ensure(ctx, ctx_buf(ctx, "mlp_gpart"), (size_t)blocks * MLP_NP * 4)) != CUPC_OK) return s;
    if ((s = ctx_ensure(ctx, ctx_buf(ctx, "mlp_lpart"), (size_t)blocks * 4)) != CUPC_OK) return s;
    return CUPC_OK;
}

float* bufp(cupc_ctx* ctx, const char* name) { return (float*)ctx_buf(ctx, name)->p; }

// gradient over [s0, s1) into mlp_gsum (and optionally an Adam step); returns
// the summed loss of the range through *loss_sum when non-null.
cupc_status grad_range(cupc_ctx* ctx, const float* X, const float* t, long long s0, long long s1, int step,
                       float lr, double* loss_sum)
{
    const int blocks = (int)std::min<long long>(ctx_num_sms(ctx), (s1 - s0 + 127) / 128);
    cudaStream_t st = ctx_stream(ctx);
    cudaError_t e = launch_mlp_grad(bufp(ctx, "mlp_P"), X, t, s0, s1, bufp(ctx, "mlp_gpart"), bufp(ctx, "mlp_lpart"),
                                    blocks, st);
    ctx_count_launch(ctx);
    if (e != cudaSuccess) return ctx_fail(ctx, CUPC_E_CUDA, "mlp gradient kernel", e);
    e = launch_mlp_apply(bufp(ctx, "mlp_P"), bufp(ctx, "mlp_M"), bufp(ctx, "mlp_V"), bufp(ctx, "mlp_gpart"), blocks,
                         bufp(ctx, "mlp_gsum"), step, lr, ctx_buf(ctx, "mlp_Pb")->p, st);
    ctx_count_launch(ctx);
    if (e != cudaSuccess) return ctx_fail(ctx, CUPC_E_CUDA, "mlp apply kernel", e);
    if (loss_sum) {
        std::vector<float> lp(blocks);
        e = cudaMemcpyAsync(lp.data(), bufp(ctx, "mlp_lpart"), blocks * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return ctx_fail(ctx, CUPC_E_CUDA, "mlp loss readback", e);
        for (int b = 0; b < blocks; ++b) *loss_sum += lp[b];
    }
    return CUPC_OK;
}

}  // namespace

extern "C" {

cupc_status cupc_mlp_set_weights(cupc_ctx* ctx, const float* params)
{
    if (!ctx || !params) return CUPC_E_INVALID;
    cupc_status s = mlp_ensure(ctx);
    if (s != CUPC_OK) return s;
    cudaStream_t st = ctx_stream(ctx);
    cudaError_t e = cudaMemcpyAsync(bufp(ctx, "mlp_P"), params, MLP_NP * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bufp(ctx, "mlp_M"), 0, MLP_NP * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bufp(ctx, "mlp_V"), 0, MLP_NP * 4, st);
    if (e == cudaSuccess) e = launch_mlp_to_bf16(bufp(ctx, "mlp_P"), ctx_buf(ctx, "mlp_Pb")->p, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ctx_fail(ctx, CUPC_E_CUDA, "mlp weight upload", e);
    ctx_set_mlp(ctx, 1, 0);
    return CUPC_OK;
}

cupc_status cupc_mlp_get_weights(cupc_ctx* ctx, float* params)
{
    if (!ctx || !params) return CUPC_E_INVALID;
    if (!ctx_mlp_ready(ctx)) return ctx_fail(ctx, CUPC_E_STATE, "no network weights loaded");
    cudaStream_t st = ctx_stream(ctx);
    cudaError_t e = cudaMemcpyAsync(params, bufp(ctx, "mlp_P"), MLP_NP * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ctx_fail(ctx, CUPC_E_CUDA, "mlp weight download", e);
    return CUPC_OK;
}

cupc_status cupc_mlp_grad(cupc_ctx* ctx, const float* X, const float* t, int64_t n, float* grad, double* loss)
{
    if (!ctx || !X || !t || !grad || n <= 0) return CUPC_E_INVALID;
    if (!ctx_mlp_ready(ctx)) return ctx_fail(ctx, CUPC_E_STATE, "no network weights loaded");
    double lsum = 0.0;
    cupc_status s = grad_range(ctx, X, t, 0, n, 0, 0.f, &lsum);
    if (s != CUPC_OK) return s;
    cudaStream_t st = ctx_stream(ctx);
    cudaError_t e = cudaMemcpyAsync(grad, bufp(ctx, "mlp_gsum"), MLP_NP * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ctx_fail(ctx, CUPC_E_CUDA, "mlp gradient readback", e);
    if (loss) *loss = lsum / (double)n;
    return CUPC_OK;
}

cupc_status cupc_mlp_forward(cupc_ctx* ctx, const float* X, int64_t n, float* y)
{
    if (!ctx || !X || !y || n < 0) return CUPC_E_INVALID;
    if (!ctx_mlp_ready(ctx)) return ctx_fail(ctx, CUPC_E_STATE, "no network weights loaded");
    cudaStream_t st = ctx_stream(ctx);
    cudaError_t e = launch_mlp_forward(ctx_buf(ctx, "mlp_Pb")->p, X, n, y, st);
    ctx_count_launch(ctx);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ctx_fail(ctx, CUPC_E_CUDA, "mlp forward", e);
    return CUPC_OK;
}

cupc_status cupc_mlp_train(cupc_ctx* ctx, const float* X, const float* t, int64_t n, int64_t batch, int epochs,
                           double lr, double* epoch_loss)
{
    if (!ctx || !X || !t || n <= 0 || batch <= 0 || epochs < 0 || !(lr > 0.0)) return CUPC_E_INVALID;
    if (!ctx_mlp_ready(ctx)) return ctx_fail(ctx, CUPC_E_STATE, "no network weights loaded");
    for (int ep = 0; ep < epochs; ++ep) {
        double lsum = 0.0;
        for (long long s0 = 0; s0 < n; s0 += batch) {
            const long long s1 = std::min<long long>(n, s0 + batch);
            const int step = ctx_mlp_step(ctx) + 1;
            cupc_status s = grad_range(ctx, X, t, s0, s1, step, (float)lr, epoch_loss ? &lsum : nullptr);
            if (s != CUPC_OK) return s;
            ctx_set_mlp(ctx, 1, step);
        }
        if (epoch_loss) epoch_loss[ep] = lsum / (double)n;
    }
    cudaError_t e = cudaStreamSynchronize(ctx_stream(ctx));
    if (e != cudaSuccess) return ctx_fail(ctx, CUPC_E_CUDA, "mlp training", e);
    return CUPC_OK;
}

cupc_status cupc_mlp_examples(const cupc_result* res, const float* C, float* X, float* t, int64_t cap, int64_t* n)
{
    if (!res || !C || !n || cap < 0 || ((X == nullptr) != (t == nullptr))) return CUPC_E_INVALID;
    cupc_ctx* ctx = res->ctx;
    std::vector<long long> off;
    std::vector<int> cols;
    cupc_status s = result_frozen_lists(res, 1, off, cols);   // (also builds the host records)
    if (s != CUPC_OK) return s;
    const std::vector<int32_t>& rec = res->hrec;
    int lmax = 0;
    for (size_t k = 0; k < rec.size(); k += 3 + (size_t)rec[k + 2]) lmax = std::max(lmax, (int)rec[k + 2]);
    // every level's frozen neighbour lists, one after another in nbs
    std::vector<std::vector<long long>> offs((size_t)lmax + 1);
    std::vector<long long> base((size_t)lmax + 1, 0);
    std::vector<int> nbs;
    for (int l = 1; l <= lmax; ++l) {
        std::vector<int> c;
        if (l == 1) {
            offs[1].swap(off);
            c.swap(cols);
        } else if ((s = result_frozen_lists(res, l, offs[(size_t)l], c)) != CUPC_OK) {
            return s;
        }
        base[(size_t)l] = (long long)nbs.size();
        nbs.insert(nbs.end(), c.begin(), c.end());
    }
    if (nbs.size() > (size_t)INT32_MAX) return ctx_fail(ctx, CUPC_E_RANGE, "training examples: neighbour lists too long");
    // (row a, candidate position, list start, list length, level, label): the side
    // whose frozen neighbourhood holds S (the smaller endpoint first), one
    // example per candidate other than the other endpoint
    std::vector<int32_t> q;
    for (size_t k = 0; k < rec.size(); k += 3 + (size_t)rec[k + 2]) {
        const int x = rec[k], y = rec[k + 1], l = rec[k + 2];
        if (l < 1) continue;
        const std::vector<long long>& o = offs[(size_t)l];
        for (int side = 0; side < 2; ++side) {
            const int a = side ? y : x, b = side ? x : y;
            const int* nb = nbs.data() + base[(size_t)l] + o[(size_t)a];
            const int d = (int)(o[(size_t)a + 1] - o[(size_t)a]);
            bool all = true;
            for (int m = 0; m < l && all; ++m) all = std::binary_search(nb, nb + d, rec[k + 3 + m]);
            if (!all) continue;
            for (int u = 0; u < d; ++u) {
                if (nb[u] == b) continue;
                bool in = false;
                for (int m = 0; m < l; ++m) in = in || rec[k + 3 + m] == nb[u];
                q.push_back(a);
                q.push_back(u);
                q.push_back((int32_t)(base[(size_t)l] + o[(size_t)a]));
                q.push_back(d);
                q.push_back(l);
                q.push_back(in ? 1 : 0);
            }
            break;
        }
    }
    const int64_t count = (int64_t)(q.size() / 6);
    *n = count;
    if (!X || count == 0 || cap == 0) return CUPC_OK;
    const int64_t m = std::min<int64_t>(cap, count);
    Buf* bq = ctx_buf(ctx, "mlp_ex_q");
    Buf* bn = ctx_buf(ctx, "mlp_ex_nb");
    if ((s = ctx_ensure(ctx, bq, (size_t)m * 24)) != CUPC_OK) return s;
    if ((s = ctx_ensure(ctx, bn, nbs.size() * 4)) != CUPC_OK) return s;
    cudaStream_t st = ctx_stream(ctx);
    cudaError_t e = cudaMemcpyAsync(bq->p, q.data(), (size_t)m * 24, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bn->p, nbs.data(), nbs.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_mlp_examples(C, res->p, (const int*)bn->p, (const int*)bq->p, m, X, t, st);
    ctx_count_launch(ctx);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ctx_fail(ctx, CUPC_E_CUDA, "training examples", e);
    return CUPC_OK;
}

}  // extern "C"
