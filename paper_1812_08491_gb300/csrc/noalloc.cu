// noalloc.cu -- cupc_correlation_noalloc: the FP64 correlation matrix without
// any device allocation.
//
// It runs the same kernels as cupc_correlation(precision = CUPC_F64) -- layout
// transpose, FP64 moments and standardised rows, the FP64 symmetric product --
// but their scratch (moments, the transposed input, the standardised rows and
// the error flag) lives in one file-scope device array instead of memory the
// library allocates. The caller passes device input and output buffers and a
// stream; nothing else is needed.
#include <mutex>

#include "kernels.cuh"

using namespace cupc;

namespace {

constexpr size_t kScratchBytes = size_t(36) << 20;          // 36 MiB per device
constexpr long long kMaxElems = 1ll << 21;                  // n * p
constexpr long long kMaxVars = 65536;                       // p
constexpr int kMaxDevices = 64;

// Scratch of cupc_correlation_noalloc. Every device that loads the library
// holds one copy until the process exits. All calls on a device share it.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of g_scratch on the current device, looked up once per device.
cupc_status scratch_address(int dev, void** out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return CUPC_E_CUDA;
        }
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    return CUPC_OK;
}

}  // namespace

extern "C" cupc_status cupc_correlation_noalloc(const void* X, int dtype, int layout, int64_t n_samples, int64_t p,
                                                int64_t ld, double* C_out, void* stream)
{
    if (!X || !C_out) return CUPC_E_INVALID;
    if (dtype != CUPC_F32 && dtype != CUPC_F64) return CUPC_E_INVALID;
    if (layout != CUPC_LAYOUT_SAMPLE_MAJOR && layout != CUPC_LAYOUT_VARIABLE_MAJOR) return CUPC_E_INVALID;
    if (n_samples < 2 || p < 1) return CUPC_E_INVALID;
    if (ld < (layout == CUPC_LAYOUT_SAMPLE_MAJOR ? p : n_samples)) return CUPC_E_INVALID;
    if (p > kMaxVars || n_samples * p > kMaxElems) return CUPC_E_RANGE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return CUPC_E_CUDA;
    }
    void* base = nullptr;
    cupc_status s = scratch_address(dev, &base);
    if (s != CUPC_OK) return s;

    const int n = (int)n_samples, pp = (int)p;
    const size_t es = dtype == CUPC_F64 ? 8 : 4;
    unsigned char* at = (unsigned char*)base;
    Meta* meta = (Meta*)at;
    at += up256(sizeof(Meta));
    double* mu = (double*)at;
    at += up256((size_t)pp * 8);
    double* isd = (double*)at;
    at += up256((size_t)pp * 8);
    void* xt = at;
    if (layout == CUPC_LAYOUT_SAMPLE_MAJOR) at += up256((size_t)n * pp * es);
    double* z64 = (double*)at;
    at += up256((size_t)n * pp * 8);
    if ((size_t)(at - (unsigned char*)base) > kScratchBytes) return CUPC_E_RANGE;

    cudaStream_t st = (cudaStream_t)stream;
    // the previous call's flag must not leak into this one
    if (cudaMemsetAsync(meta, 0, sizeof(Meta), st) != cudaSuccess) {
        cudaGetLastError();
        return CUPC_E_CUDA;
    }
    const void* xv = X;
    long long ldv = ld;
    if (layout == CUPC_LAYOUT_SAMPLE_MAJOR) {
        if (launch_transpose(dtype, X, ld, n, pp, xt, st) != cudaSuccess) return CUPC_E_CUDA;
        xv = xt;
        ldv = n;
    }
    if (launch_standardize(dtype, xv, ldv, n, pp, mu, isd, nullptr, z64, n, nullptr, nullptr, 0, meta, st) != cudaSuccess)
        return CUPC_E_CUDA;
    if (launch_syrk_f64(z64, n, n, pp, C_out, st) != cudaSuccess) return CUPC_E_CUDA;
    int err = 0;
    if (cudaMemcpyAsync(&err, &meta->error, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return CUPC_E_CUDA;
    }
    return err ? CUPC_E_NUMERIC : CUPC_OK;
}
