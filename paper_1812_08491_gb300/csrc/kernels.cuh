// kernels.cuh -- launcher declarations shared by the host driver and the kernel files.
#pragma once

#include "cupc_internal.cuh"

namespace cupc {

// Parameters of one level's CI-test kernel (levels l >= 1).
struct CIParams {
    const long long* row_off;      // p + 1 CSR offsets of A'_G
    const int* cols;               // nnz neighbour indices (increasing per row)
    const int* partner;            // nnz: slot of (j, i) for slot (i, j)
    const int* item_row;           // n_items: row of each work item
    const long long* item_off;     // p + 1: first item of each row
    const void* C;                 // p x p correlation (float or double), ld = p
    int p;
    int l;
    int chunk;                     // subset ranks per work item
    int canonical;
    Binom B;
    double r;                      // tanh(tau_l)
    double r2;                     // tanh(tau_l)^2
    double band_abs, band_rel;     // FP32 mode: recheck band on |rho|
    double rank_tol;               // pivot^2 at or below which a member of S is dependent
    double piv_floor;              // FP32 mode: smaller pivot^2 sends the test to FP64
    unsigned long long* best;      // nnz: smallest separating rank found per slot
    QEntry* queue;                 // FP32 mode recheck queue
    unsigned long long qcap;
    Meta* meta;
    unsigned long long n_items;
};

// Parameters of the FP64 recheck of queued tests.
struct RecheckParams {
    const long long* row_off;
    const int* cols;
    const int* srow;
    const double* z64;             // standardised rows (row v at z64 + v*ldz), used when c64 == nullptr
    long long ldz;
    int n;
    const double* c64;             // FP64 correlation if resident, else nullptr
    int p;
    int l;
    Binom B;
    double r2;
    double rank_tol;
    unsigned long long* best;
    const QEntry* queue;
    unsigned long long qcap;
    Meta* meta;
    unsigned* bits;                // level 0: adjacency to clear
    int W;
};

struct FinalizeParams {
    const long long* row_off;
    const int* cols;
    const int* srow;
    const int* partner;
    const unsigned long long* best;
    unsigned* bits;
    int W;
    int l;
    Binom B;
    int count_serial;
    int* rec;                      // SepSet record pool (int32)
    unsigned long long rec_cap;    // in ints
    Meta* meta;
    unsigned long long nnz;
};

cudaError_t launch_transpose(int dtype, const void* X, long long ld, int n, int p, void* Xt, cudaStream_t st);
cudaError_t launch_standardize(int dtype, const void* Xv, long long ld, int n, int p, double* mu, double* isd,
                               double* z64, long long ldz, void* zhi, void* zlo, long long ldb, Meta* meta,
                               cudaStream_t st);
cudaError_t launch_syrk_f64(const double* Z, long long ldz, int n, int p, double* C, cudaStream_t st);
void corr_tc_plan(int p, long long ldk, int num_sms, int* tiles, int* nsplit, int* kps, size_t* ws_bytes);
cudaError_t launch_corr_tc(const void* hi, const void* lo, long long ldk, int p, int n, float* ws, float* C,
                           int num_sms, int* err, cudaStream_t st);
cudaError_t launch_symmetrize(int dtype, const void* Cin, long long ld, int p, double* C64, float* C32,
                              cudaStream_t st);

cudaError_t launch_level0(int fp32, const void* C, int p, int W, double r0, double band0, unsigned* bits,
                          QEntry* q, unsigned long long qcap, Meta* meta, cudaStream_t st);
cudaError_t launch_degree(const unsigned* bits, int p, int W, int* deg, Meta* meta, cudaStream_t st);
cudaError_t launch_scan(const int* deg, int p, int l, int chunk, Binom B, long long* row_off,
                        long long* item_off, Meta* meta, cudaStream_t st);
cudaError_t launch_fill(const unsigned* bits, int p, int W, const long long* row_off, int* cols, int* srow,
                        cudaStream_t st);
cudaError_t launch_items(const long long* item_off, int p, int* item_row, cudaStream_t st);
cudaError_t launch_partner(const long long* row_off, const int* cols, const int* srow, long long nnz,
                           int* partner, cudaStream_t st);
cudaError_t launch_ci(int fp32, const CIParams& P, int grid, int block, cudaStream_t st);
cudaError_t launch_recheck(const RecheckParams& P, int grid, cudaStream_t st);
cudaError_t launch_recheck0(const RecheckParams& P, int grid, cudaStream_t st);
cudaError_t launch_finalize(const FinalizeParams& P, cudaStream_t st);
cudaError_t launch_pcor(int fp32, const void* C, int p, const int* q, long long nq, int l, double* rho,
                        cudaStream_t st);
cudaError_t launch_bits_to_u8(const unsigned* bits, int p, int W, unsigned char* out, cudaStream_t st);

int ci_max_level_supported();

}  // namespace cupc
