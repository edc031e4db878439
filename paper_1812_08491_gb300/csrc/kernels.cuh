// kernels.cuh -- launcher declarations shared by the host driver and the kernel files.
#pragma once

#include <vector>

#include "cupc_internal.cuh"

namespace cupc {

// Per-level counters of the fused level kernels (zeroed once per call).
constexpr int LV = CUPC_MAX_LEVEL + 2;
// Work items are dispatched in rounds: round c holds the c-th item (subset
// ranks [c chunk, (c + 1) chunk)) of every row that has one, for c < RND - 1;
// the last round holds every later item.
constexpr int RND = 64;
struct LevelMeta {
    unsigned long long tests[LV];          // CI tests executed
    unsigned long long rechecks[LV];       // FP64 rechecks performed
    unsigned long long removed[LV];        // edges removed
    unsigned long long serial[LV];         // serial-order test count (canonical runs)
    unsigned long long edges[LV];          // undirected edges at level start
    unsigned long long items[LV];          // CI work items
    unsigned long long next_item[LV];      // persistent work counter
    unsigned long long queue_len[LV];      // recheck entries pushed (may exceed capacity)
    unsigned long long block_entries[LV];  // sum over rows with work of (n'_i + 1)^2
    unsigned long long phase_ns[LV][4];    // compaction, CI, recheck, finalisation (wall ns)
    unsigned long long order_ns[LV][2];    // learned order: scoring, ranking (wall ns)
    unsigned long long recheck_ns[LV][3];  // recheck partial sums, combine (wall ns, all batches),
                                           // and block 0's own partial-sum work
    int maxdeg[LV];
    int chunk[LV];
    int learned_on[LV];                    // the level's rows enumerated in the network's order
    unsigned long long rec_ints;           // SepSet record ints appended
    int done_level;                        // level whose termination test stopped the loop
    int csr_level;                         // level whose A'_G arrays (cols, srow, partner, wpre) are current
    int csr_cur;                           // which of the two CSR buffers holds that level's A'_G
    int overflow_level;                    // level whose recheck queue overflowed
    int error;                             // 8: a grid barrier wait expired
    int range_error;                       // a subset count saturated 64 bits
    unsigned long long bar;                // grid barrier: arrivals (low 32 bits), generation (high 32)
    unsigned long long live[LV];           // queued tests rechecked (not decided already)
    unsigned long long rc_next[LV];        // recheck queue entries claimed by CTAs
    unsigned long long round_hist[LV][RND]; // rows by item count (bin 0: items past RND - 1)
    unsigned long long round_cur[LV][RND]; // slots of each round handed to CTAs so far
};

// One problem of a batch. The batch runs as one graph whose connected
// blocks are the problems: problem k owns the global vertex ids
// [off, off + P32) with P32 = p rounded up to 32 (ids past off + p are
// padding and stay isolated). Its adjacency is its own P32 x W bitset (W =
// P32 / 32 words a row) stored from word bw, so row v of the batch bitset
// starts at word rowbase(v) = bw + (v - off) W - wlo and the word holding
// global column c is rowbase(v) + (c >> 5), c >> 5 in [wlo, whi).
struct ProbDesc {
    int off, p, n;
    double inv_n;                  // 1 / n
    int wlo, whi;                  // off / 32, (off + P32) / 32
    int lmax;                      // last level its threshold allows (n - 4, max_level)
    long long bw;                  // first word of its bitset block
    long long c_off;               // its p x p correlation in the packed C
    long long z_off;               // its p x n standardised rows (FP64) in the packed rows
    long long x_off;               // its data (elements) in the packed input buffers
    const void* xs;                // its data as given (n x p, the batch's layout and type)
    const void* xv;                // its variable-major rows (ld = n)
    double r[LV], r2[LV];          // tanh(tau_l) for its n and alpha, and the square
};

// Problem of vertex v (nullptr descriptors: one problem, no batch).
__device__ __forceinline__ const ProbDesc* prob_of(const int* vprob, const ProbDesc* probs, int v)
{
    return vprob ? probs + vprob[v] : nullptr;
}

// Word offset such that bits[rowbase + (c >> 5)] holds column c of row v.
__device__ __forceinline__ long long rowbase(const ProbDesc* D, int W, int v)
{
    return D ? D->bw + (long long)(v - D->off) * (D->whi - D->wlo) - D->wlo : (long long)v * W;
}

// Parameters of one level (l >= 1) of the fused level kernel.
struct LevelParams {
    unsigned* bits;                // live A_G bitset, p rows of W words (batch: packed blocks)
    int W, p;
    long long nwords;              // words of the bitset
    int* deg;
    long long* row_off;            // p + 1 CSR offsets of A'_G
    long long* item_off;           // p + 1: items of the rows before each row (row-major count)
    int* item_row;                 // work items in dispatch order: the row of each
    int* item_c;                   // and the item's index within its row
    unsigned long long item_cap;
    int* cols;                     // neighbour indices (increasing per row)
    int* srow;                     // row of each slot
    int* partner;                  // slot of (j, i) for slot (i, j)
    // second CSR buffer: a level builds its A'_G from the previous level's
    // (the surviving slots, in order) into the other buffer
    long long* row_off2;
    int* cols2;
    int* srow2;
    int* partner2;
    unsigned char* alive;          // per slot of the current A'_G: 1 if its edge survived the level
    int* nrank;                    // per slot: position among its row's surviving slots, or -1
    int* wpre;                     // per row, neighbours below each 32-column word
    unsigned long long* best;      // smallest separating subset rank per slot
    unsigned long long nnz_cap;
    const void* C;                 // p x p correlation (float or double), ld = p
    Binom B;
    int chunk0;                    // preferred subset ranks per work item
    int jsplit;                    // level 1: a row's items also split its j positions in
                                   // ranges of 32 (graphs with too few rows to fill the GPU)
    int canonical;
    int l;
    double r, r2;                  // tanh(tau_l) and its square
    double band_abs, band_rel;     // FP32 mode: recheck band on |rho|
    double rank_tol;               // pivot^2 at or below which a member of S is dependent
    double piv_floor;              // FP32 mode: smaller pivot^2 sends the test to FP64
    QEntry* queue;
    unsigned long long qcap;
    const void* xv;                // variable-major data rows for the rechecks (or c64)
    long long ldx;
    int xf64;                      // element type of xv: 1 FP64, 0 FP32
    const double* mu;              // per variable: mean and 1/sd of the standardisation
    const double* isd;
    const float2* mup;             // the mean as an FP32 pair (FP32 data: compensated rechecks)
    int n;
    double inv_n;                  // 1 / n (one problem)
    int nmax;                      // batch: largest sample count
    const double* c64;
    double* part;                  // recheck partial Gram sums (tests x slices x D doubles)
    int* live;                     // qcap: queue positions of the tests rechecked
    int* rc_cnt;                   // kRcCnt: slices finished per rechecked test
    unsigned long long part_cap;   // doubles in part
    int* rec;                      // SepSet record pool (int32 groups i, j, l, S...)
    unsigned long long rec_cap;
    LevelMeta* lm;
    int* host_flags;               // device view of pinned host flags: [l] = 1 runs, 2 loop ended
    // batch: problem of each global vertex, and the problems (nullptr: one problem)
    const int* vprob;
    const ProbDesc* probs;
    const int* vlmax;              // batch: the last level of each vertex's problem
    unsigned long long* prob_serial;   // batch: serial-order tests per problem and level (nprob x LV)
    int ctas_per_sm;               // launch shape (0: as many as fit, at most 2)
    unsigned long long* scan_part; // per CTA: CSR slots, items
    const Meta* meta0;             // level 0's counters: a level does not run after an error
    unsigned long long qcap0;      // there, or an overflow of its recheck queue
    // learned ordering (levels >= 1, FP32 mode): each row of A'_G enumerated in
    // descending network score (nnz_cap entries each)
    int learned;                   // requested
    const void* mlp_w;             // bf16 network parameters
    int* perm;                     // perm[off_i + v]: row position of the row's v-th candidate
    int* iperm;                    // iperm[off_i + c]: order position of row position c
    int* vrank;                    // old slot -> order position in its new row (incremental A'_G)
    float* lscore;                 // per slot: the network's score of the candidate
    float* lrsum;                  // per row: sum of |C_ij| over the row's neighbours
    // level 1 by conditioning variable: row k of C staged in shared memory
    unsigned barrier_ns;           // 0: grid-barrier waits end after kBarrierNs; else a test of
                                   // the expiry path: CTA 0 withholds its arrival at the first
                                   // barrier and the others give up after this many ns
    int l1_pivot;                  // level 1 runs phase_l1_pivot with this many row buffers
                                   // (2: the next row is copied while one is tested), 0: off
    int pstage;                    // entries of the longest staged row (largest problem's p)
    void* cval;                    // nnz_cap entries (T): C_ij of each CSR slot (i, j)
};

// Level 1 by conditioning variable (a staged C row per pivot) or by row (S
// shared across j, C gathered through the caches), for the level1_form
// option. CUPC_L1_AUTO takes the row form: on GB300 it was the faster one on
// every workload measured (p = 10^3 to 10^4, and the 64-problem batch), while
// the pivot form reads each C row from HBM once (5x less DRAM at p = 10^4) but
// issues more instructions per visited slot.
inline bool level1_by_pivot(int form)
{
    return form == CUPC_L1_BY_PIVOT;
}

// Tests of a level whose FP64 recheck may be cut into slices over several CTAs.
constexpr int kRcCnt = 4096;

// Shared memory the level-1 pivot form may use for its staged C rows.
constexpr int kL1StageBytes = 96 * 1024;
// Bytes of one staged-row buffer for rows of up to pstage entries of es bytes
// (room for the row shifted by its misalignment, a multiple of 16).
__host__ __device__ inline size_t l1_buf_bytes(int pstage, int es)
{
    return ((size_t)(pstage + 16 / es) * es + 15) & ~(size_t)15;
}
// Row buffers the level-1 pivot form can use (0: rows too long to stage).
inline int l1_buffers(int pstage, int es)
{
    const size_t b = l1_buf_bytes(pstage, es);
    return 2 * b <= (size_t)kL1StageBytes ? 2 : b <= (size_t)kL1StageBytes ? 1 : 0;
}

// Parameters of the level-0 FP64 recheck.
struct Recheck0Params {
    const void* xv;                // variable-major data rows, their stride and type
    long long ldx;
    int xf64;
    const double* mu;
    const double* isd;
    const float2* mup;             // the mean as an FP32 pair (FP32 data)
    int n;
    double inv_n;
    const double* c64;
    int p;
    double r2;
    const QEntry* queue;
    unsigned long long qcap;
    Meta* meta;
    unsigned* bits;
    int W;
    const int* vprob;              // batch: problem of each vertex (nullptr: one problem)
    const ProbDesc* probs;
};

cudaError_t launch_transpose(int dtype, const void* X, long long ld, int n, int p, void* Xt, cudaStream_t st);
cudaError_t launch_standardize(int dtype, const void* Xv, long long ld, int n, int p, double* mu, double* isd,
                               float2* mup, double* z64, long long ldz, void* zhi, void* zlo, long long ldb,
                               Meta* meta, cudaStream_t st, const int* vprob = nullptr,
                               const ProbDesc* probs = nullptr);
cudaError_t launch_transpose_batch(int dtype, const ProbDesc* probs, int nprob, int pmax, int nmax, void* Xt,
                                   cudaStream_t st);
cudaError_t launch_syrk_f64(const double* Z, long long ldz, int n, int p, double* C, cudaStream_t st);
void corr_tc_plan(int p, long long ldk, int num_sms, int* tiles, int* nsplit, int* kps, size_t* ws_bytes);
cudaError_t launch_corr_tc(const void* hi, const void* lo, long long ldk, int p, int n, float* ws, float* C,
                           int num_sms, int* err, cudaStream_t st);
// Batched correlation: host-side plan (work units and output tiles, copied to
// the device by the caller) and the launch.
struct CorrBatchUnit {
    int ra, rb, g0, g1, kt, slot, prob, pad0;   // slot -1: the unit writes its tile of C
};
struct CorrBatchTile {
    int prob, bi, bj, slot0, nsplit, pad0, pad1, pad2;
};
void corr_tc_batch_plan(const std::vector<ProbDesc>& probs, int num_sms, int kps_req,
                        std::vector<CorrBatchUnit>& units, std::vector<CorrBatchTile>& tiles, size_t* ws_bytes,
                        int* kps_out);
cudaError_t launch_corr_tc_batch(const void* hi, const void* lo, long long ldk, int rows, const void* units,
                                 int n_units, const void* tiles, int n_tiles, const ProbDesc* probs, float* ws,
                                 float* C, int num_sms, int* err, cudaStream_t st);
cudaError_t launch_symmetrize(int dtype, const void* Cin, long long ld, int p, double* C64, float* C32,
                              cudaStream_t st);

cudaError_t launch_level0(int fp32, const void* C, int p, int W, double r0, double band0, unsigned* bits,
                          QEntry* q, unsigned long long qcap, Meta* meta, cudaStream_t st,
                          const int* vprob = nullptr, const ProbDesc* probs = nullptr, int nrows = 0);
cudaError_t launch_degree(const unsigned* bits, int p, int W, int* deg, Meta* meta, cudaStream_t st,
                          const int* vprob = nullptr, const ProbDesc* probs = nullptr);
cudaError_t launch_recheck0(const Recheck0Params& P, int grid, cudaStream_t st);
// One fused level kernel (cooperative launch). *grid receives the grid used.
cudaError_t launch_level(int fp32, const LevelParams& P, int num_sms, cudaStream_t st);
cudaError_t launch_pcor(int fp32, const void* C, int p, const int* q, long long nq, int l, double* rho,
                        cudaStream_t st);
// rho of (i, j, S) queries with the FP64 recheck arithmetic (data rows and
// moments in P; P.l = |S|).
cudaError_t launch_pcor_recheck(const LevelParams& P, const int* q, long long nq, double* rho, cudaStream_t st);
cudaError_t launch_bits_to_u8(const unsigned* bits, int p, int W, unsigned char* out, cudaStream_t st);

// global sharing of conditioning sets at one level (k_sshare.cu)
cudaError_t launch_sshare(const long long* off, const int* cols, const long long* pre, int nrows, int l, int bits,
                          const Binom& B, unsigned long long total, unsigned long long* keys, unsigned* cnt,
                          unsigned long long slots, const long long* bins, int nbins, unsigned long long* out,
                          int* err, int num_sms, cudaStream_t st);

// candidate-scoring network (k_mlp.cu)
cudaError_t launch_mlp_grad(const float* P, const float* X, const float* T, long long s0, long long s1, float* gpart,
                            float* lpart, int blocks, cudaStream_t st);
cudaError_t launch_mlp_apply(float* P, float* M, float* V, const float* gpart, int nblocks, float* gsum, int step,
                             float lr, void* Pb, cudaStream_t st);
cudaError_t launch_mlp_to_bf16(const float* P, void* Pb, cudaStream_t st);
cudaError_t launch_mlp_forward(const void* Pb, const float* X, long long N, float* y, cudaStream_t st);
cudaError_t launch_mlp_examples(const float* C, long long p, const int* nbs, const int* q, long long n, float* X,
                                float* t, cudaStream_t st);


}  // namespace cupc
