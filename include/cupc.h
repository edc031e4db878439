/*
 * cupc.h -- C ABI of the GB300 (sm_103a) PC-stable skeleton library.
 *
 * The library computes the first step of the order-independent PC algorithm
 * (PC-stable) for multivariate-normal data: the correlation matrix of the
 * data, then level by level the Gaussian conditional-independence tests on
 * partial correlations, edge removal and SepSet recording (paper: Zarebavani,
 * Jafarinejad, Hashemi, Salehkaleybar, "cuPC: CUDA-based Parallel PC Algorithm
 * for Causal Structure Learning on GPU", IEEE TPDS 2019; Algorithm 1, Algorithm
 * 2, Sec. 4.3). The problem statement follows Sec. 1 and Sec. 4.3: m samples of
 * n variables, no missing values, significance level alpha; outputs are the
 * skeleton G and the separating sets (SepSet). (In this header p = number of
 * variables, n_samples = number of samples.)
 *
 * Conventions for every entry point:
 *  - Return value: a cupc_status. No entry point aborts or exits. After an
 *    error the context stays usable; cupc_last_error() gives a message.
 *  - Pointers: plain host or device pointers as stated per argument; no
 *    framework types. Inputs are borrowed for the duration of the call only.
 *  - Device memory: the library allocates its own workspace and result storage
 *    with stream-ordered allocation on the context's stream; results own their
 *    storage until cupc_result_free().
 *  - Streams: all GPU work runs on the stream given to cupc_create() (or
 *    cupc_set_stream()). Calls that return results synchronise that stream.
 *  - Threads: a context must not be used by two host threads at once.
 */
#ifndef CUPC_H
#define CUPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CUPC_MAX_LEVEL 16        /* largest conditioning-set size the kernels support */
#define CUPC_STATS_LEVELS 24     /* per-level statistics slots */
#define CUPC_KCLASSES 8          /* kernel classes timed in cupc_stats.kernel_ms */

/* kernel classes (index into cupc_stats.kernel_ms / kernel_count) */
enum {
    CUPC_K_UPLOAD = 0,       /* host-to-device copy of the input */
    CUPC_K_STANDARDIZE = 1,  /* layout transpose + FP64 moments + standardised rows */
    CUPC_K_CORRELATION = 2,  /* the correlation product C = Z Z^T / n */
    CUPC_K_LEVEL0 = 3,       /* level-0 tests (+ their FP64 rechecks) */
    CUPC_K_COMPACT = 4,      /* A_G -> A'_G compaction and work-item planning */
    CUPC_K_CI = 5,           /* the CI-test kernel of levels >= 1 */
    CUPC_K_RECHECK = 6,      /* FP64 rechecks of levels >= 1 */
    CUPC_K_FINALIZE = 7      /* edge removal and SepSet records */
};

typedef enum {
    CUPC_OK = 0,
    CUPC_E_INVALID = -1,     /* bad argument (sizes, alpha, layout, null pointer) */
    CUPC_E_NOMEM = -2,       /* device allocation failed */
    CUPC_E_CUDA = -3,        /* a CUDA runtime call or kernel failed */
    CUPC_E_TIMEOUT = -4,     /* a bounded device-side wait gave up */
    CUPC_E_RANGE = -5,       /* a level or subset count beyond the supported range */
    CUPC_E_NUMERIC = -6,     /* non-finite data (NaN/Inf, zero variance) */
    CUPC_E_CANCELLED = -7,   /* cancelled between levels */
    CUPC_E_STATE = -8        /* entry point not valid in the current state */
} cupc_status;

/* element types */
enum { CUPC_F32 = 0, CUPC_F64 = 1 };

/* data layouts for X (n_samples x p):
 *   SAMPLE_MAJOR:   element (s, v) at X[s * ld + v], ld >= p (C order, rows are samples)
 *   VARIABLE_MAJOR: element (s, v) at X[v * ld + s], ld >= n_samples (Fortran/R order) */
enum { CUPC_LAYOUT_SAMPLE_MAJOR = 0, CUPC_LAYOUT_VARIABLE_MAJOR = 1 };

/* arithmetic of the CI tests */
enum {
    CUPC_MODE_PLAIN_FP64 = 0,    /* FP64 correlation, FP64 CI tests for every test */
    CUPC_MODE_FP32_RECHECK = 1   /* FP32 bulk tests; tests within a margin of the
                                    threshold are recomputed in FP64 on the GPU */
};

typedef struct {
    int mode;                /* CUPC_MODE_* (default CUPC_MODE_FP32_RECHECK) */
    int canonical_sepset;    /* 1: store the first separating set in serial order
                                (smaller endpoint's side first, lexicographic within
                                a side); 0: any separating set found first (default 1) */
    int learned_order;       /* 1: enumerate subsets in the order given by the
                                candidate-scoring network loaded with
                                cupc_mlp_set_weights() (levels >= 1); default 0 */
    int max_level;           /* last level to run; -1 = until no edge has enough
                                neighbours (Algorithm 1 termination); default -1 */
    double recheck_margin;   /* FP32 mode: absolute band on |rho| around tanh(tau)
                                that is recomputed in FP64; <= 0 selects the
                                built-in default */
    int threads_per_block;   /* CI kernel block size (0 = tuned default) */
    int chunk;               /* subsets per work item in the CI kernel (0 = default) */
    int ctas_per_sm;         /* CTAs per SM of the fused level kernel (0 = as many as
                                fit, at most 2) */
    int corr_kps;            /* batch: K steps per work unit of the batched
                                tensor-core product (0 = chosen by its cost model) */
    int batch_direct;        /* batch: 1 = launch the kernels directly instead of
                                capturing and replaying a CUDA graph (default 0) */
    int test_qcap;           /* testing (single-problem calls): when > 0, the initial
                                capacity of the FP64 recheck queue, in entries */
    int test_nnz_cap;        /* testing: when > 0, the initial capacity of A'_G in
                                slots (twice the edges of the densest level) */
    int test_rec_cap;        /* testing: when > 0, the initial capacity of the SepSet
                                record pool, in int32 */
    int level1_form;         /* how level 1 runs its tests (same results either way):
                                CUPC_L1_AUTO (default) lets the library choose (the
                                row form, measured faster on GB300 on every workload
                                of 10^3 to 10^4 variables and on batches);
                                CUPC_L1_BY_PIVOT walks, for each conditioning variable
                                k, the rows of k's neighbours with row k of C staged
                                in shared memory (every C row read once; needs the
                                row to fit 96 KB of shared memory, else as
                                CUPC_L1_BY_ROW); CUPC_L1_BY_ROW shares each subset
                                {k} of a row across its j and gathers C entries
                                through the caches */
    int host_lists;          /* 1: the call also builds the skeleton's edge list and
                                its SepSet records in (i, j) order on the device and
                                downloads them with its final readback (after the
                                levels' timing ends), so that cupc_result_edges and
                                cupc_result_sepset_records only copy host memory;
                                0 (default): each is built on its first request */
} cupc_options;
enum { CUPC_L1_AUTO = 0, CUPC_L1_BY_PIVOT = 1, CUPC_L1_BY_ROW = 2 };
/* The three test capacities exist to exercise the recovery paths: a level
 * whose buffer would overflow reports it, the buffer is enlarged and the
 * affected levels run again (cupc_stats.reruns counts the reruns by cause).
 * The result is the same as with the default capacities. */

typedef struct {
    int levels;                                  /* levels run, level 0 included */
    int64_t tests[CUPC_STATS_LEVELS];            /* CI tests executed on the GPU */
    int64_t serial_tests[CUPC_STATS_LEVELS];     /* tests the serial algorithm performs
                                                    (canonical lexicographic runs only,
                                                    else -1) */
    int64_t removed[CUPC_STATS_LEVELS];          /* edges removed at each level */
    int64_t rechecks[CUPC_STATS_LEVELS];         /* FP64 rechecks (FP32 mode) */
    int64_t edges_start[CUPC_STATS_LEVELS];      /* undirected edges at level start */
    int32_t max_degree[CUPC_STATS_LEVELS];       /* max degree at level start */
    float level_ms[CUPC_STATS_LEVELS];           /* device time of each level */
    float prep_ms;                               /* upload + standardise + correlation */
    float total_ms;                              /* device time of the whole call */
    int64_t edges_final;                         /* undirected edges in the skeleton */
    int64_t kernel_launches;                     /* kernels launched by the call */
    int64_t h2d_bytes, d2h_bytes;                /* bytes copied by the call */
    float kernel_ms[CUPC_KCLASSES];              /* device time per kernel class (CUDA events) */
    int32_t kernel_count[CUPC_KCLASSES];         /* launches per kernel class */
    int64_t ci_block_entries[CUPC_STATS_LEVELS]; /* sum over rows of (n'_i + 1)^2: the C
                                                    sub-block entries a level's tests read */
    float phase_ms[CUPC_STATS_LEVELS][4];        /* per level >= 1, wall time of its phases:
                                                    compaction, CI tests, FP64 rechecks,
                                                    removal + SepSets (device clock) */
    int32_t cuda_graph;                          /* batch: 1 if the device work ran as a
                                                    replayed CUDA graph, 0 if launched
                                                    directly; single calls: 0 */
    float recheck_ms[CUPC_STATS_LEVELS][3];      /* per level >= 1, the FP64 recheck phase
                                                    split into partial sums and combine,
                                                    and the first CTA's own partial sums
                                                    (device clock) */
    int64_t rechecks_queued[CUPC_STATS_LEVELS];  /* tests queued for the FP64 recheck (those
                                                    whose outcome could no longer matter are
                                                    skipped; rechecks counts the rest) */
    int32_t reruns[4];                           /* single calls: levels run again after a
                                                    buffer overflowed: [0] level 0's recheck
                                                    queue, [1] A'_G's slots, [2] the SepSet
                                                    pool, [3] a level >= 1 recheck queue */
    float order_ms[CUPC_STATS_LEVELS][2];        /* learned order, per level >= 1: scoring
                                                    the candidates and ranking them (device
                                                    clock, within the compaction phase; 0
                                                    where the level scored nothing) */
    float host_ms[2];                            /* wall time of the call on the host: [0]
                                                    from entry until its device work (and
                                                    the downloads it asked for) finished,
                                                    [1] building the result objects after */
} cupc_stats;

typedef struct cupc_ctx cupc_ctx;
typedef struct cupc_result cupc_result;

/* Fills *o with the defaults documented above. The options are the library's
 * own; the paper's inputs are only the data and alpha (Sec. 1, Sec. 4.3). */
void cupc_options_default(cupc_options* o);

/* Creates a context on CUDA device `device`. `stream` is a cudaStream_t (may be
 * NULL for the legacy default stream; a framework's stream handle may be passed).
 * The device must be sm_103 (GB300); otherwise CUPC_E_CUDA. Resource
 * management only: the paper has no counterpart (its program owns one GPU and
 * its buffers for the whole run, Sec. 5.1). */
cupc_status cupc_create(cupc_ctx** out, int device, void* stream);

/* Changes the stream subsequent calls use. The paper has no counterpart. */
cupc_status cupc_set_stream(cupc_ctx* ctx, void* stream);

/* Frees the context and its workspace. Results stay valid. The paper has no
 * counterpart. */
void cupc_destroy(cupc_ctx* ctx);

/* Requests that the call running on this context (from another host thread),
 * or the next call, stop between levels: it waits for the work already on the
 * GPU, frees its partial result and returns CUPC_E_CANCELLED; the context
 * stays usable. The request is consumed by the call it stops. Safe to call
 * from any thread. The paper has no counterpart (its runs are not
 * interruptible). */
cupc_status cupc_cancel(cupc_ctx* ctx);

/* Host-side fault injection for tests of the error paths (the paper has no
 * counterpart). kind:
 *   CUPC_FAIL_ALLOC    the k-th next device allocation of a skeleton call fails
 *                      (CUPC_E_NOMEM, nothing allocated);
 *   CUPC_FAIL_LAUNCH   the k-th next kernel launch of a skeleton call fails
 *                      (CUPC_E_CUDA, nothing launched);
 *   CUPC_FAIL_BARRIER  in the next skeleton call, the first level kernel's
 *                      CTA 0 never arrives at its first grid barrier and the
 *                      other CTAs give up waiting there after k ns (1e3 <= k
 *                      <= 1e9) instead of 2 s: the wait runs out, no CTA
 *                      passes that barrier, and the call returns
 *                      CUPC_E_TIMEOUT;
 *   CUPC_FAIL_NONE     disarms.
 * A failure fires once and disarms. The call that meets it returns the error
 * with no result; the context stays usable. */
enum { CUPC_FAIL_NONE = 0, CUPC_FAIL_ALLOC = 1, CUPC_FAIL_LAUNCH = 2, CUPC_FAIL_BARRIER = 3 };
cupc_status cupc_debug_fail(cupc_ctx* ctx, int kind, int64_t k);

/* Message for the last error on this context ("" if none). Never NULL. The
 * paper has no counterpart. */
const char* cupc_last_error(const cupc_ctx* ctx);

/* Algorithm 1 / Algorithm 2 on data: standardise X in FP64, form the
 * correlation matrix C (Sec. 4.3), run level 0 (Algorithm 3) and every level
 * l >= 1 (compaction of A_G, CI tests of Sec. 4.3, edge removal, SepSet) until
 * the termination rule or opts->max_level.
 *   X          host (on_device = 0) or device (on_device = 1) pointer to the
 *              n_samples x p data, element type `dtype` (CUPC_F32/CUPC_F64),
 *              laid out per `layout` with leading dimension `ld`.
 *   n_samples  number of samples m; must exceed max_level + 3 (Eq. threshold).
 *   p          number of variables, 2 <= p <= 2^20.
 *   alpha      significance level, 0 < alpha < 1.
 *   opts       NULL for defaults.
 *   out        receives a new result (free with cupc_result_free).
 * Errors: CUPC_E_INVALID (arguments), CUPC_E_NUMERIC (a variable with zero
 * variance or non-finite data), CUPC_E_RANGE (a level above CUPC_MAX_LEVEL would
 * be needed or a subset count exceeds 2^63), CUPC_E_NOMEM, CUPC_E_CUDA,
 * CUPC_E_TIMEOUT. On error *out is NULL. */
cupc_status cupc_skeleton(cupc_ctx* ctx, const void* X, int dtype, int layout, int on_device,
                          int64_t n_samples, int64_t p, int64_t ld, double alpha,
                          const cupc_options* opts, cupc_result** out);

/* Same as cupc_skeleton but from a p x p correlation matrix C (row-major with
 * leading dimension ld, host or device, CUPC_F32 or CUPC_F64) -- the
 * "sufficient statistics" form of the pcalg interface the paper mirrors
 * (Sec. 5.1). The diagonal is taken as exactly 1 and only the upper triangle is
 * read (the matrix is symmetrised from it). The matrix is widened to FP64 on
 * the device; in FP32 mode the bulk tests read its FP32 rounding and the
 * rechecks read the FP64 copy. */
cupc_status cupc_skeleton_corr(cupc_ctx* ctx, const void* C, int dtype, int on_device, int64_t p,
                               int64_t ld, int64_t n_samples, double alpha,
                               const cupc_options* opts, cupc_result** out);

/* ---------------------------------------------------------------------------
 * Batches of independent problems (the paper runs one problem per call; this
 * is the library's own addition for many small and mid-size problems).
 * Problem k has data X[k] (n_samples[k] x p[k], element type `dtype`, layout
 * `layout`, dense: ld = p[k] for SAMPLE_MAJOR, n_samples[k] for
 * VARIABLE_MAJOR; host pointers, or device pointers with on_device = 1) and
 * significance level alpha[k]. The problems run together as one graph whose
 * connected blocks are the problems: one standardisation launch, one
 * tensor-core launch over every problem's output tiles, one level-0 launch,
 * and per level l >= 1 one fused level kernel whose work queue holds the
 * (row, subset-rank chunk) items of all problems. Level l runs while any
 * problem still has an edge with enough neighbours; a problem whose threshold
 * (n - l - 3 > 0) or opts->max_level ends earlier takes no work from then on.
 * Each problem's skeleton and SepSets are exactly those of cupc_skeleton on
 * it alone with the same options.
 * The device work of a call is captured as a CUDA graph on the first call
 * with a given set of shapes, alphas and options, and replayed by later calls
 * with the same ones (opts->batch_direct = 1 launches it directly instead);
 * the context keeps one such plan and its buffers until the shapes change or
 * the context is destroyed. The call runs on a stream of its own, ordered
 * after the work already queued on the context stream, and returns when the
 * results are on the host.
 *   nprob        number of problems, 1 <= nprob <= 4096; sum of p[k] rounded up
 *                to 32 at most 2^20.
 *   opts         NULL for defaults; mode must be CUPC_MODE_FP32_RECHECK and
 *                learned_order 0.
 *   out          array of nprob result pointers, each a new result (free each
 *                with cupc_result_free). Their stats hold per problem:
 *                serial_tests (canonical runs), removed, edges_start,
 *                edges_final and levels; tests and rechecks per problem are -1.
 *   batch_stats  NULL, or receives the whole batch's counters and timings:
 *                total_ms = device time from the input copies to the end of
 *                the last level; kernel_ms[UPLOAD], [STANDARDIZE],
 *                [CORRELATION], [LEVEL0] the stages (event-timed, the level-0
 *                stage includes its rechecks and the degree pass); prep_ms
 *                standardisation + correlation; level_ms[1] every level >= 1
 *                together; phase_ms per level from the device clock.
 * Errors as cupc_skeleton; on error every out[k] is NULL. */
cupc_status cupc_skeleton_batch(cupc_ctx* ctx, int nprob, const void* const* X, int dtype, int layout,
                                int on_device, const int64_t* n_samples, const int64_t* p,
                                const double* alpha, const cupc_options* opts, cupc_result** out,
                                cupc_stats* batch_stats);

/* One launch configuration tried by the batch autotuner and its time. */
typedef struct {
    int chunk;          /* subsets per work item */
    int ctas_per_sm;    /* CTAs per SM of the level kernel */
    int corr_kps;       /* K steps per unit of the batched product (resolved, > 0) */
    float ms;           /* best device time of the batch over the repetitions */
} cupc_tune_entry;

/* Autotuner for batches: runs the batch described as in cupc_skeleton_batch
 * once per candidate configuration (chunk in {8, 16, 32, 64, 128} x CTAs per SM
 * in {1, 2} x product K-steps in {cost model, half, double}), each `reps`
 * times (1 <= reps <= 16), and writes up to `cap` entries into `entries`,
 * fastest first (*n_entries = number written). Every candidate must give the
 * same skeleton and the same SepSets; otherwise CUPC_E_STATE. The caller
 * stores the winner (e.g. in a table keyed by the batch's shape class) and
 * passes it through opts->chunk, opts->ctas_per_sm and opts->corr_kps. */
cupc_status cupc_batch_autotune(cupc_ctx* ctx, int nprob, const void* const* X, int dtype, int layout,
                                int on_device, const int64_t* n_samples, const int64_t* p,
                                const double* alpha, const cupc_options* base, int reps,
                                cupc_tune_entry* entries, int cap, int* n_entries);

/* Measured arithmetic peaks of the context's device, in TFLOP/s (2 flops per
 * fused multiply-add): FP64 and FP32 FMA throughput of a grid filling every SM
 * with four independent FMA chains per thread, best of three timed launches.
 * They are the denominators of the rooflines of ALU-bound kernels (the FP64
 * rechecks, the plain form's FP64 standardisation). The paper has no
 * counterpart. Synchronises the context stream. */
cupc_status cupc_device_peaks(cupc_ctx* ctx, double* fp64_tflops, double* fp32_tflops);

/* Number of variables of a result (the n of the paper's problem statement,
 * Sec. 1: the vertices of G). */
cupc_status cupc_result_p(const cupc_result* res, int64_t* p);

/* Counts of one orientation (cupc_result_orient). */
typedef struct {
    int64_t rounds;          /* rounds of Meek's rules run; the last one changed nothing */
    int64_t directed;        /* edges with an arrowhead at exactly one end */
    int64_t undirected;      /* edges with no arrowhead */
    int64_t bidirected;      /* edges two v-structures disagree on (arrowheads at both ends) */
    int64_t rule_conflicts;  /* edges a round proposed both ways (left undirected that round) */
    float ms;                /* device time from the neighbour lists to the marks (CUDA events) */
    int32_t reserved;
} cupc_orient_stats;

/* The second step of PC-stable (Sec. 2.4): the v-structures of Sec. 2.2 read
 * off the result's skeleton and SepSets, then Meek's orientation rules R1-R3,
 * giving the CPDAG of Sec. 2.2. Runs on the device (k_orient.cu).
 *   marks  host buffer of p*p bytes (caller-owned; NULL: counts only), row-major:
 *          marks[a*p + b] = 0 when a and b are not adjacent, 1 when the edge
 *          a - b has an arrowhead at b, 2 when it has a tail at b; so a -> b
 *          is (1, 2) at ([a][b], [b][a]), a - b is (2, 2), and an edge two
 *          v-structures disagree on is (1, 1).
 *   stats  may be NULL.
 * Readings (the paper names the step only): every unshielded triple
 * i - k - j (i, j not adjacent) with k outside SepSet(i, j) is a v-structure,
 * all of them applied together; the rules run in rounds that decide from the
 * marks at the start of the round and apply all their orientations together,
 * until a round changes nothing; an edge proposed both ways in a round stays
 * undirected; only undirected edges are oriented, and only directed edges
 * count as arrows in the rules' premises. Given the skeleton and the SepSets,
 * the marks do not depend on the order in which triples or edges are visited
 * (the SepSets themselves are the canonical ones of the serial order in
 * canonical mode, and any separating sets otherwise, so the marks equal the
 * oracle's for canonical results). Device scratch comes from the context's
 * pool; the result itself is not changed. Synchronises the context stream
 * once per round.
 * Errors: CUPC_E_INVALID (NULL result), CUPC_E_STATE (a result without its
 * skeleton or SepSet records), CUPC_E_NOMEM, CUPC_E_CUDA. */
cupc_status cupc_result_orient(cupc_result* res, uint8_t* marks, cupc_orient_stats* stats);

/* The skeleton G that Algorithm 1 returns (Sec. 2.4; the adjacency matrix A_G
 * of Algorithm 2 and Sec. 3, at the end of the last level) as a p x p uint8 matrix (1 = edge)
 * in the host buffer `out` (caller-owned, p*p bytes). Synchronises the context
 * stream. */
cupc_status cupc_result_adjacency(const cupc_result* res, uint8_t* out);

/* The skeleton G that Algorithm 1 returns (Sec. 2.4), as an edge list: pairs
 * (i, j) with i < j in increasing (i, j) order, written to out[2k] and
 * out[2k + 1] (host buffer, caller-owned, room for `cap` pairs); *n_edges =
 * the number of edges. With out == NULL only *n_edges is set. The list is
 * built once per result (on the device for a single call's result, downloaded
 * in one copy; from the host bitset for a batch result) and kept until
 * cupc_result_free. */
cupc_status cupc_result_edges(const cupc_result* res, int32_t* out, int64_t cap, int64_t* n_edges);

/* Copies, into the host buffer `out` (p*p int16), the level at which each pair
 * was removed (|S| of its SepSet, Algorithm 1), or -1 where the edge is present
 * (the diagonal is -1). */
cupc_status cupc_result_sep_levels(const cupc_result* res, int16_t* out);

/* SepSet(V_i, V_j) that Algorithm 1 stores when it removes the edge (the
 * second output of the skeleton phase, Sec. 2.4): writes the members
 * (increasing) to out[0..*len)
 * (caller-owned, at least CUPC_MAX_LEVEL entries) and the size to *len;
 * *len = -1 when the edge is present. Level-0 removals have *len = 0. */
cupc_status cupc_result_sepset(const cupc_result* res, int64_t i, int64_t j, int32_t* out, int* len);

/* The SepSets of Algorithm 1 (Sec. 2.4) for every removal at level >= 1, as
 * consecutive int32 groups
 * (i, j, l, S[0..l)) with i < j, sorted by (i, j). With out == NULL only
 * *n_ints is set; otherwise at most `cap` ints are written. The sorted records
 * are built once per result (put in order on the device, or on the host when
 * the result's counts do not allow it) and kept until cupc_result_free. */
cupc_status cupc_result_sepset_records(const cupc_result* res, int32_t* out, int64_t cap,
                                       int64_t* n_ints);

/* Level-boundary checkpoint of a single-problem result (the state between
 * two levels of Algorithm 2: A_G after the result's last level, A_G after
 * level 0, the SepSet records so far, the per-level counters, and p, n, alpha
 * and the options the levels ran with), as an opaque, versioned host byte
 * buffer. A run stopped after level k (opts->max_level = k) and resumed from
 * its checkpoint with cupc_skeleton_resume gives the skeleton, SepSets and
 * counters of the uninterrupted run. With buf == NULL only *size is set;
 * otherwise cap must be at least *size (else CUPC_E_RANGE). CUPC_E_STATE for
 * a batch result. The paper has no counterpart (its pcalg-style interface,
 * Sec. 5.1, runs to completion). */
cupc_status cupc_result_checkpoint(const cupc_result* res, void* buf, int64_t cap, int64_t* size);

/* Continues a run from a checkpoint: the same data (arguments as in
 * cupc_skeleton; the correlation matrix is recomputed from it, deterministically)
 * and the same alpha and options (mode, canonical_sepset, learned_order; and
 * the same network weights for the learned order), with opts->max_level = -1
 * or >= the checkpoint's level. Runs the levels after the checkpoint's last
 * one and returns a full result (counters of the checkpoint's levels
 * included). The data itself is not checked against the checkpoint: the
 * caller passes the data the checkpoint was taken on. CUPC_E_INVALID for a
 * malformed checkpoint or one of another problem or options. */
cupc_status cupc_skeleton_resume(cupc_ctx* ctx, const void* X, int dtype, int layout, int on_device,
                                 int64_t n_samples, int64_t p, int64_t ld, double alpha,
                                 const cupc_options* opts, const void* ckpt, int64_t ckpt_size,
                                 cupc_result** out);

/* Global sharing of conditioning sets at one level (Sec. 5.5, Fig. 9): on the
 * result's A'_G at the start of `level` (1 <= level <= 4; its skeleton plus the
 * pairs it removed at that level or later), every level-subset S of adj(i) of
 * each row i that runs tests there (|adj(i)| >= level + 1) is counted once per
 * row. counts[k] (host, nbins entries) receives the number of distinct sets S
 * that appear in at least bins[k] and fewer than bins[k + 1] rows (the last bin
 * has no upper end; bins increasing, bins[0] >= 1). The library shares S within
 * a row only (as the paper's cuPC-S does); stats (may be NULL) gives what a
 * global search would find and cost: pairs (row, S) -- one factorisation each
 * with row-local sharing --, distinct sets -- one each with global sharing --,
 * sets in two rows or more, the largest row count, the rows, and search_ms,
 * the device time of the search itself (a hash table over all pairs, then the
 * histogram). Synchronises the context stream. Errors: CUPC_E_INVALID,
 * CUPC_E_RANGE (level, p beyond 65535 with level > 2, or more than 2^28
 * pairs), CUPC_E_CUDA. */
typedef struct {
    int64_t pairs;
    int64_t distinct;
    int64_t redundant;
    int64_t max_rows;
    int64_t rows;
    float search_ms;
    int32_t reserved;
} cupc_sshare_stats;
cupc_status cupc_result_sshare(const cupc_result* res, int level, const int64_t* bins, int nbins,
                               int64_t* counts, cupc_sshare_stats* stats);

/* Per-level statistics of the call that produced `res`: the test counts of
 * Algorithm 1 in serial order (the paper's Fig. 2 count convention), tests
 * executed, removals, device times. The paper reports runtimes only (Sec. 5.3);
 * the counters are the library's own. */
cupc_status cupc_result_stats(const cupc_result* res, cupc_stats* out);

/* Frees a result (NULL is ignored). The paper has no counterpart. */
void cupc_result_free(cupc_result* res);

/* ---------------------------------------------------------------------------
 * Building blocks exposed for verification (same kernels as the skeleton path).
 * ------------------------------------------------------------------------- */

/* Correlation matrix (Sec. 4.3) of X into the device buffer C_out (p x p,
 * row-major, ld = p): precision CUPC_F64 uses the FP64 standardisation and the
 * FP64 product; CUPC_F32 the FP64 standardisation and the split-precision
 * tensor-core product with FP32 accumulation. Arguments for X as in
 * cupc_skeleton. */
cupc_status cupc_correlation(cupc_ctx* ctx, const void* X, int dtype, int layout, int on_device,
                             int64_t n_samples, int64_t p, int64_t ld, int precision, void* C_out);

/* Partial correlations rho(V_i, V_j | S) (Sec. 4.3, Eqs. PartialCorMat and
 * RhoCal) for nq queries from the device correlation matrix C (p x p, ld = p,
 * element type `dtype`), evaluated with the CI kernels' device arithmetic in
 * that precision. `queries` is a device int32 array of nq rows (i, j, S[0..l)).
 * rho_out is a device double array of nq entries (NaN when the conditional
 * variance is not positive). */
cupc_status cupc_pcor_batch(cupc_ctx* ctx, const void* C, int dtype, int64_t p,
                            const int32_t* queries, int64_t nq, int l, double* rho_out);

/* Partial correlations rho(V_i, V_j | S) (Sec. 4.3, Eqs. PartialCorMat and
 * RhoCal) for nq queries, evaluated from the data X with the arithmetic of the
 * FP64 rechecks: the moments of the standardisation, the Gram sums of the
 * centred data over the l + 2 variables (FP64 for FP64 data, compensated FP32
 * pairs for FP32 data), then the FP64 elimination of S. X as in cupc_skeleton
 * (host or device); `queries` is a device int32 array of nq rows
 * (i, j, S[0..l)); rho_out a device double array of nq entries (NaN when a
 * conditional variance is not positive). For verification of the recheck
 * path. */
cupc_status cupc_pcor_data(cupc_ctx* ctx, const void* X, int dtype, int layout, int on_device,
                           int64_t n_samples, int64_t p, int64_t ld, const int32_t* queries, int64_t nq,
                           int l, double* rho_out);

/* ---------------------------------------------------------------------------
 * Candidate-scoring network for learned subset ordering (the paper has no
 * learned component; these calls serve the ordering option). The network maps
 * five features of a candidate k of row i at level l (k a neighbour of i in
 * A'_G, means over the row's other neighbours j),
 * (|C_ik|, mean |C_jk|, mean |C_ij|, l/8, mean |rho_ij.k|), with the two terms
 * that need C_jk set to 0 at level 1, through 5 -> 64 -> 64 -> 1 with ReLU to a
 * score; with opts->learned_order, every level l >= 1 enumerates the subsets
 * of each row with at most 512 neighbours over its neighbours sorted by
 * descending score (ties: increasing index), lexicographic over the sorted
 * positions: every subset is still reachable, so the skeleton is unchanged,
 * and the SepSet stored is the first separating set in that order. A larger
 * row keeps the increasing order. Parameters are CUPC_MLP_PARAMS floats packed W1 (64x5), b1 (64),
 * W2 (64x64), b2 (64), w3 (64), b3 (1), row-major. Training keeps FP32
 * master weights on the device; scoring uses their bf16 rounding.
 * ------------------------------------------------------------------------- */
#define CUPC_MLP_PARAMS 4609
#define CUPC_MLP_FEATURES 5

/* Loads parameters (host array of CUPC_MLP_PARAMS floats) into the context and
 * resets the Adam moments. */
cupc_status cupc_mlp_set_weights(cupc_ctx* ctx, const float* params);

/* Copies the context's FP32 parameters to the host array `params`. */
cupc_status cupc_mlp_get_weights(cupc_ctx* ctx, float* params);

/* Gradient of the mean binary cross-entropy with logits over n examples:
 * X device float [n x 5], t device float [n] (0 or 1); grad receives
 * CUPC_MLP_PARAMS floats (host) and *loss the mean loss. Deterministic. */
cupc_status cupc_mlp_grad(cupc_ctx* ctx, const float* X, const float* t, int64_t n, float* grad, double* loss);

/* Scores of n feature rows (device float [n x 5]) into device float y[n],
 * with the bf16 weights. */
cupc_status cupc_mlp_forward(cupc_ctx* ctx, const float* X, int64_t n, float* y);

/* Adam (lr, beta1 = 0.9, beta2 = 0.999, eps = 1e-8) over `epochs` passes of
 * the n examples in order, mini-batches of `batch`; epoch_loss (host, may be
 * NULL) receives each epoch's mean loss. All arithmetic runs in the library's
 * kernels on the device. */
cupc_status cupc_mlp_train(cupc_ctx* ctx, const float* X, const float* t, int64_t n, int64_t batch, int epochs,
                           double lr, double* epoch_loss);

/* Training examples for the network from a result's SepSets (levels >= 1):
 * for each removal (x, y, l, S) at level l >= 1, the endpoint a whose neighbour
 * set in A'_G at the start of level l contains S (x first, then y; x < y)
 * gives one example per neighbour k of a other than the other endpoint: the
 * features of candidate k of row a at level l above, computed by the device
 * code the level kernel scores with, from C (device float p x p, ld = p: the
 * FP32 correlation the kernels read), and the label 1 if k is in S, else 0.
 * *n receives the number of
 * examples; with X (device float [cap x 5]) and t (device float [cap]) given,
 * the first min(cap, *n) are written (both NULL: count only). Synchronises
 * the context stream. The paper has no counterpart. */
cupc_status cupc_mlp_examples(const cupc_result* res, const float* C, float* X, float* t, int64_t cap,
                              int64_t* n);

/* Allocation-free FP64 correlation matrix (the paper has no counterpart).
 *
 * For callers that may not allocate device memory: plugins whose host
 * framework owns and pre-plans all GPU memory, and latency-critical pipelines
 * in which a cudaMalloc (which can synchronise the device and take
 * milliseconds) is not acceptable. It computes exactly what
 * cupc_correlation(precision = CUPC_F64) computes, with the same kernels, and
 * needs no context.
 *   X       device pointer to the n_samples x p data (dtype, layout, ld as in
 *           cupc_skeleton).
 *   C_out   device pointer to p x p doubles (row-major, ld = p), caller-owned.
 *   stream  cudaStream_t to run on (NULL = legacy default stream); the call
 *           returns after the stream has finished the work.
 * Scratch: a fixed 36 MiB device array inside the library (one per device that
 * loads it, kept until the process exits). Limits: p <= 65536 and
 * n_samples * p <= 2^21; larger sizes return CUPC_E_RANGE before any GPU work.
 * It calls no cudaMalloc, cudaFree or allocating library routine.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture. The address is kept for the life of the process:
 * it assumes the device's primary context (the one the CUDA runtime and
 * PyTorch use) and no cudaDeviceReset() on that device afterwards; a caller
 * that resets the device or makes another driver context current must not
 * call this entry point again in that process. Every call on a device shares the scratch: calls
 * that overlap on the GPU (other threads or streams) race and must be
 * serialised by the caller; the error flag is cleared at the start of each
 * call. Errors: CUPC_E_INVALID, CUPC_E_RANGE, CUPC_E_NUMERIC (zero variance or
 * non-finite data), CUPC_E_CUDA. */
cupc_status cupc_correlation_noalloc(const void* X, int dtype, int layout, int64_t n_samples, int64_t p,
                                     int64_t ld, double* C_out, void* stream);

/* Eq. (threshold) as the library evaluates it, on the host:
 * tau = Phi^-1(1 - alpha/2) / sqrt(n_samples - l - 3) and r = tanh(tau); a CI
 * test is independent iff |Z(rho)| <= tau, i.e. |rho| <= r (Eq.
 * FisherZTransform with atanh monotone). Either output pointer may be NULL.
 * CUPC_E_INVALID when alpha is outside (0, 1) or n_samples - l - 3 <= 0.
 * Needs no GPU. */
cupc_status cupc_fisher_threshold(double alpha, int64_t n_samples, int l, double* tau, double* r);

#ifdef __cplusplus
}
#endif
#endif /* CUPC_H */
