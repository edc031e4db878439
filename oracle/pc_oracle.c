/*
 * pc_oracle.c -- plain, slow, obviously-correct FP64 CPU reference for the
 * PC-stable skeleton with Gaussian conditional-independence tests.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or
 * calls this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg use it. It shares no code with the CUDA path.
 *
 * What it follows (paper: Zarebavani et al., "cuPC: CUDA-based Parallel PC
 * Algorithm for Causal Structure Learning on GPU", TPDS 2019):
 *   - Algorithm 1 (first step of PC-stable): start from the complete graph;
 *     at each level l freeze G' = G; for every edge test subsets S of
 *     adj(V_i, G') \ {V_j} with |S| = l until one separates; remove the edge
 *     from G and store S.
 *   - Sec. 4.2, Eq. (comb) and Algorithm 6: lexicographic unranking of the
 *     t-th l-combination, plus the two index adjustments (0-based, and
 *     skipping the position p of V_j).
 *   - Sec. 4.3, Eqs. (PartialCorMat), (RhoCal), (FisherZTransform),
 *     (threshold): M0, M1, M2 from the correlation matrix C,
 *     H = M0 - M1 M2^-1 M1^T, rho = H12 / sqrt(H11 H22),
 *     Z = |0.5 ln((1+rho)/(1-rho))|, tau = Phi^-1(1 - alpha/2)/sqrt(m-|S|-3),
 *     independent iff Z <= tau.
 *   - Sec. 4.4, Algorithm 7: Moore-Penrose pseudo-inverse through the full-rank
 *     Cholesky factor of M2^T M2, used when M2 is not positive definite.
 *   - Sec. 2.4 (second step of PC-stable) with the v-structures and the CPDAG
 *     of Sec. 2.2: orc_orient, at the end of the file, with its readings.
 *
 * Readings where the paper is silent or garbled (each is listed in the design
 * notes of the repository):
 *   - termination: repeat while (max degree of G) - 1 >= l (the printed
 *     "until" condition is inverted), and stop after max_level when given;
 *   - both endpoints supply conditioning sets, the smaller index first, and the
 *     larger side is skipped once the edge is removed; at level 0 the two
 *     sides coincide (S is empty), so one test per pair (the Fig. 2 counts);
 *   - Z == tau counts as independent; |rho| >= 1 is dependent; a zero
 *     conditional variance (H11 or H22 <= 1e-10, rounding level of the unit
 *     diagonal) means V_i or V_j is determined by S, read as independent;
 *   - M2^-1 is the ordinary inverse (Cholesky) when M2 is positive definite;
 *     Algorithm 7 is used otherwise (equal in exact arithmetic);
 *   - the stored SepSet is the first separating S in the serial order above.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (see build.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_LEVELS 256
/* H11 or H22 at or below this is a zero conditional variance: V_i or V_j is a
 * linear function of S (C has a unit diagonal, so this is an absolute scale). */
#define ORC_VAR_ZERO 1e-10

/* ------------------------------------------------------------------------ */
/* Binomial coefficients (exact, saturating at UINT64_MAX).                  */
/* ------------------------------------------------------------------------ */
uint64_t orc_binom(int64_t n, int64_t k)
{
    if (k < 0 || n < 0 || k > n) return 0;
    if (k > n - k) k = n - k;
    unsigned __int128 r = 1;
    for (int64_t a = 1; a <= k; ++a) {
        r = r * (unsigned __int128)(n - k + a) / (unsigned __int128)a;
        if (r > (unsigned __int128)UINT64_MAX) return UINT64_MAX;
    }
    return (uint64_t)r;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.2 / Algorithm 6: the t-th l-combination of {1..n} in lexicographic */
/* order. Walks each position forward while the running count of skipped     */
/* combinations stays within t (Eq. comb), then steps back one.              */
/* Output O[0..l) is 1-based and increasing. Returns 0, or -1 if t is out of */
/* range.                                                                    */
/* ------------------------------------------------------------------------ */
int orc_comb(int n, int l, uint64_t t, int* O)
{
    if (l < 0 || l > n) return -1;
    if (t >= orc_binom(n, l)) return -1;
    uint64_t sum = 0;
    int prev = 0;
    for (int c = 0; c < l; ++c) {
        int v = prev;
        uint64_t add = 0;
        for (;;) {
            v += 1;
            add = orc_binom(n - v, l - (c + 1));
            sum += add;
            if (sum > t) break;
        }
        sum -= add;
        O[c] = v;
        prev = v;
    }
    return 0;
}

/* Sec. 4.2, cuPC-S adjustment: positions within a row of n elements, 0-based. */
int orc_comb_row(int nrow, int l, uint64_t t, int* P)
{
    if (orc_comb(nrow, l, t, P) != 0) return -1;
    for (int c = 0; c < l; ++c) P[c] -= 1;
    return 0;
}

/* Sec. 4.2, cuPC-E adjustment: choose from the nrow-1 elements other than the
 * one at position p; 0-based, every value >= p is moved up by one. */
int orc_comb_skip(int nrow, int l, uint64_t t, int p, int* P)
{
    if (orc_comb(nrow - 1, l, t, P) != 0) return -1;
    for (int c = 0; c < l; ++c) {
        P[c] -= 1;
        if (P[c] >= p) P[c] += 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Correlation matrix (Sec. 4.3: C is the correlation matrix of the data).   */
/* X is addressed as X[s*s_stride + v*v_stride] for sample s, variable v.    */
/* Population moments (divide by n); the diagonal is set to exactly 1.       */
/* ------------------------------------------------------------------------ */
int orc_correlation(const double* X, int64_t n, int64_t p, int64_t s_stride, int64_t v_stride,
                    double* C, int nthreads)
{
    if (n < 2 || p < 1) return -1;
    double* Z = (double*)malloc((size_t)n * (size_t)p * sizeof(double));
    if (!Z) return -2;
    (void)nthreads;
    #pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t v = 0; v < p; ++v) {
        double mean = 0.0;
        for (int64_t s = 0; s < n; ++s) mean += X[s * s_stride + v * v_stride];
        mean /= (double)n;
        double ss = 0.0;
        for (int64_t s = 0; s < n; ++s) {
            double d = X[s * s_stride + v * v_stride] - mean;
            ss += d * d;
        }
        double sd = sqrt(ss / (double)n);
        for (int64_t s = 0; s < n; ++s)
            Z[v * n + s] = (X[s * s_stride + v * v_stride] - mean) / sd;
    }
    #pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t i = 0; i < p; ++i) {
        C[i * p + i] = 1.0;
        for (int64_t j = i + 1; j < p; ++j) {
            double acc = 0.0;
            const double* zi = Z + i * n;
            const double* zj = Z + j * n;
            for (int64_t s = 0; s < n; ++s) acc += zi[s] * zj[s];
            acc /= (double)n;
            C[i * p + j] = acc;
            C[j * p + i] = acc;
        }
    }
    free(Z);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Standard normal quantile, by bisection on Phi(x) = erfc(-x/sqrt 2)/2.     */
/* Solved in the lower tail (accurate there) and mirrored for q > 1/2.       */
/* ------------------------------------------------------------------------ */
static double orc_norm_cdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

double orc_norm_quantile(double q)
{
    if (!(q > 0.0 && q < 1.0)) return NAN;
    if (q > 0.5) return -orc_norm_quantile(1.0 - q);
    if (q == 0.5) return 0.0;
    double lo = -40.0, hi = 0.0;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (orc_norm_cdf(mid) < q) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Eq. (threshold): tau = Phi^-1(1 - alpha/2) / sqrt(m - |S| - 3). The upper
 * quantile is taken as minus the lower quantile of alpha/2 (same value,
 * without rounding 1 - alpha/2 first). */
double orc_tau(double alpha, int64_t n_samples, int l)
{
    double dof = (double)(n_samples - l - 3);
    if (!(dof > 0.0)) return NAN;
    return -orc_norm_quantile(0.5 * alpha) / sqrt(dof);
}

/* ------------------------------------------------------------------------ */
/* Matrix helpers (row-major, plain loops).                                  */
/* ------------------------------------------------------------------------ */

/* Inverse of a symmetric positive definite l x l matrix through its Cholesky
 * factor M = L L^T: M^-1 = L^-T L^-1. Returns 0, or 1 if a pivot is not
 * clearly positive (pivot^2 <= 1e-12 * max diagonal). */
int orc_inverse_spd(const double* M, int l, double* Minv)
{
    if (l == 0) return 0;
    double* L = (double*)calloc((size_t)l * l, sizeof(double));
    double* Li = (double*)calloc((size_t)l * l, sizeof(double));
    double dmax = 0.0;
    for (int a = 0; a < l; ++a) if (M[a * l + a] > dmax) dmax = M[a * l + a];
    int rc = 0;
    for (int a = 0; a < l && rc == 0; ++a) {
        for (int b = 0; b <= a; ++b) {
            double s = M[a * l + b];
            for (int k = 0; k < b; ++k) s -= L[a * l + k] * L[b * l + k];
            if (a == b) {
                if (!(s > 1e-12 * dmax)) { rc = 1; break; }
                L[a * l + a] = sqrt(s);
            } else {
                L[a * l + b] = s / L[b * l + b];
            }
        }
    }
    if (rc == 0) {
        /* Li = L^-1 by forward substitution on the identity */
        for (int c = 0; c < l; ++c) {
            for (int a = 0; a < l; ++a) {
                double s = (a == c) ? 1.0 : 0.0;
                for (int k = 0; k < a; ++k) s -= L[a * l + k] * Li[k * l + c];
                Li[a * l + c] = s / L[a * l + a];
            }
        }
        /* Minv = Li^T Li */
        for (int a = 0; a < l; ++a)
            for (int b = 0; b < l; ++b) {
                double s = 0.0;
                for (int k = 0; k < l; ++k) s += Li[k * l + a] * Li[k * l + b];
                Minv[a * l + b] = s;
            }
    }
    free(L);
    free(Li);
    return rc;
}

/* Inverse of a general r x r nonsingular matrix by Gauss-Jordan elimination
 * with partial pivoting. Returns 0, or 1 when a pivot is exactly zero. */
static int orc_inverse_gj(const double* A, int r, double* Ainv)
{
    double* W = (double*)malloc((size_t)r * 2 * r * sizeof(double));
    for (int a = 0; a < r; ++a)
        for (int b = 0; b < 2 * r; ++b)
            W[a * 2 * r + b] = (b < r) ? A[a * r + b] : ((b - r) == a ? 1.0 : 0.0);
    int rc = 0;
    for (int c = 0; c < r; ++c) {
        int piv = c;
        for (int a = c + 1; a < r; ++a)
            if (fabs(W[a * 2 * r + c]) > fabs(W[piv * 2 * r + c])) piv = a;
        if (W[piv * 2 * r + c] == 0.0) { rc = 1; break; }
        if (piv != c)
            for (int b = 0; b < 2 * r; ++b) {
                double tmp = W[c * 2 * r + b];
                W[c * 2 * r + b] = W[piv * 2 * r + b];
                W[piv * 2 * r + b] = tmp;
            }
        double d = W[c * 2 * r + c];
        for (int b = 0; b < 2 * r; ++b) W[c * 2 * r + b] /= d;
        for (int a = 0; a < r; ++a) {
            if (a == c) continue;
            double f = W[a * 2 * r + c];
            for (int b = 0; b < 2 * r; ++b) W[a * 2 * r + b] -= f * W[c * 2 * r + b];
        }
    }
    if (rc == 0)
        for (int a = 0; a < r; ++a)
            for (int b = 0; b < r; ++b) Ainv[a * r + b] = W[a * 2 * r + r + b];
    free(W);
    return rc;
}

/* Sec. 4.4 / Algorithm 7: Moore-Penrose pseudo-inverse of an l x l matrix G.
 *   A = G^T G;  L = full-rank Cholesky factor of A (l x r, A = L L^T),
 *   columns whose pivot falls below tol are dropped, with
 *   tol = 1e-9 * (smallest positive diagonal entry of A);
 *   R = (L^T L)^-1;  G+ = L R R L^T G^T.
 * Returns the numerical rank r (0 gives the zero matrix). */
int orc_pinv_alg7(const double* G, int l, double* Gp)
{
    if (l == 0) return 0;
    double* A = (double*)calloc((size_t)l * l, sizeof(double));
    for (int a = 0; a < l; ++a)
        for (int b = 0; b < l; ++b) {
            double s = 0.0;
            for (int k = 0; k < l; ++k) s += G[k * l + a] * G[k * l + b];
            A[a * l + b] = s;
        }
    double dpos = INFINITY;
    for (int a = 0; a < l; ++a)
        if (A[a * l + a] > 0.0 && A[a * l + a] < dpos) dpos = A[a * l + a];
    double tol = isinf(dpos) ? 0.0 : 1e-9 * dpos;

    /* L is l x l storage; only the first r columns are used. */
    double* L = (double*)calloc((size_t)l * l, sizeof(double));
    int r = 0;
    for (int k = 0; k < l; ++k) {
        /* candidate column: A[k:, k] - L[k:, :r] L[k, :r]^T */
        for (int a = k; a < l; ++a) {
            double s = A[a * l + k];
            for (int c = 0; c < r; ++c) s -= L[a * l + c] * L[k * l + c];
            L[a * l + r] = s;
        }
        if (L[k * l + r] > tol) {
            double piv = sqrt(L[k * l + r]);
            L[k * l + r] = piv;
            for (int a = k + 1; a < l; ++a) L[a * l + r] /= piv;
            r += 1;
        } else {
            for (int a = k; a < l; ++a) L[a * l + r] = 0.0;
        }
    }
    memset(Gp, 0, (size_t)l * l * sizeof(double));
    if (r > 0) {
        double* LtL = (double*)calloc((size_t)r * r, sizeof(double));
        double* R = (double*)calloc((size_t)r * r, sizeof(double));
        for (int a = 0; a < r; ++a)
            for (int b = 0; b < r; ++b) {
                double s = 0.0;
                for (int k = 0; k < l; ++k) s += L[k * l + a] * L[k * l + b];
                LtL[a * r + b] = s;
            }
        orc_inverse_gj(LtL, r, R);
        /* T1 = L R (l x r); T2 = T1 R (l x r); T3 = T2 L^T (l x l); Gp = T3 G^T */
        double* T1 = (double*)calloc((size_t)l * r, sizeof(double));
        double* T2 = (double*)calloc((size_t)l * r, sizeof(double));
        double* T3 = (double*)calloc((size_t)l * l, sizeof(double));
        for (int a = 0; a < l; ++a)
            for (int b = 0; b < r; ++b) {
                double s = 0.0;
                for (int k = 0; k < r; ++k) s += L[a * l + k] * R[k * r + b];
                T1[a * r + b] = s;
            }
        for (int a = 0; a < l; ++a)
            for (int b = 0; b < r; ++b) {
                double s = 0.0;
                for (int k = 0; k < r; ++k) s += T1[a * r + k] * R[k * r + b];
                T2[a * r + b] = s;
            }
        for (int a = 0; a < l; ++a)
            for (int b = 0; b < l; ++b) {
                double s = 0.0;
                for (int k = 0; k < r; ++k) s += T2[a * r + k] * L[b * l + k];
                T3[a * l + b] = s;
            }
        for (int a = 0; a < l; ++a)
            for (int b = 0; b < l; ++b) {
                double s = 0.0;
                for (int k = 0; k < l; ++k) s += T3[a * l + k] * G[b * l + k];
                Gp[a * l + b] = s;
            }
        free(LtL); free(R); free(T1); free(T2); free(T3);
    }
    free(A);
    free(L);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.3: partial correlation of V_i, V_j given S from C (p x p).         */
/* Returns 0 with *rho set, or 1 when H11 or H22 <= ORC_VAR_ZERO (degenerate). */
/* *used_pinv is set to 1 when M2 was not positive definite.                 */
/* ------------------------------------------------------------------------ */
int orc_pcor(const double* C, int64_t p, int i, int j, const int* S, int l,
             double* rho, int* used_pinv)
{
    double M0[4] = { C[(int64_t)i * p + i], C[(int64_t)i * p + j],
                     C[(int64_t)j * p + i], C[(int64_t)j * p + j] };
    double H[4] = { M0[0], M0[1], M0[2], M0[3] };
    if (used_pinv) *used_pinv = 0;
    if (l > 0) {
        double* M1 = (double*)malloc((size_t)2 * l * sizeof(double));
        double* M2 = (double*)malloc((size_t)l * l * sizeof(double));
        double* M2i = (double*)malloc((size_t)l * l * sizeof(double));
        for (int k = 0; k < l; ++k) {
            M1[0 * l + k] = C[(int64_t)i * p + S[k]];
            M1[1 * l + k] = C[(int64_t)j * p + S[k]];
        }
        for (int a = 0; a < l; ++a)
            for (int b = 0; b < l; ++b) M2[a * l + b] = C[(int64_t)S[a] * p + S[b]];
        if (orc_inverse_spd(M2, l, M2i) != 0) {
            orc_pinv_alg7(M2, l, M2i);
            if (used_pinv) *used_pinv = 1;
        }
        /* H = M0 - M1 M2^-1 M1^T */
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double s = 0.0;
                for (int u = 0; u < l; ++u)
                    for (int v = 0; v < l; ++v) s += M1[a * l + u] * M2i[u * l + v] * M1[b * l + v];
                H[a * 2 + b] = M0[a * 2 + b] - s;
            }
        free(M1); free(M2); free(M2i);
    }
    /* a conditional variance at rounding level of the unit diagonal is zero */
    if (!(H[0] > ORC_VAR_ZERO) || !(H[3] > ORC_VAR_ZERO)) { *rho = NAN; return 1; }
    *rho = H[1] / sqrt(H[0] * H[3]);
    return 0;
}

/* Eq. (FisherZTransform) and the decision Z <= tau. Returns 1 if independent.
 * *z receives Z (INFINITY when |rho| >= 1, NAN when degenerate). */
int orc_fisher_decide(double rho, int degenerate, double tau, double* z)
{
    if (degenerate) { *z = NAN; return 1; }
    if (!(fabs(rho) < 1.0)) { *z = INFINITY; return 0; }
    *z = fabs(0.5 * log((1.0 + rho) / (1.0 - rho)));
    return (*z <= tau) ? 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* d-separation in a DAG (D[u*p+v] = 1 iff u -> v) through the moralised     */
/* ancestral graph of {i, j} U S. Returns 1 iff i and j are d-separated by S. */
/* ------------------------------------------------------------------------ */
int orc_dsep(const uint8_t* D, int p, int i, int j, const int* S, int l)
{
    uint8_t* anc = (uint8_t*)calloc((size_t)p, 1);
    uint8_t* inS = (uint8_t*)calloc((size_t)p, 1);
    int* stack = (int*)malloc((size_t)p * sizeof(int));
    int top = 0;
    for (int k = 0; k < l; ++k) inS[S[k]] = 1;
    int seeds[2] = { i, j };
    for (int k = 0; k < 2; ++k) if (!anc[seeds[k]]) { anc[seeds[k]] = 1; stack[top++] = seeds[k]; }
    for (int k = 0; k < l; ++k) if (!anc[S[k]]) { anc[S[k]] = 1; stack[top++] = S[k]; }
    while (top > 0) {
        int v = stack[--top];
        for (int u = 0; u < p; ++u)
            if (D[(int64_t)u * p + v] && !anc[u]) { anc[u] = 1; stack[top++] = u; }
    }
    /* moral graph restricted to the ancestral set */
    uint8_t* M = (uint8_t*)calloc((size_t)p * p, 1);
    for (int u = 0; u < p; ++u) {
        if (!anc[u]) continue;
        for (int v = 0; v < p; ++v) {
            if (!anc[v]) continue;
            if (D[(int64_t)u * p + v]) { M[(int64_t)u * p + v] = 1; M[(int64_t)v * p + u] = 1; }
        }
    }
    for (int w = 0; w < p; ++w) {
        if (!anc[w]) continue;
        for (int a = 0; a < p; ++a) {
            if (!D[(int64_t)a * p + w]) continue;
            for (int b = a + 1; b < p; ++b)
                if (D[(int64_t)b * p + w]) { M[(int64_t)a * p + b] = 1; M[(int64_t)b * p + a] = 1; }
        }
    }
    /* reachability from i avoiding S */
    uint8_t* seen = (uint8_t*)calloc((size_t)p, 1);
    top = 0;
    seen[i] = 1;
    stack[top++] = i;
    int connected = 0;
    while (top > 0 && !connected) {
        int v = stack[--top];
        for (int u = 0; u < p; ++u) {
            if (!M[(int64_t)v * p + u] || seen[u] || inS[u]) continue;
            if (u == j) { connected = 1; break; }
            seen[u] = 1;
            stack[top++] = u;
        }
    }
    free(anc); free(inS); free(stack); free(M); free(seen);
    return connected ? 0 : 1;
}

/* ------------------------------------------------------------------------ */
/* The CI-test sources the skeleton driver can use.                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int kind;                  /* 0 Gaussian from C, 1 d-separation, 2 table of statements */
    int p;
    const double* C;           /* kind 0 */
    int64_t n_samples;
    double alpha;
    const uint8_t* dag;        /* kind 1 */
    const int* table;          /* kind 2: rows of width stride: i, j, l, S[0..l) */
    int table_rows, table_stride;
} orc_ci;

typedef struct {
    double tau;                /* per-level threshold (kind 0) */
    double min_margin;         /* min |Z - tau| seen */
    int64_t degenerate;        /* count of H11 <= 0 or H22 <= 0 */
    int64_t pinv_used;
} orc_level_ctx;

static int table_lookup(const orc_ci* ci, int i, int j, const int* S, int l)
{
    for (int r = 0; r < ci->table_rows; ++r) {
        const int* row = ci->table + (int64_t)r * ci->table_stride;
        if (row[2] != l) continue;
        if (!((row[0] == i && row[1] == j) || (row[0] == j && row[1] == i))) continue;
        /* S and the stored set are both increasing */
        int same = 1;
        for (int k = 0; k < l; ++k) if (row[3 + k] != S[k]) { same = 0; break; }
        if (same) return 1;
    }
    return 0;
}

/* One CI test. Returns 1 if independent. Updates margin/degenerate counters
 * through the per-thread context. */
static int ci_test(const orc_ci* ci, orc_level_ctx* lc, int i, int j, const int* S, int l)
{
    if (ci->kind == 1) return orc_dsep(ci->dag, ci->p, i, j, S, l);
    if (ci->kind == 2) return table_lookup(ci, i, j, S, l);
    double rho, z;
    int used = 0;
    int deg = orc_pcor(ci->C, ci->p, i, j, S, l, &rho, &used);
    if (deg) lc->degenerate += 1;
    if (used) lc->pinv_used += 1;
    int ind = orc_fisher_decide(rho, deg, lc->tau, &z);
    if (!deg && isfinite(z)) {
        double m = fabs(z - lc->tau);
        if (m < lc->min_margin) lc->min_margin = m;
    }
    return ind;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 driver.                                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    int p;
    int levels_run;            /* number of levels executed (level 0 included) */
    uint8_t* adj;              /* p*p final skeleton */
    int16_t* sep_level;        /* p*p: -1 edge present, else the removal level */
    int* rec;                  /* SepSet records for removals at l >= 1: i, j, l, S... */
    int64_t rec_len, rec_cap;  /* in ints */
    int64_t n_rec;
    int64_t tests[ORC_MAX_LEVELS];
    int64_t removed[ORC_MAX_LEVELS];
    double min_margin;
    int64_t degenerate, pinv_used;
    int status;                /* 0 ok, -3 subset count overflow */
} orc_run;

/* Tests one side (a's neighbourhood) of edge (a, b). Returns 1 if separated. */
static int test_side(const orc_ci* ci, orc_level_ctx* lc, int a, int b, const int* nb, int deg,
                     int l, int64_t* tests, int* S_out, int* status)
{
    if (deg - 1 < l) return 0;
    int pos_b = -1;
    for (int k = 0; k < deg; ++k) if (nb[k] == b) { pos_b = k; break; }
    if (pos_b < 0) return 0;
    uint64_t total = orc_binom(deg - 1, l);
    if (total == UINT64_MAX) { *status = -3; return 0; }
    int P[ORC_MAX_LEVELS], S[ORC_MAX_LEVELS];
    for (uint64_t t = 0; t < total; ++t) {
        orc_comb_skip(deg, l, t, pos_b, P);
        for (int c = 0; c < l; ++c) S[c] = nb[P[c]];
        *tests += 1;
        if (ci_test(ci, lc, a, b, S, l)) {
            for (int c = 0; c < l; ++c) S_out[c] = S[c];
            return 1;
        }
    }
    return 0;
}

void orc_run_free(orc_run* r)
{
    if (!r) return;
    free(r->adj); free(r->sep_level); free(r->rec); free(r);
}

static void rec_push(orc_run* r, int i, int j, int l, const int* S)
{
    int64_t need = r->rec_len + 3 + l;
    if (need > r->rec_cap) {
        int64_t cap = r->rec_cap ? r->rec_cap : 1024;
        while (cap < need) cap *= 2;
        r->rec = (int*)realloc(r->rec, (size_t)cap * sizeof(int));
        r->rec_cap = cap;
    }
    r->rec[r->rec_len++] = i;
    r->rec[r->rec_len++] = j;
    r->rec[r->rec_len++] = l;
    for (int c = 0; c < l; ++c) r->rec[r->rec_len++] = S[c];
    r->n_rec += 1;
}

orc_run* orc_pc_stable(const orc_ci* ci, int max_level, int nthreads)
{
    int p = ci->p;
    orc_run* r = (orc_run*)calloc(1, sizeof(orc_run));
    r->p = p;
    r->adj = (uint8_t*)malloc((size_t)p * p);
    r->sep_level = (int16_t*)malloc((size_t)p * p * sizeof(int16_t));
    for (int64_t a = 0; a < (int64_t)p * p; ++a) { r->adj[a] = 1; r->sep_level[a] = -1; }
    for (int a = 0; a < p; ++a) r->adj[(int64_t)a * p + a] = 0;
    r->min_margin = INFINITY;

    int* deg = (int*)malloc((size_t)p * sizeof(int));
    int64_t* off = (int64_t*)malloc(((size_t)p + 1) * sizeof(int64_t));
    int* nb = NULL;
    uint8_t* rem = NULL;   /* per CSR slot of the smaller endpoint: edge removed this level */
    int* spool = NULL;     /* per CSR slot: the separating set found */
    int nth = nthreads > 0 ? nthreads : 1;

    for (int l = 0; l < ORC_MAX_LEVELS; ++l) {
        if (max_level >= 0 && l > max_level) break;
        double tau = (ci->kind == 0) ? orc_tau(ci->alpha, ci->n_samples, l) : 0.0;
        double mm = INFINITY;
        int64_t degn = 0, pinv = 0, ntests = 0, nrem = 0;

        if (l == 0) {
            /* Level 0: S is empty on both sides, so one test per pair i < j.
             * Nothing reads G during the level, so removals are applied at once. */
            #pragma omp parallel num_threads(nth) reduction(min:mm) reduction(+:degn, pinv, ntests, nrem)
            {
                orc_level_ctx lc = { tau, INFINITY, 0, 0 };
                #pragma omp for schedule(dynamic, 8)
                for (int x = 0; x < p; ++x)
                    for (int y = x + 1; y < p; ++y) {
                        ntests += 1;
                        if (ci_test(ci, &lc, x, y, NULL, 0)) {
                            r->adj[(int64_t)x * p + y] = 0;
                            r->adj[(int64_t)y * p + x] = 0;
                            r->sep_level[(int64_t)x * p + y] = 0;
                            r->sep_level[(int64_t)y * p + x] = 0;
                            nrem += 1;
                        }
                    }
                if (lc.min_margin < mm) mm = lc.min_margin;
                degn += lc.degenerate;
                pinv += lc.pinv_used;
            }
        } else {
            /* frozen copy G' of G as sorted neighbour lists */
            int64_t nnz = 0;
            int maxdeg = 0;
            for (int a = 0; a < p; ++a) {
                int d = 0;
                for (int b = 0; b < p; ++b) d += r->adj[(int64_t)a * p + b];
                deg[a] = d;
                off[a] = nnz;
                nnz += d;
                if (d > maxdeg) maxdeg = d;
            }
            off[p] = nnz;
            /* termination (reading of Alg. 1's last line): level l runs only
             * while some node has degree - 1 >= l */
            if (maxdeg - 1 < l) break;
            nb = (int*)realloc(nb, (size_t)(nnz > 0 ? nnz : 1) * sizeof(int));
            rem = (uint8_t*)realloc(rem, (size_t)(nnz > 0 ? nnz : 1));
            spool = (int*)realloc(spool, (size_t)(nnz > 0 ? nnz : 1) * (size_t)l * sizeof(int));
            for (int a = 0; a < p; ++a) {
                int64_t k = off[a];
                for (int b = 0; b < p; ++b) if (r->adj[(int64_t)a * p + b]) nb[k++] = b;
            }
            int st = 0;
            /* Edges are independent within a level given G' (Sec. 2.4), so the
             * rows may be processed in any order with identical results. G is
             * only written (never read) here. */
            #pragma omp parallel num_threads(nth) reduction(min:mm) reduction(+:degn, pinv, ntests, nrem)
            {
                orc_level_ctx lc = { tau, INFINITY, 0, 0 };
                #pragma omp for schedule(dynamic, 1)
                for (int x = 0; x < p; ++x) {
                    for (int64_t k = off[x]; k < off[x + 1]; ++k) {
                        int y = nb[k];
                        rem[k] = 0;
                        if (y < x) continue;
                        int status = 0;
                        int* S = spool + k * l;
                        /* side of the smaller endpoint first; the larger side
                         * only when the edge is still present */
                        int found = test_side(ci, &lc, x, y, nb + off[x], deg[x], l, &ntests, S, &status);
                        if (!found && status == 0)
                            found = test_side(ci, &lc, y, x, nb + off[y], deg[y], l, &ntests, S, &status);
                        if (status != 0) {
                            #pragma omp critical
                            st = status;
                        }
                        if (found) {
                            rem[k] = 1;
                            r->adj[(int64_t)x * p + y] = 0;
                            r->adj[(int64_t)y * p + x] = 0;
                            r->sep_level[(int64_t)x * p + y] = (int16_t)l;
                            r->sep_level[(int64_t)y * p + x] = (int16_t)l;
                            nrem += 1;
                        }
                    }
                }
                if (lc.min_margin < mm) mm = lc.min_margin;
                degn += lc.degenerate;
                pinv += lc.pinv_used;
            }
            if (st != 0) r->status = st;
            /* SepSet records in (x, y) order */
            for (int x = 0; x < p; ++x)
                for (int64_t k = off[x]; k < off[x + 1]; ++k)
                    if (nb[k] > x && rem[k]) rec_push(r, x, nb[k], l, spool + k * l);
        }
        if (mm < r->min_margin) r->min_margin = mm;
        r->degenerate += degn;
        r->pinv_used += pinv;
        r->tests[l] = ntests;
        r->removed[l] = nrem;
        r->levels_run = l + 1;
        if (r->status != 0) break;
    }
    free(deg); free(off); free(nb); free(rem); free(spool);
    return r;
}

/* Convenience entry points for the ctypes wrapper. */
orc_run* orc_pc_gauss(const double* C, int p, int64_t n_samples, double alpha, int max_level, int nthreads)
{
    orc_ci ci;
    memset(&ci, 0, sizeof ci);
    ci.kind = 0; ci.p = p; ci.C = C; ci.n_samples = n_samples; ci.alpha = alpha;
    return orc_pc_stable(&ci, max_level, nthreads);
}

orc_run* orc_pc_dsep(const uint8_t* dag, int p, int max_level, int nthreads)
{
    orc_ci ci;
    memset(&ci, 0, sizeof ci);
    ci.kind = 1; ci.p = p; ci.dag = dag;
    return orc_pc_stable(&ci, max_level, nthreads);
}

orc_run* orc_pc_table(int p, const int* table, int rows, int stride, int max_level)
{
    orc_ci ci;
    memset(&ci, 0, sizeof ci);
    ci.kind = 2; ci.p = p; ci.table = table; ci.table_rows = rows; ci.table_stride = stride;
    return orc_pc_stable(&ci, max_level, 1);
}

/* Single Gaussian CI test: returns 1 if independent; rho and z are written. */
int orc_ci_gauss(const double* C, int64_t p, int64_t n_samples, double alpha, int i, int j,
                 const int* S, int l, double* rho, double* z)
{
    int used = 0;
    int deg = orc_pcor(C, p, i, j, S, l, rho, &used);
    double tau = orc_tau(alpha, n_samples, l);
    return orc_fisher_decide(*rho, deg, tau, z);
}

/* Accessors */
int orc_run_p(const orc_run* r) { return r->p; }
int orc_run_levels(const orc_run* r) { return r->levels_run; }
int orc_run_status(const orc_run* r) { return r->status; }
double orc_run_min_margin(const orc_run* r) { return r->min_margin; }
int64_t orc_run_degenerate(const orc_run* r) { return r->degenerate; }
int64_t orc_run_pinv_used(const orc_run* r) { return r->pinv_used; }
int64_t orc_run_rec_len(const orc_run* r) { return r->rec_len; }
int64_t orc_run_n_rec(const orc_run* r) { return r->n_rec; }
void orc_run_copy(const orc_run* r, uint8_t* adj, int16_t* sep_level, int* rec,
                  int64_t* tests, int64_t* removed)
{
    int64_t pp = (int64_t)r->p * r->p;
    if (adj) memcpy(adj, r->adj, (size_t)pp);
    if (sep_level) memcpy(sep_level, r->sep_level, (size_t)pp * sizeof(int16_t));
    if (rec && r->rec_len) memcpy(rec, r->rec, (size_t)r->rec_len * sizeof(int));
    if (tests) memcpy(tests, r->tests, sizeof r->tests);
    if (removed) memcpy(removed, r->removed, sizeof r->removed);
}

/* ------------------------------------------------------------------------ */
/* Second step of PC-stable (Sec. 2.4): the v-structures V_i -> V_k <- V_j   */
/* of Sec. 2.2, read off the SepSets, then Meek's orientation rules R1-R3,  */
/* which give the CPDAG of Sec. 2.2.                                         */
/*                                                                          */
/* Edge marks: mark[a*p + b] = 0 when a and b are not adjacent; 1 when the   */
/* edge a - b has an arrowhead at b; 2 when it has a tail at b. So a -> b is */
/* (mark[a][b], mark[b][a]) = (1, 2), a - b is (2, 2), and two v-structures  */
/* that disagree on an edge leave arrowheads at both ends, (1, 1).           */
/*                                                                          */
/* Readings (the paper only names the step): every unshielded triple         */
/* i - k - j (i, j not adjacent) with k outside SepSet(i, j) is a            */
/* v-structure, all of them applied together (order-free; conflicts give     */
/* (1, 1)); the rules then run in rounds, each deciding from the marks at    */
/* the start of the round and applying all its orientations together, until  */
/* a round changes nothing; an edge that a round would orient both ways is   */
/* left undirected. Only undirected edges are oriented, and only directed    */
/* edges (1, 2) count as arrows in the rules' premises:                      */
/*   R1  c -> a, a - b, c and b not adjacent            =>  a -> b          */
/*   R2  a -> c -> b, a - b                             =>  a -> b          */
/*   R3  a - c1 -> b, a - c2 -> b, c1 and c2 not adjacent, a - b => a -> b  */
/* SepSets: sep_level[i*p + j] is the level that removed the pair (-1 when   */
/* the edge is present); removals at level 0 have S empty; the others are    */
/* found by key i*p + j (i < j) in the ascending keys[], with members        */
/* members[off[r] .. off[r] + level).                                        */
/* Returns the number of rule rounds run (the last one changed nothing), or  */
/* -1 on bad input.                                                          */
/* ------------------------------------------------------------------------ */
static int sep_has(int64_t p, const int16_t* sep_level, const int64_t* keys, const int64_t* off,
                   const int32_t* members, int64_t nkeys, int i, int j, int k)
{
    const int a = i < j ? i : j, b = i < j ? j : i;
    const int lev = sep_level[(int64_t)a * p + b];
    if (lev <= 0) return 0;
    const int64_t key = (int64_t)a * p + b;
    int64_t lo = 0, hi = nkeys;
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (keys[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    if (lo >= nkeys || keys[lo] != key) return -1;
    for (int c = 0; c < lev; ++c)
        if (members[off[lo] + c] == k) return 1;
    return 0;
}

static int is_dir(const uint8_t* mark, int64_t p, int x, int y)
{
    return mark[(int64_t)x * p + y] == 1 && mark[(int64_t)y * p + x] == 2;
}

static int is_und(const uint8_t* mark, int64_t p, int x, int y)
{
    return mark[(int64_t)x * p + y] == 2 && mark[(int64_t)y * p + x] == 2;
}

int64_t orc_orient(int p, const uint8_t* adj, const int16_t* sep_level, const int64_t* keys, const int64_t* off,
                   const int32_t* members, int64_t nkeys, uint8_t* mark)
{
    const int64_t P = p;
    /* neighbour lists of the skeleton (it does not change in this step) */
    int64_t* nb_off = (int64_t*)malloc((size_t)(P + 1) * sizeof(int64_t));
    int64_t tot = 0;
    for (int64_t a = 0; a < P; ++a) {
        nb_off[a] = tot;
        for (int64_t b = 0; b < P; ++b) tot += (a != b && adj[a * P + b]) ? 1 : 0;
    }
    nb_off[P] = tot;
    int* nb = (int*)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int));
    for (int64_t a = 0, q = 0; a < P; ++a)
        for (int64_t b = 0; b < P; ++b)
            if (a != b && adj[a * P + b]) nb[q++] = (int)b;
    for (int64_t x = 0; x < P * P; ++x) mark[x] = adj[x] ? 2 : 0;
    for (int64_t a = 0; a < P; ++a) mark[a * P + a] = 0;

    /* v-structures: unshielded triples i - k - j with k not in SepSet(i, j) */
    int bad = 0;
    for (int64_t k = 0; k < P; ++k) {
        for (int64_t x = nb_off[k]; x < nb_off[k + 1]; ++x) {
            for (int64_t y = x + 1; y < nb_off[k + 1]; ++y) {
                const int i = nb[x], j = nb[y];
                if (adj[(int64_t)i * P + j]) continue;
                const int in = sep_has(P, sep_level, keys, off, members, nkeys, i, j, (int)k);
                if (in < 0) bad = 1;
                if (in == 0) {
                    mark[(int64_t)i * P + k] = 1;
                    mark[(int64_t)j * P + k] = 1;
                }
            }
        }
    }
    if (bad) {
        free(nb);
        free(nb_off);
        return -1;
    }

    /* Meek's rules R1-R3 in rounds */
    uint8_t* prop = (uint8_t*)malloc((size_t)(P * P > 0 ? P * P : 1));
    int64_t rounds = 0;
    for (;;) {
        memset(prop, 0, (size_t)(P * P));
        for (int64_t a = 0; a < P; ++a) {
            for (int64_t x = nb_off[a]; x < nb_off[a + 1]; ++x) {
                const int b = nb[x];
                if (!is_und(mark, P, (int)a, b)) continue;
                int hit = 0;
                for (int64_t y = nb_off[a]; y < nb_off[a + 1] && !hit; ++y) {
                    const int c = nb[y];
                    if (c == b) continue;
                    /* R1 */
                    if (is_dir(mark, P, c, (int)a) && !adj[(int64_t)c * P + b]) hit = 1;
                    /* R2 */
                    if (is_dir(mark, P, (int)a, c) && is_dir(mark, P, c, b)) hit = 1;
                }
                /* R3 */
                for (int64_t y = nb_off[a]; y < nb_off[a + 1] && !hit; ++y) {
                    const int c1 = nb[y];
                    if (c1 == b || !is_und(mark, P, (int)a, c1) || !is_dir(mark, P, c1, b)) continue;
                    for (int64_t z = y + 1; z < nb_off[a + 1] && !hit; ++z) {
                        const int c2 = nb[z];
                        if (c2 == b || !is_und(mark, P, (int)a, c2) || !is_dir(mark, P, c2, b)) continue;
                        if (!adj[(int64_t)c1 * P + c2]) hit = 1;
                    }
                }
                prop[a * P + b] = (uint8_t)hit;
            }
        }
        int64_t changed = 0;
        for (int64_t a = 0; a < P; ++a)
            for (int64_t b = 0; b < P; ++b)
                if (prop[a * P + b] && !prop[b * P + a]) {
                    mark[a * P + b] = 1;
                    ++changed;
                }
        ++rounds;
        if (!changed) break;
    }
    free(prop);
    free(nb);
    free(nb_off);
    return rounds;
}
