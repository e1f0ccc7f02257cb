/*
 * amg_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU implementation of the method the
 * CUDA library computes: a smoothed-aggregation AMG hierarchy (strength of
 * connection, distance-2 maximal independent set aggregation, Jacobi-smoothed
 * prolongator, Galerkin coarse operators, dense coarsest factorisation), the
 * V(1,1) cycle, preconditioned CG and BiCGStab, and the reverse-mode adjoint
 * of a linear solve (the paper's Eq. 1-2: A^T lambda = dL/dx,
 * dL/dA = -lambda x^T, dL/db = lambda).
 *
 * The paper wraps an external library and specifies none of the AMG
 * algorithm; every step below follows the textbook method
 * (Vanek-Mandel-Brezina smoothed aggregation, Hestenes-Stiefel CG,
 * van der Vorst BiCGStab) with one fixed, deterministic reading of each choice
 * the paper leaves open.  The readings are stated at each function.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU baseline
 * use this file.  It shares no code, header or constant with the CUDA path.
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared.
 * -ffp-contract=off matters: every multiply and add below is rounded on its
 * own, which is the arithmetic order the GPU setup kernels reproduce.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_MAXIT 1
#define OR_BREAKDOWN 2
#define OR_NOT_SPD 3
#define OR_NAN 4
#define OR_ERR_ARG (-1)
#define OR_ERR_BAD_CSR (-2)
#define OR_ERR_ZERO_DIAG (-3)
#define OR_ERR_STALL (-5)
#define OR_ERR_OOM (-6)

/* The solve phase's row loops run on all host cores in the threaded build
 * (-fopenmp, liboracle_omp.so, used only to time the CPU baseline); every
 * such loop writes each entry once, so the split does not change any value.
 * The parity build compiles them as plain serial loops. */
#ifdef _OPENMP
#define OR_PAR _Pragma("omp parallel for schedule(static)")
#else
#define OR_PAR
#endif

#define OR_MAX_LEVELS 32
#define OR_DENSE_MAX 256

typedef struct {
    int nrows, ncols;
    long long nnz;
    int *rp;   /* nrows + 1 */
    int *ci;   /* nnz */
    double *v; /* nnz */
} ocsr;

typedef struct {
    int solver;       /* 0 PCG, 1 BiCGStab, 2 CG, 3 BiCGStab (no preconditioner) */
    int smoother;     /* 0 weighted Jacobi, 1 L1-Jacobi */
    double omega;     /* Jacobi weight, default 2/3 */
    double theta;     /* strength threshold, default 0.08 */
    int coarse_max;   /* stop coarsening at <= this many rows, default 64 */
    int max_levels;   /* default 20 */
    double rtol;      /* default 1e-8 */
    int max_iter;     /* default 500 */
    int max_restarts; /* true-residual restarts, default 3 */
    int symmetric;    /* -1 detect, 0 no, 1 yes */
    int adjoint_reuse; /* nonsymmetric adjoint: 0 sets up a hierarchy of A^T, 1 transposes A's (or_transposed) */
    int amg_type;     /* 0 smoothed aggregation, 1 classical Ruge-Stueben (strength, PMIS, direct interpolation) */
} or_config;

typedef struct {
    int status, iters, restarts;
    double rel_res_true, rel_res_rec;
} or_info;

typedef struct or_hier {
    int nlevels;            /* levels 0..nlevels-1; the last one is solved densely */
    int symmetric;
    or_config cfg;
    ocsr A[OR_MAX_LEVELS];
    ocsr P[OR_MAX_LEVELS];  /* P[l]: n_l x n_{l+1}, l < nlevels-1 */
    ocsr R[OR_MAX_LEVELS];  /* R[l] = P[l]^T */
    int *agg[OR_MAX_LEVELS];
    ocsr S[OR_MAX_LEVELS];        /* strength graph the aggregation of level l used (setup only) */
    double *dinv[OR_MAX_LEVELS];  /* smoother weight / d_i, per row */
    double rho[OR_MAX_LEVELS];    /* Gershgorin estimate used for P[l] */
    /* coarsest level: dense factor (row-major), Cholesky L or LU with pivots */
    int nc;
    double *dense;
    int *piv;
    /* transposed hierarchy for nonsymmetric adjoints, built on first use */
    struct or_hier *adj;
} or_hier;

/* ------------------------------------------------------------------------ */
/* CSR helpers                                                              */
/* ------------------------------------------------------------------------ */

static void csr_free(ocsr *a) {
    free(a->rp); free(a->ci); free(a->v);
    a->rp = NULL; a->ci = NULL; a->v = NULL;
    a->nnz = 0;
}

static int csr_alloc(ocsr *a, int nrows, int ncols, long long nnz) {
    a->nrows = nrows; a->ncols = ncols; a->nnz = nnz;
    a->rp = (int *)calloc((size_t)nrows + 1, sizeof(int));
    a->ci = (int *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int));
    a->v = (double *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
    return (a->rp && a->ci && a->v) ? OR_OK : OR_ERR_OOM;
}

static int csr_copy(ocsr *dst, int n, long long nnz, const int *rp, const int *ci, const double *v) {
    if (csr_alloc(dst, n, n, nnz)) return OR_ERR_OOM;
    memcpy(dst->rp, rp, ((size_t)n + 1) * sizeof(int));
    memcpy(dst->ci, ci, (size_t)nnz * sizeof(int));
    memcpy(dst->v, v, (size_t)nnz * sizeof(double));
    return OR_OK;
}

/* Validation of the caller's CSR: row_ptr starts at 0, is non-decreasing and
 * ends at nnz; columns lie in [0, n) and are strictly ascending in each row;
 * every row stores its diagonal and the diagonal is nonzero. */
int or_validate(int n, long long nnz, const int *rp, const int *ci, const double *v) {
    if (n <= 0 || nnz < n || !rp || !ci || !v) return OR_ERR_ARG;
    if (rp[0] != 0 || (long long)rp[n] != nnz) return OR_ERR_BAD_CSR;
    for (int i = 0; i < n; ++i) {
        if (rp[i + 1] < rp[i]) return OR_ERR_BAD_CSR;
        int has_diag = 0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            if (ci[k] < 0 || ci[k] >= n) return OR_ERR_BAD_CSR;
            if (k > rp[i] && ci[k] <= ci[k - 1]) return OR_ERR_BAD_CSR;
            if (ci[k] == i) {
                has_diag = 1;
                if (v[k] == 0.0) return OR_ERR_ZERO_DIAG;
            }
        }
        if (!has_diag) return OR_ERR_ZERO_DIAG;
    }
    return OR_OK;
}

static double csr_diag(const ocsr *a, int i) {
    for (int k = a->rp[i]; k < a->rp[i + 1]; ++k)
        if (a->ci[k] == i) return a->v[k];
    return 0.0;
}

/* y = A x, each row summed in storage order starting from +0.0. */
void or_spmv(int nrows, const int *rp, const int *ci, const double *v, const double *x, double *y) {
    OR_PAR
    for (int i = 0; i < nrows; ++i) {
        double s = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) s = s + v[k] * x[ci[k]];
        y[i] = s;
    }
}

static void spmv(const ocsr *a, const double *x, double *y) {
    or_spmv(a->nrows, a->rp, a->ci, a->v, x, y);
}

/* Transpose by counting sort on the column index.  Rows are visited in
 * ascending order, so every row of the result lists its columns ascending. */
static int csr_transpose(const ocsr *a, ocsr *t) {
    if (csr_alloc(t, a->ncols, a->nrows, a->nnz)) return OR_ERR_OOM;
    for (long long k = 0; k < a->nnz; ++k) t->rp[a->ci[k] + 1]++;
    for (int j = 0; j < a->ncols; ++j) t->rp[j + 1] += t->rp[j];
    int *next = (int *)malloc(((size_t)a->ncols + 1) * sizeof(int));
    if (!next) return OR_ERR_OOM;
    memcpy(next, t->rp, ((size_t)a->ncols + 1) * sizeof(int));
    for (int i = 0; i < a->nrows; ++i)
        for (int k = a->rp[i]; k < a->rp[i + 1]; ++k) {
            int pos = next[a->ci[k]]++;
            t->ci[pos] = i;
            t->v[pos] = a->v[k];
        }
    free(next);
    return OR_OK;
}

int or_transpose(int nrows, int ncols, long long nnz, const int *rp, const int *ci, const double *v,
                 int *trp, int *tci, double *tv) {
    ocsr a = {nrows, ncols, nnz, (int *)rp, (int *)ci, (double *)v}, t;
    if (csr_transpose(&a, &t)) return OR_ERR_OOM;
    memcpy(trp, t.rp, ((size_t)ncols + 1) * sizeof(int));
    memcpy(tci, t.ci, (size_t)nnz * sizeof(int));
    memcpy(tv, t.v, (size_t)nnz * sizeof(double));
    csr_free(&t);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Strength of connection                                                   */
/* ------------------------------------------------------------------------ */

/* j is a strong neighbour of i when a_ij^2 >= theta^2 |a_ii a_jj| (equality
 * counts as strong; theta is the level's threshold, see or_setup).  The strength graph S is the symmetric union
 * S1 or S1^T of this directed relation, without the diagonal.  Result: a
 * pattern-only CSR (values unused), columns ascending. */
static int strength(const ocsr *a, double theta, ocsr *S) {
    int n = a->nrows;
    double t2 = theta * theta;
    double *diag = (double *)malloc((size_t)n * sizeof(double));
    if (!diag) return OR_ERR_OOM;
    for (int i = 0; i < n; ++i) diag[i] = csr_diag(a, i);
    /* directed S1 */
    ocsr s1;
    long long cnt = 0;
    for (int i = 0; i < n; ++i)
        for (int k = a->rp[i]; k < a->rp[i + 1]; ++k) {
            int j = a->ci[k];
            if (j == i) continue;
            double lhs = a->v[k] * a->v[k];
            double prod = diag[i] * diag[j];
            double rhs = t2 * fabs(prod);
            if (lhs >= rhs) cnt++;
        }
    if (csr_alloc(&s1, n, n, cnt)) return OR_ERR_OOM;
    long long pos = 0;
    for (int i = 0; i < n; ++i) {
        s1.rp[i] = (int)pos;
        for (int k = a->rp[i]; k < a->rp[i + 1]; ++k) {
            int j = a->ci[k];
            if (j == i) continue;
            double lhs = a->v[k] * a->v[k];
            double prod = diag[i] * diag[j];
            double rhs = t2 * fabs(prod);
            if (lhs >= rhs) { s1.ci[pos] = j; s1.v[pos] = 1.0; pos++; }
        }
    }
    s1.rp[n] = (int)pos;
    free(diag);
    ocsr s1t;
    if (csr_transpose(&s1, &s1t)) return OR_ERR_OOM;
    /* union of two ascending lists per row */
    long long tot = 0;
    for (int i = 0; i < n; ++i) {
        int p = s1.rp[i], q = s1t.rp[i];
        while (p < s1.rp[i + 1] || q < s1t.rp[i + 1]) {
            if (q >= s1t.rp[i + 1] || (p < s1.rp[i + 1] && s1.ci[p] < s1t.ci[q])) p++;
            else if (p >= s1.rp[i + 1] || s1t.ci[q] < s1.ci[p]) q++;
            else { p++; q++; }
            tot++;
        }
    }
    if (csr_alloc(S, n, n, tot)) return OR_ERR_OOM;
    pos = 0;
    for (int i = 0; i < n; ++i) {
        S->rp[i] = (int)pos;
        int p = s1.rp[i], q = s1t.rp[i];
        while (p < s1.rp[i + 1] || q < s1t.rp[i + 1]) {
            int c;
            if (q >= s1t.rp[i + 1] || (p < s1.rp[i + 1] && s1.ci[p] < s1t.ci[q])) c = s1.ci[p++];
            else if (p >= s1.rp[i + 1] || s1t.ci[q] < s1.ci[p]) c = s1t.ci[q++];
            else { c = s1.ci[p]; p++; q++; }
            S->ci[pos] = c; S->v[pos] = 1.0; pos++;
        }
    }
    S->rp[n] = (int)pos;
    csr_free(&s1);
    csr_free(&s1t);
    return OR_OK;
}

/* Exported for tests: S as (row_ptr, col_idx); caller frees with or_free_buf. */
int or_strength(int n, long long nnz, const int *rp, const int *ci, const double *v, double theta,
                int **srp, int **sci, long long *snnz) {
    ocsr a = {n, n, nnz, (int *)rp, (int *)ci, (double *)v}, S;
    int st = strength(&a, theta, &S);
    if (st) return st;
    *srp = S.rp; *sci = S.ci; *snnz = S.nnz;
    free(S.v);
    return OR_OK;
}

void or_free_buf(void *p) { free(p); }

/* ------------------------------------------------------------------------ */
/* Distance-2 maximal independent set (aggregate roots)                     */
/* ------------------------------------------------------------------------ */

/* MurmurHash3's 32-bit finaliser (Appleby, public domain): a bijection on
 * 32-bit words used as the node priority. */
uint32_t or_fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

/* Priority of node i: the pair (fmix32(i), i), compared lexicographically
 * (fmix32 is a bijection, so the hash alone already orders distinct nodes).
 * Larger pair = higher priority.  A block-diagonal batch of systems is
 * defined as the independent per-system problems, so i is always the index
 * within its own system. */
typedef struct { uint32_t h; int i; } okey;

static int key_gt(okey a, okey b) { return a.h != b.h ? a.h > b.h : a.i > b.i; }

static okey node_key(int i) {
    okey k;
    k.h = or_fmix32((uint32_t)i);
    k.i = i;
    return k;
}

static int cmp_key_desc(const void *pa, const void *pb) {
    okey ka = node_key(*(const int *)pa), kb = node_key(*(const int *)pb);
    if (key_gt(ka, kb)) return -1;
    if (key_gt(kb, ka)) return 1;
    return 0;
}

/* Serial greedy: visit nodes in decreasing priority; a node becomes a root
 * when no root lies within S-distance 2 of it.  This is the
 * lexicographically-first distance-2 MIS for the given priorities. */
static int mis2_greedy(const ocsr *S, int *root) {
    int n = S->nrows;
    int *order = (int *)malloc((size_t)n * sizeof(int));
    char *blocked = (char *)calloc((size_t)n, 1);
    if (!order || !blocked) return OR_ERR_OOM;
    for (int i = 0; i < n; ++i) order[i] = i;
    qsort(order, (size_t)n, sizeof(int), cmp_key_desc);
    memset(root, 0, (size_t)n * sizeof(int));
    for (int t = 0; t < n; ++t) {
        int i = order[t];
        if (blocked[i]) continue;
        root[i] = 1;
        blocked[i] = 1;
        for (int p = S->rp[i]; p < S->rp[i + 1]; ++p) {
            int j = S->ci[p];
            blocked[j] = 1;
            for (int q = S->rp[j]; q < S->rp[j + 1]; ++q) blocked[S->ci[q]] = 1;
        }
    }
    free(order); free(blocked);
    return OR_OK;
}

/* The same set computed by synchronous rounds, the form a parallel machine
 * uses: each node carries (state, priority) with state IN=2 > UNDECIDED=1 >
 * OUT=0.  M(i) = the largest tuple within S-distance 2 of i (closed
 * neighbourhoods, through nodes of any state).  An undecided node whose M(i)
 * is its own tuple joins; one whose M(i) has state IN leaves.  Repeat until
 * nothing is undecided.  Returns the number of rounds. */
typedef struct { int st; okey k; } otup;
static int tup_gt(otup a, otup b) { return a.st != b.st ? a.st > b.st : key_gt(a.k, b.k); }

static int mis2_rounds(const ocsr *S, int *root, int *nrounds) {
    int n = S->nrows;
    otup *t = (otup *)malloc((size_t)n * sizeof(otup));
    otup *m1 = (otup *)malloc((size_t)n * sizeof(otup));
    otup *m2 = (otup *)malloc((size_t)n * sizeof(otup));
    if (!t || !m1 || !m2) return OR_ERR_OOM;
    for (int i = 0; i < n; ++i) { t[i].st = 1; t[i].k = node_key(i); }
    int rounds = 0, und = n;
    while (und > 0) {
        rounds++;
        for (int j = 0; j < n; ++j) {
            otup m = t[j];
            for (int p = S->rp[j]; p < S->rp[j + 1]; ++p)
                if (tup_gt(t[S->ci[p]], m)) m = t[S->ci[p]];
            m1[j] = m;
        }
        for (int i = 0; i < n; ++i) {
            otup m = m1[i];
            for (int p = S->rp[i]; p < S->rp[i + 1]; ++p)
                if (tup_gt(m1[S->ci[p]], m)) m = m1[S->ci[p]];
            m2[i] = m;
        }
        und = 0;
        for (int i = 0; i < n; ++i) {
            if (t[i].st != 1) continue;
            if (m2[i].st == 1 && m2[i].k.i == i) t[i].st = 2;
            else if (m2[i].st == 2) t[i].st = 0;
            else und++;
        }
        if (rounds > n + 1) break; /* cannot happen: each round decides the top undecided node */
    }
    for (int i = 0; i < n; ++i) root[i] = (t[i].st == 2);
    if (nrounds) *nrounds = rounds;
    free(t); free(m1); free(m2);
    return und == 0 ? OR_OK : OR_ERR_STALL;
}

/* Exported for tests: roots of the MIS-2 of the strength graph given as
 * (srp, sci); method 0 = greedy, 1 = rounds. */
int or_mis2(int n, const int *srp, const int *sci, int method, int *root, int *nrounds) {
    ocsr S = {n, n, srp[n], (int *)srp, (int *)sci, NULL};
    return method == 0 ? mis2_greedy(&S, root) : mis2_rounds(&S, root, nrounds);
}

int or_aggregate_roots(int n, long long nnz, const int *rp, const int *ci, const double *v,
                       const int *srp, const int *sci, const int *root, int *agg, int *nc);

/* ------------------------------------------------------------------------ */
/* Aggregation                                                              */
/* ------------------------------------------------------------------------ */

/* Aggregates from the roots.
 *  Phase 1: roots get aggregate ids 0, 1, ... in increasing node index.
 *  Phase 2: a non-root with a root among its S-neighbours joins that root's
 *           aggregate (the root is unique: roots are >= 3 apart).
 *  Phase 3: every node still unassigned joins the aggregate of the strong
 *           neighbour j, assigned after phase 2, that maximises |a_ij|
 *           (|a_ij| = 0 when A does not store (i,j)); ties go to the smallest
 *           j.  Only the phase-2 snapshot is read, so no chains form.
 *  A node left without any assigned neighbour (impossible for a maximal
 *  MIS-2) becomes a singleton aggregate numbered after all roots, in
 *  increasing node index. */
static int aggregate(const ocsr *a, const ocsr *S, const int *root, int *agg, int *nc_out) {
    int n = a->nrows;
    int nc = 0;
    for (int i = 0; i < n; ++i) agg[i] = root[i] ? nc++ : -1;
    int *snap = (int *)malloc((size_t)n * sizeof(int));
    if (!snap) return OR_ERR_OOM;
    for (int i = 0; i < n; ++i) {
        snap[i] = agg[i];
        if (root[i]) continue;
        for (int p = S->rp[i]; p < S->rp[i + 1]; ++p)
            if (root[S->ci[p]]) { snap[i] = agg[S->ci[p]]; break; }
    }
    for (int i = 0; i < n; ++i) agg[i] = snap[i];
    for (int i = 0; i < n; ++i) {
        if (snap[i] >= 0) continue;
        int best = -1;
        double bw = -1.0;
        for (int p = S->rp[i]; p < S->rp[i + 1]; ++p) {
            int j = S->ci[p];
            if (snap[j] < 0) continue;
            double w = 0.0;
            for (int k = a->rp[i]; k < a->rp[i + 1]; ++k)
                if (a->ci[k] == j) { w = fabs(a->v[k]); break; }
            if (w > bw) { bw = w; best = j; }  /* columns ascend: first max = smallest j */
        }
        agg[i] = best >= 0 ? snap[best] : -1;
    }
    for (int i = 0; i < n; ++i)
        if (agg[i] < 0) agg[i] = nc++;
    free(snap);
    *nc_out = nc;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Prolongator                                                              */
/* ------------------------------------------------------------------------ */

/* Gershgorin bound of rho(D^-1 A): max_i (sum_j |a_ij| in storage order) / |a_ii|. */
static double gershgorin(const ocsr *a) {
    double rho = 0.0;
    for (int i = 0; i < a->nrows; ++i) {
        double s = 0.0;
        for (int k = a->rp[i]; k < a->rp[i + 1]; ++k) s = s + fabs(a->v[k]);
        double q = s / fabs(csr_diag(a, i));
        if (q > rho) rho = q;
    }
    return rho;
}

/* P = (I - omega_P D^-1 A) T with T the 0/1 aggregate indicator (column
 * agg(i) of row i) and omega_P = (4/3) / rho.
 * Row i of P stores the columns J in {agg(k) : k in row i of A}, ascending,
 * keeping exact zeros: P_iJ = [J == agg(i)] - omega_P * (s_iJ / a_ii), where
 * s_iJ = sum of a_ik over the row's entries with agg(k) = J, in storage
 * order starting from +0.0. */
static int prolongator(const ocsr *a, const int *agg, int nc, ocsr *P, double *rho_out) {
    int n = a->nrows;
    double rho = gershgorin(a);
    double c = 4.0 / 3.0;
    double omega_p = c / rho;
    *rho_out = rho;
    /* pass 1: count distinct aggregates per row */
    int *cols = (int *)malloc((size_t)nc * sizeof(int));
    int *mark = (int *)malloc((size_t)nc * sizeof(int));
    double *acc = (double *)malloc((size_t)nc * sizeof(double));
    if (!cols || !mark || !acc) return OR_ERR_OOM;
    for (int J = 0; J < nc; ++J) mark[J] = -1;
    long long tot = 0;
    for (int i = 0; i < n; ++i)
        for (int k = a->rp[i]; k < a->rp[i + 1]; ++k) {
            int J = agg[a->ci[k]];
            if (mark[J] != i) { mark[J] = i; tot++; }
        }
    if (csr_alloc(P, n, nc, tot)) return OR_ERR_OOM;
    for (int J = 0; J < nc; ++J) mark[J] = -1;
    long long pos = 0;
    for (int i = 0; i < n; ++i) {
        P->rp[i] = (int)pos;
        int m = 0;
        for (int k = a->rp[i]; k < a->rp[i + 1]; ++k) {
            int J = agg[a->ci[k]];
            if (mark[J] != i) { mark[J] = i; acc[J] = 0.0; cols[m++] = J; }
            acc[J] = acc[J] + a->v[k];
        }
        /* sort the row's columns ascending (insertion sort; rows are short) */
        for (int x = 1; x < m; ++x) {
            int c = cols[x], y = x - 1;
            while (y >= 0 && cols[y] > c) { cols[y + 1] = cols[y]; --y; }
            cols[y + 1] = c;
        }
        double aii = csr_diag(a, i);
        for (int x = 0; x < m; ++x) {
            int J = cols[x];
            double t = acc[J] / aii;
            double delta = (J == agg[i]) ? 1.0 : 0.0;
            P->ci[pos] = J;
            P->v[pos] = delta - omega_p * t;
            pos++;
        }
    }
    P->rp[n] = (int)pos;
    free(cols); free(mark); free(acc);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Galerkin product                                                         */
/* ------------------------------------------------------------------------ */

/* C = X Y (Gustavson, row by row).  For a fixed (i, J) the partial products
 * x_ik y_kJ are added in increasing k, starting from +0.0, each product and
 * each sum rounded separately.  The pattern is the structural union (exact
 * zeros kept), columns ascending. */
static int spgemm(const ocsr *X, const ocsr *Y, ocsr *C) {
    int n = X->nrows, m = Y->ncols;
    int *mark = (int *)malloc((size_t)m * sizeof(int));
    int *cols = (int *)malloc((size_t)m * sizeof(int));
    double *acc = (double *)malloc((size_t)m * sizeof(double));
    if (!mark || !cols || !acc) return OR_ERR_OOM;
    for (int J = 0; J < m; ++J) mark[J] = -1;
    long long tot = 0;
    for (int i = 0; i < n; ++i)
        for (int p = X->rp[i]; p < X->rp[i + 1]; ++p) {
            int k = X->ci[p];
            for (int q = Y->rp[k]; q < Y->rp[k + 1]; ++q) {
                int J = Y->ci[q];
                if (mark[J] != i) { mark[J] = i; tot++; }
            }
        }
    if (csr_alloc(C, n, m, tot)) return OR_ERR_OOM;
    for (int J = 0; J < m; ++J) mark[J] = -1;
    long long pos = 0;
    for (int i = 0; i < n; ++i) {
        C->rp[i] = (int)pos;
        int cnt = 0;
        for (int p = X->rp[i]; p < X->rp[i + 1]; ++p) {
            int k = X->ci[p];
            double xv = X->v[p];
            for (int q = Y->rp[k]; q < Y->rp[k + 1]; ++q) {
                int J = Y->ci[q];
                if (mark[J] != i) { mark[J] = i; acc[J] = 0.0; cols[cnt++] = J; }
                double prod = xv * Y->v[q];
                acc[J] = acc[J] + prod;
            }
        }
        for (int x = 1; x < cnt; ++x) {
            int c = cols[x], y = x - 1;
            while (y >= 0 && cols[y] > c) { cols[y + 1] = cols[y]; --y; }
            cols[y + 1] = c;
        }
        for (int x = 0; x < cnt; ++x) { C->ci[pos] = cols[x]; C->v[pos] = acc[cols[x]]; pos++; }
    }
    C->rp[n] = (int)pos;
    free(mark); free(cols); free(acc);
    return OR_OK;
}

/* A_c = P^T (A P): AP first, then R = P^T times AP, so (A_c)_IJ accumulates
 * P_iI (AP)_iJ in increasing fine index i. */
/* ------------------------------------------------------------------------ */
/* Classical (Ruge-Stueben) coarsening: the paper's other AMG family (its     */
/* Sec. 3.5 runs classical and aggregation AMG through the wrapped library;   */
/* the method itself is not given, so the textbook steps below are the       */
/* reading: Ruge & Stueben 1987, Stueben 2001, De Sterck, Yang & Heys 2006).   */
/* ------------------------------------------------------------------------ */

#define OR_THETA_CLASSICAL 0.25

/* Strong dependencies of row i (the directed relation S_i): j != i with
 * -a_ij >= theta_c max_{k != i}(-a_ik) and that maximum positive; theta_c =
 * 1/4 scales exactly.  Pattern-only CSR, columns ascending. */
static int strength_classical(const ocsr *a, ocsr *S) {
    const int n = a->nrows;
    long long cnt = 0;
    double *thr = (double *)malloc((size_t)n * sizeof(double));
    if (!thr) return OR_ERR_OOM;
    for (int pass = 0; pass < 2; ++pass) {
        long long pos = 0;
        for (int i = 0; i < n; ++i) {
            if (pass == 0) {
                double m = 0.0;
                for (int k = a->rp[i]; k < a->rp[i + 1]; ++k)
                    if (a->ci[k] != i && -a->v[k] > m) m = -a->v[k];
                thr[i] = m > 0.0 ? OR_THETA_CLASSICAL * m : -1.0; /* -1: no strong dependency */
            } else {
                S->rp[i] = (int)pos;
            }
            for (int k = a->rp[i]; k < a->rp[i + 1]; ++k) {
                const int j = a->ci[k];
                if (j == i || thr[i] < 0.0 || !(-a->v[k] >= thr[i])) continue;
                if (pass == 0) cnt++;
                else { S->ci[pos] = j; S->v[pos] = 1.0; pos++; }
            }
        }
        if (pass == 0) {
            if (csr_alloc(S, n, n, cnt)) { free(thr); return OR_ERR_OOM; }
        } else {
            S->rp[n] = (int)pos;
        }
    }
    free(thr);
    return OR_OK;
}

/* PMIS C/F splitting.  Weight w_i = |S^T_i| + fmix32(i) 2^-32 (the number of
 * points i strongly influences plus a hash fraction: no two weights tie).
 * Points that influence none (w_i < 1) start as F.  Each round, computed
 * from the state at its start: (a) every undecided point whose weight
 * exceeds that of every undecided neighbour in S_i or S^T_i becomes C;
 * (b) every still undecided point with a strong dependency on a new C point
 * becomes F.  cf[i]: 1 C, 0 F. */
static int pmis(const ocsr *S, const ocsr *St, int *cf, int *nrounds) {
    const int n = S->nrows;
    double *w = (double *)malloc((size_t)n * sizeof(double));
    int *st = (int *)malloc((size_t)n * sizeof(int));  /* -1 undecided, 0 F, 1 C */
    int *newc = (int *)malloc((size_t)n * sizeof(int));
    if (!w || !st || !newc) { free(w); free(st); free(newc); return OR_ERR_OOM; }
    for (int i = 0; i < n; ++i) {
        w[i] = (double)(St->rp[i + 1] - St->rp[i]) + ldexp((double)or_fmix32((uint32_t)i), -32);
        st[i] = w[i] < 1.0 ? 0 : -1;
    }
    int rounds = 0;
    for (;;) {
        int und = 0;
        for (int i = 0; i < n; ++i) und += st[i] < 0;
        if (!und) break;
        ++rounds;
        for (int i = 0; i < n; ++i) {
            newc[i] = 0;
            if (st[i] >= 0) continue;
            int best = 1;
            for (int k = S->rp[i]; k < S->rp[i + 1] && best; ++k) { int j = S->ci[k]; if (st[j] < 0 && w[j] >= w[i]) best = 0; }
            for (int k = St->rp[i]; k < St->rp[i + 1] && best; ++k) { int j = St->ci[k]; if (st[j] < 0 && w[j] >= w[i]) best = 0; }
            newc[i] = best;
        }
        for (int i = 0; i < n; ++i) if (newc[i]) st[i] = 1;
        for (int i = 0; i < n; ++i) {
            if (st[i] >= 0) continue;
            for (int k = S->rp[i]; k < S->rp[i + 1]; ++k) if (newc[S->ci[k]]) { st[i] = 0; break; }
        }
    }
    for (int i = 0; i < n; ++i) cf[i] = st[i];
    if (nrounds) *nrounds = rounds;
    free(w); free(st); free(newc);
    return OR_OK;
}

/* Direct interpolation (Stueben 2001): a C point keeps its value (P row e_c);
 * an F point i with strong C dependencies C_i interpolates from them with
 * w_ij = -(alpha a_ij) / d, alpha = (sum of the negative off-diagonal a_ik)
 * / (sum of a_ik over C_i), d = a_ii + (sum of the positive off-diagonal
 * a_ik); every strong dependency is negative, so the positive entries are
 * the ones lumped into d.  Sums run in CSR order.  An F point without strong
 * C dependencies gets an empty row.  cidx[i]: coarse index of C point i,
 * -1 for F. */
static int direct_interp(const ocsr *a, const ocsr *S, const int *cidx, int nc, ocsr *P) {
    const int n = a->nrows;
    long long cnt = 0;
    for (int i = 0; i < n; ++i) {
        if (cidx[i] >= 0) { cnt++; continue; }
        for (int k = S->rp[i]; k < S->rp[i + 1]; ++k) cnt += cidx[S->ci[k]] >= 0;
    }
    if (csr_alloc(P, n, nc, cnt)) return OR_ERR_OOM;
    long long pos = 0;
    for (int i = 0; i < n; ++i) {
        P->rp[i] = (int)pos;
        if (cidx[i] >= 0) { P->ci[pos] = cidx[i]; P->v[pos] = 1.0; pos++; continue; }
        double neg = 0.0, posv = 0.0, negc = 0.0, aii = 0.0;
        int s = S->rp[i];
        for (int k = a->rp[i]; k < a->rp[i + 1]; ++k) {
            const int j = a->ci[k];
            const double v = a->v[k];
            if (j == i) { aii = v; continue; }
            if (v < 0.0) neg = neg + v;
            else posv = posv + v;
            while (s < S->rp[i + 1] && S->ci[s] < j) ++s;
            if (s < S->rp[i + 1] && S->ci[s] == j && cidx[j] >= 0) negc = negc + v;
        }
        if (negc == 0.0) continue; /* no strong C dependency: empty row */
        const double alpha = neg / negc, d = aii + posv;
        s = S->rp[i];
        for (int k = a->rp[i]; k < a->rp[i + 1]; ++k) {
            const int j = a->ci[k];
            if (j == i) continue;
            while (s < S->rp[i + 1] && S->ci[s] < j) ++s;
            if (s < S->rp[i + 1] && S->ci[s] == j && cidx[j] >= 0) {
                P->ci[pos] = cidx[j];
                P->v[pos] = -(alpha * a->v[k]) / d;
                pos++;
            }
        }
    }
    P->rp[n] = (int)pos;
    P->nnz = pos;
    return OR_OK;
}

/* Exported for tests: the classical strength pattern and the PMIS splitting. */
int or_classical_split(int n, long long nnz, const int *rp, const int *ci, const double *v, int *cf, int *nrounds) {
    ocsr a = {n, n, nnz, (int *)rp, (int *)ci, (double *)v}, S, St;
    int st = strength_classical(&a, &S);
    if (st) return st;
    if ((st = csr_transpose(&S, &St))) { csr_free(&S); return st; }
    st = pmis(&S, &St, cf, nrounds);
    csr_free(&S); csr_free(&St);
    return st;
}

static int galerkin(const ocsr *A, const ocsr *P, const ocsr *R, ocsr *Ac) {
    ocsr AP;
    int st = spgemm(A, P, &AP);
    if (st) return st;
    st = spgemm(R, &AP, Ac);
    csr_free(&AP);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Dense coarsest level                                                     */
/* ------------------------------------------------------------------------ */

/* In-place Cholesky A = L L^T (lower triangle, row-major).  A pivot <= 0
 * means the matrix is not SPD. */
static int dense_cholesky(double *a, int n) {
    for (int j = 0; j < n; ++j) {
        double d = a[j * n + j];
        for (int k = 0; k < j; ++k) d = d - a[j * n + k] * a[j * n + k];
        if (!(d > 0.0)) return OR_NOT_SPD;
        double ljj = sqrt(d);
        a[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = a[i * n + j];
            for (int k = 0; k < j; ++k) s = s - a[i * n + k] * a[j * n + k];
            a[i * n + j] = s / ljj;
        }
    }
    return OR_OK;
}

/* In-place LU with partial pivoting (the first row of largest |.| in the
 * column wins ties); piv[k] = row swapped into position k. */
static int dense_lu(double *a, int *piv, int n) {
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(a[k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (fabs(a[i * n + k]) > best) { best = fabs(a[i * n + k]); p = i; }
        piv[k] = p;
        if (best == 0.0) return OR_NOT_SPD; /* singular */
        if (p != k)
            for (int j = 0; j < n; ++j) { double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
        for (int i = k + 1; i < n; ++i) {
            double l = a[i * n + k] / a[k * n + k];
            a[i * n + k] = l;
            for (int j = k + 1; j < n; ++j) a[i * n + j] = a[i * n + j] - l * a[k * n + j];
        }
    }
    return OR_OK;
}

static void dense_solve(const or_hier *h, const double *b, double *x) {
    int n = h->nc;
    const double *a = h->dense;
    for (int i = 0; i < n; ++i) x[i] = b[i];
    if (h->symmetric) {
        for (int i = 0; i < n; ++i) {   /* L y = b */
            double s = x[i];
            for (int k = 0; k < i; ++k) s = s - a[i * n + k] * x[k];
            x[i] = s / a[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {   /* L^T x = y */
            double s = x[i];
            for (int k = i + 1; k < n; ++k) s = s - a[k * n + i] * x[k];
            x[i] = s / a[i * n + i];
        }
    } else {
        for (int k = 0; k < n; ++k)
            if (h->piv[k] != k) { double t = x[k]; x[k] = x[h->piv[k]]; x[h->piv[k]] = t; }
        for (int i = 0; i < n; ++i) {
            double s = x[i];
            for (int k = 0; k < i; ++k) s = s - a[i * n + k] * x[k];
            x[i] = s;
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = x[i];
            for (int k = i + 1; k < n; ++k) s = s - a[i * n + k] * x[k];
            x[i] = s / a[i * n + i];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Setup                                                                    */
/* ------------------------------------------------------------------------ */

void or_config_default(or_config *c) {
    c->solver = 0;
    c->smoother = 0;
    c->omega = 2.0 / 3.0;
    c->theta = 0.08;
    c->coarse_max = 64;
    c->max_levels = 20;
    c->rtol = 1e-8;
    c->max_iter = 500;
    c->max_restarts = 3;
    c->symmetric = -1;
    c->adjoint_reuse = 0;
    c->amg_type = 0;
}

/* Symmetric = pattern symmetric and values bitwise equal. */
static int detect_symmetric(const ocsr *a) {
    ocsr t;
    if (csr_transpose(a, &t)) return 0;
    int sym = 1;
    for (int i = 0; i <= a->nrows && sym; ++i) if (a->rp[i] != t.rp[i]) sym = 0;
    for (long long k = 0; k < a->nnz && sym; ++k)
        if (a->ci[k] != t.ci[k] || memcmp(&a->v[k], &t.v[k], sizeof(double)) != 0) sym = 0;
    csr_free(&t);
    return sym;
}

/* Smoother: weighted Jacobi uses omega / a_ii; L1-Jacobi uses 1 / sum_j |a_ij|. */
static double *smoother_weights(const ocsr *a, const or_config *c) {
    double *d = (double *)malloc((size_t)a->nrows * sizeof(double));
    if (!d) return NULL;
    for (int i = 0; i < a->nrows; ++i) {
        if (c->smoother == 1) {
            double s = 0.0;
            for (int k = a->rp[i]; k < a->rp[i + 1]; ++k) s = s + fabs(a->v[k]);
            d[i] = 1.0 / s;
        } else {
            d[i] = c->omega / csr_diag(a, i);
        }
    }
    return d;
}

void or_hier_free(or_hier *h);

/* Builds the hierarchy.  Coarsening stops when a level has <= coarse_max
 * rows, when max_levels levels exist or when a level fails to shrink; the
 * last level must then have at most OR_DENSE_MAX rows, else OR_ERR_STALL. */
or_hier *or_setup(const or_config *cfg_in, int n, long long nnz, const int *rp, const int *ci,
                  const double *v, int *status) {
    or_config cfg;
    if (cfg_in) cfg = *cfg_in; else or_config_default(&cfg);
    int st = or_validate(n, nnz, rp, ci, v);
    if (st) { *status = st; return NULL; }
    or_hier *h = (or_hier *)calloc(1, sizeof(or_hier));
    if (!h) { *status = OR_ERR_OOM; return NULL; }
    h->cfg = cfg;
    if (csr_copy(&h->A[0], n, nnz, rp, ci, v)) { *status = OR_ERR_OOM; or_hier_free(h); return NULL; }
    h->symmetric = cfg.symmetric >= 0 ? cfg.symmetric : detect_symmetric(&h->A[0]);
    int l = 0;
    for (;;) {
        ocsr *A = &h->A[l];
        h->dinv[l] = smoother_weights(A, &cfg);
        if (A->nrows <= cfg.coarse_max || l + 1 >= cfg.max_levels || l + 1 >= OR_MAX_LEVELS) break;
        /* strength threshold halves at every coarser level: theta_l = theta 2^-l
         * (Vanek, Mandel & Brezina 1996); scaling by a power of two is exact */
        if (cfg.amg_type == 1) {
            /* classical: strength, PMIS C/F, direct interpolation; agg[l]
             * holds each row's coarse index (-1 for F points) */
            ocsr S, St;
            if ((st = strength_classical(A, &S))) { *status = st; or_hier_free(h); return NULL; }
            if ((st = csr_transpose(&S, &St))) { csr_free(&S); *status = st; or_hier_free(h); return NULL; }
            h->agg[l] = (int *)malloc((size_t)A->nrows * sizeof(int));
            st = h->agg[l] ? pmis(&S, &St, h->agg[l], NULL) : OR_ERR_OOM;
            int nc = 0;
            if (!st)
                for (int i = 0; i < A->nrows; ++i) h->agg[l][i] = h->agg[l][i] ? nc++ : -1;
            if (!st && nc > 0 && nc < A->nrows) st = direct_interp(A, &S, h->agg[l], nc, &h->P[l]);
            csr_free(&S); csr_free(&St);
            if (st) { *status = st; or_hier_free(h); return NULL; }
            if (nc == 0 || nc >= A->nrows) { free(h->agg[l]); h->agg[l] = NULL; break; } /* stalled */
            if ((st = csr_transpose(&h->P[l], &h->R[l]))) { *status = st; or_hier_free(h); return NULL; }
            if ((st = galerkin(A, &h->P[l], &h->R[l], &h->A[l + 1]))) { *status = st; or_hier_free(h); return NULL; }
            l++;
            continue;
        }
        double theta_l = ldexp(cfg.theta, -l);
        ocsr S;
        if ((st = strength(A, theta_l, &S))) { *status = st; or_hier_free(h); return NULL; }
        int *root = (int *)malloc((size_t)A->nrows * sizeof(int));
        h->agg[l] = (int *)malloc((size_t)A->nrows * sizeof(int));
        st = mis2_greedy(&S, root);
        int nc = 0;
        if (!st) st = aggregate(A, &S, root, h->agg[l], &nc);
        free(root);
        h->S[l] = S;  /* kept for the tests' export (or_hier_get_strength) */
        if (st) { *status = st; or_hier_free(h); return NULL; }
        if (nc >= A->nrows) { free(h->agg[l]); h->agg[l] = NULL; break; } /* stalled */
        if ((st = prolongator(A, h->agg[l], nc, &h->P[l], &h->rho[l]))) {
            *status = st; or_hier_free(h); return NULL;
        }
        if ((st = csr_transpose(&h->P[l], &h->R[l]))) { *status = st; or_hier_free(h); return NULL; }
        if ((st = galerkin(A, &h->P[l], &h->R[l], &h->A[l + 1]))) { *status = st; or_hier_free(h); return NULL; }
        l++;
    }
    h->nlevels = l + 1;
    ocsr *Ac = &h->A[l];
    if (Ac->nrows > OR_DENSE_MAX) { *status = OR_ERR_STALL; or_hier_free(h); return NULL; }
    int m = Ac->nrows;
    h->nc = m;
    h->dense = (double *)calloc((size_t)m * m, sizeof(double));
    h->piv = (int *)malloc((size_t)m * sizeof(int));
    for (int i = 0; i < m; ++i)
        for (int k = Ac->rp[i]; k < Ac->rp[i + 1]; ++k) h->dense[i * m + Ac->ci[k]] = Ac->v[k];
    st = h->symmetric ? dense_cholesky(h->dense, m) : dense_lu(h->dense, h->piv, m);
    if (st) { *status = st; or_hier_free(h); return NULL; }
    *status = OR_OK;
    return h;
}

/* Numeric re-setup (Sec. 2.1, C++/CUDA backend: on a cache hit the setup is
 * repeated against new coefficients while the structure of the first setup
 * is kept).  Reading: the aggregates of every level and hence every sparsity
 * pattern (P, R, the coarse operators) are those of `old`; the smoother
 * weights, omega_P, P, R, the Galerkin products and the coarsest factor are
 * recomputed from the new values v (same pattern as old's finest operator),
 * by the same formulas as or_setup.  The symmetry flag is kept. */
/* Re-setup of a classical level's interpolation: the C/F map and P's pattern
 * (each F row's interpolation set C_i) are kept and the weights recomputed
 * from the new values by the direct-interpolation formula, with the sum over
 * C_i taken over P's columns whatever the new entries' signs; a row whose
 * sum over C_i is zero gets zero weights. */
static int direct_interp_values(const ocsr *a, const int *cidx, ocsr *P) {
    const int n = a->nrows;
    for (int i = 0; i < n; ++i) {
        const int p0 = P->rp[i], p1 = P->rp[i + 1];
        if (cidx[i] >= 0 || p0 == p1) continue; /* C rows stay unit rows */
        double neg = 0.0, posv = 0.0, negc = 0.0, aii = 0.0;
        int q = p0;
        for (int k = a->rp[i]; k < a->rp[i + 1]; ++k) {
            const int j = a->ci[k];
            const double v = a->v[k];
            if (j == i) { aii = v; continue; }
            if (v < 0.0) neg = neg + v;
            else posv = posv + v;
            if (cidx[j] >= 0) {
                while (q < p1 && P->ci[q] < cidx[j]) ++q;
                if (q < p1 && P->ci[q] == cidx[j]) negc = negc + v;
            }
        }
        q = p0;
        for (int k = a->rp[i]; k < a->rp[i + 1]; ++k) {
            const int j = a->ci[k];
            if (j == i || cidx[j] < 0) continue;
            while (q < p1 && P->ci[q] < cidx[j]) ++q;
            if (q < p1 && P->ci[q] == cidx[j]) {
                if (negc == 0.0) { P->v[q] = 0.0; continue; }
                const double alpha = neg / negc, d = aii + posv;
                P->v[q] = -(alpha * a->v[k]) / d;
            }
        }
    }
    return OR_OK;
}

or_hier *or_resetup(const or_hier *old, const double *v, int *status) {
    const ocsr *A0 = &old->A[0];
    or_hier *h = (or_hier *)calloc(1, sizeof(or_hier));
    if (!h) { *status = OR_ERR_OOM; return NULL; }
    h->cfg = old->cfg;
    int st;
    if (csr_copy(&h->A[0], A0->nrows, A0->nnz, A0->rp, A0->ci, v)) { *status = OR_ERR_OOM; or_hier_free(h); return NULL; }
    if ((st = or_validate(A0->nrows, A0->nnz, A0->rp, A0->ci, v))) { *status = st; or_hier_free(h); return NULL; }
    h->symmetric = old->symmetric;
    const int L = old->nlevels;
    for (int l = 0; l < L; ++l) {
        ocsr *A = &h->A[l];
        h->dinv[l] = smoother_weights(A, &h->cfg);
        if (l == L - 1) break;
        const int n = A->nrows, nc = old->A[l + 1].nrows;
        h->agg[l] = (int *)malloc((size_t)n * sizeof(int));
        if (!h->agg[l]) { *status = OR_ERR_OOM; or_hier_free(h); return NULL; }
        memcpy(h->agg[l], old->agg[l], (size_t)n * sizeof(int));
        if (h->cfg.amg_type == 1) {
            const ocsr *Po = &old->P[l];
            if (csr_alloc(&h->P[l], Po->nrows, Po->ncols, Po->nnz)) { *status = OR_ERR_OOM; or_hier_free(h); return NULL; }
            memcpy(h->P[l].rp, Po->rp, ((size_t)Po->nrows + 1) * sizeof(int));
            memcpy(h->P[l].ci, Po->ci, (size_t)Po->nnz * sizeof(int));
            memcpy(h->P[l].v, Po->v, (size_t)Po->nnz * sizeof(double)); /* C rows: unit entries */
            direct_interp_values(A, h->agg[l], &h->P[l]);
        } else if ((st = prolongator(A, h->agg[l], nc, &h->P[l], &h->rho[l]))) {
            *status = st; or_hier_free(h); return NULL;
        }
        if ((st = csr_transpose(&h->P[l], &h->R[l]))) { *status = st; or_hier_free(h); return NULL; }
        if ((st = galerkin(A, &h->P[l], &h->R[l], &h->A[l + 1]))) { *status = st; or_hier_free(h); return NULL; }
    }
    h->nlevels = L;
    ocsr *Ac = &h->A[L - 1];
    const int m = Ac->nrows;
    h->nc = m;
    h->dense = (double *)calloc((size_t)m * m, sizeof(double));
    h->piv = (int *)malloc((size_t)m * sizeof(int));
    if (!h->dense || !h->piv) { *status = OR_ERR_OOM; or_hier_free(h); return NULL; }
    for (int i = 0; i < m; ++i)
        for (int k = Ac->rp[i]; k < Ac->rp[i + 1]; ++k) h->dense[i * m + Ac->ci[k]] = Ac->v[k];
    st = h->symmetric ? dense_cholesky(h->dense, m) : dense_lu(h->dense, h->piv, m);
    if (st) { *status = st; or_hier_free(h); return NULL; }
    *status = OR_OK;
    return h;
}

/* The hierarchy of A^T that reuses A's: the same aggregates, P and R = P^T,
 * with every level operator the transpose of A's.  Since R = P^T, the
 * transpose of A's Galerkin product is the Galerkin product of the
 * transposed operator, R A_l^T P = (R A_l P)^T = A_{l+1}^T, so this is a
 * smoothed-aggregation-style hierarchy of A^T without a second setup (reusing
 * P, which was smoothed with A rather than A^T, is the reading).  Smoother
 * weights come from the transposed operators (the same diagonal; column sums
 * for L1-Jacobi); the coarsest level is factored by LU. */
or_hier *or_transposed(const or_hier *f, int *status) {
    or_hier *h = (or_hier *)calloc(1, sizeof(or_hier));
    if (!h) { *status = OR_ERR_OOM; return NULL; }
    h->cfg = f->cfg;
    h->symmetric = 0;
    const int L = f->nlevels;
    int st;
    for (int l = 0; l < L; ++l) {
        if ((st = csr_transpose(&f->A[l], &h->A[l]))) { *status = st; or_hier_free(h); return NULL; }
        h->dinv[l] = smoother_weights(&h->A[l], &h->cfg);
        if (!h->dinv[l]) { *status = OR_ERR_OOM; or_hier_free(h); return NULL; }
        if (l == L - 1) break;
        const int n = f->A[l].nrows;
        const ocsr *P = &f->P[l], *R = &f->R[l];
        h->agg[l] = (int *)malloc((size_t)n * sizeof(int));
        if (!h->agg[l] || csr_alloc(&h->P[l], P->nrows, P->ncols, P->nnz) ||
            csr_alloc(&h->R[l], R->nrows, R->ncols, R->nnz)) {
            *status = OR_ERR_OOM; or_hier_free(h); return NULL;
        }
        memcpy(h->agg[l], f->agg[l], (size_t)n * sizeof(int));
        memcpy(h->P[l].rp, P->rp, ((size_t)P->nrows + 1) * sizeof(int));
        memcpy(h->P[l].ci, P->ci, (size_t)P->nnz * sizeof(int));
        memcpy(h->P[l].v, P->v, (size_t)P->nnz * sizeof(double));
        memcpy(h->R[l].rp, R->rp, ((size_t)R->nrows + 1) * sizeof(int));
        memcpy(h->R[l].ci, R->ci, (size_t)R->nnz * sizeof(int));
        memcpy(h->R[l].v, R->v, (size_t)R->nnz * sizeof(double));
        h->rho[l] = f->rho[l];
    }
    h->nlevels = L;
    const ocsr *Ac = &h->A[L - 1];
    const int m = Ac->nrows;
    h->nc = m;
    h->dense = (double *)calloc((size_t)m * m, sizeof(double));
    h->piv = (int *)malloc((size_t)m * sizeof(int));
    if (!h->dense || !h->piv) { *status = OR_ERR_OOM; or_hier_free(h); return NULL; }
    for (int i = 0; i < m; ++i)
        for (int k = Ac->rp[i]; k < Ac->rp[i + 1]; ++k) h->dense[i * m + Ac->ci[k]] = Ac->v[k];
    if ((st = dense_lu(h->dense, h->piv, m))) { *status = st; or_hier_free(h); return NULL; }
    *status = OR_OK;
    return h;
}

void or_hier_free(or_hier *h) {
    if (!h) return;
    for (int l = 0; l < OR_MAX_LEVELS; ++l) {
        csr_free(&h->A[l]); csr_free(&h->P[l]); csr_free(&h->R[l]); csr_free(&h->S[l]);
        free(h->agg[l]); free(h->dinv[l]);
    }
    free(h->dense); free(h->piv);
    if (h->adj) or_hier_free(h->adj);
    free(h);
}

/* Accessors for tests. */
int or_hier_nlevels(const or_hier *h) { return h->nlevels; }
int or_hier_symmetric(const or_hier *h) { return h->symmetric; }
double or_hier_rho(const or_hier *h, int l) { return h->rho[l]; }
void or_hier_dims(const or_hier *h, int l, int *n, long long *nnzA, int *nc, long long *nnzP) {
    *n = h->A[l].nrows; *nnzA = h->A[l].nnz;
    *nc = l + 1 < h->nlevels ? h->A[l + 1].nrows : 0;
    *nnzP = l + 1 < h->nlevels ? h->P[l].nnz : 0;
}
/* which: 0 = A, 1 = P, 2 = R */
void or_hier_get(const or_hier *h, int l, int which, int *rp, int *ci, double *v) {
    const ocsr *m = which == 0 ? &h->A[l] : which == 1 ? &h->P[l] : &h->R[l];
    memcpy(rp, m->rp, ((size_t)m->nrows + 1) * sizeof(int));
    memcpy(ci, m->ci, (size_t)m->nnz * sizeof(int));
    memcpy(v, m->v, (size_t)m->nnz * sizeof(double));
}
void or_hier_get_agg(const or_hier *h, int l, int *agg) {
    memcpy(agg, h->agg[l], (size_t)h->A[l].nrows * sizeof(int));
}
/* The strength graph level l's aggregation used (setup of a smoothed-
 * aggregation hierarchy; -1 when the level kept none): its entry count, then
 * its pattern into srp (n_l + 1) and sci. */
long long or_hier_strength_nnz(const or_hier *h, int l) { return h->S[l].rp ? h->S[l].nnz : -1; }
void or_hier_get_strength(const or_hier *h, int l, int *srp, int *sci) {
    memcpy(srp, h->S[l].rp, ((size_t)h->S[l].nrows + 1) * sizeof(int));
    memcpy(sci, h->S[l].ci, (size_t)h->S[l].nnz * sizeof(int));
}

/* ------------------------------------------------------------------------ */
/* V(1,1) cycle                                                             */
/* ------------------------------------------------------------------------ */

/* x = M^-1 b at level l, x0 = 0:
 *   x = W b                  (W = omega D^-1, or the L1 weights)
 *   r = b - A x
 *   x_c = V(l+1, P^T r)
 *   x = x + P x_c
 *   x = x + W (b - A x)
 * and the dense solve at the last level. */
static void vcycle(const or_hier *h, int l, const double *b, double *x) {
    if (l == h->nlevels - 1) { dense_solve(h, b, x); return; }
    const ocsr *A = &h->A[l], *P = &h->P[l], *R = &h->R[l];
    int n = A->nrows, nc = P->ncols;
    const double *w = h->dinv[l];
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *bc = (double *)malloc((size_t)nc * sizeof(double));
    double *xc = (double *)malloc((size_t)nc * sizeof(double));
    OR_PAR
    for (int i = 0; i < n; ++i) x[i] = w[i] * b[i];
    spmv(A, x, r);
    OR_PAR
    for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
    spmv(R, r, bc);
    vcycle(h, l + 1, bc, xc);
    spmv(P, xc, r);
    OR_PAR
    for (int i = 0; i < n; ++i) x[i] = x[i] + r[i];
    spmv(A, x, r);
    OR_PAR
    for (int i = 0; i < n; ++i) x[i] = x[i] + w[i] * (b[i] - r[i]);
    free(r); free(bc); free(xc);
}

void or_vcycle(const or_hier *h, const double *b, double *x) { vcycle(h, 0, b, x); }

/* ------------------------------------------------------------------------ */
/* Krylov solvers                                                           */
/* ------------------------------------------------------------------------ */

#ifdef _OPENMP
/* Threaded build (timing only): fixed chunks of OR_CHUNK entries, each summed
 * in order, then the chunk sums in order -- the same bits for any thread
 * count, though not the serial build's bits. */
#define OR_CHUNK 16384
static double dot(int n, const double *a, const double *b) {
    int nch = (n + OR_CHUNK - 1) / OR_CHUNK;
    double *part = (double *)malloc((size_t)(nch > 0 ? nch : 1) * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nch; ++c) {
        int i1 = (c + 1) * OR_CHUNK < n ? (c + 1) * OR_CHUNK : n;
        double s = 0.0;
        for (int i = c * OR_CHUNK; i < i1; ++i) s = s + a[i] * b[i];
        part[c] = s;
    }
    double s = 0.0;
    for (int c = 0; c < nch; ++c) s = s + part[c];
    free(part);
    return s;
}
#else
static double dot(int n, const double *a, const double *b) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = s + a[i] * b[i];
    return s;
}
#endif

static void precond(const or_hier *h, int use, const double *r, double *z) {
    if (use) vcycle(h, 0, r, z);
    else memcpy(z, r, (size_t)h->A[0].nrows * sizeof(double));
}

static double true_residual(const or_hier *h, const double *b, const double *x, double *r) {
    int n = h->A[0].nrows;
    spmv(&h->A[0], x, r);
    OR_PAR
    for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
    return sqrt(dot(n, r, r));
}

/* Preconditioned CG (Hestenes-Stiefel), x0 = 0.  Stops when
 * ||r||_2 <= rtol ||b||_2 on the recursive residual; then the true residual
 * b - A x decides, and while it is above rtol (at most max_restarts times) CG
 * restarts from the current x.  iters counts products q = A p. */
static int pcg(const or_hier *h, int use_prec, const double *b, double *x, or_info *info) {
    int n = h->A[0].nrows;
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *z = (double *)malloc((size_t)n * sizeof(double));
    double *p = (double *)malloc((size_t)n * sizeof(double));
    double *q = (double *)malloc((size_t)n * sizeof(double));
    double bn = sqrt(dot(n, b, b));
    int status = OR_OK, iters = 0, restarts = 0;
    double rn = 0.0;
    memset(x, 0, (size_t)n * sizeof(double));
    if (bn == 0.0) { info->status = OR_OK; info->iters = 0; info->restarts = 0; info->rel_res_true = 0.0; info->rel_res_rec = 0.0; free(r); free(z); free(p); free(q); return OR_OK; }
    if (!isfinite(bn)) status = OR_NAN;
    memcpy(r, b, (size_t)n * sizeof(double));
    for (;;) {
        if (status) break;
        precond(h, use_prec, r, z);
        memcpy(p, z, (size_t)n * sizeof(double));
        double rz = dot(n, r, z);
        int conv = 0;
        while (iters < h->cfg.max_iter) {
            spmv(&h->A[0], p, q);
            double pq = dot(n, p, q);
            iters++;
            if (!isfinite(pq) || !isfinite(rz)) { status = OR_NAN; break; }
            if (pq <= 0.0) { status = OR_BREAKDOWN; break; }
            double alpha = rz / pq;
            OR_PAR
            for (int i = 0; i < n; ++i) { x[i] = x[i] + alpha * p[i]; r[i] = r[i] - alpha * q[i]; }
            rn = sqrt(dot(n, r, r));
            if (!isfinite(rn)) { status = OR_NAN; break; }
            if (rn <= h->cfg.rtol * bn) { conv = 1; break; }
            precond(h, use_prec, r, z);
            double rz_new = dot(n, r, z);
            double beta = rz_new / rz;
            rz = rz_new;
            OR_PAR
            for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        }
        if (status) break;
        if (!conv) { status = OR_MAXIT; break; }
        double tr = true_residual(h, b, x, r);
        if (tr <= h->cfg.rtol * bn || restarts >= h->cfg.max_restarts) {
            if (tr > h->cfg.rtol * bn) status = OR_MAXIT;
            break;
        }
        restarts++;   /* r already holds the true residual */
    }
    info->rel_res_rec = rn / bn;
    info->rel_res_true = true_residual(h, b, x, q) / bn;
    info->iters = iters;
    info->restarts = restarts;
    info->status = status;
    free(r); free(z); free(p); free(q);
    return status;
}

/* Right-preconditioned BiCGStab (van der Vorst), x0 = 0, shadow residual
 * r_hat = r0.  One iteration = up to two products with A.  On breakdown
 * (rho = 0 or omega = 0) the method restarts once from the current x with
 * r_hat = r; a second breakdown returns OR_BREAKDOWN.  Same stopping rule and
 * true-residual restarts as CG. */
static int bicgstab(const or_hier *h, int use_prec, const double *b, double *x, or_info *info) {
    int n = h->A[0].nrows;
    size_t sz = (size_t)n * sizeof(double);
    double *r = malloc(sz), *rh = malloc(sz), *p = malloc(sz), *v = malloc(sz), *ph = malloc(sz);
    double *s = malloc(sz), *sh = malloc(sz), *t = malloc(sz);
    double bn = sqrt(dot(n, b, b));
    int status = OR_OK, iters = 0, restarts = 0, bd_restarts = 0;
    double rn = 0.0;
    memset(x, 0, sz);
    if (bn == 0.0) { info->status = OR_OK; info->iters = 0; info->restarts = 0; info->rel_res_true = 0; info->rel_res_rec = 0; goto done; }
    if (!isfinite(bn)) { status = OR_NAN; goto finish; }
    memcpy(r, b, sz);
    for (;;) {
        memcpy(rh, r, sz);
        memset(p, 0, sz); memset(v, 0, sz);
        double rho_old = 1.0, alpha = 1.0, omega = 1.0;
        int conv = 0, breakdown = 0;
        while (iters < h->cfg.max_iter) {
            double rho = dot(n, rh, r);
            if (!isfinite(rho)) { status = OR_NAN; break; }
            if (rho == 0.0) { breakdown = 1; break; }
            iters++;  /* an iteration counts once it goes on to its products with A */
            double beta = (rho / rho_old) * (alpha / omega);
            OR_PAR
            for (int i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
            precond(h, use_prec, p, ph);
            spmv(&h->A[0], ph, v);
            double rv = dot(n, rh, v);
            if (!isfinite(rv)) { status = OR_NAN; break; }
            if (rv == 0.0) { breakdown = 1; break; }
            alpha = rho / rv;
            OR_PAR
            for (int i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
            double sn = sqrt(dot(n, s, s));
            if (sn <= h->cfg.rtol * bn) {
                OR_PAR
                for (int i = 0; i < n; ++i) x[i] = x[i] + alpha * ph[i];
                memcpy(r, s, sz);
                rn = sn; conv = 1; break;
            }
            precond(h, use_prec, s, sh);
            spmv(&h->A[0], sh, t);
            double tt = dot(n, t, t), ts = dot(n, t, s);
            if (!isfinite(tt) || !isfinite(ts)) { status = OR_NAN; break; }
            if (tt == 0.0) { breakdown = 1; break; }
            omega = ts / tt;
            OR_PAR
            for (int i = 0; i < n; ++i) {
                x[i] = x[i] + alpha * ph[i] + omega * sh[i];
                r[i] = s[i] - omega * t[i];
            }
            rn = sqrt(dot(n, r, r));
            if (!isfinite(rn)) { status = OR_NAN; break; }
            if (rn <= h->cfg.rtol * bn) { conv = 1; break; }
            if (omega == 0.0) { breakdown = 1; break; }
            rho_old = rho;
        }
        if (status) break;
        if (breakdown) {
            if (bd_restarts >= 1) { status = OR_BREAKDOWN; break; }
            bd_restarts++;
            true_residual(h, b, x, r);
            continue;
        }
        if (!conv) { status = OR_MAXIT; break; }
        double tr = true_residual(h, b, x, r);
        if (tr <= h->cfg.rtol * bn || restarts >= h->cfg.max_restarts) {
            if (tr > h->cfg.rtol * bn) status = OR_MAXIT;
            break;
        }
        restarts++;
    }
finish:
    info->rel_res_rec = bn > 0 ? rn / bn : 0.0;
    info->rel_res_true = bn > 0 ? true_residual(h, b, x, t) / bn : 0.0;
    info->iters = iters;
    info->restarts = restarts;
    info->status = status;
done:
    free(r); free(rh); free(p); free(v); free(ph); free(s); free(sh); free(t);
    return info->status;
}

int or_solve(const or_hier *h, const double *b, double *x, or_info *info) {
    switch (h->cfg.solver) {
        case 0: return pcg(h, 1, b, x, info);
        case 1: return bicgstab(h, 1, b, x, info);
        case 2: return pcg(h, 0, b, x, info);
        case 3: return bicgstab(h, 0, b, x, info);
        default: return OR_ERR_ARG;
    }
}

/* ------------------------------------------------------------------------ */
/* Adjoint (Eq. 1-2)                                                        */
/* ------------------------------------------------------------------------ */

/* lambda solves A^T lambda = g with the same solver and configuration; for a
 * symmetric A the forward hierarchy is reused, otherwise a hierarchy is set
 * up on A^T (once, kept with the handle), or with adjoint_reuse the
 * transposed hierarchy of or_transposed.  dL/dA on the stored pattern:
 * dA_k = -lambda_{row(k)} x_{col(k)};  dL/db = lambda. */
int or_adjoint(or_hier *h, const double *x, const double *g, double *lambda, double *dA, or_info *info) {
    const or_hier *hs = h;
    if (!h->symmetric) {
        if (!h->adj && h->cfg.adjoint_reuse) {
            int st;
            h->adj = or_transposed(h, &st);
            if (!h->adj) return st;
        } else if (!h->adj) {
            ocsr At;
            if (csr_transpose(&h->A[0], &At)) return OR_ERR_OOM;
            or_config c = h->cfg;
            c.symmetric = 0;
            int st;
            h->adj = or_setup(&c, At.nrows, At.nnz, At.rp, At.ci, At.v, &st);
            csr_free(&At);
            if (!h->adj) return st;
        }
        hs = h->adj;
    }
    int st = or_solve(hs, g, lambda, info);
    const ocsr *A = &h->A[0];
    OR_PAR
    for (int i = 0; i < A->nrows; ++i)
        for (int k = A->rp[i]; k < A->rp[i + 1]; ++k) dA[k] = -(lambda[i] * x[A->ci[k]]);
    return st;
}

/* Dense helpers for tests: the coarsest factor solve and the level data. */
void or_dense_solve(const or_hier *h, const double *b, double *x) { dense_solve(h, b, x); }
int or_hier_coarse_n(const or_hier *h) { return h->nc; }

/* Exported for tests: aggregates from given roots (phases 1-3 above). */
int or_aggregate_roots(int n, long long nnz, const int *rp, const int *ci, const double *v,
                       const int *srp, const int *sci, const int *root, int *agg, int *nc) {
    ocsr a = {n, n, nnz, (int *)rp, (int *)ci, (double *)v};
    ocsr S = {n, n, srp[n], (int *)srp, (int *)sci, NULL};
    return aggregate(&a, &S, root, agg, nc);
}
