/*
 * amg_b300.h -- C ABI of libamgb300.so: an algebraic-multigrid-preconditioned
 * Krylov solver for sparse CSR systems with a reverse-mode adjoint, for one
 * NVIDIA B300 GPU (sm_103a).
 *
 * What the paper defines and this library provides:
 *   - a single solve entry on a CSR matrix with a configurable Krylov solver
 *     and AMG preconditioner (JAX-AMG paper, Sec. 2.1 "Python API": inputs are
 *     normalised to CSR; default BiCGSTAB + AMG);
 *   - setup caching: the hierarchy built once by amg_setup is reused by every
 *     amg_solve / amg_adjoint on the handle (Sec. 2.1 "C++/CUDA backend":
 *     solver handles are cached and reused across solves; Sec. 3.5 runs with a
 *     fixed hierarchy, reuse_setup=True);
 *   - the adjoint of the solve (Sec. 2.1 "JAX integration", Eq. 1-2):
 *     A^T lambda = dL/dx, dL/dA = -lambda x^T (on the stored pattern),
 *     dL/db = lambda; for symmetric A the forward hierarchy is reused, for a
 *     nonsymmetric A a hierarchy is built on A^T;
 *   - diagnostics: iteration count, final residual, convergence status and
 *     hierarchy statistics (Sec. 2.2, last paragraph).
 * The AMG method itself is not specified by the paper; this library builds a
 * smoothed-aggregation hierarchy (strength of connection, distance-2 MIS
 * aggregation, Jacobi-smoothed prolongator, Galerkin P^T A P) entirely on the
 * GPU, deterministically.
 *
 * Conventions for every entry point:
 *   - Index arrays are int32, values FP64.  A CSR matrix is square n x n with
 *     row_ptr[n+1] (row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz < 2^31)
 *     and col_idx[nnz] strictly ascending within each row; every row stores a
 *     nonzero diagonal.
 *   - Array arguments may be device pointers or host pointers (pageable or
 *     pinned); the library looks up each pointer's memory type and stages host
 *     arrays through device memory it owns.  The caller owns every array it
 *     passes; the library never keeps a caller pointer after a call returns.
 *   - cuda_stream is a cudaStream_t (NULL = the legacy default stream).  All
 *     GPU work of a call is ordered on that stream; calls that return results
 *     in amg_info, or that read host arrays, synchronise the stream before
 *     returning.
 *   - A handle may be used by one host thread at a time.
 *   - Return value: AMG_OK (0); a positive soft status (AMG_MAXIT,
 *     AMG_BREAKDOWN, AMG_NAN) after which the outputs hold the last iterate
 *     and info->status repeats the code; or a negative hard error, after which
 *     the outputs are unspecified and amg_last_error() describes the failure.
 */
#ifndef AMG_B300_H
#define AMG_B300_H

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define AMG_OK 0
#define AMG_MAXIT 1          /* max_iter reached before the tolerance */
#define AMG_BREAKDOWN 2      /* Krylov breakdown (p.q <= 0 in PCG; rho, r^.v, t.t or omega = 0 twice in BiCGStab) */
#define AMG_NOT_SPD 3        /* coarsest Cholesky met a pivot <= 0 (or LU a zero pivot) */
#define AMG_NAN 4            /* non-finite value in the right-hand side or an iterate */
#define AMG_ERR_ARG (-1)     /* bad argument (NULL handle/pointer, n <= 0, ...) */
#define AMG_ERR_BAD_CSR (-2) /* row_ptr not monotone / out of range, column out of range or not ascending */
#define AMG_ERR_ZERO_DIAG (-3) /* a row without a stored diagonal, or a zero diagonal */
#define AMG_ERR_CUDA (-4)    /* a CUDA runtime error */
#define AMG_ERR_STALL (-5)   /* coarsening stopped with more than AMG_DENSE_MAX rows on the last level */
#define AMG_ERR_OOM (-6)     /* device allocation failed */
#define AMG_ERR_UNSUPPORTED (-7) /* a size beyond a documented limit */

#define AMG_MAX_LEVELS 32
#define AMG_DENSE_MAX 256    /* largest coarsest level solved densely */

/* Solvers. */
#define AMG_SOLVER_PCG 0            /* AMG-preconditioned CG (SPD A) */
#define AMG_SOLVER_BICGSTAB 1       /* AMG right-preconditioned BiCGStab */
#define AMG_SOLVER_CG 2             /* CG without preconditioner (setup builds no coarse levels) */
#define AMG_SOLVER_BICGSTAB_NOPREC 3 /* BiCGStab without preconditioner (no coarse levels either) */

/* Smoothers. */
#define AMG_SMOOTHER_JACOBI 0    /* x <- x + omega D^-1 (b - A x) */
#define AMG_SMOOTHER_L1_JACOBI 1 /* x <- x + D_l1^-1 (b - A x), d_i = sum_j |a_ij| */

/* Precision of the V-cycle. */
#define AMG_PRECISION_FP64 0
#define AMG_PRECISION_MIXED 1 /* FP32 hierarchy values and V-cycle arithmetic inside FP64 Krylov;
                                 FP64 true residual, dot products and coarsest solve */

/* AMG families (amg_config.amg_type). */
#define AMG_TYPE_AGGREGATION 0 /* smoothed aggregation (default) */
#define AMG_TYPE_CLASSICAL 1   /* classical Ruge-Stueben: strength -a_ij >= 1/4 max_k(-a_ik), PMIS
                                  C/F splitting, direct interpolation */

/* Tile layouts of the streaming kernels that run the large operators (the
 * level operators A_l, P_l, R_l with at least 16384 rows).  By default the
 * setup times each operator's candidate layouts and keeps the fastest. */
#define AMG_LAYOUT_AUTO 0       /* timed trial over all layouts (default) */
#define AMG_LAYOUT_CSR 1        /* CSR row tiles; the vector gathered from global memory */
#define AMG_LAYOUT_WINDOWED 2   /* CSR row tiles; windows of the vector staged in shared memory */
#define AMG_LAYOUT_SLICED_ELL 3 /* 32-row slices stored slot-major, one thread per row; windows staged */
#define AMG_LAYOUT_ELL_DIRECT 4 /* the same slot-major slices read with plain coalesced loads (no staging);
                                   the vector gathered from global memory */
#define AMG_LAYOUT_TILES 5      /* the timed trial over the tile layouts (CSR, windowed, sliced-ELL) only */

typedef struct amg_handle_s *amg_handle; /* opaque, owned by the library until amg_free */

typedef struct {
    int solver;       /* AMG_SOLVER_*; default AMG_SOLVER_PCG */
    int smoother;     /* AMG_SMOOTHER_*; default weighted Jacobi */
    double omega;     /* Jacobi weight; default 2/3 */
    double theta;     /* finest-level strength threshold; level l uses theta * 2^-l; default 0.08 */
    int coarse_max;   /* coarsening stops at <= coarse_max rows; default 64 */
    int max_levels;   /* default 20 (at most AMG_MAX_LEVELS) */
    double rtol;      /* stop when ||b - A x||_2 <= rtol ||b||_2; default 1e-8 */
    int max_iter;     /* Krylov iterations (products with A in CG; pairs in BiCGStab); default 500 */
    int max_restarts; /* restarts from x while the true residual is above rtol; default 3 */
    int precision;    /* AMG_PRECISION_*; default FP64 */
    int symmetric;    /* -1 detect (pattern symmetric and values bitwise equal), 0 no, 1 yes; default -1 */
    int layout;       /* AMG_LAYOUT_*: restricts the timed trial to one tile layout (an operator that
                         layout does not fit keeps the CSR layout); default AMG_LAYOUT_AUTO */
    int adjoint_reuse; /* adjoint of a nonsymmetric A: 0 sets up a hierarchy of A^T of its own (as
                          Sec. 2.1 describes; default); 1 reuses A's aggregates, P and R = P^T with
                          every level operator transposed (R A_l^T P = A_{l+1}^T), no second setup */
    int amg_type;     /* AMG_TYPE_*; default AMG_TYPE_AGGREGATION.  theta applies to aggregation;
                         batches take aggregation hierarchies only */
    int fuse_coarse;  /* launches of the coarse levels below 16384 rows that no streaming plan covers:
                         1 (default) the single-cluster tail where those levels fit it (at most 400000
                         entries per level), else one launch per pass; 2 one cooperative whole-GPU
                         launch for the run of them with the dense end of the cycle, a grid barrier
                         between passes (same bits as one launch per pass); 0 one launch per pass */
    int device_loop;  /* 1 (default): the Krylov iterations run as one CUDA graph whose conditional
                         node repeats them on the GPU until the solve is done (one host
                         synchronisation per solve); 0: graphs of four iterations polled by the host
                         (for profilers that cannot see inside graphs with conditional nodes) */
    int outer_product; /* arithmetic of the mixed form's Krylov product q = A p on a streamed finest
                         level: -1 (default) chosen at setup by timing both on the chosen plan; 0 FP64;
                         1 double-FP32 (A's values and p as pairs of binary32 numbers, each product and
                         row sum accurate to a few 2^-48 of sum_j |a_ij p_j|; q, dot products, norms,
                         updates and the true residual stay FP64).  Ignored in the FP64 form */
} amg_config;

typedef struct {
    int status;        /* same code as the call's return value */
    int iters;         /* Krylov iterations of the last solve */
    int restarts;      /* true-residual restarts of the last solve */
    int nlevels;       /* levels in the hierarchy (the last is solved densely) */
    double rel_res_true;  /* ||b - A x||_2 / ||b||_2, recomputed in FP64 at the end */
    double rel_res_rec;   /* recursive residual estimate at the end */
    int rows[AMG_MAX_LEVELS];
    long long nnz[AMG_MAX_LEVELS];
    double operator_complexity; /* sum_l nnz(A_l) / nnz(A_0) */
    double setup_ms;   /* wall time of amg_setup */
    double solve_ms;   /* wall time of the last solve (or adjoint solve) */
} amg_info;

/* Fills *cfg with the defaults listed above.  Returns AMG_OK or AMG_ERR_ARG. */
int amg_config_default(amg_config *cfg);

/* Builds the AMG hierarchy of A on the GPU and returns it in *out.
 * Copies row_ptr/col_idx/values; the caller may free them afterwards.
 * Errors: AMG_ERR_ARG, AMG_ERR_BAD_CSR, AMG_ERR_ZERO_DIAG, AMG_NOT_SPD (the
 * coarsest level of a matrix declared or detected symmetric is not SPD),
 * AMG_ERR_STALL, AMG_ERR_OOM, AMG_ERR_UNSUPPORTED, AMG_ERR_CUDA; on error
 * *out is set to NULL and nothing is leaked. */
int amg_setup(const amg_config *cfg, int n, long long nnz, const int *row_ptr, const int *col_idx,
              const double *values, void *cuda_stream, amg_handle *out);

/* Numeric re-setup for new values on the same sparsity pattern (Sec. 2.1:
 * on a cache hit the setup is repeated against the new coefficients while
 * the structure of the first setup is reused).  values: nnz entries in the
 * order of the col_idx given to amg_setup (host or device).  Every level
 * keeps its aggregates, so P, R and every coarse operator keep their
 * patterns; the smoother weights, the prolongator's omega, P, R = P^T, the
 * Galerkin products, the coarsest factor and all FP32 copies are recomputed
 * from the new values, much faster than a new setup.  A classical hierarchy
 * keeps its C/F splittings and interpolation patterns and recomputes the
 * direct-interpolation weights.  A cached hierarchy of
 * A^T (nonsymmetric adjoint) is re-set up too.  Synchronises the stream.
 * Errors: AMG_ERR_ZERO_DIAG, AMG_NOT_SPD (coarsest level), AMG_ERR_ARG (NULL
 * argument, or new values that change the detected symmetry),
 * AMG_ERR_UNSUPPORTED (batched handles), AMG_ERR_CUDA; after an error the
 * handle's values are partly updated and the handle must be freed. */
int amg_resetup(amg_handle h, const double *values, void *cuda_stream);

/* Solves A x = b from x0 = 0 with the handle's solver; b and x have n entries.
 * info may be NULL.  Returns AMG_OK or a soft/hard status (see above). */
int amg_solve(amg_handle h, const double *b, double *x, void *cuda_stream, amg_info *info);

/* Reverse-mode adjoint of x = A^-1 b (Eq. 1-2).  Given the forward solution x
 * and g = dL/dx (n entries each), solves A^T lambda = g with the handle's
 * configuration and writes lambda = dL/db (n entries) and
 * dA[k] = -lambda[row(k)] * x[col_idx[k]] for every stored entry k (nnz
 * entries, the order of the setup's col_idx).  Either output may be NULL to
 * skip it.  For a nonsymmetric A the first call builds and caches a hierarchy
 * of A^T.  Returns like amg_solve. */
int amg_adjoint(amg_handle h, const double *x, const double *g, double *lambda, double *dA,
                void *cuda_stream, amg_info *info);

/* Applies the AMG preconditioner once: z = M^-1 r (one V(1,1) cycle from
 * z = 0), the operator the Krylov solvers use (Sec. 2.2, preconditioner
 * export).  r and z have n entries.  A handle set up for an unpreconditioned
 * solver (AMG_SOLVER_CG, AMG_SOLVER_BICGSTAB_NOPREC) holds the finest level
 * only and returns AMG_ERR_UNSUPPORTED. */
int amg_vcycle(amg_handle h, const double *r, double *z, void *cuda_stream);

/* Hierarchy statistics (nlevels, rows, nnz, operator_complexity, setup_ms).
 * The iteration fields are those of the handle's last solve. */
int amg_get_info(amg_handle h, amg_info *info);

/* Copies level data out of the hierarchy (inspection and testing).
 * which = 0: A_l (rows n_l); 1: P_l (n_l x n_{l+1}); 2: R_l = P_l^T.
 * dims[0] = rows, dims[1] = cols, dims[2] = nnz are written when dims != NULL;
 * row_ptr/col_idx/values may be NULL to query the sizes only. */
int amg_get_level(amg_handle h, int level, int which, long long *dims, int *row_ptr, int *col_idx,
                  double *values);

/* Copies the aggregate index of every row of level l (l < nlevels - 1). */
int amg_get_aggregates(amg_handle h, int level, int *agg);

/* The streaming plan chosen at setup for one operator of level l: which = 0
 * A_l W (pre-smoothing), 1 P_l (prolongation), 2 R_l (restriction), 3 A_l
 * (post-smoothing), 4 the A of the Krylov products (level 0 only).
 * plan[0] = layout (AMG_LAYOUT_CSR, _WINDOWED, _SLICED_ELL or _ELL_DIRECT; 0 when the
 * operator has no streaming plan and runs on the row-vector kernels),
 * plan[1] = rows per tile, plan[2] = threads per row, plan[3] = tiles,
 * plan[4] = pipeline stages (tiles in flight per CTA; 1 for _ELL_DIRECT,
 * which stages nothing; 0 without a plan), plan[5] = 1 when the operator's
 * product runs in double-FP32 arithmetic (which = 4 in the mixed form, where
 * setup found it faster than FP64: A's values and p as pairs of binary32
 * numbers, each product and row sum accurate to a few 2^-48 of
 * sum_j |a_ij p_j|), else 0.
 * Errors: AMG_ERR_ARG (NULL, level or which out of range). */
int amg_get_plan(amg_handle h, int level, int which, int plan[6]);

/* Per-kernel tracing of the solve phase.  The paper reports wall-clock times
 * only; this is the library's own instrumentation.  amg_profile(h, 1) clears
 * the records and brackets every later solve-phase kernel launch of the
 * handle with CUDA events on the handle's stream; amg_profile(h, 0) stops
 * bracketing and keeps the records.  Kernel launches are counted in both
 * modes (the count restarts at every amg_profile call). */
int amg_profile(amg_handle h, int enable);

/* Kernel launches since the last amg_profile call, and the number of
 * (kernel, level) records.  Either pointer may be NULL. */
int amg_profile_summary(amg_handle h, long long *launches, int *nrecords);

/* Record i (0 <= i < nrecords): kernel name (NUL-terminated, truncated to
 * name_len bytes), hierarchy level, launches, total device time in ms and
 * total algorithmic bytes (compulsory DRAM traffic of the launches: operator
 * values, indices and row pointers once, each vector once).  Output pointers
 * may be NULL. */
int amg_profile_record(amg_handle h, int i, char *name, int name_len, int *level, long long *launches,
                       double *total_ms, double *total_bytes);

/* Right-hand sides per system that one batched solve carries. */
#define AMG_BATCH_MAX_RHS 8

/* Batched systems and right-hand sides (the paper's Sec. 2.2 applies the
 * solver over a batch of right-hand sides with one cached setup; here many
 * independent systems, each with up to AMG_BATCH_MAX_RHS right-hand sides,
 * are solved concurrently).  The caller passes nsys independent square
 * systems as ONE block-diagonal CSR of n rows: system k owns rows and
 * columns sys_off[k] .. sys_off[k+1]-1 (sys_off has nsys + 1 entries, host
 * or device, sys_off[0] = 0, sys_off[nsys] = n, every system non-empty), and
 * a row of system k may store columns of system k only (AMG_ERR_BAD_CSR
 * otherwise).  Each system gets the hierarchy amg_setup would build for it
 * alone -- the same strength graph, aggregates, prolongators and Galerkin
 * operators, bit for bit -- built for all systems at once; a system whose
 * coarsening ends (at most coarse_max rows, or max_levels) is solved densely
 * on that level while the others continue.  cfg->solver must be
 * AMG_SOLVER_PCG (AMG_ERR_UNSUPPORTED otherwise); precision FP64 or MIXED.
 * The handle serves amg_solve_batched, amg_batch_level, amg_get_level,
 * amg_get_aggregates, amg_get_info, the amg_profile* calls and amg_free;
 * amg_solve, amg_adjoint and amg_vcycle return AMG_ERR_ARG on it.
 * Errors as amg_setup. */
int amg_setup_batched(const amg_config *cfg, int nsys, const int *sys_off, int n, long long nnz,
                      const int *row_ptr, const int *col_idx, const double *values, void *cuda_stream,
                      amg_handle *out);

/* Solves A_k X_k = B_k for every system k of a batched handle, each column
 * (right-hand side) on its own: preconditioned CG from x0 = 0 with one
 * V-cycle per iteration, its own step sizes, and its own stop at
 * ||b - A x||_2 <= rtol ||b||_2 (true-residual restarts as amg_solve).
 * B and X: n x nrhs, row-major ([row][rhs]), 1 <= nrhs <= AMG_BATCH_MAX_RHS,
 * host or device.  iters (int) and rel_res (double, true relative
 * residual): nsys x nrhs row-major, host or device, may be NULL.  info may be
 * NULL; its status is the worst status of any pair, iters the largest count,
 * rel_res_true the largest relative residual.  Returns that worst status or
 * a hard error. */
int amg_solve_batched(amg_handle h, int nrhs, const double *B, double *X, int *iters, double *rel_res,
                      void *cuda_stream, amg_info *info);

/* Layout of level `level` of a batched handle: *nsys_level systems live on
 * it; if the arrays are non-NULL (host, sized for the batch's nsys and
 * nsys + 1 entries), sys[j] is the j-th of them (ascending ids), row_off[j]
 * its first row on this level (row_off[*nsys_level] = the level's rows) and
 * final[j] 1 if its coarsening ends here (solved densely on this level). */
int amg_batch_level(amg_handle h, int level, int *nsys_level, int *sys, int *row_off, int *final_flags);

/* The FP64 <-> FP32 conversions of the mixed-precision form, which run on
 * the integer pipes (a hardware cvt between the two formats issues on the
 * FP64 pipe): out[i] = in[i] rounded to nearest even (amg_narrow_f64) or
 * exactly (amg_widen_f32), as IEEE 754 specifies, for i < n.  Device
 * pointers; stream-ordered on cuda_stream.  Errors: AMG_ERR_ARG (NULL
 * pointer with n > 0, n < 0), AMG_ERR_CUDA. */
int amg_narrow_f64(const double *in, float *out, long long n, void *cuda_stream);
int amg_widen_f32(const float *in, double *out, long long n, void *cuda_stream);

/* Largest system amg_cg_solve_noalloc accepts (rows). */
#define AMG_NOALLOC_MAX_N (1 << 18)

/* Unpreconditioned conjugate gradients on a caller's CSR matrix that
 * allocates no device memory.  The paper has no counterpart; this entry
 * point exists for callers that cannot allocate at the moment they solve:
 * code that runs inside a framework owning all device memory (one that only
 * hands an operator the buffers it planned, and forbids cudaMalloc while it
 * executes), or a latency-critical loop in which an allocation would stall
 * every stream.  amg_setup allocates a whole hierarchy, so such callers
 * cannot hold a handle; this call needs none.
 *
 * Computes the same iteration as amg_solve with AMG_SOLVER_CG (x0 = 0; stop at
 * ||b - A x||_2 <= rtol ||b||_2, at most 3 restarts from x while the true
 * residual is above it).  n rows, nnz stored entries; row_ptr/col_idx/values,
 * b and x must be DEVICE memory of the current device (host arrays, or
 * memory of another GPU, return AMG_ERR_ARG before any GPU work: staging
 * them would need an allocation); cuda_stream, when not NULL, must belong to
 * the current device too (else AMG_ERR_ARG).  The CSR must satisfy the
 * conventions above and is not validated.  info may be NULL (its hierarchy
 * fields are left zero).
 *
 * Work space: the vectors r, p, q, the per-block partial sums and the Krylov
 * scalars live in one fixed __device__ array of about 6.3 MB.  n above
 * AMG_NOALLOC_MAX_N returns AMG_ERR_UNSUPPORTED before any GPU work.  The
 * array belongs to the library's module: with CUDA's lazy module loading
 * (the default) its device memory is committed when the module first loads
 * on a device, which happens inside the first call on that device (its
 * cudaGetSymbolAddress), and is then held until the process exits.  That
 * first call is therefore the one that may take device memory (and may fail
 * with AMG_ERR_CUDA when none is left): make one warm-up call on each device
 * before entering a region that must not allocate; later calls take no
 * device memory.  Every call on a device
 * shares that array and it keeps the last call's contents (the call clears
 * what must start at zero), so calls whose GPU work overlaps -- on two
 * streams, or from two host threads -- race and corrupt each other:
 * serialise them.  The call reads the Krylov scalars back to the host
 * between iterations, so it waits for all earlier work on cuda_stream and
 * returns only after its own GPU work has finished: it is synchronous, and a
 * stream that is capturing into a CUDA graph cannot record it.
 * Returns AMG_OK, AMG_MAXIT, AMG_BREAKDOWN, AMG_NAN or a hard error. */
int amg_cg_solve_noalloc(int n, long long nnz, const int *row_ptr, const int *col_idx, const double *values,
                         const double *b, double *x, double rtol, int max_iter, void *cuda_stream,
                         amg_info *info);

/* Average duration (microseconds) of one launch of the finest level's Krylov
 * product -- q = A p with p.q and alpha for PCG, v = A p^ with r^.v for
 * BiCGStab -- over reps back-to-back launches
 * on the handle's stream, chained as in a solve, on the vectors the last
 * solve left (call it after a solve).  Synchronous; leaves the handle ready
 * for the next solve.  Errors: AMG_ERR_ARG (NULL, reps < 1, a finisher that
 * stops on the current vectors), AMG_ERR_UNSUPPORTED (batched handles),
 * AMG_ERR_CUDA. */
int amg_profile_product(amg_handle h, int reps, double *us_per_launch);

/* Test hook for the bounded device waits.  The paper has no counterpart: it
 * exists so that tests can run a wait into its limit without faulting or
 * hanging the GPU.  Arms a one-shot control in h's device state that the next
 * solve-phase launch doing work consumes:
 *   AMG_TEST_WITHHOLD_COPY: CTA 0 of the next bulk-copy streaming pass
 *     (CSR, windowed or sliced-ELL tiles; the direct layout waits on
 *     nothing) expects 16 bytes that no copy delivers, so its first
 *     pipeline stage never completes; its waits give up after 2^12 polls;
 *   AMG_TEST_WITHHOLD_BARRIER: the last CTA of the next cooperative coarse
 *     launch (fuse_coarse = 2) skips its grid-barrier arrivals; the others'
 *     first waits give up after 2^20 SM clocks;
 *   0: disarms.
 * A wait that gives up sets the kernel's error flag and returns; the
 * amg_solve / amg_adjoint call that ran it returns AMG_ERR_CUDA (amg_last_error
 * names the wait) and its results are not valid.  The control disarms itself
 * when consumed; the next call on the handle clears the error flag and the
 * barrier word and runs normally.  Synchronous on the handle's stream.
 * Returns AMG_OK or AMG_ERR_ARG (NULL handle, unknown kind). */
#define AMG_TEST_WITHHOLD_COPY 1
#define AMG_TEST_WITHHOLD_BARRIER 2
int amg_test_arm_wait_timeout(amg_handle h, int kind);

/* Releases every resource of the handle.  amg_free(NULL) is a no-op. */
int amg_free(amg_handle h);

/* Static description of a status code. */
const char *amg_status_string(int code);

/* Description of the last hard error raised on the calling host thread. */
const char *amg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AMG_B300_H */
