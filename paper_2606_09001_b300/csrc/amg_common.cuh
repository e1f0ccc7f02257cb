// amg_common.cuh -- internal types and helpers of libamgb300 (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "amg_b300.h"

namespace amg {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------

void set_last_error(const char *fmt, ...);

#define AMG_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t _e = (expr);                                                        \
        if (_e != cudaSuccess) {                                                        \
            ::amg::set_last_error("%s:%d: %s -> %s", __FILE__, __LINE__, #expr,          \
                                  cudaGetErrorString(_e));                              \
            return _e == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA;        \
        }                                                                               \
    } while (0)

#define AMG_TRY(expr)                 \
    do {                              \
        int _s = (expr);              \
        if (_s < 0) return _s;        \
    } while (0)

#define AMG_LAUNCH_CHECK() AMG_CUDA_TRY(cudaGetLastError())

// ---------------------------------------------------------------------------
// Device memory owned by a handle
// ---------------------------------------------------------------------------

// Records every allocation so a handle frees all of it at once.  Allocations
// are rounded up and padded by 64 bytes so that vector loads that run up to
// 16 bytes past the last element of an array stay inside the allocation.
struct DevArena {
    std::vector<void *> ptrs;
    size_t bytes = 0;
    template <typename T>
    int alloc(T **p, size_t count) {
        size_t b = (count * sizeof(T) + 64 + 255) & ~size_t(255);
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, b);
        if (e != cudaSuccess) {
            set_last_error("cudaMalloc(%zu) failed: %s", b, cudaGetErrorString(e));
            *p = nullptr;
            return e == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA;
        }
        ptrs.push_back(q);
        bytes += b;
        *p = static_cast<T *>(q);
        return AMG_OK;
    }
    void release(void *p) {
        for (auto &q : ptrs)
            if (q == p) {
                cudaFree(q);
                q = nullptr;
            }
    }
    void free_all() {
        for (void *q : ptrs)
            if (q) cudaFree(q);
        ptrs.clear();
        bytes = 0;
    }
};

// Scratch buffers freed at the end of a setup phase.
struct Scratch {
    DevArena arena;
    ~Scratch() { arena.free_all(); }
    template <typename T>
    int alloc(T **p, size_t count) { return arena.alloc(p, count); }
};

// ---------------------------------------------------------------------------
// Sparse matrices
// ---------------------------------------------------------------------------

struct DevCSR {
    int nrows = 0, ncols = 0;
    long long nnz = 0;
    int *rp = nullptr;
    int *ci = nullptr;
    double *v = nullptr;
    float *v32 = nullptr;  // FP32 copy (mixed precision), or null
};

// ---------------------------------------------------------------------------
// Device-side Krylov state
// ---------------------------------------------------------------------------

struct DevScalars {
    double bn2;       // ||b||^2
    double tol2;      // (rtol ||b||)^2
    double rz;        // PCG: r.z of the current iteration
    double rz_new;
    double pq;
    double alpha, beta;
    double rr;        // ||r||^2 (recursive)
    double rho, rho_old, omega, rv, ts, tt, ss;  // BiCGStab
    double tr;        // true residual ||b - A x||^2
    int done;         // 1: stop launching work (converged, failed or max_iter)
    int status;       // AMG_OK / AMG_MAXIT / AMG_BREAKDOWN / AMG_NAN while running
    int iters;
    int flexible;     // PCG uses the Polak-Ribiere beta (mixed-precision V-cycle)
    int max_iter;
    int first;        // PCG: the next beta starts a new recursion (beta = 0)
    int copy_timeout; // a bulk-copy wait gave up (set by the streaming kernels)
    int pad;
};

// ---------------------------------------------------------------------------
// Hierarchy
// ---------------------------------------------------------------------------

// Tiling of one operator for the bulk-copy streaming kernels: rt rows per
// tile (a multiple of 16, at most 1024), each tile holding at most cap - 8
// stored entries, vec threads per row.  rt = 0: the operator is too small or
// too irregular and uses the row-vector kernels.
struct StreamPlan {
    int rt = 0, vec = 0, cap = 0, ntiles = 0;
    int nt = 512;  // threads per CTA (768: the wide variant, 4-byte values only)
    // windowed plans (c16 != null): per tile up to 4 windows of the gathered
    // vector (start, length pairs; ntiles x 8 ints), 16-bit local column
    // indices, and the window capacity per stage in elements
    int xw = 0;
    const int *wtab = nullptr;
    const uint16_t *c16 = nullptr;
};

struct Level {
    DevCSR A, P, R;     // P: n x nc, R = P^T: nc x n (P, R unused on the last level)
    double *ahat = nullptr;  // A W: values a_ij w_j (the pre-smoother's operator), FP64
    float *ahat32 = nullptr; // and FP32
    StreamPlan sa, sp, sr;   // streaming plans of A W (pre-smoothing), P, R at the V-cycle's precision
    StreamPlan sa_post;      // streaming plan of A for post-smoothing (tuned apart on the finest
                             // level of the mixed cycle, where the two passes gather different types)
    StreamPlan sa64;         // plan of A for the outer FP64 products (level 0)
    double *w = nullptr;    // smoother weight per row (omega / a_ii, or 1 / sum |a_ij|)
    float *w32 = nullptr;
    int *agg = nullptr;     // aggregate of each row (levels < last)
    double rho = 0.0;       // Gershgorin estimate used for P
    // V-cycle work vectors: b (right-hand side, levels > 0), t (residual, then
    // prolonged iterate), x (smoothed iterate, levels > 0).
    double *b = nullptr, *t = nullptr, *x = nullptr;
    float *b32 = nullptr, *t32 = nullptr, *x32 = nullptr;
    int vec_a = 8, vec_p = 8, vec_r = 8;  // threads per row chosen per operator
};

// One level of a block-diagonal batch: which systems are present, where their
// rows start, and which of them end here (solved densely on this level).
struct BatchLevel {
    std::vector<int> sys;            // system ids present on this level, ascending
    std::vector<int> off;            // row offsets of those systems (size + 1)
    std::vector<unsigned char> fin;  // 1: the system's last level is this one
    int nfin = 0, max_m = 0;
    int *fin_r0 = nullptr, *fin_m = nullptr;  // device: first row and size of each final system
    long long *fin_off2 = nullptr;            // device: offset of its dense inverse in binv
    double *binv = nullptr;                   // device: the final systems' dense inverses, FP64
};

struct Hierarchy {
    amg_config cfg;
    int n = 0;
    long long nnz = 0;
    int symmetric = 0;
    int nlevels = 0;
    Level L[AMG_MAX_LEVELS];
    // The solve runs levels 0 .. nsolve-1; on level nsolve-1 the rest of the
    // cycle is applied as one dense nc x nc matrix (row-major): the coarsest
    // inverse when nsolve == nlevels, else the exact operator of the cycle
    // from that level down (collapsed at setup); cinv32 is its FP32 copy for
    // the mixed cycle (collapsed operators only).
    int nsolve = 0;
    int nc = 0;
    double *cinv = nullptr;
    float *cinv32 = nullptr;
    double *cinv_last = nullptr;  // the coarsest level's dense inverse (also when collapsed)
    // copies of the dense operator with rows padded to nc_ld entries (a
    // multiple of 4, zero-filled) for 16-byte vector loads
    int nc_ld = 0;
    double *cpad64 = nullptr;
    float *cpad32 = nullptr;
    // Fused coarse levels: levels tail_start..nlevels-1 run in one cluster launch
    // (tail_start = -1: not used); device tables for FP64 and FP32 cycles.
    int nsys = 0;                  // > 0: a block-diagonal batch of nsys independent systems
    std::vector<BatchLevel> bl;    // per level (batches only)
    int tail_start = -1;
    int tail_cluster = 0;
    std::vector<unsigned char> tail_args64, tail_args32;  // host copies of the kernel's parameter tables
    int tail_smem64 = 0, tail_smem32 = 0;  // dynamic shared memory of each table's launch
    // One Krylov iteration captured as a CUDA graph (replayed per iteration);
    // iter_kind: which iteration it holds, iter_kernels: launches it contains.
    cudaGraphExec_t iter_exec = nullptr;
    int iter_kind = -1;
    int iter_kernels = 0;
    DevArena arena;
    double setup_ms = 0.0;
};

// ---------------------------------------------------------------------------
// Small device helpers
// ---------------------------------------------------------------------------

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while its predecessor drains; pdl_wait() blocks
// until the predecessor grid has completed and its writes are visible (a
// no-op for kernels launched without the attribute), pdl_trigger() lets this
// kernel's own successor begin launching.  Every solve-phase kernel calls
// pdl_wait() before it reads anything a predecessor may have written.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int W, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, W);
    return v;
}

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Host utilities implemented in setup.cu.
int exclusive_scan_int(const int *in, int *out, int n, int *total_host, cudaStream_t s);
int transpose_csr(const DevCSR &a, DevCSR &t, DevArena &arena, cudaStream_t s);
int build_hierarchy(Hierarchy *h, const int *rp, const int *ci, const double *v, cudaStream_t s);
int tail_prepare(Hierarchy *h, cudaStream_t s);
// Numeric re-setup: new values on the same pattern, the structure (aggregates,
// every sparsity pattern, plans) kept and every value recomputed in place.
int resetup_hierarchy(Hierarchy *h, const double *values, cudaStream_t s);
int build_hierarchy_batched(Hierarchy *h, const int *rp, const int *ci, const double *v, const int *sys_off_host,
                            int nsys, cudaStream_t s);
void free_hierarchy(Hierarchy *h);
int num_sms();

}  // namespace amg
