// amg_common.cuh -- internal types and helpers of libamgb300 (not installed).
#pragma once

#include <cstddef>

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <type_traits>
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

struct DF;

struct DevCSR {
    int nrows = 0, ncols = 0;
    long long nnz = 0;
    int *rp = nullptr;
    int *ci = nullptr;
    double *v = nullptr;
    float *v32 = nullptr;  // FP32 copy (mixed precision), or null
    DF *vdf = nullptr;     // double-FP32 copy (the finest level of the mixed form), or null
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
    int trips;        // passes of the device-side iteration loop since the solve began
    int copy_timeout; // a bounded wait gave up: 1 a bulk-copy wait, 2 a grid-barrier wait,
                      // 4 a wait for another CTA's slice in the whole-solve cluster launch
    int test_ctl;     // one-shot test control read with copy_timeout (amg_test_arm_wait_timeout); 0 normally
    int tr_fresh;     // 1: the whole-solve cluster launch ended with tr and r = b - A x of the final x
};
// The solve-phase kernels receive &copy_timeout and read the test control one
// int further on.
static_assert(offsetof(DevScalars, test_ctl) == offsetof(DevScalars, copy_timeout) + sizeof(int),
              "test_ctl must follow copy_timeout");

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
    // windowed plans (c16 != null, or ell): per tile up to 16 windows of the
    // gathered vector (start, length pairs; ntiles x 32 ints), 16-bit local
    // column indices, and the window capacity per stage in elements
    int xw = 0;
    int stages = 2;  // pipeline stages of windowed and sliced-ELL plans (2..4)
    const int *wtab = nullptr;
    const uint16_t *c16 = nullptr;
    // sliced-ELL plans (ell = 1; windowed, rt a multiple of 32): the entries
    // of each 32-row slice g stored slot-major from soff[g] (a multiple of 32;
    // ceil(n/32) + 1 offsets), padded to the slice's longest row; ec holds the
    // local indices in that order and eperm the stored entry each of the ne
    // slots holds (-1: padding).  Value arrays are laid out in slot order per
    // plan: ev_dst[k] is the copy of CSR values ev_src[k] (vbytes[k] per value).
    int ell = 0;
    // direct sliced-ELL plans (direct = 1: the slot-major layout read with
    // plain loads, no tiles): column of every slot as a 16-bit offset from its
    // row (dcol16, square operators) or an absolute int (dcol32); rt = 32
    int direct = 0;
    int maxw = 0;  // widest slice in slots (direct plans)
    const int16_t *dcol16 = nullptr;
    const int *dcol32 = nullptr;
    long long ne = 0;
    const int *soff = nullptr;
    const uint16_t *ec = nullptr;
    const int *eperm = nullptr;
    static constexpr int EV_MAX = 4;
    int nev = 0;
    const void *ev_src[EV_MAX] = {};
    void *ev_dst[EV_MAX] = {};
    int ev_bytes[EV_MAX] = {};
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
    // kept for numeric re-setup (built at the first one): the pattern (and a
    // value buffer) of A P, and R's entries as positions in P (R = P^T)
    DevCSR AP;
    int *rperm = nullptr;
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
    // Symmetry re-detection at re-setup (the pattern is fixed): tmap[k] is the
    // position of entry k's mirror a_ji when the pattern is symmetric
    // (tmap_state 1), built at the first re-setup; -1: pattern nonsymmetric.
    int *tmap = nullptr;
    int tmap_state = 0;
    // set for the adjoint's hierarchy that reuses a forward hierarchy's
    // aggregates and prolongators (it shares their arrays)
    const Hierarchy *transposed_of = nullptr;
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
    // iter_count Krylov iterations captured as one CUDA graph (replayed between
    // the host's convergence polls); iter_kind: which iteration it holds,
    // iter_kernels: launches it contains.
    cudaGraphExec_t iter_exec = nullptr;
    int iter_kind = -1;
    int iter_count = 0;
    int iter_kernels = 0;
    // The device-side Krylov loop: a graph whose conditional WHILE node repeats
    // loop_count iterations until the device scalars say the solve is done;
    // loop_kind: which iteration it holds (-1: none built; -2: conditional
    // graphs unavailable, the host-polled graph is used).
    cudaGraph_t loop_graph = nullptr;
    cudaGraphExec_t loop_exec = nullptr;
    int loop_kind = -1;
    int loop_kernels = 0;
    DevArena arena;
    double setup_ms = 0.0;
    // the autotuner's timed rounds (ms) of the tile-layout family and the
    // direct sliced-ELL family (0: not compared); the faster one is in use
    float plan_family_ms[2] = {0.f, 0.f};
    // mixed form only: 1 when the cycle runs in FP64 after all -- a
    // hierarchy the single-cluster tail runs whole has no DRAM traffic to
    // halve, and the autotuner keeps whichever precision's cycle was faster
    int cycle64 = 0;
    float cycle_ms[2] = {0.f, 0.f};  // the trial's rounds with the FP32 and the FP64 cycle
    // Whole PCG solves in one cluster launch (cpcg.cuh), where every level's
    // operators fit the cluster's shared memory: CTAs of the cluster (0: not
    // used), the kernel's parameter table (FP32 cycle in the mixed form, FP64
    // otherwise) and its dynamic shared memory.
    int cpcg_cta = 0;
    std::vector<unsigned char> cpcg_args;
    int cpcg_smem = 0;
    // The same kernel running one V-cycle from the tail's first level when
    // that level is not the finest (vmode): CTAs (0: the tail kernel is used),
    // table (FP32 cycle in the mixed form) and dynamic shared memory.
    int vtail_cta = 0;
    std::vector<unsigned char> vtail_args;
    int vtail_smem = 0;
    int vtail_restricts = 0;  // the V-cycle table computes its first level's right-hand side (R_{t-1} t_{t-1})
    // mixed form: 1 when the outer product q = A p runs in double-FP32
    // arithmetic (A's values and p split into FP32 pairs), chosen at setup by
    // timing; krylov_us: a PCG iteration with the cycle's plan family's FP64
    // product and with the kept variant (us)
    int krylov_df = 0;
    float krylov_us[2] = {0.f, 0.f};
    // the direct family's plan of the Krylov product, kept when the tile
    // family wins the cycle (a candidate for the product alone), else rt = 0
    StreamPlan alt_sa64;
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
// The adjoint's hierarchy of A^T reusing h's aggregates and prolongators, and
// its refresh after a re-setup of h.
int build_transposed_hierarchy(Hierarchy *ht, const Hierarchy *h, cudaStream_t s);
int refresh_transposed_hierarchy(Hierarchy *ht, const Hierarchy *h, cudaStream_t s);
// Lays the sliced-ELL plans' value arrays out again from the CSR values
// (after a numeric re-setup).
int ell_refresh(Hierarchy *h, cudaStream_t s);
int build_hierarchy_batched(Hierarchy *h, const int *rp, const int *ci, const double *v, const int *sys_off_host,
                            int nsys, cudaStream_t s);
void free_hierarchy(Hierarchy *h);
int num_sms();

// ---------------------------------------------------------------------------
// FP32 <-> FP64 conversions on the integer pipes
// ---------------------------------------------------------------------------
//
// A cvt between FP32 and FP64 issues on the FP64 pipe, at the rate of an FP64
// FMA (under two per clock per SM on this GPU), and the FP64 Krylov kernels
// already keep that pipe busy.  These conversions take the IEEE 754 binary32
// and binary64 encodings apart with integer operations instead: widening is
// exact, narrowing rounds to nearest, ties to even; infinities, subnormals
// and signed zeros convert as IEEE 754 specifies, and a NaN stays a (quiet)
// NaN with its leading payload bits.

// binary32 -> binary64 (exact)
__device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    unsigned long long bits;
    if (e - 1u < 254u) {  // normal: rebias the exponent (1023 - 127), widen the fraction
        bits = sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
    } else if (e == 255u) {  // infinity, or NaN made quiet
        bits = sign | 0x7ff0000000000000ull | ((unsigned long long)m << 29) | (m ? (1ull << 51) : 0ull);
    } else if (m == 0u) {  // signed zero
        bits = sign;
    } else {  // subnormal m 2^-149 = 1.f 2^(p - 149), p the leading one's position
        const int p = 31 - __clz((int)m);
        bits = sign | ((unsigned long long)(p + 874) << 52) | (((unsigned long long)m << (52 - p)) & 0xfffffffffffffull);
    }
    return __longlong_as_double((long long)bits);
}

// binary64 -> binary32, round to nearest even
__device__ __forceinline__ float f64_to_f32_rn(double d) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
    const int e = (int)((u >> 52) & 0x7ff);
    const unsigned long long m = u & 0xfffffffffffffull;
    const int ef = e - 896;  // the binary32 biased exponent
    if (ef > 0 && ef < 255) {
        // normal range: keep 23 fraction bits and round on the 29 dropped
        // ones; a carry out of the fraction increments the exponent (up to
        // infinity), as rounding requires
        const unsigned hi = (unsigned)(m >> 29), rem = (unsigned)m & 0x1fffffffu;
        const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (hi & 1u))) ? 1u : 0u;
        return __uint_as_float(sign | (((unsigned)ef << 23) + hi + up));
    }
    if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (m ? 0x00400000u | (unsigned)(m >> 29) : 0u));
    if (ef >= 255) return __uint_as_float(sign | 0x7f800000u);  // beyond the binary32 range
    // binary32 subnormal or zero: the 53-bit significand in units of 2^-149,
    // i.e. shifted right by 30 - ef (binary64 subnormals are far below)
    const int sh = 30 - ef;
    if (e == 0 || sh > 54) return __uint_as_float(sign);
    const unsigned long long M = m | (1ull << 52);
    const unsigned long long q = M >> sh, r = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    const unsigned long long up = (r > half || (r == half && (q & 1ull))) ? 1ull : 0ull;
    return __uint_as_float(sign | (unsigned)(q + up));
}

// ---------------------------------------------------------------------------
// Double-FP32 numbers for the batched FP64 product
// ---------------------------------------------------------------------------
//
// On this GPU an FP64 FMA issues at under two per clock per SM, against 128
// FP32 FMAs.  The batched solve's finest product q = A p does eight FMAs per
// stored entry (one per right-hand side) and is bound by the FP64 pipe; it
// runs in double-length FP32 arithmetic instead (Dekker 1971; Shewchuk 1997):
// A's values and p are split once into an unevaluated sum hi + lo of two
// binary32 numbers, hi = RN32(d), lo = RN32(d - hi), so hi + lo equals d to
// within 2^-48 |d|; a product keeps the exact remainder of hi * hi (one FMA)
// and the two cross terms, and a row sum adds the hi parts with an exact
// two-sum and the remainders in FP32.  Each q_i is accurate to a few 2^-48 of
// sum_j |a_ij p_j| (FP64: 2^-53); dot products, norms and vector updates stay
// FP64.  The single-system product does one FMA per entry; on a 7-point
// operator that still keeps the FP64 pipe busier than DRAM, so the mixed form
// times it both ways at setup and keeps the faster.
struct __align__(8) DF {
    float hi, lo;
    DF() = default;
    __host__ __device__ constexpr DF(int z) : hi((float)z), lo(0.f) {}
    __host__ __device__ constexpr DF(float h, float l) : hi(h), lo(l) {}
};
static_assert(sizeof(DF) == 8, "a DF is two packed binary32 numbers");

// Read-only-path loads for the value types the streaming kernels take: the
// built-in types through __ldg, a DF as one 8-byte load.
template <typename T>
__device__ __forceinline__ T ldgv(const T *p) {
    return __ldg(p);
}
__device__ __forceinline__ DF ldgv(const DF *p) {
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return DF(v.x, v.y);
}

// d as hi + lo (hi = RN32(d), lo = RN32(d - hi); the difference is exact in FP64)
__device__ __forceinline__ DF df_split(double d) {
    const float h = f64_to_f32_rn(d);
    return DF(h, f64_to_f32_rn(d - f32_to_f64(h)));
}

// hi + lo in FP64 (both widenings exact; one rounding in the add)
__device__ __forceinline__ double df_value(DF a) { return f32_to_f64(a.hi) + f32_to_f64(a.lo); }

// a * x as (t, e): t = RN32(a.hi x.hi), e its exact remainder plus the cross
// terms a.hi x.lo + a.lo x.hi (the a.lo x.lo term, below 2^-48 |a x|, is dropped)
__device__ __forceinline__ DF operator*(DF a, DF x) {
    const float t = __fmul_rn(a.hi, x.hi);
    float e = __fmaf_rn(a.hi, x.hi, -t);
    e = __fmaf_rn(a.hi, x.lo, e);
    e = __fmaf_rn(a.lo, x.hi, e);
    return DF(t, e);
}

// s += p: the hi parts by an exact two-sum (Knuth), remainders added in FP32
__device__ __forceinline__ DF &operator+=(DF &s, DF p) {
    const float u = __fadd_rn(s.hi, p.hi);
    const float v = __fsub_rn(u, s.hi);
    const float w = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(u, v)), __fsub_rn(p.hi, v));
    s.lo = __fadd_rn(s.lo, __fadd_rn(w, p.lo));
    s.hi = u;
    return s;
}

// Value conversion between the library's floating types, FP32 <-> FP64 on
// the integer pipes.
template <typename To, typename From>
__device__ __forceinline__ To fcvt(From v) {
    if constexpr (std::is_same<To, float>::value && std::is_same<From, double>::value) return f64_to_f32_rn(v);
    else if constexpr (std::is_same<To, double>::value && std::is_same<From, float>::value) return f32_to_f64(v);
    else return static_cast<To>(v);
}

}  // namespace amg
