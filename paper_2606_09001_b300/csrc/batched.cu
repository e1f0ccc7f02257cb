// batched.cu -- many independent systems with several right-hand sides each.
//
// The systems form one block-diagonal CSR (hierarchy: build_hierarchy_batched)
// and every right-hand side of every system is its own preconditioned CG
// problem (the paper's sequential vmap over right-hand sides, Sec. 2.2, run
// concurrently): vectors are stored row-interleaved [row][K] with K = 8, so
// each stored matrix entry is read once for all K right-hand sides, and every
// (system, right-hand side) pair carries its own Krylov scalars and stops on
// its own (a per-pair convergence mask).  The V-cycle runs in FP32 or FP64
// (the handle's precision); the Krylov vectors, dot products and the
// coarsest solves are FP64.  In the mixed form the finest product q = A p,
// which does eight FMAs per stored entry and would be bound by the FP64 pipe,
// runs in double-FP32 arithmetic (A's values and p split into FP32 pairs; see
// DF), and the flexible beta takes z.(r - r_old) as -alpha z.q with the
// previous iteration's alpha and q, so no copy of r_old is kept.
//
// Finest-level row passes run over "chunks" (at most CH consecutive rows of
// one system) so that dot products reduce per system deterministically: each
// chunk writes its partial sums, and the last chunk of a system to finish
// (per-system ticket) adds them in chunk order and updates that system's
// scalars.  Rows of a system whose last level is level l (smoother weight
// 0) are written only by the dense solve of that level.
#include <algorithm>
#include <cstring>
#include <vector>

#include "solve.cuh"

namespace amg {

constexpr int K = 8;          // right-hand sides per system, interleaved
constexpr int BT = 256;       // threads per block: 32 rows x K
constexpr int CH = 512;       // rows per finest-level chunk

struct BDev {
    int n = 0, nsys = 0, npairs = 0, nchunks = 0;
    // finest-level chunks: system, first row, row count; per system: first chunk, chunks
    int *ch_sys = nullptr, *ch_r0 = nullptr, *ch_rows = nullptr;
    int *sys_ch0 = nullptr, *sys_nch = nullptr;
    unsigned *ticket = nullptr;   // per system
    double *part = nullptr;       // [chunk][K][2]
    // outer vectors [n][K], FP64
    double *B = nullptr, *X = nullptr, *R = nullptr, *Z = nullptr, *P = nullptr, *Q = nullptr;
    // FP32 copy of R for the mixed V-cycle's finest level (null in the FP64 form)
    float *R32 = nullptr;
    // mixed form: P split into FP32 pairs [n][K] and the finest operator's
    // values split likewise (the double-FP32 product); null in the FP64 form
    DF *P2 = nullptr;
    const DF *adf = nullptr;
    // per pair (system * K + rhs)
    double *bn2 = nullptr, *tol2 = nullptr, *rz = nullptr, *alpha = nullptr, *beta = nullptr, *rr = nullptr,
           *tr = nullptr;
    int *act = nullptr, *first = nullptr, *iters = nullptr, *status = nullptr;
    int *nact = nullptr;          // active pairs (device), polled by the host
    // Active pairs per system.  A chunked kernel exits early on its own
    // system's count: that count changes only in the system's last chunk,
    // after every chunk of the system has read it, so all chunks of a system
    // take the same branch (the global count may drop mid-kernel).
    int *sys_nact = nullptr;
};

}  // namespace amg

struct amg_batch_ws {
    amg::BDev d;
    // level vectors [n_l][K] at the V-cycle's precision
    void *lb[AMG_MAX_LEVELS] = {}, *lt[AMG_MAX_LEVELS] = {}, *lx[AMG_MAX_LEVELS] = {};
    cudaGraphExec_t iter_exec = nullptr;
    int iter_kernels = 0;
    int g = 1;                     // right-hand sides per thread of the V-cycle's row passes (timed trial)
    int gp = 1;                    // and of the finest Krylov product
    float g_ms[4] = {0, 0, 0, 0};  // the trials' V-cycle times for G = 1, 2, 4, 8
    float gp_ms[4] = {0, 0, 0, 0}; // and product times
    amg::DevArena arena;
};

namespace amg {

using BatchWorkspace = amg_batch_ws;

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

template <typename TA, typename TX>
__device__ __forceinline__ TA spmm_row(const int *__restrict__ rp, const int *__restrict__ ci,
                                       const TA *__restrict__ v, const TX *__restrict__ x, int i, int r) {
    TA s = 0;
    const int e = rp[i + 1];
    int k = rp[i];
    for (; k + 3 < e; k += 4) {
        const int j0 = ci[k], j1 = ci[k + 1], j2 = ci[k + 2], j3 = ci[k + 3];
        const TA a0 = v[k], a1 = v[k + 1], a2 = v[k + 2], a3 = v[k + 3];
        const TA x0 = fcvt<TA>(x[(size_t)j0 * K + r]), x1 = fcvt<TA>(x[(size_t)j1 * K + r]);
        const TA x2 = fcvt<TA>(x[(size_t)j2 * K + r]), x3 = fcvt<TA>(x[(size_t)j3 * K + r]);
        s += a0 * x0 + a1 * x1 + a2 * x2 + a3 * x3;
    }
    for (; k < e; ++k) s += v[k] * fcvt<TA>(x[(size_t)ci[k] * K + r]);
    return s;
}

// The V-cycle's row passes give each thread G consecutive right-hand sides
// of one row (8 / G threads per row, BT * G / 8 rows per block; G chosen per
// handle by timed trial): the row's indices and values load once for the G
// columns, and the G gathered entries of a column with 16-byte loads.
template <int G, typename T>
__device__ __forceinline__ void ld_g(const T *__restrict__ p, T (&v)[G]) {
    if constexpr (G * sizeof(T) >= 16) {
        using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
        constexpr int PER = 16 / sizeof(T);
#pragma unroll
        for (int q = 0; q < G / PER; ++q) {
            const V w = __ldg(reinterpret_cast<const V *>(p) + q);
            const T *u = reinterpret_cast<const T *>(&w);
#pragma unroll
            for (int c = 0; c < PER; ++c) v[q * PER + c] = u[c];
        }
    } else if constexpr (G == 2 && sizeof(T) == 4) {
        const float2 w = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = w.x;
        v[1] = w.y;
    } else if constexpr (std::is_same<T, DF>::value) {
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const float2 w = __ldg(reinterpret_cast<const float2 *>(p) + g);
            v[g] = DF(w.x, w.y);
        }
    } else {
#pragma unroll
        for (int g = 0; g < G; ++g) v[g] = __ldg(p + g);
    }
}

template <int G, typename T>
__device__ __forceinline__ void st_g(T *p, const T (&v)[G]) {
    if constexpr (G * sizeof(T) >= 16) {
        using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
        constexpr int PER = 16 / sizeof(T);
#pragma unroll
        for (int q = 0; q < G / PER; ++q) {
            V w;
            T *u = reinterpret_cast<T *>(&w);
#pragma unroll
            for (int c = 0; c < PER; ++c) u[c] = v[q * PER + c];
            reinterpret_cast<V *>(p)[q] = w;
        }
    } else {
#pragma unroll
        for (int g = 0; g < G; ++g) p[g] = v[g];
    }
}

// s[g] = sum over the row's entries of a_k x[col(k)][r0 + g], in CSR order,
// four terms at a time as spmm_row groups them
template <int G, typename TA, typename TX>
__device__ __forceinline__ void spmm_row_g(const int *__restrict__ rp, const int *__restrict__ ci,
                                           const TA *__restrict__ v, const TX *__restrict__ x, int i, int r0,
                                           TA (&s)[G]) {
#pragma unroll
    for (int g = 0; g < G; ++g) s[g] = 0;
    const int e = rp[i + 1];
    int k = rp[i];
    for (; k + 3 < e; k += 4) {
        const int j0 = ci[k], j1 = ci[k + 1], j2 = ci[k + 2], j3 = ci[k + 3];
        const TA a0 = v[k], a1 = v[k + 1], a2 = v[k + 2], a3 = v[k + 3];
        TX x0[G], x1[G], x2[G], x3[G];
        ld_g<G>(x + (size_t)j0 * K + r0, x0);
        ld_g<G>(x + (size_t)j1 * K + r0, x1);
        ld_g<G>(x + (size_t)j2 * K + r0, x2);
        ld_g<G>(x + (size_t)j3 * K + r0, x3);
#pragma unroll
        for (int g = 0; g < G; ++g)
            s[g] += a0 * fcvt<TA>(x0[g]) + a1 * fcvt<TA>(x1[g]) + a2 * fcvt<TA>(x2[g]) + a3 * fcvt<TA>(x3[g]);
    }
    for (; k < e; ++k) {
        const TA a = v[k];
        TX xv[G];
        ld_g<G>(x + (size_t)ci[k] * K + r0, xv);
#pragma unroll
        for (int g = 0; g < G; ++g) s[g] += a * fcvt<TA>(xv[g]);
    }
}

// s[g] = sum over the row's entries of a_k x[col(k)][r0 + g] in double-FP32,
// in CSR order (the values' and four columns' loads before their products)
template <int G>
__device__ __forceinline__ void spmm_row_df_g(const int *__restrict__ rp, const int *__restrict__ ci,
                                              const DF *__restrict__ v, const DF *__restrict__ x, int i, int r0,
                                              DF (&s)[G]) {
#pragma unroll
    for (int g = 0; g < G; ++g) s[g] = DF(0);
    const int e = rp[i + 1];
    int k = rp[i];
    const float2 *v2 = reinterpret_cast<const float2 *>(v);
    for (; k + 3 < e; k += 4) {
        const int j[4] = {ci[k], ci[k + 1], ci[k + 2], ci[k + 3]};
        float2 a[4];
        DF xv[4][G];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a[u] = v2[k + u];
            ld_g<G>(x + (size_t)j[u] * K + r0, xv[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int g = 0; g < G; ++g) s[g] += DF(a[u].x, a[u].y) * xv[u][g];
    }
    for (; k < e; ++k) {
        const float2 a = v2[k];
        DF xv[G];
        ld_g<G>(x + (size_t)ci[k] * K + r0, xv);
#pragma unroll
        for (int g = 0; g < G; ++g) s[g] += DF(a.x, a.y) * xv[g];
    }
}

#define ROWS_G(n)                                                                                      \
    for (long long e_ = (long long)blockIdx.x * BT + threadIdx.x; e_ < (long long)(n) * (K / G);      \
         e_ += (long long)gridDim.x * BT) {                                                           \
        const int i = (int)(e_ / (K / G)), r0 = (int)(e_ % (K / G)) * G;                              \
        const size_t e0 = (size_t)i * K + r0;

// t = b - (A W) b
template <int G, typename TB, typename TM>
__global__ void __launch_bounds__(BT) kb_presmooth(int n, const int *rp, const int *ci, const TM *ahat,
                                                   const TB *b, TM *t, const int *nact) {
    if (*nact == 0) return;
    ROWS_G(n)
    TM s[G], o[G];
    TB bv[G];
    ld_g<G>(b + e0, bv);
    spmm_row_g<G, TM, TB>(rp, ci, ahat, b, i, r0, s);
#pragma unroll
    for (int g = 0; g < G; ++g) o[g] = fcvt<TM>(bv[g]) - s[g];
    st_g<G>(t + e0, o);
}
}

// y = M x (restriction)
template <int G, typename TM>
__global__ void __launch_bounds__(BT) kb_spmm(int n, const int *rp, const int *ci, const TM *v, const TM *x, TM *y,
                                              const int *nact) {
    if (*nact == 0) return;
    ROWS_G(n)
    TM s[G];
    spmm_row_g<G, TM, TM>(rp, ci, v, x, i, r0, s);
    st_g<G>(y + e0, s);
}
}

// t = W b + P x_c
template <int G, typename TB, typename TM>
__global__ void __launch_bounds__(BT) kb_prolong(int n, const int *rp, const int *ci, const TM *pv, const TM *w,
                                                 const TB *b, const TM *xc, TM *t, const int *nact) {
    if (*nact == 0) return;
    ROWS_G(n)
    TM s[G], o[G];
    TB bv[G];
    ld_g<G>(b + e0, bv);
    spmm_row_g<G, TM, TM>(rp, ci, pv, xc, i, r0, s);
    const TM wi = w[i];
#pragma unroll
    for (int g = 0; g < G; ++g) o[g] = wi * fcvt<TM>(bv[g]) + s[g];
    st_g<G>(t + e0, o);
}
}

// x = t + W (b - A t) on rows with w > 0 (rows with w = 0 belong to a dense solve)
template <int G, typename TB, typename TM, typename TO>
__global__ void __launch_bounds__(BT) kb_postsmooth(int n, const int *rp, const int *ci, const TM *av, const TM *w,
                                                    const TB *b, const TM *t, TO *x, const int *nact) {
    if (*nact == 0) return;
    ROWS_G(n)
    const TM wi = w[i];
    if (wi != (TM)0) {
        TM s[G], tv[G];
        TB bv[G];
        TO o[G];
        ld_g<G>(b + e0, bv);
        ld_g<G>(t + e0, tv);
        spmm_row_g<G, TM, TM>(rp, ci, av, t, i, r0, s);
#pragma unroll
        for (int g = 0; g < G; ++g) o[g] = fcvt<TO>(tv[g] + wi * (fcvt<TM>(bv[g]) - s[g]));
        st_g<G>(x + e0, o);
    }
}
}

// Dense solves of the systems whose last level this is: block per system.
template <typename TB, typename TO>
__global__ void __launch_bounds__(BT) kb_dense(const int *r0s, const int *ms, const long long *off2,
                                               const double *binv, const TB *b, TO *x, const int *nact) {
    if (*nact == 0) return;
    const int f = blockIdx.x, r0 = r0s[f], m = ms[f];
    const double *inv = binv + off2[f];
    for (int e = threadIdx.x; e < m * K; e += BT) {
        const int i = e / K, r = e % K;
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += inv[(size_t)i * m + j] * fcvt<double>(b[(size_t)(r0 + j) * K + r]);
        x[(size_t)(r0 + i) * K + r] = fcvt<TO>(s);
    }
}

// Adds n values v(0), ..., v(n-1) with one warp in a fixed order (lane-strided
// partial sums, then a shuffle tree); every lane returns the total.  FP64
// adds are slow on this GPU, so the block's warps share a reduction's pairs
// rather than a few threads adding long serial chains.
template <class F>
__device__ __forceinline__ double warp_sum_n(int n, F v) {
    double a = 0.0;
    for (int t = threadIdx.x & 31; t < n; t += 32) a += v(t);
    return warp_sum(a);
}

// The system's totals from its chunks' partials, in its last chunk: one warp
// per (value, right-hand side) pair; tot[q] valid in threads tid < K for
// right-hand side tid.
template <int NV>
__device__ __forceinline__ void system_totals(int sys, const BDev &W, double (&tot)[NV]) {
    __shared__ double s_tot[NV][K];
    const int c0 = W.sys_ch0[sys], nc = W.sys_nch[sys];
    for (int pr = threadIdx.x >> 5; pr < NV * K; pr += BT / 32) {
        const int q = pr / K, r = pr % K;
        const double a = warp_sum_n(nc, [&](int c) { return __ldcg(&W.part[((size_t)(c0 + c) * K + r) * 2 + q]); });
        if ((threadIdx.x & 31) == 0) s_tot[q][r] = a;
    }
    __syncthreads();
    if (threadIdx.x < K)
        for (int q = 0; q < NV; ++q) tot[q] = s_tot[q][threadIdx.x];
}

// Block reduction of acc[NV] per right-hand side (thread r = tid % K), the
// chunk's partials, and in the last chunk of the system the per-system totals
// (returned in tot[q], valid in threads tid < K for right-hand side tid).
template <int NV>
__device__ bool chunk_reduce(double (&acc)[NV], int chunk, int sys, const BDev &W, double (&tot)[NV]) {
    __shared__ double sh[NV][BT];
    __shared__ bool s_last;
    for (int q = 0; q < NV; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    // one warp per (value, right-hand side) pair: entries r, r + K, ...
    for (int pr = threadIdx.x >> 5; pr < NV * K; pr += BT / 32) {
        const int q = pr / K, r = pr % K;
        const double a = warp_sum_n(BT / K, [&](int u) { return sh[q][r + K * u]; });
        if ((threadIdx.x & 31) == 0) W.part[((size_t)chunk * K + r) * 2 + q] = a;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&W.ticket[sys], 1u) == (unsigned)W.sys_nch[sys] - 1;
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    system_totals<NV>(sys, W, tot);
    if (threadIdx.x == 0) W.ticket[sys] = 0u;
    return true;
}

__device__ __forceinline__ void deactivate(const BDev &W, int p, int status) {
    W.status[p] = status;
    W.act[p] = 0;
    atomicSub(&W.sys_nact[p / K], 1);
    atomicSub(W.nact, 1);
}

// chunk_reduce for threads that hold G right-hand sides each (acc[q][g] for
// right-hand side r0 + g): per right-hand side, the block's values are added
// over the row slots by one warp.
template <int NV, int G>
__device__ bool chunk_reduce_g(double (&acc)[NV][G], int chunk, int sys, const BDev &W, double (&tot)[NV]) {
    constexpr int SLOTS = BT / (K / G);
    __shared__ double sh[NV][K][SLOTS];
    __shared__ bool s_last;
    const int slot = threadIdx.x / (K / G), r0 = (threadIdx.x % (K / G)) * G;
#pragma unroll
    for (int q = 0; q < NV; ++q)
#pragma unroll
        for (int g = 0; g < G; ++g) sh[q][r0 + g][slot] = acc[q][g];
    __syncthreads();
    // one warp per (value, right-hand side) pair, over its slots
    for (int pr = threadIdx.x >> 5; pr < NV * K; pr += BT / 32) {
        const int q = pr / K, r = pr % K;
        const double a = warp_sum_n(SLOTS, [&](int t) { return sh[q][r][t]; });
        if ((threadIdx.x & 31) == 0) W.part[((size_t)chunk * K + r) * 2 + q] = a;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&W.ticket[sys], 1u) == (unsigned)W.sys_nch[sys] - 1;
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    system_totals<NV>(sys, W, tot);
    if (threadIdx.x == 0) W.ticket[sys] = 0u;
    return true;
}

// Finest level, chunked: z = t + W (b - A t) (rows with w = 0 keep the dense
// solve's z), r.z and, flexible, z.q per pair -> beta.  G right-hand sides
// per thread.
template <int G, typename TM>
__global__ void __launch_bounds__(BT) kb_post0(BDev W, const int *rp, const int *ci, const TM *av,
                                               const TM *w, const TM *t, int flexible) {
    const int chunk = blockIdx.x, sys = W.ch_sys[chunk], r0c = W.ch_r0[chunk], rows = W.ch_rows[chunk];
    if (W.sys_nact[sys] == 0) return;
    const int r0 = (threadIdx.x % (K / G)) * G;
    double acc[2][G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[0][g] = acc[1][g] = 0.0;
    for (int il = threadIdx.x / (K / G); il < rows; il += BT / (K / G)) {
        const int i = r0c + il;
        const size_t e0 = (size_t)i * K + r0;
        const TM wi = w[i];
        double rv[G], o[G], qv[G];
        ld_g<G>(W.R + e0, rv);
        if (wi != (TM)0) {
            TM s[G], tv[G];
            ld_g<G>(t + e0, tv);
            spmm_row_g<G, TM, TM>(rp, ci, av, t, i, r0, s);
#pragma unroll
            for (int g = 0; g < G; ++g) o[g] = fcvt<double>(tv[g] + wi * (fcvt<TM>(rv[g]) - s[g]));
            st_g<G>(W.Z + e0, o);
        } else {
            ld_g<G>(W.Z + e0, o);
        }
        if (flexible) ld_g<G>(W.Q + e0, qv);  // q = A p of the previous iteration: r - r_old = -alpha q
#pragma unroll
        for (int g = 0; g < G; ++g) {
            acc[0][g] += rv[g] * o[g];
            if (flexible) acc[1][g] += qv[g] * o[g];
        }
    }
    double tot[2];
    if (chunk_reduce_g<2, G>(acc, chunk, sys, W, tot) && threadIdx.x < K) {
        const int p = sys * K + threadIdx.x;
        if (W.act[p]) {
            if (!isfinite(tot[0])) {
                deactivate(W, p, AMG_NAN);
            } else {
                W.beta[p] = W.first[p] ? 0.0 : (flexible ? -W.alpha[p] * tot[1] : tot[0]) / W.rz[p];
                W.first[p] = 0;
                W.rz[p] = tot[0];
            }
        }
    }
}

// p = z + beta p (active pairs), and its FP32 pairs in the mixed form
__global__ void __launch_bounds__(BT) kb_p(BDev W) {
    const int chunk = blockIdx.x, sys = W.ch_sys[chunk], r0 = W.ch_r0[chunk], rows = W.ch_rows[chunk];
    const int r = threadIdx.x % K, p = sys * K + r;
    if (!W.act[p]) return;
    const double beta = W.beta[p];
    for (int il = threadIdx.x / K; il < rows; il += BT / K) {
        const size_t e = (size_t)(r0 + il) * K + r;
        const double pe = beta == 0.0 ? W.Z[e] : W.Z[e] + beta * W.P[e];
        W.P[e] = pe;
        if (W.P2) W.P2[e] = df_split(pe);
    }
}

// one row's q = sum_k a_k p_{col(k)} for right-hand side r in double-FP32
// (four terms' loads before their products; the sum in CSR order)
__device__ __forceinline__ DF spmm_row_df(const int *__restrict__ rp, const int *__restrict__ ci,
                                          const DF *__restrict__ v, const DF *__restrict__ x, int i, int r) {
    DF s(0);
    const int e = rp[i + 1];
    int k = rp[i];
    const float2 *v2 = reinterpret_cast<const float2 *>(v), *x2 = reinterpret_cast<const float2 *>(x);
    for (; k + 3 < e; k += 4) {
        const int j0 = ci[k], j1 = ci[k + 1], j2 = ci[k + 2], j3 = ci[k + 3];
        const float2 a0 = v2[k], a1 = v2[k + 1], a2 = v2[k + 2], a3 = v2[k + 3];
        const float2 x0 = x2[(size_t)j0 * K + r], x1 = x2[(size_t)j1 * K + r];
        const float2 x2_ = x2[(size_t)j2 * K + r], x3 = x2[(size_t)j3 * K + r];
        s += DF(a0.x, a0.y) * DF(x0.x, x0.y);
        s += DF(a1.x, a1.y) * DF(x1.x, x1.y);
        s += DF(a2.x, a2.y) * DF(x2_.x, x2_.y);
        s += DF(a3.x, a3.y) * DF(x3.x, x3.y);
    }
    for (; k < e; ++k) {
        const float2 a = v2[k], xv = x2[(size_t)ci[k] * K + r];
        s += DF(a.x, a.y) * DF(xv.x, xv.y);
    }
    return s;
}

// q = A p, p.q per pair -> alpha; or (TRUE_RES) r = b - A x, ||r||^2 per pair.
// G right-hand sides per thread; in the mixed form the product runs in
// double-FP32 on p's FP32 pairs (the true residual stays FP64).
template <bool TRUE_RES, int G>
__global__ void __launch_bounds__(BT) kb_spmv0(BDev W, const int *rp, const int *ci, const double *av) {
    const int chunk = blockIdx.x, sys = W.ch_sys[chunk], r0c = W.ch_r0[chunk], rows = W.ch_rows[chunk];
    if (!TRUE_RES && W.sys_nact[sys] == 0) return;
    const int r0 = (threadIdx.x % (K / G)) * G;
    double acc[1][G];
    DF accdf[G];  // the mixed form's p.q partials, double-FP32 (one FP64 conversion a thread)
#pragma unroll
    for (int g = 0; g < G; ++g) {
        acc[0][g] = 0.0;
        accdf[g] = DF(0);
    }
    for (int il = threadIdx.x / (K / G); il < rows; il += BT / (K / G)) {
        const int i = r0c + il;
        const size_t e0 = (size_t)i * K + r0;
        if (TRUE_RES) {
            double sv[G], bv[G], rv[G];
            ld_g<G>(W.B + e0, bv);
            spmm_row_g<G, double, double>(rp, ci, av, W.X, i, r0, sv);
#pragma unroll
            for (int g = 0; g < G; ++g) {
                rv[g] = bv[g] - sv[g];
                acc[0][g] += rv[g] * rv[g];
            }
            st_g<G>(W.R + e0, rv);
            if (W.R32) {
                float rf[G];
#pragma unroll
                for (int g = 0; g < G; ++g) rf[g] = f64_to_f32_rn(rv[g]);
                st_g<G>(W.R32 + e0, rf);
            }
        } else if (W.adf) {  // mixed form: double-FP32 product on p's FP32 pairs
            DF sd[G], pv[G];
            ld_g<G>(W.P2 + e0, pv);
            spmm_row_df_g<G>(rp, ci, W.adf, W.P2, i, r0, sd);
            double q[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                q[g] = df_value(sd[g]);
                accdf[g] += pv[g] * sd[g];
            }
            st_g<G>(W.Q + e0, q);
        } else {
            double sv[G], pv[G];
            ld_g<G>(W.P + e0, pv);
            spmm_row_g<G, double, double>(rp, ci, av, W.P, i, r0, sv);
#pragma unroll
            for (int g = 0; g < G; ++g) acc[0][g] += pv[g] * sv[g];
            st_g<G>(W.Q + e0, sv);
        }
    }
    if (!TRUE_RES && W.adf)
#pragma unroll
        for (int g = 0; g < G; ++g) acc[0][g] = df_value(accdf[g]);
    double tot[1];
    if (chunk_reduce_g<1, G>(acc, chunk, sys, W, tot) && threadIdx.x < K) {
        const int p = sys * K + threadIdx.x;
        if (TRUE_RES) {
            W.tr[p] = tot[0];
        } else if (W.act[p]) {
            if (!isfinite(tot[0])) deactivate(W, p, AMG_NAN);
            else if (tot[0] <= 0.0) deactivate(W, p, AMG_BREAKDOWN);
            else W.alpha[p] = W.rz[p] / tot[0];
        }
    }
}

// The finest product at the handle's G.
template <bool TRUE_RES>
static void launch_spmv0(const BDev &d, int g, const int *rp, const int *ci, const double *av, cudaStream_t s) {
    switch (g) {
        case 8: kb_spmv0<TRUE_RES, 8><<<d.nchunks, BT, 0, s>>>(d, rp, ci, av); break;
        case 4: kb_spmv0<TRUE_RES, 4><<<d.nchunks, BT, 0, s>>>(d, rp, ci, av); break;
        case 2: kb_spmv0<TRUE_RES, 2><<<d.nchunks, BT, 0, s>>>(d, rp, ci, av); break;
        default: kb_spmv0<TRUE_RES, 1><<<d.nchunks, BT, 0, s>>>(d, rp, ci, av); break;
    }
}

// x += alpha p, r -= alpha q (active pairs), ||r||^2 -> convergence
__global__ void __launch_bounds__(BT) kb_update(BDev W, int max_iter) {
    const int chunk = blockIdx.x, sys = W.ch_sys[chunk], r0 = W.ch_r0[chunk], rows = W.ch_rows[chunk];
    if (W.sys_nact[sys] == 0) return;
    const int r = threadIdx.x % K, p = sys * K + r;
    const bool a = W.act[p] != 0;
    const double alpha = a ? W.alpha[p] : 0.0;
    double acc[1] = {0.0};
    for (int il = threadIdx.x / K; il < rows; il += BT / K) {
        const size_t e = (size_t)(r0 + il) * K + r;
        if (a) {
            W.X[e] += alpha * W.P[e];
            const double rn = W.R[e] - alpha * W.Q[e];
            W.R[e] = rn;
            if (W.R32) W.R32[e] = f64_to_f32_rn(rn);
            acc[0] += rn * rn;
        }
    }
    double tot[1];
    if (chunk_reduce<1>(acc, chunk, sys, W, tot) && threadIdx.x < K) {
        const int q = sys * K + threadIdx.x;
        if (W.act[q]) {
            W.iters[q] += 1;
            W.rr[q] = tot[0];
            if (!isfinite(tot[0])) deactivate(W, q, AMG_NAN);
            else if (tot[0] <= W.tol2[q]) deactivate(W, q, AMG_OK);
            else if (W.iters[q] >= max_iter) deactivate(W, q, AMG_MAXIT);
        }
    }
}

// x = 0, r = b, p = q = 0; ||b||^2 per pair; pairs with b = 0 are done at once.
__global__ void __launch_bounds__(BT) kb_init(BDev W, double rtol) {
    const int chunk = blockIdx.x, sys = W.ch_sys[chunk], r0 = W.ch_r0[chunk], rows = W.ch_rows[chunk];
    const int r = threadIdx.x % K;
    double acc[1] = {0.0};
    for (int il = threadIdx.x / K; il < rows; il += BT / K) {
        const size_t e = (size_t)(r0 + il) * K + r;
        const double bi = W.B[e];
        W.X[e] = 0.0;
        W.R[e] = bi;
        if (W.R32) W.R32[e] = f64_to_f32_rn(bi);
        W.P[e] = 0.0;
        W.Q[e] = 0.0;  // the flexible beta's first z.q (unused: beta = 0) reads finite values
        W.Z[e] = 0.0;
        acc[0] += bi * bi;
    }
    double tot[1];
    if (chunk_reduce<1>(acc, chunk, sys, W, tot) && threadIdx.x < K) {
        const int p = sys * K + threadIdx.x;
        W.bn2[p] = tot[0];
        W.tol2[p] = rtol * rtol * tot[0];
        W.rr[p] = tot[0];
        W.iters[p] = 0;
        W.first[p] = 1;
        W.rz[p] = 0.0;
        W.status[p] = AMG_OK;
        const bool live = tot[0] > 0.0 && isfinite(tot[0]);
        W.act[p] = live;
        if (!isfinite(tot[0])) W.status[p] = AMG_NAN;
        if (live) {
            atomicAdd(&W.sys_nact[sys], 1);
            atomicAdd(W.nact, 1);
        }
    }
}

// Restart the pairs whose true residual is still above the tolerance (r holds it).
__global__ void kb_restart(BDev W, int max_iter) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < W.npairs; p += gridDim.x * blockDim.x) {
        if (W.status[p] == AMG_OK && W.bn2[p] > 0.0 && W.tr[p] > W.tol2[p] && W.iters[p] < max_iter) {
            W.act[p] = 1;
            W.first[p] = 1;
            atomicAdd(&W.sys_nact[p / K], 1);
            atomicAdd(W.nact, 1);
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

__global__ void k_split_df(long long n, const double *__restrict__ in, DF *out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = df_split(in[i]);
}

static int workspace_build(Hierarchy *h, BatchWorkspace &W) {
    DevArena &a = W.arena;
    BDev &d = W.d;
    const int n = h->n, ns = h->nsys;
    d.n = n;
    d.nsys = ns;
    d.npairs = ns * K;
    const BatchLevel &B0 = h->bl[0];
    std::vector<int> ch_sys, ch_r0, ch_rows, sys_ch0(ns), sys_nch(ns);
    for (int s = 0; s < ns; ++s) {
        sys_ch0[s] = (int)ch_sys.size();
        for (int r0 = B0.off[s]; r0 < B0.off[s + 1]; r0 += CH) {
            ch_sys.push_back(s);
            ch_r0.push_back(r0);
            ch_rows.push_back(std::min(CH, B0.off[s + 1] - r0));
        }
        sys_nch[s] = (int)ch_sys.size() - sys_ch0[s];
    }
    d.nchunks = (int)ch_sys.size();
    AMG_TRY(a.alloc(&d.ch_sys, d.nchunks));
    AMG_TRY(a.alloc(&d.ch_r0, d.nchunks));
    AMG_TRY(a.alloc(&d.ch_rows, d.nchunks));
    AMG_TRY(a.alloc(&d.sys_ch0, ns));
    AMG_TRY(a.alloc(&d.sys_nch, ns));
    AMG_TRY(a.alloc(&d.ticket, ns));
    AMG_TRY(a.alloc(&d.part, (size_t)d.nchunks * K * 2));
    AMG_CUDA_TRY(cudaMemcpy(d.ch_sys, ch_sys.data(), sizeof(int) * d.nchunks, cudaMemcpyHostToDevice));
    AMG_CUDA_TRY(cudaMemcpy(d.ch_r0, ch_r0.data(), sizeof(int) * d.nchunks, cudaMemcpyHostToDevice));
    AMG_CUDA_TRY(cudaMemcpy(d.ch_rows, ch_rows.data(), sizeof(int) * d.nchunks, cudaMemcpyHostToDevice));
    AMG_CUDA_TRY(cudaMemcpy(d.sys_ch0, sys_ch0.data(), sizeof(int) * ns, cudaMemcpyHostToDevice));
    AMG_CUDA_TRY(cudaMemcpy(d.sys_nch, sys_nch.data(), sizeof(int) * ns, cudaMemcpyHostToDevice));
    AMG_CUDA_TRY(cudaMemset(d.ticket, 0, sizeof(unsigned) * ns));
    const size_t nk = (size_t)n * K;
    double **vecs[] = {&d.B, &d.X, &d.R, &d.Z, &d.P, &d.Q};
    for (double **v : vecs) AMG_TRY(a.alloc(v, nk));
    if (h->cfg.precision == AMG_PRECISION_MIXED) {
        AMG_TRY(a.alloc(&d.R32, nk));
        AMG_TRY(a.alloc(&d.P2, nk));
        const DevCSR &A0 = h->L[0].A;
        DF *adf = nullptr;
        AMG_TRY(a.alloc(&adf, (size_t)std::max(1LL, A0.nnz)));
        k_split_df<<<std::max(1, std::min((int)((A0.nnz + 255) / 256), 16 * num_sms())), 256>>>(A0.nnz, A0.v, adf);
        AMG_LAUNCH_CHECK();
        d.adf = adf;
    }
    double **pv[] = {&d.bn2, &d.tol2, &d.rz, &d.alpha, &d.beta, &d.rr, &d.tr};
    for (double **v : pv) AMG_TRY(a.alloc(v, (size_t)d.npairs));
    int **pi[] = {&d.act, &d.first, &d.iters, &d.status};
    for (int **v : pi) AMG_TRY(a.alloc(v, (size_t)d.npairs));
    AMG_TRY(a.alloc(&d.nact, 1));
    AMG_CUDA_TRY(cudaMemset(d.nact, 0, sizeof(int)));
    AMG_TRY(a.alloc(&d.sys_nact, ns));
    const size_t vb = h->cfg.precision == AMG_PRECISION_MIXED ? 4 : 8;
    for (int l = 0; l < h->nlevels; ++l) {
        const size_t nl = (size_t)h->L[l].A.nrows * K;
        unsigned char *p;
        AMG_TRY(a.alloc(&p, nl * vb));
        W.lt[l] = p;
        if (l > 0) {
            AMG_TRY(a.alloc(&p, nl * vb));
            W.lb[l] = p;
            AMG_TRY(a.alloc(&p, nl * vb));
            W.lx[l] = p;
        }
    }
    AMG_CUDA_TRY(cudaDeviceSynchronize());
    return AMG_OK;
}

static int tune_g(Hierarchy *h, BatchWorkspace &W);

int batch_create(Hierarchy *h, BatchWorkspace **out) {
    *out = nullptr;
    BatchWorkspace *W = new (std::nothrow) BatchWorkspace();
    if (!W) return AMG_ERR_OOM;
    int rc = workspace_build(h, *W);
    if (rc == AMG_OK) rc = tune_g(h, *W);
    if (rc < 0) {
        batch_destroy(W);
        return rc;
    }
    *out = W;
    return AMG_OK;
}

void batch_destroy(BatchWorkspace *W) {
    if (!W) return;
    if (W->iter_exec) cudaGraphExecDestroy(W->iter_exec);
    W->arena.free_all();
    delete W;
}

// blocks for n rows at G right-hand sides per thread
static int rows_grid(long long n, int G) {
    const long long g = (n * (K / G) + BT - 1) / BT;
    return (int)std::max(1LL, std::min(g, (long long)num_sms() * 16));
}

template <int G, typename TM>
static int batch_vcycle(Hierarchy *h, BatchWorkspace &W, Profiler &prof, cudaStream_t s) {
    const int L = h->nlevels;
    constexpr bool mixed = sizeof(TM) == 4;
    const BDev &d = W.d;
    const int *na = d.nact;
    auto Av = [&](const DevCSR &m) -> const TM * { return (const TM *)(mixed ? (const void *)m.v32 : (const void *)m.v); };
    auto Ah = [&](const Level &lv) -> const TM * { return (const TM *)(mixed ? (const void *)lv.ahat32 : (const void *)lv.ahat); };
    auto Wv = [&](const Level &lv) -> const TM * { return (const TM *)(mixed ? (const void *)lv.w32 : (const void *)lv.w); };
    auto T = [&](int l) { return (TM *)W.lt[l]; };
    auto Bv = [&](int l) { return (TM *)W.lb[l]; };
    auto Xv = [&](int l) { return (TM *)W.lx[l]; };
    auto dense = [&](int l) -> int {
        const BatchLevel &bl = h->bl[l];
        if (bl.nfin == 0) return AMG_OK;
        ProfScope ps(&prof, s, "b_dense", l, 0.0);
        if (l == 0)
            kb_dense<double, double><<<bl.nfin, BT, 0, s>>>(bl.fin_r0, bl.fin_m, bl.fin_off2, bl.binv, d.R, d.Z, na);
        else
            kb_dense<TM, TM><<<bl.nfin, BT, 0, s>>>(bl.fin_r0, bl.fin_m, bl.fin_off2, bl.binv, Bv(l), Xv(l), na);
        AMG_LAUNCH_CHECK();
        return AMG_OK;
    };
    const double vb = (double)sizeof(TM);
    // down: the systems ending on level l are solved there first
    AMG_TRY(dense(0));
    for (int l = 0; l < L - 1; ++l) {
        const Level &lv = h->L[l];
        const int n = lv.A.nrows, nc = lv.R.nrows;
        {
            // the input is vb bytes wide on every level (the finest: FP64 R, or its FP32 copy in the mixed form)
            ProfScope ps(&prof, s, "b_presmooth", l, lv.A.nnz * (4.0 + vb) + (double)n * K * 2.0 * vb);
            if (l == 0 && mixed)  // the FP32 copy of R: no conversion per gathered entry
                kb_presmooth<G, float, TM><<<rows_grid(n, G), BT, 0, s>>>(n, lv.A.rp, lv.A.ci, Ah(lv), d.R32, T(0), na);
            else if (l == 0)
                kb_presmooth<G, double, TM><<<rows_grid(n, G), BT, 0, s>>>(n, lv.A.rp, lv.A.ci, Ah(lv), d.R, T(0), na);
            else
                kb_presmooth<G, TM, TM><<<rows_grid(n, G), BT, 0, s>>>(n, lv.A.rp, lv.A.ci, Ah(lv), Bv(l), T(l), na);
        }
        {
            ProfScope ps(&prof, s, "b_restrict", l, lv.R.nnz * (4.0 + vb) + (double)(n + nc) * K * vb);
            kb_spmm<G, TM><<<rows_grid(nc, G), BT, 0, s>>>(nc, lv.R.rp, lv.R.ci, Av(lv.R), T(l), Bv(l + 1), na);
        }
        AMG_LAUNCH_CHECK();
        AMG_TRY(dense(l + 1));
    }
    // up
    for (int l = L - 2; l >= 0; --l) {
        const Level &lv = h->L[l];
        const int n = lv.A.nrows, nc = lv.P.ncols;
        {
            ProfScope ps(&prof, s, "b_prolong", l, lv.P.nnz * (4.0 + vb) + (double)n * vb + (double)(2 * n + nc) * K * vb);
            if (l == 0 && mixed)
                kb_prolong<G, float, TM><<<rows_grid(n, G), BT, 0, s>>>(n, lv.P.rp, lv.P.ci, Av(lv.P), Wv(lv), d.R32, Xv(1),
                                                                  T(0), na);
            else if (l == 0)
                kb_prolong<G, double, TM><<<rows_grid(n, G), BT, 0, s>>>(n, lv.P.rp, lv.P.ci, Av(lv.P), Wv(lv), d.R, Xv(1),
                                                                   T(0), na);
            else
                kb_prolong<G, TM, TM><<<rows_grid(n, G), BT, 0, s>>>(n, lv.P.rp, lv.P.ci, Av(lv.P), Wv(lv), Bv(l),
                                                               Xv(l + 1), T(l), na);
        }
        AMG_LAUNCH_CHECK();
        if (l > 0) {
            ProfScope ps(&prof, s, "b_postsmooth", l, lv.A.nnz * (4.0 + vb) + (double)n * vb + (double)n * K * 3.0 * vb);
            kb_postsmooth<G, TM, TM, TM><<<rows_grid(n, G), BT, 0, s>>>(n, lv.A.rp, lv.A.ci, Av(lv.A), Wv(lv), Bv(l), T(l),
                                                                  Xv(l), na);
            AMG_LAUNCH_CHECK();
        }
    }
    // finest post-smoothing with r.z (systems ending on level 0 keep the dense z)
    {
        const Level &l0 = h->L[0];
        const double nk = (double)l0.A.nrows * K;
        ProfScope ps(&prof, s, "b_postsmooth_rz", 0,
                     L > 1 ? l0.A.nnz * (4.0 + vb) + l0.A.nrows * vb + nk * (vb + 8.0 * (mixed ? 4.0 : 3.0)) : nk * 16.0);
        kb_post0<G, TM><<<d.nchunks, BT, 0, s>>>(d, l0.A.rp, l0.A.ci, Av(l0.A), Wv(l0), T(0), mixed ? 1 : 0);
        AMG_LAUNCH_CHECK();
    }
    return AMG_OK;
}

// One batched V-cycle at the handle's G.
static int vcycle_g(Hierarchy *h, BatchWorkspace &W, Profiler &prof, cudaStream_t s) {
    const bool mixed = h->cfg.precision == AMG_PRECISION_MIXED;
    switch (W.g) {
        case 8: return mixed ? batch_vcycle<8, float>(h, W, prof, s) : batch_vcycle<8, double>(h, W, prof, s);
        case 4: return mixed ? batch_vcycle<4, float>(h, W, prof, s) : batch_vcycle<4, double>(h, W, prof, s);
        case 2: return mixed ? batch_vcycle<2, float>(h, W, prof, s) : batch_vcycle<2, double>(h, W, prof, s);
        default: return mixed ? batch_vcycle<1, float>(h, W, prof, s) : batch_vcycle<1, double>(h, W, prof, s);
    }
}

// The autotuner of the batched V-cycle: right-hand sides per thread G in
// {1, 2, 4, 8} (threads per row 8 / G, rows per block BT G / 8), each timed
// as the best of three trials of two whole V-cycles (after one) with every
// system active; the fastest is kept.
static int tune_g(Hierarchy *h, BatchWorkspace &W) {
    BDev &d = W.d;
    cudaStream_t s = nullptr;
    AMG_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    // every system active (the kernels skip inactive ones), the vectors zero
    AMG_CUDA_TRY(cudaMemsetAsync(d.nact, 0x01, sizeof(int), s));
    AMG_CUDA_TRY(cudaMemsetAsync(d.sys_nact, 0x01, sizeof(int) * d.nsys, s));
    AMG_CUDA_TRY(cudaMemsetAsync(d.R, 0, sizeof(double) * (size_t)d.n * K, s));
    if (d.R32) AMG_CUDA_TRY(cudaMemsetAsync(d.R32, 0, sizeof(float) * (size_t)d.n * K, s));
    AMG_CUDA_TRY(cudaMemsetAsync(d.Q, 0, sizeof(double) * (size_t)d.n * K, s));
    AMG_CUDA_TRY(cudaMemsetAsync(d.P, 0, sizeof(double) * (size_t)d.n * K, s));
    if (d.P2) AMG_CUDA_TRY(cudaMemsetAsync(d.P2, 0, sizeof(DF) * (size_t)d.n * K, s));
    AMG_CUDA_TRY(cudaMemsetAsync(d.act, 0, sizeof(int) * d.npairs, s));
    Profiler prof;
    cudaEvent_t e0, e1;
    AMG_CUDA_TRY(cudaEventCreate(&e0));
    AMG_CUDA_TRY(cudaEventCreate(&e1));
    int best = 1, rc = AMG_OK;
    float best_ms = 1e30f;
    const int gs[4] = {1, 2, 4, 8};
    const Level &l0 = h->L[0];
    // the finest product first, in the form the solve runs (the systems
    // count as active while every pair is marked stopped, so the kernel does
    // its full work and its finisher changes nothing)
    int bestp = 1;
    float bestp_ms = 1e30f;
    for (int q = 0; q < 4 && rc >= 0; ++q) {
        launch_spmv0<false>(d, gs[q], l0.A.rp, l0.A.ci, l0.A.v, s);
        float t_best = 1e30f;
        for (int trial = 0; trial < 3; ++trial) {
            cudaEventRecord(e0, s);
            for (int k = 0; k < 2; ++k) launch_spmv0<false>(d, gs[q], l0.A.rp, l0.A.ci, l0.A.v, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = AMG_ERR_CUDA;
                break;
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            t_best = std::min(t_best, t);
        }
        W.gp_ms[q] = t_best;
        if (t_best < bestp_ms) {
            bestp_ms = t_best;
            bestp = gs[q];
        }
    }
    W.gp = bestp;
    for (int q = 0; q < 4 && rc >= 0; ++q) {
        W.g = gs[q];
        rc = vcycle_g(h, W, prof, s);
        float t_best = 1e30f;
        for (int trial = 0; trial < 3 && rc >= 0; ++trial) {
            cudaEventRecord(e0, s);
            for (int k = 0; k < 2 && rc >= 0; ++k) rc = vcycle_g(h, W, prof, s);
            cudaEventRecord(e1, s);
            if (rc >= 0 && cudaEventSynchronize(e1) == cudaSuccess) {
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                t_best = std::min(t_best, t);
            }
        }
        W.g_ms[q] = t_best;
        if (t_best < best_ms) {
            best_ms = t_best;
            best = gs[q];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    W.g = best;
    cudaMemsetAsync(d.nact, 0, sizeof(int), s);
    cudaMemsetAsync(d.sys_nact, 0, sizeof(int) * d.nsys, s);
    const cudaError_t se = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    AMG_TRY(rc);
    AMG_CUDA_TRY(se);
    return AMG_OK;
}

static int batch_iteration(Hierarchy *h, BatchWorkspace &W, Profiler &prof, cudaStream_t s) {
    const bool mixed = h->cfg.precision == AMG_PRECISION_MIXED;
    AMG_TRY(vcycle_g(h, W, prof, s));
    const Level &l0 = h->L[0];
    const BDev &d = W.d;
    const double nk = (double)d.n * K;
    {
        ProfScope ps(&prof, s, "b_p", 0, (mixed ? 32.0 : 24.0) * nk);
        kb_p<<<d.nchunks, BT, 0, s>>>(d);
    }
    {
        ProfScope ps(&prof, s, "b_spmv_pq", 0, l0.A.nnz * 12.0 + 4.0 * (d.n + 1) + 24.0 * nk);
        launch_spmv0<false>(d, W.gp, l0.A.rp, l0.A.ci, l0.A.v, s);
    }
    {
        ProfScope ps(&prof, s, "b_update", 0, (mixed ? 52.0 : 48.0) * nk);
        kb_update<<<d.nchunks, BT, 0, s>>>(d, h->cfg.max_iter);
    }
    AMG_LAUNCH_CHECK();
    return AMG_OK;
}

// Copies B ([n][nrhs], device) into the K-wide workspace (zero padding), and
// the result back.
__global__ void kb_pack(int n, int nrhs, const double *src, double *dst) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * K;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / K), r = (int)(e % K);
        dst[e] = r < nrhs ? src[(size_t)i * nrhs + r] : 0.0;
    }
}
__global__ void kb_unpack(int n, int nrhs, const double *src, double *dst) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * nrhs;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / nrhs), r = (int)(e % nrhs);
        dst[e] = src[(size_t)i * K + r];
    }
}

static bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int batch_solve(Hierarchy *h, BatchWorkspace *Wp, Profiler &prof, int nrhs, const double *Bin, double *Xout,
                int *iters_out, double *rel_out, cudaStream_t s, SolveResult *res) {
    BatchWorkspace &W = *Wp;
    const BDev &d = W.d;
    const amg_config &c = h->cfg;
    const Level &l0 = h->L[0];
    const int grid = std::max(1, std::min((int)(((long long)d.n * K + 255) / 256), num_sms() * 16));
    // stage: host arrays go through Q (free before the solve starts)
    const double *Bd = Bin;
    if (!on_device(Bin)) {
        AMG_CUDA_TRY(cudaMemcpyAsync(d.Q, Bin, sizeof(double) * (size_t)d.n * nrhs, cudaMemcpyDefault, s));
        Bd = d.Q;
    }
    kb_pack<<<grid, 256, 0, s>>>(d.n, nrhs, Bd, d.B);
    AMG_LAUNCH_CHECK();
    AMG_CUDA_TRY(cudaMemsetAsync(d.nact, 0, sizeof(int), s));
    AMG_CUDA_TRY(cudaMemsetAsync(d.sys_nact, 0, sizeof(int) * d.nsys, s));
    {
        ProfScope ps(&prof, s, "b_init", 0, 48.0 * d.n * K);
        kb_init<<<d.nchunks, BT, 0, s>>>(d, c.rtol);
    }
    AMG_LAUNCH_CHECK();
    int nact = 0;
    const long long cap = (long long)c.max_iter * (c.max_restarts + 1) + 16;
    long long launched = 0;
    int restarts = 0;
    for (;;) {
        AMG_CUDA_TRY(cudaMemcpyAsync(&nact, d.nact, sizeof(int), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        while (nact > 0) {
            // iterations of finished pairs are no-ops; the host polls every 4
            for (int k = 0; k < 4; ++k) {
                if (prof.on) {
                    AMG_TRY(batch_iteration(h, W, prof, s));
                    continue;
                }
                if (!W.iter_exec) {
                    const long long before = prof.launches;
                    AMG_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
                    const int rc = batch_iteration(h, W, prof, s);
                    cudaGraph_t g = nullptr;
                    const cudaError_t ce = cudaStreamEndCapture(s, &g);
                    if (rc < 0) {
                        if (g) cudaGraphDestroy(g);
                        return rc;
                    }
                    AMG_CUDA_TRY(ce);
                    const cudaError_t ie = cudaGraphInstantiate(&W.iter_exec, g, 0);
                    cudaGraphDestroy(g);
                    AMG_CUDA_TRY(ie);
                    W.iter_kernels = (int)(prof.launches - before);
                    prof.launches = before;
                }
                AMG_CUDA_TRY(cudaGraphLaunch(W.iter_exec, s));
                prof.launches += W.iter_kernels;
            }
            launched += 4;
            AMG_CUDA_TRY(cudaMemcpyAsync(&nact, d.nact, sizeof(int), cudaMemcpyDeviceToHost, s));
            AMG_CUDA_TRY(cudaStreamSynchronize(s));
            if (launched > cap) {
                set_last_error("batched solve: %lld iterations launched without every pair stopping", launched);
                return AMG_ERR_CUDA;
            }
        }
        // true residuals; restart the pairs still above the tolerance
        {
            ProfScope ps(&prof, s, "b_true_residual", 0, l0.A.nnz * 12.0 + 4.0 * (d.n + 1) + 24.0 * d.n * K);
            launch_spmv0<true>(d, W.gp, l0.A.rp, l0.A.ci, l0.A.v, s);
        }
        AMG_LAUNCH_CHECK();
        if (restarts >= c.max_restarts) break;
        kb_restart<<<std::max(1, (d.npairs + 255) / 256), 256, 0, s>>>(d, c.max_iter);
        AMG_LAUNCH_CHECK();
        AMG_CUDA_TRY(cudaMemcpyAsync(&nact, d.nact, sizeof(int), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        if (nact == 0) break;
        ++restarts;
    }
    // outputs
    double *Xd = Xout;
    const bool host_x = !on_device(Xout);
    if (host_x) Xd = d.Q;
    kb_unpack<<<grid, 256, 0, s>>>(d.n, nrhs, d.X, Xd);
    AMG_LAUNCH_CHECK();
    if (host_x) AMG_CUDA_TRY(cudaMemcpyAsync(Xout, d.Q, sizeof(double) * (size_t)d.n * nrhs, cudaMemcpyDefault, s));
    const int np = d.npairs;
    std::vector<int> st(np), it(np);
    std::vector<double> tr(np), bn(np), rr(np);
    AMG_CUDA_TRY(cudaMemcpyAsync(st.data(), d.status, sizeof(int) * np, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(it.data(), d.iters, sizeof(int) * np, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(tr.data(), d.tr, sizeof(double) * np, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(bn.data(), d.bn2, sizeof(double) * np, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(rr.data(), d.rr, sizeof(double) * np, cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    SolveResult out;
    out.restarts = restarts;
    std::vector<int> io((size_t)d.nsys * nrhs);
    std::vector<double> ro((size_t)d.nsys * nrhs);
    for (int sy = 0; sy < d.nsys; ++sy)
        for (int r = 0; r < nrhs; ++r) {
            const int p = sy * K + r;
            int sp = st[p];
            const double rel = bn[p] > 0.0 ? sqrt(tr[p] / bn[p]) : 0.0;
            if (sp == AMG_OK && bn[p] > 0.0 && !(tr[p] <= c.rtol * c.rtol * bn[p])) sp = AMG_MAXIT;
            out.status = std::max(out.status, sp);
            out.iters = std::max(out.iters, it[p]);
            out.rel_res_true = std::max(out.rel_res_true, rel);
            out.rel_res_rec = std::max(out.rel_res_rec, bn[p] > 0.0 ? sqrt(rr[p] / bn[p]) : 0.0);
            io[(size_t)sy * nrhs + r] = it[p];
            ro[(size_t)sy * nrhs + r] = rel;
        }
    if (iters_out) AMG_CUDA_TRY(cudaMemcpy(iters_out, io.data(), sizeof(int) * io.size(), cudaMemcpyDefault));
    if (rel_out) AMG_CUDA_TRY(cudaMemcpy(rel_out, ro.data(), sizeof(double) * ro.size(), cudaMemcpyDefault));
    prof.collect();
    *res = out;
    return AMG_OK;
}

}  // namespace amg
