// solve.cu -- solve phase: V(1,1) cycle, preconditioned CG and BiCGStab.
//
// Every kernel reads scal->done first and returns at once when the solve has
// finished, so the host may launch iterations ahead of the convergence check.
// Dot products are reduced deterministically: each block writes one partial
// sum, and the last block to finish (ticket counter) adds the partials in
// block order and updates the Krylov scalars on the device.
#include <algorithm>
#include <climits>
#include <type_traits>
#include <cstring>

#include "solve.cuh"
#include "stream.cuh"
#include "tail.cuh"
#include "mid.cuh"
#include "cpcg.cuh"

namespace amg {

constexpr int BLOCK = 256;

static int grid_rows(int n, int vec, int cap) {
    const int rpb = BLOCK / vec;
    return std::max(1, std::min((n + rpb - 1) / rpb, cap));
}

// Launches a solve-phase kernel with programmatic stream serialization, so
// that it starts while its predecessor drains (each such kernel waits on the
// dependency before reading what the predecessor wrote; see pdl_wait()).
template <typename... KArgs, typename... Args>
static int launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    AMG_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
    return AMG_OK;
}

#define VEC_DISPATCH(vec, ...)                          \
    switch (vec) {                                      \
        case 2: { constexpr int V = 2; __VA_ARGS__; } break;   \
        case 4: { constexpr int V = 4; __VA_ARGS__; } break;   \
        case 8: { constexpr int V = 8; __VA_ARGS__; } break;   \
        case 16: { constexpr int V = 16; __VA_ARGS__; } break; \
        default: { constexpr int V = 32; __VA_ARGS__; } break; \
    }

// ---------------------------------------------------------------------------
// Deterministic block reduction + last-block finisher
// ---------------------------------------------------------------------------

// Reduces NV values over the block, stores the block's partials, and returns
// true in the last block to arrive, with tot[] = sum over blocks in block order
// (valid in every thread of that block).
template <int NV, int NT = BLOCK>
__device__ bool reduce_last(double (&v)[NV], double *part, int cap, unsigned *counter, double (&tot)[NV]) {
    __shared__ double sh[NV][NT / 32];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double a = warp_sum(v[k]);
        if (lane == 0) sh[k][wid] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double a = 0.0;
            for (int w = 0; w < NT / 32; ++w) a += sh[k][w];
            part[k * cap + blockIdx.x] = a;
        }
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double a = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += NT) a += __ldcg(&part[k * cap + b]);
        a = warp_sum(a);
        __syncthreads();
        if (lane == 0) sh[k][wid] = a;
        __syncthreads();
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += sh[k][w];
        tot[k] = t;
    }
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

__device__ __forceinline__ bool finite(double a) { return isfinite(a); }

__device__ __forceinline__ void fail(DevScalars *sc, int status) {
    sc->status = status;
    sc->done = 1;
}

// ---------------------------------------------------------------------------
// Loads (the V-cycle may read FP64 inputs into FP32 arithmetic)
// ---------------------------------------------------------------------------

template <typename TM, typename T>
__device__ __forceinline__ TM ld(const T *p, int i) { return fcvt<TM>(__ldg(p + i)); }

// ---------------------------------------------------------------------------
// V-cycle kernels: VEC threads per row, grid-stride over warps so that every
// lane of a warp runs the same number of iterations (shuffles are warp-wide).
// ---------------------------------------------------------------------------

#define ROW_LOOP(VEC, n)                                                                     \
    const int lane_ = threadIdx.x & (VEC - 1);                                               \
    const int rows_per_warp_ = 32 / VEC;                                                     \
    const int warp_ = (blockIdx.x * BLOCK + threadIdx.x) >> 5;                               \
    const int nwarps_ = (gridDim.x * BLOCK) >> 5;                                            \
    const int sub_ = (threadIdx.x & 31) / VEC;                                               \
    for (int base_ = warp_ * rows_per_warp_; base_ < (n); base_ += nwarps_ * rows_per_warp_) { \
        const int i = base_ + sub_;                                                          \
        const bool valid = i < (n);

#define ROW_LOOP_END }

// sum over k = k0, k0 + VEC, ... < e of v[k] * g(ci[k]), in that order: the
// indices and values of ROW_UNR terms load before their gathers, so a lane
// waits on two round trips per ROW_UNR terms instead of two per term.
constexpr int ROW_UNR = 4;

template <int VEC, typename TM, class G>
__device__ __forceinline__ TM row_dot(const int *__restrict__ ci, const TM *__restrict__ v, int k0, int e, G g) {
    TM s = 0;
    for (int kb = k0; kb < e; kb += VEC * ROW_UNR) {
        int c[ROW_UNR];
        TM a[ROW_UNR];
#pragma unroll
        for (int u = 0; u < ROW_UNR; ++u) {
            const int k = kb + u * VEC;
            if (k < e) {
                c[u] = __ldg(ci + k);
                a[u] = __ldg(v + k);
            }
        }
#pragma unroll
        for (int u = 0; u < ROW_UNR; ++u)
            if (kb + u * VEC < e) s += a[u] * g(c[u]);
    }
    return s;
}

// r = b - A (W b): pre-smoothing from x = 0 fused with the residual.
template <int VEC, typename TB, typename TM>
__global__ void __launch_bounds__(BLOCK) k_presmooth(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                     const TM *__restrict__ v, const TM *__restrict__ w,
                                                     const TB *__restrict__ b, TM *__restrict__ r, const int *done) {
    pdl_wait();
    pdl_trigger();
    if (*done) return;
    ROW_LOOP(VEC, n)
    TM s = 0;
    if (valid) s = row_dot<VEC>(ci, v, rp[i] + lane_, rp[i + 1], [&](int j) { return ld<TM>(w, j) * ld<TM>(b, j); });
    s = group_sum<VEC>(s);
    if (valid && lane_ == 0) r[i] = ld<TM>(b, i) - s;
    ROW_LOOP_END
}

// y = M x (restriction by R = P^T, or any plain CSR product).
template <int VEC, typename TX, typename TM, typename TY>
__global__ void __launch_bounds__(BLOCK) k_spmv(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                const TM *__restrict__ v, const TX *__restrict__ x,
                                                TY *__restrict__ y, const int *done) {
    pdl_wait();
    pdl_trigger();
    if (*done) return;
    ROW_LOOP(VEC, n)
    TM s = 0;
    if (valid) s = row_dot<VEC>(ci, v, rp[i] + lane_, rp[i + 1], [&](int j) { return ld<TM>(x, j); });
    s = group_sum<VEC>(s);
    if (valid && lane_ == 0) y[i] = (TY)s;
    ROW_LOOP_END
}

// t = W b + P x_c: the pre-smoothed iterate (recomputed) plus the coarse correction.
template <int VEC, typename TB, typename TM>
__global__ void __launch_bounds__(BLOCK) k_prolong(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                   const TM *__restrict__ v, const TM *__restrict__ w,
                                                   const TB *__restrict__ b, const TM *__restrict__ xc,
                                                   TM *__restrict__ t, const int *done) {
    pdl_wait();
    pdl_trigger();
    if (*done) return;
    ROW_LOOP(VEC, n)
    TM s = 0;
    if (valid) s = row_dot<VEC>(ci, v, rp[i] + lane_, rp[i + 1], [&](int j) { return xc[j]; });
    s = group_sum<VEC>(s);
    if (valid && lane_ == 0) t[i] = ld<TM>(w, i) * ld<TM>(b, i) + s;
    ROW_LOOP_END
}

enum Fin { FIN_NONE = 0, FIN_PCG_BETA = 1 };

// Finisher of the PCG preconditioner application: rz_new = r.z (and, for the
// flexible form, z.q with q = A p of the previous iteration); beta = rz_new / rz,
// or for the flexible form z.(r - r_old) / rz = -alpha z.q / rz (r - r_old =
// -alpha q); the first iteration after a (re)start uses beta = 0.
__device__ void finish_pcg_beta(DevScalars *sc, const double *tot) {
    const double rz_new = tot[0];
    if (!finite(rz_new)) { fail(sc, AMG_NAN); return; }
    double beta = 0.0;
    if (!sc->first) {
        const double num = sc->flexible ? -sc->alpha * tot[1] : rz_new;
        beta = num / sc->rz;
    }
    sc->first = 0;
    sc->beta = beta;
    sc->rz = rz_new;
}

// x = t + W (b - A t): post-smoothing.  FIN_PCG_BETA also reduces r.z (r = b,
// the V-cycle input) and, for the flexible form, z.qprev (qprev = A p of the
// previous iteration), and finishes beta.
template <int VEC, typename TB, typename TM, typename TO, int FIN>
__global__ void __launch_bounds__(BLOCK) k_postsmooth(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                      const TM *__restrict__ v, const TM *__restrict__ w,
                                                      const TB *__restrict__ b, const TM *__restrict__ t,
                                                      TO *__restrict__ out, const double *__restrict__ qprev,
                                                      DevScalars *sc, double *part, int cap, unsigned *counter) {
    pdl_wait();
    pdl_trigger();
    if (sc->done) return;
    double acc[2] = {0.0, 0.0};
    ROW_LOOP(VEC, n)
    TM s = 0;
    if (valid) s = row_dot<VEC>(ci, v, rp[i] + lane_, rp[i + 1], [&](int j) { return t[j]; });
    s = group_sum<VEC>(s);
    if (valid && lane_ == 0) {
        const TM bi = ld<TM>(b, i);
        const TM xi = t[i] + ld<TM>(w, i) * (bi - s);
        const TO o = fcvt<TO>(xi);
        out[i] = o;
        if (FIN == FIN_PCG_BETA) {
            acc[0] += ld<double>(b, i) * fcvt<double>(o);
            if (qprev) acc[1] += qprev[i] * fcvt<double>(o);
        }
    }
    ROW_LOOP_END
    if (FIN == FIN_PCG_BETA) {
        double tot[2];
        if (reduce_last<2>(acc, part, cap, counter, tot) && threadIdx.x == 0) finish_pcg_beta(sc, tot);
    }
}

// Coarsest level: x = A_c^-1 b in FP64 with the stored dense inverse (one block).
template <typename TI, typename TO, int FIN>
__global__ void __launch_bounds__(BLOCK) k_coarse(int m, const double *__restrict__ cinv, const TI *__restrict__ b,
                                                  TO *__restrict__ x, const double *__restrict__ qprev,
                                                  DevScalars *sc, double *part, int cap, unsigned *counter) {
    pdl_wait();
    pdl_trigger();
    if (sc->done) return;
    __shared__ double sb[AMG_DENSE_MAX];
    for (int i = threadIdx.x; i < m; i += BLOCK) sb[i] = fcvt<double>(b[i]);
    __syncthreads();
    double acc[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < m; i += BLOCK) {
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += cinv[(size_t)i * m + j] * sb[j];
        const TO o = fcvt<TO>(s);
        x[i] = o;
        if (FIN == FIN_PCG_BETA) {
            acc[0] += sb[i] * fcvt<double>(o);
            if (qprev) acc[1] += qprev[i] * fcvt<double>(o);
        }
    }
    if (FIN == FIN_PCG_BETA) {
        double tot[2];
        if (reduce_last<2>(acc, part, cap, counter, tot) && threadIdx.x == 0) finish_pcg_beta(sc, tot);
    }
}

// The dense operator of the coarse end of the cycle, x = M b (dense_rows:
// one warp per row, 16 16-byte loads of a lane in flight, a 2048-float row in
// one round).
template <typename TMAT, typename TV>
__global__ void __launch_bounds__(BLOCK) k_dense_apply(int m, int ld, const TMAT *__restrict__ M,
                                                       const TV *__restrict__ b, TV *__restrict__ x, const int *done) {
    pdl_wait();
    pdl_trigger();
    if (*done) return;
    __shared__ __align__(16) double sb[mid::DENSE_LD];
    mid::dense_rows<16, TMAT, TV>(m, ld, M, b, x, sb);
}

// ---------------------------------------------------------------------------
// Krylov kernels (FP64)
// ---------------------------------------------------------------------------

// PCG start: x = 0, r = b, p = 0, ||b||^2.
// cg: unpreconditioned CG, whose r.z is r.r (b.b here) with no beta pass.
__global__ void __launch_bounds__(BLOCK) k_pcg_init(int n, const double *__restrict__ b, double *x, double *r,
                                                    double *p, float *r32, DevScalars *sc, double rtol,
                                                    double *part, int cap, unsigned *counter, int cg) {
    pdl_wait();
    pdl_trigger();
    double acc[1] = {0.0};
    for (int i = blockIdx.x * BLOCK + threadIdx.x; i < n; i += gridDim.x * BLOCK) {
        const double bi = b[i];
        x[i] = 0.0;
        r[i] = bi;
        if (r32) r32[i] = f64_to_f32_rn(bi);
        p[i] = 0.0;
        acc[0] += bi * bi;
    }
    double tot[1];
    if (reduce_last<1>(acc, part, cap, counter, tot) && threadIdx.x == 0) {
        sc->bn2 = tot[0];
        sc->tol2 = rtol * rtol * tot[0];
        sc->rr = tot[0];
        sc->iters = 0;
        sc->beta = 0.0;
        sc->first = 1;
        if (cg) {
            sc->rz = tot[0];
            sc->first = 0;
        }
        sc->status = AMG_OK;
        sc->done = 0;
        if (!finite(tot[0])) fail(sc, AMG_NAN);
        else if (tot[0] == 0.0) sc->done = 1;
    }
}

// p = z + beta p
__global__ void __launch_bounds__(BLOCK) k_pcg_p(int n, const double *__restrict__ z, double *p, DF *p2,
                                                 const DevScalars *sc) {
    pdl_wait();
    pdl_trigger();
    if (sc->done) return;
    const double beta = sc->beta;
    // pairs of entries as 16-byte accesses (the workspace vectors are
    // allocation-aligned), then the odd last entry; p2 (when given) takes p
    // split into FP32 pairs for the double-FP32 product
    const int n2 = n >> 1, g0 = blockIdx.x * BLOCK + threadIdx.x, gs = gridDim.x * BLOCK;
    const double2 *z2 = reinterpret_cast<const double2 *>(z);
    double2 *pp2 = reinterpret_cast<double2 *>(p);
    for (int i = g0; i < n2; i += gs) {
        const double2 zv = z2[i];
        double2 pv;
        if (beta == 0.0) {  // first step after a (re)start: p = z exactly
            pv = zv;
        } else {
            pv = pp2[i];
            pv.x = zv.x + beta * pv.x;
            pv.y = zv.y + beta * pv.y;
        }
        pp2[i] = pv;
        if (p2) {
            const DF a = df_split(pv.x), b = df_split(pv.y);
            reinterpret_cast<float4 *>(p2)[i] = make_float4(a.hi, a.lo, b.hi, b.lo);
        }
    }
    if ((n & 1) && g0 == 0) {
        const double pv = beta == 0.0 ? z[n - 1] : z[n - 1] + beta * p[n - 1];
        p[n - 1] = pv;
        if (p2) p2[n - 1] = df_split(pv);
    }
}

enum SpmvFin { SF_PCG_ALPHA = 0, SF_BICG_ALPHA = 1, SF_BICG_OMEGA = 2, SF_TRUE_RES = 3 };

// y = A x fused with a finisher:
//   SF_PCG_ALPHA : p.q           -> alpha = rz / p.q     (dvec = x)
//   SF_BICG_ALPHA: r^.v          -> alpha = rho / r^.v  (dvec = r^)
//   SF_BICG_OMEGA: t.s, t.t      -> omega = t.s / t.t   (dvec = s)
//   SF_TRUE_RES  : y = b - A x,  ||y||^2 -> tr          (dvec = b)
// Finisher of the outer products (one thread of the last block).
template <int SF>
__device__ void finish_spmv(DevScalars *sc, const double (&tot)[2]) {
    if (SF == SF_PCG_ALPHA) {
        const double pq = tot[0];
        if (!finite(pq)) fail(sc, AMG_NAN);
        else if (pq <= 0.0) fail(sc, AMG_BREAKDOWN);
        else { sc->pq = pq; sc->alpha = sc->rz / pq; }
    } else if (SF == SF_BICG_ALPHA) {
        const double rv = tot[0];
        if (!finite(rv)) fail(sc, AMG_NAN);
        else if (rv == 0.0) fail(sc, AMG_BREAKDOWN);
        else { sc->rv = rv; sc->alpha = sc->rho / rv; }
    } else if (SF == SF_BICG_OMEGA) {
        const double ts = tot[0], tt = tot[1];
        if (!finite(ts) || !finite(tt)) fail(sc, AMG_NAN);
        else if (tt == 0.0) fail(sc, AMG_BREAKDOWN);
        else { sc->ts = ts; sc->tt = tt; sc->omega = ts / tt; }
    } else {
        sc->tr = tot[0];
    }
}

template <int VEC, int SF>
__global__ void __launch_bounds__(BLOCK) k_spmv_fin(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                    const double *__restrict__ v, const double *__restrict__ x,
                                                    double *__restrict__ y, float *__restrict__ y32,
                                                    const double *__restrict__ dvec, DevScalars *sc, double *part,
                                                    int cap, unsigned *counter) {
    pdl_wait();
    pdl_trigger();
    if (SF != SF_TRUE_RES && sc->done) return;
    double acc[2] = {0.0, 0.0};
    ROW_LOOP(VEC, n)
    double s = 0.0;
    if (valid) {
        const int e = rp[i + 1];
        for (int k = rp[i] + lane_; k < e; k += VEC) s += v[k] * __ldg(x + ci[k]);
    }
    s = group_sum<VEC>(s);
    if (valid && lane_ == 0) {
        if (SF == SF_TRUE_RES) {
            const double ri = dvec[i] - s;
            y[i] = ri;
            if (y32) y32[i] = f64_to_f32_rn(ri);
            acc[0] += ri * ri;
        } else {
            y[i] = s;
            if (SF == SF_PCG_ALPHA) acc[0] += x[i] * s;
            if (SF == SF_BICG_ALPHA) acc[0] += dvec[i] * s;
            if (SF == SF_BICG_OMEGA) { acc[0] += s * dvec[i]; acc[1] += s * s; }
        }
    }
    ROW_LOOP_END
    double tot[2];
    if (reduce_last<2>(acc, part, cap, counter, tot) && threadIdx.x == 0) finish_spmv<SF>(sc, tot);
}

// x += alpha p; (r_old = r;) r -= alpha q; ||r||^2; convergence / iteration cap.
__global__ void __launch_bounds__(BLOCK) k_pcg_update(int n, double *x, double *r, const double *__restrict__ p,
                                                      const double *__restrict__ q, float *r32,
                                                      DevScalars *sc, double *part, int cap, unsigned *counter,
                                                      int cg) {
    pdl_wait();
    pdl_trigger();
    if (sc->done) return;
    const double alpha = sc->alpha;
    double acc[1] = {0.0};
    // pairs of entries as 16-byte accesses (the workspace vectors are
    // allocation-aligned), then the odd last entry
    const int n2 = n >> 1, g0 = blockIdx.x * BLOCK + threadIdx.x, gs = gridDim.x * BLOCK;
    double2 *x2 = reinterpret_cast<double2 *>(x), *r2 = reinterpret_cast<double2 *>(r);
    const double2 *p2 = reinterpret_cast<const double2 *>(p), *q2 = reinterpret_cast<const double2 *>(q);
    for (int i = g0; i < n2; i += gs) {
        double2 xv = x2[i];
        const double2 pv = p2[i], qv = q2[i];
        double2 rv = r2[i];
        xv.x += alpha * pv.x;
        xv.y += alpha * pv.y;
        rv.x = rv.x - alpha * qv.x;
        rv.y = rv.y - alpha * qv.y;
        x2[i] = xv;
        r2[i] = rv;
        if (r32) reinterpret_cast<float2 *>(r32)[i] = make_float2(f64_to_f32_rn(rv.x), f64_to_f32_rn(rv.y));
        acc[0] += rv.x * rv.x;
        acc[0] += rv.y * rv.y;
    }
    if ((n & 1) && g0 == 0) {
        const int i = n - 1;
        x[i] += alpha * p[i];
        const double rn = r[i] - alpha * q[i];
        r[i] = rn;
        if (r32) r32[i] = f64_to_f32_rn(rn);
        acc[0] += rn * rn;
    }
    double tot[1];
    if (reduce_last<1>(acc, part, cap, counter, tot) && threadIdx.x == 0) {
        sc->iters += 1;
        sc->rr = tot[0];
        if (cg) {
            // unpreconditioned CG: z = r, so the next beta is ||r_new||^2 / ||r||^2
            sc->beta = tot[0] / sc->rz;
            sc->rz = tot[0];
        }
        if (!finite(tot[0])) fail(sc, AMG_NAN);
        else if (tot[0] <= sc->tol2) sc->done = 1;
        else if (sc->iters >= sc->max_iter) fail(sc, AMG_MAXIT);
    }
}

// BiCGStab start: x = 0, r = r^ = b, p = v = 0, rho = b.b, rho_old = alpha = omega = 1.
__global__ void __launch_bounds__(BLOCK) k_bicg_init(int n, const double *__restrict__ b, double *x, double *r,
                                                     double *rh, double *p, double *v, DevScalars *sc, double rtol,
                                                     double *part, int cap, unsigned *counter) {
    pdl_wait();
    pdl_trigger();
    double acc[1] = {0.0};
    for (int i = blockIdx.x * BLOCK + threadIdx.x; i < n; i += gridDim.x * BLOCK) {
        const double bi = b[i];
        x[i] = 0.0;
        r[i] = bi;
        rh[i] = bi;
        p[i] = 0.0;
        v[i] = 0.0;
        acc[0] += bi * bi;
    }
    double tot[1];
    if (reduce_last<1>(acc, part, cap, counter, tot) && threadIdx.x == 0) {
        sc->bn2 = tot[0];
        sc->tol2 = rtol * rtol * tot[0];
        sc->rr = tot[0];
        sc->rho = tot[0];
        sc->rho_old = 1.0;
        sc->alpha = 1.0;
        sc->omega = 1.0;
        sc->iters = 0;
        sc->status = AMG_OK;
        sc->done = 0;
        if (!finite(tot[0])) fail(sc, AMG_NAN);
        else if (tot[0] == 0.0) sc->done = 1;
    }
}

// Restart from the current x with r = r^ = b - A x (r already holds it).
__global__ void __launch_bounds__(BLOCK) k_bicg_restart(int n, const double *__restrict__ r, double *rh, double *p,
                                                        double *v, DevScalars *sc, double *part, int cap,
                                                        unsigned *counter) {
    pdl_wait();
    pdl_trigger();
    double acc[1] = {0.0};
    for (int i = blockIdx.x * BLOCK + threadIdx.x; i < n; i += gridDim.x * BLOCK) {
        const double ri = r[i];
        rh[i] = ri;
        p[i] = 0.0;
        v[i] = 0.0;
        acc[0] += ri * ri;
    }
    double tot[1];
    if (reduce_last<1>(acc, part, cap, counter, tot) && threadIdx.x == 0) {
        sc->rr = tot[0];
        sc->rho = tot[0];
        sc->rho_old = 1.0;
        sc->alpha = 1.0;
        sc->omega = 1.0;
        sc->status = AMG_OK;
        sc->done = 0;
        if (!finite(tot[0])) fail(sc, AMG_NAN);
        else if (tot[0] == 0.0) sc->done = 1;
    }
}

// p = r + beta (p - omega v), beta = (rho / rho_old)(alpha / omega); counts the iteration.
__global__ void __launch_bounds__(BLOCK) k_bicg_p(int n, const double *__restrict__ r, double *p,
                                                  const double *__restrict__ v, float *p32, DevScalars *sc) {
    pdl_wait();
    pdl_trigger();
    if (sc->done) return;
    const double beta = (sc->rho / sc->rho_old) * (sc->alpha / sc->omega);
    const double omega = sc->omega;
    for (int i = blockIdx.x * BLOCK + threadIdx.x; i < n; i += gridDim.x * BLOCK) {
        const double pi = r[i] + beta * (p[i] - omega * v[i]);
        p[i] = pi;
        if (p32) p32[i] = f64_to_f32_rn(pi);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->iters += 1;
}

// s = r - alpha v; x += alpha p^; ||s||^2 (early exit when small).
__global__ void __launch_bounds__(BLOCK) k_bicg_s(int n, const double *__restrict__ r, const double *__restrict__ v,
                                                  double *s, float *s32, double *x, const double *__restrict__ ph,
                                                  DevScalars *sc, double *part, int cap, unsigned *counter) {
    pdl_wait();
    pdl_trigger();
    if (sc->done) return;
    const double alpha = sc->alpha;
    double acc[1] = {0.0};
    for (int i = blockIdx.x * BLOCK + threadIdx.x; i < n; i += gridDim.x * BLOCK) {
        const double si = r[i] - alpha * v[i];
        s[i] = si;
        if (s32) s32[i] = f64_to_f32_rn(si);
        x[i] += alpha * ph[i];
        acc[0] += si * si;
    }
    double tot[1];
    if (reduce_last<1>(acc, part, cap, counter, tot) && threadIdx.x == 0) {
        sc->ss = tot[0];
        sc->rr = tot[0];
        if (!finite(tot[0])) fail(sc, AMG_NAN);
        else if (tot[0] <= sc->tol2) sc->done = 1;
    }
}

// x += omega s^; r = s - omega t; ||r||^2 and the next rho = r^.r.
__global__ void __launch_bounds__(BLOCK) k_bicg_update(int n, double *x, const double *__restrict__ sh, double *r,
                                                       const double *__restrict__ s, const double *__restrict__ t,
                                                       const double *__restrict__ rh, DevScalars *sc, double *part,
                                                       int cap, unsigned *counter) {
    pdl_wait();
    pdl_trigger();
    if (sc->done) return;
    const double omega = sc->omega;
    double acc[2] = {0.0, 0.0};
    for (int i = blockIdx.x * BLOCK + threadIdx.x; i < n; i += gridDim.x * BLOCK) {
        x[i] += omega * sh[i];
        const double ri = s[i] - omega * t[i];
        r[i] = ri;
        acc[0] += ri * ri;
        acc[1] += rh[i] * ri;
    }
    double tot[2];
    if (reduce_last<2>(acc, part, cap, counter, tot) && threadIdx.x == 0) {
        sc->rr = tot[0];
        if (!finite(tot[0]) || !finite(tot[1])) fail(sc, AMG_NAN);
        else if (tot[0] <= sc->tol2) sc->done = 1;
        else if (omega == 0.0 || tot[1] == 0.0) fail(sc, AMG_BREAKDOWN);
        else if (sc->iters >= sc->max_iter) fail(sc, AMG_MAXIT);
        else { sc->rho_old = sc->rho; sc->rho = tot[1]; }
    }
}

__global__ void k_copy(int n, const double *__restrict__ a, double *b) {
    pdl_wait();
    pdl_trigger();
    for (int i = blockIdx.x * BLOCK + threadIdx.x; i < n; i += gridDim.x * BLOCK) b[i] = a[i];
}

// dA[k] = -lambda_i x_{col(k)} for every stored entry of row i.
template <int VEC>
__global__ void __launch_bounds__(BLOCK) k_grad_values(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                       const double *__restrict__ lambda,
                                                       const double *__restrict__ x, double *__restrict__ dA) {
    pdl_wait();
    pdl_trigger();
    ROW_LOOP(VEC, n)
    if (valid) {
        const double li = -lambda[i];
        const int e = rp[i + 1];
        for (int k = rp[i] + lane_; k < e; k += VEC) dA[k] = li * __ldg(x + ci[k]);
    }
    ROW_LOOP_END
}

// Host-chosen control fields of the device scalars.  A reset also clears the
// arrival count of the fused coarse levels' grid barrier (left nonzero only
// by a barrier wait that gave up).
__global__ void k_set_control(DevScalars *sc, int done, int status, int flexible, int max_iter, int reset_iters,
                              unsigned *gbar) {
    pdl_wait();
    pdl_trigger();
    sc->done = done;
    sc->status = status;
    sc->flexible = flexible;
    sc->max_iter = max_iter;
    sc->tr_fresh = 0;
    if (reset_iters) {
        sc->iters = 0;
        sc->trips = 0;
        sc->copy_timeout = 0;
        gbar[0] = 0;
    }
}

// The condition of the device-side Krylov loop, after each pass of its body:
// repeat while the solve is running and fewer than cap passes have run (the
// device sets done at max_iter at the latest; cap only bounds the loop).
__global__ void k_loop_cond(cudaGraphConditionalHandle hd, DevScalars *sc, int cap) {
    pdl_wait();
    pdl_trigger();
    const int t = ++sc->trips;
    cudaGraphSetConditional(hd, (sc->done == 0 && t < cap) ? 1u : 0u);
}

// The next preconditioner application starts a new recursion (beta = 0, p = z).
__global__ void k_pcg_restart(DevScalars *sc, int cg) {
    pdl_wait();
    pdl_trigger();
    if (cg) {  // unpreconditioned CG: p = r, r.z = ||r||^2 of the true residual
        sc->beta = 0.0;
        sc->rz = sc->tr;
        sc->first = 0;
    } else {
        sc->first = 1;
    }
}

// ---------------------------------------------------------------------------
// Tracing
// ---------------------------------------------------------------------------

int Profiler::find(const char *name, int level) {
    for (size_t i = 0; i < recs.size(); ++i)
        if (recs[i].level == level && strncmp(recs[i].name, name, sizeof(recs[i].name)) == 0) return (int)i;
    Rec r;
    memset(&r, 0, sizeof(r));
    strncpy(r.name, name, sizeof(r.name) - 1);
    r.level = level;
    recs.push_back(r);
    return (int)recs.size() - 1;
}

cudaEvent_t Profiler::event() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

int Profiler::collect() {
    for (const Pending &q : pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) recs[q.rec].ms += ms;
        pool.push_back(q.a);
        pool.push_back(q.b);
    }
    pending.clear();
    return AMG_OK;
}

void Profiler::reset() {
    collect();
    recs.clear();
    launches = 0;
}

void Profiler::destroy() {
    collect();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
}

ProfScope::ProfScope(Profiler *p_, cudaStream_t s_, const char *name, int level, double bytes) : p(p_), s(s_) {
    if (!p) return;
    p->launches++;
    if (!p->on) return;
    rec = p->find(name, level);
    p->recs[rec].launches++;
    p->recs[rec].bytes += bytes;
    a = p->event();
    cudaEventRecord(a, s);
}

ProfScope::~ProfScope() {
    if (!a) return;
    cudaEvent_t b = p->event();
    cudaEventRecord(b, s);
    p->pending.push_back({rec, a, b});
}

#define TRACE(name, level, bytes) ProfScope prof_scope_(&W.prof, s, name, level, (double)(bytes))

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

int workspace_init(Workspace &W, int n) {
    W.n = n;
    DevArena &a = W.arena;
    double **vecs[] = {&W.b, &W.x, &W.r, &W.z, &W.p, &W.q, &W.rh, &W.v, &W.ph, &W.s, &W.sh, &W.t, &W.aux};
    for (double **pp : vecs) AMG_TRY(a.alloc(pp, (size_t)n));
    AMG_TRY(a.alloc(&W.r32, (size_t)n));
    AMG_TRY(a.alloc(&W.p2, (size_t)n));
    AMG_TRY(a.alloc(&W.scal, 1));
    W.part_cap = num_sms() * 8;
    AMG_TRY(a.alloc(&W.part, (size_t)3 * W.part_cap));
    AMG_TRY(a.alloc(&W.counter, 4));
    AMG_CUDA_TRY(cudaMemset(W.counter, 0, 4 * sizeof(unsigned)));
    AMG_TRY(a.alloc(&W.gbar, 2));
    AMG_CUDA_TRY(cudaMemset(W.gbar, 0, 2 * sizeof(unsigned)));
    AMG_CUDA_TRY(cudaMemset(W.scal, 0, sizeof(DevScalars)));
    AMG_CUDA_TRY(cudaMallocHost(&W.scal_h, sizeof(DevScalars)));
    memset(W.scal_h, 0, sizeof(DevScalars));
    AMG_CUDA_TRY(cudaStreamSynchronize(0));  // the memsets above ran on the legacy stream
    return AMG_OK;
}

void workspace_free(Workspace &W) {
    W.prof.destroy();
    W.arena.free_all();
    if (W.scal_h) cudaFreeHost(W.scal_h);
    W.scal_h = nullptr;
}

// ---------------------------------------------------------------------------
// Epilogues of the bulk-copy streaming kernel (stream.cuh)
// ---------------------------------------------------------------------------

// r = b - (A W) b
template <typename TB, typename TM>
struct OpPre {
    const int *dn;
    const TB *b;
    TM *r;
    struct Pre {
        TB b;
    };
    __device__ bool done() const { return *dn != 0; }
    __device__ TM gather(int j) const { return fcvt<TM>(__ldg(b + j)); }
    using GX = TB;
    __device__ const GX *gsrc() const { return b; }
    __device__ Pre load(int i) const { return Pre{__ldg(b + i)}; }
    static constexpr bool SELF = true;  // the epilogue needs the gathered vector's own entry
    static constexpr int NROWV = 0, ROWV_BYTES = 0;  // row operands staged by the sliced-ELL kernel
    __device__ Pre load_rest(int) const { return Pre{}; }
    __device__ void put_self(Pre &p, GX v) const { p.b = v; }
    __device__ void finish(int i, TM s, const Pre &p, double (&)[2]) const { r[i] = fcvt<TM>(p.b) - s; }
    template <int NT>
    __device__ void reduce(double (&)[2]) const {}
};

// y = M x
template <typename TM>
struct OpSpmv {
    const int *dn;
    const TM *x;
    TM *y;
    struct Pre {};
    __device__ bool done() const { return *dn != 0; }
    __device__ TM gather(int j) const { return __ldg(x + j); }
    using GX = TM;
    __device__ const GX *gsrc() const { return x; }
    __device__ Pre load(int) const { return Pre{}; }
    static constexpr bool SELF = false;
    static constexpr int NROWV = 0, ROWV_BYTES = 0;
    __device__ Pre load_rest(int i) const { return load(i); }
    __device__ void put_self(Pre &, GX) const {}
    __device__ void finish(int i, TM s, const Pre &, double (&)[2]) const { y[i] = s; }
    template <int NT>
    __device__ void reduce(double (&)[2]) const {}
};

// y = M x with x of type TG (the autotuner's probe of a plan: gathers the type
// the plan's heaviest use gathers)
template <typename TM, typename TG>
struct OpTune {
    const int *dn;
    const TG *x;
    TM *y;
    struct Pre {};
    __device__ bool done() const { return *dn != 0; }
    __device__ TM gather(int j) const { return fcvt<TM>(__ldg(x + j)); }
    using GX = TG;
    __device__ const GX *gsrc() const { return x; }
    __device__ Pre load(int) const { return Pre{}; }
    static constexpr bool SELF = false;
    static constexpr int NROWV = 0, ROWV_BYTES = 0;
    __device__ Pre load_rest(int i) const { return load(i); }
    __device__ void put_self(Pre &, GX) const {}
    __device__ void finish(int i, TM s, const Pre &, double (&)[2]) const { y[i] = s; }
    template <int NT>
    __device__ void reduce(double (&)[2]) const {}
};

// t = W b + P x_c
template <typename TB, typename TM>
struct OpProlong {
    const int *dn;
    const TM *w;
    const TB *b;
    const TM *xc;
    TM *t;
    struct Pre {
        TM w;
        TB b;
    };
    __device__ bool done() const { return *dn != 0; }
    __device__ TM gather(int j) const { return __ldg(xc + j); }
    using GX = TM;
    __device__ const GX *gsrc() const { return xc; }
    __device__ Pre load(int i) const { return Pre{__ldg(w + i), __ldg(b + i)}; }
    static constexpr bool SELF = false;
    __device__ Pre load_rest(int i) const { return load(i); }
    // row operands the sliced-ELL kernel stages with each tile: w, b
    static constexpr int NROWV = 2, ROWV_BYTES = (int)(sizeof(TM) + sizeof(TB));
    __device__ int rowv(const void **src, int *eb) const {
        src[0] = w;
        eb[0] = (int)sizeof(TM);
        src[1] = b;
        eb[1] = (int)sizeof(TB);
        return 2;
    }
    __device__ Pre load_rowv(const unsigned char *const *rv, int rl) const {
        return Pre{reinterpret_cast<const TM *>(rv[0])[rl], reinterpret_cast<const TB *>(rv[1])[rl]};
    }
    __device__ void put_self(Pre &, GX) const {}
    __device__ void finish(int i, TM s, const Pre &p, double (&)[2]) const { t[i] = p.w * fcvt<TM>(p.b) + s; }
    template <int NT>
    __device__ void reduce(double (&)[2]) const {}
};

// out = t + W (b - A t), with the PCG beta finisher on level 0
template <typename TB, typename TM, typename TO, int FIN>
struct OpPost {
    DevScalars *sc;
    const TM *w;
    const TB *b;
    const TM *t;
    TO *out;
    const double *qprev;  // flexible PCG: A p of the previous iteration (else null)
    double *part;
    int cap;
    unsigned *counter;
    struct Pre {
        TM t, w;
        TB b;
        double ro;
    };
    __device__ bool done() const { return sc->done != 0; }
    __device__ TM gather(int j) const { return __ldg(t + j); }
    using GX = TM;
    __device__ const GX *gsrc() const { return t; }
    __device__ Pre load(int i) const {
        return Pre{__ldg(t + i), __ldg(w + i), __ldg(b + i), (FIN == FIN_PCG_BETA && qprev) ? __ldg(qprev + i) : 0.0};
    }
    static constexpr bool SELF = true;
    __device__ Pre load_rest(int i) const {
        return Pre{(TM)0, __ldg(w + i), __ldg(b + i), (FIN == FIN_PCG_BETA && qprev) ? __ldg(qprev + i) : 0.0};
    }
    // row operands the sliced-ELL kernel stages with each tile: w, b (and qprev)
    static constexpr int NROWV = FIN == FIN_PCG_BETA ? 3 : 2;
    static constexpr int ROWV_BYTES = (int)(sizeof(TM) + sizeof(TB)) + (FIN == FIN_PCG_BETA ? 8 : 0);
    __device__ int rowv(const void **src, int *eb) const {
        src[0] = w;
        eb[0] = (int)sizeof(TM);
        src[1] = b;
        eb[1] = (int)sizeof(TB);
        if (FIN != FIN_PCG_BETA || !qprev) return 2;
        src[2] = qprev;
        eb[2] = 8;
        return 3;
    }
    __device__ Pre load_rowv(const unsigned char *const *rv, int rl) const {
        return Pre{(TM)0, reinterpret_cast<const TM *>(rv[0])[rl], reinterpret_cast<const TB *>(rv[1])[rl],
                   (FIN == FIN_PCG_BETA && qprev) ? reinterpret_cast<const double *>(rv[2])[rl] : 0.0};
    }
    __device__ void put_self(Pre &p, GX v) const { p.t = v; }
    __device__ void finish(int i, TM s, const Pre &p, double (&acc)[2]) const {
        const TO o = fcvt<TO>(p.t + p.w * (fcvt<TM>(p.b) - s));
        out[i] = o;
        if (FIN == FIN_PCG_BETA) {
            acc[0] += fcvt<double>(p.b) * fcvt<double>(o);
            acc[1] += p.ro * fcvt<double>(o);
        }
    }
    template <int NT>
    __device__ void reduce(double (&acc)[2]) const {
        if (FIN == FIN_PCG_BETA) {
            double tot[2];
            if (reduce_last<2, NT>(acc, part, cap, counter, tot) && threadIdx.x == 0)
                finish_pcg_beta(sc, tot);
        }
    }
};

// the outer FP64 products with their finishers (see k_spmv_fin)
template <int SF>
struct OpFin {
    DevScalars *sc;
    const double *x;
    double *y;
    const double *dvec;
    double *part;
    int cap;
    unsigned *counter;
    float *y32;  // true residual: FP32 copy of y (may be null)
    struct Pre {
        double d;
    };
    __device__ bool done() const { return SF != SF_TRUE_RES && sc->done != 0; }
    __device__ double gather(int j) const { return __ldg(x + j); }
    using GX = double;
    __device__ const GX *gsrc() const { return x; }
    __device__ Pre load(int i) const { return Pre{SF == SF_PCG_ALPHA ? __ldg(x + i) : __ldg(dvec + i)}; }
    static constexpr bool SELF = SF == SF_PCG_ALPHA;
    static constexpr int NROWV = 0, ROWV_BYTES = 0;
    __device__ Pre load_rest(int i) const { return SELF ? Pre{} : load(i); }
    __device__ void put_self(Pre &p, GX v) const {
        if (SELF) p.d = v;
    }
    __device__ void finish(int i, double s, const Pre &p, double (&acc)[2]) const {
        if (SF == SF_TRUE_RES) {
            const double ri = p.d - s;
            y[i] = ri;
            if (y32) y32[i] = f64_to_f32_rn(ri);
            acc[0] += ri * ri;
        } else {
            y[i] = s;
            if (SF == SF_BICG_OMEGA) {
                acc[0] += s * p.d;
                acc[1] += s * s;
            } else {
                acc[0] += p.d * s;
            }
        }
    }
    template <int NT>
    __device__ void reduce(double (&acc)[2]) const {
        double tot[2];
        if (reduce_last<2, NT>(acc, part, cap, counter, tot) && threadIdx.x == 0) finish_spmv<SF>(sc, tot);
    }
};

// q = A p in double-FP32 arithmetic with p.q -> alpha (the mixed form's
// outer product where the setup found it faster): A's values and the gathered
// p are FP32 pairs (p2, written with p), each row's sum is a double-FP32
// number converted to FP64 once, and q, p.q and alpha are FP64 as in OpFin.
struct OpFinDF {
    DevScalars *sc;
    const double *p;
    const DF *p2;
    double *y;
    double *part;
    int cap;
    unsigned *counter;
    struct Pre {
        double d;
    };
    __device__ bool done() const { return sc->done != 0; }
    __device__ DF gather(int j) const { return p2[j]; }
    using GX = DF;
    __device__ const GX *gsrc() const { return p2; }
    __device__ Pre load(int i) const { return Pre{__ldg(p + i)}; }
    static constexpr bool SELF = false;
    static constexpr int NROWV = 0, ROWV_BYTES = 0;
    __device__ Pre load_rest(int i) const { return load(i); }
    __device__ void put_self(Pre &, GX) const {}
    __device__ void finish(int i, DF s, const Pre &pr, double (&acc)[2]) const {
        const double q = df_value(s);
        y[i] = q;
        acc[0] += pr.d * q;
    }
    template <int NT>
    __device__ void reduce(double (&acc)[2]) const {
        double tot[2];
        if (reduce_last<2, NT>(acc, part, cap, counter, tot) && threadIdx.x == 0) finish_spmv<SF_PCG_ALPHA>(sc, tot);
    }
};

// Resident CTAs per SM of a windowed or sliced-ELL launch (two when they fit:
// the SM's 228 KB less about 11 KB of static and reserved memory per CTA).
static int ctas_per_sm(int smem) { return std::max(1, std::min(2, (228 * 1024) / (smem + 11 * 1024))); }

template <typename TM, int VEC, class Op, int NT>
static int stream_launch_nt(const StreamPlan &pl, int n, const int *rp, const int *ci, const TM *v, const Op &op,
                            int *err, cudaStream_t s) {
    if constexpr (NT == 512) {
        if (pl.c16) {
        using GX = typename Op::GX;
        const int smem = stream::smem_bytes_win<TM, GX, NT>(pl.rt, pl.cap, pl.xw, pl.stages);
        static int attr_set = 0;
        if (smem > attr_set) {
            AMG_CUDA_TRY(cudaFuncSetAttribute(stream::k_stream_win<TM, VEC, Op, NT>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            attr_set = smem;
        }
        const int per_sm = ctas_per_sm(smem);
        const int grid = std::max(1, std::min(pl.ntiles, per_sm * num_sms()));
        AMG_TRY(launch_k(stream::k_stream_win<TM, VEC, Op, NT>, grid, NT, smem, s, n, pl.rt, pl.cap, pl.xw, pl.ntiles, rp, pl.c16,
                                                                      v, pl.wtab, op, err, pl.stages));
        AMG_LAUNCH_CHECK();
        return AMG_OK;
        }
    }
    if (pl.rt % 16 != 0) {
        // the row-pointer bulk copies need tiles starting on 16-byte boundaries
        set_last_error("streaming pass: tile height %d is not a multiple of 16", pl.rt);
        return AMG_ERR_ARG;
    }
    const int smem = stream::smem_bytes<TM, NT>(pl.rt, pl.cap);
    static int attr_set = 0;  // largest dynamic shared memory enabled for this instantiation
    if (smem > attr_set) {
        AMG_CUDA_TRY(cudaFuncSetAttribute(stream::k_stream<TM, VEC, Op, NT>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr_set = smem;
    }
    // CTAs per SM that fit the SM's 228 KB of shared memory (1 KB reserved per CTA)
    const int per_sm = std::max(1, std::min(2, (228 * 1024) / (smem + 2048)));
    const int grid = std::max(1, std::min(pl.ntiles, per_sm * num_sms()));
    AMG_TRY(launch_k(stream::k_stream<TM, VEC, Op, NT>, grid, NT, smem, s, n, pl.rt, pl.cap, pl.ntiles, rp, ci, v, op, err));
    AMG_LAUNCH_CHECK();
    return AMG_OK;
}

template <typename TM, int VEC, class Op>
static int stream_launch_vec(const StreamPlan &pl, int n, const int *rp, const int *ci, const TM *v, const Op &op,
                             int *err, cudaStream_t s) {
    if constexpr (sizeof(TM) == 4) {
        if (pl.nt == 768) return stream_launch_nt<TM, VEC, Op, 768>(pl, n, rp, ci, v, op, err, s);
    }
    return stream_launch_nt<TM, VEC, Op, 512>(pl, n, rp, ci, v, op, err, s);
}

// The slot-order copy of CSR values v bound to sliced-ELL plan pl, or null.
static const void *ell_values(const StreamPlan &pl, const void *v) {
    for (int k = 0; k < pl.nev; ++k)
        if (pl.ev_src[k] == v) return pl.ev_dst[k];
    return nullptr;
}

template <typename TM, class Op>
static int stream_launch_ell(const StreamPlan &pl, int n, const TM *v, const Op &op, int *err, cudaStream_t s) {
    const TM *ev = static_cast<const TM *>(ell_values(pl, v));
    if (!ev) {
        set_last_error("streaming pass: the operator's values are not laid out for its sliced-ELL plan");
        return AMG_ERR_ARG;
    }
    using GX = typename Op::GX;
    // the epilogue's row operands are staged while as many CTAs per SM fit
    // as without them (and the stage stays within one CTA's 227 KB)
    int smem = stream::smem_bytes_ell<TM, GX>(pl.cap, pl.xw, pl.rt, 0, pl.stages);
    int rows = 0;
    if (Op::NROWV > 0) {
        const int with = stream::smem_bytes_ell<TM, GX>(pl.cap, pl.xw, pl.rt, Op::ROWV_BYTES, pl.stages);
        if (ctas_per_sm(with) == ctas_per_sm(smem) && with <= 227 * 1024 - 11 * 1024) {
            rows = 1;
            smem = with;
        }
    }
    static int attr_set = 0;
    if (smem > attr_set) {
        AMG_CUDA_TRY(cudaFuncSetAttribute(stream::k_stream_ell<TM, Op, 512>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr_set = smem;
    }
    const int per_sm = ctas_per_sm(smem);
    const int grid = std::max(1, std::min(pl.ntiles, per_sm * num_sms()));
    AMG_TRY(launch_k(stream::k_stream_ell<TM, Op, 512>, grid, 512, smem, s, n, pl.rt, pl.cap, pl.xw, pl.ntiles, pl.soff,
                     pl.ec, ev, pl.wtab, op, rows, err, pl.stages));
    AMG_LAUNCH_CHECK();
    return AMG_OK;
}

template <typename TM, class Op>
static int stream_launch_direct(const StreamPlan &pl, int n, const TM *v, const Op &op, cudaStream_t s) {
    const TM *ev = static_cast<const TM *>(ell_values(pl, v));
    if (!ev) {
        set_last_error("streaming pass: the operator's values are not laid out for its direct plan");
        return AMG_ERR_ARG;
    }
    constexpr int NT = stream::DIRECT_THREADS;
    // one wave of resident blocks (grid-stride over the slices), at most
    // num_sms() * 8: the reductions' partial sums hold that many
    auto wave = [](const void *fn) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, 0) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        return std::min(per_sm, 8) * num_sms();
    };
    const int need = (pl.ntiles + NT / 32 - 1) / (NT / 32);
    auto go = [&](auto kern, const auto *col, int &w) -> int {
        if (!w) w = wave((const void *)kern);
        AMG_TRY(launch_k(kern, std::max(1, std::min(need, w)), NT, 0, s, n, pl.ntiles, pl.soff, col, ev, op));
        return AMG_OK;
    };
    static int w16n = 0, w16w = 0, w32n = 0, w32w = 0;
    const bool wide = pl.maxw > 8;
    if (pl.dcol16 && !wide) AMG_TRY(go(stream::k_ell_direct<TM, int16_t, Op, false, NT>, pl.dcol16, w16n));
    else if (pl.dcol16) AMG_TRY(go(stream::k_ell_direct<TM, int16_t, Op, true, NT>, pl.dcol16, w16w));
    else if (!wide) AMG_TRY(go(stream::k_ell_direct<TM, int, Op, false, NT>, pl.dcol32, w32n));
    else AMG_TRY(go(stream::k_ell_direct<TM, int, Op, true, NT>, pl.dcol32, w32w));
    AMG_LAUNCH_CHECK();
    return AMG_OK;
}

// One streaming pass of a CSR operator whose plan is usable (pl.rt > 0).
template <typename TM, class Op>
static int stream_launch(const StreamPlan &pl, int n, const int *rp, const int *ci, const TM *v, const Op &op,
                         int *err, cudaStream_t s) {
    if (pl.direct) return stream_launch_direct<TM, Op>(pl, n, v, op, s);
    if (pl.ell) return stream_launch_ell<TM, Op>(pl, n, v, op, err, s);
    switch (pl.vec) {
        case 1: return stream_launch_vec<TM, 1, Op>(pl, n, rp, ci, v, op, err, s);
        case 2: return stream_launch_vec<TM, 2, Op>(pl, n, rp, ci, v, op, err, s);
        case 4: return stream_launch_vec<TM, 4, Op>(pl, n, rp, ci, v, op, err, s);
        case 8: return stream_launch_vec<TM, 8, Op>(pl, n, rp, ci, v, op, err, s);
        case 16: return stream_launch_vec<TM, 16, Op>(pl, n, rp, ci, v, op, err, s);
        default: return stream_launch_vec<TM, 32, Op>(pl, n, rp, ci, v, op, err, s);
    }
}

// Algorithmic bytes of a CSR operator pass: values + column indices + row pointers.
static double csr_bytes(const DevCSR &m, int vb) {
    return (double)m.nnz * (4.0 + vb) + 4.0 * ((double)m.nrows + 1.0);
}

// ---------------------------------------------------------------------------
// Autotuner: timed trial of streaming plans at setup
// ---------------------------------------------------------------------------

// Candidate tilings of one operator: rows per tile (multiples of 16, whole
// consumer passes when possible, capped so that there are at least four
// tiles per resident CTA) and threads per row (the mean-length choice and
// twice it).  Every candidate keeps each tile within cap - 8 stored entries.
static std::vector<StreamPlan> plan_candidates(const DevCSR &m, const StreamPlan &base, bool wide, cudaStream_t s) {
    std::vector<StreamPlan> out;
    if (base.rt == 0) return out;
    const int n = m.nrows;
    std::vector<int> rp((size_t)n + 1);
    if (cudaMemcpyAsync(rp.data(), m.rp, sizeof(int) * ((size_t)n + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        out.push_back(base);
        return out;
    }
    auto worst = [&](int rt) {
        int w = 0;
        for (int r0 = 0; r0 < n; r0 += rt) w = std::max(w, rp[std::min(r0 + rt, n)] - rp[r0]);
        return w;
    };
    const int resident = 2 * num_sms();
    std::vector<int> rts = {base.rt};
    int rt4 = (n / (4 * resident)) / 16 * 16;  // >= 4 tiles per resident CTA
    if (rt4 >= 16 && rt4 < base.rt) rts.push_back(rt4);
    if (base.rt / 2 >= 16) rts.push_back(base.rt / 2 / 16 * 16);
    for (int vec : {base.vec, base.vec * 2}) {
        if (vec > 32) continue;
        for (int rt : rts) {
            if (rt < 16 || worst(rt) > base.cap - 8) continue;
            StreamPlan p = base;
            p.rt = rt;
            p.vec = vec;
            p.ntiles = (n + rt - 1) / rt;
            bool dup = false;
            for (const StreamPlan &q : out) dup |= q.rt == p.rt && q.vec == p.vec && q.nt == p.nt;
            if (!dup) out.push_back(p);
        }
    }
    if (wide) {
        // 768-thread CTAs (23 consumer warps, two stages of 6144 entries):
        // tiles of one or two whole consumer passes
        for (int vec : {base.vec, base.vec * 2}) {
            if (vec > 32) continue;
            const int pass = 23 * 32 / vec;
            for (int rt : {pass, 2 * pass}) {
                // tiles start at multiples of 16 rows, so every bulk copy of
                // row pointers starts on a 16-byte boundary (23 * 32 / vec is
                // not a multiple of 16 for vec >= 4)
                if (rt % 16 != 0 || rt > stream::RT_MAX || worst(rt) > 6144 - 8) continue;
                StreamPlan p = base;
                p.nt = 768;
                p.cap = 6144;
                p.rt = rt;
                p.vec = vec;
                p.ntiles = (n + rt - 1) / rt;
                out.push_back(p);
            }
        }
    }
    return out;
}

// ---------------------------------------------------------------------------
// Windowed plans: per-tile windows of the gathered vector
// ---------------------------------------------------------------------------

constexpr int WIN_SPAN_CH = 16384;  // largest column span of a tile, in 4-element chunks
constexpr int WIN_GAP_CH = 8;       // runs of touched chunks closer than this share a window
constexpr int WIN_RUNS = 1024;      // most runs a tile may have before they are grouped

// One block per tile (grid-stride): the windows covering every column the
// tile touches -- the runs of touched 4-element chunks (runs closer than
// WIN_GAP_CH chunks joined), grouped into at most WIN_NW windows by breaking
// at the WIN_NW - 1 widest gaps -- and each entry's offset into them.  Tiles
// whose windows exceed xw_max elements (or that span too many columns or
// runs) set *bad.
__global__ void __launch_bounds__(256) k_tile_windows(int n, int rt, int ntiles, const int *__restrict__ rp,
                                                      const int *__restrict__ ci, int xw_max, int *wtab,
                                                      uint16_t *c16, int *bad, int *xw_used) {
    constexpr int NW = stream::WIN_NW;
    __shared__ unsigned char ch[WIN_SPAN_CH];
    __shared__ int rs[WIN_RUNS], re[WIN_RUNS], gap[WIN_RUNS];
    __shared__ int s_min, s_max, s_ok, s_nr, s_nw;
    __shared__ int s_ws[NW], s_wl[NW], s_off[NW];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int r0 = t * rt, r1 = min(r0 + rt, n);
        const int s = rp[r0], e = rp[r1];
        if (threadIdx.x == 0) {
            s_min = INT_MAX;
            s_max = -1;
            s_ok = 1;
            s_nr = 0;
            s_nw = 0;
        }
        __syncthreads();
        int lmin = INT_MAX, lmax = -1;
        for (int k = s + threadIdx.x; k < e; k += blockDim.x) {
            const int c = ci[k];
            lmin = min(lmin, c);
            lmax = max(lmax, c);
        }
        atomicMin(&s_min, lmin);
        atomicMax(&s_max, lmax);
        __syncthreads();
        const int base = s_max >= 0 ? (s_min & ~3) : 0;
        const int nch = s_max >= 0 ? ((s_max - base) >> 2) + 1 : 0;
        if (nch <= WIN_SPAN_CH) {
            for (int q = threadIdx.x; q < nch; q += blockDim.x) ch[q] = 0;
            __syncthreads();
            for (int k = s + threadIdx.x; k < e; k += blockDim.x) ch[(ci[k] - base) >> 2] = 1;
            __syncthreads();
            if (threadIdx.x < 32) {
                // warp 0 lists the runs in order (every lane keeps the same state)
                int nr = 0, ws = -1, we = -1;
                for (int q0 = 0; q0 < nch; q0 += 32) {
                    const int q = q0 + threadIdx.x;
                    unsigned msk = __ballot_sync(0xffffffffu, q < nch && ch[q]);
                    while (msk) {
                        const int c = q0 + __ffs(msk) - 1;
                        msk &= msk - 1;
                        if (ws >= 0 && c - we < WIN_GAP_CH) {
                            we = c + 1;
                        } else {
                            if (ws >= 0) {
                                if (nr < WIN_RUNS && threadIdx.x == 0) {
                                    rs[nr] = ws;
                                    re[nr] = we;
                                }
                                ++nr;
                            }
                            ws = c;
                            we = c + 1;
                        }
                    }
                }
                if (ws >= 0) {
                    if (nr < WIN_RUNS && threadIdx.x == 0) {
                        rs[nr] = ws;
                        re[nr] = we;
                    }
                    ++nr;
                }
                if (threadIdx.x == 0) {
                    s_nr = nr;
                    if (nr > WIN_RUNS) s_ok = 0;
                }
            }
        } else if (threadIdx.x == 0) {
            s_ok = 0;
        }
        __syncthreads();
        const int nr = s_nr;
        if (s_ok && nr > NW) {
            // break at the NW - 1 widest gaps (the narrowest index on ties):
            // gap[i] between runs i and i+1, marked -1 once chosen
            for (int i = threadIdx.x; i < nr - 1; i += blockDim.x) gap[i] = rs[i + 1] - re[i];
            __syncthreads();
            if (threadIdx.x < 32) {
                for (int pick = 0; pick < NW - 1; ++pick) {
                    int best = -1, bi = -1;
                    for (int i = threadIdx.x; i < nr - 1; i += 32)
                        if (gap[i] > best) {
                            best = gap[i];
                            bi = i;
                        }
                    for (int o = 16; o > 0; o >>= 1) {
                        const int ob = __shfl_xor_sync(0xffffffffu, best, o), oi = __shfl_xor_sync(0xffffffffu, bi, o);
                        if (ob > best || (ob == best && oi >= 0 && (bi < 0 || oi < bi))) {
                            best = ob;
                            bi = oi;
                        }
                    }
                    if (threadIdx.x == 0 && bi >= 0) gap[bi] = -1;
                    __syncwarp();
                }
            }
            __syncthreads();
        }
        if (s_ok && threadIdx.x == 0) {
            int nw = 0, tot = 0, ws = nr > 0 ? rs[0] : 0;
            for (int i = 0; i < nr; ++i) {
                const bool last = i == nr - 1;
                const bool brk = last || nr <= NW || gap[i] < 0;
                if (brk) {
                    s_ws[nw] = base + 4 * ws;
                    s_wl[nw] = 4 * (re[i] - ws);
                    s_off[nw] = tot;
                    tot += 4 * (re[i] - ws);
                    ++nw;
                    if (!last) ws = rs[i + 1];
                }
            }
            s_nw = nw;
            if (tot > xw_max) s_ok = 0;
            else atomicMax(xw_used, tot);
        }
        __syncthreads();
        if (!s_ok) {
            if (threadIdx.x == 0) atomicExch(bad, 1);
        } else {
            const int nw = s_nw;
            if (threadIdx.x < 2 * NW) {
                const int w = threadIdx.x >> 1;
                wtab[(size_t)t * 2 * NW + threadIdx.x] = w < nw ? ((threadIdx.x & 1) ? s_wl[w] : s_ws[w]) : 0;
            }
            for (int k = s + threadIdx.x; k < e; k += blockDim.x) {
                const int c = ci[k];
                int w = 0;
                while (w + 1 < nw && c >= s_ws[w + 1]) ++w;
                c16[k] = (uint16_t)(s_off[w] + (c - s_ws[w]));
            }
        }
        __syncthreads();
    }
}

// Turns plan p (512 threads) into a windowed plan for operator m: tightens
// the stage capacity to the tiles' entries, budgets the windows for FP64
// gathers at two CTAs per SM, and builds the window table and local indices
// in `scr`.  Returns false when some tile does not fit.
template <typename TM>
static bool build_windows(const DevCSR &m, StreamPlan &p, int worst_tile, int gx_bytes, Scratch &scr, cudaStream_t s) {
    p.cap = (worst_tile + 8 + 255) / 256 * 256;
    const stream::WLayout<TM, double> lay(p.rt, p.cap, 0);
    // two CTAs per SM: 228 KB less 1 KB reserved per CTA and the descriptors'
    // static shared memory (about 9 KB)
    const int per_cta = (228 * 1024) / 2 - 1024 - 10 * 1024;
    const int budget = per_cta / stream::WIN_STAGES - lay.stb;
    const int xw_max = std::min(65532, budget / gx_bytes / 4 * 4);
    if (xw_max < 64) return false;
    int *wtab = nullptr, *bad = nullptr, *used = nullptr;
    uint16_t *c16 = nullptr;
    if (scr.alloc(&wtab, (size_t)p.ntiles * 2 * stream::WIN_NW) < 0 || scr.alloc(&c16, (size_t)std::max(1LL, m.nnz)) < 0 ||
        scr.alloc(&bad, 2) < 0) {
        cudaGetLastError();
        return false;
    }
    used = bad + 1;
    if (cudaMemsetAsync(bad, 0, 2 * sizeof(int), s) != cudaSuccess) return false;
    k_tile_windows<<<std::min(p.ntiles, 8 * num_sms()), 256, 0, s>>>(m.nrows, p.rt, p.ntiles, m.rp, m.ci, xw_max, wtab,
                                                                       c16, bad, used);
    int h[2] = {1, 0};
    if (cudaMemcpyAsync(h, bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (h[0]) return false;
    p.xw = std::max(4, h[1]);
    p.wtab = wtab;
    p.c16 = c16;
    return true;
}

// ---------------------------------------------------------------------------
// Sliced-ELL plans (stream::k_stream_ell)
// ---------------------------------------------------------------------------

// The width (longest row) of each 32-row slice.
__global__ void k_ell_width(int n, int nsl, const int *__restrict__ rp, int *wd) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nsl) return;
    const int r0 = g * 32, r1 = min(r0 + 32, n);
    int w = 0;
    for (int r = r0; r < r1; ++r) w = max(w, rp[r + 1] - rp[r]);
    wd[g] = w;
}

// One thread per slice row: its local indices in slot order and the stored
// entry each slot holds; padding slots (-1) repeat the row's first index (0
// for an empty row, whose tile still has a window if the slice has a slot).
__global__ void k_ell_fill(int n, int nsl, const int *__restrict__ rp, const uint16_t *__restrict__ c16,
                           const int *__restrict__ soff, int *eperm, uint16_t *ec) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (long long)nsl * 32) return;
    const int g = (int)(r >> 5), lane = (int)(r & 31);
    const int s0 = soff[g], wd = (soff[g + 1] - s0) >> 5;
    const int b = r < n ? rp[r] : 0, len = r < n ? rp[r + 1] - b : 0;
    const uint16_t pad = len > 0 ? c16[b] : (uint16_t)0;
    for (int u = 0; u < wd; ++u) {
        const int pos = s0 + u * 32 + lane;
        eperm[pos] = u < len ? b + u : -1;
        ec[pos] = u < len ? c16[b + u] : pad;
    }
}

// One thread per slice row of a direct sliced-ELL plan: the stored entry each
// slot holds (-1: padding) and its column, as an offset from the row (col16;
// *bad is set when an offset does not fit 16 bits) or absolute (col32).
// Padding slots take the row's first column, or column min(r, ncols - 1) for
// an empty row and the rows past n, so every slot's column is valid.
__global__ void k_direct_fill(int n, int ncols, int nsl, const int *__restrict__ rp, const int *__restrict__ ci,
                              const int *__restrict__ soff, int *eperm, int16_t *col16, int *col32, int *bad) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (long long)nsl * 32) return;
    const int g = (int)(r >> 5), lane = (int)(r & 31);
    const int s0 = soff[g], wd = (soff[g + 1] - s0) >> 5;
    const int b = r < n ? rp[r] : 0, len = r < n ? rp[r + 1] - b : 0;
    const int pad = len > 0 ? ci[b] : (int)min(r, (long long)ncols - 1);
    for (int u = 0; u < wd; ++u) {
        const int pos = s0 + u * 32 + lane;
        const int c = u < len ? ci[b + u] : pad;
        eperm[pos] = u < len ? b + u : -1;
        if (col16) {
            const long long d = (long long)c - r;
            if (d < -32768 || d > 32767) atomicExch(bad, 1);
            else col16[pos] = (int16_t)d;
        } else {
            col32[pos] = c;
        }
    }
}

// dst = the values of src in slot order (zero in padding slots).
template <typename T>
__global__ void k_ell_vals(long long ne, const int *__restrict__ eperm, const T *__restrict__ src, T *dst) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < ne; k += (long long)gridDim.x * blockDim.x) {
        const int e = eperm[k];
        dst[k] = e >= 0 ? src[e] : T(0);
    }
}

static int ell_lay_out(const StreamPlan &pl, const void *src, void *dst, int vbytes, cudaStream_t s) {
    if (pl.ne == 0) return AMG_OK;
    const int grid = (int)std::min<long long>((pl.ne + 255) / 256, 16LL * num_sms());
    if (vbytes == 4)
        k_ell_vals<float><<<grid, 256, 0, s>>>(pl.ne, pl.eperm, static_cast<const float *>(src), static_cast<float *>(dst));
    else
        k_ell_vals<double><<<grid, 256, 0, s>>>(pl.ne, pl.eperm, static_cast<const double *>(src),
                                                static_cast<double *>(dst));
    AMG_LAUNCH_CHECK();
    return AMG_OK;
}

// Turns windowed plan p (local indices c16 built for its tiles; rt a multiple
// of 32) into a sliced-ELL plan with its tables in `scr`.  Returns false when
// the padded tiles do not fit two CTAs per SM or the entry count overflows.
template <typename TM>
static bool build_ell(const DevCSR &m, StreamPlan &p, int gx_bytes, Scratch &scr, cudaStream_t s) {
    const int n = m.nrows, nsl = (n + 31) / 32, spt = p.rt / 32;
    int *wd = nullptr, *soff = nullptr;
    if (p.rt % 32 != 0 || !p.c16 || scr.alloc(&wd, (size_t)nsl) < 0 || scr.alloc(&soff, (size_t)nsl + 1) < 0) {
        cudaGetLastError();
        return false;
    }
    k_ell_width<<<(nsl + 255) / 256, 256, 0, s>>>(n, nsl, m.rp, wd);
    std::vector<int> w((size_t)nsl), so((size_t)nsl + 1);
    if (cudaMemcpyAsync(w.data(), wd, sizeof(int) * (size_t)nsl, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    long long tot = 0;
    for (int g = 0; g < nsl; ++g) {
        so[g] = (int)tot;
        tot += 32LL * w[g];
        if (tot > INT_MAX - 64) return false;
    }
    so[nsl] = (int)tot;
    int worst = 0;
    for (int g0 = 0; g0 < nsl; g0 += spt) worst = std::max(worst, so[std::min(g0 + spt, nsl)] - so[g0]);
    const int cap = std::max(64, (worst + 63) / 64 * 64);
    // two CTAs per SM: 228 KB less 1 KB reserved per CTA and the descriptors'
    // static shared memory (about 9 KB)
    const int per_cta = (228 * 1024) / 2 - 1024 - 10 * 1024;
    const int stage = stream::align16(cap * (int)sizeof(TM)) + stream::align16(cap * 2) +
                      stream::align16(p.xw * gx_bytes) + 16;
    if (stream::WIN_STAGES * stage > per_cta) return false;
    int *eperm = nullptr;
    uint16_t *ec = nullptr;
    if (scr.alloc(&eperm, (size_t)std::max(1LL, tot)) < 0 || scr.alloc(&ec, (size_t)std::max(1LL, tot)) < 0) {
        cudaGetLastError();
        return false;
    }
    if (cudaMemcpyAsync(soff, so.data(), sizeof(int) * so.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const long long rows = (long long)nsl * 32;
    k_ell_fill<<<(int)((rows + 255) / 256), 256, 0, s>>>(n, nsl, m.rp, p.c16, soff, eperm, ec);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    p.ell = 1;
    p.ne = tot;
    p.soff = soff;
    p.ec = ec;
    p.eperm = eperm;
    p.cap = cap;
    p.c16 = nullptr;
    p.vec = 1;
    p.nt = 512;
    return true;
}

// A direct sliced-ELL plan for operator m (the slot-major layout of 32-row
// slices, read with plain loads): slice offsets, the slot-to-entry map and
// the columns -- 16-bit offsets from the row when use16 (square operators,
// every offset within 16 bits), else absolute -- in `scr`.  Returns false
// when the offsets do not fit or the slot count overflows.
static bool build_direct(const DevCSR &m, StreamPlan &p, bool use16, Scratch &scr, cudaStream_t s) {
    const int n = m.nrows, nsl = (n + 31) / 32;
    if (use16 && m.ncols != m.nrows) return false;
    int *wd = nullptr, *soff = nullptr, *bad = nullptr, *eperm = nullptr, *c32 = nullptr;
    int16_t *c16 = nullptr;
    if (scr.alloc(&wd, (size_t)nsl) < 0 || scr.alloc(&soff, (size_t)nsl + 1) < 0 || scr.alloc(&bad, 1) < 0) {
        cudaGetLastError();
        return false;
    }
    k_ell_width<<<(nsl + 255) / 256, 256, 0, s>>>(n, nsl, m.rp, wd);
    std::vector<int> w((size_t)nsl), so((size_t)nsl + 1);
    if (cudaMemcpyAsync(w.data(), wd, sizeof(int) * (size_t)nsl, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    long long tot = 0;
    int maxw = 0;
    for (int g = 0; g < nsl; ++g) {
        so[g] = (int)tot;
        tot += 32LL * w[g];
        maxw = std::max(maxw, w[g]);
        if (tot > INT_MAX - 64) return false;
    }
    so[nsl] = (int)tot;
    const size_t ne = (size_t)std::max(1LL, tot);
    if (scr.alloc(&eperm, ne) < 0 || (use16 ? scr.alloc(&c16, ne) : scr.alloc(&c32, ne)) < 0) {
        cudaGetLastError();
        return false;
    }
    if (cudaMemcpyAsync(soff, so.data(), sizeof(int) * so.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const long long rows = (long long)nsl * 32;
    k_direct_fill<<<(int)((rows + 255) / 256), 256, 0, s>>>(n, m.ncols, nsl, m.rp, m.ci, soff, eperm, c16, c32, bad);
    int hbad = 1;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (hbad) return false;
    p = StreamPlan();
    p.direct = 1;
    p.maxw = maxw;
    p.rt = 32;
    p.vec = 1;
    p.nt = stream::DIRECT_THREADS;
    p.ntiles = nsl;
    p.ne = tot;
    p.soff = soff;
    p.eperm = eperm;
    p.dcol16 = c16;
    p.dcol32 = c32;
    return true;
}

// tune_plan's layout restriction for the tile family: every layout but the
// direct one (AMG_LAYOUT_AUTO admits all of them)
constexpr int LAYOUT_TILES = -1;

// What a plan is timed with: the pass it serves, epilogue included, on
// scratch vectors (y = M x for passes without an epilogue of their own).
enum TuneKind { TUNE_SPMV, TUNE_PRE, TUNE_POST0, TUNE_POST, TUNE_PROLONG, TUNE_ALPHA };

template <typename T>
__global__ void k_fill(size_t n, T v, T *out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) out[i] = v;
}

// Times y = M x with each candidate (the best of three trials of ten launches,
// after one warm-up) and keeps the fastest plan.  x and y are scratch vectors
// of the operator's sizes.
template <typename TM, typename TG>
static int tune_plan(const DevCSR &m, const TM *vals, StreamPlan &pl, DevArena &ar, int layout, TuneKind kind,
                     cudaStream_t s) {
    const int gx_bytes = sizeof(TG);
    std::vector<StreamPlan> cands = plan_candidates(m, pl, sizeof(TM) == 4, s);
    Scratch scr;
    // windowed variants of the 512-thread candidates
    const bool tiles = layout != AMG_LAYOUT_ELL_DIRECT;
    if (pl.rt > 0) {
        std::vector<int> rp((size_t)m.nrows + 1);
        AMG_CUDA_TRY(cudaMemcpy(rp.data(), m.rp, sizeof(int) * rp.size(), cudaMemcpyDeviceToHost));
        const size_t nbase = cands.size();
        for (size_t q = 0; q < nbase && tiles; ++q) {
            if (cands[q].nt != 512) continue;
            StreamPlan w = cands[q];
            int worst = 0;
            for (int r0 = 0; r0 < m.nrows; r0 += w.rt) worst = std::max(worst, rp[std::min(r0 + w.rt, m.nrows)] - rp[r0]);
            if (build_windows<TM>(m, w, worst, gx_bytes, scr, s)) cands.push_back(w);
        }
        // sliced-ELL variants: tiles of one or two passes of the 15 consumer
        // warps (a slice each), and of 7 slices for small operators
        for (int rt : {480, 960, 224}) {
            if (!tiles || (long long)m.nrows < 2LL * rt) continue;
            StreamPlan w;
            w.rt = rt;
            w.vec = 1;
            w.nt = 512;
            w.ntiles = (m.nrows + rt - 1) / rt;
            int worst = 0;
            for (int r0 = 0; r0 < m.nrows; r0 += rt) worst = std::max(worst, rp[std::min(r0 + rt, m.nrows)] - rp[r0]);
            if (worst + 8 > 65536 || !build_windows<TM>(m, w, worst, gx_bytes, scr, s) ||
                !build_ell<TM>(m, w, gx_bytes, scr, s))
                continue;
            TM *ev = nullptr;
            if (scr.alloc(&ev, (size_t)std::max(1LL, w.ne)) < 0) {
                cudaGetLastError();
                continue;
            }
            if (ell_lay_out(w, vals, ev, (int)sizeof(TM), s) < 0) continue;
            w.nev = 1;
            w.ev_src[0] = vals;
            w.ev_dst[0] = ev;
            w.ev_bytes[0] = (int)sizeof(TM);
            cands.push_back(w);
        }
        // the direct sliced-ELL layout: 16-bit column offsets where they fit,
        // else absolute columns
        for (bool use16 : {true, false}) {
            if (layout == LAYOUT_TILES) break;
            StreamPlan d;
            if (!build_direct(m, d, use16, scr, s)) continue;
            TM *ev = nullptr;
            if (scr.alloc(&ev, (size_t)std::max(1LL, d.ne)) < 0) {
                cudaGetLastError();
                break;
            }
            if (ell_lay_out(d, vals, ev, (int)sizeof(TM), s) < 0) break;
            d.nev = 1;
            d.ev_src[0] = vals;
            d.ev_dst[0] = ev;
            d.ev_bytes[0] = (int)sizeof(TM);
            cands.push_back(d);
            break;
        }
        // the same tiles with a deeper ring: 3 and 4 stages, at two CTAs per
        // SM where they still fit, else at one (more bytes in flight per SM).
        // Sized for FP64 gathers, the widest any pass of the plan makes (the
        // finest level's pre-smoothing reads an FP64 input when no FP32 copy
        // is given), so every launch stays within one CTA's shared memory.
        const size_t nring = cands.size();
        for (size_t q = 0; q < nring; ++q) {
            if (!cands[q].c16 && !cands[q].ell) continue;
            for (int st : {3, 4}) {
                StreamPlan d = cands[q];
                d.stages = st;
                const int smem = d.ell ? stream::smem_bytes_ell<TM, double>(d.cap, d.xw, d.rt, 0, st)
                                       : stream::smem_bytes_win<TM, double>(d.rt, d.cap, d.xw, st);
                if (smem <= 216 * 1024) cands.push_back(d);
            }
        }
    }
    if (layout != AMG_LAYOUT_AUTO) {
        // only the requested layout (LAYOUT_TILES: every tile layout), the
        // heuristic CSR plan when none fits
        auto kind = [](const StreamPlan &p) {
            return p.direct ? AMG_LAYOUT_ELL_DIRECT
                   : p.ell  ? AMG_LAYOUT_SLICED_ELL
                   : p.c16  ? AMG_LAYOUT_WINDOWED
                            : AMG_LAYOUT_CSR;
        };
        std::vector<StreamPlan> keep;
        for (const StreamPlan &c : cands)
            if (layout == LAYOUT_TILES ? kind(c) != AMG_LAYOUT_ELL_DIRECT : kind(c) == layout) keep.push_back(c);
        if (keep.empty() && !cands.empty()) keep.push_back(cands[0]);
        cands.swap(keep);
    }
    if (cands.empty()) return AMG_OK;
    if (cands.size() == 1 && !cands[0].ell && !cands[0].c16 && !cands[0].direct) {
        pl = cands[0];
        return AMG_OK;
    }
    // scratch operands: the gathered vector, weights, right-hand sides and
    // r_old set to constants (ones and halves keep every dot product finite,
    // and p.Ap = sum_ij a_ij > 0 for the M-matrices of diffusion problems),
    // outputs, and the reductions' partial sums and scalars of their own
    const size_t nr = (size_t)m.nrows, ncl = (size_t)m.ncols;
    const int cap = num_sms() * 8;
    TG *x = nullptr;
    TM *w = nullptr, *bm = nullptr;
    double *y = nullptr, *bd = nullptr, *ro = nullptr, *part = nullptr;
    unsigned *cnt = nullptr;
    DevScalars *tsc = nullptr;
    int *err = nullptr;
    AMG_TRY(scr.alloc(&x, ncl));
    AMG_TRY(scr.alloc(&y, std::max(nr, ncl)));
    AMG_TRY(scr.alloc(&w, nr));
    AMG_TRY(scr.alloc(&bm, nr));
    AMG_TRY(scr.alloc(&bd, nr));
    AMG_TRY(scr.alloc(&ro, nr));
    AMG_TRY(scr.alloc(&part, (size_t)3 * cap));
    AMG_TRY(scr.alloc(&cnt, 4));
    AMG_TRY(scr.alloc(&tsc, 1));
    AMG_TRY(scr.alloc(&err, 2));  // the error flag and the (unarmed) test control after it
    k_fill<TG><<<256, 256, 0, s>>>(ncl, (TG)1, x);
    k_fill<TM><<<256, 256, 0, s>>>(nr, (TM)0.5, w);
    k_fill<TM><<<256, 256, 0, s>>>(nr, (TM)1, bm);
    k_fill<double><<<256, 256, 0, s>>>(nr, 1.0, bd);
    k_fill<double><<<256, 256, 0, s>>>(nr, 0.5, ro);
    AMG_LAUNCH_CHECK();
    AMG_CUDA_TRY(cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned), s));
    AMG_CUDA_TRY(cudaMemsetAsync(err, 0, 2 * sizeof(int), s));
    constexpr bool same = std::is_same<TM, TG>::value;
    const TM *xm = reinterpret_cast<const TM *>(x);  // the gathered vector as TM (kinds with TG = TM)
    TM *ym = reinterpret_cast<TM *>(y);
    auto launch = [&](const StreamPlan &c) -> int {
        if constexpr (same) {
            if (kind == TUNE_POST0)
                return stream_launch<TM>(c, m.nrows, m.rp, m.ci, vals,
                                         OpPost<double, TM, double, FIN_PCG_BETA>{tsc, w, bd, xm, y, ro, part, cap, cnt},
                                         err, s);
            if (kind == TUNE_POST)
                return stream_launch<TM>(c, m.nrows, m.rp, m.ci, vals,
                                         OpPost<TM, TM, TM, FIN_NONE>{tsc, w, bm, xm, ym, nullptr, part, cap, cnt}, err, s);
            if (kind == TUNE_PROLONG)
                return stream_launch<TM>(c, m.nrows, m.rp, m.ci, vals, OpProlong<TM, TM>{&tsc->done, w, bm, xm, ym},
                                         err, s);
            if constexpr (std::is_same<TM, double>::value)
                if (kind == TUNE_ALPHA)
                    return stream_launch<TM>(c, m.nrows, m.rp, m.ci, vals,
                                             OpFin<SF_PCG_ALPHA>{tsc, x, y, nullptr, part, cap, cnt, nullptr}, err, s);
        }
        if (kind == TUNE_PRE)
            return stream_launch<TM>(c, m.nrows, m.rp, m.ci, vals, OpPre<TG, TM>{&tsc->done, x, ym}, err, s);
        return stream_launch<TM>(c, m.nrows, m.rp, m.ci, vals, OpTune<TM, TG>{&tsc->done, x, ym}, err, s);
    };
    cudaEvent_t e0, e1;
    AMG_CUDA_TRY(cudaEventCreate(&e0));
    AMG_CUDA_TRY(cudaEventCreate(&e1));
    // Among the candidates within 3 % of the fastest (the trials' noise), the
    // first by layout -- sliced-ELL, windowed, CSR -- then by candidate order
    // is kept, so near-ties resolve the same way in every run.  A pass whose
    // finisher stops the scalars (a p.Ap <= 0 on these operands) is timed as
    // y = M x instead.
    std::vector<float> times(cands.size(), 1e30f);
    StreamPlan chosen = pl;
    int rc = AMG_OK;
    for (int pass = 0; pass < 2 && rc >= 0; ++pass) {
        bool stopped_any = false;
        for (size_t ci_ = 0; ci_ < cands.size() && !stopped_any; ++ci_) {
            const StreamPlan &c = cands[ci_];
            if ((rc = cudaMemsetAsync(tsc, 0, sizeof(DevScalars), s) == cudaSuccess ? AMG_OK : AMG_ERR_CUDA) < 0) break;
            if ((rc = launch(c)) < 0) break;
            // best of three trials of ten launches
            float ms = 1e30f;
            for (int trial = 0; trial < 3 && rc >= 0; ++trial) {
                cudaEventRecord(e0, s);
                for (int r = 0; r < 10; ++r)
                    if ((rc = launch(c)) < 0) break;
                cudaEventRecord(e1, s);
                if (rc < 0 || cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = rc < 0 ? rc : AMG_ERR_CUDA;
                    break;
                }
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                ms = std::min(ms, t);
            }
            if (rc < 0) break;
            int stopped = 0;
            if (cudaMemcpy(&stopped, &tsc->done, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
                rc = AMG_ERR_CUDA;
                break;
            }
            stopped_any = stopped != 0;
            times[ci_] = ms;
        }
        if (rc < 0 || !stopped_any || kind == TUNE_SPMV) break;
        kind = TUNE_SPMV;  // time every candidate again as y = M x
    }
    if (rc >= 0) {
        const float fastest = *std::min_element(times.begin(), times.end());
        auto rank = [](const StreamPlan &p) { return p.ell ? 0 : p.direct ? 1 : p.c16 ? 2 : 3; };
        int pick = -1;
        for (size_t q = 0; q < cands.size(); ++q)
            if (times[q] <= 1.03f * fastest && (pick < 0 || rank(cands[q]) < rank(cands[pick]))) pick = (int)q;
        if (pick >= 0) chosen = cands[pick];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (rc < 0) return rc;
    if (chosen.ell) {
        // keep the chosen tables (the candidates live in scratch memory); the
        // value arrays are laid out for the plan by ell_bind
        const int nsl = (m.nrows + 31) / 32;
        int *wtab = nullptr, *soff = nullptr, *eperm = nullptr;
        uint16_t *ec = nullptr;
        const size_t ne = (size_t)std::max(1LL, chosen.ne);
        AMG_TRY(ar.alloc(&wtab, (size_t)chosen.ntiles * 2 * stream::WIN_NW));
        AMG_TRY(ar.alloc(&soff, (size_t)nsl + 1));
        AMG_TRY(ar.alloc(&eperm, ne));
        AMG_TRY(ar.alloc(&ec, ne));
        AMG_CUDA_TRY(cudaMemcpyAsync(wtab, chosen.wtab, sizeof(int) * (size_t)chosen.ntiles * 2 * stream::WIN_NW,
                                     cudaMemcpyDeviceToDevice, s));
        AMG_CUDA_TRY(cudaMemcpyAsync(soff, chosen.soff, sizeof(int) * ((size_t)nsl + 1), cudaMemcpyDeviceToDevice, s));
        AMG_CUDA_TRY(cudaMemcpyAsync(eperm, chosen.eperm, sizeof(int) * ne, cudaMemcpyDeviceToDevice, s));
        AMG_CUDA_TRY(cudaMemcpyAsync(ec, chosen.ec, sizeof(uint16_t) * ne, cudaMemcpyDeviceToDevice, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        chosen.wtab = wtab;
        chosen.soff = soff;
        chosen.eperm = eperm;
        chosen.ec = ec;
        chosen.nev = 0;
    } else if (chosen.direct) {
        // keep the chosen slice tables (the candidates live in scratch memory)
        const int nsl = (m.nrows + 31) / 32;
        const size_t ne = (size_t)std::max(1LL, chosen.ne);
        int *soff = nullptr, *eperm = nullptr, *c32 = nullptr;
        int16_t *c16 = nullptr;
        AMG_TRY(ar.alloc(&soff, (size_t)nsl + 1));
        AMG_TRY(ar.alloc(&eperm, ne));
        AMG_CUDA_TRY(cudaMemcpyAsync(soff, chosen.soff, sizeof(int) * ((size_t)nsl + 1), cudaMemcpyDeviceToDevice, s));
        AMG_CUDA_TRY(cudaMemcpyAsync(eperm, chosen.eperm, sizeof(int) * ne, cudaMemcpyDeviceToDevice, s));
        if (chosen.dcol16) {
            AMG_TRY(ar.alloc(&c16, ne));
            AMG_CUDA_TRY(cudaMemcpyAsync(c16, chosen.dcol16, sizeof(int16_t) * ne, cudaMemcpyDeviceToDevice, s));
        } else {
            AMG_TRY(ar.alloc(&c32, ne));
            AMG_CUDA_TRY(cudaMemcpyAsync(c32, chosen.dcol32, sizeof(int) * ne, cudaMemcpyDeviceToDevice, s));
        }
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        chosen.soff = soff;
        chosen.eperm = eperm;
        chosen.dcol16 = c16;
        chosen.dcol32 = c32;
        chosen.nev = 0;
    } else if (chosen.c16) {
        // keep the chosen windows (the candidates live in scratch memory)
        int *wtab = nullptr;
        uint16_t *c16 = nullptr;
        AMG_TRY(ar.alloc(&wtab, (size_t)chosen.ntiles * 2 * stream::WIN_NW));
        AMG_TRY(ar.alloc(&c16, (size_t)std::max(1LL, m.nnz)));
        AMG_CUDA_TRY(cudaMemcpyAsync(wtab, chosen.wtab, sizeof(int) * (size_t)chosen.ntiles * 2 * stream::WIN_NW,
                                     cudaMemcpyDeviceToDevice, s));
        AMG_CUDA_TRY(cudaMemcpyAsync(c16, chosen.c16, sizeof(uint16_t) * (size_t)m.nnz, cudaMemcpyDeviceToDevice, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        chosen.wtab = wtab;
        chosen.c16 = c16;
    }
    pl = chosen;
    return AMG_OK;
}

template <class F>
static void for_each_plan(Hierarchy *h, F f) {
    for (int l = 0; l < h->nlevels; ++l) {
        Level &lv = h->L[l];
        for (StreamPlan *p : {&lv.sa, &lv.sa_post, &lv.sp, &lv.sr, &lv.sa64}) f(*p);
    }
}

// Lays out, in the hierarchy's arena, CSR values src for sliced-ELL plan pl
// (nothing for other plans); plans of one layout (the same slice offsets)
// share a copy.
static int ell_bind_one(Hierarchy *h, StreamPlan &pl, const void *src, int vbytes, cudaStream_t s) {
    if (!(pl.ell || pl.direct) || !src || ell_values(pl, src)) return AMG_OK;
    if (pl.nev == StreamPlan::EV_MAX) {
        set_last_error("sliced-ELL plan: more than %d value arrays", StreamPlan::EV_MAX);
        return AMG_ERR_ARG;
    }
    void *dst = nullptr;
    for_each_plan(h, [&](StreamPlan &q) {
        if (!dst && (q.ell || q.direct) && q.soff == pl.soff) dst = const_cast<void *>(ell_values(q, src));
    });
    if (!dst) {
        const size_t ne = (size_t)std::max(1LL, pl.ne);
        if (vbytes == 4) {
            float *d = nullptr;
            AMG_TRY(h->arena.alloc(&d, ne));
            dst = d;
        } else {
            double *d = nullptr;
            AMG_TRY(h->arena.alloc(&d, ne));
            dst = d;
        }
        AMG_TRY(ell_lay_out(pl, src, dst, vbytes, s));
    }
    pl.ev_src[pl.nev] = src;
    pl.ev_dst[pl.nev] = dst;
    pl.ev_bytes[pl.nev] = vbytes;
    ++pl.nev;
    return AMG_OK;
}

// Binds every sliced-ELL plan to the value arrays the solve launches it with.
static int ell_bind(Hierarchy *h, cudaStream_t s) {
    const bool mixed = h->cfg.precision == AMG_PRECISION_MIXED;
    for (int l = 0; l < h->nlevels; ++l) {
        Level &lv = h->L[l];
        if (mixed) {
            AMG_TRY(ell_bind_one(h, lv.sa, lv.ahat32, 4, s));
            AMG_TRY(ell_bind_one(h, lv.sa_post, lv.A.v32, 4, s));
            AMG_TRY(ell_bind_one(h, lv.sp, lv.P.v32, 4, s));
            AMG_TRY(ell_bind_one(h, lv.sr, lv.R.v32, 4, s));
        } else {
            AMG_TRY(ell_bind_one(h, lv.sa, lv.ahat, 8, s));
            AMG_TRY(ell_bind_one(h, lv.sa_post, lv.A.v, 8, s));
            AMG_TRY(ell_bind_one(h, lv.sp, lv.P.v, 8, s));
            AMG_TRY(ell_bind_one(h, lv.sr, lv.R.v, 8, s));
        }
    }
    AMG_TRY(ell_bind_one(h, h->L[0].sa64, h->L[0].A.v, 8, s));
    if (mixed && h->L[0].A.vdf) AMG_TRY(ell_bind_one(h, h->L[0].sa64, h->L[0].A.vdf, 8, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    return AMG_OK;
}

int ell_refresh(Hierarchy *h, cudaStream_t s) {
    int rc = AMG_OK;
    for_each_plan(h, [&](StreamPlan &q) {
        if (!q.ell && !q.direct) return;
        for (int k = 0; k < q.nev && rc == AMG_OK; ++k) rc = ell_lay_out(q, q.ev_src[k], q.ev_dst[k], q.ev_bytes[k], s);
    });
    AMG_TRY(rc);
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    return AMG_OK;
}

// Refines every streaming plan of the hierarchy by timed trial of each
// operator's own pass, over the layouts `lay` admits.
static int tune_all(Hierarchy *h, int lay, cudaStream_t s) {
    const bool mixed = h->cfg.precision == AMG_PRECISION_MIXED;
    for (int l = 0; l < h->nsolve - 1; ++l) {
        Level &lv = h->L[l];
        // pre- and post-smoothing gather different vectors and run different
        // epilogues: their plans of A are tuned apart
        lv.sa_post = lv.sa;
        const TuneKind post = l == 0 ? TUNE_POST0 : TUNE_POST;
        if (mixed) {
            // the Krylov solvers hand the finest level FP32 copies of its input
            AMG_TRY((tune_plan<float, float>(lv.A, lv.A.v32, lv.sa, h->arena, lay, TUNE_PRE, s)));
            AMG_TRY((tune_plan<float, float>(lv.A, lv.A.v32, lv.sa_post, h->arena, lay, post, s)));
            AMG_TRY((tune_plan<float, float>(lv.P, lv.P.v32, lv.sp, h->arena, lay, TUNE_PROLONG, s)));
            AMG_TRY((tune_plan<float, float>(lv.R, lv.R.v32, lv.sr, h->arena, lay, TUNE_SPMV, s)));
        } else {
            AMG_TRY((tune_plan<double, double>(lv.A, lv.A.v, lv.sa, h->arena, lay, TUNE_PRE, s)));
            AMG_TRY((tune_plan<double, double>(lv.A, lv.A.v, lv.sa_post, h->arena, lay, post, s)));
            AMG_TRY((tune_plan<double, double>(lv.P, lv.P.v, lv.sp, h->arena, lay, TUNE_PROLONG, s)));
            AMG_TRY((tune_plan<double, double>(lv.R, lv.R.v, lv.sr, h->arena, lay, TUNE_SPMV, s)));
        }
    }
    AMG_TRY((tune_plan<double, double>(h->L[0].A, h->L[0].A.v, h->L[0].sa64, h->arena, lay, TUNE_ALPHA, s)));
    return ell_bind(h, s);
}

// ---------------------------------------------------------------------------
// Fused coarse levels (tail.cuh)
// ---------------------------------------------------------------------------

// Shared memory one tail CTA may use (the SM's 228 KB less the static part).
constexpr int TAIL_SMEM_MAX = 220 * 1024;

// Splits an operator's rows into `cta` contiguous slices of about equal
// stored entries (dense: equal rows) and picks the lanes per row.
template <typename TV>
static void tail_partition(tail::TOp<TV> &op, const std::vector<int> &rp, int cta) {
    const int n = op.n;
    const long long nnz = op.ci ? rp[n] : (long long)n * op.ncols;
    op.r0[0] = 0;
    for (int c = 1; c < cta; ++c) {
        if (op.ci) {
            const long long target = nnz * c / cta;
            op.r0[c] = (int)(std::lower_bound(rp.begin(), rp.begin() + n + 1, (int)target) - rp.begin());
        } else {
            op.r0[c] = (int)((long long)n * c / cta);
        }
        op.r0[c] = std::max(op.r0[c], op.r0[c - 1]);
    }
    for (int c = cta; c <= tail::MAX_CTAS; ++c) op.r0[c] = n;
    for (int c = 0; c <= tail::MAX_CTAS; ++c) op.e0[c] = op.ci ? rp[op.r0[c]] : 0;
    int rows_max = 1;
    for (int c = 0; c < cta; ++c) rows_max = std::max(rows_max, op.r0[c + 1] - op.r0[c]);
    const double mean = n > 0 ? (double)nnz / n : 1.0;
    int by_rows = 1;
    while (by_rows < 32 && (long long)(by_rows * 2) * rows_max <= tail::THREADS) by_rows <<= 1;
    int by_nnz = 1;
    while (by_nnz < 32 && by_nnz < mean) by_nnz <<= 1;
    op.vec = std::max(1, std::min(by_rows, by_nnz));
}

// Largest shared-memory slice (bytes, 16-aligned) of an operator over the CTAs.
template <typename TV>
static void tail_slice_bytes(const tail::TOp<TV> &op, const std::vector<int> &rp, int cta, long long &rpb,
                             long long &cib, long long &vb) {
    rpb = cib = vb = 0;
    for (int c = 0; c < cta; ++c) {
        const int r0 = op.r0[c], r1 = op.r0[c + 1];
        if (r0 >= r1) continue;
        long long e0, e1;
        if (op.ci) {
            rpb = std::max(rpb, (tail::align_hi<int>(r1 + 1) - tail::align_lo<int>(r0)) * 4);
            e0 = rp[r0];
            e1 = rp[r1];
            if (e1 > e0) cib = std::max(cib, (tail::align_hi<int>(e1) - tail::align_lo<int>(e0)) * 4);
        } else {
            e0 = (long long)r0 * op.ncols;
            e1 = (long long)r1 * op.ncols;
        }
        if (e1 > e0) vb = std::max(vb, (tail::align_hi<TV>(e1) - tail::align_lo<TV>(e0)) * (long long)sizeof(TV));
    }
}

static int host_rp(const DevCSR &m, std::vector<int> &rp) {
    rp.resize((size_t)m.nrows + 1);
    AMG_CUDA_TRY(cudaMemcpy(rp.data(), m.rp, sizeof(int) * rp.size(), cudaMemcpyDeviceToHost));
    return AMG_OK;
}

// Bytes CTA c bulk-copies for one preloaded operator (the same rounding as
// the kernel's preload()).
template <typename TV>
static long long tail_cta_bytes(const tail::TOp<TV> &op, int c) {
    if (!op.res) return 0;
    const int r0 = op.r0[c], r1 = op.r0[c + 1];
    if (r0 >= r1) return 0;
    long long by = 0, e0, e1;
    if (op.ci) {
        by += (tail::align_hi<int>(r1 + 1) - tail::align_lo<int>(r0)) * 4;
        e0 = op.e0[c];
        e1 = op.e0[c + 1];
        if (e1 > e0) by += (tail::align_hi<int>(e1) - tail::align_lo<int>(e0)) * 4;
    } else {
        e0 = (long long)r0 * op.ncols;
        e1 = (long long)r1 * op.ncols;
    }
    if (e1 > e0) by += (tail::align_hi<TV>(e1) - tail::align_lo<TV>(e0)) * (long long)sizeof(TV);
    return by;
}

// Builds the kernel's parameter table for the fused tail from level t: row
// slices, lanes per row, and the shared-memory layout -- the staged vector,
// every smoothed level's w and b, then the slices of the finest tail level's
// A, P, R, the next level's, ..., the coarsest inverse, each preloaded while
// the budget lasts.
template <typename TM>
static int build_tail_table(Hierarchy *h, int t, int cta, std::vector<unsigned char> &out, int *smem_bytes) {
    const bool mixed = sizeof(TM) == 4;
    tail::TArgs<TM> a;
    memset(&a, 0, sizeof(a));
    a.nlev = h->nsolve - t;
    a.level0 = t == 0;
    a.nc = h->nc;
    // operators and their row slices
    std::vector<std::vector<int>> rps;  // host row pointers, in placement order
    std::vector<tail::TOp<TM> *> order;
    for (int k = 0; k < a.nlev; ++k) {
        const Level &lv = h->L[t + k];
        tail::TLevel<TM> &d = a.L[k];
        d.n = lv.A.nrows;
        d.w = (const TM *)(mixed ? (const void *)lv.w32 : (const void *)lv.w);
        d.b = (TM *)(mixed ? (void *)lv.b32 : (void *)lv.b);
        d.t = (TM *)(mixed ? (void *)lv.t32 : (void *)lv.t);
        d.x = (TM *)(mixed ? (void *)lv.x32 : (void *)lv.x);
        d.ws_off = d.bs_off = -1;
        if (k == a.nlev - 1) break;  // the coarsest level is solved with its dense inverse
        struct {
            tail::TOp<TM> *op;
            const DevCSR *m;
        } ops[3] = {{&d.A, &lv.A}, {&d.P, &lv.P}, {&d.R, &lv.R}};
        for (auto &o : ops) {
            o.op->rp = o.m->rp;
            o.op->ci = o.m->ci;
            o.op->v = (const TM *)(mixed ? (const void *)o.m->v32 : (const void *)o.m->v);
            o.op->n = o.m->nrows;
            o.op->ncols = o.m->ncols;
            rps.emplace_back();
            AMG_TRY(host_rp(*o.m, rps.back()));
            tail_partition(*o.op, rps.back(), cta);
            order.push_back(o.op);
        }
    }
    const std::vector<int> none;
    a.C.rp = nullptr;
    a.C.ci = nullptr;
    a.C.v = h->cinv;
    a.C.n = a.nc;
    a.C.ncols = a.nc;
    tail_partition(a.C, none, cta);
    // shared memory: the staged vector, every smoothed level's w and b, then
    // operator slices
    long long stage = a.nc;
    for (int k = 0; k < a.nlev; ++k) stage = std::max<long long>(stage, h->L[t + k].A.nrows);
    long long off = (stage * sizeof(TM) + 127) / 128 * 128;
    a.stage_off = 0;
    if (off > TAIL_SMEM_MAX) {
        *smem_bytes = -1;  // does not fit: no fused tail
        return AMG_OK;
    }
    for (int k = 0; k < a.nlev - 1; ++k) {
        tail::TLevel<TM> &d = a.L[k];
        const long long vb = (tail::align_hi<TM>(d.n)) * (long long)sizeof(TM);
        if (off + 2 * vb <= TAIL_SMEM_MAX) {
            d.ws_off = (int)off;
            d.bs_off = (int)(off + vb);
            off += 2 * vb;
        }
    }
    auto place = [&](auto &op, const std::vector<int> &rp) {
        long long rpb, cib, vb;
        tail_slice_bytes(op, rp, cta, rpb, cib, vb);
        const long long need = rpb + cib + vb;
        if (off + need > TAIL_SMEM_MAX) {
            op.res = 0;
            return;
        }
        op.res = 1;
        op.rp_off = (int)off;
        op.ci_off = (int)(off + rpb);
        op.v_off = (int)(off + rpb + cib);
        off += need;
    };
    for (size_t q = 0; q < order.size(); ++q) place(*order[q], rps[q]);
    place(a.C, none);
    for (int c = 0; c < cta; ++c) {
        long long tx = tail_cta_bytes(a.C, c);
        for (int k = 0; k < a.nlev - 1; ++k) {
            const tail::TLevel<TM> &d = a.L[k];
            tx += tail_cta_bytes(d.A, c) + tail_cta_bytes(d.P, c) + tail_cta_bytes(d.R, c);
            if (d.ws_off >= 0) tx += tail::align_hi<TM>(d.n) * (long long)sizeof(TM);
        }
        a.tx[c] = (unsigned)tx;
    }
    out.resize(sizeof(a));
    memcpy(out.data(), &a, sizeof(a));
    *smem_bytes = (int)off;
    return AMG_OK;
}

// Raises k_tail<TM>'s dynamic shared-memory limit to at least smem.  The
// limit belongs to the kernel, shared by every hierarchy in the process, so
// it only grows: lowering it for one hierarchy (e.g. an adjoint's) would make
// another's larger tail fail to launch.
template <typename TM>
static bool tail_smem_limit(int smem) {
    static int limit = 0;
    if (smem <= limit) return true;
    if (cudaFuncSetAttribute((const void *)tail::k_tail<TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    limit = smem;
    return true;
}

template <typename TM>
static int tail_cluster_size(int smem) {
    const void *fn = (const void *)tail::k_tail<TM>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) cudaGetLastError();
    if (!tail_smem_limit<TM>(smem)) return 0;
    for (int cs : {16, 8}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(tail::THREADS);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) == cudaSuccess && nclusters > 0) return cs;
        cudaGetLastError();
    }
    return 0;
}

static int cpcg_prepare(Hierarchy *h);
static int vtail_prepare(Hierarchy *h);

// Chooses the first level of the fused tail: every level from it down is
// small -- no streaming plan, fewer than 16384 rows and at most 400K stored
// entries, a few MB that one cluster of 16 SMs reads faster than a
// full-GPU launch can start -- and at least one of them is smoothed.  Builds
// the device tables (the cluster size is the largest of 16 and 8 that the
// device schedules with the tables' shared memory).
int tail_prepare(Hierarchy *h, cudaStream_t) {
    h->tail_start = -1;
    const int L = h->nsolve;
    if (L < 2 || h->cfg.fuse_coarse != 1) return AMG_OK;
    int t = L - 1;
    while (t > 0 && h->L[t - 1].sa.rt == 0 && h->L[t - 1].A.nrows < 16384 && h->L[t - 1].A.nnz <= 400000) --t;
    if (t > L - 2 || L - t > tail::MAX_LEVELS) return AMG_OK;
    const bool mixed = h->cfg.precision == AMG_PRECISION_MIXED;
    for (int cs : {16, 8}) {
        int s64 = 0, s32 = 0;
        std::vector<unsigned char> a64, a32;
        AMG_TRY(build_tail_table<double>(h, t, cs, a64, &s64));
        if (mixed) AMG_TRY(build_tail_table<float>(h, t, cs, a32, &s32));
        if (s64 < 0 || s32 < 0) continue;
        const int got = tail_cluster_size<double>(s64);
        const int got32 = mixed ? tail_cluster_size<float>(s32) : got;
        if (got >= cs && got32 >= cs) {
            h->tail_cluster = cs;
            h->tail_args64 = a64;
            h->tail_args32 = a32;
            h->tail_smem64 = s64;
            h->tail_smem32 = s32;
            h->tail_start = t;
            AMG_TRY(vtail_prepare(h));
            return cpcg_prepare(h);
        }
    }
    return AMG_OK;
}

template <typename TM>
static int launch_tail(Hierarchy *h, Workspace &W, const double *b0, double *z0, const double *qprev, int fin,
                       cudaStream_t s) {
    const bool mixed = sizeof(TM) == 4;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(h->tail_cluster);
    cfg.blockDim = dim3(tail::THREADS);
    cfg.dynamicSmemBytes = mixed ? h->tail_smem32 : h->tail_smem64;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = h->tail_cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const tail::TArgs<TM> &args = *(const tail::TArgs<TM> *)(mixed ? h->tail_args32.data() : h->tail_args64.data());
    if (!tail_smem_limit<TM>((int)cfg.dynamicSmemBytes)) {
        set_last_error("fused tail: %d bytes of shared memory refused", (int)cfg.dynamicSmemBytes);
        return AMG_ERR_CUDA;
    }
    AMG_CUDA_TRY(cudaLaunchKernelEx(&cfg, tail::k_tail<TM>, args, b0, z0, qprev, fin, W.scal));
    return AMG_OK;
}

// ---------------------------------------------------------------------------
// Whole PCG solves in one cluster (cpcg.cuh)
// ---------------------------------------------------------------------------

// Dynamic shared memory of one whole-solve CTA: the SM's 227 KB less the
// kernel's static part (the reductions' partials and the table, about 18 KB).
constexpr int CPCG_SMEM_MAX = 208 * 1024;

// A level's row split: `cta` slices of about equal stored entries of A (of
// rows for the dense level), inner bounds rounded to multiples of 4.
static void cpcg_split(int n, const std::vector<int> *rp, int cta, int *r0) {
    r0[0] = 0;
    const long long tot = rp ? (long long)(*rp)[n] : n;
    for (int c = 1; c < cta; ++c) {
        const long long t = tot * c / cta;
        int r = rp ? (int)(std::lower_bound(rp->begin(), rp->begin() + n + 1, (int)t) - rp->begin()) : (int)t;
        r = (r + 2) / 4 * 4;
        r0[c] = std::min(std::max(r, r0[c - 1]), n);
    }
    for (int c = cta; c <= cpcg::MAX_CTAS; ++c) r0[c] = n;
}

// Fills an operator's entry bounds per slice and its lanes per row (the
// fused tail's rule: as many lanes as the mean row length asks, while the
// largest slice's rows still fill the CTA's threads).
template <typename TV>
static void cpcg_op(cpcg::COp<TV> &op, const DevCSR *m, const TV *v, const std::vector<int> *rp, const int *r0,
                    int cta, int ncols) {
    op.rp = m ? m->rp : nullptr;
    op.ci = m ? m->ci : nullptr;
    op.v = v;
    op.ncols = ncols;
    op.copy = 3;
    const int n = r0[cta];
    for (int c = 0; c <= cpcg::MAX_CTAS; ++c) op.e0[c] = rp ? (*rp)[r0[std::min(c, cta)]] : 0;
    const long long nnz = rp ? (long long)(*rp)[n] : (long long)n * ncols;
    int rows_max = 1;
    for (int c = 0; c < cta; ++c) rows_max = std::max(rows_max, r0[c + 1] - r0[c]);
    const double mean = n > 0 ? (double)nnz / n : 1.0;
    int by_rows = 1;
    while (by_rows < 32 && (long long)(by_rows * 2) * rows_max <= cpcg::THREADS) by_rows <<= 1;
    int by_nnz = 1;
    while (by_nnz < 32 && by_nnz < mean) by_nnz <<= 1;
    op.vec = std::max(1, std::min(by_rows, by_nnz));
}

// Largest slice of an operator over the CTAs: bytes of row pointers,
// indices and values, each region 16-byte aligned.
template <typename TV>
static void cpcg_slice_max(const cpcg::COp<TV> &op, const int *r0, int cta, long long &rpb, long long &cib,
                           long long &vb) {
    rpb = cib = vb = 0;
    for (int c = 0; c < cta; ++c) {
        const int a = r0[c], z = r0[c + 1];
        if (a >= z) continue;
        long long e0, e1;
        if (op.ci) {
            rpb = std::max(rpb, (tail::align_hi<int>(z + 1) - tail::align_lo<int>(a)) * 4);
            e0 = op.e0[c];
            e1 = op.e0[c + 1];
            if (e1 > e0) cib = std::max(cib, (tail::align_hi<int>(e1) - tail::align_lo<int>(e0)) * 4);
        } else {
            e0 = (long long)a * op.ncols;
            e1 = (long long)z * op.ncols;
        }
        if (e1 > e0) vb = std::max(vb, (tail::align_hi<TV>(e1) - tail::align_lo<TV>(e0)) * (long long)sizeof(TV));
    }
}

static long long round16(long long b) { return (b + 15) / 16 * 16; }

// The parameter table of the whole-solve cluster kernel with `cta` CTAs and
// its dynamic shared memory, or *smem_bytes = -1 where the operators and
// vectors do not all fit.  Shared memory: the two staging buffers (a whole
// vector of the largest level, FP64 for the outer product), the CTA's FP64
// slices of x, r, p, q, z, each smoothed level's slices of w and b, then the
// operator slices.
//
// collapsed = 1 takes the hierarchy as the V-cycle runs it, levels 0 ..
// nsolve-1 with the dense operator of the collapsed coarse end (its FP32
// copy in the mixed form); collapsed = 0 takes every level, 0 .. nlevels-1,
// with the coarsest level's dense inverse -- the same preconditioner up to
// rounding, the collapse being exact.
//
// vmode = 1 builds the table of one V-cycle from level t (the kernel's level
// 0; no Krylov vectors or outer product), with level t's b and x in global
// memory.
// Whether the V-cycle cluster launch from level t computes level t's
// right-hand side itself (R_{t-1} t_{t-1}): when R_{t-1} does not stream
// (its rows are level t's, fewer than 16384) and is small enough for the
// cluster's SMs to read in about a microsecond.
static bool vtail_folds_restriction(const Hierarchy *h, int t) {
    if (t < 1) return false;
    const Level &lp = h->L[t - 1];
    return !lp.sr.rt && lp.R.nnz <= 400000;
}

template <typename TM>
static int build_cpcg_table(Hierarchy *h, int cta, int collapsed, int t, int vmode, std::vector<unsigned char> &out,
                            int *smem_bytes) {
    const bool mixed = sizeof(TM) == 4;
    *smem_bytes = -1;
    const int nl = (collapsed ? h->nsolve : h->nlevels) - t;
    const bool dense32 = collapsed && mixed && h->nsolve < h->nlevels && h->cinv32;
    if (nl < 2 || nl > cpcg::MAX_LEVELS) return AMG_OK;
    cpcg::CArgs<TM> a;
    memset(&a, 0, sizeof(a));
    a.nlev = nl;
    a.cta = cta;
    a.vmode = vmode;
    if (vmode) {
        const Level &lt = h->L[t];
        a.vb = (const TM *)(mixed ? (const void *)lt.b32 : (const void *)lt.b);
        a.vx = (TM *)(mixed ? (void *)lt.x32 : (void *)lt.x);
        if (vtail_folds_restriction(h, t)) {
            const Level &lp = h->L[t - 1];
            a.vr_rp = lp.R.rp;
            a.vr_ci = lp.R.ci;
            a.vr_v = (const TM *)(mixed ? (const void *)lp.R.v32 : (const void *)lp.R.v);
            a.vr_x = (const TM *)(mixed ? (const void *)lp.t32 : (const void *)lp.t);
        }
    }
    std::vector<std::vector<int>> rpA(nl), rpP(nl), rpR(nl);
    for (int k = 0; k < nl; ++k) {
        cpcg::CLevel<TM> &d = a.L[k];
        d.w_off = d.b_off = -1;
        if (k < nl - 1) {
            const Level &lv = h->L[t + k];
            d.n = lv.A.nrows;
            AMG_TRY(host_rp(lv.A, rpA[k]));
            AMG_TRY(host_rp(lv.P, rpP[k]));
            AMG_TRY(host_rp(lv.R, rpR[k]));
            cpcg_split(d.n, &rpA[k], cta, d.r0);
            d.w = (const TM *)(mixed ? (const void *)lv.w32 : (const void *)lv.w);
        } else {
            d.n = collapsed ? h->nc : h->L[t + k].A.nrows;
            cpcg_split(d.n, nullptr, cta, d.r0);
        }
    }
    for (int k = 0; k < nl - 1; ++k) {
        const Level &lv = h->L[t + k];
        cpcg::CLevel<TM> &d = a.L[k];
        auto vals = [&](const DevCSR &m) { return (const TM *)(mixed ? (const void *)m.v32 : (const void *)m.v); };
        cpcg_op(d.A, &lv.A, vals(lv.A), &rpA[k], d.r0, cta, lv.A.ncols);
        cpcg_op(d.P, &lv.P, vals(lv.P), &rpP[k], d.r0, cta, lv.P.ncols);
        cpcg_op(d.R, &lv.R, vals(lv.R), &rpR[k], a.L[k + 1].r0, cta, lv.R.ncols);
    }
    if (!vmode) cpcg_op(a.K, &h->L[0].A, (const double *)h->L[0].A.v, &rpA[0], a.L[0].r0, cta, h->L[0].A.ncols);
    const int nd = a.L[nl - 1].n;
    cpcg_op(a.C, (const DevCSR *)nullptr, (const double *)(collapsed ? h->cinv : h->cinv_last), nullptr,
            a.L[nl - 1].r0, cta, nd);
    cpcg_op(a.C32, (const DevCSR *)nullptr, (const float *)h->cinv32, nullptr, a.L[nl - 1].r0, cta, nd);
    a.c32 = dense32 ? 1 : 0;
    a.C.copy = dense32 ? 0 : 3;
    a.C32.copy = dense32 ? 3 : 0;
    // the outer operator shares A_0's row pointers and indices (and in the
    // FP64 form its values)
    a.K.copy = mixed && !vmode ? 2 : 0;

    long long vec_bytes = vmode ? 0 : 8LL * h->n;
    for (int k = 0; k < nl; ++k) vec_bytes = std::max<long long>(vec_bytes, (long long)a.L[k].n * sizeof(TM));
    const long long bufb = round16(vec_bytes);
    long long off = 0;
    a.buf_bytes = (int)bufb;
    a.buf_off[0] = 0;
    a.buf_off[1] = (int)bufb;
    off = 2 * bufb;
    auto slice_rows = [&](int k) {
        int m = 0;
        for (int c = 0; c < cta; ++c) m = std::max(m, a.L[k].r0[c + 1] - a.L[k].r0[c]);
        return m;
    };
    const long long kb = vmode ? 0 : round16(8LL * slice_rows(0));
    int *koffs[5] = {&a.x_off, &a.r_off, &a.p_off, &a.q_off, &a.z_off};
    for (int *o : koffs) {
        *o = (int)off;
        off += kb;
    }
    for (int k = 0; k < nl - 1; ++k) {
        const long long vb = round16((long long)sizeof(TM) * slice_rows(k));
        a.L[k].w_off = (int)off;
        off += vb;
        if (k > 0 || vmode) {
            a.L[k].b_off = (int)off;
            off += vb;
        }
    }
    auto place = [&](auto &op, const int *r0) {
        long long rpb, cib, vb;
        if (!op.copy) return;
        cpcg_slice_max(op, r0, cta, rpb, cib, vb);
        if (op.copy & 1) {
            op.rp_off = (int)off;
            op.ci_off = (int)(off + rpb);
            off += rpb + cib;
        }
        if (op.copy & 2) {
            op.v_off = (int)off;
            off += vb;
        }
    };
    for (int k = 0; k < nl - 1; ++k) {
        place(a.L[k].A, a.L[k].r0);
        place(a.L[k].P, a.L[k].r0);
        place(a.L[k].R, a.L[k + 1].r0);
    }
    place(a.C, a.L[nl - 1].r0);
    place(a.C32, a.L[nl - 1].r0);
    if (!vmode) {
        a.K.rp_off = a.L[0].A.rp_off;
        a.K.ci_off = a.L[0].A.ci_off;
        if (mixed) place(a.K, a.L[0].r0);
        else a.K.v_off = a.L[0].A.v_off;  // the FP64 cycle's A_0 itself
    }
    if (off > CPCG_SMEM_MAX) return AMG_OK;
    for (int c = 0; c < cta; ++c) {
        long long tx = 0;
        for (int k = 0; k < nl - 1; ++k) {
            const cpcg::CLevel<TM> &d = a.L[k], &nx = a.L[k + 1];
            tx += cpcg::slice_copy(d.A, d.r0[c], d.r0[c + 1], c, nullptr, nullptr, false);
            tx += cpcg::slice_copy(d.P, d.r0[c], d.r0[c + 1], c, nullptr, nullptr, false);
            tx += cpcg::slice_copy(d.R, nx.r0[c], nx.r0[c + 1], c, nullptr, nullptr, false);
        }
        tx += cpcg::slice_copy(a.K, a.L[0].r0[c], a.L[0].r0[c + 1], c, nullptr, nullptr, false);
        tx += cpcg::slice_copy(a.C, a.L[nl - 1].r0[c], a.L[nl - 1].r0[c + 1], c, nullptr, nullptr, false);
        tx += cpcg::slice_copy(a.C32, a.L[nl - 1].r0[c], a.L[nl - 1].r0[c + 1], c, nullptr, nullptr, false);
        a.tx[c] = (unsigned)tx;
    }
    out.resize(sizeof(a));
    memcpy(out.data(), &a, sizeof(a));
    *smem_bytes = (int)off;
    return AMG_OK;
}

// Raises k_cpcg<TM, VM>'s dynamic shared-memory limit to at least smem (the
// limit belongs to the kernel and only grows, as the tail's) and allows
// 16-CTA clusters.
template <typename TM, bool VM>
static bool cpcg_smem_limit(int smem) {
    static int limit = 0;
    const void *fn = (const void *)cpcg::k_cpcg<TM, VM>;
    if (smem <= limit) return true;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) cudaGetLastError();
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    limit = smem;
    return true;
}

// Whether k_cpcg<TM, VM> schedules a cluster of `cta` CTAs with smem bytes
// of dynamic shared memory (checked once, at setup).
template <typename TM, bool VM>
static bool cpcg_fits(int cta, int smem) {
    const void *fn = (const void *)cpcg::k_cpcg<TM, VM>;
    if (!cpcg_smem_limit<TM, VM>(smem)) return false;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cta);
    cfg.blockDim = dim3(cpcg::THREADS);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cta;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) == cudaSuccess && nclusters > 0) return true;
    cudaGetLastError();
    return false;
}

// Prepares whole-solve cluster launches for a hierarchy whose whole cycle
// already runs in the single-cluster tail: the hierarchy as collapsed (fewer
// phases a cycle), else every level with the coarsest inverse, on the
// largest cluster (16, then 8 CTAs) whose shared memory holds every operator
// slice and vector.
static int cpcg_prepare(Hierarchy *h) {
    h->cpcg_cta = 0;
    if (h->tail_start != 0 || h->nsys > 0) return AMG_OK;
    const bool mixed = h->cfg.precision == AMG_PRECISION_MIXED;
    for (int collapsed : {1, 0}) {
        if (!collapsed && h->nsolve == h->nlevels) break;
        for (int cs : {16, 8}) {
            std::vector<unsigned char> args;
            int smem = -1;
            if (mixed) AMG_TRY(build_cpcg_table<float>(h, cs, collapsed, 0, 0, args, &smem));
            else AMG_TRY(build_cpcg_table<double>(h, cs, collapsed, 0, 0, args, &smem));
            if (smem < 0) continue;
            if (mixed ? cpcg_fits<float, false>(cs, smem) : cpcg_fits<double, false>(cs, smem)) {
                h->cpcg_cta = cs;
                h->cpcg_args = args;
                h->cpcg_smem = smem;
                return AMG_OK;
            }
        }
    }
    return AMG_OK;
}

// Prepares one-V-cycle cluster launches from the tail's first level when it is
// a coarse level (the finest level streams): collapsed first, on 16 then 8
// CTAs, as for the whole solve.
static int vtail_prepare(Hierarchy *h) {
    h->vtail_cta = 0;
    h->vtail_restricts = 0;
    const int t = h->tail_start;
    if (t <= 0 || h->nsys > 0) return AMG_OK;
    const bool mixed = h->cfg.precision == AMG_PRECISION_MIXED;
    for (int collapsed : {1, 0}) {
        if (!collapsed && h->nsolve == h->nlevels) break;
        if (collapsed && h->nsolve - t < 2) continue;
        for (int cs : {16, 8}) {
            std::vector<unsigned char> args;
            int smem = -1;
            if (mixed) AMG_TRY(build_cpcg_table<float>(h, cs, collapsed, t, 1, args, &smem));
            else AMG_TRY(build_cpcg_table<double>(h, cs, collapsed, t, 1, args, &smem));
            if (smem < 0) continue;
            if (mixed ? cpcg_fits<float, true>(cs, smem) : cpcg_fits<double, true>(cs, smem)) {
                h->vtail_cta = cs;
                h->vtail_args = args;
                h->vtail_smem = smem;
                h->vtail_restricts = vtail_folds_restriction(h, t) ? 1 : 0;  // as the table was built
                return AMG_OK;
            }
        }
    }
    return AMG_OK;
}

// One V-cycle from the tail's first level as one cluster launch.
template <typename TM>
static int launch_vtail(Hierarchy *h, Workspace &W, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(h->vtail_cta);
    cfg.blockDim = dim3(cpcg::THREADS);
    cfg.dynamicSmemBytes = h->vtail_smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = h->vtail_cta;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    if (!cpcg_smem_limit<TM, true>(h->vtail_smem)) {
        set_last_error("V-cycle cluster: %d bytes of shared memory refused", h->vtail_smem);
        return AMG_ERR_CUDA;
    }
    const auto &args = *(const cpcg::CArgs<TM> *)h->vtail_args.data();
    AMG_CUDA_TRY(cudaLaunchKernelEx(&cfg, cpcg::k_cpcg<TM, true>, args, (const double *)nullptr, (double *)nullptr,
                                    (double *)nullptr, (double *)nullptr, (double *)nullptr, (double *)nullptr,
                                    (float *)nullptr, W.scal));
    return AMG_OK;
}

// Bytes one whole-solve launch moves to and from global memory: the operator
// slices every CTA bulk-copies once (the table's transaction counts), x, r,
// p, q read and x, r, p, q, z (and r's FP32 copy) written.
static double cpcg_bytes(const Hierarchy *h) {
    const bool mixed = h->cfg.precision == AMG_PRECISION_MIXED;
    const unsigned *tx = mixed ? ((const cpcg::CArgs<float> *)h->cpcg_args.data())->tx
                               : ((const cpcg::CArgs<double> *)h->cpcg_args.data())->tx;
    double by = 0.0;
    for (int c = 0; c < h->cpcg_cta; ++c) by += tx[c];
    return by + (72.0 + (mixed ? 4.0 : 0.0)) * h->n;
}

// One launch that iterates the PCG solve to its end (the scalars say why).
static int launch_cpcg(Hierarchy *h, Workspace &W, cudaStream_t s) {
    const bool mixed = h->cfg.precision == AMG_PRECISION_MIXED;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(h->cpcg_cta);
    cfg.blockDim = dim3(cpcg::THREADS);
    cfg.dynamicSmemBytes = h->cpcg_smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = h->cpcg_cta;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    TRACE("cluster_pcg", 0, cpcg_bytes(h));
    if (mixed) {
        if (!cpcg_smem_limit<float, false>(h->cpcg_smem)) {
            set_last_error("whole-solve cluster: %d bytes of shared memory refused", h->cpcg_smem);
            return AMG_ERR_CUDA;
        }
        const auto &args = *(const cpcg::CArgs<float> *)h->cpcg_args.data();
        AMG_CUDA_TRY(cudaLaunchKernelEx(&cfg, cpcg::k_cpcg<float, false>, args, (const double *)W.b, W.x, W.r, W.p, W.q, W.z,
                                        W.r32, W.scal));
    } else {
        if (!cpcg_smem_limit<double, false>(h->cpcg_smem)) {
            set_last_error("whole-solve cluster: %d bytes of shared memory refused", h->cpcg_smem);
            return AMG_ERR_CUDA;
        }
        const auto &args = *(const cpcg::CArgs<double> *)h->cpcg_args.data();
        AMG_CUDA_TRY(cudaLaunchKernelEx(&cfg, cpcg::k_cpcg<double, false>, args, (const double *)W.b, W.x, W.r, W.p, W.q,
                                        W.z, (float *)nullptr, W.scal));
    }
    return AMG_OK;
}

// Algorithmic bytes of the fused tail (levels t.. of one V-cycle).
static double tail_bytes(const Hierarchy *h, int vb) {
    double by = 0.0;
    for (int l = h->tail_start; l < h->nsolve - 1; ++l) {
        const Level &lv = h->L[l];
        by += 2.0 * (lv.A.nnz * (4.0 + vb) + 4.0 * (lv.A.nrows + 1.0)) + 2.0 * (lv.P.nnz * (4.0 + vb)) +
              4.0 * (lv.A.nrows + lv.R.nrows + 2.0) + 8.0 * vb * lv.A.nrows;
    }
    return by + 8.0 * h->nc * h->nc + 2.0 * vb * h->nc;
}

// First level m of the cooperative coarse launch (mid.cuh; fuse_coarse = 2),
// or -1: levels m..L-2 all have fewer than 16384 rows and no streaming plan,
// m >= 1 (the finest level reads the FP64 input and finishes the Krylov
// scalars) and the cycle ends in the dense operator.
static int mid_level(const Hierarchy *h) {
    const int L = h->nsolve;
    if (h->cfg.fuse_coarse != 2 || h->tail_start >= 0 || L < 3 || h->nc_ld > mid::DENSE_LD) return -1;
    auto small = [](const Level &lv) {
        return !lv.sa.rt && !lv.sa_post.rt && !lv.sp.rt && !lv.sr.rt && lv.A.nrows < 16384;
    };
    int m = L - 1;
    while (m - 1 >= 1 && L - m < mid::MAX_LEVELS + 1 && small(h->L[m - 1])) --m;
    return m < L - 1 ? m : -1;
}

// CTAs of the cooperative launch: up to two per SM, as the occupancy allows.
template <typename TM, typename TMAT>
static int mid_grid() {
    static int g = 0;
    if (!g) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mid::k_mid<TM, TMAT>, mid::THREADS, 0) != cudaSuccess)
            return 0;
        g = std::min(per_sm, 2) * num_sms();
    }
    return g;
}

// Levels m..L-1 of one V-cycle (and the restriction into level m when it is
// not streamed) as one cooperative launch.
template <typename TM>
static int launch_mid(Hierarchy *h, Workspace &W, int m, cudaStream_t s) {
    const bool mixed = sizeof(TM) == 4;
    auto Av = [&](const DevCSR &a) -> const TM * { return (const TM *)(mixed ? (const void *)a.v32 : (const void *)a.v); };
    auto Wv = [&](const Level &lv) -> const TM * { return (const TM *)(mixed ? (const void *)lv.w32 : (const void *)lv.w); };
    auto Tv = [&](const Level &lv) -> TM * { return (TM *)(mixed ? (void *)lv.t32 : (void *)lv.t); };
    auto Bv = [&](const Level &lv) -> TM * { return (TM *)(mixed ? (void *)lv.b32 : (void *)lv.b); };
    auto Xv = [&](const Level &lv) -> TM * { return (TM *)(mixed ? (void *)lv.x32 : (void *)lv.x); };
    const int L = h->nsolve;
    mid::MArgs<TM> a = {};
    a.nlev = L - 1 - m;
    const Level &lp = h->L[m - 1];
    if (!lp.sr.rt) {
        a.r0n = lp.R.nrows;
        a.r0vec = lp.vec_r;
        a.r0rp = lp.R.rp;
        a.r0ci = lp.R.ci;
        a.r0v = Av(lp.R);
        a.r0x = Tv(lp);
    }
    for (int k = 0; k < a.nlev; ++k) {
        const Level &lv = h->L[m + k];
        mid::MLevel<TM> &o = a.L[k];
        o.n = lv.A.nrows;
        o.nc = lv.R.nrows;
        o.vec_a = lv.vec_a;
        o.vec_p = lv.vec_p;
        o.vec_r = lv.vec_r;
        o.arp = lv.A.rp, o.aci = lv.A.ci, o.av = Av(lv.A);
        o.prp = lv.P.rp, o.pci = lv.P.ci, o.pv = Av(lv.P);
        o.rrp = lv.R.rp, o.rci = lv.R.ci, o.rv = Av(lv.R);
        o.w = Wv(lv);
        o.b = Bv(lv), o.t = Tv(lv), o.x = Xv(lv);
    }
    const Level &lc = h->L[L - 1];
    const bool m32 = mixed && h->cpad32;
    a.dm = h->nc;
    a.dld = h->nc_ld;
    a.M = m32 ? (const void *)h->cpad32 : (const void *)h->cpad64;
    a.db = Bv(lc);
    a.dx = Xv(lc);
    const int grid = m32 ? mid_grid<TM, float>() : mid_grid<TM, double>();
    if (grid <= 0) {
        set_last_error("fused coarse levels: no resident CTA");
        return AMG_ERR_CUDA;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(mid::THREADS);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const int *done = &W.scal->done;
    int *err = &W.scal->copy_timeout;
    if (m32)
        AMG_CUDA_TRY(cudaLaunchKernelEx(&cfg, mid::k_mid<TM, float>, a, W.gbar, done, err));
    else
        AMG_CUDA_TRY(cudaLaunchKernelEx(&cfg, mid::k_mid<TM, double>, a, W.gbar, done, err));
    return AMG_OK;
}

// Algorithmic bytes of the fused coarse levels (one V-cycle).
static double mid_bytes(const Hierarchy *h, int m, int vb) {
    const bool m32 = vb == 4 && h->cpad32;
    const Level &lp = h->L[m - 1];
    double by = lp.sr.rt ? 0.0 : csr_bytes(lp.R, vb) + (double)vb * (lp.A.nrows + lp.R.nrows);
    for (int l = m; l < h->nsolve - 1; ++l) {  // the sum of the per-pass figures
        const Level &lv = h->L[l];
        by += 2.0 * csr_bytes(lv.A, vb) + csr_bytes(lv.P, vb) + csr_bytes(lv.R, vb) + 11.0 * vb * lv.A.nrows +
              2.0 * vb * lv.R.nrows;
    }
    const double nc = h->nc;
    return by + nc * nc * (m32 ? 4.0 : 8.0) + 2.0 * vb * nc;
}

// One V-cycle: z0 = M^-1 b0.  TM = float for the mixed form.
template <typename TM>
static int launch_vcycle(Hierarchy *h, Workspace &W, const double *b0, double *z0, int fin, cudaStream_t s,
                         const float *b032) {
    const int L = h->nsolve;
    const int cap = W.part_cap;
    const int *done = &W.scal->done;
    const bool mixed = sizeof(TM) == 4;
    const int vb = sizeof(TM);
    auto Av = [&](const DevCSR &m) -> const TM * { return (const TM *)(mixed ? (const void *)m.v32 : (const void *)m.v); };
    auto Wv = [&](const Level &lv) -> const TM * { return (const TM *)(mixed ? (const void *)lv.w32 : (const void *)lv.w); };
    auto Tv = [&](const Level &lv) -> TM * { return (TM *)(mixed ? (void *)lv.t32 : (void *)lv.t); };
    auto Bv = [&](const Level &lv) -> TM * { return (TM *)(mixed ? (void *)lv.b32 : (void *)lv.b); };
    auto Xv = [&](const Level &lv) -> TM * { return (TM *)(mixed ? (void *)lv.x32 : (void *)lv.x); };
    // the flexible beta's z.q with the previous iteration's q = A p
    const double *qprev = (fin == FIN_PCG_BETA && h->cfg.precision == AMG_PRECISION_MIXED) ? W.q : nullptr;

    if (L == 1) {
        const double m = h->nc;
        TRACE("coarse", 0, m * m * 8.0 + 16.0 * m + (fin == FIN_PCG_BETA ? 8.0 * m : 0.0));
        if (fin == FIN_PCG_BETA)
            AMG_TRY(launch_k(k_coarse<double, double, FIN_PCG_BETA>, 1, BLOCK, 0, s, h->nc, h->cinv, b0, z0, qprev, W.scal, W.part, cap, W.counter));
        else
            AMG_TRY(launch_k(k_coarse<double, double, FIN_NONE>, 1, BLOCK, 0, s, h->nc, h->cinv, b0, z0, qprev, W.scal, W.part, cap, W.counter));
        AMG_LAUNCH_CHECK();
        return AMG_OK;
    }
    const int mm = mid_level(h);  // first level of the cooperative coarse launch, or -1
    // first level handled by the fused tail or the cooperative launch
    const int tl = h->tail_start >= 0 ? h->tail_start : (mm > 0 ? mm : L - 1);
    // the cluster kernel's V-cycle where its table fits (built for the form's
    // cycle type), else the tail kernel; the cluster V-cycle restricts into
    // its first level itself when its table says so
    const bool vt = h->tail_start > 0 && h->vtail_cta &&
                    (sizeof(TM) == 4) == (h->cfg.precision == AMG_PRECISION_MIXED);
    const bool vt_restricts = vt && h->vtail_restricts;
    if (h->tail_start == 0) {
        TRACE("tail", 0, tail_bytes(h, vb));
        return launch_tail<TM>(h, W, b0, z0, qprev, fin == FIN_PCG_BETA, s);
    }
    // down
    for (int l = 0; l < tl; ++l) {
        Level &lv = h->L[l];
        Level &nx = h->L[l + 1];
        const int n = lv.A.nrows;
        const double bb = l == 0 ? (b032 ? 4.0 : 8.0) : vb;  // the finest input: FP32 copy or FP64
        int *err = &W.scal->copy_timeout;
        if (lv.sa.rt) {
            TRACE("presmooth", l, csr_bytes(lv.A, vb) + n * (bb + vb));
            const TM *ah = (const TM *)(mixed ? (const void *)lv.ahat32 : (const void *)lv.ahat);
            if (l == 0 && b032 && mixed)
                AMG_TRY(stream_launch<TM>(lv.sa, n, lv.A.rp, lv.A.ci, ah,
                                          OpPre<float, TM>{done, reinterpret_cast<const float *>(b032), Tv(lv)}, err, s));
            else if (l == 0)
                AMG_TRY(stream_launch<TM>(lv.sa, n, lv.A.rp, lv.A.ci, ah, OpPre<double, TM>{done, b0, Tv(lv)}, err, s));
            else
                AMG_TRY(stream_launch<TM>(lv.sa, n, lv.A.rp, lv.A.ci, ah, OpPre<TM, TM>{done, Bv(lv), Tv(lv)}, err, s));
        } else {
            TRACE("presmooth", l, csr_bytes(lv.A, vb) + n * (bb + 2.0 * vb));
            if (l == 0 && b032 && mixed) {
                VEC_DISPATCH(lv.vec_a, AMG_TRY(launch_k(k_presmooth<V, TM, TM>, grid_rows(n, V, cap), BLOCK, 0, s, n,
                                           lv.A.rp, lv.A.ci, Av(lv.A), Wv(lv), reinterpret_cast<const TM *>(b032),
                                           Tv(lv), done)));
            } else if (l == 0) {
                VEC_DISPATCH(lv.vec_a, AMG_TRY(launch_k(k_presmooth<V, double, TM>, grid_rows(n, V, cap), BLOCK, 0, s, 
                                           n, lv.A.rp, lv.A.ci, Av(lv.A), Wv(lv), b0, Tv(lv), done)));
            } else {
                VEC_DISPATCH(lv.vec_a, AMG_TRY(launch_k(k_presmooth<V, TM, TM>, grid_rows(n, V, cap), BLOCK, 0, s, 
                                           n, lv.A.rp, lv.A.ci, Av(lv.A), Wv(lv), Bv(lv), Tv(lv), done)));
            }
        }
        const int nc = lv.R.nrows;
        // the cooperative launch and the cluster V-cycle restrict into their first level themselves
        if ((l != mm - 1 || lv.sr.rt) && !(vt_restricts && l == tl - 1)) {
            TRACE("restrict", l, csr_bytes(lv.R, vb) + (double)vb * (n + nc));
            if (lv.sr.rt)
                AMG_TRY(stream_launch<TM>(lv.sr, nc, lv.R.rp, lv.R.ci, Av(lv.R), OpSpmv<TM>{done, Tv(lv), Bv(nx)}, err, s));
            else
                VEC_DISPATCH(lv.vec_r, AMG_TRY(launch_k(k_spmv<V, TM, TM, TM>, grid_rows(nc, V, cap), BLOCK, 0, s, 
                                           nc, lv.R.rp, lv.R.ci, Av(lv.R), Tv(lv), Bv(nx), done)));
        }
        AMG_LAUNCH_CHECK();
    }
    if (h->tail_start > 0) {
        if (vt) {
            const Level &lp = h->L[tl - 1];
            TRACE("cluster_cycle", tl,
                  tail_bytes(h, vb) + (vt_restricts ? csr_bytes(lp.R, vb) + (double)vb * lp.A.nrows : 0.0));
            AMG_TRY(launch_vtail<TM>(h, W, s));
        } else {
            TRACE("tail", tl, tail_bytes(h, vb));
            AMG_TRY(launch_tail<TM>(h, W, nullptr, nullptr, nullptr, 0, s));
        }
    } else if (mm > 0) {
        TRACE("mid", mm, mid_bytes(h, mm, vb));
        AMG_TRY(launch_mid<TM>(h, W, mm, s));
        AMG_LAUNCH_CHECK();
    } else {
        Level &lc = h->L[L - 1];
        const double m = h->nc;
        const bool m32 = mixed && h->cpad32;
        TRACE("coarse", L - 1, m * m * (m32 ? 4.0 : 8.0) + 2.0 * vb * m);
        const int grid = std::max(1, std::min((h->nc + BLOCK / 32 - 1) / (BLOCK / 32), 4 * num_sms()));
        if (m32)
            AMG_TRY(launch_k(k_dense_apply<float, TM>, grid, BLOCK, 0, s, h->nc, h->nc_ld, h->cpad32, Bv(lc), Xv(lc), done));
        else
            AMG_TRY(launch_k(k_dense_apply<double, TM>, grid, BLOCK, 0, s, h->nc, h->nc_ld, h->cpad64, Bv(lc), Xv(lc), done));
        AMG_LAUNCH_CHECK();
    }
    // up
    for (int l = tl - 1; l >= 0; --l) {
        Level &lv = h->L[l];
        Level &nx = h->L[l + 1];
        const int n = lv.A.nrows;
        const int nc = nx.A.nrows;
        const double bb = l == 0 ? 8.0 : vb;
        const double bbp = l == 0 && b032 ? 4.0 : bb;  // prolongation reads the FP32 copy when given
        int *err = &W.scal->copy_timeout;
        if (lv.sp.rt) {
            TRACE("prolong", l, csr_bytes(lv.P, vb) + (double)vb * nc + n * (bbp + 2.0 * vb));
            if (l == 0 && b032 && mixed)
                AMG_TRY(stream_launch<TM>(lv.sp, n, lv.P.rp, lv.P.ci, Av(lv.P),
                                          OpProlong<float, TM>{done, Wv(lv), reinterpret_cast<const float *>(b032), Xv(nx),
                                                               Tv(lv)}, err, s));
            else if (l == 0)
                AMG_TRY(stream_launch<TM>(lv.sp, n, lv.P.rp, lv.P.ci, Av(lv.P),
                                          OpProlong<double, TM>{done, Wv(lv), b0, Xv(nx), Tv(lv)}, err, s));
            else
                AMG_TRY(stream_launch<TM>(lv.sp, n, lv.P.rp, lv.P.ci, Av(lv.P),
                                          OpProlong<TM, TM>{done, Wv(lv), Bv(lv), Xv(nx), Tv(lv)}, err, s));
        } else {
            TRACE("prolong", l, csr_bytes(lv.P, vb) + (double)vb * nc + n * (bb + 2.0 * vb));
            if (l == 0) {
                VEC_DISPATCH(lv.vec_p, AMG_TRY(launch_k(k_prolong<V, double, TM>, grid_rows(n, V, cap), BLOCK, 0, s, 
                                           n, lv.P.rp, lv.P.ci, Av(lv.P), Wv(lv), b0, Xv(nx), Tv(lv), done)));
            } else {
                VEC_DISPATCH(lv.vec_p, AMG_TRY(launch_k(k_prolong<V, TM, TM>, grid_rows(n, V, cap), BLOCK, 0, s, 
                                           n, lv.P.rp, lv.P.ci, Av(lv.P), Wv(lv), Bv(lv), Xv(nx), Tv(lv), done)));
            }
        }
        {
            const double ob = l == 0 ? 8.0 : vb;
            TRACE("postsmooth", l, csr_bytes(lv.A, vb) + n * (2.0 * vb + bb + ob) + (qprev && l == 0 ? 8.0 * n : 0.0));
            if (lv.sa_post.rt) {
                const int *rp_ = lv.A.rp, *ci_ = lv.A.ci;
                if (l == 0 && fin == FIN_PCG_BETA)
                    AMG_TRY(stream_launch<TM>(lv.sa_post, n, rp_, ci_, Av(lv.A),
                                              OpPost<double, TM, double, FIN_PCG_BETA>{W.scal, Wv(lv), b0, Tv(lv), z0, qprev,
                                                                                         W.part, cap, W.counter},
                                              err, s));
                else if (l == 0)
                    AMG_TRY(stream_launch<TM>(lv.sa_post, n, rp_, ci_, Av(lv.A),
                                              OpPost<double, TM, double, FIN_NONE>{W.scal, Wv(lv), b0, Tv(lv), z0, nullptr,
                                                                                     W.part, cap, W.counter},
                                              err, s));
                else
                    AMG_TRY(stream_launch<TM>(lv.sa_post, n, rp_, ci_, Av(lv.A),
                                              OpPost<TM, TM, TM, FIN_NONE>{W.scal, Wv(lv), Bv(lv), Tv(lv), Xv(lv), nullptr,
                                                                             W.part, cap, W.counter},
                                              err, s));
            } else if (l == 0) {
                if (fin == FIN_PCG_BETA) {
                    VEC_DISPATCH(lv.vec_a, AMG_TRY(launch_k(k_postsmooth<V, double, TM, double, FIN_PCG_BETA>, grid_rows(n, V, cap), BLOCK, 0, s, 
                                               n, lv.A.rp, lv.A.ci, Av(lv.A), Wv(lv), b0, Tv(lv), z0, qprev, W.scal, W.part, cap, W.counter)));
                } else {
                    VEC_DISPATCH(lv.vec_a, AMG_TRY(launch_k(k_postsmooth<V, double, TM, double, FIN_NONE>, grid_rows(n, V, cap), BLOCK, 0, s, 
                                               n, lv.A.rp, lv.A.ci, Av(lv.A), Wv(lv), b0, Tv(lv), z0, nullptr, W.scal, W.part, cap, W.counter)));
                }
            } else {
                VEC_DISPATCH(lv.vec_a, AMG_TRY(launch_k(k_postsmooth<V, TM, TM, TM, FIN_NONE>, grid_rows(n, V, cap), BLOCK, 0, s, 
                                           n, lv.A.rp, lv.A.ci, Av(lv.A), Wv(lv), Bv(lv), Tv(lv), Xv(lv), nullptr, W.scal, W.part, cap, W.counter)));
            }
        }
        AMG_LAUNCH_CHECK();
    }
    return AMG_OK;
}

// b032: an FP32 copy of b0 (mixed form, may be null), read by the finest
// level's pre-smoothing and prolongation in place of converting b0.
static int vcycle(Hierarchy *h, Workspace &W, const double *b0, double *z0, int fin, cudaStream_t s,
                  const float *b032 = nullptr) {
    if (h->cfg.precision == AMG_PRECISION_MIXED && !h->cycle64)
        return launch_vcycle<float>(h, W, b0, z0, fin, s, b032);
    return launch_vcycle<double>(h, W, b0, z0, fin, s, nullptr);
}

static int stream_grid(int n, int cap) { return std::max(1, std::min((n + BLOCK - 1) / BLOCK, cap)); }

// q = A x with a finisher (the outer, FP64 operator).
template <int SF>
static int spmv_fin(Hierarchy *h, Workspace &W, const char *name, const double *x, double *y, const double *dvec,
                    cudaStream_t s, float *y32 = nullptr) {
    const int n = h->n, cap = W.part_cap;
    const Level &l0 = h->L[0];
    if constexpr (SF == SF_PCG_ALPHA) {
        if (h->krylov_df && x == W.p) {
            // the operation's algorithmic bytes, as for the FP64 product (this
            // launch also reads p itself for p.q beside the split copy it gathers)
            TRACE(name, 0, csr_bytes(l0.A, 8) + 16.0 * n);
            const OpFinDF op{W.scal, W.p, W.p2, y, W.part, cap, W.counter};
            if (l0.sa64.direct) AMG_TRY(stream_launch_direct<DF>(l0.sa64, n, l0.A.vdf, op, s));
            else AMG_TRY(stream_launch_ell<DF>(l0.sa64, n, l0.A.vdf, op, &W.scal->copy_timeout, s));
            return AMG_OK;
        }
    }
    TRACE(name, 0, csr_bytes(l0.A, 8) + 16.0 * n + (SF == SF_PCG_ALPHA ? 0.0 : 8.0 * n));
    if (l0.sa64.rt) {
        AMG_TRY(stream_launch<double>(l0.sa64, n, l0.A.rp, l0.A.ci, l0.A.v,
                                      OpFin<SF>{W.scal, x, y, dvec, W.part, cap, W.counter, y32}, &W.scal->copy_timeout, s));
        return AMG_OK;
    }
    VEC_DISPATCH(l0.vec_a, AMG_TRY(launch_k(k_spmv_fin<V, SF>, grid_rows(n, V, cap), BLOCK, 0, s, 
                               n, l0.A.rp, l0.A.ci, l0.A.v, x, y, y32, dvec, W.scal, W.part, cap, W.counter)));
    AMG_LAUNCH_CHECK();
    return AMG_OK;
}

// One PCG iteration: z = M r (with beta), p = z + beta p, q = A p (alpha), update.
static int pcg_iteration(Hierarchy *h, Workspace &W, cudaStream_t s) {
    const int n = h->n, cap = W.part_cap;
    const bool mixed = h->cfg.precision == AMG_PRECISION_MIXED;
    AMG_TRY(vcycle(h, W, W.r, W.z, FIN_PCG_BETA, s, mixed ? W.r32 : nullptr));
    {
        TRACE("pcg_p", 0, 24.0 * n);
        AMG_TRY(launch_k(k_pcg_p, stream_grid(n, cap), BLOCK, 0, s, n, W.z, W.p, h->krylov_df ? W.p2 : nullptr,
                         W.scal));
    }
    AMG_TRY(spmv_fin<SF_PCG_ALPHA>(h, W, "spmv_pq", W.p, W.q, W.p, s));
    {
        TRACE("pcg_update", 0, (mixed ? 52.0 : 48.0) * n);
        AMG_TRY(launch_k(k_pcg_update, stream_grid(n, cap), BLOCK, 0, s, n, W.x, W.r, W.p, W.q,
                         mixed ? W.r32 : nullptr, W.scal,
                                                           W.part, cap, W.counter, 0));
    }
    AMG_LAUNCH_CHECK();
    return AMG_OK;
}

static int cg_iteration(Hierarchy *h, Workspace &W, cudaStream_t s) {
    const int n = h->n, cap = W.part_cap;
    {
        TRACE("pcg_p", 0, 24.0 * n);
        AMG_TRY(launch_k(k_pcg_p, stream_grid(n, cap), BLOCK, 0, s, n, W.r, W.p, h->krylov_df ? W.p2 : nullptr,
                         W.scal));
    }
    AMG_TRY(spmv_fin<SF_PCG_ALPHA>(h, W, "spmv_pq", W.p, W.q, W.p, s));
    {
        TRACE("pcg_update", 0, 48.0 * n);
        AMG_TRY(launch_k(k_pcg_update, stream_grid(n, cap), BLOCK, 0, s, n, W.x, W.r, W.p, W.q, nullptr, W.scal,
                         W.part, cap, W.counter, 1));
    }
    AMG_LAUNCH_CHECK();
    return AMG_OK;
}

static int bicg_iteration(Hierarchy *h, Workspace &W, bool precond, cudaStream_t s) {
    const int n = h->n, cap = W.part_cap;
    // the mixed V-cycle reads FP32 copies of p and s (one buffer, used in turn)
    float *v32 = precond && h->cfg.precision == AMG_PRECISION_MIXED ? W.r32 : nullptr;
    {
        TRACE("bicg_p", 0, (v32 ? 36.0 : 32.0) * n);
        AMG_TRY(launch_k(k_bicg_p, stream_grid(n, cap), BLOCK, 0, s, n, W.r, W.p, W.v, v32, W.scal));
    }
    const double *ph = W.p;
    if (precond) {
        AMG_TRY(vcycle(h, W, W.p, W.ph, FIN_NONE, s, v32));
        ph = W.ph;
    }
    AMG_TRY(spmv_fin<SF_BICG_ALPHA>(h, W, "spmv_rv", ph, W.v, W.rh, s));
    {
        TRACE("bicg_s", 0, 48.0 * n);
        AMG_TRY(launch_k(k_bicg_s, stream_grid(n, cap), BLOCK, 0, s, n, W.r, W.v, W.s, v32, W.x, ph, W.scal, W.part, cap,
                         W.counter));
    }
    const double *sh = W.s;
    if (precond) {
        AMG_TRY(vcycle(h, W, W.s, W.sh, FIN_NONE, s, v32));
        sh = W.sh;
    }
    AMG_TRY(spmv_fin<SF_BICG_OMEGA>(h, W, "spmv_ts", sh, W.t, W.s, s));
    {
        TRACE("bicg_update", 0, 64.0 * n);
        AMG_TRY(launch_k(k_bicg_update, stream_grid(n, cap), BLOCK, 0, s, n, W.x, sh, W.r, W.s, W.t, W.rh, W.scal, W.part, cap, W.counter));
    }
    AMG_LAUNCH_CHECK();
    return AMG_OK;
}

static int iterate(Hierarchy *h, Workspace &W, int kind, cudaStream_t s) {
    switch (kind) {
        case 0: return cg_iteration(h, W, s);
        case 1: return pcg_iteration(h, W, s);
        case 2: return bicg_iteration(h, W, false, s);
        default: return bicg_iteration(h, W, true, s);
    }
}

// One Krylov iteration (kind: 0 CG, 1 PCG, 2 BiCGStab, 3 AMG-BiCGStab).  The
// iteration's kernels are captured once per hierarchy as a CUDA graph and
// replayed, which removes most of the per-launch cost of the ~25 kernels; the
// launch count still advances by the kernels the graph holds.  With
// per-kernel tracing on, the kernels are launched directly.
// `count` Krylov iterations: one CUDA graph (captured once per solver kind)
// whose iterations are chained by programmatic edges like the kernels within
// one, or, while tracing, plain launches.
static int run_iterations(Hierarchy *h, Workspace &W, int kind, int count, cudaStream_t s) {
    if (W.prof.on) {
        for (int k = 0; k < count; ++k) AMG_TRY(iterate(h, W, kind, s));
        return AMG_OK;
    }
    if (!h->iter_exec || h->iter_kind != kind || h->iter_count != count) {
        if (h->iter_exec) cudaGraphExecDestroy(h->iter_exec);
        h->iter_exec = nullptr;
        const long long before = W.prof.launches;
        AMG_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int rc = AMG_OK;
        for (int k = 0; k < count && rc >= 0; ++k) rc = iterate(h, W, kind, s);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(s, &g);
        if (rc < 0) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        AMG_CUDA_TRY(ce);
        const cudaError_t ie = cudaGraphInstantiate(&h->iter_exec, g, 0);
        cudaGraphDestroy(g);
        AMG_CUDA_TRY(ie);
        h->iter_kind = kind;
        h->iter_count = count;
        h->iter_kernels = (int)(W.prof.launches - before);
        W.prof.launches = before;
    }
    AMG_CUDA_TRY(cudaGraphLaunch(h->iter_exec, s));
    W.prof.launches += h->iter_kernels;
    return AMG_OK;
}

// Iterations in one pass of the device-side loop's body.  A pass ends in a
// one-thread condition kernel; after convergence the rest of a pass's
// kernels return at once, so two iterations a pass trade that overshoot
// against the condition launches.
constexpr int LOOP_ITERS = 2;

// The device-side loop for iteration kind `kind`: a graph holding one
// conditional WHILE node whose body -- LOOP_ITERS iterations and the
// condition kernel -- the GPU repeats until the solve is done, so a solve
// launches it once and synchronises once.  Built on first use per kind;
// returns false (and marks the hierarchy) where conditional nodes cannot be
// built, the host-polled graph then being used.
static bool build_loop(Hierarchy *h, Workspace &W, int kind, int cap, cudaStream_t s) {
    if (h->loop_kind == kind && h->loop_exec) return true;
    if (h->loop_kind == -2) return false;
    if (h->loop_exec) cudaGraphExecDestroy(h->loop_exec);
    if (h->loop_graph) cudaGraphDestroy(h->loop_graph);
    h->loop_exec = nullptr;
    h->loop_graph = nullptr;
    h->loop_kind = -2;
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    auto fail = [&]() {
        cudaGetLastError();
        cudaGraphDestroy(g);
        return false;
    };
    cudaGraphConditionalHandle hd;
    if (cudaGraphConditionalHandleCreate(&hd, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) return fail();
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hd;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) != cudaSuccess) return fail();
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail();
    const long long before = W.prof.launches;
    int rc = AMG_OK;
    for (int k = 0; k < LOOP_ITERS && rc >= 0; ++k) rc = iterate(h, W, kind, s);
    if (rc >= 0) rc = launch_k(k_loop_cond, 1, 1, 0, s, hd, W.scal, cap);
    cudaGraph_t got = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &got);
    if (rc < 0 || ce != cudaSuccess) return fail();
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) return fail();
    h->loop_graph = g;
    h->loop_exec = ex;
    h->loop_kind = kind;
    h->loop_kernels = (int)(W.prof.launches - before) + 1;  // and the condition kernel
    W.prof.launches = before;
    return true;
}

static int read_scalars(Workspace &W, cudaStream_t s) {
    AMG_CUDA_TRY(cudaMemcpyAsync(W.scal_h, W.scal, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    return AMG_OK;
}

// r = b - A x and ||r||^2 into scal->tr; the host reads the scalars.
static int true_residual(Hierarchy *h, Workspace &W, cudaStream_t s) {
    AMG_TRY(spmv_fin<SF_TRUE_RES>(h, W, "true_residual", W.x, W.r, W.b, s,
                                  h->cfg.precision == AMG_PRECISION_MIXED ? W.r32 : nullptr));
    return read_scalars(W, s);
}

static int set_control(Workspace &W, cudaStream_t s, int done, int status, int flexible, int max_iter, int reset) {
    TRACE("control", 0, 0.0);
    AMG_TRY(launch_k(k_set_control, 1, 1, 0, s, W.scal, done, status, flexible, max_iter, reset, W.gbar));
    AMG_LAUNCH_CHECK();
    return AMG_OK;
}

static int bicg_restart(Hierarchy *h, Workspace &W, cudaStream_t s) {
    const int n = h->n, cap = W.part_cap;
    TRACE("bicg_restart", 0, 32.0 * n);
    AMG_TRY(launch_k(k_bicg_restart, stream_grid(n, cap), BLOCK, 0, s, n, W.r, W.rh, W.p, W.v, W.scal, W.part, cap, W.counter));
    AMG_LAUNCH_CHECK();
    return AMG_OK;
}

int krylov_solve(Hierarchy *h, Workspace &W, cudaStream_t s, SolveResult *res) {
    const amg_config &c = h->cfg;
    const int n = h->n, cap = W.part_cap;
    const bool bicg = c.solver == AMG_SOLVER_BICGSTAB || c.solver == AMG_SOLVER_BICGSTAB_NOPREC;
    const bool precond = c.solver == AMG_SOLVER_PCG || c.solver == AMG_SOLVER_BICGSTAB;
    const int flexible = c.precision == AMG_PRECISION_MIXED ? 1 : 0;

    AMG_TRY(set_control(W, s, 0, AMG_OK, flexible, c.max_iter, 1));
    {
        TRACE(bicg ? "bicg_init" : "pcg_init", 0, (bicg ? 48.0 : 32.0) * n);
        if (bicg)
            AMG_TRY(launch_k(k_bicg_init, stream_grid(n, cap), BLOCK, 0, s, n, W.b, W.x, W.r, W.rh, W.p, W.v, W.scal, c.rtol, W.part,
                                                              cap, W.counter));
        else
            AMG_TRY(launch_k(k_pcg_init, stream_grid(n, cap), BLOCK, 0, s, n, W.b, W.x, W.r, W.p,
                             c.precision == AMG_PRECISION_MIXED ? W.r32 : nullptr, W.scal, c.rtol, W.part, cap,
                             W.counter, precond ? 0 : 1));
    }
    AMG_LAUNCH_CHECK();
    // The start's scalars (||b||^2, a failure) are read with the first
    // iterations': the start leaves done set for b = 0 or a non-finite b, so
    // those iterations return at once.
    int status = AMG_OK;
    int restarts = 0, bd_restarts = 0;
    bool first_read = true;
    // W.scal_h holds the scalars of a true residual of the current x
    bool fresh = false;
    const int chunk = 4;
    const int kind = bicg ? (precond ? 3 : 2) : (precond ? 1 : 0);
    long long launched = 0;
    const long long launch_cap = (long long)c.max_iter * (c.max_restarts + 2) + 4 * chunk;
    const int trip_cap = (int)std::min<long long>(INT_MAX - 1, launch_cap / LOOP_ITERS + 2);
    // PCG on a hierarchy that fits one cluster: each pass of the loop below
    // is one whole-solve launch; else the device-side loop, where conditional
    // graphs build (not while tracing)
    const bool cluster = c.device_loop && kind == 1 && h->cpcg_cta > 0;
    const bool device_loop = !cluster && c.device_loop && !W.prof.on && build_loop(h, W, kind, trip_cap, s);
    int trips_seen = 0;
    while (status == AMG_OK) {
        // iterate until the device marks the solve done; the device sets done
        // at max_iter at the latest, launch_cap only guards the host loop
        for (;;) {
            if (cluster) {
                AMG_TRY(launch_cpcg(h, W, s));
                launched += launch_cap / 2 + 1;  // one launch runs the solve to its end
                AMG_TRY(read_scalars(W, s));
            } else if (device_loop) {
                AMG_CUDA_TRY(cudaGraphLaunch(h->loop_exec, s));
                launched += launch_cap / 2 + 1;  // one launch runs the loop to its end
                AMG_TRY(read_scalars(W, s));
                // kernels launched: the body's (with its condition kernel) per pass
                W.prof.launches += (long long)h->loop_kernels * std::max(0, W.scal_h->trips - trips_seen);
                trips_seen = W.scal_h->trips;
            } else {
                AMG_TRY(run_iterations(h, W, kind, chunk, s));
                launched += chunk;
                AMG_TRY(read_scalars(W, s));
            }
            if (first_read) {
                first_read = false;
                if (W.scal_h->bn2 == 0.0 && W.scal_h->status == AMG_OK) {
                    // b = 0: x = 0 exactly
                    res->status = AMG_OK;
                    res->iters = 0;
                    res->restarts = 0;
                    res->rel_res_true = res->rel_res_rec = 0.0;
                    W.prof.collect();
                    return AMG_OK;
                }
            }
            if (W.scal_h->done) break;
            if (launched > launch_cap) {
                set_last_error("solver loop exceeded %lld iterations without finishing", launch_cap);
                return AMG_ERR_CUDA;
            }
        }
        status = W.scal_h->status;
        if (bicg && status == AMG_BREAKDOWN && bd_restarts < 1) {
            // restart once from the current x with r^ = r = b - A x
            bd_restarts++;
            AMG_TRY(true_residual(h, W, s));
            AMG_TRY(bicg_restart(h, W, s));
            AMG_TRY(read_scalars(W, s));
            status = W.scal_h->status;
            if (W.scal_h->done) break;
            continue;
        }
        // the cluster launch ends with the true residual of its final x
        const bool tr_done = cluster && W.scal_h->tr_fresh;
        if (status != AMG_OK) {
            fresh = tr_done;
            break;
        }
        // converged on the recursive residual: check the true residual
        if (!tr_done) AMG_TRY(true_residual(h, W, s));
        fresh = true;
        const double tr = W.scal_h->tr;
        if (tr <= W.scal_h->tol2) break;
        if (restarts >= c.max_restarts || W.scal_h->iters >= c.max_iter) {
            status = AMG_MAXIT;
            break;
        }
        restarts++;
        fresh = false;
        // r already holds b - A x; restart the recursion from the current x
        if (bicg) {
            AMG_TRY(bicg_restart(h, W, s));
        } else {
            AMG_TRY(set_control(W, s, 0, AMG_OK, flexible, c.max_iter, 0));
            TRACE("control", 0, 0.0);
            AMG_TRY(launch_k(k_pcg_restart, 1, 1, 0, s, W.scal, precond ? 0 : 1));
            AMG_LAUNCH_CHECK();
        }
    }
    if (!fresh) AMG_TRY(read_scalars(W, s));
    const double rec = W.scal_h->rr;
    res->iters = W.scal_h->iters;
    if (!fresh) AMG_TRY(true_residual(h, W, s));
    const double bn2 = W.scal_h->bn2;
    res->status = status;
    res->restarts = restarts;
    res->rel_res_true = sqrt(W.scal_h->tr / bn2);
    res->rel_res_rec = sqrt(rec / bn2);
    if (status == AMG_OK && !(res->rel_res_true <= c.rtol)) res->status = AMG_MAXIT;
    W.prof.collect();
    if (W.scal_h->copy_timeout) {
        set_last_error(W.scal_h->copy_timeout & 4   ? "a distributed-shared-memory wait of the whole-solve cluster launch timed out"
                       : W.scal_h->copy_timeout & 2 ? "a grid-barrier wait of the fused coarse levels timed out"
                                                  : "a bulk-copy wait in a streaming kernel timed out");
        return AMG_ERR_CUDA;
    }
    return AMG_OK;
}

int test_arm_wait_timeout(Workspace &W, int kind, cudaStream_t s) {
    static_assert(stream::TEST_WITHHOLD_COPY == AMG_TEST_WITHHOLD_COPY &&
                      mid::TEST_WITHHOLD_BARRIER == AMG_TEST_WITHHOLD_BARRIER,
                  "test control values");
    AMG_CUDA_TRY(cudaMemcpyAsync(&W.scal->test_ctl, &kind, sizeof(int), cudaMemcpyHostToDevice, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    return AMG_OK;
}

int vcycle_apply(Hierarchy *h, Workspace &W, const double *r, double *z, cudaStream_t s) {
    if (h->nc == 0) {
        set_last_error("amg_vcycle: the handle was set up for an unpreconditioned solver (no hierarchy)");
        return AMG_ERR_UNSUPPORTED;
    }
    AMG_TRY(set_control(W, s, 0, AMG_OK, 0, h->cfg.max_iter, 1));
    return vcycle(h, W, r, z, FIN_NONE, s);
}

// Average duration of the finest level's Krylov product with its finisher
// (PCG: q = A p, p.q, alpha; BiCGStab: v = A p, r^.v) over `reps`
// back-to-back launches on the handle's stream after two, on the workspace's
// current vectors (the last solve's).  Launches are chained exactly as in a
// solve (programmatic dependent launch), so the figure is the kernel's
// steady-state duration without the per-launch events of a trace.  The
// scalars' control fields are reset before and after.
int time_product(Hierarchy *h, Workspace &W, int reps, cudaStream_t s, double *us) {
    const bool bicg = h->cfg.solver == AMG_SOLVER_BICGSTAB || h->cfg.solver == AMG_SOLVER_BICGSTAB_NOPREC;
    auto one = [&]() -> int {
        if (bicg) return spmv_fin<SF_BICG_ALPHA>(h, W, "spmv_rv", W.p, W.v, W.rh, s);
        return spmv_fin<SF_PCG_ALPHA>(h, W, "spmv_pq", W.p, W.q, W.p, s);
    };
    AMG_TRY(set_control(W, s, 0, AMG_OK, 0, h->cfg.max_iter, 1));
    for (int k = 0; k < 2; ++k) AMG_TRY(one());
    cudaEvent_t e0, e1;
    AMG_CUDA_TRY(cudaEventCreate(&e0));
    AMG_CUDA_TRY(cudaEventCreate(&e1));
    int rc = AMG_OK;
    cudaEventRecord(e0, s);
    for (int k = 0; k < reps && rc >= 0; ++k) rc = one();
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (rc >= 0 && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    AMG_TRY(rc);
    AMG_TRY(read_scalars(W, s));
    const int stopped = W.scal_h->done;
    AMG_TRY(set_control(W, s, 1, AMG_OK, 0, h->cfg.max_iter, 1));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (stopped) {
        set_last_error("product timing: the finisher stopped on the current vectors (run a solve first)");
        return AMG_ERR_ARG;
    }
    *us = 1e3 * (double)ms / std::max(1, reps);
    return AMG_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: plan family by timed trial of whole cycles
// ---------------------------------------------------------------------------

// Every streaming plan of h (the order of for_each_plan).
static std::vector<StreamPlan> plans_of(Hierarchy *h) {
    std::vector<StreamPlan> v;
    for_each_plan(h, [&](StreamPlan &p) { v.push_back(p); });
    return v;
}

static void set_plans(Hierarchy *h, const std::vector<StreamPlan> &v) {
    size_t k = 0;
    for_each_plan(h, [&](StreamPlan &p) { p = v[k++]; });
}

// Best of three trials of four rounds (after two), a round being one V-cycle
// followed by the finest level's FP64 product -- the passes of one Krylov
// iteration, in their order -- on constant vectors, with h's current plans.
// The product's finisher (the true residual's) never stops the scalars, so
// every round does its full work.
static int time_rounds(Hierarchy *h, Workspace &W, cudaStream_t s, float *ms_out) {
    const int n = h->n;
    const bool mixed = h->cfg.precision == AMG_PRECISION_MIXED;
    k_fill<double><<<256, 256, 0, s>>>((size_t)n, 1.0, W.r);
    k_fill<double><<<256, 256, 0, s>>>((size_t)n, 1.0, W.b);
    k_fill<float><<<256, 256, 0, s>>>((size_t)n, 1.0f, W.r32);
    AMG_LAUNCH_CHECK();
    auto round = [&]() -> int {
        AMG_TRY(set_control(W, s, 0, AMG_OK, 0, h->cfg.max_iter, 1));
        if (h->nc > 0) AMG_TRY(vcycle(h, W, W.r, W.z, FIN_NONE, s, mixed ? W.r32 : nullptr));
        return spmv_fin<SF_TRUE_RES>(h, W, "true_residual", h->nc > 0 ? W.z : W.r, W.t, W.b, s);
    };
    cudaEvent_t e0, e1;
    AMG_CUDA_TRY(cudaEventCreate(&e0));
    AMG_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int rc = AMG_OK;
    for (int k = 0; k < 2 && rc >= 0; ++k) rc = round();
    for (int trial = 0; trial < 3 && rc >= 0; ++trial) {
        cudaEventRecord(e0, s);
        for (int k = 0; k < 4 && rc >= 0; ++k) rc = round();
        cudaEventRecord(e1, s);
        if (rc >= 0 && cudaEventSynchronize(e1) == cudaSuccess) {
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            best = std::min(best, t);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    AMG_TRY(rc);
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    *ms_out = best;
    return AMG_OK;
}

// The mixed form on a hierarchy whose whole cycle is one cluster launch (the
// tail from level 0): its operators sit in shared memory and L2, so the FP32
// cycle saves no DRAM traffic and only adds conversions; the rounds are timed
// with the FP32 and the FP64 cycle and the faster is kept.
static int tune_cycle_precision(Hierarchy *h, Workspace &W, cudaStream_t s) {
    h->cycle64 = 0;
    if (h->cfg.precision != AMG_PRECISION_MIXED || h->tail_start != 0 || h->nc == 0) return AMG_OK;
    AMG_TRY(time_rounds(h, W, s, &h->cycle_ms[0]));
    h->cycle64 = 1;
    AMG_TRY(time_rounds(h, W, s, &h->cycle_ms[1]));
    h->cycle64 = h->cycle_ms[1] < h->cycle_ms[0] ? 1 : 0;
    return AMG_OK;
}

static int autotune_layouts(Hierarchy *h, Workspace &W, cudaStream_t s);

// The mixed form's outer product q = A p: its plan launched in FP64 and in
// double-FP32 arithmetic, and, when the tile family won the cycle, the direct
// family's plan of the product both ways too.  Whole PCG iterations decide
// (the cycle, p = z + beta p -- which also writes the split p for the
// double-FP32 product -- the product and the update, launched as the solve
// launches them): a faster product alone measured slower iterations when it
// added the split's writes or put direct blocks between the cycle's tile
// rings.  The chosen plan in FP64 is kept unless another is 3 % faster.  Each
// iteration starts from reset scalars, so a finisher that stops on the
// constant vectors (p.Ap <= 0) stops none of the others.
static int tune_krylov_df(Hierarchy *h, Workspace &W, cudaStream_t s) {
    h->krylov_df = 0;
    Level &l0 = h->L[0];
    const StreamPlan alt = h->alt_sa64;
    h->alt_sa64 = StreamPlan{};
    auto df_ok = [&](const StreamPlan &p) { return (p.ell || p.direct) && l0.A.vdf && ell_values(p, l0.A.vdf); };
    // the double-FP32 product serves PCG and CG (BiCGStab's products stay FP64)
    const bool cg = h->cfg.solver == AMG_SOLVER_CG;
    if (h->cfg.precision != AMG_PRECISION_MIXED || h->cfg.outer_product == 0 || !df_ok(l0.sa64) ||
        !(cg || h->cfg.solver == AMG_SOLVER_PCG))
        return AMG_OK;
    if (h->cfg.outer_product == 1) {
        h->krylov_df = 1;
        return AMG_OK;
    }
    struct Cand {
        StreamPlan plan;
        int df;
    };
    std::vector<Cand> cands = {{l0.sa64, 0}, {l0.sa64, 1}};
    if (alt.direct && ell_values(alt, l0.A.v)) {
        cands.push_back({alt, 0});
        if (df_ok(alt)) cands.push_back({alt, 1});
    }
    const int n = h->n;
    for (double *v : {W.p, W.q, W.r, W.b}) k_fill<double><<<256, 256, 0, s>>>((size_t)n, 1.0, v);
    k_fill<double><<<256, 256, 0, s>>>((size_t)n, 0.0, W.x);
    k_fill<float><<<256, 256, 0, s>>>((size_t)n, 1.0f, W.r32);
    k_fill<DF><<<256, 256, 0, s>>>((size_t)n, DF(1.f, 0.f), W.p2);
    AMG_LAUNCH_CHECK();
    cudaEvent_t e0, e1;
    AMG_CUDA_TRY(cudaEventCreate(&e0));
    AMG_CUDA_TRY(cudaEventCreate(&e1));
    std::vector<float> best(cands.size(), 1e30f);
    const StreamPlan chosen = l0.sa64;
    int rc = AMG_OK;
    for (size_t q = 0; q < cands.size() && rc >= 0; ++q) {
        l0.sa64 = cands[q].plan;
        h->krylov_df = cands[q].df;
        auto one = [&]() -> int {
            AMG_TRY(set_control(W, s, 0, AMG_OK, cg ? 0 : 1, h->cfg.max_iter, 1));
            return cg ? cg_iteration(h, W, s) : pcg_iteration(h, W, s);
        };
        for (int k = 0; k < 2 && rc >= 0; ++k) rc = one();
        for (int trial = 0; trial < 3 && rc >= 0; ++trial) {
            cudaEventRecord(e0, s);
            for (int k = 0; k < 4 && rc >= 0; ++k) rc = one();
            cudaEventRecord(e1, s);
            if (rc >= 0 && cudaEventSynchronize(e1) == cudaSuccess) {
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                best[q] = std::min(best[q], t);
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    l0.sa64 = chosen;
    h->krylov_df = 0;
    AMG_TRY(rc);
    AMG_TRY(set_control(W, s, 1, AMG_OK, 0, h->cfg.max_iter, 1));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    size_t pick = 0;
    for (size_t q = 1; q < cands.size(); ++q)
        if (best[q] < 0.97f * best[0] && best[q] < best[pick]) pick = q;
    l0.sa64 = cands[pick].plan;
    h->krylov_df = cands[pick].df;
    h->krylov_us[0] = 250.f * best[0];  // ms for 4 iterations -> us per iteration
    h->krylov_us[1] = 250.f * best[pick];
    return AMG_OK;
}

// The autotuner: the streaming plans (autotune_layouts), then, in the mixed
// form, the outer product's arithmetic and, for a tail-only hierarchy, the
// cycle's precision.
int autotune_plans(Hierarchy *h, Workspace &W, cudaStream_t s) {
    AMG_TRY(autotune_layouts(h, W, s));
    AMG_TRY(tune_krylov_df(h, W, s));
    return tune_cycle_precision(h, W, s);
}

// With a requested layout, each operator's plan is the fastest of that
// layout in a timed trial of its own pass.  With AMG_LAYOUT_AUTO the two
// families are tuned apart -- the tile layouts (CSR, windowed and sliced-ELL
// tiles through a shared-memory ring) and the direct sliced-ELL layout -- and
// whole V-cycles with the finest product decide between them: a cycle that
// interleaves the two families runs slower than either alone (the persistent
// tile kernels' CTAs wait behind the direct kernels' blocks), which the
// per-pass trials cannot see.
static int autotune_layouts(Hierarchy *h, Workspace &W, cudaStream_t s) {
    if (h->cfg.layout == AMG_LAYOUT_TILES) return tune_all(h, LAYOUT_TILES, s);
    if (h->cfg.layout != AMG_LAYOUT_AUTO) return tune_all(h, h->cfg.layout, s);
    const std::vector<StreamPlan> base = plans_of(h);
    AMG_TRY(tune_all(h, LAYOUT_TILES, s));
    const std::vector<StreamPlan> tiles = plans_of(h);
    set_plans(h, base);
    AMG_TRY(tune_all(h, AMG_LAYOUT_ELL_DIRECT, s));
    const std::vector<StreamPlan> direct = plans_of(h);
    bool any_direct = false;
    for (const StreamPlan &p : direct) any_direct |= p.direct != 0;
    if (!any_direct) {
        set_plans(h, tiles);
        return AMG_OK;
    }
    float ms_tiles = 0.f, ms_direct = 0.f;
    set_plans(h, tiles);
    AMG_TRY(time_rounds(h, W, s, &ms_tiles));
    set_plans(h, direct);
    AMG_TRY(time_rounds(h, W, s, &ms_direct));
    if (ms_tiles <= ms_direct) {
        set_plans(h, tiles);
        h->alt_sa64 = direct[4];  // level 0's Krylov plan (the order of for_each_plan)
        if (!h->alt_sa64.direct) h->alt_sa64 = StreamPlan{};
    }
    h->plan_family_ms[0] = ms_tiles;
    h->plan_family_ms[1] = ms_direct;
    return AMG_OK;
}

int grad_values(Hierarchy *h, Workspace &W, const double *lambda, const double *x, double *dA, cudaStream_t s) {
    const Level &l0 = h->L[0];
    const int n = h->n;
    TRACE("grad_values", 0, csr_bytes(l0.A, 0) + 16.0 * n + 8.0 * l0.A.nnz);
    VEC_DISPATCH(l0.vec_a, AMG_TRY(launch_k(k_grad_values<V>, grid_rows(n, V, num_sms() * 8), BLOCK, 0, s, 
                               n, l0.A.rp, l0.A.ci, lambda, x, dA)));
    AMG_LAUNCH_CHECK();
    return AMG_OK;
}

}  // namespace amg
