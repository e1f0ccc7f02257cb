// noalloc.cu -- amg_cg_solve_noalloc: conjugate gradients on a caller's CSR
// matrix without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// solve: code running inside a framework that owns all device memory and
// forbids allocation while it executes (a memory-planned runtime or a custom
// operator that may only use the buffers it is handed), or a latency-critical
// loop where a cudaMalloc would stall every stream.  amg_setup allocates the
// whole hierarchy, so those callers cannot use a handle.  This entry point
// needs nothing but the caller's arrays: its work vectors (r, p, q), the
// per-block partial sums and the Krylov scalars live in one file-scope
// __device__ array of fixed size.  Under CUDA's lazy module loading the
// array's device memory is committed when this file's module first loads on a
// device -- inside the first call there -- and held until the process exits,
// so a caller makes one warm-up call before a region that must not allocate.
//
// The iteration is the same unpreconditioned CG as amg_solve with
// AMG_SOLVER_CG: x0 = 0, stop when ||r||_2 <= rtol ||b||_2 on the recursive
// residual, then restart from x while the true residual b - A x is above the
// tolerance (at most 3 restarts).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "amg_common.cuh"

namespace {

constexpr int NA_BLOCK = 256;
constexpr int NA_MAX_N = AMG_NOALLOC_MAX_N;   // rows the scratch holds
constexpr int NA_PARTS = 1024;                // partial sums (at most this many blocks)
constexpr int NA_RESTARTS = 3;

struct NaScalars {
    double bn2, tol2, rr, rz, pq, alpha, beta, tr;
    int done, status, iters, first, max_iter;
    unsigned ticket;
};

// r, p, q (NA_MAX_N each), NA_PARTS partial sums, then the scalars.
constexpr size_t NA_SCALAR_DOUBLES = (sizeof(NaScalars) + sizeof(double) - 1) / sizeof(double);
constexpr size_t NA_DOUBLES = 3 * (size_t)NA_MAX_N + NA_PARTS + NA_SCALAR_DOUBLES + 8;

static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

struct NaView {
    double *r, *p, *q, *part;
    NaScalars *sc;
};

__host__ __device__ inline NaView carve(double *base) {
    NaView v;
    v.r = base;
    v.p = base + NA_MAX_N;
    v.q = base + 2 * (size_t)NA_MAX_N;
    v.part = base + 3 * (size_t)NA_MAX_N;
    v.sc = reinterpret_cast<NaScalars *>(base + 3 * (size_t)NA_MAX_N + NA_PARTS);
    return v;
}

// Per-device address of g_noalloc_scratch, looked up once with the device current.
std::mutex g_na_mutex;
double *g_na_ptr[64] = {nullptr};

int scratch_address(double **out) {
    int dev = 0;
    AMG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        amg::set_last_error("amg_cg_solve_noalloc: device ordinal %d out of range", dev);
        return AMG_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            amg::set_last_error("amg_cg_solve_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return AMG_ERR_CUDA;
        }
        g_na_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_na_ptr[dev];
    return AMG_OK;
}

// Deterministic block reduction; the last block adds the partials in block order.
template <int NV>
__device__ bool na_reduce_last(double (&v)[NV], double *part, unsigned *ticket, double (&tot)[NV]) {
    __shared__ double sh[NV][NA_BLOCK / 32];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < NV; ++k) {
        double a = amg::warp_sum(v[k]);
        if (lane == 0) sh[k][wid] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < NV; ++k) {
            double a = 0.0;
            for (int w = 0; w < NA_BLOCK / 32; ++w) a += sh[k][w];
            part[k * (NA_PARTS / NV) + blockIdx.x] = a;
        }
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    for (int k = 0; k < NV; ++k) {
        double a = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += NA_BLOCK) a += __ldcg(&part[k * (NA_PARTS / NV) + b]);
        a = amg::warp_sum(a);
        __syncthreads();
        if (lane == 0) sh[k][wid] = a;
        __syncthreads();
        double t = 0.0;
        for (int w = 0; w < NA_BLOCK / 32; ++w) t += sh[k][w];
        tot[k] = t;
    }
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

__global__ void na_init(int n, const double *__restrict__ b, double *x, NaView s, double rtol, int max_iter) {
    double acc[1] = {0.0};
    for (int i = blockIdx.x * NA_BLOCK + threadIdx.x; i < n; i += gridDim.x * NA_BLOCK) {
        const double bi = b[i];
        x[i] = 0.0;
        s.r[i] = bi;
        s.p[i] = 0.0;
        acc[0] += bi * bi;
    }
    double tot[1];
    if (na_reduce_last<1>(acc, s.part, &s.sc->ticket, tot) && threadIdx.x == 0) {
        NaScalars *c = s.sc;
        c->bn2 = tot[0];
        c->tol2 = rtol * rtol * tot[0];
        c->rr = tot[0];
        c->iters = 0;
        c->first = 1;
        c->max_iter = max_iter;
        c->status = AMG_OK;
        c->done = 0;
        if (!isfinite(tot[0])) { c->status = AMG_NAN; c->done = 1; }
        else if (tot[0] == 0.0) c->done = 1;
    }
}

// rz = r.r, beta = rz / rz_old (0 right after a (re)start)
__global__ void na_beta(int n, NaView s) {
    if (s.sc->done) return;
    double acc[1] = {0.0};
    for (int i = blockIdx.x * NA_BLOCK + threadIdx.x; i < n; i += gridDim.x * NA_BLOCK) acc[0] += s.r[i] * s.r[i];
    double tot[1];
    if (na_reduce_last<1>(acc, s.part, &s.sc->ticket, tot) && threadIdx.x == 0) {
        NaScalars *c = s.sc;
        if (!isfinite(tot[0])) { c->status = AMG_NAN; c->done = 1; return; }
        c->beta = c->first ? 0.0 : tot[0] / c->rz;
        c->first = 0;
        c->rz = tot[0];
    }
}

// p = r + beta p
__global__ void na_p(int n, NaView s) {
    if (s.sc->done) return;
    const double beta = s.sc->beta;
    for (int i = blockIdx.x * NA_BLOCK + threadIdx.x; i < n; i += gridDim.x * NA_BLOCK)
        s.p[i] = beta == 0.0 ? s.r[i] : s.r[i] + beta * s.p[i];
}

// q = A p (8 threads per row), alpha = rz / p.q;  or, with TRUE_RES, r = b - A x and ||r||^2.
template <bool TRUE_RES>
__global__ void na_spmv(int n, const int *__restrict__ rp, const int *__restrict__ ci, const double *__restrict__ v,
                        const double *__restrict__ xin, const double *__restrict__ b, NaView s) {
    if (!TRUE_RES && s.sc->done) return;
    constexpr int VEC = 8;
    double acc[1] = {0.0};
    const int lane = threadIdx.x & (VEC - 1);
    const int sub = (threadIdx.x & 31) / VEC;
    const int warp = (blockIdx.x * NA_BLOCK + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * NA_BLOCK) >> 5;
    for (int base = warp * (32 / VEC); base < n; base += nwarps * (32 / VEC)) {
        const int i = base + sub;
        const bool valid = i < n;
        double sum = 0.0;
        if (valid)
            for (int k = rp[i] + lane; k < rp[i + 1]; k += VEC) sum += v[k] * xin[ci[k]];
        sum = amg::group_sum<VEC>(sum);
        if (valid && lane == 0) {
            if (TRUE_RES) {
                const double ri = b[i] - sum;
                s.r[i] = ri;
                acc[0] += ri * ri;
            } else {
                s.q[i] = sum;
                acc[0] += xin[i] * sum;
            }
        }
    }
    double tot[1];
    if (na_reduce_last<1>(acc, s.part, &s.sc->ticket, tot) && threadIdx.x == 0) {
        NaScalars *c = s.sc;
        if (TRUE_RES) {
            c->tr = tot[0];
        } else if (!isfinite(tot[0])) {
            c->status = AMG_NAN;
            c->done = 1;
        } else if (tot[0] <= 0.0) {
            c->status = AMG_BREAKDOWN;
            c->done = 1;
        } else {
            c->pq = tot[0];
            c->alpha = c->rz / tot[0];
        }
    }
}

// x += alpha p; r -= alpha q; ||r||^2; convergence and the iteration cap.
__global__ void na_update(int n, double *x, NaView s) {
    if (s.sc->done) return;
    const double alpha = s.sc->alpha;
    double acc[1] = {0.0};
    for (int i = blockIdx.x * NA_BLOCK + threadIdx.x; i < n; i += gridDim.x * NA_BLOCK) {
        x[i] += alpha * s.p[i];
        const double ri = s.r[i] - alpha * s.q[i];
        s.r[i] = ri;
        acc[0] += ri * ri;
    }
    double tot[1];
    if (na_reduce_last<1>(acc, s.part, &s.sc->ticket, tot) && threadIdx.x == 0) {
        NaScalars *c = s.sc;
        c->iters += 1;
        c->rr = tot[0];
        if (!isfinite(tot[0])) { c->status = AMG_NAN; c->done = 1; }
        else if (tot[0] <= c->tol2) c->done = 1;
        else if (c->iters >= c->max_iter) { c->status = AMG_MAXIT; c->done = 1; }
    }
}

// Restart the recursion from the current x: r already holds b - A x.
__global__ void na_restart(NaView s) {
    s.sc->done = 0;
    s.sc->status = AMG_OK;
    s.sc->first = 1;
}

// True when p is device (or managed) memory of device `dev`, the device the
// kernels run on: memory of another GPU would be dereferenced from this one.
bool device_accessible(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

int read_scalars(const NaScalars *dev_sc, NaScalars *host, cudaStream_t st) {
    AMG_CUDA_TRY(cudaMemcpyAsync(host, dev_sc, sizeof(NaScalars), cudaMemcpyDeviceToHost, st));
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    return AMG_OK;
}

}  // namespace

extern "C" int amg_cg_solve_noalloc(int n, long long nnz, const int *row_ptr, const int *col_idx,
                                    const double *values, const double *b, double *x, double rtol, int max_iter,
                                    void *cuda_stream, amg_info *info) {
    if (n <= 0 || nnz < 0 || !row_ptr || !col_idx || !values || !b || !x || !(rtol > 0.0) || max_iter < 1) {
        amg::set_last_error("amg_cg_solve_noalloc: invalid argument (n=%d, nnz=%lld)", n, nnz);
        return AMG_ERR_ARG;
    }
    if (n > NA_MAX_N) {
        amg::set_last_error("amg_cg_solve_noalloc: n = %d exceeds the %d rows its fixed scratch holds", n, NA_MAX_N);
        return AMG_ERR_UNSUPPORTED;
    }
    if (nnz >= (1LL << 31)) {
        amg::set_last_error("amg_cg_solve_noalloc: nnz = %lld exceeds the int32 index range", nnz);
        return AMG_ERR_UNSUPPORTED;
    }
    int dev = 0;
    AMG_CUDA_TRY(cudaGetDevice(&dev));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (st) {
        // a stream of another device would run the kernels there
        int sdev = -1;
        AMG_CUDA_TRY(cudaStreamGetDevice(st, &sdev));
        if (sdev != dev) {
            amg::set_last_error("amg_cg_solve_noalloc: the stream belongs to device %d, the current device is %d", sdev,
                                dev);
            return AMG_ERR_ARG;
        }
    }
    const void *ptrs[] = {row_ptr, col_idx, values, b, x};
    for (const void *p : ptrs)
        if (!device_accessible(p, dev)) {
            amg::set_last_error("amg_cg_solve_noalloc: every array must be device memory of the current device %d "
                                "(no staging without allocation)", dev);
            return AMG_ERR_ARG;
        }
    double *base = nullptr;
    AMG_TRY(scratch_address(&base));
    const NaView s = carve(base);
    int sms = 148;
    AMG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::max(1, std::min((n + NA_BLOCK - 1) / NA_BLOCK, std::min(NA_PARTS, sms * 4)));
    const int grid_spmv = std::max(1, std::min((n + NA_BLOCK / 8 - 1) / (NA_BLOCK / 8), std::min(NA_PARTS, sms * 4)));

    // the ticket counter must start at zero (the scratch keeps the last call's contents)
    AMG_CUDA_TRY(cudaMemsetAsync(&s.sc->ticket, 0, sizeof(unsigned), st));
    na_init<<<grid, NA_BLOCK, 0, st>>>(n, b, x, s, rtol, max_iter);
    AMG_LAUNCH_CHECK();
    NaScalars h;
    AMG_TRY(read_scalars(s.sc, &h, st));
    int status = h.status, restarts = 0;
    const double bn2 = h.bn2;
    if (bn2 == 0.0 && status == AMG_OK) {
        if (info) {
            memset(info, 0, sizeof(*info));
        }
        return AMG_OK;
    }
    const long long cap = (long long)max_iter * (NA_RESTARTS + 2) + 16;
    long long launched = 0;
    bool have_true = false;  // h.tr holds ||b - A x||^2 of the final x
    while (status == AMG_OK) {
        for (;;) {
            for (int k = 0; k < 4; ++k) {
                na_beta<<<grid, NA_BLOCK, 0, st>>>(n, s);
                na_p<<<grid, NA_BLOCK, 0, st>>>(n, s);
                na_spmv<false><<<grid_spmv, NA_BLOCK, 0, st>>>(n, row_ptr, col_idx, values, s.p, nullptr, s);
                na_update<<<grid, NA_BLOCK, 0, st>>>(n, x, s);
            }
            AMG_LAUNCH_CHECK();
            launched += 4;
            AMG_TRY(read_scalars(s.sc, &h, st));
            if (h.done) break;
            if (launched > cap) {
                amg::set_last_error("amg_cg_solve_noalloc: iteration loop did not finish");
                return AMG_ERR_CUDA;
            }
        }
        status = h.status;
        if (status != AMG_OK) break;
        na_spmv<true><<<grid_spmv, NA_BLOCK, 0, st>>>(n, row_ptr, col_idx, values, x, b, s);
        AMG_LAUNCH_CHECK();
        AMG_TRY(read_scalars(s.sc, &h, st));
        if (h.tr <= h.tol2) {
            have_true = true;  // x is final: its true residual is already known
            break;
        }
        if (restarts >= NA_RESTARTS || h.iters >= max_iter) {
            status = AMG_MAXIT;
            break;
        }
        restarts++;
        na_restart<<<1, 1, 0, st>>>(s);
        AMG_LAUNCH_CHECK();
    }
    const double rec = h.rr;
    const int iters = h.iters;
    if (!have_true) {
        na_spmv<true><<<grid_spmv, NA_BLOCK, 0, st>>>(n, row_ptr, col_idx, values, x, b, s);
        AMG_LAUNCH_CHECK();
        AMG_TRY(read_scalars(s.sc, &h, st));
    }
    const double rel_true = sqrt(h.tr / bn2);
    if (status == AMG_OK && !(rel_true <= rtol)) status = AMG_MAXIT;
    if (info) {
        memset(info, 0, sizeof(*info));
        info->status = status;
        info->iters = iters;
        info->restarts = restarts;
        info->rel_res_true = rel_true;
        info->rel_res_rec = sqrt(rec / bn2);
    }
    return status;
}
