// api.cu -- the C ABI of libamgb300 (declared in include/amg_b300.h).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <new>

#include "solve.cuh"

namespace amg {
const char *last_error();
}

using namespace amg;

struct amg_handle_s {
    Hierarchy H;              // hierarchy of A
    Hierarchy *HT = nullptr;  // hierarchy of A^T (nonsymmetric adjoint), built on first use
    Workspace W;
    amg_batch_ws *BW = nullptr;  // batched handles only
    cudaStream_t s = nullptr; // private stream; ordered after/before the caller's stream by events
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // side stream of the adjoint's host copy of x (created on first use)
    cudaStream_t s_aux = nullptr;
    cudaEvent_t ev_aux0 = nullptr, ev_aux1 = nullptr;
    double *dA_stage = nullptr;  // device staging of dL/dA for host outputs
    DevArena extra;
    SolveResult last;
    double last_solve_ms = 0.0;
};

namespace {

using clk = std::chrono::steady_clock;

int check_config(const amg_config &c) {
    if (c.solver < 0 || c.solver > 3 || (c.smoother != 0 && c.smoother != 1) || !(c.omega > 0.0) ||
        !(c.theta >= 0.0) || c.coarse_max < 1 || c.max_levels < 1 || c.max_levels > AMG_MAX_LEVELS ||
        !(c.rtol > 0.0) || c.max_iter < 1 || c.max_restarts < 0 || (c.precision != 0 && c.precision != 1) ||
        c.symmetric < -1 || c.symmetric > 1 || c.layout < AMG_LAYOUT_AUTO || c.layout > AMG_LAYOUT_TILES ||
        (c.adjoint_reuse != 0 && c.adjoint_reuse != 1) ||
        (c.amg_type != AMG_TYPE_AGGREGATION && c.amg_type != AMG_TYPE_CLASSICAL) ||
        c.fuse_coarse < 0 || c.fuse_coarse > 2 || (c.device_loop != 0 && c.device_loop != 1) ||
        c.outer_product < -1 || c.outer_product > 1) {
        set_last_error("invalid amg_config");
        return AMG_ERR_ARG;
    }
    return AMG_OK;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Orders the private stream after the caller's stream.
int enter(amg_handle h, void *cuda_stream) {
    cudaStream_t us = (cudaStream_t)cuda_stream;
    AMG_CUDA_TRY(cudaEventRecord(h->ev_in, us));
    AMG_CUDA_TRY(cudaStreamWaitEvent(h->s, h->ev_in, 0));
    return AMG_OK;
}

// Orders the caller's stream after the private stream.
int leave(amg_handle h, void *cuda_stream, bool sync) {
    cudaStream_t us = (cudaStream_t)cuda_stream;
    AMG_CUDA_TRY(cudaEventRecord(h->ev_out, h->s));
    AMG_CUDA_TRY(cudaStreamWaitEvent(us, h->ev_out, 0));
    if (sync) AMG_CUDA_TRY(cudaStreamSynchronize(h->s));
    return AMG_OK;
}

void fill_info(amg_handle h, const Hierarchy &H, amg_info *info) {
    memset(info, 0, sizeof(*info));
    info->status = h->last.status;
    info->iters = h->last.iters;
    info->restarts = h->last.restarts;
    info->rel_res_true = h->last.rel_res_true;
    info->rel_res_rec = h->last.rel_res_rec;
    info->nlevels = H.nlevels;
    long long tot = 0;
    for (int l = 0; l < H.nlevels; ++l) {
        info->rows[l] = H.L[l].A.nrows;
        info->nnz[l] = H.L[l].A.nnz;
        tot += H.L[l].A.nnz;
    }
    info->operator_complexity = H.nnz ? (double)tot / (double)H.nnz : 0.0;
    info->setup_ms = H.setup_ms;
    info->solve_ms = h->last_solve_ms;
}

void destroy(amg_handle h) {
    if (!h) return;
    if (h->s) cudaStreamSynchronize(h->s);
    free_hierarchy(&h->H);
    if (h->HT) {
        free_hierarchy(h->HT);
        delete h->HT;
    }
    workspace_free(h->W);
    batch_destroy(h->BW);
    h->extra.free_all();
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->ev_aux0) cudaEventDestroy(h->ev_aux0);
    if (h->ev_aux1) cudaEventDestroy(h->ev_aux1);
    if (h->s_aux) cudaStreamDestroy(h->s_aux);
    if (h->s) cudaStreamDestroy(h->s);
    delete h;
}

int single_only(amg_handle h, const char *fn) {
    if (h->H.nsys > 0) {
        set_last_error("%s: the handle holds a batch of systems (use amg_solve_batched)", fn);
        return AMG_ERR_ARG;
    }
    return AMG_OK;
}

int make_handle(amg_handle *out, void *cuda_stream) {
    amg_handle h = new (std::nothrow) amg_handle_s();
    if (!h) return AMG_ERR_OOM;
    if (cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        set_last_error("stream/event creation failed: %s", cudaGetErrorString(cudaGetLastError()));
        destroy(h);
        return AMG_ERR_CUDA;
    }
    const int rc = enter(h, cuda_stream);
    if (rc < 0) {
        destroy(h);
        return rc;
    }
    *out = h;
    return AMG_OK;
}

int run_solve(amg_handle h, Hierarchy *H, cudaStream_t s) {
    const auto t0 = clk::now();
    SolveResult r;
    int rc = krylov_solve(H, h->W, s, &r);
    h->last_solve_ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    if (rc < 0) return rc;
    h->last = r;
    return r.status;
}

}  // namespace

extern "C" {

int amg_config_default(amg_config *c) {
    if (!c) return AMG_ERR_ARG;
    c->solver = AMG_SOLVER_PCG;
    c->smoother = AMG_SMOOTHER_JACOBI;
    c->omega = 2.0 / 3.0;
    c->theta = 0.08;
    c->coarse_max = 64;
    c->max_levels = 20;
    c->rtol = 1e-8;
    c->max_iter = 500;
    c->max_restarts = 3;
    c->precision = AMG_PRECISION_FP64;
    c->symmetric = -1;
    c->layout = AMG_LAYOUT_AUTO;
    c->adjoint_reuse = 0;
    c->amg_type = AMG_TYPE_AGGREGATION;
    c->fuse_coarse = 1;
    c->device_loop = 1;
    c->outer_product = -1;
    return AMG_OK;
}

int amg_setup(const amg_config *cfg, int n, long long nnz, const int *row_ptr, const int *col_idx,
              const double *values, void *cuda_stream, amg_handle *out) {
    if (!out) return AMG_ERR_ARG;
    *out = nullptr;
    if (n <= 0 || nnz < n || nnz >= (1LL << 31) - 1 || !row_ptr || !col_idx || !values) {
        set_last_error("amg_setup: invalid sizes or null array (n=%d, nnz=%lld)", n, nnz);
        return AMG_ERR_ARG;
    }
    amg_config c;
    if (cfg) c = *cfg;
    else amg_config_default(&c);
    AMG_TRY(check_config(c));
    amg_handle h = new (std::nothrow) amg_handle_s();
    if (!h) return AMG_ERR_OOM;
    const auto t0 = clk::now();
    int rc = AMG_OK;
    do {
        if (cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess) {
            set_last_error("amg_setup: stream/event creation failed: %s", cudaGetErrorString(cudaGetLastError()));
            rc = AMG_ERR_CUDA;
            break;
        }
        if ((rc = enter(h, cuda_stream)) < 0) break;
        h->H.cfg = c;
        h->H.n = n;
        h->H.nnz = nnz;
        if ((rc = build_hierarchy(&h->H, row_ptr, col_idx, values, h->s)) != AMG_OK) break;
        if ((rc = workspace_init(h->W, n)) < 0) break;
        if ((rc = autotune_plans(&h->H, h->W, h->s)) < 0) break;
        if ((rc = leave(h, cuda_stream, true)) < 0) break;
    } while (0);
    if (rc != AMG_OK) {
        destroy(h);
        return rc;
    }
    h->H.setup_ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    *out = h;
    return AMG_OK;
}

int amg_solve(amg_handle h, const double *b, double *x, void *cuda_stream, amg_info *info) {
    if (!h || !b || !x) return AMG_ERR_ARG;
    AMG_TRY(single_only(h, "amg_solve"));
    const int n = h->H.n;
    AMG_TRY(enter(h, cuda_stream));
    AMG_CUDA_TRY(cudaMemcpyAsync(h->W.b, b, sizeof(double) * n, cudaMemcpyDefault, h->s));
    int rc = run_solve(h, &h->H, h->s);
    if (rc < 0) return rc;
    AMG_CUDA_TRY(cudaMemcpyAsync(x, h->W.x, sizeof(double) * n, cudaMemcpyDefault, h->s));
    AMG_TRY(leave(h, cuda_stream, info != nullptr || !is_device_ptr(x)));
    if (info) fill_info(h, h->H, info);
    return rc;
}

int amg_adjoint(amg_handle h, const double *x, const double *g, double *lambda, double *dA, void *cuda_stream,
                amg_info *info) {
    if (!h || !x || !g) return AMG_ERR_ARG;
    AMG_TRY(single_only(h, "amg_adjoint"));
    const int n = h->H.n;
    const long long nnz = h->H.nnz;
    AMG_TRY(enter(h, cuda_stream));
    Hierarchy *H = &h->H;
    if (!h->H.symmetric) {
        if (!h->HT) {
            // A^T: transpose on the device, then a full setup of its own, or
            // (adjoint_reuse, preconditioned solvers) the transpose of A's hierarchy
            Hierarchy *HT = new (std::nothrow) Hierarchy();
            if (!HT) return AMG_ERR_OOM;
            DevArena tmp;
            DevCSR At;
            const bool reuse = h->H.cfg.adjoint_reuse && h->H.nc > 0;
            int rc = reuse ? AMG_OK : transpose_csr(h->H.L[0].A, At, tmp, h->s);
            if (rc == AMG_OK && reuse) {
                const auto t0 = clk::now();
                rc = build_transposed_hierarchy(HT, &h->H, h->s);
                if (rc == AMG_OK) rc = autotune_plans(HT, h->W, h->s);
                HT->setup_ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
            } else if (rc == AMG_OK) {
                HT->cfg = h->H.cfg;
                HT->cfg.symmetric = 0;
                HT->n = n;
                HT->nnz = nnz;
                const auto t0 = clk::now();
                rc = build_hierarchy(HT, At.rp, At.ci, At.v, h->s);
                if (rc == AMG_OK) rc = autotune_plans(HT, h->W, h->s);
                HT->setup_ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
            }
            cudaStreamSynchronize(h->s);
            tmp.free_all();
            if (rc != AMG_OK) {
                free_hierarchy(HT);
                delete HT;
                return rc;
            }
            h->HT = HT;
        }
        H = h->HT;
    }
    // x is read only by the gradient, after the solve.  On the device the
    // gradient reads it in place; from the host it is copied on a side stream
    // while the solve runs (after the work already queued on the private
    // stream, which may still read W.aux).
    const double *xg = x;
    bool side = false;
    auto overlaps = [](const void *a, size_t na, const void *b, size_t nb) {
        const char *pa = static_cast<const char *>(a), *pb = static_cast<const char *>(b);
        return b && pa < pb + nb && pb < pa + na;
    };
    const size_t xb = sizeof(double) * n;
    if (dA && is_device_ptr(x) &&
        (overlaps(x, xb, lambda, xb) || overlaps(x, xb, dA, sizeof(double) * (size_t)nnz))) {
        // x shares memory with an output written before the gradient reads it
        AMG_CUDA_TRY(cudaMemcpyAsync(h->W.aux, x, xb, cudaMemcpyDefault, h->s));
        xg = h->W.aux;
    } else if (dA && !is_device_ptr(x)) {
        if (!h->s_aux && (cudaStreamCreateWithFlags(&h->s_aux, cudaStreamNonBlocking) != cudaSuccess ||
                          cudaEventCreateWithFlags(&h->ev_aux0, cudaEventDisableTiming) != cudaSuccess ||
                          cudaEventCreateWithFlags(&h->ev_aux1, cudaEventDisableTiming) != cudaSuccess)) {
            set_last_error("amg_adjoint: side stream not created");
            return AMG_ERR_CUDA;
        }
        AMG_CUDA_TRY(cudaEventRecord(h->ev_aux0, h->s));
        AMG_CUDA_TRY(cudaStreamWaitEvent(h->s_aux, h->ev_aux0, 0));
        AMG_CUDA_TRY(cudaMemcpyAsync(h->W.aux, x, sizeof(double) * n, cudaMemcpyDefault, h->s_aux));
        AMG_CUDA_TRY(cudaEventRecord(h->ev_aux1, h->s_aux));
        xg = h->W.aux;
        side = true;
    }
    AMG_CUDA_TRY(cudaMemcpyAsync(h->W.b, g, sizeof(double) * n, cudaMemcpyDefault, h->s));
    int rc = run_solve(h, H, h->s);
    if (rc < 0) {
        if (side) cudaStreamSynchronize(h->s_aux);  // the copy reads the caller's buffer
        return rc;
    }
    // W.x = lambda
    bool host_out = false;
    if (lambda) {
        AMG_CUDA_TRY(cudaMemcpyAsync(lambda, h->W.x, sizeof(double) * n, cudaMemcpyDefault, h->s));
        host_out |= !is_device_ptr(lambda);
    }
    if (dA) {
        if (side) AMG_CUDA_TRY(cudaStreamWaitEvent(h->s, h->ev_aux1, 0));
        if (is_device_ptr(dA)) {
            AMG_TRY(grad_values(&h->H, h->W, h->W.x, xg, dA, h->s));
        } else {
            if (!h->dA_stage) AMG_TRY(h->extra.alloc(&h->dA_stage, (size_t)nnz));
            AMG_TRY(grad_values(&h->H, h->W, h->W.x, xg, h->dA_stage, h->s));
            AMG_CUDA_TRY(cudaMemcpyAsync(dA, h->dA_stage, sizeof(double) * nnz, cudaMemcpyDefault, h->s));
            host_out = true;
        }
    }
    AMG_TRY(leave(h, cuda_stream, info != nullptr || host_out));
    if (info) fill_info(h, *H, info);
    return rc;
}

int amg_vcycle(amg_handle h, const double *r, double *z, void *cuda_stream) {
    if (!h || !r || !z) return AMG_ERR_ARG;
    AMG_TRY(single_only(h, "amg_vcycle"));
    const int n = h->H.n;
    AMG_TRY(enter(h, cuda_stream));
    AMG_CUDA_TRY(cudaMemcpyAsync(h->W.b, r, sizeof(double) * n, cudaMemcpyDefault, h->s));
    AMG_TRY(vcycle_apply(&h->H, h->W, h->W.b, h->W.z, h->s));
    AMG_CUDA_TRY(cudaMemcpyAsync(z, h->W.z, sizeof(double) * n, cudaMemcpyDefault, h->s));
    AMG_TRY(leave(h, cuda_stream, !is_device_ptr(z)));
    return AMG_OK;
}

int amg_get_info(amg_handle h, amg_info *info) {
    if (!h || !info) return AMG_ERR_ARG;
    fill_info(h, h->H, info);
    return AMG_OK;
}

int amg_get_level(amg_handle h, int level, int which, long long *dims, int *row_ptr, int *col_idx,
                  double *values) {
    if (!h || level < 0 || level >= h->H.nlevels || which < 0 || which > 2) return AMG_ERR_ARG;
    if (which > 0 && level >= h->H.nlevels - 1) return AMG_ERR_ARG;
    const Level &lv = h->H.L[level];
    const DevCSR &m = which == 0 ? lv.A : which == 1 ? lv.P : lv.R;
    if (dims) {
        dims[0] = m.nrows;
        dims[1] = m.ncols;
        dims[2] = m.nnz;
    }
    if (row_ptr) AMG_CUDA_TRY(cudaMemcpy(row_ptr, m.rp, sizeof(int) * ((size_t)m.nrows + 1), cudaMemcpyDefault));
    if (col_idx) AMG_CUDA_TRY(cudaMemcpy(col_idx, m.ci, sizeof(int) * (size_t)m.nnz, cudaMemcpyDefault));
    if (values) AMG_CUDA_TRY(cudaMemcpy(values, m.v, sizeof(double) * (size_t)m.nnz, cudaMemcpyDefault));
    return AMG_OK;
}

int amg_get_aggregates(amg_handle h, int level, int *agg) {
    if (!h || !agg || level < 0 || level >= h->H.nlevels - 1) return AMG_ERR_ARG;
    AMG_CUDA_TRY(cudaMemcpy(agg, h->H.L[level].agg, sizeof(int) * (size_t)h->H.L[level].A.nrows, cudaMemcpyDefault));
    return AMG_OK;
}

namespace {
__global__ void k_narrow(const double *__restrict__ in, float *out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = amg::f64_to_f32_rn(in[i]);
}
__global__ void k_widen(const float *__restrict__ in, double *out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = amg::f32_to_f64(in[i]);
}
int conv_grid(long long n) { return (int)std::max(1LL, std::min((n + 255) / 256, 4096LL)); }
}  // namespace

int amg_narrow_f64(const double *in, float *out, long long n, void *cuda_stream) {
    if (n < 0 || (n > 0 && (!in || !out))) return AMG_ERR_ARG;
    if (n == 0) return AMG_OK;
    k_narrow<<<conv_grid(n), 256, 0, (cudaStream_t)cuda_stream>>>(in, out, n);
    AMG_LAUNCH_CHECK();
    return AMG_OK;
}

int amg_widen_f32(const float *in, double *out, long long n, void *cuda_stream) {
    if (n < 0 || (n > 0 && (!in || !out))) return AMG_ERR_ARG;
    if (n == 0) return AMG_OK;
    k_widen<<<conv_grid(n), 256, 0, (cudaStream_t)cuda_stream>>>(in, out, n);
    AMG_LAUNCH_CHECK();
    return AMG_OK;
}

int amg_get_plan(amg_handle h, int level, int which, int plan[6]) {
    if (!h || !plan || level < 0 || level >= h->H.nlevels || which < 0 || which > 4 || (which == 4 && level != 0))
        return AMG_ERR_ARG;
    const Level &lv = h->H.L[level];
    const StreamPlan *ps[] = {&lv.sa, &lv.sp, &lv.sr, &lv.sa_post, &lv.sa64};
    const StreamPlan &p = *ps[which];
    plan[0] = p.rt == 0      ? 0
              : p.direct     ? AMG_LAYOUT_ELL_DIRECT
              : p.ell        ? AMG_LAYOUT_SLICED_ELL
              : p.c16        ? AMG_LAYOUT_WINDOWED
                             : AMG_LAYOUT_CSR;
    plan[1] = p.rt;
    plan[2] = p.vec;
    plan[3] = p.ntiles;
    // CSR tiles: three stages of 4-byte values at 512 threads, else two
    const bool v4 = which != 4 && h->H.cfg.precision == AMG_PRECISION_MIXED;
    plan[4] = p.rt == 0 ? 0 : p.direct ? 1 : (p.ell || p.c16) ? p.stages : (p.nt == 512 && v4 ? 3 : 2);
    plan[5] = which == 4 && h->H.krylov_df ? 1 : 0;
    return AMG_OK;
}

int amg_profile(amg_handle h, int enable) {
    if (!h) return AMG_ERR_ARG;
    AMG_CUDA_TRY(cudaStreamSynchronize(h->s));
    h->W.prof.reset();
    h->W.prof.on = enable != 0;
    return AMG_OK;
}

int amg_profile_summary(amg_handle h, long long *launches, int *nrecords) {
    if (!h) return AMG_ERR_ARG;
    AMG_CUDA_TRY(cudaStreamSynchronize(h->s));
    h->W.prof.collect();
    if (launches) *launches = h->W.prof.launches;
    if (nrecords) *nrecords = (int)h->W.prof.recs.size();
    return AMG_OK;
}

int amg_profile_record(amg_handle h, int i, char *name, int name_len, int *level, long long *launches,
                       double *total_ms, double *total_bytes) {
    if (!h || i < 0 || i >= (int)h->W.prof.recs.size()) return AMG_ERR_ARG;
    const Profiler::Rec &r = h->W.prof.recs[i];
    if (name && name_len > 0) {
        strncpy(name, r.name, (size_t)name_len - 1);
        name[name_len - 1] = 0;
    }
    if (level) *level = r.level;
    if (launches) *launches = r.launches;
    if (total_ms) *total_ms = r.ms;
    if (total_bytes) *total_bytes = r.bytes;
    return AMG_OK;
}

int amg_resetup(amg_handle h, const double *values, void *cuda_stream) {
    if (!h || !values) return AMG_ERR_ARG;
    if (h->H.nsys > 0) {
        set_last_error("amg_resetup: not provided for batched handles");
        return AMG_ERR_UNSUPPORTED;
    }
    AMG_TRY(enter(h, cuda_stream));
    const auto t0 = clk::now();
    int rc = resetup_hierarchy(&h->H, values, h->s);
    if (rc == AMG_OK && h->HT && h->HT->transposed_of) {
        // the transposed hierarchy follows A's: its operators are transposed again
        rc = refresh_transposed_hierarchy(h->HT, &h->H, h->s);
    } else if (rc == AMG_OK && h->HT) {
        // the cached hierarchy of A^T follows: its values are the transpose of the new ones
        DevArena tmp;
        DevCSR At;
        rc = transpose_csr(h->H.L[0].A, At, tmp, h->s);
        if (rc == AMG_OK) rc = resetup_hierarchy(h->HT, At.v, h->s);
        const cudaError_t e = cudaStreamSynchronize(h->s);
        tmp.free_all();
        if (rc == AMG_OK && e != cudaSuccess) {
            set_last_error("amg_resetup: %s", cudaGetErrorString(e));
            rc = AMG_ERR_CUDA;
        }
    }
    if (rc != AMG_OK) return rc;
    AMG_TRY(leave(h, cuda_stream, true));
    h->H.setup_ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    return AMG_OK;
}

int amg_setup_batched(const amg_config *cfg, int nsys, const int *sys_off, int n, long long nnz,
                      const int *row_ptr, const int *col_idx, const double *values, void *cuda_stream,
                      amg_handle *out) {
    if (!out) return AMG_ERR_ARG;
    *out = nullptr;
    if (nsys <= 0 || nsys > n || n <= 0 || nnz < n || nnz >= (1LL << 31) - 1 || !sys_off || !row_ptr || !col_idx ||
        !values) {
        set_last_error("amg_setup_batched: invalid sizes or null array (nsys=%d, n=%d, nnz=%lld)", nsys, n, nnz);
        return AMG_ERR_ARG;
    }
    amg_config c;
    if (cfg) c = *cfg;
    else amg_config_default(&c);
    AMG_TRY(check_config(c));
    if (c.solver != AMG_SOLVER_PCG || c.amg_type != AMG_TYPE_AGGREGATION) {
        set_last_error("amg_setup_batched: only AMG_SOLVER_PCG with aggregation AMG is supported for batches");
        return AMG_ERR_UNSUPPORTED;
    }
    std::vector<int> off((size_t)nsys + 1);
    AMG_CUDA_TRY(cudaMemcpy(off.data(), sys_off, sizeof(int) * off.size(), cudaMemcpyDefault));
    const auto t0 = clk::now();
    amg_handle h = nullptr;
    AMG_TRY(make_handle(&h, cuda_stream));
    int rc = AMG_OK;
    do {
        h->H.cfg = c;
        h->H.n = n;
        h->H.nnz = nnz;
        if ((rc = build_hierarchy_batched(&h->H, row_ptr, col_idx, values, off.data(), nsys, h->s)) != AMG_OK) break;
        if ((rc = batch_create(&h->H, &h->BW)) < 0) break;
        if ((rc = leave(h, cuda_stream, true)) < 0) break;
    } while (0);
    if (rc != AMG_OK) {
        destroy(h);
        return rc;
    }
    h->H.setup_ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    *out = h;
    return AMG_OK;
}

int amg_solve_batched(amg_handle h, int nrhs, const double *B, double *X, int *iters, double *rel_res,
                      void *cuda_stream, amg_info *info) {
    if (!h || !B || !X || nrhs < 1 || nrhs > AMG_BATCH_MAX_RHS) return AMG_ERR_ARG;
    if (!h->BW) {
        set_last_error("amg_solve_batched: the handle was not made by amg_setup_batched");
        return AMG_ERR_ARG;
    }
    AMG_TRY(enter(h, cuda_stream));
    const auto t0 = clk::now();
    SolveResult r;
    const int rc = batch_solve(&h->H, h->BW, h->W.prof, nrhs, B, X, iters, rel_res, h->s, &r);
    h->last_solve_ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    if (rc < 0) return rc;
    h->last = r;
    AMG_TRY(leave(h, cuda_stream, true));
    if (info) fill_info(h, h->H, info);
    return r.status;
}

int amg_batch_level(amg_handle h, int level, int *nsys_level, int *sys, int *row_off, int *final_flags) {
    if (!h || !nsys_level || h->H.nsys <= 0 || level < 0 || level >= h->H.nlevels) return AMG_ERR_ARG;
    const BatchLevel &b = h->H.bl[level];
    const int ns = (int)b.sys.size();
    *nsys_level = ns;
    for (int j = 0; j < ns; ++j) {
        if (sys) sys[j] = b.sys[j];
        if (final_flags) final_flags[j] = b.fin[j];
    }
    if (row_off)
        for (int j = 0; j <= ns; ++j) row_off[j] = b.off[j];
    return AMG_OK;
}

int amg_profile_product(amg_handle h, int reps, double *us_per_launch) {
    if (!h || reps < 1 || !us_per_launch) return AMG_ERR_ARG;
    AMG_TRY(single_only(h, "amg_profile_product"));
    return time_product(&h->H, h->W, reps, h->s, us_per_launch);
}

int amg_test_arm_wait_timeout(amg_handle h, int kind) {
    if (!h || kind < 0 || kind > AMG_TEST_WITHHOLD_BARRIER) {
        set_last_error("amg_test_arm_wait_timeout: invalid handle or kind %d", kind);
        return AMG_ERR_ARG;
    }
    return test_arm_wait_timeout(h->W, kind, h->s);
}

int amg_free(amg_handle h) {
    destroy(h);
    return AMG_OK;
}

const char *amg_status_string(int code) {
    switch (code) {
        case AMG_OK: return "ok";
        case AMG_MAXIT: return "maximum iterations reached";
        case AMG_BREAKDOWN: return "Krylov breakdown";
        case AMG_NOT_SPD: return "coarsest operator not SPD / singular";
        case AMG_NAN: return "non-finite value";
        case AMG_ERR_ARG: return "invalid argument";
        case AMG_ERR_BAD_CSR: return "invalid CSR structure";
        case AMG_ERR_ZERO_DIAG: return "zero or missing diagonal";
        case AMG_ERR_CUDA: return "CUDA error";
        case AMG_ERR_STALL: return "coarsening stalled";
        case AMG_ERR_OOM: return "out of device memory";
        case AMG_ERR_UNSUPPORTED: return "size beyond a supported limit";
        default: return "unknown status";
    }
}

const char *amg_last_error(void) { return amg::last_error(); }

}  // extern "C"
