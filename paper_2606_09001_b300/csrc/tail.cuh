// tail.cuh -- the coarse levels of a V-cycle in one launch.
//
// Below the streaming threshold every level is small (at most a few
// thousand rows): one launch per operator there costs more in launch latency
// than in memory traffic.  k_tail runs all levels t..L-1 of the cycle --
// pre-smoothing with the residual, restriction, the dense coarsest solve,
// prolongation and post-smoothing -- as phases of a single thread-block
// cluster (up to 16 CTAs of 1024 threads, one per SM), separated by hardware
// cluster barriers (barrier.cluster arrive.release / wait.acquire).  Vectors
// written inside the kernel are read back through L2 (ld.global.cg); the
// operators are read-only.  Every thread runs every phase and barrier, and
// the early exit on a finished solve is taken before the first barrier, by
// all threads alike, so no barrier can wait for a thread that left.
#pragma once

#include <cooperative_groups.h>

#include "amg_common.cuh"

namespace amg {
namespace tail {

namespace cg = cooperative_groups;

constexpr int THREADS = 1024;
constexpr int MAX_LEVELS = 12;

template <typename TM>
struct TLevel {
    int n, vec_a, vec_p, vec_r;
    const int *arp, *aci;
    const TM *av, *ahat, *w;   // A, A W, smoother weights
    const int *prp, *pci;
    const TM *pv;              // P (n x n_next)
    const int *rrp, *rci;
    const TM *rv;              // R (n_next x n)
    TM *b, *t, *x;             // right-hand side (levels > t), residual / prolonged iterate, result
};

// Fixed per-hierarchy table (device memory, built once at setup).
template <typename TM>
struct TArgs {
    int nlev;                  // levels t .. L-1 (the last is the dense coarsest)
    int level0;                // 1: the first tail level is the finest (b0 in, z0 out, FP64)
    int nc;
    const double *cinv;        // dense inverse of the coarsest operator
    TLevel<TM> L[MAX_LEVELS];
};

__device__ __forceinline__ float ldcg(const float *p) { return __ldcg(p); }
__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }

// y_i = f(i, sum_j M_ij g(j)) over the rows, vec threads per row, all threads
// of the cluster; every warp runs the same number of iterations.
template <typename TM, class G, class F>
__device__ __forceinline__ void row_pass(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                         const TM *__restrict__ v, int vec, int gtid, int gthreads, G g, F f) {
    constexpr int UNR = 4;  // entries per lane with their loads in flight together
    const int lane = gtid & (vec - 1);
    const int group = gtid / vec, ngroups = gthreads / vec;
    for (int base = 0; base < n; base += ngroups) {
        const int i = base + group;
        TM s = 0;
        if (i < n) {
            const int e = __ldg(rp + i + 1);
            for (int kb = __ldg(rp + i) + lane; kb < e; kb += UNR * vec) {
                TM av[UNR];
                int cj[UNR];
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    const int k = kb + u * vec;
                    const bool in = k < e;
                    av[u] = in ? __ldg(v + k) : (TM)0;
                    cj[u] = in ? __ldg(ci + k) : -1;
                }
                TM xv[UNR];
#pragma unroll
                for (int u = 0; u < UNR; ++u) xv[u] = cj[u] >= 0 ? g(cj[u]) : (TM)0;
#pragma unroll
                for (int u = 0; u < UNR; ++u) s += av[u] * xv[u];
            }
        }
        for (int o = vec >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, vec);
        if (i < n && lane == 0) f(i, s);
    }
}

// b0/z0: finest right-hand side and result when the tail starts at level 0
// (FP64); rold: flexible PCG's previous residual (mixed); fin: compute the PCG
// beta from r.z (level-0 tails only).
template <typename TM>
__global__ void __launch_bounds__(THREADS) k_tail(const TArgs<TM> *__restrict__ ap, const double *__restrict__ b0,
                                                  double *__restrict__ z0, const double *__restrict__ rold, int fin,
                                                  DevScalars *sc) {
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ double red[2][THREADS / 32];
    if (sc->done) return;  // uniform: read before any barrier by every thread
    const TArgs<TM> &a = *ap;
    const int gtid = (int)cluster.block_rank() * THREADS + threadIdx.x;
    const int gthreads = (int)cluster.num_blocks() * THREADS;
    const int nl = a.nlev;
    const bool l0 = a.level0 != 0;
    double acc[2] = {0.0, 0.0};

    // down: pre-smoothing + residual, restriction
    for (int k = 0; k < nl - 1; ++k) {
        const TLevel<TM> &lv = a.L[k];
        const TLevel<TM> &nx = a.L[k + 1];
        const bool fin0 = l0 && k == 0;
        // r = b - (A W) b
        row_pass<TM>(lv.n, lv.arp, lv.aci, lv.ahat, lv.vec_a, gtid, gthreads,
                     [&](int j) { return fin0 ? (TM)__ldg(b0 + j) : ldcg(lv.b + j); },
                     [&](int i, TM s) { lv.t[i] = (fin0 ? (TM)__ldg(b0 + i) : ldcg(lv.b + i)) - s; });
        cluster.sync();
        // b_next = R r
        row_pass<TM>(nx.n, lv.rrp, lv.rci, lv.rv, lv.vec_r, gtid, gthreads, [&](int j) { return ldcg(lv.t + j); },
                     [&](int i, TM s) { nx.b[i] = s; });
        cluster.sync();
    }
    // coarsest: x = A_c^-1 b, FP64, one warp per row
    {
        const TLevel<TM> &lc = a.L[nl - 1];
        const int warp = gtid >> 5, lane = gtid & 31, nwarps = gthreads >> 5;
        for (int base = 0; base < a.nc; base += nwarps) {
            const int i = base + warp;
            double s = 0.0;
            if (i < a.nc)
                for (int j = lane; j < a.nc; j += 32) s += __ldg(a.cinv + (size_t)i * a.nc + j) * (double)ldcg(lc.b + j);
            s = warp_sum(s);
            if (i < a.nc && lane == 0) lc.x[i] = (TM)s;
        }
        cluster.sync();
    }
    // up: prolongation, post-smoothing
    for (int k = nl - 2; k >= 0; --k) {
        const TLevel<TM> &lv = a.L[k];
        const TLevel<TM> &nx = a.L[k + 1];
        const bool fin0 = l0 && k == 0;
        // t = W b + P x_next
        row_pass<TM>(lv.n, lv.prp, lv.pci, lv.pv, lv.vec_p, gtid, gthreads, [&](int j) { return ldcg(nx.x + j); },
                     [&](int i, TM s) {
                         const TM bi = fin0 ? (TM)__ldg(b0 + i) : ldcg(lv.b + i);
                         lv.t[i] = __ldg(lv.w + i) * bi + s;
                     });
        cluster.sync();
        // x = t + W (b - A t)
        row_pass<TM>(lv.n, lv.arp, lv.aci, lv.av, lv.vec_a, gtid, gthreads, [&](int j) { return ldcg(lv.t + j); },
                     [&](int i, TM s) {
                         const TM bi = fin0 ? (TM)__ldg(b0 + i) : ldcg(lv.b + i);
                         const TM xi = ldcg(lv.t + i) + __ldg(lv.w + i) * (bi - s);
                         if (fin0) {
                             const double o = (double)xi;
                             z0[i] = o;
                             if (fin) {
                                 acc[0] += __ldg(b0 + i) * o;
                                 if (rold) acc[1] += __ldg(rold + i) * o;
                             }
                         } else {
                             lv.x[i] = xi;
                         }
                     });
        if (k > 0) cluster.sync();
    }
    if (l0 && fin) {
        // cluster-wide reduction of r.z (and z.r_old) into CTA 0, then beta
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int q = 0; q < 2; ++q) {
            double v = warp_sum(acc[q]);
            if (lane == 0) red[q][wid] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int q = 0; q < 2; ++q) {
                double v = 0.0;
                for (int w = 0; w < THREADS / 32; ++w) v += red[q][w];
                red[q][0] = v;
            }
        }
        cluster.sync();
        if (cluster.block_rank() == 0 && threadIdx.x == 0) {
            double tot[2] = {0.0, 0.0};
            for (unsigned r = 0; r < cluster.num_blocks(); ++r) {
                const double *remote = cluster.map_shared_rank(&red[0][0], r);
                tot[0] += remote[0];
                tot[1] += remote[THREADS / 32];
            }
            if (!isfinite(tot[0])) {
                sc->status = AMG_NAN;
                sc->done = 1;
            } else {
                double beta = 0.0;
                if (!sc->first) beta = (sc->flexible ? tot[0] - tot[1] : tot[0]) / sc->rz;
                sc->first = 0;
                sc->beta = beta;
                sc->rz = tot[0];
            }
        }
        cluster.sync();  // keep every CTA's shared memory alive until CTA 0 has read it
    }
}

}  // namespace tail
}  // namespace amg
