// tail.cuh -- the coarse levels of a V-cycle in one launch.
//
// Below the streaming threshold every level is small (at most a few
// thousand rows): one launch per operator there costs more in launch latency
// than in memory traffic.  k_tail runs all levels t..L-1 of the cycle --
// pre-smoothing with the residual, restriction, the dense coarsest solve,
// prolongation and post-smoothing -- as phases of a single thread-block
// cluster (up to 16 CTAs of 1024 threads, one per SM), separated by hardware
// cluster barriers (barrier.cluster arrive.release / wait.acquire).
//
// Every operator of the tail is split into contiguous row slices of about
// equal stored entries, one per CTA.  At launch each CTA bulk-copies its
// slices (row pointers, column indices, values; the coarsest inverse's rows)
// into shared memory with cp.async.bulk on one mbarrier, as far as its
// shared-memory budget allows; the rest is read from global memory.  Each
// smoothed level's weights are preloaded too, and its right-hand side is kept
// in shared memory from the pre-smoothing stage to the end of the cycle.
// Each phase first stages the vector it gathers from (written by every CTA in
// the previous phase, read back through L2 with ld.global.cg) into the CTA's
// shared memory, so a row pass never waits on a global load for x.  Every
// thread runs every phase and barrier, and the early exit on a finished solve
// is taken before the first barrier, by all threads alike, so no barrier can
// wait for a thread that left.
#pragma once

#include <cooperative_groups.h>

#include "amg_common.cuh"
#include "stream.cuh"

namespace amg {
namespace tail {

namespace cg = cooperative_groups;

constexpr int THREADS = 1024;
constexpr int MAX_LEVELS = 12;
constexpr int MAX_CTAS = 16;

// One CSR operator of the tail (or the coarsest dense inverse, ci = null),
// split over the cluster's CTAs: CTA c owns rows r0[c] .. r0[c+1]-1.
template <typename TV>
struct TOp {
    const int *rp, *ci;
    const TV *v;
    int n;                     // rows
    int ncols;                 // dense inverse: row length
    int vec;                   // lanes per row
    int res;                   // 1: every CTA's slice is preloaded into shared memory
    int rp_off, ci_off, v_off; // byte offsets of the slices in each CTA's shared memory
    int r0[MAX_CTAS + 1];
    int e0[MAX_CTAS + 1];      // CSR: row_ptr at each slice boundary
};

template <typename TM>
struct TLevel {
    int n;
    TOp<TM> A, P, R;           // A (pre- and post-smoothing), P (n x n_next), R (n_next x n)
    const TM *w;               // smoother weights
    TM *b, *t, *x;             // right-hand side (levels > t), residual / prolonged iterate, result
    int ws_off, bs_off;        // shared-memory copies of w (preloaded) and b (kept from the
                               // pre-smoothing stage) for the whole cycle; -1: read from global
};

// Fixed per-hierarchy table, built once at setup and passed by value as a
// kernel parameter (it reaches every SM with the launch instead of through
// dependent global loads).
template <typename TM>
struct TArgs {
    int nlev;                  // levels t .. L-1 (the last is the dense coarsest)
    int level0;                // 1: the first tail level is the finest (b0 in, z0 out, FP64)
    int nc;
    int stage_off;             // byte offset of the staged vector in shared memory
    unsigned tx[MAX_CTAS];     // bytes each CTA preloads (for the mbarrier's transaction count)
    TOp<double> C;             // dense inverse of the coarsest operator (nc x nc, row-major)
    TLevel<TM> L[MAX_LEVELS];
};

__device__ __forceinline__ float ldcg(const float *p) { return __ldcg(p); }
__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }

// Element index at which a 16-byte-aligned copy of entries from e starts.
template <typename T>
__host__ __device__ __forceinline__ long long align_lo(long long e) {
    return e & ~(long long)(16 / sizeof(T) - 1);
}
template <typename T>
__host__ __device__ __forceinline__ long long align_hi(long long e) {
    return (e + 16 / sizeof(T) - 1) & ~(long long)(16 / sizeof(T) - 1);
}

// Issues the bulk copies of this CTA's slice of one operator (thread 0), or
// adds up their bytes (bytes_only).
template <typename TV>
__device__ uint32_t preload(const TOp<TV> &op, int c, unsigned char *smem, uint64_t *bar, bool bytes_only) {
    if (!op.res) return 0;
    const int r0 = op.r0[c], r1 = op.r0[c + 1];
    if (r0 >= r1) return 0;
    uint32_t bytes = 0;
    long long e0, e1;
    if (op.ci) {
        const long long a = align_lo<int>(r0), z = align_hi<int>(r1 + 1);
        const uint32_t b = (uint32_t)((z - a) * 4);
        if (!bytes_only) stream::bulk_g2s(smem + op.rp_off, op.rp + a, b, bar);
        bytes += b;
        e0 = op.e0[c];
        e1 = op.e0[c + 1];
        if (e1 > e0) {
            const long long ca = align_lo<int>(e0), cz = align_hi<int>(e1);
            const uint32_t cb = (uint32_t)((cz - ca) * 4);
            if (!bytes_only) stream::bulk_g2s(smem + op.ci_off, op.ci + ca, cb, bar);
            bytes += cb;
        }
    } else {
        e0 = (long long)r0 * op.ncols;
        e1 = (long long)r1 * op.ncols;
    }
    if (e1 > e0) {
        const long long va = align_lo<TV>(e0), vz = align_hi<TV>(e1);
        const uint32_t vb = (uint32_t)((vz - va) * sizeof(TV));
        if (!bytes_only) stream::bulk_g2s(smem + op.v_off, op.v + va, vb, bar);
        bytes += vb;
    }
    return bytes;
}

// Rows of this CTA's slice: f(i, sum_j M_ij xs[j]), vec lanes per row, the
// operator read from shared memory when preloaded.  The loop bound is the same
// for every thread of the CTA, so the shuffles see whole warps.
template <typename TV, typename TS, typename TA, class F>
__device__ __forceinline__ void op_rows(const TOp<TV> &op, int c, const unsigned char *smem, const TS *xs, F f) {
    const int r0 = op.r0[c], r1 = op.r0[c + 1];
    const int vec = op.vec;
    const int lane = threadIdx.x & (vec - 1), group = threadIdx.x / vec, ngroups = THREADS / vec;
    const int *rp = op.rp, *ci = op.ci;
    const TV *v = op.v;
    long long rpb = 0, cib = 0, vb = 0;
    if (op.res && r0 < r1) {
        if (ci) {
            rp = reinterpret_cast<const int *>(smem + op.rp_off);
            rpb = align_lo<int>(r0);
            const long long e0 = rp[r0 - rpb];
            ci = reinterpret_cast<const int *>(smem + op.ci_off);
            cib = align_lo<int>(e0);
            vb = align_lo<TV>(e0);
        } else {
            vb = align_lo<TV>((long long)r0 * op.ncols);
        }
        v = reinterpret_cast<const TV *>(smem + op.v_off);
    }
    for (int base = r0; base < r1; base += ngroups) {
        const int i = base + group;
        TA s = 0;
        if (i < r1) {
            if (ci) {
                const int e = rp[i + 1 - rpb];
#pragma unroll 4
                for (int k = rp[i - rpb] + lane; k < e; k += vec) s += (TA)v[k - vb] * (TA)xs[ci[k - cib]];
            } else {
                const long long o = (long long)i * op.ncols - vb;
#pragma unroll 4
                for (int j = lane; j < op.ncols; j += vec) s += (TA)v[o + j] * (TA)xs[j];
            }
        }
        for (int o = vec >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, vec);
        if (i < r1 && lane == 0) f(i, s);
    }
}

// xs[j] = g(j) for j < len, by every thread of the CTA, then a CTA barrier.
template <typename TM, class G>
__device__ __forceinline__ void stage(TM *xs, int len, G g) {
    for (int j = threadIdx.x; j < len; j += THREADS) xs[j] = g(j);
    __syncthreads();
}

// b0/z0: finest right-hand side and result when the tail starts at level 0
// (FP64); qprev: flexible PCG's previous iteration's q = A p (mixed); fin:
// compute the PCG beta from r.z (level-0 tails only).
template <typename TM>
__global__ void __launch_bounds__(THREADS) k_tail(const __grid_constant__ TArgs<TM> a, const double *__restrict__ b0,
                                                  double *__restrict__ z0, const double *__restrict__ qprev, int fin,
                                                  DevScalars *sc) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ double red[2][THREADS / 32];
    cg::cluster_group cluster = cg::this_cluster();
    pdl_wait();
    pdl_trigger();
    if (sc->done) return;  // uniform: read before any barrier by every thread
    const int c = (int)cluster.block_rank();
    const int nl = a.nlev;
    const bool l0 = a.level0 != 0;
    TM *xs = reinterpret_cast<TM *>(smem + a.stage_off);

    // Preload this CTA's operator slices and every level's weights: warp 0
    // arms one mbarrier with the CTA's byte count, then its lanes issue the
    // bulk copies of different operators at once.
    if (threadIdx.x < 32) {
        if (threadIdx.x == 0) {
            stream::mbar_init(&bar, 1);
            stream::fence_mbar_init();
            stream::mbar_expect_tx(&bar, a.tx[c]);
        }
        __syncwarp();
        const int nops = 3 * (nl - 1);
        for (int it = threadIdx.x; it < nops + nl; it += 32) {
            if (it < nops) {
                const TLevel<TM> &lv = a.L[it / 3];
                preload(it % 3 == 0 ? lv.A : it % 3 == 1 ? lv.P : lv.R, c, smem, &bar, false);
            } else if (it == nops) {
                preload(a.C, c, smem, &bar, false);
            } else {
                const TLevel<TM> &lv = a.L[it - nops - 1];
                if (lv.ws_off >= 0)
                    stream::bulk_g2s(smem + lv.ws_off, lv.w, (uint32_t)(align_hi<TM>(lv.n) * sizeof(TM)), &bar);
            }
        }
    }
    __syncthreads();
    double acc[2] = {0.0, 0.0};
    bool ok = true, waited = false;
    // before the first row pass: the preloaded slices must have landed
    auto ready = [&]() {
        if (waited) return;
        waited = true;
        ok = __syncthreads_and(stream::mbar_wait(&bar, 0)) != 0;
        if (!ok && threadIdx.x == 0) atomicExch(&sc->copy_timeout, 1);
    };

    // down: pre-smoothing + residual, restriction
    for (int k = 0; k < nl - 1; ++k) {
        const TLevel<TM> &lv = a.L[k];
        const TLevel<TM> &nx = a.L[k + 1];
        const bool fin0 = l0 && k == 0;
        TM *ws = lv.ws_off >= 0 && k > 0 ? reinterpret_cast<TM *>(smem + lv.ws_off) : nullptr;  // landed after level 0
        TM *bs = lv.bs_off >= 0 ? reinterpret_cast<TM *>(smem + lv.bs_off) : nullptr;
        // t = b - A (W b)
        stage(xs, lv.n, [&](int j) {
            const TM bj = fin0 ? fcvt<TM>(__ldg(b0 + j)) : ldcg(lv.b + j);
            if (bs) bs[j] = bj;
            return (ws ? ws[j] : __ldg(lv.w + j)) * bj;
        });
        ready();
        if (ok)
            op_rows<TM, TM, TM>(lv.A, c, smem, xs, [&](int i, TM s) {
                lv.t[i] = (bs ? bs[i] : fin0 ? fcvt<TM>(__ldg(b0 + i)) : ldcg(lv.b + i)) - s;
            });
        cluster.sync();
        // b_next = R t
        stage(xs, lv.n, [&](int j) { return ldcg(lv.t + j); });
        if (ok) op_rows<TM, TM, TM>(lv.R, c, smem, xs, [&](int i, TM s) { nx.b[i] = s; });
        cluster.sync();
    }
    // coarsest: x = A_c^-1 b in FP64
    {
        const TLevel<TM> &lc = a.L[nl - 1];
        stage(xs, a.nc, [&](int j) { return ldcg(lc.b + j); });
        ready();
        if (ok) op_rows<double, TM, double>(a.C, c, smem, xs, [&](int i, double s) { lc.x[i] = fcvt<TM>(s); });
        cluster.sync();
    }
    // up: prolongation, post-smoothing
    for (int k = nl - 2; k >= 0; --k) {
        const TLevel<TM> &lv = a.L[k];
        const TLevel<TM> &nx = a.L[k + 1];
        const bool fin0 = l0 && k == 0;
        const TM *ws = lv.ws_off >= 0 ? reinterpret_cast<const TM *>(smem + lv.ws_off) : nullptr;
        const TM *bs = lv.bs_off >= 0 ? reinterpret_cast<const TM *>(smem + lv.bs_off) : nullptr;
        auto wof = [&](int i) { return ws ? ws[i] : __ldg(lv.w + i); };
        auto bof = [&](int i) { return bs ? bs[i] : fin0 ? fcvt<TM>(__ldg(b0 + i)) : ldcg(lv.b + i); };
        // t = W b + P x_next
        stage(xs, nx.n, [&](int j) { return ldcg(nx.x + j); });
        if (ok) op_rows<TM, TM, TM>(lv.P, c, smem, xs, [&](int i, TM s) { lv.t[i] = wof(i) * bof(i) + s; });
        cluster.sync();
        // x = t + W (b - A t)
        stage(xs, lv.n, [&](int j) { return ldcg(lv.t + j); });
        if (ok)
            op_rows<TM, TM, TM>(lv.A, c, smem, xs, [&](int i, TM s) {
                const TM xi = xs[i] + wof(i) * (bof(i) - s);
                if (fin0) {
                    const double o = fcvt<double>(xi);
                    z0[i] = o;
                    if (fin) {
                        acc[0] += __ldg(b0 + i) * o;
                        if (qprev) acc[1] += __ldg(qprev + i) * o;
                    }
                } else {
                    lv.x[i] = xi;
                }
            });
        if (k > 0) cluster.sync();
    }
    if (l0 && fin) {
        // cluster-wide reduction of r.z (and z.qprev) into CTA 0, then beta
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
        if (c == 0 && threadIdx.x == 0 && ok) {
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
                if (!sc->first) beta = (sc->flexible ? -sc->alpha * tot[1] : tot[0]) / sc->rz;  // z.(r - r_old) = -alpha z.q
                sc->first = 0;
                sc->beta = beta;
                sc->rz = tot[0];
            }
        }
        cluster.sync();  // keep every CTA's shared memory alive until CTA 0 has read it
    }
    if (!ok) {
        // a bounded chance for copies still in flight to land before exit
        stream::mbar_wait(&bar, 0);
    }
}

}  // namespace tail
}  // namespace amg
