// cpcg.cuh -- a whole PCG solve in one thread-block cluster.
//
// When every level of the hierarchy is small enough that all operators fit
// in the shared memory of one cluster (up to 16 CTAs of 512 threads, one
// per SM), k_cpcg runs the preconditioned CG iterations of Sec. 2.1 -- the
// V-cycle, the outer FP64 product q = A p, the vector updates and the dot
// products -- in a single launch, until the recursive residual meets the
// tolerance, the iteration cap is reached or a scalar fails.  The host then
// checks the true residual and restarts as for any other solve.
//
// Rows.  Every level's rows are split into contiguous slices, one per CTA,
// and the split is shared by all operators whose rows belong to that level
// (A_k and P_k, and R_{k-1}, whose rows are level k's); slice bounds are
// multiples of 4.  A CTA bulk-copies its slices of every operator into shared
// memory at launch and keeps its slices of the per-row vectors there: w_k
// and b_k of each smoothed level, and the outer x, r, p, q, z in FP64.
//
// Exchange.  A row pass gathers from a whole vector held in the CTA's
// shared memory.  Each phase computes the CTA's rows of the next such vector
// into its own staging buffer, then sends that slice to the same place in
// every other CTA's buffer with st.async: 16-byte remote stores that count
// their bytes on the receiving CTA's mbarrier.  A CTA arms that mbarrier
// with the bytes it will receive and waits on it (bounded), so a phase waits
// only for its own inputs: no cluster barrier and no memory fence in the
// loop, and no vector passes through global memory.  Two staging buffers
// alternate; a CTA writes into a peer's buffer only after receiving that
// peer's output of the phase before, which the peer sends after it has read
// the buffer, so a phase never overwrites what a slower CTA still gathers.
//
// V-cycle mode (k_cpcg<TM, true>, for a table built with vmode = 1): the
// same phases from a coarse level t down and back, for a hierarchy whose
// levels above t stream: level t's right-hand side is computed here from
// level t-1's residual (the restriction R_{t-1}, read from global memory:
// one launch fewer a cycle) or read from global memory, and the result goes
// back there (read by the prolongation above); no reduction and no
// data-dependent branch, so every CTA runs the same phases.  The mode is a
// template parameter: the V-cycle instance carries none of the Krylov code
// (71 registers a thread instead of 114-124, 4 KB of static shared memory
// instead of 17 KB).
//
// Reductions.  A CTA's partial dot products go into a slot per CTA in every
// CTA's shared memory the same way; each CTA adds the slots in rank order,
// so every CTA holds the same bits and takes the same decision (beta, alpha,
// convergence, failure) without a further exchange, and all CTAs leave the
// loop after the same phase.  A CTA whose bulk copies did not land in time
// skips its row passes, and one whose wait ran out puts a NaN into its next
// partial, which ends the solve everywhere.
#pragma once

#include <cooperative_groups.h>

#include "amg_common.cuh"
#include "stream.cuh"
#include "tail.cuh"

namespace amg {
namespace cpcg {

namespace cg = cooperative_groups;

constexpr int THREADS = 512;
constexpr int MAX_LEVELS = 8;
constexpr int MAX_CTAS = 16;
// The last warp arms the mbarriers and issues the sends: the row passes of
// the small levels leave it idle, so the bookkeeping stays off the path of
// the warps that hold rows.
constexpr int AUX_WARP = THREADS / 32 - 1;

// One operator's slices: CSR (ci != null) or the dense coarsest operator
// (row-major, ncols entries a row).  The shared-memory offsets are the same
// in every CTA (each region is sized for the largest slice).
template <typename TV>
struct COp {
    const int *rp, *ci;
    const TV *v;
    int ncols;
    int vec;                   // lanes per row
    int copy;                  // bulk copies of its own: 1 row pointers and indices, 2 values
                               // (the outer FP64 A_0 shares A_0's row pointers and indices)
    int rp_off, ci_off, v_off;
    int e0[MAX_CTAS + 1];      // CSR: row_ptr at each slice boundary of the rows' level
};

template <typename TM>
struct CLevel {
    int n;
    int r0[MAX_CTAS + 1];      // the level's row split (multiples of 4, then n)
    COp<TM> A, P;              // rows of this level (smoothed levels only)
    COp<TM> R;                 // R_k: rows of level k+1, split as level k+1
    const TM *w;               // smoother weights (global; the CTA's slice is loaded at w_off)
    int w_off, b_off;          // shared-memory slices of w and b (b: levels > 0)
};

template <typename TM>
struct CArgs {
    int nlev;                  // levels 0 .. nlev-1; the last one is the dense coarsest
    // 1: one V-cycle from a coarse level t (table level 0) -- its right-hand
    // side vb and result vx in global memory, the levels above it run as
    // separate passes -- instead of a whole PCG solve; launched as
    // k_cpcg<TM, true>
    int vmode;
    const TM *vb;
    TM *vx;
    // V-cycle mode, where vr_rp is set: level t's right-hand side computed
    // here as R_{t-1} t_{t-1} (R's rows are level t's, split as level t; R
    // and t_{t-1} are read from global memory), in place of the restriction
    // pass above and the read of vb
    const int *vr_rp, *vr_ci;
    const TM *vr_v, *vr_x;
    int cta;
    int buf_off[2], buf_bytes; // the two staging buffers
    int x_off, r_off, p_off, q_off, z_off;  // the CTA's level-0 slices of the FP64 Krylov vectors
    unsigned tx[MAX_CTAS];     // bytes each CTA bulk-copies (the mbarrier's transaction count)
    COp<double> K;             // level-0 A in FP64 for q = A p (shares A_0's row pointers and indices)
    // the dense operator of the last level, split as level nlev-1: FP64 with
    // FP64 sums (C), or in the mixed form the collapsed coarse end's FP32 copy
    // with FP32 sums (C32, c32 = 1)
    COp<double> C;
    COp<float> C32;
    int c32;
    CLevel<TM> L[MAX_LEVELS];
};

// Issues CTA c's bulk copies of one operator's slice, rows [r0, r1) (thread
// of warp 0), or only adds up their bytes.
template <typename TV>
__device__ __host__ inline uint32_t slice_copy(const COp<TV> &op, int r0, int r1, int c, unsigned char *smem,
                                               uint64_t *bar, bool issue) {
    if (!op.copy || r0 >= r1) return 0;
    uint32_t bytes = 0;
    long long e0, e1;
    if (op.ci) {
        e0 = op.e0[c];
        e1 = op.e0[c + 1];
    } else {
        e0 = (long long)r0 * op.ncols;
        e1 = (long long)r1 * op.ncols;
    }
    if (op.ci && (op.copy & 1)) {
        const long long a = tail::align_lo<int>(r0), z = tail::align_hi<int>(r1 + 1);
        const uint32_t b = (uint32_t)((z - a) * 4);
#ifdef __CUDA_ARCH__
        if (issue) stream::bulk_g2s(smem + op.rp_off, op.rp + a, b, bar);
#endif
        bytes += b;
        if (e1 > e0) {
            const long long ca = tail::align_lo<int>(e0), cz = tail::align_hi<int>(e1);
            const uint32_t cb = (uint32_t)((cz - ca) * 4);
#ifdef __CUDA_ARCH__
            if (issue) stream::bulk_g2s(smem + op.ci_off, op.ci + ca, cb, bar);
#endif
            bytes += cb;
        }
    }
    if ((op.copy & 2) && e1 > e0) {
        const long long va = tail::align_lo<TV>(e0), vz = tail::align_hi<TV>(e1);
        const uint32_t vb = (uint32_t)((vz - va) * sizeof(TV));
#ifdef __CUDA_ARCH__
        if (issue) stream::bulk_g2s(smem + op.v_off, op.v + va, vb, bar);
#endif
        bytes += vb;
    }
    return bytes;
}

#ifdef __CUDACC__

// Rows [r0, r1) of CTA c: f(i, sum_j M_ij xs[j]), vec lanes a row, the
// operator's slice read from shared memory.  Every lane of a row's group
// ends with the row's sum; lane 0 calls f.  The loop bound is the same for
// all threads of the CTA, so the shuffles see whole warps.
template <typename TV, typename TS, typename TA, class F>
__device__ __forceinline__ void rows(const COp<TV> &op, int r0, int r1, int c, const unsigned char *smem,
                                     const TS *xs, F f) {
    const int vec = op.vec;
    const int lane = threadIdx.x & (vec - 1), group = threadIdx.x / vec, ngroups = THREADS / vec;
    if (op.ci) {
        const int e0 = op.e0[c];
        // slices indexed by row and entry (the copies start at 16-byte aligned elements)
        const int *rp = reinterpret_cast<const int *>(smem + op.rp_off) - (int)tail::align_lo<int>(r0);
        const int *ci = reinterpret_cast<const int *>(smem + op.ci_off) - (int)tail::align_lo<int>(e0);
        const TV *v = reinterpret_cast<const TV *>(smem + op.v_off) - (int)tail::align_lo<TV>(e0);
        for (int base = r0; base < r1; base += ngroups) {
            const int i = base + group;
            TA s = 0;
            if (i < r1) {
                const int e = rp[i + 1];
#pragma unroll 4
                for (int k = rp[i] + lane; k < e; k += vec) s += (TA)v[k] * (TA)xs[ci[k]];
            }
            for (int o = vec >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, vec);
            if (i < r1 && lane == 0) f(i, s);
        }
    } else {
        const TV *v = reinterpret_cast<const TV *>(smem + op.v_off) - (int)tail::align_lo<TV>((long long)r0 * op.ncols);
        for (int base = r0; base < r1; base += ngroups) {
            const int i = base + group;
            TA s = 0;
            if (i < r1) {
                const TV *row = v + i * op.ncols;
#pragma unroll 4
                for (int j = lane; j < op.ncols; j += vec) s += (TA)row[j] * (TA)xs[j];
            }
            for (int o = vec >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, vec);
            if (i < r1 && lane == 0) f(i, s);
        }
    }
}

__device__ __forceinline__ uint32_t mapa(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
// A bulk copy of `bytes` (a multiple of 16) from this CTA's shared memory to
// another CTA's (dst and bar shared::cluster), completing on that CTA's
// mbarrier.
__device__ __forceinline__ void bulk_s2peer(uint32_t dst, uint32_t src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "r"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void st_async8(uint32_t dst, double v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(dst),
                 "l"(__double_as_longlong(v)), "r"(bar)
                 : "memory");
}
// Arrives on an mbarrier and adds `bytes` to its expected transaction count,
// without ordering the thread's earlier memory operations (the arrival
// publishes nothing).
__device__ __forceinline__ void arm_relaxed(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.relaxed.cta.shared::cta.b64 _, [%0], %1;" ::"r"(stream::smem_u32(b)),
                 "r"(bytes)
                 : "memory");
}

// Bounded wait for an mbarrier phase whose bytes other CTAs of the cluster
// wrote (acquire at cluster scope).
constexpr uint32_t WAIT_POLLS = 1u << 22;
__device__ __forceinline__ bool wait_cluster(uint64_t *b, uint32_t parity) {
    const uint32_t a = stream::smem_u32(b);
    for (uint32_t it = 0; it < WAIT_POLLS; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Bytes of the slice of rows [r0, r1) of a vector of `size`-byte entries,
// rounded out to 16 bytes (r0 is a multiple of 4; the last slice's tail runs
// into the buffer's padding).
__device__ __forceinline__ int slice_b0(int r0, int size) { return r0 * size; }
__device__ __forceinline__ int slice_b1(int r0, int r1, int size) {
    return r1 > r0 ? (r1 * size + 15) & ~15 : r0 * size;
}
// Bytes CTA c receives of a vector split by r0: every other CTA's slice.
__device__ __forceinline__ uint32_t incoming(const int *r0, int size, int c, int C) {
    uint32_t by = 0;
    for (int d = 0; d < C; ++d)
        if (d != c) by += (uint32_t)(slice_b1(r0[d], r0[d + 1], size) - slice_b0(r0[d], size));
    return by;
}

// The CTA's NV partial sums (acc, one per thread) into tot[0..NV-1]
// (shared).  Every thread's partials go to part (NV x THREADS); warp q then
// adds value q's in a fixed order (lane l: threads l, l+32, ..., then a
// shuffle tree), the values in parallel on different warps: FP64 adds are
// slow, so few warps should issue them.  Only threads below np hold
// partials.  *poison (read after the barrier) makes tot[0] a NaN.
template <int NV>
__device__ __forceinline__ void cta_sum(const double (&acc)[NV], double *part, double *tot, const int *poison,
                                        int np) {
#pragma unroll
    for (int q = 0; q < NV; ++q) part[q * THREADS + threadIdx.x] = acc[q];
    __syncthreads();
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (wid < NV) {
        double v = 0.0;
        for (int k = lane; k < np; k += 32) v += part[wid * THREADS + k];
        v = warp_sum(v);
        if (lane == 0) tot[wid] = *poison && wid == 0 ? __longlong_as_double(0x7ff8000000000000ll) : v;
    }
    __syncthreads();
}

// The Krylov scalars, kept in shared memory: thread 0 alone updates them
// (from the reduction slots), the other threads read them after a barrier.
struct KScal {
    double rz, alpha, beta, pq, rr;
    int iters, first, status, stop;
    int have_rr;  // an update preceded this V-cycle: its ||r||^2 is reduced with r.z
};

// b: the right-hand side; x, r, p, q, z: the solve's FP64 vectors in global
// memory (x and r the current iterate and residual; p and q the previous
// iteration's, read when the recursion continues); r32: the FP32 copy of r
// (mixed form), or null.  The kernel reads and writes the scalars in sc as
// the per-iteration kernels do and leaves done = 1; when the iterations end
// converged or at the cap it also leaves r = b - A x and tr = ||r||^2 of the
// final x (tr_fresh = 1), the true residual the host checks.
template <typename TM, bool VM>
__global__ void __launch_bounds__(THREADS, 1) k_cpcg(const __grid_constant__ CArgs<TM> ga, const double *__restrict__ gb,
                                                     double *__restrict__ gx,
                                                     double *__restrict__ gr, double *__restrict__ gp,
                                                     double *__restrict__ gq, double *__restrict__ gz,
                                                     float *__restrict__ gr32, DevScalars *sc) {
    extern __shared__ __align__(128) unsigned char smem[];
    // bar: the operator slices' bulk copies; xbar[k]: staging buffer k's
    // incoming slices; rbar: the two reductions' incoming partials
    __shared__ __align__(8) uint64_t bar, xbar[2], rbar[2];
    __shared__ double part[3 * THREADS];
    __shared__ double tot[3], sums[3];
    __shared__ __align__(16) double slot_rz[MAX_CTAS * 3], slot_pq[MAX_CTAS];
    __shared__ KScal S;
    __shared__ int bad;  // 1: the bulk copies did not land; 2: an exchange wait ran out
    // the table, copied to shared memory: the phases index it by level and
    // rank, which the constant cache serves slowly
    __shared__ __align__(16) CArgs<TM> a;
    cg::cluster_group cl = cg::this_cluster();
    // What depends on no earlier kernel -- the table, the mbarriers, the bulk
    // copies of the operator slices and the smoother weights, all written at
    // setup -- is issued before the wait on the preceding kernel (launched
    // with programmatic stream serialisation, this overlaps its end).
    {
        static_assert(sizeof(CArgs<TM>) % 4 == 0, "table copied in words");
        const int *src = reinterpret_cast<const int *>(&ga);
        int *dst = reinterpret_cast<int *>(&a);
        for (int k = threadIdx.x; k < (int)(sizeof(CArgs<TM>) / 4); k += THREADS) dst[k] = src[k];
        __syncthreads();
    }
    const int c = (int)cl.block_rank(), C = a.cta, nl = a.nlev;
    const int tid = threadIdx.x;

    // bulk copies of the CTA's operator slices (warp 0), one mbarrier
    if (tid < 32) {
        if (tid == 0) {
            stream::mbar_init(&bar, 1);
            for (int k = 0; k < 2; ++k) stream::mbar_init(&xbar[k], 1);
            for (int k = 0; k < 2; ++k) stream::mbar_init(&rbar[k], 1);
            stream::fence_mbar_init();
            stream::mbar_expect_tx(&bar, a.tx[c]);
        }
        __syncwarp();
        const int nops = 3 * (nl - 1);
        const int q0 = a.L[nl - 1].r0[c], q1 = a.L[nl - 1].r0[c + 1];
        for (int it = tid; it < nops + 3; it += 32) {
            if (it < nops) {
                const CLevel<TM> &lv = a.L[it / 3], &nx = a.L[it / 3 + 1];
                const int k = it % 3;
                if (k == 2) slice_copy(lv.R, nx.r0[c], nx.r0[c + 1], c, smem, &bar, true);
                else slice_copy(k == 0 ? lv.A : lv.P, lv.r0[c], lv.r0[c + 1], c, smem, &bar, true);
            } else if (it == nops) {
                slice_copy(a.K, a.L[0].r0[c], a.L[0].r0[c + 1], c, smem, &bar, true);
            } else if (it == nops + 1) {
                slice_copy(a.C, q0, q1, c, smem, &bar, true);
            } else {
                slice_copy(a.C32, q0, q1, c, smem, &bar, true);
            }
        }
    }
    for (int k = 0; k < nl - 1; ++k) {
        const CLevel<TM> &lv = a.L[k];
        TM *w = reinterpret_cast<TM *>(smem + lv.w_off);
        for (int i = lv.r0[c] + tid; i < lv.r0[c + 1]; i += THREADS) w[i - lv.r0[c]] = lv.w[i];
    }
    pdl_wait();
    pdl_trigger();
    if (sc->done) {
        // uniform (every thread of every CTA reads the same word, before any
        // cluster barrier); the copies land before the shared memory is released
        stream::mbar_wait(&bar, 0);
        return;
    }
    const double tol2 = sc->tol2;
    const int max_iter = sc->max_iter, flexible = sc->flexible, first0 = sc->first;
    if (tid == 0) {
        S.rz = sc->rz;
        S.alpha = sc->alpha;
        S.beta = sc->beta;
        S.pq = sc->pq;
        S.rr = sc->rr;
        S.iters = sc->iters;
        S.first = first0;
        S.status = AMG_OK;
        S.stop = 0;
        S.have_rr = 0;
        bad = 0;
    }

    // the CTA's slices of the vectors
    const int r0 = a.L[0].r0[c], r1 = a.L[0].r0[c + 1];
    double *X = reinterpret_cast<double *>(smem + a.x_off), *R = reinterpret_cast<double *>(smem + a.r_off);
    double *P = reinterpret_cast<double *>(smem + a.p_off), *Q = reinterpret_cast<double *>(smem + a.q_off);
    double *Z = reinterpret_cast<double *>(smem + a.z_off);
    if (VM && a.vr_rp) {
        // b_t = R_{t-1} t_{t-1} on the CTA's rows, four lanes a row
        constexpr int G = 4;
        TM *b0 = reinterpret_cast<TM *>(smem + a.L[0].b_off);
        const int g = tid & (G - 1);
        for (int base = r0; base < r1; base += THREADS / G) {
            const int i = base + tid / G;
            TM s = 0;
            if (i < r1) {
                const int e = __ldg(a.vr_rp + i + 1);
                for (int k = __ldg(a.vr_rp + i) + g; k < e; k += G) s += __ldg(a.vr_v + k) * __ldg(a.vr_x + __ldg(a.vr_ci + k));
            }
            s = group_sum<G>(s);
            if (i < r1 && g == 0) b0[i - r0] = s;
        }
    } else if (VM) {
        TM *b0 = reinterpret_cast<TM *>(smem + a.L[0].b_off);
        for (int i = r0 + tid; i < r1; i += THREADS) b0[i - r0] = a.vb[i];
    } else {
        for (int i = r0 + tid; i < r1; i += THREADS) {
            X[i - r0] = gx[i];
            R[i - r0] = gr[i];
            P[i - r0] = first0 ? 0.0 : gp[i];
            Q[i - r0] = first0 ? 0.0 : gq[i];
        }
    }
    // every CTA has started and initialised its mbarriers: remote stores may begin
    cl.sync();
    auto buf = [&](int k) { return smem + a.buf_off[k]; };
    uint32_t xpar = 0, rpar = 0;  // phase parities of xbar[k] (bit k) and rbar[k] (bit k)
    int cur = 0;
    double rr_part = 0.0;         // the thread's share of the last update's ||r||^2

    // Sends this CTA's rows [q0, q1) of the vector in buf(nb) to every other
    // CTA -- one bulk copy a peer -- then waits for theirs.  The caller has
    // armed xbar[nb] with the incoming bytes and written its rows (made
    // visible to the copies by the proxy fence and the barrier here).
    auto exchange = [&](int nb, int q0, int q1, int size) {
        stream::fence_proxy_async();
        __syncthreads();
        const int b0 = slice_b0(q0, size), bytes = slice_b1(q0, q1, size) - b0;
        const int d = tid - AUX_WARP * 32;
        if (d >= 0 && d < C && d != c && bytes > 0) {
            const uint32_t src = stream::smem_u32(buf(nb) + b0);
            bulk_s2peer(mapa(src, (uint32_t)d), src, (uint32_t)bytes, mapa(stream::smem_u32(&xbar[nb]), (uint32_t)d));
        }
        if (!wait_cluster(&xbar[nb], (xpar >> nb) & 1u)) atomicOr(&bad, 2);
        xpar ^= 1u << nb;
        cur = nb;
    };
    // Puts the CTA's nv totals (tot) into slot c of every CTA's slots; warp 0
    // waits for the others' and adds them in a fixed order (a shuffle tree
    // over the ranks, the same bits in every CTA) into sums[0..nv-1], read by
    // thread 0 after the warp's sync.
    auto reduce = [&](int j, double *slots, int nv) {
        const uint32_t sb = stream::smem_u32(slots), rb = stream::smem_u32(&rbar[j]);
        const int d = tid - AUX_WARP * 32;
        if (d >= 0 && d < C && d != c)
            for (int q = 0; q < nv; ++q)
                st_async8(mapa(sb + 8u * (c * nv + q), (uint32_t)d), tot[q], mapa(rb, (uint32_t)d));
        if (tid < 32) {
            if (tid == 0)
                for (int q = 0; q < nv; ++q) slots[c * nv + q] = tot[q];
            if (!wait_cluster(&rbar[j], (rpar >> j) & 1u)) atomicOr(&bad, 2);
            __syncwarp();
            const int d = tid & (MAX_CTAS - 1);
            for (int q0 = 0; q0 < nv; q0 += 2) {
                const int q = q0 + (tid >> 4);
                double v = q < nv && d < C ? slots[d * nv + q] : 0.0;
                v = group_sum<MAX_CTAS>(v);
                if (d == 0 && q < nv) sums[q] = v;
            }
            __syncwarp();
        }
        rpar ^= 1u << j;
    };
    auto arm_vec = [&](int nb, const int *split, int size) {
        if (tid == AUX_WARP * 32) arm_relaxed(&xbar[nb], incoming(split, size, c, C));
    };
    auto arm_red = [&](int j, int nv) {
        if (tid == AUX_WARP * 32) arm_relaxed(&rbar[j], (uint32_t)(8 * nv * (C - 1)));
    };

    // the first pre-smoothing gathers W b with b = r (a V-cycle: level t's b)
    {
        arm_vec(0, a.L[0].r0, (int)sizeof(TM));
        TM *ys = reinterpret_cast<TM *>(buf(0));
        const TM *w0 = reinterpret_cast<const TM *>(smem + a.L[0].w_off);
        const TM *b0 = reinterpret_cast<const TM *>(smem + a.L[0].b_off);
        for (int i = r0 + tid; i < r1; i += THREADS)
            ys[i] = w0[i - r0] * (VM ? b0[i - r0] : fcvt<TM>(R[i - r0]));
        exchange(0, r0, r1, (int)sizeof(TM));
    }
    const bool loaded = __syncthreads_and(stream::mbar_wait(&bar, 0)) != 0;
    if (!loaded && tid == 0) {
        atomicOr(&sc->copy_timeout, 1);
        atomicOr(&bad, 1);
    }

    for (;;) {
        // V-cycle, down: pre-smoothing with the residual, restriction
        for (int k = 0; k < nl - 1; ++k) {
            const CLevel<TM> &lv = a.L[k], &nx = a.L[k + 1];
            const int s0 = lv.r0[c], s1 = lv.r0[c + 1];
            const TM *bk = reinterpret_cast<const TM *>(smem + lv.b_off);
            {
                // t = b - A (W b)
                const int nb = cur ^ 1;
                arm_vec(nb, lv.r0, (int)sizeof(TM));
                const TM *xs = reinterpret_cast<const TM *>(buf(cur));
                TM *ys = reinterpret_cast<TM *>(buf(nb));
                if (loaded)
                    rows<TM, TM, TM>(lv.A, s0, s1, c, smem, xs, [&](int i, TM s) {
                        const TM bi = k == 0 && !VM ? fcvt<TM>(R[i - s0]) : bk[i - s0];
                        ys[i] = bi - s;
                    });
                exchange(nb, s0, s1, (int)sizeof(TM));
            }
            {
                // b_next = R t; the next pre-smoothing gathers W b_next, the
                // dense operator b_next itself
                const int q0 = nx.r0[c], q1 = nx.r0[c + 1];
                const bool last = k + 1 == nl - 1;
                const int nb = cur ^ 1;
                arm_vec(nb, nx.r0, (int)sizeof(TM));
                const TM *xs = reinterpret_cast<const TM *>(buf(cur));
                TM *ys = reinterpret_cast<TM *>(buf(nb));
                TM *bn = reinterpret_cast<TM *>(smem + nx.b_off);
                const TM *wn = reinterpret_cast<const TM *>(smem + nx.w_off);
                if (loaded)
                    rows<TM, TM, TM>(lv.R, q0, q1, c, smem, xs, [&](int i, TM s) {
                        if (last) {
                            ys[i] = s;
                        } else {
                            bn[i - q0] = s;
                            ys[i] = wn[i - q0] * s;
                        }
                    });
                exchange(nb, q0, q1, (int)sizeof(TM));
            }
        }
        // the dense operator of the last level
        {
            const CLevel<TM> &lc = a.L[nl - 1];
            const int s0 = lc.r0[c], s1 = lc.r0[c + 1];
            const int nb = cur ^ 1;
            arm_vec(nb, lc.r0, (int)sizeof(TM));
            const TM *xs = reinterpret_cast<const TM *>(buf(cur));
            TM *ys = reinterpret_cast<TM *>(buf(nb));
            if (loaded) {
                if (a.c32)
                    rows<float, TM, TM>(a.C32, s0, s1, c, smem, xs, [&](int i, TM s) { ys[i] = s; });
                else
                    rows<double, TM, double>(a.C, s0, s1, c, smem, xs,
                                             [&](int i, double s) { ys[i] = fcvt<TM>(s); });
            }
            exchange(nb, s0, s1, (int)sizeof(TM));
        }
        // V-cycle, up: prolongation, post-smoothing; level 0 ends in z and r.z
        bool stop = false;
        for (int k = nl - 2; k >= 0; --k) {
            const CLevel<TM> &lv = a.L[k];
            const int s0 = lv.r0[c], s1 = lv.r0[c + 1];
            const TM *wk = reinterpret_cast<const TM *>(smem + lv.w_off);
            const TM *bk = reinterpret_cast<const TM *>(smem + lv.b_off);
            auto bof = [&](int i) { return k == 0 && !VM ? fcvt<TM>(R[i - s0]) : bk[i - s0]; };
            {
                // t = W b + P x_next
                const int nb = cur ^ 1;
                arm_vec(nb, lv.r0, (int)sizeof(TM));
                const TM *xs = reinterpret_cast<const TM *>(buf(cur));
                TM *ys = reinterpret_cast<TM *>(buf(nb));
                if (loaded)
                    rows<TM, TM, TM>(lv.P, s0, s1, c, smem, xs,
                                     [&](int i, TM s) { ys[i] = wk[i - s0] * bof(i) + s; });
                exchange(nb, s0, s1, (int)sizeof(TM));
            }
            // x = t + W (b - A t)
            const TM *ts = reinterpret_cast<const TM *>(buf(cur));
            if (k > 0) {
                const int nb = cur ^ 1;
                arm_vec(nb, lv.r0, (int)sizeof(TM));
                TM *ys = reinterpret_cast<TM *>(buf(nb));
                if (loaded)
                    rows<TM, TM, TM>(lv.A, s0, s1, c, smem, ts,
                                     [&](int i, TM s) { ys[i] = ts[i] + wk[i - s0] * (bof(i) - s); });
                exchange(nb, s0, s1, (int)sizeof(TM));
            } else if (VM) {
                // the cycle's result, read by the prolongation of the level above
                if (loaded)
                    rows<TM, TM, TM>(lv.A, s0, s1, c, smem, ts,
                                     [&](int i, TM s) { a.vx[i] = ts[i] + wk[i - s0] * (bof(i) - s); });
            } else {
                // r.z, z.q and the last update's ||r||^2 in one reduction
                arm_red(0, 3);
                double acc[3] = {0.0, 0.0, rr_part};
                if (loaded)
                    rows<TM, TM, TM>(lv.A, s0, s1, c, smem, ts, [&](int i, TM s) {
                        const double zi = fcvt<double>(ts[i] + wk[i - s0] * (bof(i) - s));
                        Z[i - s0] = zi;
                        acc[0] += R[i - s0] * zi;
                        acc[1] += Q[i - s0] * zi;  // z.q: the flexible beta's z.(r - r_old) = -alpha z.q
                    });
                // partials sit in the rows' lane-0 threads and the update's
                // threads: below rows x lanes
                cta_sum<3>(acc, part, tot, &bad, min(THREADS, (s1 - s0) * lv.A.vec));  // a NaN ends the solve everywhere
                reduce(0, slot_rz, 3);
                if (tid == 0) {
                    // the last update's convergence test, then beta: an update
                    // that converged costs one V-cycle more, not an iteration
                    if (S.have_rr) {
                        S.rr = sums[2];
                        if (!isfinite(sums[2])) {
                            S.status = AMG_NAN;
                            S.stop = 1;
                        } else if (sums[2] <= tol2) {
                            S.stop = 1;
                        } else if (S.iters >= max_iter) {
                            S.status = AMG_MAXIT;
                            S.stop = 1;
                        }
                    }
                    if (S.stop) {
                    } else if (!isfinite(sums[0])) {
                        S.status = AMG_NAN;
                        S.stop = 1;
                    } else {
                        S.beta = S.first ? 0.0 : (flexible ? -S.alpha * sums[1] : sums[0]) / S.rz;
                        S.first = 0;
                        S.rz = sums[0];
                    }
                }
                __syncthreads();
                stop = S.stop != 0;
            }
        }
        if (stop || VM) break;
        // p = z + beta p
        {
            const int nb = cur ^ 1;
            arm_vec(nb, a.L[0].r0, 8);
            double *ps = reinterpret_cast<double *>(buf(nb));
            const double beta = S.beta;
            for (int i = r0 + tid; i < r1; i += THREADS) {
                const double pv = beta == 0.0 ? Z[i - r0] : Z[i - r0] + beta * P[i - r0];
                P[i - r0] = pv;
                ps[i] = pv;
            }
            exchange(nb, r0, r1, 8);
        }
        // q = A p (FP64) and p.q -> alpha
        {
            arm_red(1, 1);
            const double *ps = reinterpret_cast<const double *>(buf(cur));
            double acc[1] = {0.0};
            rows<double, double, double>(a.K, r0, r1, c, smem, ps, [&](int i, double s) {
                Q[i - r0] = s;
                acc[0] += P[i - r0] * s;
            });
            cta_sum<1>(acc, part, tot, &bad, min(THREADS, (r1 - r0) * a.K.vec));
            reduce(1, slot_pq, 1);
            if (tid == 0) {
                if (!isfinite(sums[0]) || sums[0] <= 0.0) {
                    S.status = isfinite(sums[0]) ? AMG_BREAKDOWN : AMG_NAN;
                    S.stop = 1;
                } else {
                    S.pq = sums[0];
                    S.alpha = S.rz / sums[0];
                }
            }
            __syncthreads();
            if (S.stop) break;
        }
        // x += alpha p, r -= alpha q, r.r; the next pre-smoothing gathers W r
        {
            const int nb = cur ^ 1;
            arm_vec(nb, a.L[0].r0, (int)sizeof(TM));
            TM *ys = reinterpret_cast<TM *>(buf(nb));
            const TM *w0 = reinterpret_cast<const TM *>(smem + a.L[0].w_off);
            const double alpha = S.alpha;
            rr_part = 0.0;
            for (int i = r0 + tid; i < r1; i += THREADS) {
                X[i - r0] += alpha * P[i - r0];
                const double rn = R[i - r0] - alpha * Q[i - r0];
                R[i - r0] = rn;
                rr_part += rn * rn;
                ys[i] = w0[i - r0] * fcvt<TM>(rn);
            }
            if (tid == 0) {
                S.iters += 1;
                S.have_rr = 1;
            }
            exchange(nb, r0, r1, (int)sizeof(TM));
        }
    }
    // the true residual of the final x: x to every CTA, then r = b - A x
    // (the FP64 operator) and ||r||^2
    const bool true_res = !VM && (S.status == AMG_OK || S.status == AMG_MAXIT);
    if (true_res) {
        {
            const int nb = cur ^ 1;
            arm_vec(nb, a.L[0].r0, 8);
            double *xs = reinterpret_cast<double *>(buf(nb));
            for (int i = r0 + tid; i < r1; i += THREADS) xs[i] = X[i - r0];
            exchange(nb, r0, r1, 8);
        }
        arm_red(1, 1);
        const double *xs = reinterpret_cast<const double *>(buf(cur));
        double acc[1] = {0.0};
        if (loaded)
            rows<double, double, double>(a.K, r0, r1, c, smem, xs, [&](int i, double s) {
                const double ri = gb[i] - s;
                R[i - r0] = ri;
                acc[0] += ri * ri;
            });
        cta_sum<1>(acc, part, tot, &bad, min(THREADS, (r1 - r0) * a.K.vec));
        reduce(1, slot_pq, 1);
        __syncthreads();  // R's new entries, for the write-back below
    }
    if ((bad & 2) && tid == 0) atomicOr(&sc->copy_timeout, 4);
    // the state back to global memory for the true residual and a restart
    if (!VM)
        for (int i = r0 + tid; i < r1; i += THREADS) {
            gx[i] = X[i - r0];
            gr[i] = R[i - r0];
            gp[i] = P[i - r0];
            gq[i] = Q[i - r0];
            gz[i] = Z[i - r0];
            if (gr32) gr32[i] = f64_to_f32_rn(R[i - r0]);
        }
    if (c == 0 && tid == 0 && !VM) {
        sc->rz = S.rz;
        sc->alpha = S.alpha;
        sc->beta = S.beta;
        sc->pq = S.pq;
        sc->rr = S.rr;
        sc->iters = S.iters;
        sc->first = S.first;
        sc->status = S.status;
        if (true_res) sc->tr = sums[0];
        sc->tr_fresh = true_res ? 1 : 0;
        sc->done = 1;
    }
    if (!loaded) stream::mbar_wait(&bar, 0);  // a bounded chance for late copies to land before exit
    // no CTA leaves while another may still store into its shared memory
    cl.sync();
}

#endif  // __CUDACC__

}  // namespace cpcg
}  // namespace amg
