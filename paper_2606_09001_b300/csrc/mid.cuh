// mid.cuh -- the coarse levels of a V-cycle in one whole-GPU launch
// (amg_config.fuse_coarse = 2).
//
// Below the streaming threshold (16384 rows) each pass of the cycle is a
// small grid-stride CSR kernel.  k_mid runs the run of such levels m..L-2 --
// the restriction into level m, then for every level pre-smoothing with the
// residual and restriction, the dense operator of the cycle's end, and back
// up prolongation and post-smoothing -- as phases of one cooperative launch
// (one 1024-thread CTA per SM, all resident) with a software grid barrier
// between phases.  Each phase computes its rows exactly as the per-pass
// kernel does, so the two give the same bits.
//
// Measured on the 128^3 diffusion hierarchy (levels 2-3 of 6) it is slower
// than the per-pass kernels chained with programmatic dependent launch: a
// barrier costs about 1.4 us, but at 64 registers a thread the launch holds
// 32 warps an SM against 64 for the 256-thread per-pass kernels, and the
// latency-bound row passes take about twice as long.  It is therefore not
// the default.
//
// Vectors written in this launch are read with plain loads (never the
// non-coherent read-only path): the barrier's acquire orders them after every
// CTA's writes of the previous phase.  Operators and weights, read-only for
// the launch, take the read-only path.  The early exit on a finished solve is
// taken before the first barrier by every CTA alike.  The barrier's wait is
// bounded by the clock: a CTA that gives up sets an error flag and the
// kernel's results are discarded by the host.
#pragma once

#include "amg_common.cuh"

namespace amg {
namespace mid {

constexpr int THREADS = 1024;  // one CTA per SM
constexpr int MAX_LEVELS = 8;

template <typename TM>
struct MLevel {
    int n, nc;                 // rows of this level and of the next
    int vec_a, vec_p, vec_r;   // lanes per row of A, P, R
    const int *arp, *aci;
    const TM *av;
    const int *prp, *pci;
    const TM *pv;
    const int *rrp, *rci;
    const TM *rv;
    const TM *w;
    TM *b, *t, *x;
};

template <typename TM>
struct MArgs {
    int nlev;                  // smoothed levels m .. m+nlev-1 (then the dense end)
    // phase 0: b_m = R_{m-1} t_{m-1}
    int r0n, r0vec;
    const int *r0rp, *r0ci;
    const TM *r0v;
    const TM *r0x;
    // the dense end: x = M b, M dm x dm with rows padded to dld entries
    int dm, dld;
    const void *M;
    TM *db, *dx;
    MLevel<TM> L[MAX_LEVELS];
};

__device__ __forceinline__ unsigned atom_add_release(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.release.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier on one word whose low 31 bits are zero between barriers: CTA 0
// adds 2^31 - (nblocks - 1), every other CTA adds 1, so the top bit flips
// when, and only when, the last CTA has arrived, and the low bits are zero
// again.  Each CTA waits for the top bit to differ from the one its own add
// saw.  The add releases the CTA's writes (ordered before it by the CTA
// barrier), the load that sees the flip acquires everyone's.  A wait gives up
// after `limit` SM clocks (2^31, about a second, unless a test shortens it)
// and returns false.  `skip` (tests only) neither adds nor waits.
constexpr long long BARRIER_CLOCKS = 1LL << 31;
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned nblocks, bool skip = false,
                                             long long limit = BARRIER_CLOCKS) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0 && !skip) {
        s_ok = 1;
        const unsigned inc = blockIdx.x == 0 ? 0x80000000u - (nblocks - 1) : 1u;
        const unsigned old = atom_add_release(bar, inc);
        const long long t0 = clock64();
        while (((ld_acquire(bar) ^ old) & 0x80000000u) == 0) {
            if (clock64() - t0 > limit) {
                s_ok = 0;
                break;
            }
        }
    } else if (threadIdx.x == 0) {
        s_ok = 1;
    }
    __syncthreads();
    return s_ok != 0;
}

// The test control read at err[1] (see amg_test_arm_wait_timeout): with
// TEST_WITHHOLD_BARRIER the last CTA of the next launch that does work skips
// every grid-barrier arrival, so every other CTA's first wait runs out after
// TEST_CLOCKS clocks; those CTAs set err[0] |= 2, disarm the control and
// return, and the skipping CTA runs its phases unsynchronised to the end
// (results discarded; no wait of its own).
constexpr int TEST_WITHHOLD_BARRIER = 2;
constexpr long long TEST_CLOCKS = 1LL << 20;

// Row passes: VEC lanes per row, warps grid-stride over the rows.
#define MID_ROWS(VEC, n)                                                              \
    const int lane_ = threadIdx.x & (VEC - 1);                                        \
    const int rpw_ = 32 / VEC;                                                        \
    const int warp_ = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;                   \
    const int nwarps_ = (gridDim.x * blockDim.x) >> 5;                                \
    const int sub_ = (threadIdx.x & 31) / VEC;                                        \
    for (int base_ = warp_ * rpw_; base_ < (n); base_ += nwarps_ * rpw_) {            \
        const int i = base_ + sub_;                                                   \
        const bool valid = i < (n);

// y = M x
template <int VEC, typename TM>
__device__ void p_spmv(int n, const int *__restrict__ rp, const int *__restrict__ ci, const TM *__restrict__ v,
                       const TM *x, TM *y) {
    MID_ROWS(VEC, n)
    TM s = 0;
    if (valid) {
        const int e = __ldg(rp + i + 1);
        for (int k = __ldg(rp + i) + lane_; k < e; k += VEC) s += __ldg(v + k) * x[__ldg(ci + k)];
    }
    s = group_sum<VEC>(s);
    if (valid && lane_ == 0) y[i] = s;
    }
}

// t = b - A (W b)
template <int VEC, typename TM>
__device__ void p_pre(const MLevel<TM> &lv) {
    MID_ROWS(VEC, lv.n)
    TM s = 0;
    if (valid) {
        const int e = __ldg(lv.arp + i + 1);
        for (int k = __ldg(lv.arp + i) + lane_; k < e; k += VEC) {
            const int j = __ldg(lv.aci + k);
            s += __ldg(lv.av + k) * (__ldg(lv.w + j) * lv.b[j]);
        }
    }
    s = group_sum<VEC>(s);
    if (valid && lane_ == 0) lv.t[i] = lv.b[i] - s;
    }
}

// t = W b + P x_next
template <int VEC, typename TM>
__device__ void p_prolong(const MLevel<TM> &lv, const TM *xc) {
    MID_ROWS(VEC, lv.n)
    TM s = 0;
    if (valid) {
        const int e = __ldg(lv.prp + i + 1);
        for (int k = __ldg(lv.prp + i) + lane_; k < e; k += VEC) s += __ldg(lv.pv + k) * xc[__ldg(lv.pci + k)];
    }
    s = group_sum<VEC>(s);
    if (valid && lane_ == 0) lv.t[i] = __ldg(lv.w + i) * lv.b[i] + s;
    }
}

// x = t + W (b - A t)
template <int VEC, typename TM>
__device__ void p_post(const MLevel<TM> &lv) {
    MID_ROWS(VEC, lv.n)
    TM s = 0;
    if (valid) {
        const int e = __ldg(lv.arp + i + 1);
        for (int k = __ldg(lv.arp + i) + lane_; k < e; k += VEC) s += __ldg(lv.av + k) * lv.t[__ldg(lv.aci + k)];
    }
    s = group_sum<VEC>(s);
    if (valid && lane_ == 0) lv.x[i] = lv.t[i] + __ldg(lv.w + i) * (lv.b[i] - s);
    }
}

#undef MID_ROWS

// x = M b, the dense end of the cycle (M m x m, rows padded to ld entries
// with zeros): one warp per row reading 16-byte vectors, U of a lane's loads
// of the row in flight together; b is staged in sb (DENSE_LD doubles of
// shared memory; zero beyond m).  The mixed cycle (FP32 entries, FP32
// vectors) sums in FP32, two chains a lane, like its other passes and like
// the cluster kernel's FP32 coarse end; otherwise b is staged and summed in
// FP64, FP32 entries widened on the integer pipes (exact, like any widening)
// so that the FP64 pipe runs only the products' FMAs.  A lane's partial sums
// run over its vectors in order whatever U, then the warp's sum: the
// per-level cycle's kernel and the cooperative mid kernel give the same bits.
constexpr int DENSE_LD = 2048;

template <int U, typename TMAT, typename TV>
__device__ void dense_rows(int m, int ld, const TMAT *__restrict__ M, const TV *b, TV *x, void *sbuf) {
    constexpr bool F32 = std::is_same<TMAT, float>::value && std::is_same<TV, float>::value;
    using TS = typename std::conditional<F32, float, double>::type;
    TS *sb = reinterpret_cast<TS *>(sbuf);
#pragma unroll 8
    for (int j = threadIdx.x; j < ld; j += blockDim.x) sb[j] = j < m ? fcvt<TS>(b[j]) : TS(0);
    __syncthreads();
    using V = typename std::conditional<sizeof(TMAT) == 4, float4, double2>::type;
    constexpr int VW = sizeof(V) / sizeof(TMAT);
    const int lane = threadIdx.x & 31;
    const int nv = ld / VW;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += (gridDim.x * blockDim.x) >> 5) {
        const V *row = reinterpret_cast<const V *>(M + (size_t)i * ld);
        TS s = 0, s1 = 0;
        for (int q0 = lane; q0 < nv; q0 += 32 * U) {
            V a[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = q0 + 32 * u;
                if (q < nv) a[u] = __ldg(row + q);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = q0 + 32 * u;
                if (q < nv) {
                    if constexpr (F32) {
                        const float4 c = reinterpret_cast<const float4 *>(sb)[q];
                        s = fmaf(a[u].x, c.x, s);
                        s1 = fmaf(a[u].y, c.y, s1);
                        s = fmaf(a[u].z, c.z, s);
                        s1 = fmaf(a[u].w, c.w, s1);
                    } else if constexpr (VW == 4) {
                        const double2 *bd = reinterpret_cast<const double2 *>(sb);
                        const double2 c0 = bd[2 * q], c1 = bd[2 * q + 1];
                        s += f32_to_f64(a[u].x) * c0.x + f32_to_f64(a[u].y) * c0.y + f32_to_f64(a[u].z) * c1.x +
                             f32_to_f64(a[u].w) * c1.y;
                    } else {
                        const double2 c = reinterpret_cast<const double2 *>(sb)[q];
                        s += a[u].x * c.x + a[u].y * c.y;
                    }
                }
            }
        }
        s = group_sum<32>(s + s1);
        if (lane == 0) x[i] = fcvt<TV>(s);
    }
}

#define MID_VEC(vec, CALL)                                      \
    switch (vec) {                                              \
        case 2: { constexpr int V = 2; CALL; } break;           \
        case 4: { constexpr int V = 4; CALL; } break;           \
        case 8: { constexpr int V = 8; CALL; } break;           \
        case 16: { constexpr int V = 16; CALL; } break;         \
        default: { constexpr int V = 32; CALL; } break;         \
    }

// The phases, with a grid barrier between each two:
//   b_m = R_{m-1} t_{m-1};
//   for each level l = m..: t_l = b_l - A_l W_l b_l, then b_{l+1} = R_l t_l;
//   x_end = M b_end;
//   for each level l = ..m: t_l = W_l b_l + P_l x_{l+1}, then x_l = t_l + W_l (b_l - A_l t_l).
// bar: the two barrier words (zero count on entry); err: set to 2 when a
// barrier wait gave up.
template <typename TM, typename TMAT>
__global__ void __launch_bounds__(THREADS) k_mid(const __grid_constant__ MArgs<TM> a, unsigned *bar,
                                                 const int *done, int *err) {
    // no kernel writes these flags while this one runs (it is launched without
    // programmatic overlap): every CTA returns or none.  After a barrier wait
    // gave up the barrier word is inconsistent until the next call's control
    // kernel clears it, so later launches of the same call do nothing.
    if (*done || (*err & 2)) return;
    __shared__ __align__(16) double sb[DENSE_LD];
    const unsigned nb = gridDim.x;
    // every CTA reads the test control before any CTA can disarm it (that
    // happens only after a barrier wait has run out)
    const bool test = __ldcg(err + 1) == TEST_WITHHOLD_BARRIER;
    const bool skip = test && blockIdx.x == nb - 1 && nb > 1;
    const long long lim = test ? TEST_CLOCKS : BARRIER_CLOCKS;
    auto sync = [&]() -> bool {
        if (grid_barrier(bar, nb, skip, lim)) return true;
        if (threadIdx.x == 0) {
            atomicOr(err, 2);
            atomicExch(err + 1, 0);
        }
        return false;
    };
    MID_VEC(a.r0vec, (p_spmv<V, TM>(a.r0n, a.r0rp, a.r0ci, a.r0v, a.r0x, a.L[0].b)));
    for (int k = 0; k < a.nlev; ++k) {
        const MLevel<TM> &lv = a.L[k];
        TM *bn = k + 1 < a.nlev ? a.L[k + 1].b : a.db;
        if (!sync()) return;
        MID_VEC(lv.vec_a, (p_pre<V, TM>(lv)));
        if (!sync()) return;
        MID_VEC(lv.vec_r, (p_spmv<V, TM>(lv.nc, lv.rrp, lv.rci, lv.rv, lv.t, bn)));
    }
    if (!sync()) return;
    dense_rows<8, TMAT, TM>(a.dm, a.dld, reinterpret_cast<const TMAT *>(a.M), a.db, a.dx, sb);
    for (int k = a.nlev - 1; k >= 0; --k) {
        const MLevel<TM> &lv = a.L[k];
        const TM *xn = k + 1 < a.nlev ? a.L[k + 1].x : a.dx;
        if (!sync()) return;
        MID_VEC(lv.vec_p, (p_prolong<V, TM>(lv, xn)));
        if (!sync()) return;
        MID_VEC(lv.vec_a, (p_post<V, TM>(lv)));
    }
}

#undef MID_VEC

}  // namespace mid
}  // namespace amg
