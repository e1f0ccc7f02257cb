// stream.cuh -- row-tiled CSR passes staged through shared memory by TMA bulk
// copies (cp.async.bulk + mbarrier), used for every large operator of the
// V-cycle and the outer Krylov products.
//
// Warp-specialised persistent CTAs of NT threads (512, or 768 for 4-byte
// values) walk the tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ... of rt consecutive rows.
//   * Warp 0, lane 0 is the producer: for each tile it issues three bulk copies
//     into a pipeline stage -- the tile's row pointers, column indices and
//     values, each range rounded out to 16-byte boundaries (every array the
//     library owns is padded so the rounded range stays inside it) -- and
//     arms the stage's "full" mbarrier with the byte count.
//   * Warps 1..15 consume: wait on "full", reduce the tile's rows from shared
//     memory (VEC threads per row, UNR entries in flight per thread, the input
//     vector gathered from global memory), hand each row to an epilogue
//     functor, then arrive on the stage's "empty" mbarrier.  The producer
//     waits on "empty" before refilling the stage.
// No block-wide barrier runs inside the loop, so consumer warps drift freely
// across STAGES tiles.  The wider CTA keeps more gathers in flight per SM (two
// CTAs of 23 consumer warps instead of 15) with two pipeline stages.  Every wait is bounded; a timeout sets an error flag
// and the CTA leaves the loop.  Optional dot products end in the
// deterministic last-block reduction (the one __syncthreads of the kernel).
#pragma once

#include "amg_common.cuh"

namespace amg {
namespace stream {

constexpr int THREADS = 512;  // the default CTA width
constexpr int MAX_STAGES = 4;
constexpr int RT_MAX = 1024;
constexpr int CAP = 4096;  // stage capacity in stored entries
// Tile descriptors (entry range, window table row) of a CTA's first META_T
// tiles are loaded into shared memory at launch, in one round trip by all
// threads, so the producer never waits on a global load before a refill.
constexpr int META_T = 64;

// Pipeline depth per value type and CTA width: 3 stages of 4-byte values or
// 2 of 8-byte values keep two 512-thread CTAs resident per SM (about 104 KB
// each); 768-thread CTAs use 2 stages.
template <typename TM, int NT = THREADS>
__host__ __device__ constexpr int stages() { return NT == 512 && sizeof(TM) == 4 ? 3 : 2; }

__host__ __device__ constexpr int align16(int b) { return (b + 15) & ~15; }

// Stage layout (bytes): [row pointers | column indices | values | header]
template <typename TM>
struct Layout {
    int rpb, cib, vab, stb;
    __host__ __device__ Layout(int rt, int cap)
        : rpb(align16((rt + 8) * 4)), cib(align16((cap + 8) * 4)), vab(align16((cap + 8) * (int)sizeof(TM))),
          stb(rpb + cib + vab + 16) {}
};

template <typename TM, int NT = THREADS>
inline int smem_bytes(int rt, int cap) { return stages<TM, NT>() * Layout<TM>(rt, cap).stb; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
// Adds to the current phase's expected transaction bytes without arriving.
__device__ __forceinline__ void mbar_expect_tx_only(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(b))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after `limit` polls (2^22 unless a test shortens it)
// and reports it.
constexpr uint32_t WAIT_POLLS = 1u << 22;
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, uint32_t limit = WAIT_POLLS) {
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}

// The test control the kernels read at err[1] (armed by the host, see
// amg_test_arm_wait_timeout).  With TEST_WITHHOLD_COPY, CTA 0 of the next
// streaming launch that does work adds 16 bytes that no copy delivers to its
// first stage's expected count, so the stage never completes: its consumers'
// and producer's waits run out after TEST_POLLS polls, set err[0] and leave
// the loop; by then every copy the CTA issued has landed (the real bytes of
// both stages arrive microseconds after issue).  CTA 0 disarms the control.
constexpr int TEST_WITHHOLD_COPY = 1;
constexpr uint32_t TEST_POLLS = 1u << 12;

// Called by every thread of the CTA after the dependency wait, with c = err[1]
// as CTA 0 loaded it (0 elsewhere): true in every thread of CTA 0 when the
// control is armed; thread 0 disarms it.
__device__ __forceinline__ bool test_withhold(int c, int *err) {
    if (blockIdx.x != 0) return false;
    const bool w = __syncthreads_or(c == TEST_WITHHOLD_COPY) != 0;
    if (w && threadIdx.x == 0) atomicExch(err + 1, 0);
    return w;
}

// The row pass.  Op provides: bool done(); TM gather(int j); Pre load(int i)
// (the row's epilogue operands, loaded before the gathers so the latencies
// overlap); finish(int i, TM s, const Pre&, double (&acc)[2]);
// reduce<NT>(double (&acc)[2]) (called by every thread of every CTA at the end).
template <typename TM, int VEC, class Op, int NT = THREADS>
__global__ void __launch_bounds__(NT, 2) k_stream(int n, int rt, int cap, int ntiles, const int *__restrict__ rp,
                                                  const int *__restrict__ ci, const TM *__restrict__ v, Op op,
                                                  int *err) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int STAGES = stages<TM, NT>();
    constexpr int CONSUMER_WARPS = NT / 32 - 1;
    __shared__ __align__(8) uint64_t full[MAX_STAGES], empty[MAX_STAGES];
    const Layout<TM> L(rt, cap);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int k = 0; k < STAGES; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], CONSUMER_WARPS);
        }
        fence_mbar_init();
    }
    __syncthreads();
    __shared__ int2 m_se[META_T];
    const int my_tiles = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    for (int j = tid; j < min(my_tiles, META_T); j += NT) {
        const int t = blockIdx.x + j * gridDim.x;
        m_se[j] = make_int2(__ldg(rp + t * rt), __ldg(rp + min(t * rt + rt, n)));
    }
    __syncthreads();
    // Issues tile t (the CTA's j-th) into stage st: the expected bytes are
    // added without arriving when `pre` (the first tiles, copied before the
    // dependency wait: the operator is constant), else with the producer's
    // arrival.
    auto issue = [&](int t, int j, int st, bool pre) {
        unsigned char *stage = smem + st * L.stb;
        const int r0 = t * rt, r1 = min(r0 + rt, n);
        const int2 se = j < META_T ? m_se[j] : make_int2(__ldg(rp + r0), __ldg(rp + r1));
        const int s = se.x, e = se.y;
        const int rp_cnt = (r1 - r0 + 1 + 3) & ~3;  // r0 is a multiple of 4
        const int cs = s & ~3, ce = (e + 3) & ~3;
        constexpr int PER = 16 / sizeof(TM);
        const int vs = s & ~(PER - 1), ve = (e + PER - 1) & ~(PER - 1);
        int *hdr = reinterpret_cast<int *>(stage + L.rpb + L.cib + L.vab);
        hdr[0] = cs;
        hdr[1] = vs;
        const uint32_t b_rp = rp_cnt * 4, b_ci = (ce - cs) * 4, b_v = (ve - vs) * (uint32_t)sizeof(TM);
        if (pre) mbar_expect_tx_only(&full[st], b_rp + b_ci + b_v);
        else mbar_expect_tx(&full[st], b_rp + b_ci + b_v);
        bulk_g2s(stage, rp + r0, b_rp, &full[st]);
        if (b_ci) bulk_g2s(stage + L.rpb, ci + cs, b_ci, &full[st]);
        if (b_v) bulk_g2s(stage + L.rpb + L.cib, v + vs, b_v, &full[st]);
    };
    int npre = 0;
    if (tid == 0)
        for (; npre < STAGES && (int)blockIdx.x + npre * (int)gridDim.x < ntiles; ++npre)
            issue(blockIdx.x + npre * gridDim.x, npre, npre, true);
    pdl_wait();
    pdl_trigger();
    const int ctl = blockIdx.x == 0 ? __ldcg(err + 1) : 0;  // in flight with the done flag's load
    if (op.done()) {
        // the prefetched copies land before the CTA leaves
        if (tid == 0)
            for (int k = 0; k < npre; ++k) {
                mbar_arrive(&full[k]);
                mbar_wait(&full[k], 0);
            }
        return;
    }
    const bool wh = test_withhold(ctl, err);
    const uint32_t lim = wh ? TEST_POLLS : WAIT_POLLS;
    double acc[2] = {0.0, 0.0};
    bool ok = true;
    if (warp == 0) {
        if (lane == 0) {
            for (int j = 0;; ++j) {
                const int t = blockIdx.x + j * gridDim.x;
                if (t >= ntiles) break;
                const int st = j % STAGES;
                if (j < npre) {
                    if (j == 0 && wh) mbar_expect_tx_only(&full[0], 16);  // bytes no copy delivers
                    mbar_arrive(&full[st]);  // copies already issued
                    continue;
                }
                if (!mbar_wait(&empty[st], (uint32_t)(((j / STAGES) - 1) & 1), lim)) {
                    ok = false;
                    break;
                }
                fence_proxy_async();
                issue(t, j, st, false);
            }
        }
    } else {
        constexpr int UNR = VEC == 1 ? 8 : 4;
        const int ct = tid - 32;
        constexpr int ROWS_PER_PASS = CONSUMER_WARPS * 32 / VEC;
        const int rsub = ct / VEC, vl = ct % VEC;
        // the first pass's epilogue operands of tile t (written by
        // predecessors, so after the dependency wait): loaded a tile ahead,
        // so that their latency overlaps the tile before, where the registers
        // allow it (up to 512 threads), else before the stage wait
        constexpr bool AHEAD = NT <= 512;
        typename Op::Pre pnext{};
        if constexpr (AHEAD) {
            if ((int)blockIdx.x < ntiles && rsub < min(rt, n - (int)blockIdx.x * rt) && vl == 0)
                pnext = op.load(blockIdx.x * rt + rsub);
        }
        for (int j = 0;; ++j) {
            const int t = blockIdx.x + j * gridDim.x;
            if (t >= ntiles) break;
            const int st = j % STAGES;
            const int r0 = t * rt;
            const int rows = min(rt, n - r0);
            typename Op::Pre pre0{};
            if constexpr (AHEAD) {
                pre0 = pnext;
                const int tn = t + gridDim.x;
                if (tn < ntiles && rsub < min(rt, n - tn * rt) && vl == 0) pnext = op.load(tn * rt + rsub);
            } else if (rsub < rows && vl == 0) {
                pre0 = op.load(r0 + rsub);
            }
            if (!__all_sync(0xffffffffu, mbar_wait(&full[st], (uint32_t)((j / STAGES) & 1), lim))) {  // warp-uniform
                ok = false;
                break;
            }
            const unsigned char *stage = smem + st * L.stb;
            const int *rps = reinterpret_cast<const int *>(stage);
            const int *cis = reinterpret_cast<const int *>(stage + L.rpb);
            const TM *vals = reinterpret_cast<const TM *>(stage + L.rpb + L.cib);
            const int *hdr = reinterpret_cast<const int *>(stage + L.rpb + L.cib + L.vab);
            const int cs = hdr[0], vsb = hdr[1];
            for (int base = 0; base < rows; base += ROWS_PER_PASS) {
                const int rl = base + rsub;
                TM sum = 0;
                typename Op::Pre pre = pre0;
                if (rl < rows) {
                    if (vl == 0 && base > 0) pre = op.load(r0 + rl);
                    const int k1 = rps[rl + 1];
                    for (int kb = rps[rl] + vl; kb < k1; kb += UNR * VEC) {
                        TM av[UNR], xv[UNR];
#pragma unroll
                        for (int u = 0; u < UNR; ++u) {
                            const int k = kb + u * VEC;
                            if (k < k1) {
                                av[u] = vals[k - vsb];
                                xv[u] = op.gather(cis[k - cs]);
                            } else {
                                av[u] = 0;
                                xv[u] = 0;
                            }
                        }
#pragma unroll
                        for (int u = 0; u < UNR; ++u) sum += av[u] * xv[u];
                    }
                }
                if (VEC > 1) sum = group_sum<VEC>(sum);
                if (vl == 0 && rl < rows) op.finish(r0 + rl, sum, pre, acc);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
        }
    }
    if (!ok) {
        atomicExch(err, 1);
        // a bounded chance for copies still in flight to land before exit
        for (int k = 0; k < STAGES; ++k) mbar_try_wait(&full[k], 0);
    }
    op.template reduce<NT>(acc);
}

// ---------------------------------------------------------------------------
// Windowed variant: the gathered vector staged too
// ---------------------------------------------------------------------------
//
// For operators whose tiles each touch only a few short ranges of columns
// (the stencil structure of PDE matrices), setup finds, per tile, up to
// WIN_NW windows of the gathered vector -- 4-element aligned ranges that
// cover every column the tile touches, split at the tile's largest gaps --
// and rewrites each stored column
// index as a 16-bit offset into the tile's windows laid end to end.  The
// producer then bulk-copies those windows of the vector into the stage with
// the tile, and consumers gather from shared memory: no global load waits
// inside the row loop, and the index stream shrinks from 4 to 2 bytes per
// entry.  Op additionally provides GX (the gathered vector's type),
// const GX *gsrc(), and for epilogues that need the gathered vector's entry
// of their own row (SELF: square operators, where every row stores its
// diagonal, so a tile's own rows lie in one window) load_rest() and
// put_self(): that entry is then read from the staged window.

constexpr int WIN_NW = 16;

template <typename TM, typename GX>
struct WLayout {
    int rpb, cib, vab, xwb, stb;
    __host__ __device__ WLayout(int rt, int cap, int xw)
        : rpb(align16((rt + 8) * 4)), cib(align16((cap + 8) * 2)), vab(align16((cap + 8) * (int)sizeof(TM))),
          xwb(align16(xw * (int)sizeof(GX))), stb(rpb + cib + vab + xwb + 16) {}
};

// Pipeline stages of the windowed and sliced-ELL kernels: a plan's own count
// (2 to MAX_STAGES).  Bytes in flight per SM set the bandwidth a pass
// reaches, so the autotuner also tries more stages of the same tiles (at one
// CTA per SM when two no longer fit) and smaller tiles with more stages.
constexpr int WIN_STAGES = 2;  // the default

template <typename TM, typename GX, int NT = THREADS>
inline int smem_bytes_win(int rt, int cap, int xw, int stages = WIN_STAGES) {
    return stages * WLayout<TM, GX>(rt, cap, xw).stb;
}

// Producer side of the windowed kernels: bulk-copies the windows of the
// gathered vector gx for tile t (the CTA's j-th; its descriptors from the
// shared table m_w for the first META_T tiles, else from wtab) into xs, and
// stores at *dl0_out the offset of column r0 in the windows when one window
// holds the tile's own rows r0 .. r1-1 (else -1).  The copies' bytes are
// expected with the caller's arrival on `full`.
template <typename GX>
__device__ __forceinline__ void issue_windows(const int *__restrict__ wtab, const int4 (*m_w)[WIN_NW / 2], int t, int j,
                                              int r0, int r1, const GX *gx, unsigned char *xs, int *dl0_out,
                                              uint64_t *full) {
    const int4 *wrow = reinterpret_cast<const int4 *>(wtab) + (size_t)t * (WIN_NW / 2);
    int4 wq[WIN_NW / 2];
#pragma unroll
    for (int q = 0; q < WIN_NW / 2; ++q) wq[q] = j < META_T ? m_w[j][q] : __ldg(wrow + q);
    int dl0 = -1;
    {
        int woff = 0;
#pragma unroll
        for (int q = 0; q < WIN_NW / 2; ++q) {
            if (dl0 < 0 && wq[q].y > 0 && r0 >= wq[q].x && r1 <= wq[q].x + wq[q].y) dl0 = woff + r0 - wq[q].x;
            woff += wq[q].y;
            if (dl0 < 0 && wq[q].w > 0 && r0 >= wq[q].z && r1 <= wq[q].z + wq[q].w) dl0 = woff + r0 - wq[q].z;
            woff += wq[q].w;
        }
    }
    *dl0_out = dl0;
    uint32_t b_x = 0;
#pragma unroll
    for (int q = 0; q < WIN_NW / 2; ++q) b_x += (uint32_t)(wq[q].y + wq[q].w) * (uint32_t)sizeof(GX);
    mbar_expect_tx(full, b_x);
    uint32_t off = 0;
#pragma unroll
    for (int q = 0; q < WIN_NW / 2; ++q) {
        if (wq[q].y > 0) {
            bulk_g2s(xs + off, gx + wq[q].x, (uint32_t)wq[q].y * (uint32_t)sizeof(GX), full);
            off += (uint32_t)wq[q].y * (uint32_t)sizeof(GX);
        }
        if (wq[q].w > 0) {
            bulk_g2s(xs + off, gx + wq[q].z, (uint32_t)wq[q].w * (uint32_t)sizeof(GX), full);
            off += (uint32_t)wq[q].w * (uint32_t)sizeof(GX);
        }
    }
}

template <typename TM, int VEC, class Op, int NT = THREADS>
__global__ void __launch_bounds__(NT, 2) k_stream_win(int n, int rt, int cap, int xw, int ntiles,
                                                      const int *__restrict__ rp, const uint16_t *__restrict__ c16,
                                                      const TM *__restrict__ v, const int *__restrict__ wtab, Op op,
                                                      int *err, int stages) {
    using GX = typename Op::GX;
    extern __shared__ __align__(128) unsigned char smem[];
    const int STAGES = stages;
    constexpr int CONSUMER_WARPS = NT / 32 - 1;
    __shared__ __align__(8) uint64_t full[MAX_STAGES], empty[MAX_STAGES];
    const WLayout<TM, GX> L(rt, cap, xw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int k = 0; k < STAGES; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], CONSUMER_WARPS);
        }
        fence_mbar_init();
    }
    __syncthreads();
    __shared__ int2 m_se[META_T];
    __shared__ int4 m_w[META_T][WIN_NW / 2];
    const int my_tiles = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    {
        constexpr int PARTS = 1 + WIN_NW / 2;
        for (int q = tid; q < min(my_tiles, META_T) * PARTS; q += NT) {
            const int j = q / PARTS, part = q % PARTS;
            const int t = blockIdx.x + j * gridDim.x;
            if (part == 0) m_se[j] = make_int2(__ldg(rp + t * rt), __ldg(rp + min(t * rt + rt, n)));
            else m_w[j][part - 1] = __ldg(reinterpret_cast<const int4 *>(wtab) + (size_t)t * (WIN_NW / 2) + part - 1);
        }
    }
    __syncthreads();
    // The operator part of tile t (the CTA's j-th: row pointers, local
    // indices, values), its bytes expected without arriving: constant data,
    // so the first tiles' are copied before the dependency wait.
    auto issue_op = [&](int t, int j, int st) {
        unsigned char *stage = smem + st * L.stb;
        const int r0 = t * rt, r1 = min(r0 + rt, n);
        const int2 se = j < META_T ? m_se[j] : make_int2(__ldg(rp + r0), __ldg(rp + r1));
        const int s = se.x, e = se.y;
        const int rp_cnt = (r1 - r0 + 1 + 3) & ~3;  // r0 is a multiple of 4
        const int cs = s & ~7, ce = (e + 7) & ~7;
        constexpr int PER = 16 / sizeof(TM);
        const int vs = s & ~(PER - 1), ve = (e + PER - 1) & ~(PER - 1);
        int *hdr = reinterpret_cast<int *>(stage + L.rpb + L.cib + L.vab + L.xwb);
        hdr[0] = cs;
        hdr[1] = vs;
        const uint32_t b_rp = rp_cnt * 4, b_ci = (ce - cs) * 2, b_v = (ve - vs) * (uint32_t)sizeof(TM);
        mbar_expect_tx_only(&full[st], b_rp + b_ci + b_v);
        bulk_g2s(stage, rp + r0, b_rp, &full[st]);
        if (b_ci) bulk_g2s(stage + L.rpb, c16 + cs, b_ci, &full[st]);
        if (b_v) bulk_g2s(stage + L.rpb + L.cib, v + vs, b_v, &full[st]);
    };
    // The windows of the gathered vector for tile t (written by the
    // predecessor: after the dependency wait), expected with the producer's
    // arrival.
    auto issue_win = [&](int t, int j, int st) {
        unsigned char *stage = smem + st * L.stb;
        const int r0 = t * rt, r1 = min(r0 + rt, n);
        issue_windows<GX>(wtab, m_w, t, j, r0, r1, op.gsrc(), stage + L.rpb + L.cib + L.vab,
                          reinterpret_cast<int *>(stage + L.rpb + L.cib + L.vab + L.xwb) + 2, &full[st]);
    };
    int npre = 0;
    if (tid == 0)
        for (; npre < STAGES && (int)blockIdx.x + npre * (int)gridDim.x < ntiles; ++npre)
            issue_op(blockIdx.x + npre * gridDim.x, npre, npre);
    pdl_wait();
    pdl_trigger();
    const int ctl = blockIdx.x == 0 ? __ldcg(err + 1) : 0;  // in flight with the done flag's load
    if (op.done()) {
        // the prefetched copies land before the CTA leaves
        if (tid == 0)
            for (int k = 0; k < npre; ++k) {
                mbar_arrive(&full[k]);
                mbar_wait(&full[k], 0);
            }
        return;
    }
    const bool wh = test_withhold(ctl, err);
    const uint32_t lim = wh ? TEST_POLLS : WAIT_POLLS;
    double acc[2] = {0.0, 0.0};
    bool ok = true;
    if (warp == 0) {
        if (lane == 0) {
            for (int j = 0;; ++j) {
                const int t = blockIdx.x + j * gridDim.x;
                if (t >= ntiles) break;
                const int st = j % STAGES;
                if (j >= npre) {
                    if (!mbar_wait(&empty[st], (uint32_t)(((j / STAGES) - 1) & 1), lim)) {
                        ok = false;
                        break;
                    }
                    fence_proxy_async();
                    issue_op(t, j, st);
                }
                if (j == 0 && wh) mbar_expect_tx_only(&full[0], 16);  // bytes no copy delivers
                issue_win(t, j, st);
            }
        }
    } else {
        constexpr int UNR = VEC == 1 ? 8 : 4;
        const int ct = tid - 32;
        constexpr int ROWS_PER_PASS = CONSUMER_WARPS * 32 / VEC;
        const int rsub = ct / VEC, vl = ct % VEC;
        for (int j = 0;; ++j) {
            const int t = blockIdx.x + j * gridDim.x;
            if (t >= ntiles) break;
            const int st = j % STAGES;
            const int r0 = t * rt;
            const int rows = min(rt, n - r0);
            typename Op::Pre pre0{};
            if (rsub < rows && vl == 0) pre0 = op.load_rest(r0 + rsub);
            if (!__all_sync(0xffffffffu, mbar_wait(&full[st], (uint32_t)((j / STAGES) & 1), lim))) {  // warp-uniform
                ok = false;
                break;
            }
            const unsigned char *stage = smem + st * L.stb;
            const int *rps = reinterpret_cast<const int *>(stage);
            const uint16_t *cis = reinterpret_cast<const uint16_t *>(stage + L.rpb);
            const TM *vals = reinterpret_cast<const TM *>(stage + L.rpb + L.cib);
            const GX *xs = reinterpret_cast<const GX *>(stage + L.rpb + L.cib + L.vab);
            const int *hdr = reinterpret_cast<const int *>(stage + L.rpb + L.cib + L.vab + L.xwb);
            const int cs = hdr[0], vsb = hdr[1], dl0 = hdr[2];
            for (int base = 0; base < rows; base += ROWS_PER_PASS) {
                const int rl = base + rsub;
                TM sum = 0;
                typename Op::Pre pre = pre0;
                if (rl < rows) {
                    if (vl == 0 && base > 0) pre = op.load_rest(r0 + rl);
                    if (Op::SELF && vl == 0) op.put_self(pre, dl0 >= 0 ? xs[dl0 + rl] : __ldg(op.gsrc() + r0 + rl));
                    const int k1 = rps[rl + 1];
                    for (int kb = rps[rl] + vl; kb < k1; kb += UNR * VEC) {
#pragma unroll
                        for (int u = 0; u < UNR; ++u) {
                            const int k = kb + u * VEC;
                            if (k < k1) sum += vals[k - vsb] * fcvt<TM>(xs[cis[k - cs]]);
                        }
                    }
                }
                if (VEC > 1) sum = group_sum<VEC>(sum);
                if (vl == 0 && rl < rows) op.finish(r0 + rl, sum, pre, acc);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
        }
    }
    if (!ok) {
        atomicExch(err, 1);
        for (int k = 0; k < STAGES; ++k) mbar_try_wait(&full[k], 0);
    }
    op.template reduce<NT>(acc);
}

// ---------------------------------------------------------------------------
// Sliced-ELL variant: one thread per row, slot-major tiles
// ---------------------------------------------------------------------------
//
// The windowed layout with each 32-row slice's entries stored slot-major:
// entry u of row 32g + l sits at soff[g] + 32u + l, the slice padded to its
// longest row with zero values (whose local index is some valid window
// offset, so the padding adds +-0 to the row's sum).  A warp takes a slice,
// one lane per row: per slot its 32 lanes read 32 consecutive values and
// indices, and on stencil operators 32 consecutive entries of the staged
// vector, which is the fewest shared-memory wavefronts a stored entry can
// cost; the CSR kernels' lanes instead read entries strided by the row
// length.  Each row is summed in CSR order, and the epilogue runs on all 32
// lanes with coalesced loads and stores.  Tiles are rt rows, a multiple of
// 32; soff[g] is a multiple of 32 entries, so every bulk copy starts on a
// 16-byte boundary and moves a multiple of 16 bytes.
//
// The epilogue's own row operands (Op::rowv: up to three vectors indexed by
// row, e.g. the smoother weights and right-hand side) are staged too when
// `rows` is set: each tile's range of each vector, in whole 16-byte chunks,
// bulk-copied with the tile, so the epilogue reads shared memory instead of
// waiting on global loads.  The rows of a ragged chunk (the last tile's last
// n % 4 rows) and vectors not 16-byte aligned fall back to global loads.

constexpr int ROWV_MAX = 3;

template <typename TM, typename GX>
struct ELayout {
    int vab, cib, xwb, rvb, stb;
    // rvbytes: staged row-operand bytes per row (0: none)
    __host__ __device__ ELayout(int cap, int xw, int rt, int rvbytes)
        : vab(align16(cap * (int)sizeof(TM))), cib(align16(cap * 2)), xwb(align16(xw * (int)sizeof(GX))),
          rvb(rvbytes ? align16(rt * rvbytes + 16 * ROWV_MAX) : 0), stb(vab + cib + xwb + rvb + 16) {}
};

template <typename TM, typename GX>
inline int smem_bytes_ell(int cap, int xw, int rt, int rvbytes, int stages = WIN_STAGES) {
    return stages * ELayout<TM, GX>(cap, xw, rt, rvbytes).stb;
}

// One lane's row of a slice with exactly W slots: every value, index and
// staged-vector load issues before the first FMA; the sum keeps slot order.
template <int W, typename TM, typename GX>
__device__ __forceinline__ TM slot_sum(const TM *vp, const uint16_t *cp, const GX *xs) {
    TM a[W];
    int c[W];
#pragma unroll
    for (int q = 0; q < W; ++q) {
        a[q] = vp[q * 32];
        c[q] = cp[q * 32];
    }
    TM sum = 0;
#pragma unroll
    for (int q = 0; q < W; ++q) sum += a[q] * fcvt<TM>(xs[c[q]]);
    return sum;
}

template <typename TM, class Op, int NT = THREADS>
__global__ void __launch_bounds__(NT, 2) k_stream_ell(int n, int rt, int cap, int xw, int ntiles,
                                                      const int *__restrict__ soff, const uint16_t *__restrict__ ec,
                                                      const TM *__restrict__ ev, const int *__restrict__ wtab, Op op,
                                                      int rows, int *err, int stages) {
    using GX = typename Op::GX;
    extern __shared__ __align__(128) unsigned char smem[];
    const int STAGES = stages;
    constexpr int CONSUMER_WARPS = NT / 32 - 1;
    __shared__ __align__(8) uint64_t full[MAX_STAGES], empty[MAX_STAGES];
    const ELayout<TM, GX> L(cap, xw, rt, rows ? Op::ROWV_BYTES : 0);
    // the staged row operands: sources, element sizes, offsets in a stage
    const void *rsrc[ROWV_MAX] = {};
    int reb[ROWV_MAX] = {0, 0, 0}, roff[ROWV_MAX] = {0, 0, 0}, nrv = 0;
    if constexpr (Op::NROWV > 0) {
        if (rows) {
            nrv = op.rowv(rsrc, reb);
            int o = 0;
#pragma unroll
            for (int k = 0; k < ROWV_MAX; ++k) {
                if (k >= nrv) reb[k] = 0;
                else if (reinterpret_cast<uintptr_t>(rsrc[k]) & 15) nrv = 0;  // not bulk-copyable: global loads
                roff[k] = o;
                o += align16(rt * reb[k]);
            }
        }
    }
    const bool staged = nrv > 0;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int spt = rt >> 5;          // slices per tile
    const int nsl_all = (n + 31) >> 5;  // slices of the operator
    if (tid == 0) {
        for (int k = 0; k < STAGES; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], CONSUMER_WARPS);
        }
        fence_mbar_init();
    }
    __syncthreads();
    __shared__ int2 m_se[META_T];
    __shared__ int4 m_w[META_T][WIN_NW / 2];
    const int my_tiles = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    {
        constexpr int PARTS = 1 + WIN_NW / 2;
        for (int q = tid; q < min(my_tiles, META_T) * PARTS; q += NT) {
            const int j = q / PARTS, part = q % PARTS;
            const int t = blockIdx.x + j * gridDim.x;
            if (part == 0) m_se[j] = make_int2(__ldg(soff + t * spt), __ldg(soff + min(t * spt + spt, nsl_all)));
            else m_w[j][part - 1] = __ldg(reinterpret_cast<const int4 *>(wtab) + (size_t)t * (WIN_NW / 2) + part - 1);
        }
    }
    __syncthreads();
    // The operator part of tile t (values, local indices), its bytes expected
    // without arriving: constant data, copied for the first tiles before the
    // dependency wait.
    auto issue_op = [&](int t, int j, int st) {
        unsigned char *stage = smem + st * L.stb;
        const int g0 = t * spt;
        const int2 se = j < META_T ? m_se[j] : make_int2(__ldg(soff + g0), __ldg(soff + min(g0 + spt, nsl_all)));
        reinterpret_cast<int *>(stage + L.vab + L.cib + L.xwb + L.rvb)[0] = se.x;
        const uint32_t ne = (uint32_t)(se.y - se.x);
        const uint32_t b_v = ne * (uint32_t)sizeof(TM), b_c = ne * 2u;
        mbar_expect_tx_only(&full[st], b_v + b_c);
        if (ne) {
            bulk_g2s(stage, ev + se.x, b_v, &full[st]);
            bulk_g2s(stage + L.vab, ec + se.x, b_c, &full[st]);
        }
    };
    // the row operands and windows of tile t (written by predecessors: after
    // the dependency wait), the windows' copies arriving for the producer
    auto issue_win = [&](int t, int j, int st) {
        unsigned char *stage = smem + st * L.stb;
        const int r0 = t * rt, r1 = min(r0 + rt, n);
        if (staged) {
            const int rs = (r1 - r0) & ~3;  // whole 16-byte chunks of every operand
            uint32_t bytes = 0;
#pragma unroll
            for (int k = 0; k < ROWV_MAX; ++k) bytes += (uint32_t)(rs * reb[k]);
            if (bytes) {
                mbar_expect_tx_only(&full[st], bytes);
                unsigned char *rvb = stage + L.vab + L.cib + L.xwb;
#pragma unroll
                for (int k = 0; k < ROWV_MAX; ++k)
                    if (reb[k])
                        bulk_g2s(rvb + roff[k], static_cast<const unsigned char *>(rsrc[k]) + (size_t)r0 * reb[k],
                                 (uint32_t)(rs * reb[k]), &full[st]);
            }
        }
        issue_windows<GX>(wtab, m_w, t, j, r0, r1, op.gsrc(), stage + L.vab + L.cib,
                          reinterpret_cast<int *>(stage + L.vab + L.cib + L.xwb + L.rvb) + 1, &full[st]);
    };
    int npre = 0;
    if (tid == 0)
        for (; npre < STAGES && (int)blockIdx.x + npre * (int)gridDim.x < ntiles; ++npre)
            issue_op(blockIdx.x + npre * gridDim.x, npre, npre);
    pdl_wait();
    pdl_trigger();
    const int ctl = blockIdx.x == 0 ? __ldcg(err + 1) : 0;  // in flight with the done flag's load
    if (op.done()) {
        // the prefetched copies land before the CTA leaves
        if (tid == 0)
            for (int k = 0; k < npre; ++k) {
                mbar_arrive(&full[k]);
                mbar_wait(&full[k], 0);
            }
        return;
    }
    const bool wh = test_withhold(ctl, err);
    const uint32_t lim = wh ? TEST_POLLS : WAIT_POLLS;
    double acc[2] = {0.0, 0.0};
    bool ok = true;
    if (warp == 0) {
        if (lane == 0) {
            for (int j = 0;; ++j) {
                const int t = blockIdx.x + j * gridDim.x;
                if (t >= ntiles) break;
                const int st = j % STAGES;
                if (j >= npre) {
                    if (!mbar_wait(&empty[st], (uint32_t)(((j / STAGES) - 1) & 1), lim)) {
                        ok = false;
                        break;
                    }
                    fence_proxy_async();
                    issue_op(t, j, st);
                }
                if (j == 0 && wh) mbar_expect_tx_only(&full[0], 16);  // bytes no copy delivers
                issue_win(t, j, st);
            }
        }
    } else {
        const int cw = warp - 1;
        // the entry range of the warp's first slice of tile t, loaded a tile
        // ahead (the table is constant) so that its latency overlaps the
        // tile before instead of the stage wait alone
        auto first_range = [&](int t, int &a, int &b) {
            const int g0 = t * spt;
            if (cw < min(spt, nsl_all - g0)) {
                a = __ldg(soff + g0 + cw);
                b = __ldg(soff + g0 + cw + 1);
            }
        };
        int nb0 = 0, nb1 = 0;
        if ((int)blockIdx.x < ntiles) first_range(blockIdx.x, nb0, nb1);
        for (int j = 0;; ++j) {
            const int t = blockIdx.x + j * gridDim.x;
            if (t >= ntiles) break;
            const int st = j % STAGES;
            const int r0 = t * rt, g0 = t * spt;
            const int nsl = min(spt, nsl_all - g0);
            // the warp's first slice: its entry range (loaded during the tile
            // before) and the rows' epilogue operands, loaded before the stage
            // wait so the latencies overlap; then the next tile's range
            int sl = cw;
            int sb0 = nb0, sb1 = nb1;
            if (t + (int)gridDim.x < ntiles) first_range(t + gridDim.x, nb0, nb1);
            typename Op::Pre pre{};
            if (sl < nsl) {
                const int row = r0 + sl * 32 + lane;
                if (!staged && row < n) pre = op.load_rest(row);
            }
            if (!__all_sync(0xffffffffu, mbar_wait(&full[st], (uint32_t)((j / STAGES) & 1), lim))) {  // warp-uniform
                ok = false;
                break;
            }
            const unsigned char *stage = smem + st * L.stb;
            const TM *vals = reinterpret_cast<const TM *>(stage);
            const uint16_t *cis = reinterpret_cast<const uint16_t *>(stage + L.vab);
            const GX *xs = reinterpret_cast<const GX *>(stage + L.vab + L.cib);
            const int *hdr = reinterpret_cast<const int *>(stage + L.vab + L.cib + L.xwb + L.rvb);
            const int e0 = hdr[0], dl0 = hdr[1];
            const int rs = (min(r0 + rt, n) - r0) & ~3;  // rows whose operands are staged
            while (sl < nsl) {
                const int rl = sl * 32 + lane, row = r0 + rl;
                if constexpr (Op::NROWV > 0) {
                    if (staged) {
                        const unsigned char *rvb = stage + L.vab + L.cib + L.xwb;
                        const unsigned char *rv[ROWV_MAX] = {rvb + roff[0], rvb + roff[1], rvb + roff[2]};
                        if (rl < rs) pre = op.load_rowv(rv, rl);
                        else if (row < n) pre = op.load_rest(row);
                    }
                }
                const int wd = (sb1 - sb0) >> 5;  // warp-uniform
                const TM *vp = vals + (sb0 - e0) + lane;
                const uint16_t *cp = cis + (sb0 - e0) + lane;
                // stencil widths run fully unrolled (wd is warp-uniform)
                TM sum = 0;
                switch (wd) {
                    case 0: break;
                    case 1: sum = slot_sum<1>(vp, cp, xs); break;
                    case 2: sum = slot_sum<2>(vp, cp, xs); break;
                    case 3: sum = slot_sum<3>(vp, cp, xs); break;
                    case 4: sum = slot_sum<4>(vp, cp, xs); break;
                    case 5: sum = slot_sum<5>(vp, cp, xs); break;
                    case 6: sum = slot_sum<6>(vp, cp, xs); break;
                    case 7: sum = slot_sum<7>(vp, cp, xs); break;
                    case 8: sum = slot_sum<8>(vp, cp, xs); break;
                    default: {
                        int u = 0;
                        for (; u + 4 <= wd; u += 4) {
                            TM a[4];
                            int c[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                a[q] = vp[(u + q) * 32];
                                c[q] = cp[(u + q) * 32];
                            }
#pragma unroll
                            for (int q = 0; q < 4; ++q) sum += a[q] * fcvt<TM>(xs[c[q]]);
                        }
                        for (; u < wd; ++u) sum += vp[u * 32] * fcvt<TM>(xs[cp[u * 32]]);
                    }
                }
                if (row < n) {
                    if (Op::SELF) op.put_self(pre, dl0 >= 0 ? xs[dl0 + rl] : ldgv(op.gsrc() + row));
                    op.finish(row, sum, pre, acc);
                }
                sl += CONSUMER_WARPS;
                if (sl < nsl) {
                    sb0 = __ldg(soff + g0 + sl);
                    sb1 = __ldg(soff + g0 + sl + 1);
                    const int row2 = r0 + sl * 32 + lane;
                    if (!staged) pre = row2 < n ? op.load_rest(row2) : typename Op::Pre{};
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
        }
    }
    if (!ok) {
        atomicExch(err, 1);
        for (int k = 0; k < STAGES; ++k) mbar_try_wait(&full[k], 0);
    }
    op.template reduce<NT>(acc);
}

}  // namespace stream
}  // namespace amg

namespace amg {
namespace stream {

// ---------------------------------------------------------------------------
// Direct sliced-ELL variant: no bulk copies
// ---------------------------------------------------------------------------
//
// The sliced-ELL value layout (entry u of row 32g + l at soff[g] + 32u + l)
// read straight from global memory: a warp takes a 32-row slice, one lane
// per row, so each slot is one coalesced load of 32 values and one of 32
// column indices; the gathered vector is read from global memory (L2: the
// vectors of a pass fit in it), and the epilogue's row operands with
// coalesced loads issued before the row's.  IDX is int16_t (column minus row,
// for square operators whose couplings stay within 32767 rows) or int
// (absolute columns).  Padding slots hold value 0 and a valid column.  With
// many small independent loads per warp and no producer thread, the pass
// keeps more memory requests in flight than a tile ring whose copies are
// small; the autotuner times both.  Each row sums in slot (= CSR) order.
constexpr int DIRECT_THREADS = 256;

template <typename IDX>
__device__ __forceinline__ int direct_col(IDX c, int i) {
    if constexpr (sizeof(IDX) == 2) return i + (int)c;
    else return (int)c;
}

template <typename TM, typename IDX, class Op, bool WIDE, int NT = DIRECT_THREADS>
__global__ void __launch_bounds__(NT) k_ell_direct(int n, int nsl, const int *__restrict__ soff,
                                                    const IDX *__restrict__ ecol, const TM *__restrict__ ev, Op op) {
    constexpr int U = 8;  // slots whose loads are in flight together
    const int lane = threadIdx.x & 31;
    const int nw = (int)((gridDim.x * (unsigned)NT) >> 5);
    int g = (int)((blockIdx.x * (unsigned)NT + threadIdx.x) >> 5);
    // a slice's first U slots (values, columns): the operator is constant, so
    // the warp's first slice loads before the dependency wait; without WIDE
    // (every slice at most U slots wide) each next slice's loads also go out
    // behind the current slice's gathers
    TM a[U];
    IDX c[U];
    int s0 = 0, wd = 0;
    auto fetch = [&](int gg, TM (&av)[U], IDX (&cv)[U], int &s0v, int &wdv) {
        s0v = __ldg(soff + gg);
        wdv = (__ldg(soff + gg + 1) - s0v) >> 5;  // warp-uniform
#pragma unroll
        for (int q = 0; q < U; ++q)
            if (q < wdv) {
                av[q] = ldgv(ev + s0v + q * 32 + lane);
                cv[q] = __ldg(ecol + s0v + q * 32 + lane);
            }
    };
    if (g < nsl) fetch(g, a, c, s0, wd);
    pdl_wait();
    pdl_trigger();
    if (op.done()) return;
    double acc[2] = {0.0, 0.0};
    while (g < nsl) {
        const int i = g * 32 + lane;
        typename Op::Pre pre{};
        if (i < n) pre = op.load(i);
        TM x[U];
#pragma unroll
        for (int q = 0; q < U; ++q)
            if (q < wd) x[q] = op.gather(direct_col(c[q], i));
        const int gn = g + nw;
        TM sum = 0;
        if constexpr (!WIDE) {
            TM an[U];
            IDX cn[U];
            int s0n = 0, wdn = 0;
            if (gn < nsl) fetch(gn, an, cn, s0n, wdn);
#pragma unroll
            for (int q = 0; q < U; ++q)
                if (q < wd) sum += a[q] * x[q];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                a[q] = an[q];
                c[q] = cn[q];
            }
            s0 = s0n;
            wd = wdn;
        } else {
#pragma unroll
            for (int q = 0; q < U; ++q)
                if (q < wd) sum += a[q] * x[q];
            // slots beyond the first U: U at a time, loads first
            for (int u = U; u < wd; u += U) {
#pragma unroll
                for (int q = 0; q < U; ++q)
                    if (u + q < wd) {
                        a[q] = ldgv(ev + s0 + (u + q) * 32 + lane);
                        c[q] = __ldg(ecol + s0 + (u + q) * 32 + lane);
                    }
#pragma unroll
                for (int q = 0; q < U; ++q)
                    if (u + q < wd) x[q] = op.gather(direct_col(c[q], i));
#pragma unroll
                for (int q = 0; q < U; ++q)
                    if (u + q < wd) sum += a[q] * x[q];
            }
            if (gn < nsl) fetch(gn, a, c, s0, wd);
        }
        if (i < n) op.finish(i, sum, pre, acc);
        g = gn;
    }
    op.template reduce<NT>(acc);
}

}  // namespace stream
}  // namespace amg
