// stream.cuh -- row-tiled CSR passes staged through shared memory by TMA bulk
// copies (cp.async.bulk + mbarrier), used for every large operator of the
// V-cycle and the outer Krylov products.
//
// A persistent CTA walks the tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...
// of RT consecutive rows.  For each tile one thread issues three bulk copies
// into a pipeline stage: the tile's row pointers, column indices and values
// (each range rounded out to 16-byte boundaries; every array the library
// owns is padded so the rounded range stays inside its allocation).  STAGES
// tiles are in flight per CTA, so the copy engine keeps enough bytes moving to
// saturate HBM with few threads.  Consumers wait on the stage's mbarrier (a
// bounded wait), then VEC threads per row reduce the row from shared memory,
// gathering the input vector from global memory (L2), and an epilogue functor
// finishes the row.  Optional dot products end in the deterministic
// last-block reduction.
#pragma once

#include "amg_common.cuh"

namespace amg {
namespace stream {

constexpr int THREADS = 512;
constexpr int CAP = 4096;   // entries per stage (values and column indices)
constexpr int RT_MAX = 512;

template <typename TM>
struct Stages;
template <>
struct Stages<float> { static constexpr int N = 3; };
template <>
struct Stages<double> { static constexpr int N = 2; };

// Shared-memory layout of one stage (bytes, 16-byte multiples).
constexpr int RP_BYTES = (RT_MAX + 8) * 4;
constexpr int CI_BYTES = (CAP + 8) * 4;
template <typename TM>
constexpr int stage_bytes() { return RP_BYTES + CI_BYTES + (CAP + 8) * (int)sizeof(TM) + 16; }
template <typename TM>
constexpr int smem_bytes() { return Stages<TM>::N * stage_bytes<TM>(); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
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

// Bounded wait: gives up after 2^22 polls and reports it.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity) {
    for (uint32_t it = 0; it < (1u << 22); ++it)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}

// Issues the copies of tile t into stage buffers; called by one thread.
template <typename TM>
__device__ __forceinline__ void issue_tile(int t, int rt, int n, const int *__restrict__ rp,
                                           const int *__restrict__ ci, const TM *__restrict__ v,
                                           unsigned char *stage, uint64_t *bar) {
    const int r0 = t * rt;
    const int r1 = min(r0 + rt, n);
    const int s = __ldg(rp + r0), e = __ldg(rp + r1);
    const int rp_cnt = (r1 - r0 + 1 + 3) & ~3;                  // r0 is a multiple of 4
    const int cs = s & ~3, ce = (e + 3) & ~3;                   // int32: 4 per 16 bytes
    constexpr int PER = 16 / sizeof(TM);
    const int vs = s & ~(PER - 1), ve = (e + PER - 1) & ~(PER - 1);
    int *hdr = reinterpret_cast<int *>(stage + RP_BYTES + CI_BYTES + (CAP + 8) * sizeof(TM));
    hdr[0] = cs;
    hdr[1] = vs;
    const uint32_t b_rp = rp_cnt * 4, b_ci = (ce - cs) * 4, b_v = (ve - vs) * (uint32_t)sizeof(TM);
    mbar_expect_tx(bar, b_rp + b_ci + b_v);
    bulk_g2s(stage, rp + r0, b_rp, bar);
    if (b_ci) bulk_g2s(stage + RP_BYTES, ci + cs, b_ci, bar);
    if (b_v) bulk_g2s(stage + RP_BYTES + CI_BYTES, v + vs, b_v, bar);
}

// The row pass.  Op provides: bool done() const; TM gather(int j) const;
// void finish(int i, TM s, double* acc) const; void reduce(double* acc) const
// (called by every thread of every CTA at the end).
template <typename TM, int VEC, class Op>
__global__ void __launch_bounds__(THREADS) k_stream(int n, int rt, int ntiles, const int *__restrict__ rp,
                                                    const int *__restrict__ ci, const TM *__restrict__ v, Op op,
                                                    int *err) {
    constexpr int S = Stages<TM>::N;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[S];
    if (op.done()) return;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int k = 0; k < S; ++k) mbar_init(&bars[k], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < S; ++k) {
            const int t = blockIdx.x + k * gridDim.x;
            if (t < ntiles) issue_tile<TM>(t, rt, n, rp, ci, v, smem + k * stage_bytes<TM>(), &bars[k]);
        }
    double acc[2] = {0.0, 0.0};
    const int row_local = tid / VEC, lane = tid % VEC;
    bool ok = true;
    for (int j = 0;; ++j) {
        const int t = blockIdx.x + j * gridDim.x;
        if (t >= ntiles) break;
        const int st = j % S;
        unsigned char *stage = smem + st * stage_bytes<TM>();
        const bool got = mbar_wait(&bars[st], (uint32_t)((j / S) & 1));
        if (__syncthreads_or(!got)) {  // block-uniform decision
            ok = false;
            break;
        }
        const int *rps = reinterpret_cast<const int *>(stage);
        const int *cis = reinterpret_cast<const int *>(stage + RP_BYTES);
        const TM *vs_ = reinterpret_cast<const TM *>(stage + RP_BYTES + CI_BYTES);
        const int *hdr = reinterpret_cast<const int *>(stage + RP_BYTES + CI_BYTES + (CAP + 8) * sizeof(TM));
        const int cs = hdr[0], vsb = hdr[1];
        const int r0 = t * rt;
        const int rows = min(rt, n - r0);
        TM sum = 0;
        if (row_local < rows) {
            const int k1 = rps[row_local + 1];
            for (int k = rps[row_local] + lane; k < k1; k += VEC) sum += vs_[k - vsb] * op.gather(cis[k - cs]);
        }
        if (VEC > 1) sum = group_sum<VEC>(sum);
        if (lane == 0 && row_local < rows) op.finish(r0 + row_local, sum, acc);
        __syncthreads();  // every read of this stage is done
        if (tid == 0) {
            const int tn = t + S * gridDim.x;
            if (tn < ntiles) {
                fence_proxy_async();
                issue_tile<TM>(tn, rt, n, rp, ci, v, stage, &bars[st]);
            }
        }
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        // give the copies in flight a bounded chance to land before the CTA exits
        for (int k = 0; k < S; ++k) mbar_try_wait(&bars[k], 0);
    }
    op.reduce(acc);
}

}  // namespace stream
}  // namespace amg
