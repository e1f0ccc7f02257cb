// setup.cu -- construction of the smoothed-aggregation AMG hierarchy on the GPU.
//
// Every integer decision (strength, independent set, aggregates, sparsity
// patterns) is deterministic, and every floating-point value that feeds a
// later decision is computed in a fixed order with each multiply and add
// rounded separately (__dmul_rn / __dadd_rn / __ddiv_rn; this file is also
// built with -fmad=false), so the hierarchy does not depend on thread
// scheduling.  The steps are:
//   validation of the CSR input               (CSR normalisation, Sec. 2.1)
//   strength of connection S = S1 or S1^T      a_ij^2 >= theta_l^2 |a_ii a_jj|
//   distance-2 maximal independent set         synchronous rounds of max-tuple propagation
//   aggregates                                 roots, their neighbours, then best strong neighbour
//   prolongator P = (I - omega_P D^-1 A) T     omega_P = (4/3) / Gershgorin bound
//   R = P^T                                    CSR transpose
//   Galerkin A_c = R (A P)                     row-wise SpGEMM, fixed summation order
//   coarsest level                             dense Cholesky / LU, explicit inverse
#include <cstdarg>
#include <cstring>
#include <algorithm>
#include <vector>

#include "amg_common.cuh"

namespace amg {

static thread_local char g_last_error[1024] = "";

void set_last_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

const char *last_error() { return g_last_error; }

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 148;
    }
    return sms;
}

// ===========================================================================
// Exclusive scan of int counts (out has n + 1 entries; out[n] = total)
// ===========================================================================

constexpr int SCAN_T = 256, SCAN_I = 8, SCAN_TILE = SCAN_T * SCAN_I;

template <typename TIn, typename TOut>
__global__ void k_scan_tile(const TIn *in, TOut *out, long long *sums, int n) {
    __shared__ long long sh[SCAN_T];
    const int tid = threadIdx.x;
    const long long base = (long long)blockIdx.x * SCAN_TILE + (long long)tid * SCAN_I;
    long long v[SCAN_I];
    long long s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        v[i] = (base + i < n) ? (long long)in[base + i] : 0;
        s += v[i];
    }
    sh[tid] = s;
    __syncthreads();
    for (int off = 1; off < SCAN_T; off <<= 1) {
        long long add = tid >= off ? sh[tid - off] : 0;
        __syncthreads();
        sh[tid] += add;
        __syncthreads();
    }
    long long run = tid ? sh[tid - 1] : 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        if (base + i < n) out[base + i] = (TOut)run;
        run += v[i];
    }
    if (tid == SCAN_T - 1) sums[blockIdx.x] = sh[SCAN_T - 1];
}

template <typename TOut>
__global__ void k_scan_add(TOut *out, const long long *sums, int n) {
    long long i = (long long)blockIdx.x * SCAN_TILE + threadIdx.x;
    long long add = sums[blockIdx.x];
    for (int k = 0; k < SCAN_I; ++k, i += SCAN_T)
        if (i < n) out[i] = (TOut)((long long)out[i] + add);
}

// Exclusive scan of long long in place; returns the total.
static int scan_ll_inplace(long long *a, int n, long long *total, cudaStream_t s) {
    int nb = ceil_div(n, SCAN_TILE);
    long long *sums = nullptr;
    Scratch sc;
    AMG_TRY(sc.alloc(&sums, nb + 1));
    k_scan_tile<long long, long long><<<nb, SCAN_T, 0, s>>>(a, a, sums, n);
    AMG_LAUNCH_CHECK();
    if (nb > 1) {
        long long t = 0;
        AMG_TRY(scan_ll_inplace(sums, nb, &t, s));
        k_scan_add<long long><<<nb, SCAN_T, 0, s>>>(a, sums, n);
        AMG_LAUNCH_CHECK();
        *total = t;
    } else {
        AMG_CUDA_TRY(cudaMemcpyAsync(total, sums, sizeof(long long), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return AMG_OK;
}

int exclusive_scan_int(const int *in, int *out, int n, int *total_host, cudaStream_t s) {
    if (n <= 0) {
        AMG_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int), s));
        if (total_host) *total_host = 0;
        return AMG_OK;
    }
    int nb = ceil_div(n, SCAN_TILE);
    long long *sums = nullptr;
    Scratch sc;
    AMG_TRY(sc.alloc(&sums, nb + 1));
    k_scan_tile<int, int><<<nb, SCAN_T, 0, s>>>(in, out, sums, n);
    AMG_LAUNCH_CHECK();
    long long total = 0;
    if (nb > 1) {
        AMG_TRY(scan_ll_inplace(sums, nb, &total, s));
        k_scan_add<int><<<nb, SCAN_T, 0, s>>>(out, sums, n);
        AMG_LAUNCH_CHECK();
    } else {
        AMG_CUDA_TRY(cudaMemcpyAsync(&total, sums, sizeof(long long), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (total >= (1LL << 31) - 1) {
        set_last_error("scan total %lld exceeds the int32 index range", total);
        return AMG_ERR_UNSUPPORTED;
    }
    int t32 = (int)total;
    AMG_CUDA_TRY(cudaMemcpyAsync(out + n, &t32, sizeof(int), cudaMemcpyHostToDevice, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));  // t32 lives on this stack frame
    if (total_host) *total_host = t32;
    return AMG_OK;
}

// ===========================================================================
// Generic small kernels
// ===========================================================================

__global__ void k_fill_int(int *a, int n, int v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = v;
}

__global__ void k_iota(int *a, int n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = (int)i;
}

__global__ void k_fill_double(double *a, long long n, double v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = v;
}

// d[k] = v[k] as an unevaluated FP32 pair hi + lo (the double-FP32 copy of the
// finest operator for the mixed form's outer product).
__global__ void k_to_df(const double *__restrict__ v, DF *__restrict__ d, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        d[k] = df_split(v[k]);
}

__global__ void k_to_f32(const double *in, float *out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = __double2float_rn(in[i]);
}

static int grid_for(long long n, int threads = 256) {
    long long g = (n + threads - 1) / threads;
    long long cap = (long long)num_sms() * 16;
    return (int)std::max(1LL, std::min(g, cap));
}

// ===========================================================================
// CSR transpose (deterministic: each output row lists its columns ascending)
// ===========================================================================

__global__ void k_count_cols(const int *ci, long long nnz, int *cnt) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x)
        atomicAdd(&cnt[ci[k]], 1);
}

__global__ void k_transpose_scatter(int nrows, const int *rp, const int *ci, const double *v, int *next,
                                    int *tci, double *tv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += gridDim.x * blockDim.x)
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            int pos = atomicAdd(&next[ci[k]], 1);
            tci[pos] = i;
            if (v) tv[pos] = v[k];
        }
}

// One warp per segment: stable order by key (keys in a segment are unique),
// by rank counting.  Writes the sorted segment to (out_k, out_v).
__global__ void k_sort_segments(int nseg, const int *seg_ptr, const int *in_k, const double *in_v, int *out_k,
                                double *out_v) {
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int sgm = wid; sgm < nseg; sgm += nw) {
        const int s = seg_ptr[sgm], e = seg_ptr[sgm + 1];
        const int len = e - s;
        for (int a = lane; a < len; a += 32) {
            int key = in_k[s + a];
            int rank = 0;
            for (int b = 0; b < len; ++b) rank += in_k[s + b] < key;
            out_k[s + rank] = key;
            if (in_v) out_v[s + rank] = in_v[s + a];
        }
    }
}

int transpose_csr(const DevCSR &a, DevCSR &t, DevArena &arena, cudaStream_t s) {
    t.nrows = a.ncols;
    t.ncols = a.nrows;
    t.nnz = a.nnz;
    AMG_TRY(arena.alloc(&t.rp, (size_t)t.nrows + 1));
    AMG_TRY(arena.alloc(&t.ci, (size_t)std::max(1LL, a.nnz)));
    t.v = nullptr;
    if (a.v) AMG_TRY(arena.alloc(&t.v, (size_t)std::max(1LL, a.nnz)));
    Scratch sc;
    int *cnt, *next, *tmp_k;
    double *tmp_v = nullptr;
    AMG_TRY(sc.alloc(&cnt, (size_t)t.nrows + 1));
    AMG_TRY(sc.alloc(&next, (size_t)t.nrows + 1));
    AMG_TRY(sc.alloc(&tmp_k, (size_t)std::max(1LL, a.nnz)));
    if (a.v) AMG_TRY(sc.alloc(&tmp_v, (size_t)std::max(1LL, a.nnz)));
    AMG_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * ((size_t)t.nrows + 1), s));
    if (a.nnz > 0) {
        k_count_cols<<<grid_for(a.nnz), 256, 0, s>>>(a.ci, a.nnz, cnt);
        AMG_LAUNCH_CHECK();
    }
    int total = 0;
    AMG_TRY(exclusive_scan_int(cnt, t.rp, t.nrows, &total, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(next, t.rp, sizeof(int) * ((size_t)t.nrows + 1), cudaMemcpyDeviceToDevice, s));
    if (a.nnz > 0) {
        k_transpose_scatter<<<grid_for(a.nrows), 256, 0, s>>>(a.nrows, a.rp, a.ci, a.v, next, tmp_k, tmp_v);
        AMG_LAUNCH_CHECK();
        k_sort_segments<<<grid_for((long long)t.nrows * 32), 256, 0, s>>>(t.nrows, t.rp, tmp_k, tmp_v, t.ci, t.v);
        AMG_LAUNCH_CHECK();
    }
    AMG_CUDA_TRY(cudaStreamSynchronize(s));  // scratch is freed on return
    return AMG_OK;
}

// ===========================================================================
// Validation and diagonal
// ===========================================================================

// Per row, the first violation in storage order: code 1 = bad CSR, 2 = zero
// or missing diagonal.  The lowest failing row wins (key = row * 4 + code).
__global__ void k_validate(int n, long long nnz, const int *rp, const int *ci, const double *v, int *diag_pos,
                           unsigned long long *first_err) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int code = 0;
        const int s = rp[i], e = rp[i + 1];
        int dpos = -1;
        if (e < s || s < 0 || (long long)e > nnz) {
            code = 1;
        } else {
            for (int k = s; k < e; ++k) {
                const int c = ci[k];
                if (c < 0 || c >= n || (k > s && c <= ci[k - 1])) { code = 1; break; }
                if (c == i) {
                    dpos = k;
                    if (v[k] == 0.0) { code = 2; break; }
                }
            }
            if (!code && dpos < 0) code = 2;
        }
        diag_pos[i] = dpos;
        if (code) atomicMin(first_err, (unsigned long long)i * 4ull + (unsigned long long)code);
    }
}

__global__ void k_find_diag(int n, const int *rp, const int *ci, const double *v, double *diag, int *bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] == i) { d = v[k]; break; }
        diag[i] = d;
        if (d == 0.0) atomicExch(bad, 1);
    }
}

// Bitwise comparison of A and its transpose (symmetry detection).
__global__ void k_compare_csr(int n, long long nnz, const int *rp1, const int *ci1, const double *v1,
                              const int *rp2, const int *ci2, const double *v2, int *differ) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz + n + 1;
         k += (long long)gridDim.x * blockDim.x) {
        bool d;
        if (k < nnz)
            d = ci1[k] != ci2[k] || __double_as_longlong(v1[k]) != __double_as_longlong(v2[k]);
        else
            d = rp1[k - nnz] != rp2[k - nnz];
        if (d) atomicExch(differ, 1);
    }
}

// ===========================================================================
// Strength of connection
// ===========================================================================

__device__ __forceinline__ bool strong_link(double aij, double aii, double ajj, double t2) {
    const double lhs = __dmul_rn(aij, aij);
    const double prod = __dmul_rn(aii, ajj);
    const double rhs = __dmul_rn(t2, fabs(prod));
    return lhs >= rhs;
}

template <bool FILL>
__global__ void k_strength(int n, const int *rp, const int *ci, const double *v, const double *diag, double t2,
                           int *cnt, const int *srp, int *sci) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double aii = diag[i];
        int c = 0;
        int pos = FILL ? srp[i] : 0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            const int j = ci[k];
            if (j == i) continue;
            if (strong_link(v[k], aii, diag[j], t2)) {
                if (FILL) sci[pos++] = j;
                else c++;
            }
        }
        if (!FILL) cnt[i] = c;
    }
}

// Union of two ascending column lists per row.
template <bool FILL>
__global__ void k_union(int n, const int *arp, const int *aci, const int *brp, const int *bci, int *cnt,
                        const int *orp, int *oci) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int p = arp[i], pe = arp[i + 1], q = brp[i], qe = brp[i + 1];
        int pos = FILL ? orp[i] : 0, c = 0;
        while (p < pe || q < qe) {
            int col;
            if (q >= qe || (p < pe && aci[p] < bci[q])) col = aci[p++];
            else if (p >= pe || bci[q] < aci[p]) col = bci[q++];
            else { col = aci[p]; ++p; ++q; }
            if (FILL) oci[pos++] = col;
            else c++;
        }
        if (!FILL) cnt[i] = c;
    }
}

// ===========================================================================
// Distance-2 maximal independent set by synchronous rounds
// ===========================================================================
// Node tuple = (state << 32) | fmix32(local index), state IN = 2 > UNDECIDED = 1
// > OUT = 0.  fmix32 (MurmurHash3's finaliser) is a bijection of 32-bit words,
// and two nodes within distance 2 always belong to the same system, so tuples
// within any neighbourhood are distinct.

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__global__ void k_mis_init(int n, const int *row_start, unsigned long long *t) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int local = row_start ? i - row_start[i] : i;
        t[i] = (1ull << 32) | (unsigned long long)fmix32((uint32_t)local);
    }
}

__global__ void k_mis_max(int n, const int *srp, const int *sci, const unsigned long long *in,
                          unsigned long long *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        unsigned long long m = in[i];
        for (int p = srp[i]; p < srp[i + 1]; ++p) m = max(m, in[sci[p]]);
        out[i] = m;
    }
}

__global__ void k_mis_update(int n, const int *srp, const int *sci, const unsigned long long *m1,
                             unsigned long long *t, int *undecided) {
    int und = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned long long ti = t[i];
        if ((ti >> 32) != 1ull) continue;
        unsigned long long m = m1[i];
        for (int p = srp[i]; p < srp[i + 1]; ++p) m = max(m, m1[sci[p]]);
        if (m == ti) t[i] = (2ull << 32) | (ti & 0xffffffffull);
        else if ((m >> 32) == 2ull) t[i] = ti & 0xffffffffull;
        else und++;
    }
    und = __reduce_add_sync(0xffffffffu, und);
    if ((threadIdx.x & 31) == 0 && und) atomicAdd(undecided, und);
}

// ===========================================================================
// Aggregation
// ===========================================================================

// active (may be null): rows of systems still coarsening in a batch.
// ===========================================================================
// Classical (Ruge-Stueben) coarsening: strength, PMIS splitting, direct
// interpolation (amg_type = AMG_TYPE_CLASSICAL; the same readings as the
// oracle, step for step)
// ===========================================================================

constexpr double THETA_CLASSICAL = 0.25;

// Strong dependencies of row i: j != i with -a_ij >= 1/4 max_{k != i}(-a_ik)
// and that maximum positive.  FILL = false counts per row, true fills.
template <bool FILL>
__global__ void k_strength_classical(int n, const int *rp, const int *ci, const double *v, int *cnt, const int *srp,
                                     int *sci) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double m = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] != i && -v[k] > m) m = -v[k];
        const double thr = m > 0.0 ? __dmul_rn(THETA_CLASSICAL, m) : -1.0;
        int c = 0, pos = FILL ? srp[i] : 0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            const int j = ci[k];
            if (j == i || thr < 0.0 || !(-v[k] >= thr)) continue;
            if (FILL) sci[pos++] = j;
            else ++c;
        }
        if (!FILL) cnt[i] = c;
    }
}

// PMIS weights w_i = |S^T_i| + fmix32(i) 2^-32; points influencing none start F.
__global__ void k_pmis_init(int n, const int *strp, double *w, int *st) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        w[i] = (double)(strp[i + 1] - strp[i]) + ldexp((double)fmix32((uint32_t)i), -32);
        st[i] = w[i] < 1.0 ? 0 : -1;
    }
}

// A round's selection, from the state at its start: an undecided point whose
// weight exceeds every undecided neighbour's in S_i and S^T_i becomes C.
__global__ void k_pmis_select(int n, const int *srp, const int *sci, const int *strp, const int *stci, const double *w,
                              const int *st, int *newc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int best = st[i] < 0;
        for (int k = srp[i]; k < srp[i + 1] && best; ++k) {
            const int j = sci[k];
            if (st[j] < 0 && w[j] >= w[i]) best = 0;
        }
        for (int k = strp[i]; k < strp[i + 1] && best; ++k) {
            const int j = stci[k];
            if (st[j] < 0 && w[j] >= w[i]) best = 0;
        }
        newc[i] = best;
    }
}

// The round's update: new C points, then undecided points with a strong
// dependency on a new C point become F; *und counts the undecided left.
__global__ void k_pmis_update(int n, const int *srp, const int *sci, const int *newc, int *st, int *und) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (newc[i]) {
            st[i] = 1;
            continue;
        }
        if (st[i] >= 0) continue;
        bool f = false;
        for (int k = srp[i]; k < srp[i + 1] && !f; ++k) f = newc[sci[k]] != 0;
        if (f) st[i] = 0;
        else atomicAdd(und, 1);
    }
}

__global__ void k_c_flags(int n, const int *st, int *flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) flag[i] = st[i] == 1;
}

__global__ void k_c_index(int n, const int *st, const int *scan, int *cidx) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        cidx[i] = st[i] == 1 ? scan[i] : -1;
}

// Direct interpolation.  FILL = false counts each row's entries (a C row 1,
// an F row its strong C dependencies); FILL = true writes them: a C row the
// unit entry, an F row w_ij = -(alpha a_ij) / d with alpha = (sum of the
// negative off-diagonal a_ik) / (sum over its strong C dependencies) and
// d = a_ii + (sum of the positive off-diagonal a_ik), sums in CSR order.
template <bool FILL>
__global__ void k_interp_direct(int n, const int *rp, const int *ci, const double *v, const int *srp, const int *sci,
                                const int *cidx, int *cnt, const int *prp, int *pci, double *pv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (cidx[i] >= 0) {
            if (FILL) {
                pci[prp[i]] = cidx[i];
                pv[prp[i]] = 1.0;
            } else {
                cnt[i] = 1;
            }
            continue;
        }
        double neg = 0.0, posv = 0.0, negc = 0.0, aii = 0.0;
        int nc_i = 0;
        int sp = srp[i];
        const int se = srp[i + 1];
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            const int j = ci[k];
            const double a = v[k];
            if (j == i) {
                aii = a;
                continue;
            }
            if (a < 0.0) neg = __dadd_rn(neg, a);
            else posv = __dadd_rn(posv, a);
            while (sp < se && sci[sp] < j) ++sp;
            if (sp < se && sci[sp] == j && cidx[j] >= 0) {
                negc = __dadd_rn(negc, a);
                ++nc_i;
            }
        }
        if (negc == 0.0) nc_i = 0;  // no strong C dependency: an empty row
        if (!FILL) {
            cnt[i] = nc_i;
            continue;
        }
        if (nc_i == 0) continue;
        const double alpha = __ddiv_rn(neg, negc), d = __dadd_rn(aii, posv);
        int pos = prp[i];
        sp = srp[i];
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            const int j = ci[k];
            if (j == i) continue;
            while (sp < se && sci[sp] < j) ++sp;
            if (sp < se && sci[sp] == j && cidx[j] >= 0) {
                pci[pos] = cidx[j];
                pv[pos] = __ddiv_rn(-__dmul_rn(alpha, v[k]), d);
                ++pos;
            }
        }
    }
}

// Re-setup of a classical level's interpolation: P's pattern (each F row's
// interpolation set, as coarse columns) and the C/F map are kept; the
// direct-interpolation weights are recomputed from the new values, the sum
// over the set taken whatever the new entries' signs, zero weights where it
// is zero.  C rows keep their unit entries.
__global__ void k_interp_direct_values(int n, const int *rp, const int *ci, const double *v, const int *cidx,
                                       const int *prp, const int *pci, double *pv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p0 = prp[i], p1 = prp[i + 1];
        if (cidx[i] >= 0 || p0 == p1) continue;
        double neg = 0.0, posv = 0.0, negc = 0.0, aii = 0.0;
        int q = p0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            const int j = ci[k];
            const double a = v[k];
            if (j == i) {
                aii = a;
                continue;
            }
            if (a < 0.0) neg = __dadd_rn(neg, a);
            else posv = __dadd_rn(posv, a);
            const int c = cidx[j];
            if (c >= 0) {
                while (q < p1 && pci[q] < c) ++q;
                if (q < p1 && pci[q] == c) negc = __dadd_rn(negc, a);
            }
        }
        q = p0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            const int j = ci[k];
            const int c = cidx[j];
            if (j == i || c < 0) continue;
            while (q < p1 && pci[q] < c) ++q;
            if (q < p1 && pci[q] == c) {
                if (negc == 0.0) {
                    pv[q] = 0.0;
                    continue;
                }
                const double alpha = __ddiv_rn(neg, negc), d = __dadd_rn(aii, posv);
                pv[q] = __ddiv_rn(-__dmul_rn(alpha, v[k]), d);
            }
        }
    }
}

__global__ void k_root_flags(int n, const unsigned long long *t, int *flag, const unsigned char *active = nullptr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flag[i] = (t[i] >> 32) == 2ull && (!active || active[i]);
}

// Phases 1-2: roots take their id; a non-root adjacent to a root takes that
// root's aggregate (unique: roots are at least 3 apart).
__global__ void k_agg_phase12(int n, const int *srp, const int *sci, const unsigned long long *t,
                              const int *root_id, int *snap,
                              const unsigned char *active = nullptr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int a = -1;
        if (active && !active[i]) {
            a = -1;
        } else if ((t[i] >> 32) == 2ull) {
            a = root_id[i];
        } else {
            for (int p = srp[i]; p < srp[i + 1]; ++p) {
                const int j = sci[p];
                if ((t[j] >> 32) == 2ull) { a = root_id[j]; break; }
            }
        }
        snap[i] = a;
    }
}

// Phase 3: an unassigned node joins the aggregate of the phase-2-assigned
// strong neighbour j with the largest |a_ij| (0 when (i,j) is not stored);
// ties go to the smallest j.  Reads only the phase-2 snapshot.
__global__ void k_agg_phase3(int n, const int *rp, const int *ci, const double *v, const int *srp,
                             const int *sci, const int *snap, int *agg, int *unassigned,
                             const unsigned char *active = nullptr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int a = snap[i];
        if (active && !active[i]) {
            agg[i] = -1;
            unassigned[i] = 0;
            continue;
        }
        if (a < 0) {
            int best = -1;
            double bw = -1.0;
            int k = rp[i];
            const int ke = rp[i + 1];
            for (int p = srp[i]; p < srp[i + 1]; ++p) {
                const int j = sci[p];
                while (k < ke && ci[k] < j) ++k;  // both lists ascend
                if (snap[j] < 0) continue;
                const double w = (k < ke && ci[k] == j) ? fabs(v[k]) : 0.0;
                if (w > bw) { bw = w; best = j; }
            }
            a = best >= 0 ? snap[best] : -1;
        }
        agg[i] = a;
        unassigned[i] = a < 0;
    }
}

__global__ void k_agg_singletons(int n, const int *rank, int base, int *agg) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (agg[i] < 0) agg[i] = base + rank[i];
}

// ===========================================================================
// Prolongator pieces
// ===========================================================================

// rho_i = (sum_j |a_ij| in storage order) / |a_ii|; the maximum is taken over
// the bit patterns (non-negative doubles order like their bits).
__global__ void k_gershgorin(int n, const int *rp, const double *v, const double *diag,
                             unsigned long long *rho_bits) {
    unsigned long long m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) s = __dadd_rn(s, fabs(v[k]));
        const double q = __ddiv_rn(s, fabs(diag[i]));
        m = max(m, (unsigned long long)__double_as_longlong(q));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(rho_bits, m);
}

__global__ void k_smoother_weights(int n, const int *rp, const double *v, const double *diag, double omega,
                                   int l1, double *w) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (l1) {
            double s = 0.0;
            for (int k = rp[i]; k < rp[i + 1]; ++k) s = __dadd_rn(s, fabs(v[k]));
            w[i] = __ddiv_rn(1.0, s);
        } else {
            w[i] = __ddiv_rn(omega, diag[i]);
        }
    }
}

// ===========================================================================
// Row-wise SpGEMM C = X Y with a per-warp hash accumulator in shared memory
// ===========================================================================
// One warp builds one row of C.  The entries of row i of X are taken one at a
// time in storage (ascending column) order; the lanes spread over the
// matching row of Y, whose columns are distinct, so within a step no two
// lanes touch the same accumulator.  Hence for each (i, J) the products
// x_ik y_kJ are added in increasing k, starting from +0.0, each product and
// sum rounded separately: the order the FP64 reference computes in.
// Symbolic pass: counts distinct columns.  Numeric pass: values, then the row
// is compacted and sorted by column (rank counting) and written.
// A row whose distinct count does not fit the table is listed in `overflow`
// and redone by a second launch with one larger table per block.

constexpr int SPG_EMPTY = -1;

enum { EPI_NONE = 0, EPI_PROLONG = 1 };

struct ProlongEpi {
    const int *agg;      // aggregate of each fine row
    const double *diag;  // a_ii
    double omega_p;      // (4/3) / rho
    const double *omega_row = nullptr;  // per-row omega_P (block-diagonal batches: per system), or null
};

template <bool NUMERIC, int EPI>
__global__ void k_spgemm(int nrows, const int *xrp, const int *xci, const double *xv, const int *yrp,
                         const int *yci, const double *yv, int hcap, const int *row_list, int nlist,
                         int *cnt_out, const int *crp, int *cci, double *cv, ProlongEpi epi, int *overflow_rows,
                         int *overflow_count) {
    extern __shared__ unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    int *keys = reinterpret_cast<int *>(smem_raw) + (size_t)wib * hcap;
    double *vals = reinterpret_cast<double *>(smem_raw + (size_t)wpb * hcap * sizeof(int)) + (size_t)wib * hcap;
    const int mask = hcap - 1;
    const int nwork = row_list ? nlist : nrows;
    for (int w = blockIdx.x * wpb + wib; w < nwork; w += gridDim.x * wpb) {
        const int i = row_list ? row_list[w] : w;
        for (int s = lane; s < hcap; s += 32) {
            keys[s] = SPG_EMPTY;
            if (NUMERIC) vals[s] = 0.0;
        }
        __syncwarp();
        bool ovf = false;
        const int pe = xrp[i + 1];
        for (int p = xrp[i]; p < pe && !ovf; ++p) {
            const int k = xci[p];
            const double xk = NUMERIC ? (xv ? xv[p] : 1.0) : 0.0;
            const int qe = yrp[k + 1];
            for (int q0 = yrp[k]; q0 < qe; q0 += 32) {
                const int q = q0 + lane;
                bool lane_ovf = false;
                if (q < qe) {
                    const int J = yci[q];
                    unsigned h = ((unsigned)J * 2654435761u) & (unsigned)mask;
                    int probes = 0;
                    int slot = -1;
                    while (probes < hcap) {
                        int cur = keys[h];
                        if (cur == J) { slot = (int)h; break; }
                        if (cur == SPG_EMPTY) {
                            int prev = atomicCAS(&keys[h], SPG_EMPTY, J);
                            if (prev == SPG_EMPTY || prev == J) { slot = (int)h; break; }
                        }
                        h = (h + 1) & (unsigned)mask;
                        ++probes;
                    }
                    if (slot < 0) lane_ovf = true;
                    else if (NUMERIC) {
                        const double yJ = yv ? yv[q] : 1.0;
                        vals[slot] = __dadd_rn(vals[slot], __dmul_rn(xk, yJ));
                    }
                }
                __syncwarp();
                if (__any_sync(0xffffffffu, lane_ovf)) { ovf = true; break; }
            }
        }
        // count (and compact in place, preserving slot order)
        int count = 0;
        if (!ovf) {
            for (int base = 0; base < hcap; base += 32) {
                const int s = base + lane;
                const int key = keys[s];
                double val = NUMERIC ? vals[s] : 0.0;
                const unsigned ball = __ballot_sync(0xffffffffu, key != SPG_EMPTY);
                const int pos = count + __popc(ball & ((1u << lane) - 1u));
                __syncwarp();
                if (key != SPG_EMPTY) {
                    keys[pos] = key;
                    if (NUMERIC) vals[pos] = val;
                }
                __syncwarp();
                count += __popc(ball);
            }
            // A table filled beyond 3/4 is treated as an overflow so that probing stays short.
            if (count > (hcap * 3) / 4) ovf = true;
        }
        if (ovf) {
            if (lane == 0) {
                int slot_o = atomicAdd(overflow_count, 1);
                overflow_rows[slot_o] = i;
            }
            __syncwarp();
            continue;
        }
        if (!NUMERIC) {
            if (lane == 0) cnt_out[i] = count;
        } else {
            const int out0 = crp[i];
            for (int a = lane; a < count; a += 32) {
                const int key = keys[a];
                int rank = 0;
                for (int b = 0; b < count; ++b) rank += keys[b] < key;
                double val = vals[a];
                if (EPI == EPI_PROLONG) {
                    const double t = __ddiv_rn(val, epi.diag[i]);
                    const double delta = (key == epi.agg[i]) ? 1.0 : 0.0;
                    const double om = epi.omega_row ? epi.omega_row[i] : epi.omega_p;
                    val = __dsub_rn(delta, __dmul_rn(om, t));
                }
                cci[out0 + rank] = key;
                cv[out0 + rank] = val;
            }
        }
        __syncwarp();
    }
}

// C = X Y (X: nrows x *, Y: * x ncols).  xv/yv may be null (all ones).
template <int EPI>
static int spgemm(int nrows, int ncols, const int *xrp, const int *xci, const double *xv, const int *yrp,
                  const int *yci, const double *yv, ProlongEpi epi, DevCSR &C, DevArena &arena, cudaStream_t s) {
    C.nrows = nrows;
    C.ncols = ncols;
    Scratch sc;
    int *cnt, *ovf_rows, *ovf_cnt;
    AMG_TRY(sc.alloc(&cnt, (size_t)nrows + 1));
    AMG_TRY(sc.alloc(&ovf_rows, (size_t)nrows + 1));
    AMG_TRY(sc.alloc(&ovf_cnt, 2));
    AMG_TRY(arena.alloc(&C.rp, (size_t)nrows + 1));
    const int small_cap = 512, warps = 8;
    const size_t small_smem = (size_t)warps * small_cap * (sizeof(int) + sizeof(double));
    int big_cap = 8192;
    size_t big_smem = (size_t)big_cap * (sizeof(int) + sizeof(double));
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    while (big_smem > (size_t)optin && big_cap > 1024) {
        big_cap >>= 1;
        big_smem = (size_t)big_cap * (sizeof(int) + sizeof(double));
    }
    AMG_CUDA_TRY(cudaFuncSetAttribute(k_spgemm<false, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big_smem));
    AMG_CUDA_TRY(cudaFuncSetAttribute(k_spgemm<true, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big_smem));

    for (int pass = 0; pass < 2; ++pass) {
        const bool numeric = pass == 1;
        AMG_CUDA_TRY(cudaMemsetAsync(ovf_cnt, 0, sizeof(int), s));
        const int blocks = (int)std::min<long long>((nrows + warps - 1) / warps, (long long)num_sms() * 8);
        if (!numeric)
            k_spgemm<false, EPI><<<std::max(blocks, 1), warps * 32, small_smem, s>>>(
                nrows, xrp, xci, xv, yrp, yci, yv, small_cap, nullptr, 0, cnt, nullptr, nullptr, nullptr, epi,
                ovf_rows, ovf_cnt);
        else
            k_spgemm<true, EPI><<<std::max(blocks, 1), warps * 32, small_smem, s>>>(
                nrows, xrp, xci, xv, yrp, yci, yv, small_cap, nullptr, 0, nullptr, C.rp, C.ci, C.v, epi, ovf_rows,
                ovf_cnt);
        AMG_LAUNCH_CHECK();
        int novf = 0;
        AMG_CUDA_TRY(cudaMemcpyAsync(&novf, ovf_cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        if (novf > 0) {
            AMG_CUDA_TRY(cudaMemsetAsync(ovf_cnt, 0, sizeof(int), s));
            int *ovf2;
            AMG_TRY(sc.alloc(&ovf2, (size_t)novf + 1));
            const int blocks2 = std::min(novf, num_sms() * 2);
            if (!numeric)
                k_spgemm<false, EPI><<<blocks2, 32, big_smem, s>>>(nrows, xrp, xci, xv, yrp, yci, yv, big_cap,
                                                                   ovf_rows, novf, cnt, nullptr, nullptr, nullptr,
                                                                   epi, ovf2, ovf_cnt);
            else
                k_spgemm<true, EPI><<<blocks2, 32, big_smem, s>>>(nrows, xrp, xci, xv, yrp, yci, yv, big_cap,
                                                                  ovf_rows, novf, nullptr, C.rp, C.ci, C.v, epi,
                                                                  ovf2, ovf_cnt);
            AMG_LAUNCH_CHECK();
            int novf2 = 0;
            AMG_CUDA_TRY(cudaMemcpyAsync(&novf2, ovf_cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
            AMG_CUDA_TRY(cudaStreamSynchronize(s));
            if (novf2 > 0) {
                set_last_error("a product row has more than %d distinct columns", (big_cap * 3) / 4);
                return AMG_ERR_UNSUPPORTED;
            }
        }
        if (!numeric) {
            int total = 0;
            AMG_TRY(exclusive_scan_int(cnt, C.rp, nrows, &total, s));
            C.nnz = total;
            AMG_TRY(arena.alloc(&C.ci, (size_t)std::max(1, total)));
            AMG_TRY(arena.alloc(&C.v, (size_t)std::max(1, total)));
        }
    }
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    return AMG_OK;
}

// Numeric products on a known pattern (re-setup): C = X Y where C's sorted
// row pattern (crp, cci) is that of an earlier product of the same patterns.
// Every product x_ik y_kJ is added at J's position in its row (binary search
// of the row's columns), in increasing k as in k_spgemm -- whose results
// these kernels equal bit for bit -- and the epilogue runs on the finished
// sums.  A product outside the pattern (never, for the setup's patterns) is
// reported through *bad and dropped.  Two shapes:
//   k_spgemm_known_thread: a thread per output row, for products whose rows
//     pair few entries (the finest levels): 32 rows' loads in flight per warp;
//   k_spgemm_known_warp: a warp per output row, entries of X in order and the
//     lanes over the (distinct) columns of each Y row, the row's columns and
//     sums in shared memory when it has at most KCAP entries.
constexpr int KCAP = 512;
constexpr int KWARPS = 8;

__device__ __forceinline__ int lower_bound_col(const int *c, int n, int J) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (c[mid] < J) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <int EPI>
__device__ __forceinline__ double prolong_epilogue(double val, int col, int i, const ProlongEpi &epi) {
    if (EPI == EPI_PROLONG) {
        const double t = __ddiv_rn(val, epi.diag[i]);
        const double delta = (col == epi.agg[i]) ? 1.0 : 0.0;
        const double om = epi.omega_row ? epi.omega_row[i] : epi.omega_p;
        val = __dsub_rn(delta, __dmul_rn(om, t));
    }
    return val;
}

template <int EPI>
__global__ void __launch_bounds__(256) k_spgemm_known_thread(int nrows, const int *__restrict__ xrp,
                                                            const int *__restrict__ xci, const double *__restrict__ xv,
                                                            const int *__restrict__ yrp, const int *__restrict__ yci,
                                                            const double *__restrict__ yv,
                                                            const int *__restrict__ crp, const int *__restrict__ cci,
                                                            double *cv, ProlongEpi epi, int *bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += gridDim.x * blockDim.x) {
        const int c0 = crp[i], cn = crp[i + 1] - c0;
        const int *cols = cci + c0;
        double *vals = cv + c0;
        for (int a = 0; a < cn; ++a) vals[a] = 0.0;
        const int pe = xrp[i + 1];
        for (int p = xrp[i]; p < pe; ++p) {
            const int k = xci[p];
            const double xk = xv ? xv[p] : 1.0;
            const int qe = yrp[k + 1];
            for (int q = yrp[k]; q < qe; ++q) {
                const int J = yci[q];
                const int pos = lower_bound_col(cols, cn, J);
                if (pos >= cn || cols[pos] != J) {
                    atomicExch(bad, 1);
                    continue;
                }
                vals[pos] = __dadd_rn(vals[pos], __dmul_rn(xk, yv ? yv[q] : 1.0));
            }
        }
        if (EPI == EPI_PROLONG)
            for (int a = 0; a < cn; ++a) vals[a] = prolong_epilogue<EPI>(vals[a], cols[a], i, epi);
    }
}

template <int EPI>
__global__ void __launch_bounds__(KWARPS * 32) k_spgemm_known_warp(int nrows, const int *__restrict__ xrp,
                                                                  const int *__restrict__ xci,
                                                                  const double *__restrict__ xv,
                                                                  const int *__restrict__ yrp,
                                                                  const int *__restrict__ yci,
                                                                  const double *__restrict__ yv,
                                                                  const int *__restrict__ crp,
                                                                  const int *__restrict__ cci, double *cv,
                                                                  ProlongEpi epi, int *bad) {
    __shared__ int s_cols[KWARPS][KCAP];
    __shared__ double s_vals[KWARPS][KCAP];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int i = blockIdx.x * KWARPS + wib; i < nrows; i += gridDim.x * KWARPS) {
        const int c0 = crp[i], cn = crp[i + 1] - c0;
        const bool staged = cn <= KCAP;
        const int *cols = staged ? s_cols[wib] : cci + c0;
        double *vals = staged ? s_vals[wib] : cv + c0;
        for (int a = lane; a < cn; a += 32) {
            if (staged) s_cols[wib][a] = cci[c0 + a];
            vals[a] = 0.0;
        }
        __syncwarp();
        const int pe = xrp[i + 1];
        for (int p = xrp[i]; p < pe; ++p) {
            const int k = xci[p];
            const double xk = xv ? xv[p] : 1.0;
            const int qe = yrp[k + 1];
            for (int q = yrp[k] + lane; q < qe; q += 32) {
                const int J = yci[q];
                const int pos = lower_bound_col(cols, cn, J);
                if (pos >= cn || cols[pos] != J) {
                    atomicExch(bad, 1);
                    continue;
                }
                vals[pos] = __dadd_rn(vals[pos], __dmul_rn(xk, yv ? yv[q] : 1.0));
            }
            __syncwarp();
        }
        for (int a = lane; a < cn; a += 32) cv[c0 + a] = prolong_epilogue<EPI>(vals[a], cols[a], i, epi);
        __syncwarp();
    }
}

// C.v = X Y on C's known pattern (C.rp, C.ci, C.nnz as set up before);
// *bad is set if a product falls outside it.  ypairs: the mean number of
// entries of Y's rows, which with X's picks the kernel shape.
template <int EPI>
static int spgemm_known(int nrows, const int *xrp, const int *xci, const double *xv, long long xnnz, const int *yrp,
                        const int *yci, const double *yv, double ymean, ProlongEpi epi, const DevCSR &C, int *bad,
                        cudaStream_t s) {
    if (nrows == 0) return AMG_OK;
    const double pairs = (double)xnnz / nrows * ymean;
    if (pairs <= 96.0) {
        const int blocks = (int)std::min<long long>((nrows + 255) / 256, (long long)num_sms() * 16);
        k_spgemm_known_thread<EPI><<<std::max(blocks, 1), 256, 0, s>>>(nrows, xrp, xci, xv, yrp, yci, yv, C.rp, C.ci,
                                                                         C.v, epi, bad);
    } else {
        const int blocks = (int)std::min<long long>((nrows + KWARPS - 1) / KWARPS, (long long)num_sms() * 8);
        k_spgemm_known_warp<EPI><<<std::max(blocks, 1), KWARPS * 32, 0, s>>>(nrows, xrp, xci, xv, yrp, yci, yv, C.rp,
                                                                               C.ci, C.v, epi, bad);
    }
    AMG_LAUNCH_CHECK();
    return AMG_OK;
}

// dst[k] = src[perm[k]]
__global__ void k_gather_values(long long n, const int *__restrict__ perm, const double *__restrict__ src, double *dst) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        dst[k] = src[perm[k]];
}

// ===========================================================================
// Dense coarsest level: factor (Cholesky if symmetric, else LU with partial
// pivoting) and explicit inverse, one thread block, FP64.
// ===========================================================================

__global__ void k_csr_to_dense(int n, const int *rp, const int *ci, const double *v, double *d) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * n; i += gridDim.x * blockDim.x) d[i] = 0.0;
    __syncthreads();
    // one block
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int k = rp[i]; k < rp[i + 1]; ++k) d[(size_t)i * n + ci[k]] = v[k];
}

// One thread block factors an n x n dense matrix in place and writes its inverse.
__device__ void dense_factor_inverse_block(int n, int symmetric, double *a, int *piv, double *inv, int *status) {
    __shared__ int s_piv;
    __shared__ int s_fail;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) s_fail = 0;
    __syncthreads();
    if (symmetric) {
        for (int j = 0; j < n; ++j) {
            if (tid == 0) {
                double d = a[(size_t)j * n + j];
                for (int k = 0; k < j; ++k) d -= a[(size_t)j * n + k] * a[(size_t)j * n + k];
                if (!(d > 0.0)) s_fail = 1;
                else a[(size_t)j * n + j] = sqrt(d);
            }
            __syncthreads();
            if (s_fail) break;
            const double ljj = a[(size_t)j * n + j];
            for (int i = j + 1 + tid; i < n; i += nt) {
                double s = a[(size_t)i * n + j];
                for (int k = 0; k < j; ++k) s -= a[(size_t)i * n + k] * a[(size_t)j * n + k];
                a[(size_t)i * n + j] = s / ljj;
            }
            __syncthreads();
        }
    } else {
        for (int k = 0; k < n; ++k) {
            if (tid == 0) {
                int p = k;
                double best = fabs(a[(size_t)k * n + k]);
                for (int i = k + 1; i < n; ++i) {
                    const double c = fabs(a[(size_t)i * n + k]);
                    if (c > best) { best = c; p = i; }
                }
                s_piv = p;
                piv[k] = p;
                if (best == 0.0) s_fail = 1;
            }
            __syncthreads();
            if (s_fail) break;
            const int p = s_piv;
            if (p != k)
                for (int j = tid; j < n; j += nt) {
                    const double t = a[(size_t)k * n + j];
                    a[(size_t)k * n + j] = a[(size_t)p * n + j];
                    a[(size_t)p * n + j] = t;
                }
            __syncthreads();
            for (int i = k + 1 + tid; i < n; i += nt) a[(size_t)i * n + k] /= a[(size_t)k * n + k];
            __syncthreads();
            for (int idx = tid; idx < (n - k - 1) * (n - k - 1); idx += nt) {
                const int i = k + 1 + idx / (n - k - 1), j = k + 1 + idx % (n - k - 1);
                a[(size_t)i * n + j] -= a[(size_t)i * n + k] * a[(size_t)k * n + j];
            }
            __syncthreads();
        }
    }
    if (s_fail) {
        if (tid == 0) *status = AMG_NOT_SPD;
        return;
    }
    // inverse: column c of inv solves A x = e_c (one thread per column)
    for (int c = tid; c < n; c += nt) {
        double *x = inv + (size_t)c;  // column c, stride n
        for (int i = 0; i < n; ++i) x[(size_t)i * n] = (i == c) ? 1.0 : 0.0;
        if (symmetric) {
            for (int i = 0; i < n; ++i) {
                double s = x[(size_t)i * n];
                for (int k = 0; k < i; ++k) s -= a[(size_t)i * n + k] * x[(size_t)k * n];
                x[(size_t)i * n] = s / a[(size_t)i * n + i];
            }
            for (int i = n - 1; i >= 0; --i) {
                double s = x[(size_t)i * n];
                for (int k = i + 1; k < n; ++k) s -= a[(size_t)k * n + i] * x[(size_t)k * n];
                x[(size_t)i * n] = s / a[(size_t)i * n + i];
            }
        } else {
            for (int k = 0; k < n; ++k) {
                const int p = piv[k];
                if (p != k) {
                    const double t = x[(size_t)k * n];
                    x[(size_t)k * n] = x[(size_t)p * n];
                    x[(size_t)p * n] = t;
                }
            }
            for (int i = 0; i < n; ++i) {
                double s = x[(size_t)i * n];
                for (int k = 0; k < i; ++k) s -= a[(size_t)i * n + k] * x[(size_t)k * n];
                x[(size_t)i * n] = s;
            }
            for (int i = n - 1; i >= 0; --i) {
                double s = x[(size_t)i * n];
                for (int k = i + 1; k < n; ++k) s -= a[(size_t)i * n + k] * x[(size_t)k * n];
                x[(size_t)i * n] = s / a[(size_t)i * n + i];
            }
        }
    }
    if (tid == 0) *status = AMG_OK;
}

__global__ void k_dense_factor_inverse(int n, int symmetric, double *a, int *piv, double *inv, int *status) {
    dense_factor_inverse_block(n, symmetric, a, piv, inv, status);
}

// Batched: block b factors system b's m[b] x m[b] block (dense at off2[b],
// pivots at off1[b], inverse at off2[b] of inv).
__global__ void k_dense_factor_inverse_batch(const int *m, const long long *off2, const int *off1, int symmetric,
                                             double *a, int *piv, double *inv, int *status) {
    const int b = blockIdx.x;
    dense_factor_inverse_block(m[b], symmetric, a + off2[b], piv + off1[b], inv + off2[b], status + b);
}

// Batched dense extraction: block b copies rows [r0, r0 + m) of the CSR into
// an m x m block with columns shifted by r0.
__global__ void k_csr_to_dense_batch(const int *r0s, const int *m, const long long *off2, const int *rp,
                                     const int *ci, const double *v, double *d) {
    const int b = blockIdx.x, r0 = r0s[b], mb = m[b];
    double *db = d + off2[b];
    for (int i = threadIdx.x; i < mb * mb; i += blockDim.x) db[i] = 0.0;
    __syncthreads();
    for (int i = threadIdx.x; i < mb; i += blockDim.x)
        for (int k = rp[r0 + i]; k < rp[r0 + i + 1]; ++k) db[(size_t)i * mb + (ci[k] - r0)] = v[k];
}

// ===========================================================================
// Hierarchy construction
// ===========================================================================

// a_ij w_j for every stored entry (the pre-smoother applies A W to b).
__global__ void k_scale_cols(int n, const int *rp, const int *ci, const double *v, const double *w, double *out,
                             float *out32) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            const double a = v[k] * w[ci[k]];
            out[k] = a;
            if (out32) out32[k] = __double2float_rn(a);
        }
}

// Tiling for the streaming kernels: the largest rt (multiple of 16, <= 1024)
// whose every tile holds at most cap - 8 stored entries, and vec threads per
// row from the mean row length.  Operators below 16384 rows keep the
// row-vector kernels.
static int plan_stream(const DevCSR &m, int cap, StreamPlan &pl, cudaStream_t s) {
    pl = StreamPlan();
    const int n = m.nrows;
    if (n < 16384) return AMG_OK;
    std::vector<int> rp((size_t)n + 1);
    AMG_CUDA_TRY(cudaMemcpyAsync(rp.data(), m.rp, sizeof(int) * ((size_t)n + 1), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    auto worst = [&](int rt) {
        int w = 0;
        for (int r0 = 0; r0 < n; r0 += rt) w = std::max(w, rp[std::min(r0 + rt, n)] - rp[r0]);
        return w;
    };
    const double mean = (double)m.nnz / n;
    int v = 1;
    while (v < 32 && mean > 12.0 * v) v <<= 1;
    // 480 consumer threads take a tile in passes of 480 / v rows: prefer tile
    // heights that are whole passes (and multiples of 16), else any multiple of 16
    const int pass = 480 / v;
    int unit = 16;
    while (unit % pass != 0) unit += 16;
    int best = 0;
    for (int u : {unit, 16}) {
        int lo = 0, hi = 1024 / u;  // search rt = u k
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (worst(u * mid) <= cap - 8) lo = mid;
            else hi = mid - 1;
        }
        if (lo > 0) {
            best = u * lo;
            break;
        }
    }
    if (best == 0) return AMG_OK;
    pl.rt = best;
    pl.cap = cap;
    pl.vec = v;
    pl.ntiles = (n + pl.rt - 1) / pl.rt;
    return AMG_OK;
}

static int choose_vec(long long nnz, int nrows) {
    const double mean = nrows > 0 ? (double)nnz / nrows : 1.0;
    int v = 2;
    while (v < 32 && v < mean) v <<= 1;
    return v;
}

static int collapse_coarse(Hierarchy *h, cudaStream_t s);

// The part of a setup after the levels' operators exist (levels 0 ..
// h->nlevels - 1 with A, and P, R, agg, w on all but the last): the coarsest
// dense factor and inverse, FP32 copies, work vectors, streaming plans, the
// collapsed coarse end and the fused tail.
static int finish_build(Hierarchy *h, bool precond, cudaStream_t s) {
    const amg_config &cfg = h->cfg;
    DevArena &ar = h->arena;

    // ---- coarsest level: dense factor + inverse ----
    const int l = h->nlevels - 1;
    Level &Lc = h->L[l];
    h->nc = precond ? Lc.A.nrows : 0;
    if (h->nc > AMG_DENSE_MAX) {
        set_last_error("coarsening stopped at level %d with %d rows (> %d)", l, h->nc, AMG_DENSE_MAX);
        return AMG_ERR_STALL;
    }
    if (precond) {
        Scratch sc;
        double *dense;
        int *piv, *st;
        const int m = h->nc;
        AMG_TRY(sc.alloc(&dense, (size_t)m * m));
        AMG_TRY(sc.alloc(&piv, (size_t)m));
        AMG_TRY(sc.alloc(&st, 1));
        AMG_TRY(ar.alloc(&h->cinv, (size_t)m * m));
        h->cinv_last = h->cinv;
        k_csr_to_dense<<<1, 256, 0, s>>>(m, Lc.A.rp, Lc.A.ci, Lc.A.v, dense);
        k_dense_factor_inverse<<<1, 256, 0, s>>>(m, h->symmetric, dense, piv, h->cinv, st);
        AMG_LAUNCH_CHECK();
        int hst = -1;
        AMG_CUDA_TRY(cudaMemcpyAsync(&hst, st, sizeof(int), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        if (hst != AMG_OK) {
            set_last_error("coarsest level (%d rows) is not %s", m, h->symmetric ? "SPD" : "invertible");
            return AMG_NOT_SPD;
        }
    }

    // ---- FP32 copies, work vectors, launch shapes ----
    const bool mixed = cfg.precision == AMG_PRECISION_MIXED;
    for (int k = 0; k < h->nlevels; ++k) {
        Level &Lv = h->L[k];
        const int nl = Lv.A.nrows;
        const bool last = k == h->nlevels - 1;
        Lv.vec_a = choose_vec(Lv.A.nnz, nl);
        if (!last) {
            Lv.vec_p = choose_vec(Lv.P.nnz, nl);
            Lv.vec_r = choose_vec(Lv.R.nnz, Lv.R.nrows);
        }
        AMG_TRY(ar.alloc(&Lv.t, (size_t)nl));
        if (k > 0) {
            AMG_TRY(ar.alloc(&Lv.b, (size_t)nl));
            AMG_TRY(ar.alloc(&Lv.x, (size_t)nl));
        }
        const int cap = 4096;  // stage capacity (stream::CAP)
        if (k == 0) AMG_TRY(plan_stream(Lv.A, cap, Lv.sa64, s));
        if (!last) {
            AMG_TRY(plan_stream(Lv.A, cap, Lv.sa, s));
            Lv.sa_post = Lv.sa;
            AMG_TRY(plan_stream(Lv.P, cap, Lv.sp, s));
            AMG_TRY(plan_stream(Lv.R, cap, Lv.sr, s));
            AMG_TRY(ar.alloc(&Lv.ahat, (size_t)std::max(1LL, Lv.A.nnz)));
            if (mixed) AMG_TRY(ar.alloc(&Lv.ahat32, (size_t)std::max(1LL, Lv.A.nnz)));
            k_scale_cols<<<grid_for(nl), 256, 0, s>>>(nl, Lv.A.rp, Lv.A.ci, Lv.A.v, Lv.w, Lv.ahat, Lv.ahat32);
            AMG_LAUNCH_CHECK();
        }
        if (mixed) {
            AMG_TRY(ar.alloc(&Lv.A.v32, (size_t)std::max(1LL, Lv.A.nnz)));
            k_to_f32<<<grid_for(Lv.A.nnz), 256, 0, s>>>(Lv.A.v, Lv.A.v32, Lv.A.nnz);
            AMG_TRY(ar.alloc(&Lv.w32, (size_t)nl));
            k_to_f32<<<grid_for(nl), 256, 0, s>>>(Lv.w, Lv.w32, nl);
            if (!last) {
                AMG_TRY(ar.alloc(&Lv.P.v32, (size_t)std::max(1LL, Lv.P.nnz)));
                k_to_f32<<<grid_for(Lv.P.nnz), 256, 0, s>>>(Lv.P.v, Lv.P.v32, Lv.P.nnz);
                AMG_TRY(ar.alloc(&Lv.R.v32, (size_t)std::max(1LL, Lv.R.nnz)));
                k_to_f32<<<grid_for(Lv.R.nnz), 256, 0, s>>>(Lv.R.v, Lv.R.v32, Lv.R.nnz);
            }
            if (k == 0) {
                AMG_TRY(ar.alloc(&Lv.A.vdf, (size_t)std::max(1LL, Lv.A.nnz)));
                k_to_df<<<grid_for(Lv.A.nnz), 256, 0, s>>>(Lv.A.v, Lv.A.vdf, Lv.A.nnz);
            }
            AMG_LAUNCH_CHECK();
            AMG_TRY(ar.alloc(&Lv.t32, (size_t)nl));
            if (k > 0) {
                AMG_TRY(ar.alloc(&Lv.b32, (size_t)nl));
                AMG_TRY(ar.alloc(&Lv.x32, (size_t)nl));
            }
        }
    }
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (!precond) {
        h->nsolve = 1;
        return AMG_OK;
    }
    AMG_TRY(collapse_coarse(h, s));
    return tail_prepare(h, s);
}

int build_hierarchy(Hierarchy *h, const int *rp_in, const int *ci_in, const double *v_in, cudaStream_t s) {
    const amg_config &cfg = h->cfg;
    const int n = h->n;
    const long long nnz = h->nnz;
    DevArena &ar = h->arena;

    // ---- level 0: copy and validate ----
    Level &L0 = h->L[0];
    L0.A.nrows = L0.A.ncols = n;
    L0.A.nnz = nnz;
    AMG_TRY(ar.alloc(&L0.A.rp, (size_t)n + 1));
    AMG_TRY(ar.alloc(&L0.A.ci, (size_t)nnz));
    AMG_TRY(ar.alloc(&L0.A.v, (size_t)nnz));
    AMG_CUDA_TRY(cudaMemcpyAsync(L0.A.rp, rp_in, sizeof(int) * ((size_t)n + 1), cudaMemcpyDefault, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(L0.A.ci, ci_in, sizeof(int) * (size_t)nnz, cudaMemcpyDefault, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(L0.A.v, v_in, sizeof(double) * (size_t)nnz, cudaMemcpyDefault, s));
    int ends[2] = {0, 0};
    AMG_CUDA_TRY(cudaMemcpyAsync(&ends[0], L0.A.rp, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(&ends[1], L0.A.rp + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (ends[0] != 0 || (long long)ends[1] != nnz) {
        set_last_error("row_ptr[0] = %d, row_ptr[n] = %d, nnz = %lld", ends[0], ends[1], nnz);
        return AMG_ERR_BAD_CSR;
    }
    {
        Scratch sc;
        int *dpos;
        unsigned long long *err;
        AMG_TRY(sc.alloc(&dpos, (size_t)n));
        AMG_TRY(sc.alloc(&err, 1));
        unsigned long long init = ~0ull;
        AMG_CUDA_TRY(cudaMemcpyAsync(err, &init, sizeof(init), cudaMemcpyHostToDevice, s));
        k_validate<<<grid_for(n), 256, 0, s>>>(n, nnz, L0.A.rp, L0.A.ci, L0.A.v, dpos, err);
        AMG_LAUNCH_CHECK();
        unsigned long long first = 0;
        AMG_CUDA_TRY(cudaMemcpyAsync(&first, err, sizeof(first), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        if (first != ~0ull) {
            const int row = (int)(first >> 2), code = (int)(first & 3);
            set_last_error("invalid CSR at row %d (%s)", row, code == 1 ? "bad structure" : "zero or missing diagonal");
            return code == 1 ? AMG_ERR_BAD_CSR : AMG_ERR_ZERO_DIAG;
        }
    }

    // ---- symmetry ----
    if (cfg.symmetric >= 0) {
        h->symmetric = cfg.symmetric;
    } else {
        DevArena tmp;
        DevCSR At;
        int rc = transpose_csr(L0.A, At, tmp, s);
        if (rc < 0) { tmp.free_all(); return rc; }
        int *differ = nullptr;
        rc = tmp.alloc(&differ, 1);
        if (rc < 0) { tmp.free_all(); return rc; }
        cudaMemsetAsync(differ, 0, sizeof(int), s);
        k_compare_csr<<<grid_for(nnz + n + 1), 256, 0, s>>>(n, nnz, L0.A.rp, L0.A.ci, L0.A.v, At.rp, At.ci, At.v,
                                                             differ);
        int d = 1;
        cudaMemcpyAsync(&d, differ, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        tmp.free_all();
        AMG_CUDA_TRY(e);
        h->symmetric = d ? 0 : 1;
    }

    // ---- levels ----
    // Unpreconditioned Krylov solvers keep the finest level only: no coarse
    // levels, coarse solve or cycle are built (nor re-set up).
    const bool precond = cfg.solver == AMG_SOLVER_PCG || cfg.solver == AMG_SOLVER_BICGSTAB;
    int l = 0;
    for (;;) {
        Level &Lv = h->L[l];
        DevCSR &A = Lv.A;
        const int nl = A.nrows;
        Scratch sc;
        double *diag;
        int *bad;
        AMG_TRY(sc.alloc(&diag, (size_t)nl));
        AMG_TRY(sc.alloc(&bad, 1));
        AMG_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
        k_find_diag<<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.ci, A.v, diag, bad);
        AMG_LAUNCH_CHECK();
        int hbad = 0;
        AMG_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        if (hbad) {
            set_last_error("level %d has a zero diagonal", l);
            return AMG_ERR_ZERO_DIAG;
        }
        AMG_TRY(ar.alloc(&Lv.w, (size_t)nl));
        k_smoother_weights<<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.v, diag, cfg.omega,
                                                        cfg.smoother == AMG_SMOOTHER_L1_JACOBI, Lv.w);
        AMG_LAUNCH_CHECK();
        if (!precond || nl <= cfg.coarse_max || l + 1 >= cfg.max_levels || l + 1 >= AMG_MAX_LEVELS) break;

        if (cfg.amg_type == AMG_TYPE_CLASSICAL) {
            // classical: strength, PMIS splitting, direct interpolation; agg
            // holds each row's coarse index (-1 for an F point)
            int *cnt, *srp, *sci;
            AMG_TRY(sc.alloc(&cnt, (size_t)nl + 1));
            AMG_TRY(sc.alloc(&srp, (size_t)nl + 1));
            k_strength_classical<false><<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.ci, A.v, cnt, nullptr, nullptr);
            AMG_LAUNCH_CHECK();
            int snnz = 0;
            AMG_TRY(exclusive_scan_int(cnt, srp, nl, &snnz, s));
            AMG_TRY(sc.alloc(&sci, (size_t)std::max(1, snnz)));
            k_strength_classical<true><<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.ci, A.v, nullptr, srp, sci);
            AMG_LAUNCH_CHECK();
            DevCSR S, St;
            S.nrows = S.ncols = nl;
            S.nnz = snnz;
            S.rp = srp;
            S.ci = sci;
            AMG_TRY(transpose_csr(S, St, sc.arena, s));
            double *w;
            int *st, *newc, *und;
            AMG_TRY(sc.alloc(&w, (size_t)nl));
            AMG_TRY(sc.alloc(&st, (size_t)nl));
            AMG_TRY(sc.alloc(&newc, (size_t)nl));
            AMG_TRY(sc.alloc(&und, 1));
            k_pmis_init<<<grid_for(nl), 256, 0, s>>>(nl, St.rp, w, st);
            AMG_LAUNCH_CHECK();
            int rounds = 0, hund = 1;
            while (hund > 0) {
                if (++rounds > 100000) {
                    set_last_error("PMIS rounds did not terminate at level %d", l);
                    return AMG_ERR_STALL;
                }
                AMG_CUDA_TRY(cudaMemsetAsync(und, 0, sizeof(int), s));
                k_pmis_select<<<grid_for(nl), 256, 0, s>>>(nl, srp, sci, St.rp, St.ci, w, st, newc);
                k_pmis_update<<<grid_for(nl), 256, 0, s>>>(nl, srp, sci, newc, st, und);
                AMG_LAUNCH_CHECK();
                AMG_CUDA_TRY(cudaMemcpyAsync(&hund, und, sizeof(int), cudaMemcpyDeviceToHost, s));
                AMG_CUDA_TRY(cudaStreamSynchronize(s));
            }
            int *flag, *cscan;
            AMG_TRY(sc.alloc(&flag, (size_t)nl + 1));
            AMG_TRY(sc.alloc(&cscan, (size_t)nl + 1));
            k_c_flags<<<grid_for(nl), 256, 0, s>>>(nl, st, flag);
            AMG_LAUNCH_CHECK();
            int ncc = 0;
            AMG_TRY(exclusive_scan_int(flag, cscan, nl, &ncc, s));
            if (ncc == 0 || ncc >= nl) break;  // coarsening stalled: this level is the last
            AMG_TRY(ar.alloc(&Lv.agg, (size_t)nl));
            k_c_index<<<grid_for(nl), 256, 0, s>>>(nl, st, cscan, Lv.agg);
            int *pcnt;
            AMG_TRY(sc.alloc(&pcnt, (size_t)nl + 1));
            k_interp_direct<false><<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.ci, A.v, srp, sci, Lv.agg, pcnt, nullptr,
                                                                 nullptr, nullptr);
            AMG_LAUNCH_CHECK();
            DevCSR &P = Lv.P;
            P.nrows = nl;
            P.ncols = ncc;
            AMG_TRY(ar.alloc(&P.rp, (size_t)nl + 1));
            int pnnz = 0;
            AMG_TRY(exclusive_scan_int(pcnt, P.rp, nl, &pnnz, s));
            P.nnz = pnnz;
            AMG_TRY(ar.alloc(&P.ci, (size_t)std::max(1, pnnz)));
            AMG_TRY(ar.alloc(&P.v, (size_t)std::max(1, pnnz)));
            k_interp_direct<true><<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.ci, A.v, srp, sci, Lv.agg, nullptr, P.rp,
                                                                P.ci, P.v);
            AMG_LAUNCH_CHECK();
            Lv.rho = 0.0;
            AMG_TRY(transpose_csr(P, Lv.R, ar, s));
            DevCSR AP;
            AMG_TRY((spgemm<EPI_NONE>(nl, ncc, A.rp, A.ci, A.v, P.rp, P.ci, P.v, ProlongEpi{}, AP, sc.arena, s)));
            Level &Ln = h->L[l + 1];
            AMG_TRY((spgemm<EPI_NONE>(ncc, ncc, Lv.R.rp, Lv.R.ci, Lv.R.v, AP.rp, AP.ci, AP.v, ProlongEpi{}, Ln.A, ar, s)));
            AMG_CUDA_TRY(cudaStreamSynchronize(s));
            ++l;
            continue;
        }

        // strength
        const double theta_l = ldexp(cfg.theta, -l);
        const double t2 = theta_l * theta_l;
        int *cnt, *s1rp, *s1ci, *srp, *sci;
        AMG_TRY(sc.alloc(&cnt, (size_t)nl + 1));
        AMG_TRY(sc.alloc(&s1rp, (size_t)nl + 1));
        k_strength<false><<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.ci, A.v, diag, t2, cnt, nullptr, nullptr);
        AMG_LAUNCH_CHECK();
        int s1nnz = 0;
        AMG_TRY(exclusive_scan_int(cnt, s1rp, nl, &s1nnz, s));
        AMG_TRY(sc.alloc(&s1ci, (size_t)std::max(1, s1nnz)));
        k_strength<true><<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.ci, A.v, diag, t2, nullptr, s1rp, s1ci);
        AMG_LAUNCH_CHECK();
        DevCSR S1;
        S1.nrows = S1.ncols = nl;
        S1.nnz = s1nnz;
        S1.rp = s1rp;
        S1.ci = s1ci;
        DevCSR S1t;
        AMG_TRY(transpose_csr(S1, S1t, sc.arena, s));
        AMG_TRY(sc.alloc(&srp, (size_t)nl + 1));
        k_union<false><<<grid_for(nl), 256, 0, s>>>(nl, s1rp, s1ci, S1t.rp, S1t.ci, cnt, nullptr, nullptr);
        AMG_LAUNCH_CHECK();
        int snnz = 0;
        AMG_TRY(exclusive_scan_int(cnt, srp, nl, &snnz, s));
        AMG_TRY(sc.alloc(&sci, (size_t)std::max(1, snnz)));
        k_union<true><<<grid_for(nl), 256, 0, s>>>(nl, s1rp, s1ci, S1t.rp, S1t.ci, nullptr, srp, sci);
        AMG_LAUNCH_CHECK();

        // distance-2 MIS
        unsigned long long *t, *m1;
        int *und;
        AMG_TRY(sc.alloc(&t, (size_t)nl));
        AMG_TRY(sc.alloc(&m1, (size_t)nl));
        AMG_TRY(sc.alloc(&und, 1));
        k_mis_init<<<grid_for(nl), 256, 0, s>>>(nl, nullptr, t);
        AMG_LAUNCH_CHECK();
        int rounds = 0, hund = 1;
        while (hund > 0) {
            if (++rounds > 100000) {
                set_last_error("independent-set rounds did not terminate at level %d", l);
                return AMG_ERR_STALL;
            }
            AMG_CUDA_TRY(cudaMemsetAsync(und, 0, sizeof(int), s));
            k_mis_max<<<grid_for(nl), 256, 0, s>>>(nl, srp, sci, t, m1);
            k_mis_update<<<grid_for(nl), 256, 0, s>>>(nl, srp, sci, m1, t, und);
            AMG_LAUNCH_CHECK();
            AMG_CUDA_TRY(cudaMemcpyAsync(&hund, und, sizeof(int), cudaMemcpyDeviceToHost, s));
            AMG_CUDA_TRY(cudaStreamSynchronize(s));
        }

        // aggregates
        int *flag, *root_id, *snap, *rank;
        AMG_TRY(sc.alloc(&flag, (size_t)nl + 1));
        AMG_TRY(sc.alloc(&root_id, (size_t)nl + 1));
        AMG_TRY(sc.alloc(&snap, (size_t)nl));
        AMG_TRY(sc.alloc(&rank, (size_t)nl + 1));
        AMG_TRY(ar.alloc(&Lv.agg, (size_t)nl));
        k_root_flags<<<grid_for(nl), 256, 0, s>>>(nl, t, flag);
        AMG_LAUNCH_CHECK();
        int nroots = 0;
        AMG_TRY(exclusive_scan_int(flag, root_id, nl, &nroots, s));
        k_agg_phase12<<<grid_for(nl), 256, 0, s>>>(nl, srp, sci, t, root_id, snap);
        k_agg_phase3<<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.ci, A.v, srp, sci, snap, Lv.agg, flag);
        AMG_LAUNCH_CHECK();
        int nsingle = 0;
        AMG_TRY(exclusive_scan_int(flag, rank, nl, &nsingle, s));
        if (nsingle > 0) {
            k_agg_singletons<<<grid_for(nl), 256, 0, s>>>(nl, rank, nroots, Lv.agg);
            AMG_LAUNCH_CHECK();
        }
        const int nc = nroots + nsingle;
        if (nc >= nl) {  // coarsening stalled: this level is the last
            ar.release(Lv.agg);
            Lv.agg = nullptr;
            break;
        }

        // prolongator P = (I - omega_P D^-1 A) T
        unsigned long long *rho_bits;
        AMG_TRY(sc.alloc(&rho_bits, 1));
        AMG_CUDA_TRY(cudaMemsetAsync(rho_bits, 0, sizeof(unsigned long long), s));
        k_gershgorin<<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.v, diag, rho_bits);
        AMG_LAUNCH_CHECK();
        unsigned long long hb = 0;
        AMG_CUDA_TRY(cudaMemcpyAsync(&hb, rho_bits, sizeof(hb), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        double rho;
        memcpy(&rho, &hb, sizeof(rho));
        Lv.rho = rho;
        const double c43 = 4.0 / 3.0;
        ProlongEpi epi{Lv.agg, diag, c43 / rho};
        int *trp;
        AMG_TRY(sc.alloc(&trp, (size_t)nl + 1));
        k_iota<<<grid_for(nl + 1), 256, 0, s>>>(trp, nl + 1);
        AMG_LAUNCH_CHECK();
        AMG_TRY((spgemm<EPI_PROLONG>(nl, nc, A.rp, A.ci, A.v, trp, Lv.agg, nullptr, epi, Lv.P, ar, s)));
        AMG_TRY(transpose_csr(Lv.P, Lv.R, ar, s));
        // Galerkin A_c = R (A P)
        DevCSR AP;
        AMG_TRY((spgemm<EPI_NONE>(nl, nc, A.rp, A.ci, A.v, Lv.P.rp, Lv.P.ci, Lv.P.v, ProlongEpi{}, AP, sc.arena, s)));
        Level &Ln = h->L[l + 1];
        AMG_TRY((spgemm<EPI_NONE>(nc, nc, Lv.R.rp, Lv.R.ci, Lv.R.v, AP.rp, AP.ci, AP.v, ProlongEpi{}, Ln.A, ar, s)));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        ++l;
    }
    h->nlevels = l + 1;
    return finish_build(h, precond, s);
}


// ===========================================================================
// Block-diagonal batches of independent systems
// ===========================================================================
// The hierarchy of a batch is, system by system, the hierarchy each system
// would have alone: independent-set priorities use the row's index within its
// system, the Gershgorin estimate and omega_P are per system, and a system
// stops coarsening on its own (<= coarse_max rows, the level cap, or no
// shrink).  A system that stops on level l is "final" there: its rows keep
// zero smoother weights (the smoothing kernels leave zeros), get no
// prolongator rows (it is absent from level l + 1), and a per-system dense
// inverse solves it on level l.

__global__ void k_rows_of_sys(int n, int nsys, const int *off, int *row_sys, int *row_start) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int lo = 0, hi = nsys - 1;
        while (lo < hi) {  // last system with off <= i
            const int mid = (lo + hi + 1) / 2;
            if (off[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        row_sys[i] = lo;
        row_start[i] = off[lo];
    }
}

__global__ void k_active_rows(int n, const int *row_sys, const unsigned char *fin, unsigned char *active, double *w) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const bool a = !fin[row_sys[i]];
        active[i] = a;
        if (!a) w[i] = 0.0;
    }
}

__global__ void k_gershgorin_sys(int n, const int *rp, const double *v, const double *diag, const int *row_sys,
                                 const unsigned char *active, unsigned long long *rho_bits) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!active[i]) continue;
        double s = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) s = __dadd_rn(s, fabs(v[k]));
        const double q = __ddiv_rn(s, fabs(diag[i]));
        atomicMax(rho_bits + row_sys[i], (unsigned long long)__double_as_longlong(q));
    }
}

__global__ void k_omega_rows(int n, const int *row_sys, const unsigned char *active, const double *om_sys,
                             double *om_row) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        om_row[i] = active[i] ? om_sys[row_sys[i]] : 0.0;
}

__global__ void k_assigned(int n, const int *agg, int *flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) flag[i] = agg[i] >= 0;
}

__global__ void k_t_fill(int n, const int *agg, const int *trp, int *tci) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (agg[i] >= 0) tci[trp[i]] = agg[i];
}

// Dense inverses of the systems final on this level (each <= AMG_DENSE_MAX rows).
static int batch_dense(Hierarchy *h, int l, cudaStream_t s) {
    BatchLevel &B = h->bl[l];
    const DevCSR &A = h->L[l].A;
    std::vector<int> r0, m, off1;
    std::vector<long long> off2;
    long long tot2 = 0;
    int tot1 = 0;
    for (size_t k = 0; k < B.sys.size(); ++k) {
        if (!B.fin[k]) continue;
        const int mk = B.off[k + 1] - B.off[k];
        if (mk > AMG_DENSE_MAX) {
            set_last_error("system %d stopped coarsening on level %d with %d rows (> %d)", B.sys[k], l, mk,
                           AMG_DENSE_MAX);
            return AMG_ERR_STALL;
        }
        r0.push_back(B.off[k]);
        m.push_back(mk);
        off1.push_back(tot1);
        off2.push_back(tot2);
        tot1 += mk;
        tot2 += (long long)mk * mk;
        B.max_m = std::max(B.max_m, mk);
    }
    B.nfin = (int)r0.size();
    if (B.nfin == 0) return AMG_OK;
    DevArena &ar = h->arena;
    Scratch sc;
    int *d_r0s, *d_m, *d_off1, *piv, *st;
    long long *d_off2;
    double *dense;
    AMG_TRY(ar.alloc(&B.fin_r0, r0.size()));
    AMG_TRY(ar.alloc(&B.fin_m, m.size()));
    AMG_TRY(ar.alloc(&B.fin_off2, off2.size()));
    AMG_TRY(ar.alloc(&B.binv, (size_t)tot2));
    AMG_TRY(sc.alloc(&d_off1, off1.size()));
    AMG_TRY(sc.alloc(&piv, (size_t)tot1));
    AMG_TRY(sc.alloc(&st, r0.size()));
    AMG_TRY(sc.alloc(&dense, (size_t)tot2));
    d_r0s = B.fin_r0;
    d_m = B.fin_m;
    d_off2 = B.fin_off2;
    AMG_CUDA_TRY(cudaMemcpyAsync(d_r0s, r0.data(), sizeof(int) * r0.size(), cudaMemcpyHostToDevice, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(d_m, m.data(), sizeof(int) * m.size(), cudaMemcpyHostToDevice, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(d_off2, off2.data(), sizeof(long long) * off2.size(), cudaMemcpyHostToDevice, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(d_off1, off1.data(), sizeof(int) * off1.size(), cudaMemcpyHostToDevice, s));
    k_csr_to_dense_batch<<<B.nfin, 256, 0, s>>>(d_r0s, d_m, d_off2, A.rp, A.ci, A.v, dense);
    k_dense_factor_inverse_batch<<<B.nfin, 256, 0, s>>>(d_m, d_off2, d_off1, h->symmetric, dense, piv, B.binv, st);
    AMG_LAUNCH_CHECK();
    std::vector<int> hst(r0.size());
    AMG_CUDA_TRY(cudaMemcpyAsync(hst.data(), st, sizeof(int) * hst.size(), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    for (size_t k = 0; k < hst.size(); ++k)
        if (hst[k] != AMG_OK) {
            set_last_error("the last level of a system of the batch (level %d) is not %s", l,
                           h->symmetric ? "SPD" : "invertible");
            return AMG_NOT_SPD;
        }
    return AMG_OK;
}

// ---------------------------------------------------------------------------
// Collapsing the coarse end of the cycle into one dense operator
// ---------------------------------------------------------------------------
//
// With a fixed hierarchy and a zero initial iterate, the V(1,1) cycle from
// level l down is a fixed linear map x_l = M_l b_l.  From the cycle's steps
// (pre-smoothing x = W b, residual, restriction, the coarser cycle,
// prolongation, post-smoothing):
//   T   = W + P_l M_{l+1} R_l (I - A_l W)     (the iterate after the correction)
//   M_l = W + T - W (A_l T)                   (after post-smoothing)
// with M_{L-1} the coarsest inverse.  Every product below is a plain sum in
// a fixed order (CSR order, then increasing index), separately rounded.

// E = I - A W (dense n x n, zero-filled beforehand)
__global__ void k_dense_i_minus_aw(int n, const int *rp, const int *ci, const double *v, const double *w, double *E) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        E[(size_t)i * n + i] = 1.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            const int j = ci[k];
            E[(size_t)i * n + j] = (i == j ? 1.0 : 0.0) - v[k] * w[j];
        }
    }
}

// C = S B: S sparse (rows), B dense row-major with nb columns
__global__ void k_spmm_dense(int rows, int nb, const int *rp, const int *ci, const double *v, const double *B, double *C) {
    const long long total = (long long)rows * nb;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / nb), j = (int)(e % nb);
        double s = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) s = s + v[k] * B[(size_t)ci[k] * nb + j];
        C[e] = s;
    }
}

// C = M B: M dense m x m, B dense m x nb
__global__ void k_gemm_dense(int m, int nb, const double *M, const double *B, double *C) {
    const long long total = (long long)m * nb;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / nb), j = (int)(e % nb);
        double s = 0.0;
        for (int q = 0; q < m; ++q) s = s + M[(size_t)i * m + q] * B[(size_t)q * nb + j];
        C[e] = s;
    }
}

// T += W (diagonal)
__global__ void k_add_diag(int n, double *T, const double *w) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) T[(size_t)i * n + i] += w[i];
}

// M = W + T - W U
__global__ void k_collapse_combine(int n, const double *T, const double *U, const double *w, double *M) {
    const long long total = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        M[e] = ((i == j ? w[i] : 0.0) + T[e]) - w[i] * U[e];
    }
}

// padded row-major copies of a dense m x m operator: rows of ld entries, zero beyond m
__global__ void k_pad_dense(int m, int ld, const double *in, double *out64, float *out32) {
    const long long total = (long long)m * ld;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / ld), j = (int)(e % ld);
        const double v = j < m ? in[(size_t)i * m + j] : 0.0;
        out64[e] = v;
        if (out32) out32[e] = (float)v;
    }
}

__global__ void k_to_f32_ll(const double *in, float *out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

static int grid_ll(long long n);

// The padded copies of the dense operator the solve applies (h->cinv).
static int pad_dense(Hierarchy *h, cudaStream_t s) {
    const int m = h->nc;
    const int ld = (m + 3) / 4 * 4;
    const long long tot = (long long)m * ld;
    h->nc_ld = ld;
    if (!h->cpad64) AMG_TRY(h->arena.alloc(&h->cpad64, (size_t)tot));
    if (h->cfg.precision == AMG_PRECISION_MIXED && !h->cpad32) AMG_TRY(h->arena.alloc(&h->cpad32, (size_t)tot));
    k_pad_dense<<<grid_ll(tot), 256, 0, s>>>(m, ld, h->cinv, h->cpad64, h->cpad32);
    AMG_LAUNCH_CHECK();
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    return AMG_OK;
}

static int grid_ll(long long n) { return (int)std::max(1LL, std::min((n + 255) / 256, (long long)num_sms() * 32)); }

// Chooses the first level below the finest with at most COLLAPSE_MAX rows and,
// if coarser levels follow it, replaces the rest of the cycle from there by
// its dense operator (h->nsolve, h->nc, h->cinv, h->cinv32).
constexpr int COLLAPSE_MAX = 2048;

static int collapse_coarse(Hierarchy *h, cudaStream_t s) {
    const int L = h->nlevels;
    // a re-setup keeps the collapsed level and writes into the existing buffers
    const bool again = h->nsolve > 0 && h->nsolve < L;
    int tc = 1;
    if (again) tc = h->nsolve - 1;
    else
        while (tc < L && h->L[tc].A.nrows > COLLAPSE_MAX) ++tc;
    h->nsolve = L;
    if (tc >= L - 1) return pad_dense(h, s);
    DevArena &ar = h->arena;
    Scratch sc;
    const int nmax = h->L[tc].A.nrows;
    const size_t sq = (size_t)nmax * nmax;
    double *E, *Y, *Z, *T, *U, *Mnext = h->cinv_last, *Mcur = nullptr;
    AMG_TRY(sc.alloc(&E, sq));
    AMG_TRY(sc.alloc(&Y, sq));
    AMG_TRY(sc.alloc(&Z, sq));
    AMG_TRY(sc.alloc(&T, sq));
    AMG_TRY(sc.alloc(&U, sq));
    for (int l = L - 2; l >= tc; --l) {
        const Level &lv = h->L[l];
        const int n = lv.A.nrows, m = lv.R.nrows;
        const long long nn = (long long)n * n, mn = (long long)m * n;
        if (l == tc) {
            if (again) Mcur = h->cinv;
            else AMG_TRY(ar.alloc(&Mcur, (size_t)nn));
        } else {
            AMG_TRY(sc.alloc(&Mcur, (size_t)nn));
        }
        AMG_CUDA_TRY(cudaMemsetAsync(E, 0, sizeof(double) * nn, s));
        k_dense_i_minus_aw<<<grid_for(n), 256, 0, s>>>(n, lv.A.rp, lv.A.ci, lv.A.v, lv.w, E);
        k_spmm_dense<<<grid_ll(mn), 256, 0, s>>>(m, n, lv.R.rp, lv.R.ci, lv.R.v, E, Y);   // Y = R (I - A W)
        k_gemm_dense<<<grid_ll(mn), 256, 0, s>>>(m, n, Mnext, Y, Z);                      // Z = M_{l+1} Y
        k_spmm_dense<<<grid_ll(nn), 256, 0, s>>>(n, n, lv.P.rp, lv.P.ci, lv.P.v, Z, T);   // T = P Z
        k_add_diag<<<grid_for(n), 256, 0, s>>>(n, T, lv.w);                                // T += W
        k_spmm_dense<<<grid_ll(nn), 256, 0, s>>>(n, n, lv.A.rp, lv.A.ci, lv.A.v, T, U);   // U = A T
        k_collapse_combine<<<grid_ll(nn), 256, 0, s>>>(n, T, U, lv.w, Mcur);
        AMG_LAUNCH_CHECK();
        Mnext = Mcur;
    }
    h->nsolve = tc + 1;
    h->nc = nmax;
    h->cinv = Mcur;
    if (h->cfg.precision == AMG_PRECISION_MIXED) {
        if (!h->cinv32) AMG_TRY(ar.alloc(&h->cinv32, sq));
        k_to_f32_ll<<<grid_ll((long long)sq), 256, 0, s>>>(Mcur, h->cinv32, (long long)sq);
        AMG_LAUNCH_CHECK();
    }
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    return pad_dense(h, s);
}

// Numeric re-setup (Sec. 2.1: on a cache hit the setup is repeated against
// the new coefficients while the structure of the first setup is reused).
// Every level keeps its aggregates, so P, R and every coarse operator keep
// their patterns; the smoother weights, omega_P, P, R (= P^T), the Galerkin
// products, the coarsest inverse, the collapsed operator and all FP32 copies
// are recomputed from the new values by the same kernels as the setup, and
// written into the existing arrays -- every pointer the streaming plans,
// windows, tail tables and captured graphs hold stays valid.
// The index of every stored entry, as a value (exact in FP64 below 2^53).
__global__ void k_entry_index(long long nnz, double *v) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x)
        v[k] = (double)k;
}

// Entry positions carried through a transpose as values, back to ints.
__global__ void k_to_int(long long n, const double *v, int *out) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        out[k] = (int)v[k];
}

// Pattern of the transpose equal to the pattern: record the mirror map.
__global__ void k_mirror_map(int n, long long nnz, const int *rp1, const int *ci1, const int *rp2, const int *ci2,
                             const double *idx2, int *tmap, int *differ) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz + n + 1;
         k += (long long)gridDim.x * blockDim.x) {
        if (k < nnz) {
            if (ci1[k] != ci2[k]) atomicExch(differ, 1);
            tmap[k] = (int)idx2[k];
        } else if (rp1[k - nnz] != rp2[k - nnz]) {
            atomicExch(differ, 1);
        }
    }
}

// Values symmetric (bitwise) through the mirror map.
__global__ void k_compare_mirror(long long nnz, const double *v, const int *tmap, int *differ) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x)
        if (__double_as_longlong(v[k]) != __double_as_longlong(__ldg(v + tmap[k]))) atomicExch(differ, 1);
}

// Whether the finest level's current values are symmetric (bitwise), by the
// mirror map of its fixed pattern (built on first use).
static int values_symmetric(Hierarchy *h, cudaStream_t s, bool *sym) {
    Level &L0 = h->L[0];
    const int n = L0.A.nrows;
    const long long nnz = L0.A.nnz;
    if (h->tmap_state == 0) {
        DevArena tmp;
        DevCSR I = L0.A, It;
        int *differ = nullptr;
        int rc = tmp.alloc(&I.v, (size_t)std::max(1LL, nnz));
        if (rc == AMG_OK) rc = tmp.alloc(&differ, 1);
        if (rc == AMG_OK) {
            k_entry_index<<<grid_for(nnz), 256, 0, s>>>(nnz, I.v);
            rc = transpose_csr(I, It, tmp, s);
        }
        if (rc == AMG_OK) rc = h->arena.alloc(&h->tmap, (size_t)std::max(1LL, nnz));
        if (rc < 0) {
            tmp.free_all();
            return rc;
        }
        cudaMemsetAsync(differ, 0, sizeof(int), s);
        k_mirror_map<<<grid_for(nnz + n + 1), 256, 0, s>>>(n, nnz, L0.A.rp, L0.A.ci, It.rp, It.ci, It.v, h->tmap, differ);
        int d = 1;
        cudaMemcpyAsync(&d, differ, sizeof(int), cudaMemcpyDeviceToHost, s);
        const cudaError_t e = cudaStreamSynchronize(s);
        tmp.free_all();
        AMG_CUDA_TRY(e);
        h->tmap_state = d ? -1 : 1;
        if (d) {
            h->arena.release(h->tmap);
            h->tmap = nullptr;
        }
    }
    if (h->tmap_state < 0) {
        *sym = false;
        return AMG_OK;
    }
    Scratch sc;
    int *differ = nullptr;
    AMG_TRY(sc.alloc(&differ, 1));
    AMG_CUDA_TRY(cudaMemsetAsync(differ, 0, sizeof(int), s));
    k_compare_mirror<<<grid_for(nnz), 256, 0, s>>>(nnz, L0.A.v, h->tmap, differ);
    AMG_LAUNCH_CHECK();
    int d = 1;
    AMG_CUDA_TRY(cudaMemcpyAsync(&d, differ, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    *sym = d == 0;
    return AMG_OK;
}

// The part of a re-setup after every level operator, P, R and weight holds
// its new values: the coarsest inverse, A W and the FP32 copies, the
// collapsed coarse end (or the padded dense copies) and the sliced-ELL plans'
// value copies.
static int refresh_derived(Hierarchy *h, cudaStream_t s) {
    const amg_config &cfg = h->cfg;
    const int L = h->nlevels;
    // coarsest inverse (none for unpreconditioned handles)
    if (h->nc > 0) {
        Level &Lc = h->L[L - 1];
        Scratch sc;
        double *dense;
        int *piv, *st;
        const int m = Lc.A.nrows;
        AMG_TRY(sc.alloc(&dense, (size_t)m * m));
        AMG_TRY(sc.alloc(&piv, (size_t)m));
        AMG_TRY(sc.alloc(&st, 1));
        k_csr_to_dense<<<1, 256, 0, s>>>(m, Lc.A.rp, Lc.A.ci, Lc.A.v, dense);
        k_dense_factor_inverse<<<1, 256, 0, s>>>(m, h->symmetric, dense, piv, h->cinv_last, st);
        AMG_LAUNCH_CHECK();
        int hst = -1;
        AMG_CUDA_TRY(cudaMemcpyAsync(&hst, st, sizeof(int), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        if (hst != AMG_OK) {
            set_last_error("coarsest level (%d rows) is not %s", m, h->symmetric ? "SPD" : "invertible");
            return AMG_NOT_SPD;
        }
    }
    // A W and the FP32 copies
    const bool mixed = cfg.precision == AMG_PRECISION_MIXED;
    for (int k = 0; k < L; ++k) {
        Level &Lv = h->L[k];
        const int nl = Lv.A.nrows;
        const bool last = k == L - 1;
        if (Lv.ahat) k_scale_cols<<<grid_for(nl), 256, 0, s>>>(nl, Lv.A.rp, Lv.A.ci, Lv.A.v, Lv.w, Lv.ahat, Lv.ahat32);
        if (mixed) {
            k_to_f32<<<grid_for(Lv.A.nnz), 256, 0, s>>>(Lv.A.v, Lv.A.v32, Lv.A.nnz);
            if (Lv.A.vdf) k_to_df<<<grid_for(Lv.A.nnz), 256, 0, s>>>(Lv.A.v, Lv.A.vdf, Lv.A.nnz);
            k_to_f32<<<grid_for(nl), 256, 0, s>>>(Lv.w, Lv.w32, nl);
            if (!last) {
                k_to_f32<<<grid_for(Lv.P.nnz), 256, 0, s>>>(Lv.P.v, Lv.P.v32, Lv.P.nnz);
                k_to_f32<<<grid_for(Lv.R.nnz), 256, 0, s>>>(Lv.R.v, Lv.R.v32, Lv.R.nnz);
            }
        }
        AMG_LAUNCH_CHECK();
    }
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    // the collapsed coarse end (in place) and the padded dense copies
    if (h->nc > 0) AMG_TRY(h->nsolve < h->nlevels ? collapse_coarse(h, s) : pad_dense(h, s));
    // the sliced-ELL plans' slot-order copies of the new values
    return ell_refresh(h, s);
}

int resetup_hierarchy(Hierarchy *h, const double *v_in, cudaStream_t s) {
    const amg_config &cfg = h->cfg;
    const int L = h->nlevels;
    Level &L0 = h->L[0];
    AMG_CUDA_TRY(cudaMemcpyAsync(L0.A.v, v_in, sizeof(double) * (size_t)L0.A.nnz, cudaMemcpyDefault, s));
    if (cfg.symmetric < 0) {
        // the detected symmetry fixes the coarsest factor and the adjoint's hierarchy
        bool sym = false;
        AMG_TRY(values_symmetric(h, s, &sym));
        if ((sym ? 1 : 0) != h->symmetric) {
            set_last_error("the new values change the matrix's symmetry: set up a new handle");
            return AMG_ERR_ARG;
        }
    }
    for (int l = 0; l < L; ++l) {
        Level &Lv = h->L[l];
        DevCSR &A = Lv.A;
        const int nl = A.nrows;
        Scratch sc;
        double *diag;
        int *bad;
        AMG_TRY(sc.alloc(&diag, (size_t)nl));
        AMG_TRY(sc.alloc(&bad, 1));
        AMG_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
        k_find_diag<<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.ci, A.v, diag, bad);
        AMG_LAUNCH_CHECK();
        int hbad = 0;
        AMG_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        if (hbad) {
            set_last_error("level %d has a zero diagonal", l);
            return AMG_ERR_ZERO_DIAG;
        }
        k_smoother_weights<<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.v, diag, cfg.omega,
                                                        cfg.smoother == AMG_SMOOTHER_L1_JACOBI, Lv.w);
        AMG_LAUNCH_CHECK();
        if (l == L - 1) break;
        const int nc = Lv.R.nrows;
        unsigned long long *rho_bits;
        AMG_TRY(sc.alloc(&rho_bits, 1));
        AMG_CUDA_TRY(cudaMemsetAsync(rho_bits, 0, sizeof(unsigned long long), s));
        k_gershgorin<<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.v, diag, rho_bits);
        AMG_LAUNCH_CHECK();
        unsigned long long hb = 0;
        AMG_CUDA_TRY(cudaMemcpyAsync(&hb, rho_bits, sizeof(hb), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        double rho;
        memcpy(&rho, &hb, sizeof(rho));
        Lv.rho = rho;
        const double c43 = 4.0 / 3.0;
        ProlongEpi epi{Lv.agg, diag, c43 / rho};
        int *trp;
        AMG_TRY(sc.alloc(&trp, (size_t)nl + 1));
        k_iota<<<grid_for(nl + 1), 256, 0, s>>>(trp, nl + 1);
        AMG_LAUNCH_CHECK();
        // the patterns are those of the setup: every product is numeric only,
        // written in place (A P's pattern and R's permutation kept from the
        // first re-setup)
        AMG_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
        if (cfg.amg_type == AMG_TYPE_CLASSICAL) {
            k_interp_direct_values<<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.ci, A.v, Lv.agg, Lv.P.rp, Lv.P.ci, Lv.P.v);
            AMG_LAUNCH_CHECK();
        } else {
            AMG_TRY((spgemm_known<EPI_PROLONG>(nl, A.rp, A.ci, A.v, A.nnz, trp, Lv.agg, nullptr, 1.0, epi, Lv.P, bad, s)));
        }
        if (!Lv.rperm) {
            DevCSR I = Lv.P, It;
            AMG_TRY(sc.alloc(&I.v, (size_t)std::max(1LL, Lv.P.nnz)));
            k_entry_index<<<grid_for(Lv.P.nnz), 256, 0, s>>>(Lv.P.nnz, I.v);
            AMG_TRY(transpose_csr(I, It, sc.arena, s));
            AMG_TRY(h->arena.alloc(&Lv.rperm, (size_t)std::max(1LL, Lv.R.nnz)));
            k_to_int<<<grid_for(Lv.R.nnz), 256, 0, s>>>(Lv.R.nnz, It.v, Lv.rperm);
            AMG_LAUNCH_CHECK();
        }
        k_gather_values<<<grid_for(Lv.R.nnz), 256, 0, s>>>(Lv.R.nnz, Lv.rperm, Lv.P.v, Lv.R.v);
        AMG_LAUNCH_CHECK();
        if (!Lv.AP.rp) {
            AMG_TRY((spgemm<EPI_NONE>(nl, nc, A.rp, A.ci, A.v, Lv.P.rp, Lv.P.ci, Lv.P.v, ProlongEpi{}, Lv.AP, h->arena, s)));
        } else {
            AMG_TRY((spgemm_known<EPI_NONE>(nl, A.rp, A.ci, A.v, A.nnz, Lv.P.rp, Lv.P.ci, Lv.P.v,
                                             (double)Lv.P.nnz / std::max(1, Lv.P.nrows), ProlongEpi{}, Lv.AP, bad, s)));
        }
        AMG_TRY((spgemm_known<EPI_NONE>(nc, Lv.R.rp, Lv.R.ci, Lv.R.v, Lv.R.nnz, Lv.AP.rp, Lv.AP.ci, Lv.AP.v,
                                         (double)Lv.AP.nnz / std::max(1, Lv.AP.nrows), ProlongEpi{}, h->L[l + 1].A,
                                         bad, s)));
        hbad = 0;
        AMG_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        if (hbad) {
            set_last_error("re-setup: a product left the setup's pattern on level %d", l);
            return AMG_ERR_CUDA;
        }
    }
    return refresh_derived(h, s);
}

int build_hierarchy_batched(Hierarchy *h, const int *rp_in, const int *ci_in, const double *v_in,
                            const int *sys_off_host, int nsys, cudaStream_t s) {
    const amg_config &cfg = h->cfg;
    const int n = h->n;
    const long long nnz = h->nnz;
    DevArena &ar = h->arena;
    h->nsys = nsys;
    if (sys_off_host[0] != 0 || sys_off_host[nsys] != n) {
        set_last_error("system offsets must start at 0 and end at n");
        return AMG_ERR_ARG;
    }
    for (int k = 0; k < nsys; ++k)
        if (sys_off_host[k + 1] <= sys_off_host[k]) {
            set_last_error("system %d is empty", k);
            return AMG_ERR_ARG;
        }
    // level 0: copy and validate, then check the matrix is block diagonal
    Level &L0 = h->L[0];
    L0.A.nrows = L0.A.ncols = n;
    L0.A.nnz = nnz;
    AMG_TRY(ar.alloc(&L0.A.rp, (size_t)n + 1));
    AMG_TRY(ar.alloc(&L0.A.ci, (size_t)nnz));
    AMG_TRY(ar.alloc(&L0.A.v, (size_t)nnz));
    AMG_CUDA_TRY(cudaMemcpyAsync(L0.A.rp, rp_in, sizeof(int) * ((size_t)n + 1), cudaMemcpyDefault, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(L0.A.ci, ci_in, sizeof(int) * (size_t)nnz, cudaMemcpyDefault, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(L0.A.v, v_in, sizeof(double) * (size_t)nnz, cudaMemcpyDefault, s));
    {
        std::vector<int> hrp((size_t)n + 1), hci((size_t)nnz);
        AMG_CUDA_TRY(cudaMemcpyAsync(hrp.data(), L0.A.rp, sizeof(int) * hrp.size(), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaMemcpyAsync(hci.data(), L0.A.ci, sizeof(int) * hci.size(), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        if (hrp[0] != 0 || (long long)hrp[n] != nnz) {
            set_last_error("row_ptr[0] = %d, row_ptr[n] = %d, nnz = %lld", hrp[0], hrp[n], nnz);
            return AMG_ERR_BAD_CSR;
        }
        for (int k = 0; k < nsys; ++k)
            for (int i = sys_off_host[k]; i < sys_off_host[k + 1]; ++i) {
                if (hrp[i + 1] < hrp[i] || hrp[i] < 0 || (long long)hrp[i + 1] > nnz) {
                    set_last_error("invalid CSR at row %d", i);
                    return AMG_ERR_BAD_CSR;
                }
                for (int q = hrp[i]; q < hrp[i + 1]; ++q)
                    if (hci[q] < sys_off_host[k] || hci[q] >= sys_off_host[k + 1]) {
                        set_last_error("row %d of system %d couples to column %d outside its block", i, k, hci[q]);
                        return AMG_ERR_BAD_CSR;
                    }
            }
    }
    {
        Scratch sc;
        int *dpos;
        unsigned long long *err;
        AMG_TRY(sc.alloc(&dpos, (size_t)n));
        AMG_TRY(sc.alloc(&err, 1));
        unsigned long long init = ~0ull;
        AMG_CUDA_TRY(cudaMemcpyAsync(err, &init, sizeof(init), cudaMemcpyHostToDevice, s));
        k_validate<<<grid_for(n), 256, 0, s>>>(n, nnz, L0.A.rp, L0.A.ci, L0.A.v, dpos, err);
        AMG_LAUNCH_CHECK();
        unsigned long long first = 0;
        AMG_CUDA_TRY(cudaMemcpyAsync(&first, err, sizeof(first), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        if (first != ~0ull) {
            const int code = (int)(first & 3);
            set_last_error("invalid CSR at row %d", (int)(first >> 2));
            return code == 1 ? AMG_ERR_BAD_CSR : AMG_ERR_ZERO_DIAG;
        }
    }
    if (cfg.symmetric >= 0) {
        h->symmetric = cfg.symmetric;
    } else {
        DevArena tmp;
        DevCSR At;
        int rc = transpose_csr(L0.A, At, tmp, s);
        int *differ = nullptr;
        if (rc == AMG_OK) rc = tmp.alloc(&differ, 1);
        if (rc < 0) { tmp.free_all(); return rc; }
        cudaMemsetAsync(differ, 0, sizeof(int), s);
        k_compare_csr<<<grid_for(nnz + n + 1), 256, 0, s>>>(n, nnz, L0.A.rp, L0.A.ci, L0.A.v, At.rp, At.ci, At.v,
                                                             differ);
        int d = 1;
        cudaMemcpyAsync(&d, differ, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        tmp.free_all();
        AMG_CUDA_TRY(e);
        h->symmetric = d ? 0 : 1;
    }

    h->bl.assign(AMG_MAX_LEVELS, BatchLevel());
    h->bl[0].sys.resize(nsys);
    h->bl[0].off.assign(sys_off_host, sys_off_host + nsys + 1);
    for (int k = 0; k < nsys; ++k) h->bl[0].sys[k] = k;
    int l = 0;
    for (;;) {
        Level &Lv = h->L[l];
        BatchLevel &B = h->bl[l];
        DevCSR &A = Lv.A;
        const int nl = A.nrows;
        const int ns = (int)B.sys.size();
        Scratch sc;
        double *diag;
        int *bad, *d_off, *row_sys, *row_start;
        unsigned char *d_fin, *active;
        AMG_TRY(sc.alloc(&diag, (size_t)nl));
        AMG_TRY(sc.alloc(&bad, 1));
        AMG_TRY(sc.alloc(&d_off, (size_t)ns + 1));
        AMG_TRY(sc.alloc(&row_sys, (size_t)nl));
        AMG_TRY(sc.alloc(&row_start, (size_t)nl));
        AMG_TRY(sc.alloc(&d_fin, (size_t)ns));
        AMG_TRY(sc.alloc(&active, (size_t)nl));
        AMG_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
        AMG_CUDA_TRY(cudaMemcpyAsync(d_off, B.off.data(), sizeof(int) * (ns + 1), cudaMemcpyHostToDevice, s));
        k_rows_of_sys<<<grid_for(nl), 256, 0, s>>>(nl, ns, d_off, row_sys, row_start);
        k_find_diag<<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.ci, A.v, diag, bad);
        AMG_LAUNCH_CHECK();
        int hbad = 0;
        AMG_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        if (hbad) {
            set_last_error("level %d has a zero diagonal", l);
            return AMG_ERR_ZERO_DIAG;
        }
        AMG_TRY(ar.alloc(&Lv.w, (size_t)nl));
        B.fin.assign(ns, 0);
        for (int k = 0; k < ns; ++k) {
            const int m = B.off[k + 1] - B.off[k];
            B.fin[k] = !(m > cfg.coarse_max && l + 1 < cfg.max_levels && l + 1 < AMG_MAX_LEVELS);
        }
        const double theta_l = ldexp(cfg.theta, -l);
        const double t2 = theta_l * theta_l;
        std::vector<int> nc_sys(ns, 0);
        int nc = 0;
        for (int attempt = 0;; ++attempt) {
            k_smoother_weights<<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.v, diag, cfg.omega,
                                                            cfg.smoother == AMG_SMOOTHER_L1_JACOBI, Lv.w);
            AMG_CUDA_TRY(cudaMemcpyAsync(d_fin, B.fin.data(), ns, cudaMemcpyHostToDevice, s));
            k_active_rows<<<grid_for(nl), 256, 0, s>>>(nl, row_sys, d_fin, active, Lv.w);
            AMG_LAUNCH_CHECK();
            bool any_active = false;
            for (int k = 0; k < ns; ++k) any_active |= !B.fin[k];
            if (!any_active) break;
            Scratch sa;
            int *cnt, *s1rp, *s1ci, *srp, *sci;
            AMG_TRY(sa.alloc(&cnt, (size_t)nl + 1));
            AMG_TRY(sa.alloc(&s1rp, (size_t)nl + 1));
            k_strength<false><<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.ci, A.v, diag, t2, cnt, nullptr, nullptr);
            AMG_LAUNCH_CHECK();
            int s1nnz = 0;
            AMG_TRY(exclusive_scan_int(cnt, s1rp, nl, &s1nnz, s));
            AMG_TRY(sa.alloc(&s1ci, (size_t)std::max(1, s1nnz)));
            k_strength<true><<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.ci, A.v, diag, t2, nullptr, s1rp, s1ci);
            AMG_LAUNCH_CHECK();
            DevCSR S1;
            S1.nrows = S1.ncols = nl;
            S1.nnz = s1nnz;
            S1.rp = s1rp;
            S1.ci = s1ci;
            DevCSR S1t;
            AMG_TRY(transpose_csr(S1, S1t, sa.arena, s));
            AMG_TRY(sa.alloc(&srp, (size_t)nl + 1));
            k_union<false><<<grid_for(nl), 256, 0, s>>>(nl, s1rp, s1ci, S1t.rp, S1t.ci, cnt, nullptr, nullptr);
            AMG_LAUNCH_CHECK();
            int snnz = 0;
            AMG_TRY(exclusive_scan_int(cnt, srp, nl, &snnz, s));
            AMG_TRY(sa.alloc(&sci, (size_t)std::max(1, snnz)));
            k_union<true><<<grid_for(nl), 256, 0, s>>>(nl, s1rp, s1ci, S1t.rp, S1t.ci, nullptr, srp, sci);
            AMG_LAUNCH_CHECK();
            unsigned long long *t, *m1;
            int *und;
            AMG_TRY(sa.alloc(&t, (size_t)nl));
            AMG_TRY(sa.alloc(&m1, (size_t)nl));
            AMG_TRY(sa.alloc(&und, 1));
            k_mis_init<<<grid_for(nl), 256, 0, s>>>(nl, row_start, t);
            AMG_LAUNCH_CHECK();
            int rounds = 0, hund = 1;
            while (hund > 0) {
                if (++rounds > 100000) {
                    set_last_error("independent-set rounds did not terminate at level %d", l);
                    return AMG_ERR_STALL;
                }
                AMG_CUDA_TRY(cudaMemsetAsync(und, 0, sizeof(int), s));
                k_mis_max<<<grid_for(nl), 256, 0, s>>>(nl, srp, sci, t, m1);
                k_mis_update<<<grid_for(nl), 256, 0, s>>>(nl, srp, sci, m1, t, und);
                AMG_LAUNCH_CHECK();
                AMG_CUDA_TRY(cudaMemcpyAsync(&hund, und, sizeof(int), cudaMemcpyDeviceToHost, s));
                AMG_CUDA_TRY(cudaStreamSynchronize(s));
            }
            int *flag, *root_id, *snap;
            AMG_TRY(sa.alloc(&flag, (size_t)nl + 1));
            AMG_TRY(sa.alloc(&root_id, (size_t)nl + 1));
            AMG_TRY(sa.alloc(&snap, (size_t)nl));
            if (!Lv.agg) AMG_TRY(ar.alloc(&Lv.agg, (size_t)nl));
            k_root_flags<<<grid_for(nl), 256, 0, s>>>(nl, t, flag, active);
            AMG_LAUNCH_CHECK();
            int nroots = 0;
            AMG_TRY(exclusive_scan_int(flag, root_id, nl, &nroots, s));
            k_agg_phase12<<<grid_for(nl), 256, 0, s>>>(nl, srp, sci, t, root_id, snap, active);
            k_agg_phase3<<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.ci, A.v, srp, sci, snap, Lv.agg, flag, active);
            AMG_LAUNCH_CHECK();
            int nsingle = 0;
            AMG_TRY(exclusive_scan_int(flag, snap, nl, &nsingle, s));  // snap reused as scratch
            if (nsingle > 0) {
                set_last_error("aggregation left %d nodes unassigned at level %d", nsingle, l);
                return AMG_ERR_UNSUPPORTED;
            }
            // aggregates per system: the roots inside each system's row range
            std::vector<int> hroot((size_t)nl + 1);
            AMG_CUDA_TRY(cudaMemcpyAsync(hroot.data(), root_id, sizeof(int) * ((size_t)nl + 1), cudaMemcpyDeviceToHost, s));
            AMG_CUDA_TRY(cudaStreamSynchronize(s));
            bool stalled = false;
            for (int k = 0; k < ns; ++k) {
                nc_sys[k] = B.fin[k] ? 0 : hroot[B.off[k + 1]] - hroot[B.off[k]];
                const int m = B.off[k + 1] - B.off[k];
                if (!B.fin[k] && nc_sys[k] >= m) {
                    B.fin[k] = 1;  // no shrink: this system ends here
                    stalled = true;
                }
            }
            nc = nroots;
            if (!stalled) break;
            if (attempt > ns) {
                set_last_error("batched coarsening did not settle at level %d", l);
                return AMG_ERR_STALL;
            }
        }
        Lv.A.v32 = nullptr;
        AMG_TRY(batch_dense(h, l, s));
        bool any_active = false;
        for (int k = 0; k < ns; ++k) any_active |= !B.fin[k];
        if (!any_active) break;

        // prolongator with per-system omega_P
        unsigned long long *rho_bits;
        double *om_sys, *om_row;
        AMG_TRY(sc.alloc(&rho_bits, (size_t)ns));
        AMG_TRY(sc.alloc(&om_sys, (size_t)ns));
        AMG_TRY(sc.alloc(&om_row, (size_t)nl));
        AMG_CUDA_TRY(cudaMemsetAsync(rho_bits, 0, sizeof(unsigned long long) * ns, s));
        k_gershgorin_sys<<<grid_for(nl), 256, 0, s>>>(nl, A.rp, A.v, diag, row_sys, active, rho_bits);
        AMG_LAUNCH_CHECK();
        std::vector<unsigned long long> hb(ns);
        AMG_CUDA_TRY(cudaMemcpyAsync(hb.data(), rho_bits, sizeof(unsigned long long) * ns, cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        std::vector<double> hom(ns, 0.0);
        double rho_max = 0.0;
        for (int k = 0; k < ns; ++k) {
            if (B.fin[k]) continue;
            double rho;
            memcpy(&rho, &hb[k], sizeof(rho));
            const double c43 = 4.0 / 3.0;
            hom[k] = c43 / rho;
            rho_max = std::max(rho_max, rho);
        }
        Lv.rho = rho_max;
        AMG_CUDA_TRY(cudaMemcpyAsync(om_sys, hom.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s));
        k_omega_rows<<<grid_for(nl), 256, 0, s>>>(nl, row_sys, active, om_sys, om_row);
        int *tflag, *trp, *tci;
        AMG_TRY(sc.alloc(&tflag, (size_t)nl + 1));
        AMG_TRY(sc.alloc(&trp, (size_t)nl + 1));
        k_assigned<<<grid_for(nl), 256, 0, s>>>(nl, Lv.agg, tflag);
        AMG_LAUNCH_CHECK();
        int tnnz = 0;
        AMG_TRY(exclusive_scan_int(tflag, trp, nl, &tnnz, s));
        AMG_TRY(sc.alloc(&tci, (size_t)std::max(1, tnnz)));
        k_t_fill<<<grid_for(nl), 256, 0, s>>>(nl, Lv.agg, trp, tci);
        AMG_LAUNCH_CHECK();
        ProlongEpi epi{Lv.agg, diag, 0.0, om_row};
        AMG_TRY((spgemm<EPI_PROLONG>(nl, nc, A.rp, A.ci, A.v, trp, tci, nullptr, epi, Lv.P, ar, s)));
        AMG_TRY(transpose_csr(Lv.P, Lv.R, ar, s));
        DevCSR AP;
        AMG_TRY((spgemm<EPI_NONE>(nl, nc, A.rp, A.ci, A.v, Lv.P.rp, Lv.P.ci, Lv.P.v, ProlongEpi{}, AP, sc.arena, s)));
        Level &Ln = h->L[l + 1];
        AMG_TRY((spgemm<EPI_NONE>(nc, nc, Lv.R.rp, Lv.R.ci, Lv.R.v, AP.rp, AP.ci, AP.v, ProlongEpi{}, Ln.A, ar, s)));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        // the next level holds the systems still coarsening
        BatchLevel &Bn = h->bl[l + 1];
        Bn.sys.clear();
        Bn.off.assign(1, 0);
        for (int k = 0; k < ns; ++k)
            if (!B.fin[k]) {
                Bn.sys.push_back(B.sys[k]);
                Bn.off.push_back(Bn.off.back() + nc_sys[k]);
            }
        ++l;
    }
    h->nlevels = l + 1;
    h->nsolve = h->nlevels;
    h->nc = 0;
    h->cinv = nullptr;
    // Ahat = A W, FP32 copies; work vectors are allocated by the batched workspace
    const bool mixed = cfg.precision == AMG_PRECISION_MIXED;
    for (int k = 0; k < h->nlevels; ++k) {
        Level &Lv = h->L[k];
        const int nl = Lv.A.nrows;
        const bool last = k == h->nlevels - 1;
        Lv.vec_a = choose_vec(Lv.A.nnz, nl);
        AMG_TRY(ar.alloc(&Lv.ahat, (size_t)std::max(1LL, Lv.A.nnz)));
        if (mixed) AMG_TRY(ar.alloc(&Lv.ahat32, (size_t)std::max(1LL, Lv.A.nnz)));
        k_scale_cols<<<grid_for(nl), 256, 0, s>>>(nl, Lv.A.rp, Lv.A.ci, Lv.A.v, Lv.w, Lv.ahat, Lv.ahat32);
        if (!last) {
            Lv.vec_p = choose_vec(Lv.P.nnz, nl);
            Lv.vec_r = choose_vec(Lv.R.nnz, Lv.R.nrows);
        }
        if (mixed) {
            AMG_TRY(ar.alloc(&Lv.A.v32, (size_t)std::max(1LL, Lv.A.nnz)));
            k_to_f32<<<grid_for(Lv.A.nnz), 256, 0, s>>>(Lv.A.v, Lv.A.v32, Lv.A.nnz);
            AMG_TRY(ar.alloc(&Lv.w32, (size_t)nl));
            k_to_f32<<<grid_for(nl), 256, 0, s>>>(Lv.w, Lv.w32, nl);
            if (!last) {
                AMG_TRY(ar.alloc(&Lv.P.v32, (size_t)std::max(1LL, Lv.P.nnz)));
                k_to_f32<<<grid_for(Lv.P.nnz), 256, 0, s>>>(Lv.P.v, Lv.P.v32, Lv.P.nnz);
                AMG_TRY(ar.alloc(&Lv.R.v32, (size_t)std::max(1LL, Lv.R.nnz)));
                k_to_f32<<<grid_for(Lv.R.nnz), 256, 0, s>>>(Lv.R.v, Lv.R.v32, Lv.R.nnz);
            }
        }
        AMG_LAUNCH_CHECK();
    }
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    return AMG_OK;
}

// The adjoint's hierarchy of A^T reusing A's (ht set up from h, which must
// be preconditioned and nonsymmetric): the same aggregates, P and R = P^T
// (their index and FP64 value arrays shared with h, which outlives ht),
// every level operator the exact transpose of h's -- since R = P^T, the
// Galerkin product of the transposed level above -- and smoother weights
// from the transposed operators; the rest is built as for any hierarchy.
static int transpose_levels(Hierarchy *ht, const Hierarchy *h, bool alloc, cudaStream_t s) {
    const amg_config &cfg = ht->cfg;
    for (int l = 0; l < h->nlevels; ++l) {
        Level &Lt = ht->L[l];
        const Level &Lf = h->L[l];
        const int nl = Lf.A.nrows;
        if (alloc) {
            AMG_TRY(transpose_csr(Lf.A, Lt.A, ht->arena, s));
        } else {
            DevArena tmp;
            DevCSR At;
            int rc = transpose_csr(Lf.A, At, tmp, s);
            if (rc == AMG_OK && cudaMemcpyAsync(Lt.A.v, At.v, sizeof(double) * (size_t)At.nnz, cudaMemcpyDeviceToDevice,
                                                s) != cudaSuccess)
                rc = AMG_ERR_CUDA;
            const cudaError_t e = cudaStreamSynchronize(s);
            tmp.free_all();
            AMG_TRY(rc);
            AMG_CUDA_TRY(e);
        }
        Scratch sc;
        double *diag;
        int *bad;
        AMG_TRY(sc.alloc(&diag, (size_t)nl));
        AMG_TRY(sc.alloc(&bad, 1));
        AMG_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
        k_find_diag<<<grid_for(nl), 256, 0, s>>>(nl, Lt.A.rp, Lt.A.ci, Lt.A.v, diag, bad);
        if (alloc) AMG_TRY(ht->arena.alloc(&Lt.w, (size_t)nl));
        k_smoother_weights<<<grid_for(nl), 256, 0, s>>>(nl, Lt.A.rp, Lt.A.v, diag, cfg.omega,
                                                        cfg.smoother == AMG_SMOOTHER_L1_JACOBI, Lt.w);
        AMG_LAUNCH_CHECK();
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        if (alloc && l < h->nlevels - 1) {
            // shared with h: patterns and FP64 values (FP32 copies are ht's own)
            Lt.P = Lf.P;
            Lt.R = Lf.R;
            Lt.P.v32 = nullptr;
            Lt.R.v32 = nullptr;
            Lt.agg = Lf.agg;
            Lt.rho = Lf.rho;
        }
    }
    return AMG_OK;
}

int build_transposed_hierarchy(Hierarchy *ht, const Hierarchy *h, cudaStream_t s) {
    ht->cfg = h->cfg;
    ht->cfg.symmetric = 0;
    ht->symmetric = 0;
    ht->n = h->n;
    ht->nnz = h->nnz;
    ht->transposed_of = h;
    AMG_TRY(transpose_levels(ht, h, true, s));
    ht->nlevels = h->nlevels;
    return finish_build(ht, true, s);
}

int refresh_transposed_hierarchy(Hierarchy *ht, const Hierarchy *h, cudaStream_t s) {
    AMG_TRY(transpose_levels(ht, h, false, s));
    return refresh_derived(ht, s);
}

void free_hierarchy(Hierarchy *h) {
    if (!h) return;
    if (h->iter_exec) cudaGraphExecDestroy(h->iter_exec);
    h->iter_exec = nullptr;
    if (h->loop_exec) cudaGraphExecDestroy(h->loop_exec);
    if (h->loop_graph) cudaGraphDestroy(h->loop_graph);
    h->loop_exec = nullptr;
    h->loop_graph = nullptr;
    h->arena.free_all();
}

}  // namespace amg
