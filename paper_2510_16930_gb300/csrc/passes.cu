// The two streaming passes of one HOQRI block update (mode n).
//
// Both passes walk the mode-n sorted nonzeros.  For a non-empty row i of X_(n)
// (the index set I^(n)_i of Table 1) they form
//     y_i = sum_{z in I^(n)_i} x_z * kron_{m != n} U_m(i_m(z), :)      (P_{-n} values)
// which is row i of Y_(n), Y = X x_{-n} {U^T} (Eq. ttmctc), without ever
// storing Y.  Then
//     core pass:   G_(n) += U_n(i, :)^T y_i^T      (G = X x {U^T} = U_n^T Y_(n))
//     TTMcTC pass: A_n(i, :) = G_(n) y_i          (A_n = Y_(n) G_(n)^T)
// This regroups the sums of Alg. 3 by row, which costs nnz*P_{-n} + R_n*P
// multiply-adds, the second complexity of Table 2.
//
// Work split: the sorted stream is cut into chunks of C consecutive nonzeros,
// one warp task each.  A row that crosses a chunk boundary is summed in pieces:
// the core pass is linear in y_i, so pieces add into G directly; the TTMcTC pass
// writes the piece's K_n-vector G_(n) y_piece to a per-chunk slot and a fix-up
// kernel adds the pieces of each crossing row in chunk order.  No floating
// point atomics anywhere: every sum has a fixed order for a given context, so
// results are bitwise reproducible run to run.
#include <algorithm>

#include "internal.cuh"

namespace hoqri {

namespace {

constexpr int GEN_WARPS = 4;  // warps per CTA of the generic pass kernel
constexpr int RED_TPB = 256;

template <typename T>
struct PassArgs {
    int nm1;                       // N - 1
    int Kn;                        // K_n
    int Ko[HOQRI_MAXN - 1];        // ranks of the other modes (ascending m != n)
    int roff[HOQRI_MAXN - 1];      // offset of each gathered row in the row buffer
    int rtot;                      // sum of Ko
    int Pm;                        // prod Ko = P_{-n}
    int Kl;                        // Ko[nm1-1] (last other mode: fastest in y)
    int L;                         // Pm / Kl
    const int32_t *oidx[HOQRI_MAXN - 1];
    const T *Uo[HOQRI_MAXN - 1];
    const T *Un;
    const T *vals;
    const int64_t *row_ptr;
    const int32_t *row_id;
    const int32_t *chunk_row;
    int64_t nchunks;
    int64_t nnz;
    int C;
    int wstride;                   // per-warp shared memory (elements of T)
    int acc_in_smem;               // core accumulator in shared memory (else global)
    T *acc_glob;                   // [grid*GEN_WARPS][Kn*Pm] when not in smem
    const T *Gn;                   // TTMcTC: G_(n) as [Kn][Pm]
    int gn_in_smem;
    T *A;                          // TTMcTC output, I_n x K_n
    T *apart;                      // [nchunks][2][Kn]
    T *cpart;                      // core: [grid][Kn*Pm]
};

__device__ __forceinline__ float shfl_idx(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double shfl_idx(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ int shfl_idx(int v, int src) { return __shfl_sync(0xffffffffu, v, src); }

template <typename T>
__device__ __forceinline__ T warp_allsum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Generic pass: any N <= 8, K <= 64, P_{-n} <= 32*PL.  y lives in registers
// (element e = lane + 32*j of the lane); each nonzero's factor rows are staged
// in the warp's shared row buffer, the Kronecker prefix z (all other modes but
// the last) is formed once per nonzero in shared memory, and
// y[e] += z[e / Kl] * u_last[e % Kl].
template <typename T, int PL, bool CORE>
__global__ void __launch_bounds__(GEN_WARPS * 32) k_pass_generic(PassArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int KnPm = a.Kn * a.Pm;
    // shared layout: [Gn (TTMcTC, optional)] [per-warp: rowbuf | zbuf | acc (core, optional)]
    T *gn = a.Gn ? (T *)a.Gn : nullptr;
    T *wbase = sm;
    if (!CORE && a.gn_in_smem) {
        for (int p = threadIdx.x; p < KnPm; p += blockDim.x) sm[p] = a.Gn[p];
        gn = sm;
        wbase = sm + KnPm;
    }
    T *rowbuf = wbase + (size_t)wib * a.wstride;
    T *zbuf = rowbuf + a.rtot;
    T *acc = nullptr;
    if (CORE) {
        acc = a.acc_in_smem ? zbuf + a.L
                            : a.acc_glob + ((size_t)blockIdx.x * GEN_WARPS + wib) * KnPm;
        for (int p = lane; p < KnPm; p += 32) acc[p] = T(0);
    }
    __syncthreads();

    int qj[PL], rj[PL];
#pragma unroll
    for (int j = 0; j < PL; ++j) {
        int e = lane + 32 * j;
        qj[j] = e / a.Kl;
        rj[j] = e % a.Kl;
    }
    const int lastoff = a.roff[a.nm1 - 1];
    const int64_t gw = (int64_t)blockIdx.x * GEN_WARPS + wib;
    const int64_t nw = (int64_t)gridDim.x * GEN_WARPS;

    for (int64_t ch = gw; ch < a.nchunks; ch += nw) {
        const int64_t s0 = ch * a.C;
        const int64_t s1 = min(s0 + (int64_t)a.C, a.nnz);
        const int32_t r_first = a.chunk_row[ch];
        int32_t rr = r_first;
        int64_t pos = s0;
        while (pos < s1) {
            const int64_t rs = a.row_ptr[rr], re = a.row_ptr[rr + 1];
            const int64_t a0 = pos, a1 = min(re, s1);
            if (a1 <= a0) break;  // row descriptors always advance; never spin on bad input
            T y[PL];
#pragma unroll
            for (int j = 0; j < PL; ++j) y[j] = T(0);
            for (int64_t b = a0; b < a1; b += 32) {
                const int nb = (int)min((int64_t)32, a1 - b);
                int mi[HOQRI_MAXN - 1];
                T mx = T(0);
                for (int j = 0; j < a.nm1; ++j) mi[j] = 0;
                if (lane < nb) {
                    for (int j = 0; j < a.nm1; ++j) mi[j] = a.oidx[j][b + lane];
                    mx = a.vals[b + lane];
                }
                for (int t = 0; t < nb; ++t) {
                    const T x = shfl_idx(mx, t);
                    for (int j = 0; j < a.nm1; ++j) {
                        const int i = shfl_idx(mi[j], t);
                        const T *src = a.Uo[j] + (int64_t)i * a.Ko[j];
                        for (int k = lane; k < a.Ko[j]; k += 32) rowbuf[a.roff[j] + k] = src[k];
                    }
                    __syncwarp();
                    for (int l = lane; l < a.L; l += 32) {
                        T z = x;
                        int rem = l;
                        for (int j = a.nm1 - 2; j >= 0; --j) {
                            const int k = rem % a.Ko[j];
                            rem /= a.Ko[j];
                            z *= rowbuf[a.roff[j] + k];
                        }
                        zbuf[l] = z;
                    }
                    __syncwarp();
#pragma unroll
                    for (int j = 0; j < PL; ++j)
                        if (lane + 32 * j < a.Pm) y[j] += zbuf[qj[j]] * rowbuf[lastoff + rj[j]];
                    __syncwarp();
                }
            }
            const int32_t row = a.row_id[rr];
            if (CORE) {
                for (int kn = 0; kn < a.Kn; ++kn) {
                    const T u = a.Un[(int64_t)row * a.Kn + kn];
                    T *ak = acc + (size_t)kn * a.Pm;
#pragma unroll
                    for (int j = 0; j < PL; ++j) {
                        const int e = lane + 32 * j;
                        if (e < a.Pm) ak[e] += u * y[j];
                    }
                }
            } else {
                const bool full = (rs >= s0) && (re <= s1);
                T *dst = full ? a.A + (int64_t)row * a.Kn
                              : a.apart + (ch * 2 + (rr == r_first ? 0 : 1)) * a.Kn;
                for (int kn = 0; kn < a.Kn; ++kn) {
                    const T *g = gn + (size_t)kn * a.Pm;
                    T s = T(0);
#pragma unroll
                    for (int j = 0; j < PL; ++j) {
                        const int e = lane + 32 * j;
                        if (e < a.Pm) s += g[e] * y[j];
                    }
                    s = warp_allsum(s);
                    if (lane == 0) dst[kn] = s;
                }
            }
            pos = a1;
            ++rr;
        }
    }
    if (CORE) {
        __syncthreads();
        // CTA partial = sum of the warp accumulators in warp order
        for (int p = threadIdx.x; p < KnPm; p += blockDim.x) {
            T s = T(0);
            for (int w = 0; w < GEN_WARPS; ++w) {
                const T *aw = a.acc_in_smem ? (wbase + (size_t)w * a.wstride + a.rtot + a.L)
                                            : a.acc_glob + ((size_t)blockIdx.x * GEN_WARPS + w) * KnPm;
                s += aw[p];
            }
            a.cpart[(size_t)blockIdx.x * KnPm + p] = s;
        }
    }
}

// sum of the per-chunk pieces of each row that crosses chunk boundaries
template <typename T>
__global__ void k_fixup(const int32_t *split_row, int64_t nsplit, const int64_t *row_ptr, const int32_t *row_id,
                        const int32_t *chunk_row, int C, const T *apart, int Kn, T *A) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nsplit) return;
    const int32_t r = split_row[w];
    const int64_t c0 = row_ptr[r] / C, c1 = (row_ptr[r + 1] - 1) / C;
    const int first_slot = (chunk_row[c0] == r) ? 0 : 1;
    for (int kn = 0; kn < Kn; ++kn) {
        double s = 0.0;
        for (int64_t c = c0 + lane; c <= c1; c += 32)
            s += (double)apart[(c * 2 + (c == c0 ? first_slot : 0)) * Kn + kn];
        s = warp_allsum(s);
        if (lane == 0) A[(int64_t)row_id[r] * Kn + kn] = (T)s;
    }
}

struct CoreMap {
    int nm1, Kn, Pm;
    int Ko[HOQRI_MAXN - 1];
    int64_t gso[HOQRI_MAXN - 1];
    int64_t gsn;
};

__device__ __forceinline__ int64_t rowmajor_of(const CoreMap &m, int p) {
    int kn = p / m.Pm;
    int e = p - kn * m.Pm;
    int64_t g = (int64_t)kn * m.gsn;
    for (int j = m.nm1 - 1; j >= 0; --j) {
        int k = e % m.Ko[j];
        e /= m.Ko[j];
        g += (int64_t)k * m.gso[j];
    }
    return g;
}

// G (row-major) = sum over CTAs of the [Kn][Pm] partials, in CTA order; block
// partial sums of ||G||^2.
template <typename T>
__global__ void k_core_reduce(const T *cpart, int nblk, CoreMap m, T *G, double *gpart) {
    __shared__ double sh[RED_TPB];
    const int P = m.Kn * m.Pm;
    double sq = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += (double)cpart[(size_t)b * P + p];
        const T v = (T)s;
        G[rowmajor_of(m, p)] = v;
        sq += (double)v * (double)v;
    }
    sh[threadIdx.x] = sq;
    __syncthreads();
    for (int w = RED_TPB / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) gpart[blockIdx.x] = sh[0];
}

__global__ void k_sum_into(const double *part, int n, double *out, double *out2) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = s;
        if (out2) *out2 = s;
    }
}

// Gn[kn][e] = G(row-major) for the TTMcTC pass
template <typename T>
__global__ void k_core_to_unfolded(const T *G, CoreMap m, T *Gn) {
    const int P = m.Kn * m.Pm;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) Gn[p] = G[rowmajor_of(m, p)];
}

template <typename T>
void fill_common(hoqri_ctx *c, int n, PassArgs<T> &a) {
    const ModeStore &M = c->ms[n];
    a.nm1 = c->N - 1;
    a.Kn = c->K[n];
    int j = 0, off = 0;
    a.Pm = 1;
    for (int m = 0; m < c->N; ++m) {
        if (m == n) continue;
        a.Ko[j] = c->K[m];
        a.roff[j] = off;
        off += c->K[m];
        a.Pm *= c->K[m];
        a.oidx[j] = M.oidx[j];
        a.Uo[j] = (const T *)c->U[m];
        ++j;
    }
    a.rtot = off;
    a.Kl = a.Ko[a.nm1 - 1];
    a.L = a.Pm / a.Kl;
    a.Un = (const T *)c->U[n];
    a.vals = (const T *)M.vals;
    a.row_ptr = M.row_ptr;
    a.row_id = M.row_id;
    a.chunk_row = M.chunk_row;
    a.nchunks = M.nchunks;
    a.nnz = c->nnz;
    a.C = M.C;
}

CoreMap core_map(hoqri_ctx *c, int n) {
    CoreMap m{};
    int64_t st[HOQRI_MAXN];
    st[c->N - 1] = 1;
    for (int q = c->N - 2; q >= 0; --q) st[q] = st[q + 1] * c->K[q + 1];
    m.nm1 = c->N - 1;
    m.Kn = c->K[n];
    m.gsn = st[n];
    m.Pm = 1;
    int j = 0;
    for (int q = 0; q < c->N; ++q) {
        if (q == n) continue;
        m.Ko[j] = c->K[q];
        m.gso[j] = st[q];
        m.Pm *= c->K[q];
        ++j;
    }
    return m;
}

int pl_for(int Pm) {
    int pl = 1;
    while (32 * pl < Pm) pl <<= 1;
    return pl;
}

template <typename T, bool CORE>
hoqri_status launch_generic(hoqri_ctx *c, PassArgs<T> &a, int grid, size_t smem) {
    const int pl = pl_for(a.Pm);
#define HQ_GEN(PLV)                                                                                   \
    case PLV: {                                                                                       \
        auto kern = k_pass_generic<T, PLV, CORE>;                                                     \
        HQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        kern<<<grid, GEN_WARPS * 32, smem, c->stream>>>(a);                                           \
        c->nlaunch++;                                                                                 \
        break;                                                                                        \
    }
    switch (pl) {
        HQ_GEN(1)
        HQ_GEN(2)
        HQ_GEN(4)
        HQ_GEN(8)
        HQ_GEN(16)
        HQ_GEN(32)
        HQ_GEN(64)
        default:
            set_error("P_{-n} = prod_{m != n} K_m above 2048 is not supported by this build");
            return HOQRI_ERR_UNSUPPORTED;
    }
#undef HQ_GEN
    HQ_CUDA(cudaGetLastError());
    return HOQRI_OK;
}

constexpr size_t SMEM_CAP = 200 * 1024;

template <typename T>
hoqri_status core_pass_t(hoqri_ctx *c, int n, void *G_out, double *normG2_slot) {
    PassArgs<T> a{};
    fill_common<T>(c, n, a);
    const int KnPm = a.Kn * a.Pm;
    a.wstride = (a.rtot + a.L + KnPm + 3) & ~3;
    size_t smem = (size_t)GEN_WARPS * a.wstride * sizeof(T);
    a.acc_in_smem = smem <= SMEM_CAP;
    if (!a.acc_in_smem) {
        a.wstride = (a.rtot + a.L + 3) & ~3;
        smem = (size_t)GEN_WARPS * a.wstride * sizeof(T);
    }
    const int grid = c->core_grid;
    a.acc_glob = (T *)c->a_part;  // only used when the accumulator does not fit in smem
    a.cpart = (T *)c->core_part;
    if (!a.acc_in_smem && (int64_t)grid * GEN_WARPS * KnPm * (int64_t)sizeof(T) > c->a_part_bytes) {
        set_error("core pass: accumulator workspace too small");
        return HOQRI_ERR_UNSUPPORTED;
    }
    HQ_TRY((launch_generic<T, true>(c, a, grid, smem)));
    CoreMap m = core_map(c, n);
    const int rb = std::max(1, std::min(64, (KnPm + RED_TPB - 1) / RED_TPB));
    k_core_reduce<T><<<rb, RED_TPB, 0, c->stream>>>((const T *)c->core_part, grid, m, (T *)G_out, c->gnorm_part);
    k_sum_into<<<1, 32, 0, c->stream>>>(c->gnorm_part, rb, c->dnorm + 1, normG2_slot);
    c->nlaunch += 2;
    HQ_CUDA(cudaGetLastError());
    return HOQRI_OK;
}

template <typename T>
hoqri_status ttmctc_pass_t(hoqri_ctx *c, int n, const void *G, void *A_out) {
    const ModeStore &M = c->ms[n];
    PassArgs<T> a{};
    fill_common<T>(c, n, a);
    const int KnPm = a.Kn * a.Pm;
    CoreMap m = core_map(c, n);
    T *Gn = (T *)c->core_part;  // core partials are consumed; reuse the buffer for G_(n)
    k_core_to_unfolded<T><<<std::max(1, std::min(64, (KnPm + 255) / 256)), 256, 0, c->stream>>>((const T *)G, m, Gn);
    c->nlaunch++;
    HQ_CUDA(cudaMemsetAsync(A_out, 0, (size_t)c->dims[n] * a.Kn * sizeof(T), c->stream));
    a.Gn = Gn;
    a.A = (T *)A_out;
    a.apart = (T *)c->a_part;
    if ((int64_t)M.nchunks * 2 * a.Kn * (int64_t)sizeof(T) > c->a_part_bytes) {
        set_error("TTMcTC pass: partial-row workspace too small");
        return HOQRI_ERR_UNSUPPORTED;
    }
    a.wstride = (a.rtot + a.L + 3) & ~3;
    size_t smem = (size_t)GEN_WARPS * a.wstride * sizeof(T);
    a.gn_in_smem = (smem + (size_t)KnPm * sizeof(T)) <= SMEM_CAP;
    if (a.gn_in_smem) smem += (size_t)KnPm * sizeof(T);
    const int grid = c->pass_grid;
    HQ_TRY((launch_generic<T, false>(c, a, grid, smem)));
    if (M.nsplit > 0) {
        const int tpb = 256;
        const int64_t blocks = ceil_div(M.nsplit * 32, tpb);
        k_fixup<T><<<(unsigned)blocks, tpb, 0, c->stream>>>(M.split_row, M.nsplit, M.row_ptr, M.row_id, M.chunk_row,
                                                            M.C, (const T *)c->a_part, a.Kn, (T *)A_out);
        c->nlaunch++;
    }
    HQ_CUDA(cudaGetLastError());
    return HOQRI_OK;
}

}  // namespace

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Sizes the partition and the scratch buffers of the passes.
hoqri_status passes_init(hoqri_ctx *c) {
    int32_t C = c->opt.chunk_nnz;
    if (C <= 0) {
        // about 8 tasks per resident warp, within [32, 2048]
        int64_t target = ceil_div(c->nnz, (int64_t)c->num_sms * 16 * 8);
        C = 32;
        while (C < target && C < 2048) C <<= 1;
    }
    int64_t max_chunks = 0;
    for (int n = 0; n < c->N; ++n) {
        HQ_TRY(build_partition(c, n, C));
        max_chunks = std::max(max_chunks, c->ms[n].nchunks);
    }
    const int64_t want = ceil_div(std::max<int64_t>(max_chunks, 1), GEN_WARPS);
    c->pass_grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)c->num_sms * 4));
    c->core_grid = c->pass_grid;
    int maxK = 1;
    for (int n = 0; n < c->N; ++n) maxK = std::max(maxK, (int)c->K[n]);
    // core partials [grid][P]; also holds G_(n) for the TTMcTC pass
    c->core_part_bytes = (int64_t)std::max(c->core_grid, 1) * c->P * (int64_t)c->rsize;
    HQ_TRY(dalloc(c, &c->core_part, c->core_part_bytes));
    // per-chunk partial rows [nchunks][2][Kn], or per-warp core accumulators
    int64_t ab = std::max<int64_t>(max_chunks, 1) * 2 * maxK * (int64_t)c->rsize;
    for (int n = 0; n < c->N; ++n) {
        // same test as core_pass_t: does the per-warp accumulator fit in shared memory?
        int64_t rtot = 0, Pm = 1;
        for (int m = 0; m < c->N; ++m)
            if (m != n) {
                rtot += c->K[m];
                Pm *= c->K[m];
            }
        const int64_t Kl = c->K[n == c->N - 1 ? c->N - 2 : c->N - 1];
        const int64_t wst = (rtot + Pm / Kl + c->P + 3) & ~3LL;
        if ((int64_t)GEN_WARPS * wst * (int64_t)c->rsize > (int64_t)SMEM_CAP)
            ab = std::max(ab, (int64_t)c->core_grid * GEN_WARPS * c->P * (int64_t)c->rsize);
    }
    c->a_part_bytes = ab;
    HQ_TRY(dalloc(c, &c->a_part, c->a_part_bytes));
    HQ_TRY(dalloc(c, (void **)&c->gnorm_part, 64 * sizeof(double)));
    return HOQRI_OK;
}

hoqri_status core_pass(hoqri_ctx *c, int n, void *G_out, double *normG2_slot) {
    cudaEvent_t e0 = nullptr;
    HQ_TRY(prof_begin(c, 0, &e0));
    hoqri_status s = (c->prec == HOQRI_FP64) ? core_pass_t<double>(c, n, G_out, normG2_slot)
                                             : core_pass_t<float>(c, n, G_out, normG2_slot);
    HQ_TRY(s);
    return prof_end(c, 0, e0);
}

hoqri_status ttmctc_pass(hoqri_ctx *c, int n, const void *G, void *A_out) {
    cudaEvent_t e0 = nullptr;
    HQ_TRY(prof_begin(c, 1, &e0));
    hoqri_status s = (c->prec == HOQRI_FP64) ? ttmctc_pass_t<double>(c, n, G, A_out)
                                             : ttmctc_pass_t<float>(c, n, G, A_out);
    HQ_TRY(s);
    return prof_end(c, 1, e0);
}

}  // namespace hoqri
