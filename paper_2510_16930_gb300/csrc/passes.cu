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
// Work split: the sorted stream is cut into chunks of at most C nonzeros, one
// warp task each; whole rows are packed into a chunk, and a row longer than C
// is cut into pieces that are chunks of their own.  The core pass is linear in
// y_i, so pieces add into G directly; the TTMcTC pass writes each piece's
// K_n-vector G_(n) y_piece to a per-chunk slot and a fix-up kernel adds the
// pieces of each long row in chunk order.  No floating point atomics anywhere:
// every sum has a fixed order for a given context, so results are bitwise
// reproducible run to run.
//
// Two kernels implement the passes:
//  - k_pass_fast (FP32): the y_i of a row is a sum of rank-1 terms z (x) v, with
//    v the last other mode's factor row and z = x * (Kronecker product of the
//    remaining ones).  Each lane owns a TL x TV register tile of y; the lanes
//    of a warp form groups that take every NG-th nonzero of the row (split over
//    nonzeros), and the group partial sums are added with warp shuffles at the
//    row end.  The chunk's index and value streams are staged in shared memory
//    by TMA bulk copies (cp.async.bulk, completion on an mbarrier), double
//    buffered, so the next chunk is in flight while the current one computes.
//  - k_pass_generic (any N <= 8, K <= 64, FP32 or FP64): y in registers, factor
//    rows staged per nonzero in shared memory.
#include <algorithm>
#include <type_traits>

#include "internal.cuh"

namespace hoqri {

namespace {

constexpr int GEN_WARPS = 4;  // warps per CTA of the generic pass kernel
constexpr int RED_TPB = 256;
constexpr size_t SMEM_CAP = 200 * 1024;
constexpr int FAST_MAX_CTAS_PER_SM = 4;

// ------------------------------------------------------------------ helpers

template <typename T>
__device__ __forceinline__ T shfl_idx(T v, int src) {
    return __shfl_sync(0xffffffffu, v, src);
}

template <typename T>
__device__ __forceinline__ T warp_allsum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// bounded wait on an mbarrier phase; false (and *err set) if the limit ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int32_t *err) {
    const uint32_t a = smem_addr(bar);
    for (int it = 0; it < (1 << 21); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    if (err) atomicExch(err, 1);
    return false;
}

// 1-D TMA bulk copy global -> shared, completion counted on an mbarrier.
// dst, src and bytes are multiples of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ------------------------------------------------------------ generic kernel

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
    // column block of this launch: columns [e0, e0 + Pb) of Y_(n) and G_(n)
    // (e0 and Pb multiples of Kl; one block covers every column when Pm <= 2048)
    int e0, Pb, q0, Lb;            // q0 = e0 / Kl, Lb = Pb / Kl Kronecker prefixes
    int accum;                     // TTMcTC: add into A / apart (blocks after the first)
    const int32_t *oidx[HOQRI_MAXN - 1];
    const T *Uo[HOQRI_MAXN - 1];
    const T *Un;
    const T *vals;
    const int64_t *row_ptr;
    const int32_t *row_id;
    const int64_t *chunk_start;
    const int32_t *chunk_row;
    int64_t nchunks;
    int wstride;                   // per-warp shared memory (elements of T)
    int acc_in_smem;               // core accumulator in shared memory (else global)
    T *acc_glob;                   // [grid*GEN_WARPS][Kn*Pm] when not in smem
    const T *Gn;                   // TTMcTC: G_(n) as [Kn][Pm]
    int gn_in_smem;
    T *A;                          // TTMcTC output, I_n x K_n
    T *apart;                      // [nchunks][Kn] pieces of long rows
    T *cpart;                      // core: [grid][Kn*Pm]
};

// Generic pass: y lives in registers (element e = e0 + lane + 32*j of the
// lane, over the launch's column block); each nonzero's factor rows are staged
// in the warp's shared row buffer, the block's Kronecker prefixes z (all other
// modes but the last) are formed once per nonzero in shared memory, and
// y[e] += z[e / Kl] * u_last[e % Kl].  P_{-n} above 2048 runs as several
// launches, one per column block: the core pass fills its block's columns of
// the CTA partials, the TTMcTC pass adds its block's share of A_n(i, :) =
// G_(n) y_i in block order.
template <typename T, int PL, bool CORE>
__global__ void __launch_bounds__(GEN_WARPS * 32) k_pass_generic(PassArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int KnPm = a.Kn * a.Pm;
    const T *gn = a.Gn;
    T *wbase = sm;
    if (!CORE && a.gn_in_smem) {
        for (int p = threadIdx.x; p < KnPm; p += blockDim.x) sm[p] = a.Gn[p];
        gn = sm;
        wbase = sm + KnPm;
    }
    T *rowbuf = wbase + (size_t)wib * a.wstride;
    T *zbuf = rowbuf + a.rtot;
    const int KnPb = a.Kn * a.Pb;
    T *acc = nullptr;
    if (CORE) {
        acc = a.acc_in_smem ? zbuf + a.Lb : a.acc_glob + ((size_t)blockIdx.x * GEN_WARPS + wib) * KnPb;
        for (int p = lane; p < KnPb; p += 32) acc[p] = T(0);
    }
    __syncthreads();

    int qj[PL], rj[PL];  // prefix (relative to the block's first) and last-mode index of column e
#pragma unroll
    for (int j = 0; j < PL; ++j) {
        int e = a.e0 + lane + 32 * j;
        qj[j] = e / a.Kl - a.q0;
        rj[j] = e % a.Kl;
    }
    const int lastoff = a.roff[a.nm1 - 1];
    const int64_t gw = (int64_t)blockIdx.x * GEN_WARPS + wib;
    const int64_t nw = (int64_t)gridDim.x * GEN_WARPS;

    for (int64_t ch = gw; ch < a.nchunks; ch += nw) {
        const int64_t s0 = a.chunk_start[ch];
        const int64_t s1 = a.chunk_start[ch + 1];
        int32_t rr = a.chunk_row[ch];
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
                    for (int l = lane; l < a.Lb; l += 32) {
                        T z = x;
                        int rem = a.q0 + l;
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
                        if (lane + 32 * j < a.Pb) y[j] += zbuf[qj[j]] * rowbuf[lastoff + rj[j]];
                    __syncwarp();
                }
            }
            const int32_t row = a.row_id[rr];
            if (CORE) {
                for (int kn = 0; kn < a.Kn; ++kn) {
                    const T u = a.Un[(int64_t)row * a.Kn + kn];
                    T *ak = acc + (size_t)kn * a.Pb;
#pragma unroll
                    for (int j = 0; j < PL; ++j) {
                        const int e = lane + 32 * j;
                        if (e < a.Pb) ak[e] += u * y[j];
                    }
                }
            } else {
                const bool full = (rs >= s0) && (re <= s1);
                T *dst = full ? a.A + (int64_t)row * a.Kn : a.apart + ch * a.Kn;
                for (int kn = 0; kn < a.Kn; ++kn) {
                    const T *g = gn + (size_t)kn * a.Pm + a.e0;
                    T s = T(0);
#pragma unroll
                    for (int j = 0; j < PL; ++j) {
                        const int e = lane + 32 * j;
                        if (e < a.Pb) s += g[e] * y[j];
                    }
                    s = warp_allsum(s);
                    if (lane == 0) dst[kn] = a.accum ? dst[kn] + s : s;
                }
            }
            pos = a1;
            ++rr;
        }
    }
    if (CORE) {
        __syncthreads();
        // CTA partial = sum of the warp accumulators in warp order (the block's columns)
        for (int p = threadIdx.x; p < KnPb; p += blockDim.x) {
            T s = T(0);
            for (int w = 0; w < GEN_WARPS; ++w) {
                const T *aw = a.acc_in_smem ? (wbase + (size_t)w * a.wstride + a.rtot + a.Lb)
                                            : a.acc_glob + ((size_t)blockIdx.x * GEN_WARPS + w) * KnPb;
                s += aw[p];
            }
            const int kn = p / a.Pb, e = p - kn * a.Pb;
            a.cpart[(size_t)blockIdx.x * KnPm + (size_t)kn * a.Pm + a.e0 + e] = s;
        }
    }
}

// --------------------------------------------------------------- fast kernel

struct FastArgs {
    int Kn, Pm, Kl;                // K_n, P_{-n}, rank of the last other mode
    int Ka, Kb;                    // row strides of Ua / Ub
    int GL, GV, lpn;               // lane grid of one nonzero group: GL x GV lanes, lpn = GL*GV
    const int32_t *ia, *ib, *ic;   // other-mode index streams (ascending m != n)
    const float *Ua, *Ub, *Uc;
    const float *Un;
    const float *vals;
    const int64_t *row_ptr;
    const int32_t *row_id;
    const int64_t *chunk_start;
    const int32_t *chunk_row;
    int64_t nchunks;
    int Cbuf;                      // elements per staged array (C + 4)
    int warps;                     // warps per CTA
    int gs_off, w_off, w_stride;   // shared memory layout (floats): Gs, first warp, per-warp stride
    const float *Gn;               // [Kn][Pm]
    float *A;
    float *apart;
    float *cpart;                  // [grid][Kn*Pm]
    int32_t *err;
};

template <int TN>
__device__ __forceinline__ void ldg_vec(float (&d)[TN], const float *p) {
#pragma unroll
    for (int q = 0; q < TN / 4; ++q) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p) + q);
        d[4 * q + 0] = t.x;
        d[4 * q + 1] = t.y;
        d[4 * q + 2] = t.z;
        d[4 * q + 3] = t.w;
    }
}

// NM1 = N - 1 in {2, 3}.  For NM1 = 2, y = sum (x u_a) (x) u_b: z-rows from Ua,
// v-rows from Ub.  For NM1 = 3, y = sum (x u_a(ka) u_b) (x) u_c over the tile's
// single ka: scalar from Ua, z-rows from Ub, v-rows from Uc.
template <int NM1, int TL, int TV, bool CORE>
__global__ void __launch_bounds__(256) k_pass_fast(FastArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *smf = reinterpret_cast<float *>(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);  // 2 per warp, at the start
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int lpn = a.lpn;
    const int NG = 32 / lpn;
    const int g = lane / lpn;
    const int sub = lane - g * lpn;
    const int gl = sub / a.GV;
    const int gv = sub - gl * a.GV;
    const int l0 = gl * TL;  // first y row of the lane's tile
    const int v0 = gv * TV;  // first y column
    int ka = 0, kb0 = l0;
    if (NM1 == 3) {
        ka = l0 / a.Kb;
        kb0 = l0 - ka * a.Kb;
    }
    const int KnPm = a.Kn * a.Pm;
    const float *Gs = smf + a.gs_off;
    float *wbase = smf + a.w_off + (size_t)w * a.w_stride;
    constexpr int NARR = NM1 + 1;
    float *acc = wbase + 2 * NARR * a.Cbuf;  // core accumulator [Kn][Pm] (CORE only)
    uint64_t *bar = bars + 2 * w;

    if (threadIdx.x == 0)
        for (int q = 0; q < 2 * a.warps; ++q) mbar_init(bars + q, 1);
    if (!CORE)
        for (int p = threadIdx.x; p < KnPm; p += blockDim.x) smf[a.gs_off + p] = a.Gn[p];
    if (CORE)
        for (int p = lane; p < KnPm; p += 32) acc[p] = 0.f;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();

    const int64_t gw = (int64_t)blockIdx.x * a.warps + w;
    const int64_t nw = (int64_t)gridDim.x * a.warps;

    auto issue = [&](int64_t ch, int buf) {
        if (lane == 0) {
            const int64_t s0 = a.chunk_start[ch], s1 = a.chunk_start[ch + 1];
            const int64_t al = s0 & ~(int64_t)3;
            const uint32_t n4 = (uint32_t)(((s1 - al) + 3) & ~(int64_t)3);
            const uint32_t bytes = n4 * 4u;
            float *dst = wbase + (size_t)buf * NARR * a.Cbuf;
            fence_proxy_async();
            mbar_expect_tx(bar + buf, bytes * NARR);
            bulk_g2s(dst, a.ia + al, bytes, bar + buf);
            bulk_g2s(dst + a.Cbuf, a.ib + al, bytes, bar + buf);
            if (NM1 == 3) bulk_g2s(dst + 2 * a.Cbuf, a.ic + al, bytes, bar + buf);
            bulk_g2s(dst + (NARR - 1) * a.Cbuf, a.vals + al, bytes, bar + buf);
        }
    };

    bool ok = true;
    int it = 0;
    if (gw < a.nchunks) issue(gw, 0);
    for (int64_t ch = gw; ch < a.nchunks; ch += nw, ++it) {
        const int buf = it & 1;
        if (ch + nw < a.nchunks) issue(ch + nw, buf ^ 1);
        if (!mbar_wait(bar + buf, (uint32_t)((it >> 1) & 1), a.err)) {
            ok = false;
            break;
        }
        const int64_t s0 = a.chunk_start[ch], s1 = a.chunk_start[ch + 1];
        const int off = (int)(s0 & 3);
        const float *mb = wbase + (size_t)buf * NARR * a.Cbuf;
        const int32_t *mia = reinterpret_cast<const int32_t *>(mb) + off;
        const int32_t *mib = reinterpret_cast<const int32_t *>(mb + a.Cbuf) + off;
        const int32_t *mic = reinterpret_cast<const int32_t *>(mb + 2 * a.Cbuf) + off;
        const float *mval = mb + (NARR - 1) * a.Cbuf + off;

        auto load_nz = [&](int q, float (&z)[TL], float (&v)[TV]) {
            const float x = mval[q];
            if (NM1 == 2) {
                ldg_vec<TL>(z, a.Ua + (int64_t)mia[q] * a.Ka + l0);
                ldg_vec<TV>(v, a.Ub + (int64_t)mib[q] * a.Kl + v0);
#pragma unroll
                for (int j = 0; j < TL; ++j) z[j] *= x;
            } else {
                const float s = x * __ldg(a.Ua + (int64_t)mia[q] * a.Ka + ka);
                ldg_vec<TL>(z, a.Ub + (int64_t)mib[q] * a.Kb + kb0);
                ldg_vec<TV>(v, a.Uc + (int64_t)mic[q] * a.Kl + v0);
#pragma unroll
                for (int j = 0; j < TL; ++j) z[j] *= s;
            }
        };

        int32_t rr = a.chunk_row[ch];
        int64_t pos = s0;
        while (pos < s1) {
            const int64_t rs = a.row_ptr[rr], re = a.row_ptr[rr + 1];
            const int64_t a1 = min(re, s1);
            if (a1 <= pos) break;  // row descriptors always advance; never spin on bad input
            float y[TL][TV];
#pragma unroll
            for (int j = 0; j < TL; ++j)
#pragma unroll
                for (int k = 0; k < TV; ++k) y[j][k] = 0.f;
            const int qe = (int)(a1 - s0);
            int q = (int)(pos - s0) + g;
            float z0[TL], w0[TV], z1[TL], w1[TV];
            if (q < qe) load_nz(q, z0, w0);
            while (q < qe) {
                int qn = q + NG;
                if (qn < qe) load_nz(qn, z1, w1);
#pragma unroll
                for (int j = 0; j < TL; ++j)
#pragma unroll
                    for (int k = 0; k < TV; ++k) y[j][k] = fmaf(z0[j], w0[k], y[j][k]);
                q = qn;
                if (q >= qe) break;
                qn = q + NG;
                if (qn < qe) load_nz(qn, z0, w0);
#pragma unroll
                for (int j = 0; j < TL; ++j)
#pragma unroll
                    for (int k = 0; k < TV; ++k) y[j][k] = fmaf(z1[j], w1[k], y[j][k]);
                q = qn;
            }
            __syncwarp();
            // sum the groups' partial y (every lane then holds its tile of the full y_i)
            for (int o = lpn; o < 32; o <<= 1) {
#pragma unroll
                for (int j = 0; j < TL; ++j)
#pragma unroll
                    for (int k = 0; k < TV; ++k) y[j][k] += __shfl_xor_sync(0xffffffffu, y[j][k], o);
            }
            const int32_t row = a.row_id[rr];
            if (CORE) {
                // acc[kn][e] += U_n(row, kn) * y[e]; group g owns kn = g, g + NG, ...
                for (int kn = g; kn < a.Kn; kn += NG) {
                    const float u = __ldg(a.Un + (int64_t)row * a.Kn + kn);
#pragma unroll
                    for (int j = 0; j < TL; ++j) {
                        float4 *ap = reinterpret_cast<float4 *>(acc + (size_t)kn * a.Pm + (size_t)(l0 + j) * a.Kl + v0);
#pragma unroll
                        for (int k4 = 0; k4 < TV / 4; ++k4) {
                            float4 t = ap[k4];
                            t.x = fmaf(u, y[j][4 * k4 + 0], t.x);
                            t.y = fmaf(u, y[j][4 * k4 + 1], t.y);
                            t.z = fmaf(u, y[j][4 * k4 + 2], t.z);
                            t.w = fmaf(u, y[j][4 * k4 + 3], t.w);
                            ap[k4] = t;
                        }
                    }
                }
            } else {
                const bool full = (rs >= s0) && (re <= s1);
                float *dst = full ? a.A + (int64_t)row * a.Kn : a.apart + ch * a.Kn;
                const int rounds = (a.Kn + NG - 1) / NG;
                for (int t = 0; t < rounds; ++t) {
                    const int kn = t * NG + g;
                    float s = 0.f;
                    if (kn < a.Kn) {
#pragma unroll
                        for (int j = 0; j < TL; ++j) {
                            const float4 *gp =
                                reinterpret_cast<const float4 *>(Gs + (size_t)kn * a.Pm + (size_t)(l0 + j) * a.Kl + v0);
#pragma unroll
                            for (int k4 = 0; k4 < TV / 4; ++k4) {
                                const float4 gq = gp[k4];
                                s = fmaf(gq.x, y[j][4 * k4 + 0], s);
                                s = fmaf(gq.y, y[j][4 * k4 + 1], s);
                                s = fmaf(gq.z, y[j][4 * k4 + 2], s);
                                s = fmaf(gq.w, y[j][4 * k4 + 3], s);
                            }
                        }
                    }
                    for (int o = 1; o < lpn; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    if (sub == 0 && kn < a.Kn) dst[kn] = s;
                }
            }
            pos = a1;
            ++rr;
        }
        __syncwarp();
    }
    if (!ok) {
        // a staged copy never completed: wait (bounded) for the other buffer, then leave
        mbar_wait(bar + ((it + 1) & 1), (uint32_t)(((it + 1) >> 1) & 1), nullptr);
    }
    if (CORE) {
        __syncthreads();
        for (int p = threadIdx.x; p < KnPm; p += blockDim.x) {
            float s = 0.f;
            for (int q = 0; q < a.warps; ++q) s += smf[a.w_off + (size_t)q * a.w_stride + 2 * NARR * a.Cbuf + p];
            a.cpart[(size_t)blockIdx.x * KnPm + p] = s;
        }
    }
}

// ------------------------------------------------------------------ fix-up

// A(row, :) of every row longer than C = sum of its pieces' slots, in chunk order.
template <typename T>
__global__ void __launch_bounds__(128) k_fixup(const int32_t *big, const int32_t *row_id, const T *apart, int Kn,
                                               T *A) {
    __shared__ double sh[128];
    const int b = blockIdx.x;
    const int32_t r = big[3 * b], c0 = big[3 * b + 1], c1 = big[3 * b + 2];
    for (int kn = 0; kn < Kn; ++kn) {
        double s = 0.0;
        for (int c = c0 + (int)threadIdx.x; c <= c1; c += blockDim.x) s += (double)apart[(int64_t)c * Kn + kn];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int o = 64; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) A[(int64_t)row_id[r] * Kn + kn] = (T)sh[0];
        __syncthreads();
    }
}

// Entries of the unfolding G_(n) as [Kn][Pm] (the partial and unfolded layouts)
// against the row-major core.  The sliced pass of a padded plan works on columns
// over the padded ranks KoP (PmP columns); columns with a padded index are not
// entries of G (their sums are zero).
struct CoreMap {
    int nm1, Kn, Pm, PmP;
    int Ko[HOQRI_MAXN - 1], KoP[HOQRI_MAXN - 1];
    int64_t gso[HOQRI_MAXN - 1];
    int64_t gsn;
};

// row-major index of unfolded entry p (over the padded columns), -1 for a padded column
__device__ __forceinline__ int64_t rowmajor_of(const CoreMap &m, int p) {
    int kn = p / m.PmP;
    int e = p - kn * m.PmP;
    int64_t g = (int64_t)kn * m.gsn;
    for (int j = m.nm1 - 1; j >= 0; --j) {
        int k = e % m.KoP[j];
        e /= m.KoP[j];
        if (k >= m.Ko[j]) return -1;
        g += (int64_t)k * m.gso[j];
    }
    return g;
}

// G (row-major) = sum over CTAs of the [Kn][Pm] partials, in CTA order; block
// partial sums of ||G||^2.
// Each block owns 32 consecutive entries p; its 8 warps sum the partials
// b = w, w + 8, ... of those entries (lane = entry), then warp 0 adds the 8
// warp sums in warp order.  The order of every sum is fixed.
template <typename T>
__global__ void __launch_bounds__(RED_TPB) k_core_reduce(const T *cpart, int nblk, CoreMap m, T *G, double *gpart) {
    __shared__ double sh[RED_TPB / 32][33];
    const int P = m.Kn * m.PmP;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = RED_TPB / 32;
    const int p = blockIdx.x * 32 + lane;
    double s = 0.0;
    if (p < P) {
        // eight loads in flight, added in the same order (b = w, w + nw, ...)
        int b = w;
        for (; b + 7 * nw < nblk; b += 8 * nw) {
            T x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = cpart[(size_t)(b + u * nw) * P + p];
#pragma unroll
            for (int u = 0; u < 8; ++u) s += (double)x[u];
        }
        for (; b < nblk; b += nw) s += (double)cpart[(size_t)b * P + p];
    }
    sh[w][lane] = s;
    __syncthreads();
    if (w == 0) {
        double t = 0.0;
        for (int q = 0; q < nw; ++q) t += sh[q][lane];
        double sq = 0.0;
        const int64_t g = p < P ? rowmajor_of(m, p) : -1;
        if (g >= 0) {
            G[g] = (T)t;
            sq = t * t;  // the FP64 sum, before the entry is rounded to T
        }
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (lane == 0) gpart[blockIdx.x] = sq;
    }
}

// out = sum of part[0..n) by one warp: lane-strided sums, then a fixed butterfly
__global__ void k_sum_into(const double *part, int n, double *out, double *out2) {
    const int lane = threadIdx.x & 31;
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += part[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        *out = s;
        if (out2) *out2 = s;
    }
}

// Gn[kn][e] = G(row-major) for the TTMcTC pass
template <typename T>
__global__ void k_core_to_unfolded(const T *G, CoreMap m, T *Gn) {
    const int P = m.Kn * m.PmP;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const int64_t g = rowmajor_of(m, p);
        Gn[p] = g >= 0 ? G[g] : T(0);
    }
}

// ------------------------------------------------------------ host side

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
        m.KoP[j] = c->K[q];
        m.gso[j] = st[q];
        m.Pm *= c->K[q];
        ++j;
    }
    m.PmP = m.Pm;
    return m;
}

// the map of the sliced pass of mode n: over padded columns when its plan is padded
CoreMap core_map_hyb(hoqri_ctx *c, int n) {
    CoreMap m = core_map(c, n);
    FastTile p;
    if (hyb_tile(c, n, &p) && p.pad) {
        m.PmP = 1;
        for (int j = 0; j < m.nm1; ++j) {
            m.KoP[j] = padded_rank(m.Ko[j]);
            m.PmP *= m.KoP[j];
        }
    }
    return m;
}

int pl_for(int Pm) {
    int pl = 1;
    while (32 * pl < Pm) pl <<= 1;
    return pl;
}

// columns of Y_(n) per launch of the generic pass: all of them up to 2048,
// else the largest multiple of K_l (the last other mode's rank) not above 2048
int gen_block(int Pm, int Kl) { return Pm <= 2048 ? Pm : (2048 / Kl) * Kl; }

// columns per launch of the generic core pass: as gen_block, but narrower where
// the warps' K_n x Pb accumulators would not fit in shared memory (a multiple of
// K_l), so the accumulators never live in global memory: a row's rank-1 update
// of the core is K_n x P_{-n} read-modify-writes, far too many for global memory
int gen_block_core(int Pm, int Kl, int Kn, int rtot, size_t rsize) {
    int Pb = gen_block(Pm, Kl);
    auto fits = [&](int pb) {
        return (size_t)GEN_WARPS * (size_t)(rtot + pb / Kl + Kn * pb + 3) * rsize <= SMEM_CAP;
    };
    while (Pb > Kl && !fits(Pb)) Pb = std::max(Kl, ((Pb / 2) / Kl) * Kl);
    return Pb;
}

// ---- fast-path plan for mode n

bool pow2_ge4(int k) { return k >= 4 && k <= 64 && (k & (k - 1)) == 0; }

// register-tile plan from the ranks of the other modes (powers of two >= 4)
FastTile plan_of(int N, const int (&Ko)[3]) {
    FastTile p;
    for (int q = 0; q < N - 1; ++q)
        if (!pow2_ge4(Ko[q])) return p;
    p.nm1 = N - 1;
    p.Kl = Ko[p.nm1 - 1];
    p.TV = std::min(8, p.Kl);
    p.GV = p.Kl / p.TV;
    int L;
    if (p.nm1 == 2) {
        p.Ka = Ko[0];
        L = Ko[0];
        p.TL = std::min(8, L);
    } else {
        p.Ka = Ko[0];
        p.Kb = Ko[1];
        L = Ko[0] * Ko[1];
        p.TL = std::min(8, Ko[1]);
    }
    p.GL = L / p.TL;
    p.lpn = p.GL * p.GV;
    p.Pm = L * p.Kl;
    if (p.lpn > 32) return p;
    p.ok = true;
    return p;
}

FastTile fast_plan(const hoqri_ctx *c, int n) {
    FastTile p;
    if (c->prec != HOQRI_FP32 || (c->N != 3 && c->N != 4)) return p;
    int Ko[3] = {0, 0, 0}, j = 0;
    for (int m = 0; m < c->N; ++m)
        if (m != n) Ko[j++] = c->K[m];
    return plan_of(c->N, Ko);
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
    a.chunk_start = M.chunk_start;
    a.chunk_row = M.chunk_row;
    a.nchunks = M.nchunks;
}

template <typename T, bool CORE>
hoqri_status launch_generic(hoqri_ctx *c, PassArgs<T> &a, int grid, size_t smem, int Pblk) {
    // one launch per column block of Pblk columns (in block order: the TTMcTC pass adds into A)
    for (int e0 = 0; e0 < a.Pm; e0 += Pblk) {
        a.e0 = e0;
        a.Pb = std::min(Pblk, a.Pm - e0);
        a.q0 = e0 / a.Kl;
        a.Lb = a.Pb / a.Kl;
        a.accum = e0 > 0;
        const int pl = pl_for(a.Pb);
#define HQ_GEN(PLV)                                                                                   \
    case PLV: {                                                                                       \
        auto kern = k_pass_generic<T, PLV, CORE>;                                                     \
        HQ_CUDA(smem_limit(kern, smem)); \
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
                set_error("generic pass: column block above 2048 (internal)");
                return HOQRI_ERR_UNSUPPORTED;
        }
#undef HQ_GEN
    }
    HQ_CUDA(cudaGetLastError());
    return HOQRI_OK;
}

// fast kernel configuration: warps per CTA and shared memory bytes
struct FastLaunch {
    int warps = 0;
    size_t smem = 0;
    int gs_off = 0, w_off = 0, w_stride = 0;
};

FastLaunch fast_launch(const hoqri_ctx *c, int n, const FastTile &p, bool core) {
    FastLaunch L;
    const int Kn = c->K[n];
    const int KnPm = Kn * p.Pm;
    const int Cbuf = c->ms[n].C + 4;
    const int narr = p.nm1 + 1;
    L.warps = core ? 4 : 8;
    // floats: [mbarriers: 2 per warp, padded to 32 floats] [Gs (TTMcTC)] [per warp: 2 x narr x Cbuf (+ acc)]
    L.gs_off = 32;
    int gs = core ? 0 : ((KnPm + 31) & ~31);
    L.w_off = L.gs_off + gs;
    L.w_stride = ((2 * narr * Cbuf + (core ? KnPm : 0)) + 31) & ~31;
    L.smem = (size_t)(L.w_off + L.warps * L.w_stride) * sizeof(float);
    return L;
}

// Grid = resident CTAs (SMs x CTAs per SM from the occupancy calculator),
// capped by the number of warp tasks; it depends only on the device, kernel
// and shape, so a context always uses the same grid (fixed summation order).
template <int NM1, bool CORE>
hoqri_status launch_fast_nm1(hoqri_ctx *c, const FastTile &p, FastArgs &a, const FastLaunch &L, int *grid) {
#define HQ_FAST(TLV, TVV)                                                                                  \
    if (p.TL == TLV && p.TV == TVV) {                                                                      \
        auto kern = k_pass_fast<NM1, TLV, TVV, CORE>;                                                      \
        HQ_CUDA(smem_limit(kern, L.smem));    \
        int per_sm = 0;                                                                                    \
        HQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, L.warps * 32, L.smem));      \
        per_sm = std::max(1, std::min(per_sm, FAST_MAX_CTAS_PER_SM));                                      \
        *grid = (int)std::max<int64_t>(                                                                    \
            1, std::min<int64_t>((int64_t)c->num_sms * per_sm, ceil_div(std::max<int64_t>(a.nchunks, 1), L.warps))); \
        kern<<<*grid, L.warps * 32, L.smem, c->stream>>>(a);                                               \
        c->nlaunch++;                                                                                      \
        HQ_CUDA(cudaGetLastError());                                                                       \
        return HOQRI_OK;                                                                                   \
    }
    HQ_FAST(8, 8)
    HQ_FAST(8, 4)
    HQ_FAST(4, 8)
    HQ_FAST(4, 4)
#undef HQ_FAST
    set_error("fast pass: no kernel for this tile");
    return HOQRI_ERR_UNSUPPORTED;
}

template <bool CORE>
hoqri_status launch_fast(hoqri_ctx *c, int n, const FastTile &p, const float *Gn, float *A_out, int *grid) {
    const ModeStore &M = c->ms[n];
    FastArgs a{};
    a.Kn = c->K[n];
    a.Pm = p.Pm;
    a.Kl = p.Kl;
    a.Ka = p.Ka;
    a.Kb = p.Kb;
    a.GL = p.GL;
    a.GV = p.GV;
    a.lpn = p.lpn;
    const float *Uo[3] = {nullptr, nullptr, nullptr};
    int j = 0;
    for (int m = 0; m < c->N; ++m)
        if (m != n) Uo[j++] = (const float *)c->U[m];
    a.ia = M.oidx[0];
    a.ib = M.oidx[1];
    a.ic = p.nm1 == 3 ? M.oidx[2] : nullptr;
    a.Ua = Uo[0];
    a.Ub = Uo[1];
    a.Uc = Uo[2];
    a.Un = (const float *)c->U[n];
    a.vals = (const float *)M.vals;
    a.row_ptr = M.row_ptr;
    a.row_id = M.row_id;
    a.chunk_start = M.chunk_start;
    a.chunk_row = M.chunk_row;
    a.nchunks = M.nchunks;
    a.Cbuf = M.C + 4;
    FastLaunch L = fast_launch(c, n, p, CORE);
    a.warps = L.warps;
    a.gs_off = L.gs_off;
    a.w_off = L.w_off;
    a.w_stride = L.w_stride;
    a.Gn = Gn;
    a.A = A_out;
    a.apart = (float *)c->a_part;
    a.cpart = (float *)c->core_part;
    a.err = c->dflag + 2;
    if (p.nm1 == 2) return launch_fast_nm1<2, CORE>(c, p, a, L, grid);
    return launch_fast_nm1<3, CORE>(c, p, a, L, grid);
}

bool use_fast(const hoqri_ctx *c, int n, bool core, FastTile *out) {
    FastTile p = fast_plan(c, n);
    if (!p.ok || c->ms[n].C % 4 != 0) return false;
    FastLaunch L = fast_launch(c, n, p, core);
    if (L.smem > SMEM_CAP) return false;
    *out = p;
    return true;
}

template <typename T>
hoqri_status core_pass_t(hoqri_ctx *c, int n, void *G_out, double *normG2_slot) {
    PassArgs<T> a{};
    fill_common<T>(c, n, a);
    const int KnPm = a.Kn * a.Pm;
    int grid = c->core_grid;
    FastTile fp;
    if (std::is_same<T, float>::value && use_fast(c, n, true, &fp)) {
        HQ_TRY(launch_fast<true>(c, n, fp, nullptr, nullptr, &grid));
    } else {
        const int Pb = gen_block_core(a.Pm, a.Kl, a.Kn, a.rtot, sizeof(T)), Lb = Pb / a.Kl;
        a.wstride = (a.rtot + Lb + a.Kn * Pb + 3) & ~3;
        size_t smem = (size_t)GEN_WARPS * a.wstride * sizeof(T);
        a.acc_in_smem = smem <= SMEM_CAP;
        if (!a.acc_in_smem) {
            a.wstride = (a.rtot + Lb + 3) & ~3;
            smem = (size_t)GEN_WARPS * a.wstride * sizeof(T);
        }
        a.acc_glob = (T *)c->a_part;  // only used when the accumulator does not fit in smem
        a.cpart = (T *)c->core_part;
        if (!a.acc_in_smem && (int64_t)grid * GEN_WARPS * a.Kn * Pb * (int64_t)sizeof(T) > c->a_part_bytes) {
            set_error("core pass: accumulator workspace too small");
            return HOQRI_ERR_UNSUPPORTED;
        }
        HQ_TRY((launch_generic<T, true>(c, a, grid, smem, Pb)));
    }
    CoreMap m = core_map(c, n);
    const int rb = (KnPm + 31) / 32;
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
    if ((int64_t)M.nchunks * a.Kn * (int64_t)sizeof(T) > c->a_part_bytes) {
        set_error("TTMcTC pass: partial-row workspace too small");
        return HOQRI_ERR_UNSUPPORTED;
    }
    FastTile fp;
    if (std::is_same<T, float>::value && use_fast(c, n, false, &fp)) {
        int grid = 0;
        HQ_TRY(launch_fast<false>(c, n, fp, (const float *)Gn, (float *)A_out, &grid));
    } else {
        a.Gn = Gn;
        a.A = (T *)A_out;
        a.apart = (T *)c->a_part;
        const int Pb = gen_block(a.Pm, a.Kl);
        a.wstride = (a.rtot + Pb / a.Kl + 3) & ~3;
        size_t smem = (size_t)GEN_WARPS * a.wstride * sizeof(T);
        a.gn_in_smem = Pb == a.Pm && (smem + (size_t)KnPm * sizeof(T)) <= SMEM_CAP;
        if (a.gn_in_smem) smem += (size_t)KnPm * sizeof(T);
        HQ_TRY((launch_generic<T, false>(c, a, c->pass_grid, smem, Pb)));
    }
    if (M.nbig > 0) {
        k_fixup<T><<<(unsigned)M.nbig, 128, 0, c->stream>>>(M.big, M.row_id, (const T *)c->a_part, a.Kn, (T *)A_out);
        c->nlaunch++;
    }
    HQ_CUDA(cudaGetLastError());
    return HOQRI_OK;
}

}  // namespace

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

int padded_rank(int K) {
    int k = 4;
    while (k < K) k <<= 1;
    return k;
}

// the plan of the sliced pass over padded ranks (FP32 storage, orders 3 and 4);
// ok only when some other rank actually needs padding
bool padded_plan(const hoqri_ctx *c, int n, FastTile *out) {
    if (c->prec != HOQRI_FP32 || (c->N != 3 && c->N != 4)) return false;
    int Ko[3] = {0, 0, 0}, j = 0;
    bool any = false;
    for (int m = 0; m < c->N; ++m)
        if (m != n) {
            Ko[j] = padded_rank(c->K[m]);
            any = any || Ko[j] != c->K[m];
            ++j;
        }
    if (!any) return false;
    FastTile p = plan_of(c->N, Ko);
    if (!p.ok) return false;
    p.pad = true;
    *out = p;
    return true;
}

bool fast_tile(const hoqri_ctx *c, int n, FastTile *out) {
    FastTile p = fast_plan(c, n);
    if (!p.ok) return false;
    *out = p;
    return true;
}

hoqri_status core_reduce(hoqri_ctx *c, int n, int nblk, void *G_out, double *normG2_slot) {
    CoreMap m = core_map_hyb(c, n);
    const int KnPm = m.Kn * m.PmP;
    const int rb = (KnPm + 31) / 32;
    if (c->prec == HOQRI_FP64)
        k_core_reduce<double><<<rb, RED_TPB, 0, c->stream>>>((const double *)c->core_part, nblk, m, (double *)G_out,
                                                              c->gnorm_part);
    else
        k_core_reduce<float><<<rb, RED_TPB, 0, c->stream>>>((const float *)c->core_part, nblk, m, (float *)G_out,
                                                            c->gnorm_part);
    k_sum_into<<<1, 32, 0, c->stream>>>(c->gnorm_part, rb, c->dnorm + 1, normG2_slot);
    c->nlaunch += 2;
    HQ_CUDA(cudaGetLastError());
    return HOQRI_OK;
}

hoqri_status unfold_core(hoqri_ctx *c, int n, const void *G, void *Gn) {
    CoreMap m = core_map_hyb(c, n);
    const int KnPm = m.Kn * m.PmP;
    const int g = std::max(1, std::min(64, (KnPm + 255) / 256));
    if (c->prec == HOQRI_FP64)
        k_core_to_unfolded<double><<<g, 256, 0, c->stream>>>((const double *)G, m, (double *)Gn);
    else
        k_core_to_unfolded<float><<<g, 256, 0, c->stream>>>((const float *)G, m, (float *)Gn);
    c->nlaunch++;
    HQ_CUDA(cudaGetLastError());
    return HOQRI_OK;
}

// Sizes the partition and the scratch buffers of the passes.
hoqri_status passes_init(hoqri_ctx *c) {
    int32_t C = c->opt.chunk_nnz;
    if (C <= 0) {
        // about 8 tasks per resident warp, within [32, 256]
        int64_t target = ceil_div(c->nnz, (int64_t)c->num_sms * 16 * 8);
        C = 32;
        while (C < target && C < 256) C <<= 1;
    }
    C = std::max<int32_t>(4, (C + 3) & ~3);
    int64_t max_chunks = 0;
    for (int n = 0; n < c->N; ++n) {
        HQ_TRY(build_partition(c, n, C));
        max_chunks = std::max(max_chunks, c->ms[n].nchunks);
    }
    const int64_t want = ceil_div(std::max<int64_t>(max_chunks, 1), GEN_WARPS);
    c->pass_grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)c->num_sms * 4));
    // the core partials hold one copy of G per CTA: at most 256 MB of them
    c->core_grid = (int)std::max<int64_t>(
        1, std::min<int64_t>(c->pass_grid, ((int64_t)256 << 20) / (c->P * (int64_t)c->rsize)));
    // the register-tiled kernels run at most FAST_MAX_CTAS_PER_SM resident CTAs per SM
    c->core_grid_fast = c->num_sms * FAST_MAX_CTAS_PER_SM;
    c->pass_grid_fast = c->core_grid_fast;
    int maxK = 1;
    for (int n = 0; n < c->N; ++n) maxK = std::max(maxK, (int)c->K[n]);
    // core partials [grid][P]; also holds G_(n) for the TTMcTC pass
    const int gmax = std::max(std::max(c->core_grid, c->core_grid_fast), 1);
    c->core_part_bytes = (int64_t)gmax * c->P * (int64_t)c->rsize;
    HQ_TRY(dalloc(c, &c->core_part, c->core_part_bytes));
    // per-chunk partial rows [nchunks][Kn], or per-warp core accumulators of the generic kernel
    int64_t ab = std::max<int64_t>(max_chunks, 1) * maxK * (int64_t)c->rsize;
    for (int n = 0; n < c->N; ++n) {
        // same test as core_pass_t: does the per-warp accumulator fit in shared memory?
        int64_t rtot = 0, Pm = 1;
        for (int m = 0; m < c->N; ++m)
            if (m != n) {
                rtot += c->K[m];
                Pm *= c->K[m];
            }
        const int64_t Kl = c->K[n == c->N - 1 ? c->N - 2 : c->N - 1];
        const int64_t Pb = gen_block_core((int)Pm, (int)Kl, c->K[n], (int)rtot, c->rsize);
        const int64_t wst = (rtot + Pb / Kl + c->K[n] * Pb + 3) & ~3LL;
        if ((int64_t)GEN_WARPS * wst * (int64_t)c->rsize > (int64_t)SMEM_CAP)
            ab = std::max(ab, (int64_t)c->core_grid * GEN_WARPS * c->K[n] * Pb * (int64_t)c->rsize);
    }
    // hybrid layout + dense Y for the FP32 modes with a register-tile plan
    int64_t ybytes = 0, ypb = 0;
    // ~16 work items per resident warp (8 warps per SM) for balance across SMs
    const int64_t Tt = std::max<int64_t>(256, std::min<int64_t>(16384, ceil_div(c->nnz, (int64_t)c->num_sms * 128)));
    const int64_t T32 = (Tt + 31) & ~(int64_t)31;
    int64_t fpb = 0, core_pad = 0, gn_pad = 0;
    for (int n = 0; n < c->N; ++n) {
        if (c->opt.one_stream == 2) continue;
        if (c->opt.one_stream == 3 && fib_shape(c, n, nullptr)) {
            // fiber-factored pass: the mode-n sorted stream plus piece descriptors
            HQ_TRY(build_fiber(c, n));
            ybytes = std::max<int64_t>(ybytes, c->ms[n].R * (c->P / c->K[n]) * 4);
            fpb = std::max<int64_t>(fpb, fib_part_bytes(c, n));
            continue;
        }
        FastTile p;
        if (!hyb_tile(c, n, &p)) continue;
        if (hyb_smem_need(c, n) > hyb_smem_cap()) continue;
        HQ_TRY(build_hybrid(c, n, 256, T32, 32 / p.lpn));
        const ModeStore &M = c->ms[n];
        ab = std::max<int64_t>(ab, std::max<int64_t>(M.nitem_long, 1) * 2 * c->K[n] * (int64_t)c->rsize);
        ybytes = std::max<int64_t>(ybytes, M.R * (int64_t)p.Pm * 4);
        // partials of G_(n) over padded columns (k_core_from_y*: at most 2 CTAs per SM)
        core_pad = std::max<int64_t>(core_pad, (int64_t)2 * c->num_sms * c->K[n] * p.Pm * 4);
        gn_pad = std::max<int64_t>(gn_pad, (int64_t)c->K[n] * p.Pm);
        if (p.pad)
            for (int m = 0; m < c->N; ++m)
                if (m != n && padded_rank(c->K[m]) != c->K[m] && !c->Upad[m])
                    HQ_TRY(dalloc(c, (void **)&c->Upad[m], (size_t)c->dims[m] * padded_rank(c->K[m]) * sizeof(float)));
        // pieces of rows cut by warp ranges: at most one range per warp of the pass
        // (any layout the autotuner may build)
        ypb = std::max<int64_t>(ypb, (int64_t)c->num_sms * HY_BLOCKS_PER_SM * 8 * 2 * (int64_t)p.Pm * 4);
    }
    c->a_part_bytes = ab;
    HQ_TRY(dalloc(c, &c->a_part, c->a_part_bytes));
    const int64_t ybudget = (int64_t)8 << 30;
    if (ybytes > 0 && c->opt.one_stream != 2 && ybytes <= ybudget) {
        HQ_TRY(dalloc(c, (void **)&c->Y, ybytes));
        c->Y_bytes = ybytes;
        HQ_TRY(dalloc(c, (void **)&c->ypart, std::max<int64_t>(ypb, 16)));
        c->ypart_bytes = ypb;
        if (fpb > 0) {
            HQ_TRY(dalloc(c, (void **)&c->fpart, fpb));
            c->fpart_bytes = fpb;
        }
    } else {
        // no Y buffer: the modes fall back to the two-pass kernels
        for (int n = 0; n < c->N; ++n)
            if (c->ms[n].fib) free_fiber(c, n);
    }
    if (core_pad > c->core_part_bytes) {
        // the sliced pass of a padded plan writes wider partials than the two-pass core
        dfree(c->core_part, c->stream);
        c->device_bytes -= c->core_part_bytes;
        c->core_part_bytes = core_pad;
        HQ_TRY(dalloc(c, &c->core_part, c->core_part_bytes));
    }
    HQ_TRY(dalloc(c, (void **)&c->gnorm_part, ((std::max<int64_t>(c->P, gn_pad) + 31) / 32 + 1) * sizeof(double)));
    HQ_TRY(dalloc(c, (void **)&c->claim, sizeof(unsigned long long)));
    if (c->mix && c->Y) {
        int64_t sb = 0;
        for (int m = 0; m < c->N; ++m) sb = std::max<int64_t>(sb, c->dims[m] * padded_rank(c->K[m]) * 4);
        HQ_TRY(dalloc(c, &c->usplit, sb));
    }
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
