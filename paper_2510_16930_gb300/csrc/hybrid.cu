// One-stream-per-mode TTMcTC for FP32 on the hybrid layout.
//
// For mode n the pass forms every row y_i of Y_(n) = (X x_{-n} {U^T})_(n) once
// (Eq. ttmctc, Y is "the mode-n matricization of X x_{-n} {U^T}"), writes
//   A_n(i, :) = G_(n) y_i      (the TTMcTC output, Eq. ttmctc)
// and stores y_i in a dense R_n x P_{-n} buffer.  After the QR of A_n the core
// for the next block update is the dense product
//   G_(n) = U_n^T Y_(n)        (G = X x {U^T}, Sec. 2.2; Alg. 3 first step)
// so each block update streams the nonzeros once instead of twice.  Storing Y
// is the memory of Table 2's MET/TTMc row (R_n * P_{-n} words for the current
// mode only); the paper's O(IK) variant (two streams, no Y) is the fallback
// when Y does not fit the budget.
//
// Layout (built by build_hybrid): long rows contiguous, short rows in slices of
// SW rows (SW = number of lane groups of the warp), element (step s, row g) of
// a slice at sbase + SW*s + g.
//  - Long tasks: the warp's lane groups split a row's nonzeros (group g takes
//    every SW-th one); partial tiles are added with warp shuffles at the row
//    end; y carries across staging windows; a row cut by a task boundary writes
//    its pieces to per-task slots that k_span_fix adds in task order.
//  - Slice tasks: lane group g owns row g of the slice, so no cross-group sum
//    is needed; padding entries have value 0 and gather row 0.
// Each window of the index/value streams (HY_W elements) is staged in shared
// memory by TMA bulk copies completing on an mbarrier, double buffered across
// the warp's windows; all waits are bounded.
#include <algorithm>

#include "internal.cuh"

namespace hoqri {

namespace {

constexpr int HY_WARPS = 8;
constexpr int HY_W = 512;           // staged elements per window (multiple of 32)
constexpr int HY_WB = HY_W + 8;     // floats per staged array
constexpr size_t HY_SMEM_CAP = 200 * 1024;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int32_t *err) {
    const uint32_t a = smem_addr(bar);
    for (int it = 0; it < (1 << 24); ++it) {
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

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

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

struct HybArgs {
    int Kn, Pm, Kl, Ka, Kb, GV, lpn;
    const int32_t *ia, *ib, *ic;
    const float *Ua, *Ub, *Uc;
    const float *vals;
    const int32_t *row_id;
    const int64_t *lrp;
    const int32_t *lrow;
    const int64_t *sbase;
    const int32_t *srow;
    const int64_t *item_s, *item_e;
    const int32_t *item_aux;
    int64_t nitem, nitem_long;
    int warps, gs_off, w_off, w_stride;
    const float *Gn;  // [Kn][Pm]
    float *A;
    float *Y;
    float *apart;  // [nitem_long][2][Kn]
    float *ypart;  // [nitem_long][2][Pm]
    int32_t *err;
};

template <int NM1, int TL, int TV, bool WA, bool WY>
__global__ void __launch_bounds__(HY_WARPS * 32) k_hyb(HybArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *smf = reinterpret_cast<float *>(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int lpn = a.lpn;
    const int NG = 32 / lpn;  // lane groups = rows per slice
    const int g = lane / lpn;
    const int sub = lane - g * lpn;
    const int gl = sub / a.GV;
    const int gv = sub - gl * a.GV;
    const int l0 = gl * TL;
    const int v0 = gv * TV;
    int ka = 0, kb0 = l0;
    if (NM1 == 3) {
        ka = l0 / a.Kb;
        kb0 = l0 - ka * a.Kb;
    }
    const int KnPm = a.Kn * a.Pm;
    const float *Gs = smf + a.gs_off;
    float *wbase = smf + a.w_off + (size_t)w * a.w_stride;
    constexpr int NARR = NM1 + 1;
    uint64_t *bar = bars + 2 * w;

    if (threadIdx.x == 0)
        for (int q = 0; q < 2 * a.warps; ++q) mbar_init(bars + q, 1);
    if (WA)
        for (int p = threadIdx.x; p < KnPm; p += blockDim.x) smf[a.gs_off + p] = a.Gn[p];
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();

    const int64_t gw = (int64_t)blockIdx.x * a.warps + w;
    const int64_t nw = (int64_t)gridDim.x * a.warps;

    auto issue = [&](int64_t p0, int64_t p1, int buf) {
        if (lane == 0) {
            const uint32_t n4 = (uint32_t)(((p1 - p0) + 3) & ~(int64_t)3);
            const uint32_t bytes = n4 * 4u;
            float *dst = wbase + (size_t)buf * NARR * HY_WB;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(bar + buf, bytes * NARR);
            bulk_g2s(dst, a.ia + p0, bytes, bar + buf);
            bulk_g2s(dst + HY_WB, a.ib + p0, bytes, bar + buf);
            if (NM1 == 3) bulk_g2s(dst + 2 * HY_WB, a.ic + p0, bytes, bar + buf);
            bulk_g2s(dst + (NARR - 1) * HY_WB, a.vals + p0, bytes, bar + buf);
        }
    };

    float y[TL][TV];
    auto zero_y = [&]() {
#pragma unroll
        for (int j = 0; j < TL; ++j)
#pragma unroll
            for (int k = 0; k < TV; ++k) y[j][k] = 0.f;
    };

    // write this lane's tile of y to dst (a P_{-n} vector)
    auto store_tile = [&](float *dst) {
#pragma unroll
        for (int j = 0; j < TL; ++j) {
            float4 *p = reinterpret_cast<float4 *>(dst + (size_t)(l0 + j) * a.Kl + v0);
#pragma unroll
            for (int k4 = 0; k4 < TV / 4; ++k4)
                p[k4] = make_float4(y[j][4 * k4], y[j][4 * k4 + 1], y[j][4 * k4 + 2], y[j][4 * k4 + 3]);
        }
    };

    // partial G_(n)[kn] . y over this lane's tile
    auto dot_tile = [&](int kn) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < TL; ++j) {
            const float4 *gp = reinterpret_cast<const float4 *>(Gs + (size_t)kn * a.Pm + (size_t)(l0 + j) * a.Kl + v0);
#pragma unroll
            for (int k4 = 0; k4 < TV / 4; ++k4) {
                const float4 gq = gp[k4];
                s = fmaf(gq.x, y[j][4 * k4 + 0], s);
                s = fmaf(gq.y, y[j][4 * k4 + 1], s);
                s = fmaf(gq.z, y[j][4 * k4 + 2], s);
                s = fmaf(gq.w, y[j][4 * k4 + 3], s);
            }
        }
        return s;
    };

    bool ok = true;
    int k = 0;  // windows processed by this warp (buffer = k & 1, phase = (k >> 1) & 1)
    int64_t it = gw;
    int64_t p0 = it < a.nitem ? a.item_s[it] : 0;
    if (it < a.nitem) issue(p0, min(p0 + (int64_t)HY_W, a.item_e[it]), 0);
    int64_t j = 0;  // current long row or slice
    while (it < a.nitem) {
        const int buf = k & 1;
        const int64_t ts = a.item_s[it], te = a.item_e[it];
        const int64_t p1 = min(p0 + (int64_t)HY_W, te);
        int64_t nit = it, np0 = p0 + HY_W;
        if (np0 >= te) {
            nit = it + nw;
            np0 = nit < a.nitem ? a.item_s[nit] : 0;
        }
        if (nit < a.nitem) issue(np0, min(np0 + (int64_t)HY_W, a.item_e[nit]), buf ^ 1);
        if (!mbar_wait(bar + buf, (uint32_t)((k >> 1) & 1), a.err)) {
            ok = false;
            break;
        }
        const float *mb = wbase + (size_t)buf * NARR * HY_WB;
        const int32_t *mia = reinterpret_cast<const int32_t *>(mb);
        const int32_t *mib = reinterpret_cast<const int32_t *>(mb + HY_WB);
        const int32_t *mic = reinterpret_cast<const int32_t *>(mb + 2 * HY_WB);
        const float *mval = mb + (NARR - 1) * HY_WB;
        auto load_nz = [&](int q, float (&z)[TL], float (&v)[TV]) {
            const float x = mval[q];
            if (NM1 == 2) {
                ldg_vec<TL>(z, a.Ua + (int64_t)mia[q] * a.Ka + l0);
                ldg_vec<TV>(v, a.Ub + (int64_t)mib[q] * a.Kl + v0);
#pragma unroll
                for (int jj = 0; jj < TL; ++jj) z[jj] *= x;
            } else {
                const float sc = x * __ldg(a.Ua + (int64_t)mia[q] * a.Ka + ka);
                ldg_vec<TL>(z, a.Ub + (int64_t)mib[q] * a.Kb + kb0);
                ldg_vec<TV>(v, a.Uc + (int64_t)mic[q] * a.Kl + v0);
#pragma unroll
                for (int jj = 0; jj < TL; ++jj) z[jj] *= sc;
            }
        };
        // accumulate the window-local elements q = q0, q0 + NG, ... < qe into y
        auto accumulate = [&](int q0, int qe) {
            int q = q0;
            float z0[TL], w0[TV], z1[TL], w1[TV];
            if (q < qe) load_nz(q, z0, w0);
            while (q < qe) {
                int qn = q + NG;
                if (qn < qe) load_nz(qn, z1, w1);
#pragma unroll
                for (int jj = 0; jj < TL; ++jj)
#pragma unroll
                    for (int kk = 0; kk < TV; ++kk) y[jj][kk] = fmaf(z0[jj], w0[kk], y[jj][kk]);
                q = qn;
                if (q >= qe) break;
                qn = q + NG;
                if (qn < qe) load_nz(qn, z0, w0);
#pragma unroll
                for (int jj = 0; jj < TL; ++jj)
#pragma unroll
                    for (int kk = 0; kk < TV; ++kk) y[jj][kk] = fmaf(z1[jj], w1[kk], y[jj][kk]);
                q = qn;
            }
        };

        if (it < a.nitem_long) {
            // ---------------- long rows: groups split a row's nonzeros
            if (p0 == ts) {
                j = a.item_aux[it];
                zero_y();
            }
            int64_t pos = p0;
            while (pos < p1) {
                const int64_t rs = a.lrp[j], re = a.lrp[j + 1];
                const int64_t a1 = min(re, p1);
                if (a1 <= pos) break;  // descriptors always advance; never spin on bad input
                accumulate((int)(pos - p0) + g, (int)(a1 - p0));
                const bool row_end = (a1 == re);
                if (row_end || a1 == te) {
                    __syncwarp();
                    for (int o = lpn; o < 32; o <<= 1) {
#pragma unroll
                        for (int jj = 0; jj < TL; ++jj)
#pragma unroll
                            for (int kk = 0; kk < TV; ++kk)
                                y[jj][kk] += __shfl_xor_sync(0xffffffffu, y[jj][kk], o);
                    }
                    const int32_t r = a.lrow[j];
                    const bool full = (rs >= ts) && (re <= te);
                    const int slot = (j == a.item_aux[it]) ? 0 : 1;
                    if (WA) {
                        float *dst = full ? a.A + (int64_t)a.row_id[r] * a.Kn : a.apart + (it * 2 + slot) * a.Kn;
                        const int rounds = (a.Kn + NG - 1) / NG;
                        for (int t = 0; t < rounds; ++t) {
                            const int kn = t * NG + g;
                            float s = kn < a.Kn ? dot_tile(kn) : 0.f;
                            for (int o = 1; o < lpn; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                            if (sub == 0 && kn < a.Kn) dst[kn] = s;
                        }
                    }
                    if (WY && g == 0) store_tile(full ? a.Y + (int64_t)r * a.Pm : a.ypart + (it * 2 + slot) * a.Pm);
                    zero_y();
                    if (row_end) ++j;
                }
                pos = a1;
            }
        } else {
            // ---------------- slices: lane group g owns row g of the slice
            if (p0 == ts) {
                j = a.item_aux[it];
                zero_y();
            }
            int64_t pos = p0;
            while (pos < p1) {
                const int64_t se = a.sbase[j + 1];
                const int64_t a1 = min(se, p1);
                if (a1 <= pos) break;
                accumulate((int)(pos - p0) + g, (int)(a1 - p0));
                if (a1 == se) {
                    __syncwarp();
                    const int32_t r = a.srow[j * NG + g];
                    if (WA) {
                        const int32_t row = r >= 0 ? a.row_id[r] : 0;
                        for (int kn = 0; kn < a.Kn; ++kn) {
                            float s = dot_tile(kn);
                            for (int o = 1; o < lpn; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                            if (r >= 0 && sub == (kn & (lpn - 1))) a.A[(int64_t)row * a.Kn + kn] = s;
                        }
                    }
                    if (WY && r >= 0) store_tile(a.Y + (int64_t)r * a.Pm);
                    zero_y();
                    ++j;
                }
                pos = a1;
            }
        }
        __syncwarp();
        it = nit;
        p0 = np0;
        ++k;
    }
    if (!ok) mbar_wait(bar + ((k + 1) & 1), (uint32_t)(((k + 1) >> 1) & 1), nullptr);
}

// A and Y rows of the long rows cut by task boundaries: sum of the pieces in task order.
__global__ void __launch_bounds__(256) k_span_fix(const int32_t *span, const int32_t *lrow, const int32_t *row_id,
                                                  const int32_t *item_aux, const float *apart, const float *ypart,
                                                  int Kn, int Pm, float *A, float *Y) {
    const int b = blockIdx.x;
    const int32_t jl = span[3 * b], t0 = span[3 * b + 1], t1 = span[3 * b + 2];
    const int s0 = (item_aux[t0] == jl) ? 0 : 1;
    const int32_t r = lrow[jl];
    if (A)
        for (int kn = threadIdx.x; kn < Kn; kn += blockDim.x) {
            double s = apart[((int64_t)t0 * 2 + s0) * Kn + kn];
            for (int t = t0 + 1; t <= t1; ++t) s += apart[((int64_t)t * 2) * Kn + kn];
            A[(int64_t)row_id[r] * Kn + kn] = (float)s;
        }
    if (Y)
        for (int e = threadIdx.x; e < Pm; e += blockDim.x) {
            double s = ypart[((int64_t)t0 * 2 + s0) * Pm + e];
            for (int t = t0 + 1; t <= t1; ++t) s += ypart[((int64_t)t * 2) * Pm + e];
            Y[(int64_t)r * Pm + e] = (float)s;
        }
}

// CTA partials of G_(n)[kn][e] = sum_r U_n(row_id[r], kn) * Y[r][e] over a fixed
// row range per CTA.  Thread t owns columns e = t + 256*s (s < ES) and KC values
// of kn per round.
template <int ES, int KC>
__global__ void __launch_bounds__(256) k_core_from_y(const float *Y, const float *Un, const int32_t *row_id, int64_t R,
                                                     int Kn, int Pm, int64_t rpb, float *cpart) {
    constexpr int RB = 64;
    __shared__ float Us[RB * KC];
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = min(r0 + rpb, R);
    const int KnPm = Kn * Pm;
    for (int kc = 0; kc < Kn; kc += KC) {
        float acc[ES][KC];
#pragma unroll
        for (int s = 0; s < ES; ++s)
#pragma unroll
            for (int q = 0; q < KC; ++q) acc[s][q] = 0.f;
        for (int64_t rb = r0; rb < r1; rb += RB) {
            const int nr = (int)min((int64_t)RB, r1 - rb);
            __syncthreads();
            for (int t = threadIdx.x; t < nr * KC; t += blockDim.x) {
                const int rr = t / KC, q = t - rr * KC;
                Us[t] = (kc + q < Kn) ? Un[(int64_t)row_id[rb + rr] * Kn + kc + q] : 0.f;
            }
            __syncthreads();
            for (int rr = 0; rr < nr; ++rr) {
                const float *yr = Y + (rb + rr) * Pm;
#pragma unroll
                for (int s = 0; s < ES; ++s) {
                    const int e = threadIdx.x + 256 * s;
                    const float yv = e < Pm ? yr[e] : 0.f;
#pragma unroll
                    for (int q = 0; q < KC; ++q) acc[s][q] = fmaf(Us[rr * KC + q], yv, acc[s][q]);
                }
            }
        }
#pragma unroll
        for (int s = 0; s < ES; ++s) {
            const int e = threadIdx.x + 256 * s;
            if (e >= Pm) continue;
#pragma unroll
            for (int q = 0; q < KC; ++q)
                if (kc + q < Kn) cpart[(size_t)blockIdx.x * KnPm + (size_t)(kc + q) * Pm + e] = acc[s][q];
        }
    }
}

struct HybLaunch {
    size_t smem = 0;
    int gs_off = 0, w_off = 0, w_stride = 0;
};

HybLaunch hyb_launch(const hoqri_ctx *c, int n, const FastTile &p, bool wa) {
    HybLaunch L;
    const int KnPm = c->K[n] * p.Pm;
    const int narr = p.nm1 + 1;
    L.gs_off = 32;
    L.w_off = L.gs_off + (wa ? ((KnPm + 31) & ~31) : 0);
    L.w_stride = (2 * narr * HY_WB + 31) & ~31;
    L.smem = (size_t)(L.w_off + HY_WARPS * L.w_stride) * sizeof(float);
    return L;
}

template <int NM1, bool WA, bool WY>
hoqri_status launch_hyb_nm1(hoqri_ctx *c, const FastTile &p, HybArgs &a, const HybLaunch &L) {
#define HQ_HYB(TLV, TVV)                                                                                    \
    if (p.TL == TLV && p.TV == TVV) {                                                                       \
        auto kern = k_hyb<NM1, TLV, TVV, WA, WY>;                                                           \
        HQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));     \
        int per_sm = 0;                                                                                     \
        HQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, HY_WARPS * 32, L.smem));      \
        per_sm = std::max(1, std::min(per_sm, 4));                                                          \
        const int grid = (int)std::max<int64_t>(                                                            \
            1, std::min<int64_t>((int64_t)c->num_sms * per_sm, ceil_div(std::max<int64_t>(a.nitem, 1), HY_WARPS))); \
        kern<<<grid, HY_WARPS * 32, L.smem, c->stream>>>(a);                                                \
        c->nlaunch++;                                                                                       \
        HQ_CUDA(cudaGetLastError());                                                                        \
        return HOQRI_OK;                                                                                    \
    }
    HQ_HYB(8, 8)
    HQ_HYB(8, 4)
    HQ_HYB(4, 8)
    HQ_HYB(4, 4)
#undef HQ_HYB
    set_error("hybrid pass: no kernel for this tile");
    return HOQRI_ERR_UNSUPPORTED;
}

}  // namespace

bool hyb_mode(const hoqri_ctx *c, int n) { return c->ms[n].hyb && c->Y != nullptr; }

// The pass over mode n's hybrid stream.  Gn (unfolded core [Kn][Pm], device)
// and A_out are used when A_out != nullptr; Y is written when write_y.
hoqri_status hyb_pass(hoqri_ctx *c, int n, const float *Gn, float *A_out, bool write_y) {
    const ModeStore &M = c->ms[n];
    FastTile p;
    if (!fast_tile(c, n, &p)) {
        set_error("hybrid pass: mode has no register-tile plan");
        return HOQRI_ERR_UNSUPPORTED;
    }
    HybArgs a{};
    a.Kn = c->K[n];
    a.Pm = p.Pm;
    a.Kl = p.Kl;
    a.Ka = p.Ka;
    a.Kb = p.Kb;
    a.GV = p.GV;
    a.lpn = p.lpn;
    const float *Uo[3] = {nullptr, nullptr, nullptr};
    int j = 0;
    for (int m = 0; m < c->N; ++m)
        if (m != n) Uo[j++] = (const float *)c->U[m];
    a.ia = M.hidx[0];
    a.ib = M.hidx[1];
    a.ic = p.nm1 == 3 ? M.hidx[2] : nullptr;
    a.Ua = Uo[0];
    a.Ub = Uo[1];
    a.Uc = Uo[2];
    a.vals = (const float *)M.hvals;
    a.row_id = M.row_id;
    a.lrp = M.lrp;
    a.lrow = M.lrow;
    a.sbase = M.sbase;
    a.srow = M.srow;
    a.item_s = M.item_s;
    a.item_e = M.item_e;
    a.item_aux = M.item_aux;
    a.nitem = M.nitem;
    a.nitem_long = M.nitem_long;
    const bool wa = A_out != nullptr;
    HybLaunch L = hyb_launch(c, n, p, wa);
    a.warps = HY_WARPS;
    a.gs_off = L.gs_off;
    a.w_off = L.w_off;
    a.w_stride = L.w_stride;
    a.Gn = Gn;
    a.A = A_out;
    a.Y = c->Y;
    a.apart = (float *)c->a_part;
    a.ypart = c->ypart;
    a.err = c->dflag + 2;
    if (wa) HQ_CUDA(cudaMemsetAsync(A_out, 0, (size_t)c->dims[n] * a.Kn * sizeof(float), c->stream));
    hoqri_status s;
    if (p.nm1 == 2) {
        if (wa && write_y) s = launch_hyb_nm1<2, true, true>(c, p, a, L);
        else if (wa) s = launch_hyb_nm1<2, true, false>(c, p, a, L);
        else s = launch_hyb_nm1<2, false, true>(c, p, a, L);
    } else {
        if (wa && write_y) s = launch_hyb_nm1<3, true, true>(c, p, a, L);
        else if (wa) s = launch_hyb_nm1<3, true, false>(c, p, a, L);
        else s = launch_hyb_nm1<3, false, true>(c, p, a, L);
    }
    HQ_TRY(s);
    if (M.nspan > 0) {
        k_span_fix<<<(unsigned)M.nspan, 256, 0, c->stream>>>(M.span, M.lrow, M.row_id, M.item_aux,
                                                              (const float *)c->a_part, c->ypart, a.Kn, a.Pm,
                                                              wa ? A_out : nullptr, write_y ? c->Y : nullptr);
        c->nlaunch++;
    }
    HQ_CUDA(cudaGetLastError());
    return HOQRI_OK;
}

// G_(n) = U_n^T Y_(n) (Y written by the last hyb_pass of mode n) into CTA
// partials; returns the number of CTAs (the partial count).
hoqri_status hyb_core_partials(hoqri_ctx *c, int n, int *nblk) {
    const ModeStore &M = c->ms[n];
    const int Kn = c->K[n];
    const int Pm = (int)(c->P / Kn);
    const int64_t R = M.R;
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(R, 1), 256),
                                                          (int64_t)c->num_sms * 2));
    const int64_t rpb = ceil_div(std::max<int64_t>(R, 1), grid);
    float *cp = (float *)c->core_part;
    const float *Un = (const float *)c->U[n];
    if (Pm <= 256)
        k_core_from_y<1, 16><<<grid, 256, 0, c->stream>>>(c->Y, Un, M.row_id, R, Kn, Pm, rpb, cp);
    else if (Pm <= 512)
        k_core_from_y<2, 16><<<grid, 256, 0, c->stream>>>(c->Y, Un, M.row_id, R, Kn, Pm, rpb, cp);
    else if (Pm <= 1024)
        k_core_from_y<4, 8><<<grid, 256, 0, c->stream>>>(c->Y, Un, M.row_id, R, Kn, Pm, rpb, cp);
    else
        k_core_from_y<8, 4><<<grid, 256, 0, c->stream>>>(c->Y, Un, M.row_id, R, Kn, Pm, rpb, cp);
    c->nlaunch++;
    HQ_CUDA(cudaGetLastError());
    *nblk = grid;
    return HOQRI_OK;
}

size_t hyb_smem_need(const hoqri_ctx *c, int n, bool wa) {
    FastTile p;
    if (!fast_tile(c, n, &p)) return (size_t)-1;
    return hyb_launch(c, n, p, wa).smem;
}

size_t hyb_smem_cap() { return HY_SMEM_CAP; }

}  // namespace hoqri
