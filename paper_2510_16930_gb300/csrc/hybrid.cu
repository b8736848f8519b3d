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
#include <cuda.h>

#include <algorithm>

#include "internal.cuh"

namespace hoqri {

namespace {

constexpr int HY_WARPS = 8;
constexpr int HY_W = 256;           // staged elements per window (multiple of 32)
constexpr int HY_WB = HY_W + 8;     // floats per staged array
constexpr int HY_NB = 4;            // factor-row stages in flight per warp (32 nonzeros each), power of two
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

struct HybArgs {
    int Kn, Pm, Kl, Ka, Kb, Kc, GV, lpn;
    const int32_t *ia, *ib, *ic;
    const float *vals;
    const int32_t *row_id;
    const int64_t *lrp;
    const int32_t *lrow;
    const int64_t *sbase;
    const int32_t *srow;
    const int64_t *item_s, *item_e;
    const int32_t *item_aux;
    int64_t nitem, nitem_long;
    int64_t ipw, nrange;                   // items per warp range, number of ranges
    int bar_off, gs_off, w_off, w_stride;  // shared memory layout (bytes)
    int meta_bytes;                        // one staged array of a window (HY_WB floats)
    int ring_off, stage_bytes;             // gathered factor rows: NB stages per warp
    int stage_tx;                          // bytes the gathers of one stage deliver
    int sa, sb, sc;                        // bytes per 4-row gather slot of Ua / Ub / Uc
    int offb, offc;                        // offsets of the Ub / Uc rows inside a stage
    const float *Gn;  // [Kn][Pm]
    float *A;
    float *Y;
    float *apart;  // [nitem_long][2][Kn]
    float *ypart;  // [nitem_long][2][Pm]
    int32_t *err;
};

// 4 rows (r0..r3) of a 2-D row-major factor, full width, into shared memory.
__device__ __forceinline__ void gather4(void *dst, const CUtensorMap *tm, int r0, int r1, int r2, int r3,
                                        uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(smem_addr(bar))
        : "memory");
}

template <int NM1, int TL, int TV>
__global__ void __launch_bounds__(HY_WARPS * 32) k_hyb(const __grid_constant__ CUtensorMap tmA,
                                                       const __grid_constant__ CUtensorMap tmB,
                                                       const __grid_constant__ CUtensorMap tmC, HybArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int lpn = a.lpn;
    const int lg_lpn = __ffs(lpn) - 1;
    const int NG = 32 >> lg_lpn;  // lane groups = rows per slice = nonzeros per step
    const int lg_ng = 5 - lg_lpn;
    const int g = lane >> lg_lpn;
    const int sub = lane & (lpn - 1);
    const int gl = sub / a.GV;
    const int gv = sub - gl * a.GV;
    const int l0 = gl * TL;
    const int v0 = gv * TV;
    int ka = 0, kb0 = l0;
    if (NM1 == 3) {
        ka = l0 / a.Kb;
        kb0 = l0 - ka * a.Kb;
    }
    constexpr int NARR = NM1 + 1;
    unsigned char *wbase = smem_raw + a.w_off + (size_t)w * a.w_stride;
    unsigned char *ring = wbase + a.ring_off;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw + a.bar_off) + (size_t)w * (2 + HY_NB);
    uint64_t *sbar = mbar + 2;

    if (lane == 0)
        for (int q = 0; q < 2 + HY_NB; ++q) mbar_init(mbar + q, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();

    const int64_t gw = (int64_t)blockIdx.x * HY_WARPS + w;
    const int64_t nw = (int64_t)gridDim.x * HY_WARPS;

    // stage the index and value streams of window [p0, p1) into meta buffer `buf`
    auto issue_meta = [&](int64_t p0, int64_t p1, int buf) {
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)(((p1 - p0) + 3) & ~(int64_t)3) * 4u;
            unsigned char *dst = wbase + (size_t)buf * NARR * a.meta_bytes;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(mbar + buf, bytes * NARR);
            bulk_g2s(dst, a.ia + p0, bytes, mbar + buf);
            bulk_g2s(dst + a.meta_bytes, a.ib + p0, bytes, mbar + buf);
            if (NM1 == 3) bulk_g2s(dst + 2 * a.meta_bytes, a.ic + p0, bytes, mbar + buf);
            bulk_g2s(dst + (NARR - 1) * a.meta_bytes, a.vals + p0, bytes, mbar + buf);
        }
    };

    // y tile as column pairs: y2[j][k] holds columns (2k, 2k+1) of tile row j
    float2 y2[TL][TV / 2];
    auto zero_y = [&]() {
#pragma unroll
        for (int j = 0; j < TL; ++j)
#pragma unroll
            for (int k = 0; k < TV / 2; ++k) y2[j][k] = make_float2(0.f, 0.f);
    };
    auto store_tile = [&](float *dst) {
#pragma unroll
        for (int j = 0; j < TL; ++j) {
            float4 *p = reinterpret_cast<float4 *>(dst + (size_t)(l0 + j) * a.Kl + v0);
#pragma unroll
            for (int k4 = 0; k4 < TV / 4; ++k4)
                p[k4] = make_float4(y2[j][2 * k4].x, y2[j][2 * k4].y, y2[j][2 * k4 + 1].x, y2[j][2 * k4 + 1].y);
        }
    };
    bool ok = true;
    int mk = 0;         // meta windows consumed by this warp
    int gst = 0;        // factor-row stages consumed by this warp (wraps harmlessly)
    // work of this warp: a contiguous range of long-row items (rows carry across
    // items inside the range), then every nw-th slice item
    const int64_t rg = gw;
    const int64_t r0 = rg * a.ipw;
    const int64_t r1 = rg < a.nrange ? min(r0 + a.ipw, a.nitem_long) : r0;
    auto next_item = [&](int64_t cur) -> int64_t {
        if (cur < a.nitem_long) {
            if (cur + 1 < r1) return cur + 1;
            return a.nitem_long + gw;
        }
        return cur + nw;
    };
    const int64_t lfirst = (r0 < r1) ? a.item_aux[r0] : -1;
    const int64_t lbeg = (r0 < r1) ? a.item_s[r0] : 0;
    const int64_t lend = (r0 < r1) ? a.item_e[r1 - 1] : 0;
    int64_t it = (r0 < r1) ? r0 : a.nitem_long + gw;
    int64_t p0 = it < a.nitem ? a.item_s[it] : 0;
    if (it < a.nitem) issue_meta(p0, min(p0 + (int64_t)HY_W, a.item_e[it]), 0);
    int64_t j = 0;
    bool carry = false;  // a long row continues from the previous item of this range
    while (it < a.nitem) {
        const int mbuf = mk & 1;
        const int64_t ts = a.item_s[it], te = a.item_e[it];
        const int64_t p1 = min(p0 + (int64_t)HY_W, te);
        int64_t nit = it, np0 = p0 + HY_W;
        if (np0 >= te) {
            nit = next_item(it);
            np0 = nit < a.nitem ? a.item_s[nit] : 0;
        }
        if (nit < a.nitem) issue_meta(np0, min(np0 + (int64_t)HY_W, a.item_e[nit]), mbuf ^ 1);
        if (!mbar_wait(mbar + mbuf, (uint32_t)((mk >> 1) & 1), a.err)) {
            ok = false;
            break;
        }
        const unsigned char *mb = wbase + (size_t)mbuf * NARR * a.meta_bytes;
        const int32_t *mia = reinterpret_cast<const int32_t *>(mb);
        const int32_t *mib = reinterpret_cast<const int32_t *>(mb + a.meta_bytes);
        const int32_t *mic = reinterpret_cast<const int32_t *>(mb + 2 * a.meta_bytes);
        const float *mval = reinterpret_cast<const float *>(mb + (NARR - 1) * a.meta_bytes);
        const int len = (int)(p1 - p0);
        const int nst = (len + 31) >> 5;

        // gather the factor rows of stage s (elements 32s .. 32s+31 of the window)
        auto issue_stage = [&](int s) {
            const int slot = (gst + s) & (HY_NB - 1);
            unsigned char *st = ring + (size_t)slot * a.stage_bytes;
            __syncwarp();
            if (lane == 0) mbar_expect_tx(sbar + slot, (uint32_t)a.stage_tx);
            __syncwarp();
            if (lane < 8 * NM1) {
                const int arr = lane >> 3, gi = lane & 7;
                const int e0 = 32 * s + 4 * gi;
                const int32_t *src = arr == 0 ? mia : (arr == 1 ? mib : mic);
                int r[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) r[q] = (e0 + q < len) ? src[e0 + q] : 0;
                const CUtensorMap *tm = arr == 0 ? &tmA : (arr == 1 ? &tmB : &tmC);
                const int sz = arr == 0 ? a.sa : (arr == 1 ? a.sb : a.sc);
                const int off = arr == 0 ? 0 : (arr == 1 ? a.offb : a.offc);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                gather4(st + off + (size_t)gi * sz, tm, r[0], r[1], r[2], r[3], sbar + slot);
            }
        };
        for (int s = 0; s < nst && s < HY_NB; ++s) issue_stage(s);
        int cur = -1;  // highest stage waited for in this window
        // make stage s readable; release (re-issue) the stages before it
        auto need_stage = [&](int s) {
            while (cur < s) {
                if (cur >= 0 && cur + HY_NB < nst) issue_stage(cur + HY_NB);
                ++cur;
                const int slot = (gst + cur) & (HY_NB - 1);
                if (!mbar_wait(sbar + slot, (uint32_t)(((gst + cur) >> 2) & 1), a.err)) ok = false;
            }
        };
        // operands of window element q (its stage has landed): z = x * (Kronecker
        // prefix rows), v = last other mode's row, both restricted to the lane's tile
        auto load_elem = [&](const unsigned char *st, int q, float (&z)[TL], float2 (&v)[TV / 2]) {
            const int e = q & 31;
            float x = mval[q];
            const float *rz;
            const float4 *rv;
            if (NM1 == 2) {
                rz = reinterpret_cast<const float *>(st + (e >> 2) * a.sa) + (e & 3) * a.Ka + l0;
                rv = reinterpret_cast<const float4 *>(
                    reinterpret_cast<const float *>(st + a.offb + (e >> 2) * a.sb) + (e & 3) * a.Kl + v0);
            } else {
                const float *ra = reinterpret_cast<const float *>(st + (e >> 2) * a.sa) + (e & 3) * a.Ka;
                x *= ra[ka];
                rz = reinterpret_cast<const float *>(st + a.offb + (e >> 2) * a.sb) + (e & 3) * a.Kb + kb0;
                rv = reinterpret_cast<const float4 *>(
                    reinterpret_cast<const float *>(st + a.offc + (e >> 2) * a.sc) + (e & 3) * a.Kl + v0);
            }
#pragma unroll
            for (int t = 0; t < TL / 4; ++t) {
                const float4 u = reinterpret_cast<const float4 *>(rz)[t];
                z[4 * t] = u.x;
                z[4 * t + 1] = u.y;
                z[4 * t + 2] = u.z;
                z[4 * t + 3] = u.w;
            }
            const float2 xx = make_float2(x, x);
#pragma unroll
            for (int t = 0; t < TV / 4; ++t) {
                const float4 u = rv[t];
                v[2 * t] = __fmul2_rn(make_float2(u.x, u.y), xx);
                v[2 * t + 1] = __fmul2_rn(make_float2(u.z, u.w), xx);
            }
        };
        auto fma_tile = [&](const float (&z)[TL], const float2 (&v)[TV / 2]) {
#pragma unroll
            for (int jj = 0; jj < TL; ++jj) {
                const float2 zz = make_float2(z[jj], z[jj]);
#pragma unroll
                for (int kk = 0; kk < TV / 2; ++kk) y2[jj][kk] = __ffma2_rn(zz, v[kk], y2[jj][kk]);
            }
        };
        // y += window elements q in [qa, qb) owned by this lane's group (q = step*NG + g).
        // Stage bookkeeping once per 32 elements; all_valid: every element of the
        // range is a stored entry (slices), so no per-step bounds test is needed.
        auto accumulate = [&](int qa, int qb, bool all_valid) {
            int k0 = (qa >> lg_ng) << lg_ng;
            while (k0 < qb) {
                const int s = k0 >> 5;
                need_stage(s);
                const unsigned char *st = ring + (size_t)((gst + s) & (HY_NB - 1)) * a.stage_bytes;
                const int kend = min(qb, (s + 1) << 5);
                if (all_valid) {
                    float z0[TL], z1[TL];
                    float2 v0r[TV / 2], v1r[TV / 2];
                    load_elem(st, k0 + g, z0, v0r);
                    for (; k0 < kend; k0 += 2 * NG) {
                        const bool two = k0 + NG < kend;
                        if (two) load_elem(st, k0 + NG + g, z1, v1r);
                        fma_tile(z0, v0r);
                        if (!two) {
                            k0 += NG;
                            break;
                        }
                        if (k0 + 2 * NG < kend) load_elem(st, k0 + 2 * NG + g, z0, v0r);
                        fma_tile(z1, v1r);
                    }
                } else {
                    for (; k0 < kend; k0 += NG) {
                        const int q = k0 + g;
                        if (q >= qa && q < qb) {
                            float z[TL];
                            float2 v[TV / 2];
                            load_elem(st, q, z, v);
                            fma_tile(z, v);
                        }
                    }
                }
                k0 = kend > k0 ? kend : k0;
                k0 = ((k0 + NG - 1) >> lg_ng) << lg_ng;
            }
        };

        if (it < a.nitem_long) {
            // ---------------- long rows: groups split a row's nonzeros; a row that
            // runs into the next item of the same range carries its partial y over
            if (p0 == ts && !carry) {
                j = a.item_aux[it];
                zero_y();
            }
            carry = false;
            int64_t pos = p0;
            while (pos < p1) {
                const int64_t rs = a.lrp[j], re = a.lrp[j + 1];
                const int64_t a1 = min(re, p1);
                if (a1 <= pos) break;  // descriptors always advance; never spin on bad input
                accumulate((int)(pos - p0), (int)(a1 - p0), false);
                const bool row_end = (a1 == re);
                const bool item_end = (a1 == te);
                if (!row_end && item_end && it + 1 < r1) {
                    carry = true;  // same row continues in the next item of this range
                } else if (row_end || item_end) {
                    __syncwarp();
                    for (int o = lpn; o < 32; o <<= 1) {
#pragma unroll
                        for (int jj = 0; jj < TL; ++jj)
#pragma unroll
                            for (int kk = 0; kk < TV / 2; ++kk) {
                                y2[jj][kk].x += __shfl_xor_sync(0xffffffffu, y2[jj][kk].x, o);
                                y2[jj][kk].y += __shfl_xor_sync(0xffffffffu, y2[jj][kk].y, o);
                            }
                    }
                    const int32_t r = a.lrow[j];
                    const bool full = (rs >= lbeg) && (re <= lend);
                    const int slot = (j == lfirst) ? 0 : 1;
                    if (g == 0) store_tile(full ? a.Y + (int64_t)r * a.Pm : a.ypart + (rg * 2 + slot) * a.Pm);
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
                accumulate((int)(pos - p0), (int)(a1 - p0), true);
                if (a1 == se) {
                    __syncwarp();
                    const int32_t r = a.srow[j * NG + g];
                    if (r >= 0) store_tile(a.Y + (int64_t)r * a.Pm);
                    zero_y();
                    ++j;
                }
                pos = a1;
            }
        }
        // stages issued but not consumed (none: every stage of the window is waited for)
        need_stage(nst - 1);
        __syncwarp();
        gst += nst;
        it = nit;
        p0 = np0;
        ++mk;
        if (!ok) break;
    }
    if (!ok) {
        // a staged copy never completed: bounded waits for this warp's other copies, then leave
        mbar_wait(mbar + ((mk + 1) & 1), (uint32_t)(((mk + 1) >> 1) & 1), nullptr);
        for (int q = 0; q < HY_NB; ++q) mbar_wait(sbar + q, (uint32_t)(((gst + q) >> 2) & 1), nullptr);
    }
}

// Y rows of the long rows cut by warp-range boundaries.  Piece of range t0
// (slot s0) and pieces of ranges t0+1..t1 (slot 0) are summed: warp w adds the
// pieces t0+1+w, t0+1+w+8, ... in order, then the 8 warp sums and the first
// piece are added in a fixed order, so the result does not depend on scheduling.
__global__ void __launch_bounds__(256) k_span_fix(const int32_t *span, const int32_t *lrow, const int32_t *item_aux,
                                                  int64_t ipw, const float *ypart, int Pm, float *Y) {
    extern __shared__ __align__(16) float part[];  // [8][Pm]
    const int b = blockIdx.x;
    const int32_t jl = span[3 * b], t0 = span[3 * b + 1], t1 = span[3 * b + 2];
    const int s0 = (item_aux[(int64_t)t0 * ipw] == jl) ? 0 : 1;
    const int32_t r = lrow[jl];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e = lane; e < Pm; e += 32) {
        float s = 0.f;
        for (int t = t0 + 1 + w; t <= t1; t += 8) s += ypart[((int64_t)t * 2) * Pm + e];
        part[w * Pm + e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < Pm; e += blockDim.x) {
        double s = ypart[((int64_t)t0 * 2 + s0) * Pm + e];
        for (int q = 0; q < 8; ++q) s += part[q * Pm + e];
        Y[(int64_t)r * Pm + e] = (float)s;
    }
}

// A(row_id[r], :) = G_(n) y_r for every stored row (the TTMcTC output, Eq.
// ttmctc, from the rows of Y_(n)).  Register tiles of 4 rows x 4 values of k_n
// per thread; Y and G_(n) are staged through shared memory in chunks of EC
// columns.  Rows of A without nonzeros stay as cleared by the caller.
__global__ void __launch_bounds__(256) k_a_from_y(const float *Y, const float *Gn, const int32_t *row_id, int64_t R,
                                                  int Kn, int Knp, int Pm, int RT, float *A) {
    extern __shared__ __align__(16) float dsm[];
    const int EC = Pm < 32 ? Pm : 32;
    float *YT = dsm;                    // [EC][RT + 4]
    float *GT = dsm + EC * (RT + 4);    // [EC][Knp]
    const int nkq = Knp >> 2;
    const int t = threadIdx.x;
    const int kq = t % nkq, rq = t / nkq;
    const bool active = rq < (RT >> 2);
    for (int64_t r0 = (int64_t)blockIdx.x * RT; r0 < R; r0 += (int64_t)gridDim.x * RT) {
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][k] = 0.f;
        for (int e0 = 0; e0 < Pm; e0 += EC) {
            __syncthreads();
            const int nq = EC >> 2;
            for (int idx = t; idx < RT * nq; idx += blockDim.x) {
                const int rr = idx / nq, c4 = idx - rr * nq;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (r0 + rr < R) v = *reinterpret_cast<const float4 *>(Y + (r0 + rr) * Pm + e0 + 4 * c4);
                YT[(4 * c4 + 0) * (RT + 4) + rr] = v.x;
                YT[(4 * c4 + 1) * (RT + 4) + rr] = v.y;
                YT[(4 * c4 + 2) * (RT + 4) + rr] = v.z;
                YT[(4 * c4 + 3) * (RT + 4) + rr] = v.w;
            }
            for (int idx = t; idx < EC * Knp; idx += blockDim.x) {
                const int e = idx / Knp, kn = idx - e * Knp;
                GT[idx] = kn < Kn ? Gn[(size_t)kn * Pm + e0 + e] : 0.f;
            }
            __syncthreads();
            if (active) {
                for (int e = 0; e < EC; ++e) {
                    const float4 y4 = *reinterpret_cast<const float4 *>(YT + e * (RT + 4) + 4 * rq);
                    const float4 g4 = *reinterpret_cast<const float4 *>(GT + e * Knp + 4 * kq);
                    const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
                    const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int k = 0; k < 4; ++k) acc[i][k] = fmaf(yv[i], gv[k], acc[i][k]);
                }
            }
        }
        if (active) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t r = r0 + 4 * rq + i;
                if (r >= R) continue;
                float *arow = A + (int64_t)row_id[r] * Kn;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (4 * kq + k < Kn) arow[4 * kq + k] = acc[i][k];
            }
        }
    }
}

// CTA partials of G_(n)[kn][e] = sum_r U_n(row_id[r], kn) * Y[r][e] over a
// fixed row range per CTA (Sec. 2.2: G = U_n^T Y_(n)).  Each thread owns 4 x 4
// (kn, e) tiles; U rows are staged in shared memory 64 at a time.
__global__ void __launch_bounds__(256) k_core_from_y(const float *Y, const float *Un, const int32_t *row_id, int64_t R,
                                                     int Kn, int Knp, int Pm, int64_t rpb, float *cpart) {
    constexpr int RB = 64;
    extern __shared__ __align__(16) float Us[];  // [RB][Knp]
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = min(r0 + rpb, R);
    const int KnPm = Kn * Pm;
    const int nkq = Knp >> 2, neq = Pm >> 2;
    const int nasg = nkq * neq;
    for (int base = 0; base < nasg; base += blockDim.x) {
        const int asg = base + threadIdx.x;
        const bool active = asg < nasg;
        const int kq = active ? asg / neq : 0;
        const int eq = active ? asg - kq * neq : 0;
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][k] = 0.f;
        for (int64_t rb = r0; rb < r1; rb += RB) {
            const int nr = (int)min((int64_t)RB, r1 - rb);
            __syncthreads();
            for (int t = threadIdx.x; t < nr * Knp; t += blockDim.x) {
                const int rr = t / Knp, q = t - rr * Knp;
                Us[t] = q < Kn ? Un[(int64_t)row_id[rb + rr] * Kn + q] : 0.f;
            }
            __syncthreads();
            if (active) {
                // 8 rows at a time: their loads are all in flight before the FMAs
                for (int rr0 = 0; rr0 < nr; rr0 += 8) {
                    float4 yb[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        yb[u] = rr0 + u < nr ? __ldg(reinterpret_cast<const float4 *>(Y + (rb + rr0 + u) * Pm) + eq)
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        if (rr0 + u >= nr) break;
                        const float4 u4 = *reinterpret_cast<const float4 *>(Us + (rr0 + u) * Knp + 4 * kq);
                        const float uv[4] = {u4.x, u4.y, u4.z, u4.w};
                        const float yv[4] = {yb[u].x, yb[u].y, yb[u].z, yb[u].w};
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int k = 0; k < 4; ++k) acc[i][k] = fmaf(uv[i], yv[k], acc[i][k]);
                    }
                }
            }
        }
        if (active) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int kn = 4 * kq + i;
                if (kn >= Kn) continue;
                float4 *dst = reinterpret_cast<float4 *>(cpart + (size_t)blockIdx.x * KnPm + (size_t)kn * Pm) + eq;
                *dst = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            }
        }
    }
}

struct HybLaunch {
    size_t smem = 0;
    int bar_off = 0, gs_off = 0, w_off = 0, w_stride = 0, meta_bytes = 0, ring_off = 0, stage_bytes = 0;
    int stage_tx = 0, sa = 0, sb = 0, sc = 0, offb = 0, offc = 0;
};

inline int al128(int x) { return (x + 127) & ~127; }

HybLaunch hyb_launch(const hoqri_ctx *c, int n, const FastTile &p) {
    HybLaunch L;
    const int narr = p.nm1 + 1;
    // ranks of the gathered rows: (Ua, Ub[, Uc]) = other modes in ascending order
    int K3[3] = {0, 0, 0}, j = 0;
    for (int m = 0; m < c->N; ++m)
        if (m != n) K3[j++] = c->K[m];
    L.sa = std::max(16 * K3[0], 128);
    L.sb = std::max(16 * K3[1], 128);
    L.sc = p.nm1 == 3 ? std::max(16 * K3[2], 128) : 0;
    L.offb = 8 * L.sa;
    L.offc = L.offb + 8 * L.sb;
    L.stage_bytes = al128(8 * (L.sa + L.sb + L.sc));
    L.stage_tx = 128 * (K3[0] + K3[1] + (p.nm1 == 3 ? K3[2] : 0));
    L.meta_bytes = HY_WB * 4;
    L.bar_off = 0;
    L.gs_off = al128(HY_WARPS * (2 + HY_NB) * 8);
    L.w_off = L.gs_off;
    L.ring_off = al128(2 * narr * L.meta_bytes);
    L.w_stride = al128(L.ring_off + HY_NB * L.stage_bytes);
    L.smem = (size_t)L.w_off + (size_t)HY_WARPS * L.w_stride;
    return L;
}

template <int NM1>
hoqri_status launch_hyb_nm1(hoqri_ctx *c, int n, const FastTile &p, HybArgs &a, const HybLaunch &L) {
    int oth[3] = {0, 0, 0}, j = 0;
    for (int m = 0; m < c->N; ++m)
        if (m != n) oth[j++] = m;
    const CUtensorMap &tA = c->tmap[oth[0]];
    const CUtensorMap &tB = c->tmap[oth[1]];
    const CUtensorMap &tC = c->tmap[NM1 == 3 ? oth[2] : oth[0]];
#define HQ_HYB(TLV, TVV)                                                                                    \
    if (p.TL == TLV && p.TV == TVV) {                                                                       \
        auto kern = k_hyb<NM1, TLV, TVV>;                                                           \
        HQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));     \
        const int grid = c->num_sms;                                                                        \
        kern<<<grid, HY_WARPS * 32, L.smem, c->stream>>>(tA, tB, tC, a);                                    \
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

bool hyb_mode(const hoqri_ctx *c, int n) { return c->ms[n].hyb && c->Y != nullptr && c->tmap_ok; }

// One 2-D tensor map per factor U_m (I_m x K_m FP32, row-major), box = one full
// row, for the gather4 loads of the hybrid pass.  The factors keep their device
// buffers for the life of the context, so the maps are encoded once.
hoqri_status encode_factor_maps(hoqri_ctx *c) {
    c->tmap_ok = false;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return HOQRI_OK;  // no tensor maps: the modes fall back to the two-pass kernels
    }
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    for (int m = 0; m < c->N; ++m) {
        if (c->prec != HOQRI_FP32 || c->K[m] % 4 != 0) continue;
        const cuuint64_t gdim[2] = {(cuuint64_t)c->K[m], (cuuint64_t)c->dims[m]};
        const cuuint64_t gstride[1] = {(cuuint64_t)c->K[m] * sizeof(float)};
        const cuuint32_t box[2] = {(cuuint32_t)c->K[m], 1};
        const cuuint32_t estr[2] = {1, 1};
        CUresult r = encode(&c->tmap[m], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->U[m], gdim, gstride, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            set_error("cuTensorMapEncodeTiled failed for a factor");
            return HOQRI_ERR_CUDA;
        }
    }
    c->tmap_ok = true;
    return HOQRI_OK;
}

// The pass over mode n's hybrid stream: writes every row y_r of Y_(n) into the
// dense R_n x P_{-n} buffer c->Y (rows cut by task boundaries are completed by
// k_span_fix).
hoqri_status hyb_pass(hoqri_ctx *c, int n) {
    const ModeStore &M = c->ms[n];
    FastTile p;
    if (!fast_tile(c, n, &p) || !c->tmap_ok) {
        set_error("hybrid pass: mode has no register-tile plan or tensor maps");
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
    a.ia = M.hidx[0];
    a.ib = M.hidx[1];
    a.ic = p.nm1 == 3 ? M.hidx[2] : nullptr;
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
    a.ipw = M.ipw;
    a.nrange = M.nrange;
    HybLaunch L = hyb_launch(c, n, p);
    a.bar_off = L.bar_off;
    a.gs_off = L.gs_off;
    a.w_off = L.w_off;
    a.w_stride = L.w_stride;
    a.meta_bytes = L.meta_bytes;
    a.ring_off = L.ring_off;
    a.stage_bytes = L.stage_bytes;
    a.stage_tx = L.stage_tx;
    a.sa = L.sa;
    a.sb = L.sb;
    a.sc = L.sc;
    a.offb = L.offb;
    a.offc = L.offc;
    a.Y = c->Y;
    a.ypart = c->ypart;
    a.err = c->dflag + 2;
    HQ_TRY(p.nm1 == 2 ? launch_hyb_nm1<2>(c, n, p, a, L) : launch_hyb_nm1<3>(c, n, p, a, L));
    if (M.nspan > 0) {
        const size_t sm = 8 * (size_t)a.Pm * sizeof(float);
        HQ_CUDA(cudaFuncSetAttribute(k_span_fix, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_span_fix<<<(unsigned)M.nspan, 256, sm, c->stream>>>(M.span, M.lrow, M.item_aux, M.ipw, c->ypart, a.Pm,
                                                               c->Y);
        c->nlaunch++;
    }
    HQ_CUDA(cudaGetLastError());
    return HOQRI_OK;
}

// A_n = Y_(n) G_(n)^T from the stored rows (Gn: G_(n) as [Kn][Pm] on the device).
hoqri_status hyb_a_from_y(hoqri_ctx *c, int n, const float *Gn, float *A_out) {
    const ModeStore &M = c->ms[n];
    const int Kn = c->K[n];
    const int Pm = (int)(c->P / Kn);
    const int Knp = (Kn + 3) & ~3;
    const int RT = std::min(256, 4 * (256 / (Knp / 4)));
    const int EC = Pm < 32 ? Pm : 32;
    const size_t smem = ((size_t)EC * (RT + 4) + (size_t)EC * Knp) * sizeof(float);
    HQ_CUDA(cudaMemsetAsync(A_out, 0, (size_t)c->dims[n] * Kn * sizeof(float), c->stream));
    if (M.R > 0) {
        HQ_CUDA(cudaFuncSetAttribute(k_a_from_y, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(M.R, RT), (int64_t)c->num_sms * 4));
        k_a_from_y<<<grid, 256, smem, c->stream>>>(c->Y, Gn, M.row_id, M.R, Kn, Knp, Pm, RT, A_out);
        c->nlaunch++;
    }
    HQ_CUDA(cudaGetLastError());
    return HOQRI_OK;
}

// G_(n) = U_n^T Y_(n) (Y from the last hyb_pass of mode n) into CTA partials;
// *nblk receives the number of partials.
hoqri_status hyb_core_partials(hoqri_ctx *c, int n, int *nblk) {
    const ModeStore &M = c->ms[n];
    const int Kn = c->K[n];
    const int Pm = (int)(c->P / Kn);
    const int Knp = (Kn + 3) & ~3;
    const int64_t R = M.R;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(R, 1), 256),
                                                                (int64_t)c->num_sms * 2));
    const int64_t rpb = ceil_div(std::max<int64_t>(R, 1), grid);
    const size_t smem = (size_t)64 * Knp * sizeof(float);
    k_core_from_y<<<grid, 256, smem, c->stream>>>(c->Y, (const float *)c->U[n], M.row_id, R, Kn, Knp, Pm, rpb,
                                                  (float *)c->core_part);
    c->nlaunch++;
    HQ_CUDA(cudaGetLastError());
    *nblk = grid;
    return HOQRI_OK;
}

size_t hyb_smem_need(const hoqri_ctx *c, int n) {
    FastTile p;
    if (!fast_tile(c, n, &p)) return (size_t)-1;
    return hyb_launch(c, n, p).smem;
}

size_t hyb_smem_cap() { return HY_SMEM_CAP; }

}  // namespace hoqri
