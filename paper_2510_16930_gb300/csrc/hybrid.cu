// One-stream-per-mode TTMcTC for FP32 on the hybrid layout.
//
// For mode n the pass forms every row y_i of Y_(n) = (X x_{-n} {U^T})_(n) once
// (Eq. ttmctc: Y_(n) unfolds the product of X with U_m^T along every mode m != n), writes
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
// Each window of the index/value streams (hw elements) is staged in shared
// memory by TMA bulk copies completing on an mbarrier, double buffered across
// the warp's windows; all waits are bounded.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.cuh"

namespace hoqri {

namespace {

constexpr int HY_WARPS = 8;
// staged elements per window (multiple of 32): as large as two blocks per SM
// allow (512 for three index arrays, 256 for four); larger windows mean fewer
// window turns (waits, descriptor updates, restarts of the software pipeline)
constexpr int HY_W_MAX = 512;
constexpr int HY_NMETA = 2;         // index/value windows per warp: the next one loads during this one
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

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

struct HybArgs {
    int Kn, Pm, Kl, Ka, Kb, Kc, GV, lpn;
    const float *Ua, *Ub, *Uc;  // gathered factors (other modes in ascending order)
    int Kr0, Kr1, Kr2;          // their ranks (row lengths, powers of two >= 4)
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
    int meta_bytes;                        // one staged array of a window (hw + 8 floats)
    int hw;                                // elements per window
    const float *Ulsplit;                  // last other factor as BF16 (hi | lo) rows, same bytes per row
    const float *Gn;  // [Kn][Pm]
    float *A;
    float *Y;
    float *apart;  // [nitem_long][2][Kn]
    float *ypart;  // [nitem_long][2][Pm]
    int32_t *err;
    unsigned long long *claim;  // slice items handed out so far (part 1 takes them dynamically)
};

// ---- split-BF16 tensor-core helpers (legacy warp-level mma.sync: the per-row
// tiles are 16 x 16 or 64 x 8, below the 64-row minimum of tcgen05.mma)

// v = hi + lo with hi = bf16(v) and lo = bf16(v - hi) (v - hi is exact in FP32)
__device__ __forceinline__ void split2(float2 v, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat162 h = __float22bfloat162_rn(v);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __float22bfloat162_rn(make_float2(v.x - hf.x, v.y - hf.y));
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

// d += a (16 x 16, row) * b (16 x 8, col), BF16 in, FP32 accumulate
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One pass over mode n's hybrid stream, part PART: 0 = the long rows (a
// contiguous range of items per warp), 1 = the slices (every nw-th item).
// Factor rows are read straight from global memory (L1-cached, read-only path)
// into registers: at two blocks of 8 warps per SM the loads of one warp overlap
// the arithmetic of the others.  MT > 0: long rows on the split-BF16 tensor-core
// path (MT x NT tiles of 16 x 8); MT == 0: FP32 FMA tiles (TL x TV per lane).
template <int NM1, int TL, int TV, int MT, int NT, int PART>
__global__ void __launch_bounds__(HY_WARPS * 32, 2) k_hyb(HybArgs a) {
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
    constexpr bool MMA = MT > 0 && PART == 0;
    unsigned char *wbase = smem_raw + a.w_off + (size_t)w * a.w_stride;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw + a.bar_off) + (size_t)w * 3;
    // window barriers: one arrival each (lane 0's expect_tx)
    if (lane == 0)
        for (int q = 0; q < 3; ++q) mbar_init(mbar + q, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();

    const int64_t gw = (int64_t)blockIdx.x * HY_WARPS + w;

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

    // ---- FP32 FMA tiles: y tile as column pairs, y2[j][k] = columns (2k, 2k+1) of row j
    constexpr int TLs = MMA ? 1 : TL, TVs = MMA ? 2 : TV;  // unused by the tensor-core part
    float2 y2[TLs][TVs / 2];
    auto zero_y = [&]() {
#pragma unroll
        for (int j = 0; j < TLs; ++j)
#pragma unroll
            for (int k = 0; k < TVs / 2; ++k) y2[j][k] = make_float2(0.f, 0.f);
    };
    auto store_tile = [&](float *dst) {
#pragma unroll
        for (int j = 0; j < TLs; ++j) {
            float4 *p = reinterpret_cast<float4 *>(dst + (size_t)(l0 + j) * a.Kl + v0);
#pragma unroll
            for (int k4 = 0; k4 < TVs / 4; ++k4)
                p[k4] = make_float4(y2[j][2 * k4].x, y2[j][2 * k4].y, y2[j][2 * k4 + 1].x, y2[j][2 * k4 + 1].y);
        }
    };

    // ---- split-BF16 tensor-core tiles.  The tensor cores add into their FP32
    // accumulator without rounding to nearest, so a long chain of mma into one
    // accumulator drifts (a relative bias growing with the chain).  Each group of
    // mma of two 16-nonzero steps goes to a fresh accumulator dtmp, which is then
    // added to dacc in FP32 (round to nearest): chains stay 6 mma long.
    constexpr int MTs = MMA ? MT : 1, NTs = MMA ? NT : 1;
    constexpr int KS_FLUSH = 2;
    float dacc[MTs][NTs][4];
    float dtmp[MTs][NTs][4];
    int ksteps = 0;  // 16-nonzero steps accumulated in dtmp
    auto zero_d = [&]() {
#pragma unroll
        for (int mt = 0; mt < MTs; ++mt)
#pragma unroll
            for (int nt = 0; nt < NTs; ++nt)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    dacc[mt][nt][r] = 0.f;
                    dtmp[mt][nt][r] = 0.f;
                }
        ksteps = 0;
    };
    auto flush_d = [&]() {
#pragma unroll
        for (int mt = 0; mt < MTs; ++mt)
#pragma unroll
            for (int nt = 0; nt < NTs; ++nt)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    dacc[mt][nt][r] += dtmp[mt][nt][r];
                    dtmp[mt][nt][r] = 0.f;
                }
        ksteps = 0;
    };
    // lane holds D(mt*16 + gq (+8), nt*8 + 2 tq (+1)), gq = lane / 4, tq = lane % 4
    auto store_d = [&](float *dst) {
        flush_d();
        const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
        for (int mt = 0; mt < MTs; ++mt)
#pragma unroll
            for (int nt = 0; nt < NTs; ++nt) {
                float *p = dst + (size_t)(mt * 16 + gq) * a.Kl + nt * 8 + 2 * tq;
                *reinterpret_cast<float2 *>(p) = make_float2(dacc[mt][nt][0], dacc[mt][nt][1]);
                *reinterpret_cast<float2 *>(p + 8 * a.Kl) = make_float2(dacc[mt][nt][2], dacc[mt][nt][3]);
            }
    };
    if (MMA) zero_d(); else zero_y();

    bool ok = true;
    int mk = 0;  // windows consumed by this warp
    // work list of this warp: part 0, a contiguous range of long-row items (rows
    // carry across items inside the range); part 1, every nw-th slice item
    const int64_t rg = gw;
    const int64_t r0 = PART == 0 ? rg * a.ipw : 0;
    const int64_t r1 = PART == 0 ? (rg < a.nrange ? min(r0 + a.ipw, a.nitem_long) : r0) : 0;
    const int64_t iend = PART == 0 ? r1 : a.nitem;
    // part 1: a warp claims its next slice item from a device counter, so warps
    // that finish early take more items (the item a row is computed in does not
    // change its arithmetic, so results stay the same from run to run)
    auto claim_slice = [&]() -> int64_t {
        unsigned long long v = 0;
        if (lane == 0) v = atomicAdd(a.claim, 1ull);
        v = __shfl_sync(0xffffffffu, v, 0);
        return a.nitem_long + (int64_t)v;
    };
    auto next_item = [&](int64_t cur) -> int64_t { return PART == 0 ? cur + 1 : claim_slice(); };
    const int64_t lfirst = (PART == 0 && r0 < r1) ? a.item_aux[r0] : -1;
    const int64_t lbeg = (PART == 0 && r0 < r1) ? a.item_s[r0] : 0;
    const int64_t lend = (PART == 0 && r0 < r1) ? a.item_e[r1 - 1] : 0;
    // windows of the work list: item, first element, length, item end; the
    // index/value streams of window k+2 are requested while window k is used
    struct Win {
        int64_t it, p0, te;
        int len;
        bool first;  // first window of its item
    };
    auto item_win = [&](int64_t item) -> Win {
        Win wv{item, 0, 0, 0, true};
        if (item < iend) {
            wv.p0 = a.item_s[item];
            wv.te = a.item_e[item];
            wv.len = (int)min((int64_t)a.hw, wv.te - wv.p0);
        }
        return wv;
    };
    auto next_win = [&](const Win &wv) -> Win {
        if (wv.len == 0) return wv;
        const int64_t np0 = wv.p0 + a.hw;
        if (np0 < wv.te) return Win{wv.it, np0, wv.te, (int)min((int64_t)a.hw, wv.te - np0), false};
        return item_win(next_item(wv.it));
    };
    Win W0 = item_win(PART == 0 ? r0 : claim_slice());
    Win W1 = next_win(W0);
    int issued = 0;  // windows whose streams were requested (buffer = window index mod HY_NMETA)
    if (W0.len > 0) issue_meta(W0.p0, W0.p0 + W0.len, 0), ++issued;
    if (HY_NMETA == 3 && W1.len > 0) issue_meta(W1.p0, W1.p0 + W1.len, 1), ++issued;
    int64_t j = 0;
    int64_t jc = -1, crs = 0, cre = 0;  // cached bounds (lrp or sbase) of row / slice jc
    bool carry = false;  // a long row continues from the previous item of this range
    int b0 = 0, b1 = 1, b2 = 2;  // meta buffers of windows mk, mk+1 (, mk+2)
    while (W0.len > 0) {
        Win W2 = W1;
        if (HY_NMETA == 3) {
            W2 = next_win(W1);
            if (W2.len > 0) issue_meta(W2.p0, W2.p0 + W2.len, b2), ++issued;
        } else if (W1.len > 0) {
            issue_meta(W1.p0, W1.p0 + W1.len, b1), ++issued;
        }
        if (!mbar_wait(mbar + b0, (uint32_t)((mk / HY_NMETA) & 1), a.err)) {
            ok = false;
            break;
        }
        const int64_t it = W0.it;
        const int64_t p0 = W0.p0, te = W0.te;
        const int64_t p1 = p0 + W0.len;
        const unsigned char *mb = wbase + (size_t)b0 * NARR * a.meta_bytes;
        const int32_t *mia = reinterpret_cast<const int32_t *>(mb);
        const int32_t *mib = reinterpret_cast<const int32_t *>(mb + a.meta_bytes);
        const int32_t *mic = reinterpret_cast<const int32_t *>(mb + 2 * a.meta_bytes);
        const float *mval = reinterpret_cast<const float *>(mb + (NARR - 1) * a.meta_bytes);

        // operands of window element q: z = x * (Kronecker prefix rows), v = the
        // last other mode's row, both restricted to the lane's tile
        auto load_elem = [&](int q, float (&z)[TLs], float2 (&v)[TVs / 2]) {
            float x = mval[q];
            const float *rz;
            const float4 *rv;
            if (NM1 == 2) {
                rz = a.Ua + (size_t)mia[q] * a.Kr0 + l0;
                rv = reinterpret_cast<const float4 *>(a.Ub + (size_t)mib[q] * a.Kr1 + v0);
            } else {
                x *= __ldg(a.Ua + (size_t)mia[q] * a.Kr0 + ka);
                rz = a.Ub + (size_t)mib[q] * a.Kr1 + kb0;
                rv = reinterpret_cast<const float4 *>(a.Uc + (size_t)mic[q] * a.Kr2 + v0);
            }
#pragma unroll
            for (int t = 0; t < TLs / 4; ++t) {
                const float4 u = __ldg(reinterpret_cast<const float4 *>(rz) + t);
                z[4 * t] = u.x;
                z[4 * t + 1] = u.y;
                z[4 * t + 2] = u.z;
                z[4 * t + 3] = u.w;
            }
            const float2 xx = make_float2(x, x);
#pragma unroll
            for (int t = 0; t < TVs / 4; ++t) {
                const float4 u = __ldg(rv + t);
                v[2 * t] = __fmul2_rn(make_float2(u.x, u.y), xx);
                v[2 * t + 1] = __fmul2_rn(make_float2(u.z, u.w), xx);
            }
        };
        auto fma_tile = [&](const float (&z)[TLs], const float2 (&v)[TVs / 2]) {
#pragma unroll
            for (int jj = 0; jj < TLs; ++jj) {
                const float2 zz = make_float2(z[jj], z[jj]);
#pragma unroll
                for (int kk = 0; kk < TVs / 2; ++kk) y2[jj][kk] = __ffma2_rn(zz, v[kk], y2[jj][kk]);
            }
        };
        auto one_step = [&](int q, int lo, int hi) {
            if (q >= lo && q < hi) {
                float z[TLs];
                float2 v[TVs / 2];
                load_elem(q, z, v);
                fma_tile(z, v);
            }
        };
        // y += window elements q in [qa, qb) owned by this lane's group (q = step*NG + g).
        // Steps whose NG elements all lie in [qa, qb) run software-pipelined (the
        // loads of the next step are issued before the multiply-adds of this
        // one); a step cut by qa or qb tests its element.  all_valid: every
        // element of the range is a stored entry (slices; their rows are NG-aligned).
        auto accumulate = [&](int qa, int qb, bool all_valid) {
            int k0 = (qa >> lg_ng) << lg_ng;
            if (!all_valid && k0 < qa) {
                one_step(k0 + g, qa, qb);
                k0 += NG;
            }
            const int kfull = all_valid ? qb : k0 + ((max(qb - k0, 0) >> lg_ng) << lg_ng);
            if (k0 < kfull) {
                float z0[TLs], z1[TLs];
                float2 v0r[TVs / 2], v1r[TVs / 2];
                load_elem(k0 + g, z0, v0r);
                for (; k0 < kfull; k0 += 2 * NG) {
                    const bool two = k0 + NG < kfull;
                    if (two) load_elem(k0 + NG + g, z1, v1r);
                    fma_tile(z0, v0r);
                    if (!two) {
                        k0 += NG;
                        break;
                    }
                    if (k0 + 2 * NG < kfull) load_elem(k0 + 2 * NG + g, z0, v0r);
                    fma_tile(z1, v1r);
                }
            }
            if (!all_valid && k0 < qb) one_step(k0 + g, qa, qb);
        };

        // D += contributions of window nonzeros [qa, qb) of one row on the tensor
        // cores, 16 nonzeros per step:
        //   D += A B,  A(m, k) = x_k * (Kronecker prefix rows of k)(m),  B(k, :) = U_l row of k
        // with A = Ah + Al and B = Bh + Bl split into BF16 and D += Ah Bh + Ah Bl + Al Bh
        // in FP32 (the Al Bl term is below FP32 rounding of the sum).  B comes
        // pre-split from Ulsplit (hi row, then lo row); A is formed and split in
        // registers.  Lane (gq, tq) holds A(gq (+8), k) and B(k, gq) of the
        // nonzeros k = 2tq, 2tq+1, 2tq+8, 2tq+9 of the step (the mma fragments).
        auto mma_accumulate = [&](int qa, int qb) {
            if constexpr (MMA) {
                const int gq = lane >> 2, tq = lane & 3;
                const uint16_t *Bs = reinterpret_cast<const uint16_t *>(a.Ulsplit);
                for (int k0 = qa & ~15; k0 < qb; k0 += 16) {
                    float av[4][MT][2];
                    uint32_t hb[4][NT], lb[4][NT];
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        const int kq = k0 + 2 * tq + (q4 & 1) + 8 * (q4 >> 1);
                        const bool valid = kq >= qa && kq < qb;
                        const float x = valid ? mval[kq] : 0.f;
                        const int32_t ra = valid ? mia[kq] : 0;
                        const int32_t rl = valid ? (NM1 == 2 ? mib[kq] : mic[kq]) : 0;
                        if (NM1 == 2) {
                            // A(m, k) = x * Ua(row, m), m = mt*16 + gq (+8)
#pragma unroll
                            for (int mt = 0; mt < MT; ++mt) {
                                av[q4][mt][0] = x * __ldg(a.Ua + (size_t)ra * a.Kr0 + mt * 16 + gq);
                                av[q4][mt][1] = x * __ldg(a.Ua + (size_t)ra * a.Kr0 + mt * 16 + gq + 8);
                            }
                        } else {
                            // Ka = Kb = 8: m = p*8 + r, so rows m = mt*16 + gq (+8) are p = 2mt (+1), r = gq
                            const int32_t rb = valid ? mib[kq] : 0;
                            const float xb = x * __ldg(a.Ub + (size_t)rb * 8 + gq);
#pragma unroll
                            for (int mt = 0; mt < MT; ++mt) {
                                av[q4][mt][0] = xb * __ldg(a.Ua + (size_t)ra * 8 + 2 * mt);
                                av[q4][mt][1] = xb * __ldg(a.Ua + (size_t)ra * 8 + 2 * mt + 1);
                            }
                        }
                        const uint16_t *brow = Bs + (size_t)rl * 2 * a.Kl;
#pragma unroll
                        for (int nt = 0; nt < NT; ++nt) {
                            hb[q4][nt] = valid ? __ldg(brow + nt * 8 + gq) : 0u;
                            lb[q4][nt] = valid ? __ldg(brow + a.Kl + nt * 8 + gq) : 0u;
                        }
                    }
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt) {
                        uint32_t ah[4], al[4];
                        split2(make_float2(av[0][mt][0], av[1][mt][0]), ah[0], al[0]);
                        split2(make_float2(av[0][mt][1], av[1][mt][1]), ah[1], al[1]);
                        split2(make_float2(av[2][mt][0], av[3][mt][0]), ah[2], al[2]);
                        split2(make_float2(av[2][mt][1], av[3][mt][1]), ah[3], al[3]);
#pragma unroll
                        for (int nt = 0; nt < NT; ++nt) {
                            const uint32_t bh0 = hb[0][nt] | (hb[1][nt] << 16), bh1 = hb[2][nt] | (hb[3][nt] << 16);
                            const uint32_t bl0 = lb[0][nt] | (lb[1][nt] << 16), bl1 = lb[2][nt] | (lb[3][nt] << 16);
                            mma_bf16(dtmp[mt][nt], al, bh0, bh1);
                            mma_bf16(dtmp[mt][nt], ah, bl0, bl1);
                            mma_bf16(dtmp[mt][nt], ah, bh0, bh1);
                        }
                    }
                    if (++ksteps == KS_FLUSH) flush_d();
                }
            }
        };

        if (PART == 0) {
            // ---------------- long rows; a row that runs into the next item of
            // the same range carries its partial tile over
            if (W0.first && !carry) {
                j = a.item_aux[it];
                if (MMA) zero_d(); else zero_y();
            }
            carry = false;
            int64_t pos = p0;
            while (pos < p1) {
                if (jc != j) {
                    jc = j;
                    crs = a.lrp[j];
                    cre = a.lrp[j + 1];
                }
                const int64_t rs = crs, re = cre;
                const int64_t a1 = min(re, p1);
                if (a1 <= pos) break;  // descriptors always advance; never spin on bad input
                if (MMA) mma_accumulate((int)(pos - p0), (int)(a1 - p0));
                else accumulate((int)(pos - p0), (int)(a1 - p0), false);
                const bool row_end = (a1 == re);
                const bool item_end = (a1 == te);
                if (!row_end && item_end && it + 1 < r1) {
                    carry = true;  // same row continues in the next item of this range
                } else if (row_end || item_end) {
                    const int32_t r = a.lrow[j];
                    const bool full = (rs >= lbeg) && (re <= lend);
                    const int slot = (j == lfirst) ? 0 : 1;
                    float *dst = full ? a.Y + (int64_t)r * a.Pm : a.ypart + (rg * 2 + slot) * a.Pm;
                    if (MMA) {
                        store_d(dst);
                        zero_d();
                    } else {
                        // lane groups split the row's nonzeros: add their tiles
                        __syncwarp();
                        for (int o = lpn; o < 32; o <<= 1) {
#pragma unroll
                            for (int jj = 0; jj < TLs; ++jj)
#pragma unroll
                                for (int kk = 0; kk < TVs / 2; ++kk) {
                                    y2[jj][kk].x += __shfl_xor_sync(0xffffffffu, y2[jj][kk].x, o);
                                    y2[jj][kk].y += __shfl_xor_sync(0xffffffffu, y2[jj][kk].y, o);
                                }
                        }
                        if (g == 0) store_tile(dst);
                        zero_y();
                    }
                    if (row_end) ++j;
                }
                pos = a1;
            }
        } else {
            // ---------------- slices: lane group g owns row g of the slice
            if (W0.first) {
                j = a.item_aux[it];
                zero_y();
                jc = -1;
            }
            int64_t pos = p0;
            while (pos < p1) {
                if (jc != j) {
                    jc = j;
                    cre = a.sbase[j + 1];
                }
                const int64_t se = cre;
                const int64_t a1 = min(se, p1);
                if (a1 <= pos) break;
                accumulate((int)(pos - p0), (int)(a1 - p0), true);
                if (a1 == se) {
                    const int32_t r = a.srow[j * NG + g];
                    if (r >= 0) store_tile(a.Y + (int64_t)r * a.Pm);
                    zero_y();
                    ++j;
                }
                pos = a1;
            }
        }
        __syncwarp();  // every lane is done with window mk's buffer before it is refilled
        if (HY_NMETA == 3) {
            W0 = W1;
            W1 = W2;
            const int bt = b0;
            b0 = b1;
            b1 = b2;
            b2 = bt;
        } else {
            W0 = W1;
            W1 = next_win(W1);
            b0 ^= 1;
            b1 ^= 1;
        }
        ++mk;
    }
    if (!ok) {
        // a window's copy never completed: bounded waits for this warp's requested
        // windows that were not consumed, then leave
        for (int wq = mk; wq < issued; ++wq)
            mbar_wait(mbar + wq % HY_NMETA, (uint32_t)((wq / HY_NMETA) & 1), nullptr);
    }
}

// Y rows of the long rows cut by warp-range boundaries.  The row's piece from
// range t0 (slot s0) and its pieces from ranges t0+1..t1 (slot 0) are summed.
// Thread (j, c) adds the 16-byte column group c of pieces t0+1+j, t0+1+j+ns,
// ... (ns = SF_THREADS / (Pm/4) piece streams, at most 32, at least 1) in
// SF_ACC interleaved running sums, so that SF_ACC loads are in flight (a
// Zipf-heavy row spans hundreds of ranges), combined in a fixed order; then
// the ns stream sums and the first piece are added in order, in FP64.  The
// result does not depend on scheduling.
constexpr int SF_THREADS = 256;
constexpr int SF_ACC = 8;

__host__ __device__ constexpr int span_fix_ns(int Pm) {
    return SF_THREADS / (Pm / 4) < 1 ? 1 : (SF_THREADS / (Pm / 4) < 32 ? SF_THREADS / (Pm / 4) : 32);
}

__global__ void __launch_bounds__(SF_THREADS, 1) k_span_fix(const int32_t *span, const int32_t *lrow,
                                                         const int32_t *item_aux, int64_t ipw, const float *ypart,
                                                         int Pm, float *Y) {
    extern __shared__ __align__(16) float4 part4[];  // [ns][Pm / 4]
    const int b = blockIdx.x;
    const int32_t jl = span[3 * b], t0 = span[3 * b + 1], t1 = span[3 * b + 2];
    const int s0 = (item_aux[(int64_t)t0 * ipw] == jl) ? 0 : 1;
    const int32_t r = lrow[jl];
    const int P4 = Pm >> 2;
    const int ns = span_fix_ns(Pm);
    const int cw = P4 < SF_THREADS ? P4 : SF_THREADS;  // column groups covered by one stream of threads
    const int j = threadIdx.x / cw, c0 = threadIdx.x - j * cw;
    const float4 *yp4 = reinterpret_cast<const float4 *>(ypart);
    auto add4 = [](float4 &a, const float4 v) {
        a.x += v.x;
        a.y += v.y;
        a.z += v.z;
        a.w += v.w;
    };
    if (j < ns) {
        for (int c = c0; c < P4; c += cw) {
            float4 a[SF_ACC];
#pragma unroll
            for (int u = 0; u < SF_ACC; ++u) a[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            int t = t0 + 1 + j;
            for (; t + (SF_ACC - 1) * ns <= t1; t += SF_ACC * ns) {
                float4 v[SF_ACC];
#pragma unroll
                for (int u = 0; u < SF_ACC; ++u) v[u] = yp4[(int64_t)(t + u * ns) * 2 * P4 + c];
#pragma unroll
                for (int u = 0; u < SF_ACC; ++u) add4(a[u], v[u]);
            }
#pragma unroll
            for (int u = 0; u < SF_ACC - 1; ++u)
                if (t + u * ns <= t1) add4(a[u], yp4[(int64_t)(t + u * ns) * 2 * P4 + c]);
#pragma unroll
            for (int w = 1; w < SF_ACC; w *= 2)
#pragma unroll
                for (int u = 0; u < SF_ACC; u += 2 * w) add4(a[u], a[u + w]);
            part4[j * P4 + c] = a[0];
        }
    }
    __syncthreads();
    const float *part = reinterpret_cast<const float *>(part4);
    for (int e = threadIdx.x; e < Pm; e += blockDim.x) {
        double s = ypart[((int64_t)t0 * 2 + s0) * Pm + e];
        for (int q = 0; q < ns; ++q) s += part[q * Pm + e];
        Y[(int64_t)r * Pm + e] = (float)s;
    }
}

// Upad(i, k) = U(i, k) for k < K, 0 for K <= k < Kp: the factor as the sliced
// pass of a padded plan gathers it
__global__ void k_pad_factor(const float *U, int64_t rows, int K, int Kp, float *Upad) {
    const int64_t n = rows * Kp;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / Kp;
        const int k = (int)(t - r * Kp);
        Upad[t] = k < K ? U[r * K + k] : 0.f;
    }
}

struct HybLaunch {
    size_t smem = 0;
    int hw = 0;
    int bar_off = 0, gs_off = 0, w_off = 0, w_stride = 0, meta_bytes = 0;
    int MT = 0, NT = 0;  // tensor-core tiles of the long rows (0: FP32 FMA tiles)
};

inline int al128(int x) { return (x + 127) & ~127; }

// Split-BF16 tensor-core tiles for mode n's long rows, if the context computes
// in HOQRI_BF16X3 and the shape has a kernel: N = 3 with K_a in {16, 32} rows of
// the tile and K_l in {8, 16, 32} columns; N = 4 with K_a = K_b = 8 (64 rows)
// and K_l in {8, 16, 32}.  Other shapes keep the FP32 FMA tiles.
void mix_shape(const hoqri_ctx *c, int n, const FastTile &p, int *MT, int *NT) {
    *MT = 0;
    *NT = 0;
    if (!c->mix || p.TL != 8 || p.TV != 8) return;
    (void)n;
    const int K3[3] = {p.Ka, p.nm1 == 3 ? p.Kb : p.Kl, p.Kl};  // the plan's (possibly padded) ranks
    const int Kl = p.Kl;
    if (Kl != 8 && Kl != 16 && Kl != 32) return;
    if (p.nm1 == 2 && (K3[0] == 16 || K3[0] == 32)) {
        *MT = K3[0] / 16;
        *NT = Kl / 8;
    } else if (p.nm1 == 3 && K3[0] == 8 && K3[1] == 8) {
        *MT = 4;
        *NT = Kl / 8;
    }
}

HybLaunch hyb_launch(const hoqri_ctx *c, int n, const FastTile &p) {
    HybLaunch L;
    const int narr = p.nm1 + 1;
    mix_shape(c, n, p, &L.MT, &L.NT);
    // shared memory: HY_NMETA index/value windows per warp and their barriers
    L.hw = narr == 3 ? HY_W_MAX : HY_W_MAX / 2;
    L.meta_bytes = (L.hw + 8) * 4;
    L.bar_off = 0;
    L.gs_off = al128(HY_WARPS * 3 * 8);  // three barriers per warp (at most HY_NMETA used)
    L.w_off = L.gs_off;
    L.w_stride = al128(HY_NMETA * narr * L.meta_bytes);
    L.smem = (size_t)L.w_off + (size_t)HY_WARPS * L.w_stride;
    return L;
}

// U_l as BF16 (hi | lo) rows: out row r = K/2 words of hi pairs, K/2 words of lo pairs
__global__ void k_split_bf16(const float *U, int64_t rows, int K, uint32_t *out) {
    const int hk = K / 2;
    const int64_t npair = rows * hk;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npair; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / hk;
        const int cpair = (int)(t - r * hk);
        uint32_t hi, lo;
        split2(reinterpret_cast<const float2 *>(U)[t], hi, lo);
        out[r * K + cpair] = hi;
        out[r * K + hk + cpair] = lo;
    }
}

template <int NM1>
hoqri_status launch_hyb_nm1(hoqri_ctx *c, int n, const FastTile &p, HybArgs &a, const HybLaunch &L) {
    // hyb_blocks_per_sm blocks of HY_WARPS warps per SM: part 0 (long rows), then part 1 (slices)
    const int grid = hyb_blocks_per_sm(p) * c->num_sms;
    // shared-memory share of the SM's unified L1 / shared store: just what the
    // resident blocks need, so the rest stays L1 for the factor rows of the most
    // frequent indices (a skewed index law gathers most rows from a few thousand)
    int smem_sm = 0;
    HQ_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device));
    const int carve = (int)std::min<int64_t>(
        100, ceil_div((int64_t)hyb_blocks_per_sm(p) * ((int64_t)L.smem + 1024) * 100, std::max(smem_sm, 1)));
#define HQ_HYB(TLV, TVV, MTV, NTV)                                                                           \
    if (p.TL == TLV && p.TV == TVV && L.MT == MTV && L.NT == NTV) {                                          \
        auto k0 = k_hyb<NM1, TLV, TVV, MTV, NTV, 0>;                                                         \
        auto k1 = k_hyb<NM1, TLV, TVV, 0, 0, 1>;                                                             \
        HQ_CUDA(smem_limit(k0, L.smem));        \
        HQ_CUDA(smem_limit(k1, L.smem));        \
        HQ_CUDA(cudaFuncSetAttribute(k0, cudaFuncAttributePreferredSharedMemoryCarveout, carve));           \
        HQ_CUDA(cudaFuncSetAttribute(k1, cudaFuncAttributePreferredSharedMemoryCarveout, carve));           \
        if (a.nitem_long > 0) {                                                                              \
            k0<<<grid, HY_WARPS * 32, L.smem, c->stream>>>(a);                                               \
            c->nlaunch++;                                                                                    \
        }                                                                                                    \
        if (a.nitem > a.nitem_long) {                                                                        \
            HQ_CUDA(cudaMemsetAsync(a.claim, 0, sizeof(unsigned long long), c->stream));                     \
            k1<<<grid, HY_WARPS * 32, L.smem, c->stream>>>(a);                                               \
            c->nlaunch++;                                                                                    \
        }                                                                                                    \
        HQ_CUDA(cudaGetLastError());                                                                         \
        return HOQRI_OK;                                                                                     \
    }
    HQ_HYB(8, 8, 0, 0)
    HQ_HYB(8, 4, 0, 0)
    HQ_HYB(4, 8, 0, 0)
    HQ_HYB(4, 4, 0, 0)
    if constexpr (NM1 == 2) {
        HQ_HYB(8, 8, 1, 1)
        HQ_HYB(8, 8, 1, 2)
        HQ_HYB(8, 8, 1, 4)
        HQ_HYB(8, 8, 2, 1)
        HQ_HYB(8, 8, 2, 2)
        HQ_HYB(8, 8, 2, 4)
    } else {
        HQ_HYB(8, 8, 4, 1)
        HQ_HYB(8, 8, 4, 2)
        HQ_HYB(8, 8, 4, 4)
    }
#undef HQ_HYB
    set_error("hybrid pass: no kernel for this tile");
    return HOQRI_ERR_UNSUPPORTED;
}

}  // namespace

// the register-tile plan of mode n, with the lane tile the autotuner chose if any
// (FP32 only: the split-BF16 tiles keep the plan's 8 x 8)
bool padded_plan(const hoqri_ctx *c, int n, FastTile *out);  // passes.cu

bool hyb_tile(const hoqri_ctx *c, int n, FastTile *out) {
    FastTile p;
    // ranks that are not powers of two >= 4: the plan of the padded ranks (the
    // pass gathers zero-padded factor copies; the padded columns of Y_(n) are 0)
    if (!fast_tile(c, n, &p) && !padded_plan(c, n, &p)) return false;
    const ModeStore &M = c->ms[n];
    if (!c->mix && M.tune_TL > 0 && M.tune_TV > 0) {
        const int L = p.GL * p.TL;
        if (L % M.tune_TL == 0 && p.Kl % M.tune_TV == 0 && (L / M.tune_TL) * (p.Kl / M.tune_TV) <= 32 &&
            (p.nm1 == 2 || p.Kb % M.tune_TL == 0)) {  // order 4: a lane's rows stay in one K_b block
            p.TL = M.tune_TL;
            p.TV = M.tune_TV;
            p.GL = L / p.TL;
            p.GV = p.Kl / p.TV;
            p.lpn = p.GL * p.GV;
        }
    }
    *out = p;
    return true;
}

int hyb_blocks_per_sm(const FastTile &p) {
    (void)p;
    return 2;
}

bool hyb_mode(const hoqri_ctx *c, int n) { return (c->ms[n].hyb || c->ms[n].fib) && c->Y != nullptr; }

// The pass over mode n's hybrid stream: writes every row y_r of Y_(n) into the
// dense R_n x P_{-n} buffer c->Y (rows cut by task boundaries are completed by
// k_span_fix).
hoqri_status hyb_pass(hoqri_ctx *c, int n) {
    if (c->ms[n].fib) return fib_pass(c, n);
    const ModeStore &M = c->ms[n];
    FastTile p;
    if (!hyb_tile(c, n, &p)) {
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
    a.hw = L.hw;
    {
        int j = 0;
        const float *Uo[3] = {nullptr, nullptr, nullptr};
        int Ko[3] = {4, 4, 4};
        for (int m = 0; m < c->N; ++m)
            if (m != n) {
                Uo[j] = (const float *)c->U[m];
                Ko[j] = c->K[m];
                if (p.pad && padded_rank(c->K[m]) != c->K[m]) {
                    // refresh the zero-padded copy from the current factor
                    const int Kp = padded_rank(c->K[m]);
                    const int64_t tot = c->dims[m] * (int64_t)Kp;
                    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(tot, 256), 8 * (int64_t)c->num_sms));
                    k_pad_factor<<<g, 256, 0, c->stream>>>((const float *)c->U[m], c->dims[m], c->K[m], Kp, c->Upad[m]);
                    c->nlaunch++;
                    Uo[j] = c->Upad[m];
                    Ko[j] = Kp;
                }
                ++j;
            }
        a.Ua = Uo[0];
        a.Ub = Uo[1];
        a.Uc = Uo[2];
        a.Kr0 = Ko[0];
        a.Kr1 = Ko[1];
        a.Kr2 = Ko[2];
        a.Ulsplit = nullptr;
        if (L.MT > 0) {
            // the last other factor, split into BF16 hi / lo rows for the B operand
            const int Kl = Ko[p.nm1 - 1];
            int ml = -1;
            for (int m = c->N - 1; m >= 0 && ml < 0; --m)
                if (m != n) ml = m;
            const int64_t rows = c->dims[ml];
            const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows * Kl / 2, 256), 8 * (int64_t)c->num_sms));
            k_split_bf16<<<grid, 256, 0, c->stream>>>(Uo[p.nm1 - 1], rows, Kl, (uint32_t *)c->usplit);
            c->nlaunch++;
            a.Ulsplit = (const float *)c->usplit;
        }
    }
    a.Y = c->Y;
    a.ypart = c->ypart;
    a.err = c->dflag + 2;
    a.claim = c->claim;
    cudaEvent_t e0 = nullptr;
    HQ_TRY(prof_begin(c, 3, &e0));
    HQ_TRY(p.nm1 == 2 ? launch_hyb_nm1<2>(c, n, p, a, L) : launch_hyb_nm1<3>(c, n, p, a, L));
    HQ_TRY(prof_end(c, 3, e0));
    if (M.nspan > 0) {
        const size_t sm = (size_t)span_fix_ns(a.Pm) * a.Pm * sizeof(float);
        HQ_CUDA(smem_limit(k_span_fix, sm));
        k_span_fix<<<(unsigned)M.nspan, SF_THREADS, sm, c->stream>>>(M.span, M.lrow, M.item_aux, M.ipw, c->ypart,
                                                                      a.Pm, c->Y);
        c->nlaunch++;
    }
    HQ_CUDA(cudaGetLastError());
    return HOQRI_OK;
}

size_t hyb_smem_need(const hoqri_ctx *c, int n) {
    FastTile p;
    if (!hyb_tile(c, n, &p)) return (size_t)-1;
    return hyb_launch(c, n, p).smem;
}

size_t hyb_smem_cap() { return HY_SMEM_CAP; }

}  // namespace hoqri
