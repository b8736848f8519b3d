// Fiber-factored nonzero-stream pass (FP32): the rows y_i of Y_(n).
//
// Row i of X_(n) holds the nonzeros whose mode-n index is i (I^(n)_i, Table 1).
// Let l be the last of the other modes and the prefix the others before it
// (one mode for N = 3, two for N = 4).  The nonzeros of a row that share their
// prefix indices form a fiber f, and
//   y_i = sum_{z in I^(n)_i} x_z  (U_a(a_z) [(x) U_b(b_z)]) (x) U_l(l_z)     (Eq. ttmctc)
//       = sum_f  z_f (x) w_f,   z_f = U_a(a_f) [(x) U_b(b_f)],
//                               w_f = sum_{z in f} x_z U_l(l_z)
// (the Kronecker order of Eq. (2): the last mode fastest).  A fiber of L
// nonzeros costs L*K_l + P_{-n} multiply-adds and L + 1 gathered factor rows
// instead of L*P_{-n} and 2L: the same sum, grouped.
//
// Layout (built once per mode by build_fiber): the mode-n sorted stream itself
// (within a row the nonzeros are in lexicographic order of the other modes, so
// a fiber is a run of consecutive positions), cut into pieces of at most
// FB_LP nonzeros of one fiber, in stream order.  Per piece: first position,
// length | FB_HEAD (first piece of its row), prefix indices.  Warp t owns the
// contiguous piece range [prange[t], prange[t+1]) of about equal cost.
//
// A warp takes NG pieces at a time (a batch; its nonzeros are one contiguous
// run of the stream, at most NG * FB_LP long).  Every operand of a batch is
// brought to the warp's shared memory by cp.async in three stages, each
// started FB_S batches before the next needs it, so FB_S batches of copies are
// in flight while the warp computes:
//   stage A (batch k + 3 FB_S): the piece descriptors;
//   stage B (batch k + 2 FB_S): the run's indices and values;
//   stage C (batch k + FB_S):   the U_l rows of the run's nonzeros and the
//                               prefix rows of the pieces;
//   compute (batch k), from shared memory only:
//     phase 1: lane group g (K_l/4 lanes) sums w of piece g, a float4 per lane;
//     phase 2: every lane adds z_f (x) w_f of the batch's pieces into its TR x TC
//              tile of y_i (a K_pre x K_l matrix, row-major); at the first piece
//              of a row the finished row is stored.
// A row cut by a range boundary is stored in the range's slot 0 (the range's
// first row, begun in an earlier range) or slot 1 (its last row, continued in
// a later range); k_fib_span adds the pieces in range order.  No atomics and a
// fixed order: results are the same from run to run.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hoqri {

constexpr int FB_WARPS = 4;               // warps per CTA
constexpr int FB_LP = 4;                  // most nonzeros in a piece
constexpr int FB_PIECE_COST = 4;          // cost of a piece beyond its nonzeros (balance of ranges)
constexpr uint32_t FB_HEAD = 0x80000000u; // plenf bit: first piece of its row
constexpr int FB_S = 2;                   // batches between a stage's copy and its use
constexpr int FB_ND = 3 * FB_S + 1;       // descriptor slots (batches k .. k + 3 FB_S)
constexpr int FB_NS = 2 * FB_S + 1;       // index/value slots (batches k .. k + 2 FB_S)
constexpr int FB_NR = FB_S + 1;           // row slots (batches k .. k + FB_S)

struct FibArgs {
    const int32_t *lidx;    // [nnz] last other mode's index, mode-n sorted order
    const float *vals;      // [nnz]
    const int32_t *pstart;  // [np] first position of each piece
    const uint32_t *plenf;  // [np] length | FB_HEAD
    const int32_t *pa;      // [np] prefix index of the first prefix mode
    const int32_t *pb;      // [np] second prefix mode (N = 4; else pa)
    const int32_t *prange;  // [W+1]
    const int32_t *rrow0;   // [W] compact row of each range's first piece
    const float *Ua, *Ub, *Ul;  // prefix factors and the last other factor
    int KA, KB, lgKB;        // prefix ranks (N = 3: KB = 1)
    int W;                   // ranges (warps)
    int zs_floats;           // prefix floats per piece in shared memory (KA [+ KB])
    int warp_floats;         // shared memory per warp (4-byte words)
    int64_t np;
    float *Y;                // [R][P_{-n}]
    float *ypart;            // [W][2][P_{-n}]
};

template <int PP, int KL>
struct FibShape {
    static constexpr int PM = PP * KL;
    static constexpr int LPF = KL / 4;                        // lanes per piece in phase 1
    static constexpr int NG = 32 / LPF;                       // pieces per batch
    static constexpr int RUN = NG * FB_LP;                    // most nonzeros in a batch
    static constexpr int TC = (PM / 32) < 4 ? (PM / 32) : 4;  // tile columns per lane (phase 2)
    static constexpr int NCB = KL / TC;
    static constexpr int NRB = 32 / NCB;
    static constexpr int TR = PP / NRB;                       // tile rows per lane
    static_assert(PM >= 32 && KL >= 4 && TC >= 1 && NCB * NRB == 32 && TR * NRB == PP, "tile shape");
    // per-warp shared memory (4-byte words) before the prefix slots: descriptors
    // [ND][4][NG], indices/values [NS][2][RUN], rows [NR][RUN][KL], w [NG][KL]
    static constexpr int OFF_S = FB_ND * 4 * NG;
    static constexpr int OFF_R = OFF_S + FB_NS * 2 * RUN;
    static constexpr int OFF_W = OFF_R + FB_NR * RUN * KL;
    static constexpr int OFF_P = OFF_W + NG * KL;             // prefix [NR][NG][zs_floats]
    static_assert(OFF_S % 4 == 0 && OFF_R % 4 == 0 && OFF_W % 4 == 0 && OFF_P % 4 == 0, "16-byte slots");
};

// shared memory words per warp of k_fib<., PP, KL> with zs prefix floats per piece
template <int PP, int KL>
constexpr int fib_warp_floats(int zs) {
    return FibShape<PP, KL>::OFF_P + FB_NR * FibShape<PP, KL>::NG * zs;
}

__device__ __forceinline__ uint32_t fb_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void fb_cp16(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(fb_smem(dst)), "l"(src) : "memory");
}

// 4 bytes, or 4 zero bytes when !valid (src is then not read)
__device__ __forceinline__ void fb_cp4(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(fb_smem(dst)), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}

__device__ __forceinline__ void fb_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// every group but the newest FB_S - 1 has landed (for this thread)
__device__ __forceinline__ void fb_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(FB_S - 1) : "memory"); }

__device__ __forceinline__ void fb_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int NM1, int PP, int KL>
__global__ void __launch_bounds__(FB_WARPS * 32) k_fib(FibArgs a) {
    using S = FibShape<PP, KL>;
    constexpr int PM = S::PM, LPF = S::LPF, NG = S::NG, RUN = S::RUN, TC = S::TC, TR = S::TR, NCB = S::NCB;
    constexpr int CPR = KL / 4;  // float4 per U_l row
    extern __shared__ __align__(16) float fsm[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int t = blockIdx.x * FB_WARPS + wid;
    if (t >= a.W) return;
    const int32_t p0 = a.prange[t], p1 = a.prange[t + 1];
    if (p0 >= p1) return;
    float *wsm = fsm + (size_t)wid * a.warp_floats;
    int32_t *Dsm = reinterpret_cast<int32_t *>(wsm);    // [ND][4][NG]: st, lf, pa, pb
    int32_t *Ssm = reinterpret_cast<int32_t *>(wsm + S::OFF_S);  // [NS][2][RUN]: idx, value bits
    float *Rsm = wsm + S::OFF_R;                        // [NR][RUN][KL]
    float *Wsm = wsm + S::OFF_W;                        // [NG][KL]
    float *Psm = wsm + S::OFF_P;                        // [NR][NG][zs]
    const int zs = a.zs_floats;
    const int g = lane / LPF, c = lane - g * LPF;       // phase 1: piece g, float4 c of U_l
    const int r0 = (lane / NCB) * TR, c0 = (lane % NCB) * TC;  // phase 2 tile
    const int nbatch = (p1 - p0 + NG - 1) / NG;
    int32_t j = a.rrow0[t];
    const bool cut_start = !(a.plenf[p0] & FB_HEAD);
    const bool cut_end = p1 < a.np && !(a.plenf[p1] & FB_HEAD);
    bool first = true;

    float2 acc[TR][(TC + 1) / 2];
    auto zero_acc = [&]() {
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int q = 0; q < (TC + 1) / 2; ++q) acc[r][q] = make_float2(0.f, 0.f);
    };
    auto flush = [&](bool last) {
        float *dst;
        if (first && cut_start) dst = a.ypart + ((size_t)t * 2) * PM;
        else if (last && cut_end) dst = a.ypart + ((size_t)t * 2 + 1) * PM;
        else dst = a.Y + (size_t)j * PM;
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            float *p = dst + (size_t)(r0 + r) * KL + c0;
            if constexpr (TC == 4)
                *reinterpret_cast<float4 *>(p) = make_float4(acc[r][0].x, acc[r][0].y, acc[r][1].x, acc[r][1].y);
            else if constexpr (TC == 2)
                *reinterpret_cast<float2 *>(p) = acc[r][0];
            else
                p[0] = acc[r][0].x;
        }
    };
    zero_acc();
    // pieces of batch b: [p0 + b*NG, p0 + b*NG + nb(b))
    auto nb_of = [&](int b) { return min(NG, p1 - (p0 + b * NG)); };
    // the nonzero run of batch b (its descriptors in slot b % ND): [first start, last start + last length)
    auto run_of = [&](int b, int32_t &rs, int &rl) {
        const int32_t *D = Dsm + (b % FB_ND) * 4 * NG;
        const int last = nb_of(b) - 1;
        rs = D[0];
        rl = D[last] + (int)((uint32_t)D[NG + last] & 0xffffu) - rs;
    };

    for (int k = -3 * FB_S; k < nbatch; ++k) {
        fb_wait();
        __syncwarp();
        // ---- stage A: descriptors of batch k + 3 FB_S
        {
            const int b = k + 3 * FB_S;
            if (b < nbatch && lane < NG) {
                int32_t *D = Dsm + (b % FB_ND) * 4 * NG;
                const int32_t p = p0 + b * NG + lane;
                const bool v = p < p1;
                const int32_t ps = v ? p : p0;
                fb_cp4(D + lane, a.pstart + ps, v);
                fb_cp4(D + NG + lane, a.plenf + ps, v);
                fb_cp4(D + 2 * NG + lane, a.pa + ps, v);
                if constexpr (NM1 == 3) fb_cp4(D + 3 * NG + lane, a.pb + ps, v);
            }
        }
        // ---- stage B: indices and values of batch k + 2 FB_S
        {
            const int b = k + 2 * FB_S;
            if (b >= 0 && b < nbatch) {
                int32_t rs;
                int rl;
                run_of(b, rs, rl);
                int32_t *Sx = Ssm + (b % FB_NS) * 2 * RUN;
                for (int q = lane; q < rl; q += 32) {
                    fb_cp4(Sx + q, a.lidx + rs + q, true);
                    fb_cp4(Sx + RUN + q, a.vals + rs + q, true);
                }
            }
        }
        // ---- stage C: U_l rows and prefix rows of batch k + FB_S
        {
            const int b = k + FB_S;
            if (b >= 0 && b < nbatch) {
                int32_t rs;
                int rl;
                run_of(b, rs, rl);
                const int32_t *Sx = Ssm + (b % FB_NS) * 2 * RUN;
                float *Rx = Rsm + (b % FB_NR) * RUN * KL;
                for (int q = lane; q < rl * CPR; q += 32) {
                    const int e = q / CPR, cc = q - e * CPR;
                    fb_cp16(Rx + e * KL + 4 * cc, a.Ul + (size_t)Sx[e] * KL + 4 * cc);
                }
                const int32_t *D = Dsm + (b % FB_ND) * 4 * NG;
                float *Px = Psm + (b % FB_NR) * NG * zs;
                const int nbb = nb_of(b);
                if constexpr (NM1 == 2) {
                    constexpr int QPR = PP / 4;
                    for (int q = lane; q < nbb * QPR; q += 32) {
                        const int gg = q / QPR, qq = q - gg * QPR;
                        fb_cp16(Px + gg * PP + 4 * qq, a.Ua + (size_t)D[2 * NG + gg] * PP + 4 * qq);
                    }
                } else {
                    const int qa = a.KA >> 2, qr = qa + (a.KB >> 2);
                    for (int q = lane; q < nbb * qr; q += 32) {
                        const int gg = q / qr, qq = q - gg * qr;
                        const float *src = qq < qa ? a.Ua + (size_t)D[2 * NG + gg] * a.KA + 4 * qq
                                                   : a.Ub + (size_t)D[3 * NG + gg] * a.KB + 4 * (qq - qa);
                        fb_cp16(Px + gg * zs + 4 * qq, src);
                    }
                }
            }
        }
        fb_commit();
        if (k < 0) continue;
        // ---- compute batch k
        const int nb = nb_of(k);
        const int32_t *D = Dsm + (k % FB_ND) * 4 * NG;
        const int32_t *Sx = Ssm + (k % FB_NS) * 2 * RUN;
        const float *Rx = Rsm + (k % FB_NR) * RUN * KL;
        const float *Px = Psm + (k % FB_NR) * NG * zs;
        {
            // phase 1: w of piece g (lanes of pieces past the range add nothing)
            const int32_t rs = D[0];
            const int off = D[g] - rs;
            const int len = g < nb ? (int)((uint32_t)D[NG + g] & 0xffffu) : 0;
            float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int u = 0; u < len; ++u) {
                const float x = __int_as_float(Sx[RUN + off + u]);
                const float4 r = *reinterpret_cast<const float4 *>(Rx + (off + u) * KL + 4 * c);
                w.x = fmaf(x, r.x, w.x);
                w.y = fmaf(x, r.y, w.y);
                w.z = fmaf(x, r.z, w.z);
                w.w = fmaf(x, r.w, w.w);
            }
            *reinterpret_cast<float4 *>(Wsm + g * KL + 4 * c) = w;
        }
        __syncwarp();
        // phase 2: y += z_f (x) w_f over the batch, rows stored at row starts
        const uint32_t heads = __ballot_sync(0xffffffffu, lane < nb && ((uint32_t)D[NG + min(lane, NG - 1)] & FB_HEAD));
        for (int gg = 0; gg < nb; ++gg) {
            if (((heads >> gg) & 1u) && p0 + k * NG + gg > p0) {
                flush(false);
                first = false;
                ++j;
                zero_acc();
            }
            float z[TR];
            if constexpr (NM1 == 2) {
                const float *zp = Px + gg * PP + r0;
                if constexpr (TR % 4 == 0) {
#pragma unroll
                    for (int r = 0; r < TR; r += 4) {
                        const float4 v = *reinterpret_cast<const float4 *>(zp + r);
                        z[r] = v.x;
                        z[r + 1] = v.y;
                        z[r + 2] = v.z;
                        z[r + 3] = v.w;
                    }
                } else if constexpr (TR == 2) {
                    const float2 v = *reinterpret_cast<const float2 *>(zp);
                    z[0] = v.x;
                    z[1] = v.y;
                } else {
#pragma unroll
                    for (int r = 0; r < TR; ++r) z[r] = zp[r];
                }
            } else {
                const float *za = Px + gg * zs;
                const float *zb = za + a.KA;
#pragma unroll
                for (int r = 0; r < TR; ++r) {
                    const int rr = r0 + r;
                    z[r] = za[rr >> a.lgKB] * zb[rr & (a.KB - 1)];
                }
            }
            const float *wp = Wsm + gg * KL + c0;
            if constexpr (TC >= 2) {
                float2 wv[(TC + 1) / 2];
#pragma unroll
                for (int q = 0; q < TC / 2; ++q) wv[q] = *reinterpret_cast<const float2 *>(wp + 2 * q);
#pragma unroll
                for (int r = 0; r < TR; ++r) {
                    const float2 zz = make_float2(z[r], z[r]);
#pragma unroll
                    for (int q = 0; q < TC / 2; ++q) acc[r][q] = __ffma2_rn(zz, wv[q], acc[r][q]);
                }
            } else {
                const float wv = wp[0];
#pragma unroll
                for (int r = 0; r < TR; ++r) acc[r][0].x = fmaf(z[r], wv, acc[r][0].x);
            }
        }
        __syncwarp();  // every lane is done with batch k's slots before they are refilled
    }
    fb_wait_all();
    flush(true);
}

// Rows cut by range boundaries: Y[j] = slot 1 of range t0 + slot 0 of ranges
// t0+1 .. t1, added in that order in FP64 (one CTA per cut row).
__global__ void __launch_bounds__(256) k_fib_span(const int32_t *span, const float *ypart, int Pm, float *Y);

}  // namespace hoqri
