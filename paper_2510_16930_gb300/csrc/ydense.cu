// Dense products over the stored rows of Y_(n) (the R_n x P_{-n} buffer the
// nonzero-stream pass of hybrid.cu writes):
//   A_n = Y_(n) G_(n)^T   (the TTMcTC output, Eq. ttmctc)
//   G_(n) = U_n^T Y_(n)   (the core after the QR of mode n, Sec. 2.2; Alg. 3 first step)
// Both stream Y once; the core is left as per-CTA partials that k_core_reduce
// adds in a fixed order.
#include <algorithm>

#include "internal.cuh"

namespace hoqri {

namespace {

__device__ __forceinline__ int64_t ceil_div_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }

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

// 16-byte global -> shared copies that bypass L1 (cp.async, grouped and waited
// on per thread; a __syncthreads after the wait makes every thread's copies visible)
__device__ __forceinline__ void cp16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int KN>
__host__ __device__ constexpr int ay_rt() { return KN >= 32 ? 1 : 2; }  // rows per thread (KN = 32: registers)

// acc[i][:] += sum over e' in [e, e + 4) of yv[i](e' - e) G_(n)(:, e'), in
// increasing e' (Gt = G_(n) transposed, [e][kn])
template <int KN, int AY_RT>
__device__ __forceinline__ void ay_step(const float *Gt, int e, const float4 (&yv)[AY_RT],
                                        float2 (&acc)[AY_RT][KN / 2]) {
#pragma unroll
    for (int ee = 0; ee < 4; ++ee) {
        const float4 *g4 = reinterpret_cast<const float4 *>(Gt + (size_t)(e + ee) * KN);
#pragma unroll
        for (int k4 = 0; k4 < KN / 4; ++k4) {
            const float4 g = g4[k4];
#pragma unroll
            for (int i = 0; i < AY_RT; ++i) {
                const float yy = ee == 0 ? yv[i].x : (ee == 1 ? yv[i].y : (ee == 2 ? yv[i].z : yv[i].w));
                const float2 y2 = make_float2(yy, yy);
                acc[i][2 * k4] = __ffma2_rn(y2, make_float2(g.x, g.y), acc[i][2 * k4]);
                acc[i][2 * k4 + 1] = __ffma2_rn(y2, make_float2(g.z, g.w), acc[i][2 * k4 + 1]);
            }
        }
    }
}

// A(row_id[r], :) = G_(n) y_r for KN = K_n in {4, 8, 16, 32} and P_{-n} a
// multiple of 16.  Each CTA takes a contiguous range of rows (equal ranges, one
// wave of CTAs) in tiles of AY_RB = 256 * ay_rt rows; a thread owns ay_rt rows
// of the tile and all KN outputs of each.  The tile's columns arrive in chunks
// of AY_EC: every chunk is copied into shared memory by coalesced cp.async
// (whole 64-byte row pieces, rows padded to AY_LD floats so that consecutive
// threads read their rows without bank conflicts), AY_NS - 1 chunks ahead of
// the one being multiplied; G_(n) is staged transposed ([e][kn]) once and read
// as broadcasts.  Each output is summed over e in increasing order.
constexpr int AY_EC = 16;
constexpr int AY_LD = AY_EC + 4;
constexpr int AY_NS = 3;

template <int KN>
__host__ __device__ constexpr int ay_rb() { return 256 * ay_rt<KN>(); }

template <int KN>
__global__ void __launch_bounds__(256, 1) k_a_from_y2(const float *Y, const float *Gn, const int32_t *row_id,
                                                      int64_t R, int64_t rpb, int Pm, float *A) {
    constexpr int RT = ay_rt<KN>();
    constexpr int RB = ay_rb<KN>();
    extern __shared__ __align__(16) float dsm[];
    float *Gt = dsm;                 // [Pm][KN]
    float *Ys = dsm + (size_t)Pm * KN;  // [AY_NS][RB][AY_LD]
    // Gt[e][k] = G_(n)(k, e): reads along e (coalesced), eight in flight per thread
    for (int t0 = 0; t0 < Pm * KN; t0 += 8 * 256) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int t = t0 + u * 256 + (int)threadIdx.x;
            v[u] = t < Pm * KN ? __ldg(Gn + t) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int t = t0 + u * 256 + (int)threadIdx.x;
            if (t < Pm * KN) {
                const int k = t / Pm, e = t - k * Pm;
                Gt[e * KN + k] = v[u];
            }
        }
    }
    const int64_t rbeg = (int64_t)blockIdx.x * rpb, rend = min(rbeg + rpb, R);
    const int nch = Pm / AY_EC;
    const int64_t nsteps = rend > rbeg ? ceil_div_dev(rend - rbeg, (int64_t)RB) * nch : 0;
    // step s = (tile s / nch, column chunk s % nch) into buffer s % AY_NS
    auto issue = [&](int64_t s) {
        if (s < nsteps) {
            const int64_t tile = s / nch;
            const int ch = (int)(s - tile * nch);
            const int64_t r0 = rbeg + tile * RB;
            const int nr = (int)min((int64_t)RB, rend - r0);
            float *dst = Ys + (size_t)(s % AY_NS) * RB * AY_LD;
            const float *src = Y + (size_t)r0 * Pm + (size_t)ch * AY_EC;
            for (int q = threadIdx.x; q < nr * (AY_EC / 4); q += blockDim.x) {
                const int rr = q / (AY_EC / 4), c = q - rr * (AY_EC / 4);
                cp16(dst + rr * AY_LD + 4 * c, src + (size_t)rr * Pm + 4 * c);
            }
        }
        cp_commit();
    };
#pragma unroll
    for (int s = 0; s < AY_NS - 1; ++s) issue(s);
    float2 acc[RT][KN / 2];
    for (int64_t s = 0; s < nsteps; ++s) {
        issue(s + AY_NS - 1);
        cp_wait<AY_NS - 1>();
        __syncthreads();  // this step's chunk (and, at s = 0, Gt) visible to every thread
        const int64_t tile = s / nch;
        const int ch = (int)(s - tile * nch);
        if (ch == 0) {
#pragma unroll
            for (int i = 0; i < RT; ++i)
#pragma unroll
                for (int k = 0; k < KN / 2; ++k) acc[i][k] = make_float2(0.f, 0.f);
        }
        const float *ys = Ys + (size_t)(s % AY_NS) * RB * AY_LD;
        if (RT == 1 || rend - (rbeg + tile * RB) > 256) {
#pragma unroll
            for (int e4 = 0; e4 < AY_EC / 4; ++e4) {
                float4 yv[RT];
#pragma unroll
                for (int i = 0; i < RT; ++i)
                    yv[i] = *reinterpret_cast<const float4 *>(ys + (size_t)(threadIdx.x + 256 * i) * AY_LD + 4 * e4);
                ay_step<KN, RT>(Gt, ch * AY_EC + 4 * e4, yv, acc);
            }
        } else {
            // a tile of at most 256 rows: one row per thread
            float2(&acc1)[1][KN / 2] = *reinterpret_cast<float2(*)[1][KN / 2]>(&acc[0]);
#pragma unroll
            for (int e4 = 0; e4 < AY_EC / 4; ++e4) {
                float4 yv[1];
                yv[0] = *reinterpret_cast<const float4 *>(ys + (size_t)threadIdx.x * AY_LD + 4 * e4);
                ay_step<KN, 1>(Gt, ch * AY_EC + 4 * e4, yv, acc1);
            }
        }
        if (ch == nch - 1) {
            const int64_t r0 = rbeg + tile * RB;
#pragma unroll
            for (int i = 0; i < RT; ++i) {
                const int64_t r = r0 + threadIdx.x + 256 * i;
                if (r >= rend) break;
                float2 *arow = reinterpret_cast<float2 *>(A + (size_t)row_id[r] * KN);
#pragma unroll
                for (int k = 0; k < KN / 2; ++k) arow[k] = acc[i][k];
            }
        }
        __syncthreads();  // buffer s % AY_NS is refilled by the next iteration's issue
    }
    cp_wait<0>();
}

// CTA partials of G_(n)[kn][e] = sum_r U_n(row_id[r], kn) Y[r][e] for KN in
// {4, 8, 16, 32} and P_{-n} <= 1024: Pm/4 threads cover a row (4 columns of e
// each, all KN rows of G), the block's ng = 1024 / Pm row groups take every
// ng-th row of the CTA's range (row r to group (r - r0) mod ng, each group in
// increasing r), and the groups are added in group order at the end.  Chunks of
// ch rows (a multiple of ng) of Y and their U rows are copied into shared
// memory by cp.async, CY_NS - 1 chunks ahead of the one being multiplied; the
// rows of a chunk are contiguous in Y, so the copies are fully coalesced.
constexpr int CY_NS = 3;

__host__ __device__ constexpr int cy_rows(int Pm) {
    const int ng = 1024 / Pm;
    const int c = 8192 / Pm < 32 ? 8192 / Pm : 32;
    return c > ng ? c : ng;
}

template <int KN>
__global__ void __launch_bounds__(256, KN >= 32 ? 1 : 2) k_core_from_y2(const float *Y, const float *Un, const int32_t *row_id, int64_t R,
                                                         int Pm, int64_t rpb, float *cpart) {
    extern __shared__ __align__(16) float csm[];  // [CY_NS][ch * (Pm + KN)]; after the loop [ng][KN * Pm]
    const int tpr = Pm >> 2;
    const int ng = blockDim.x / tpr;
    const int gi = threadIdx.x / tpr, eq = threadIdx.x - gi * tpr;
    const int KnPm = KN * Pm;
    const int CH = cy_rows(Pm);
    const int stage_f = CH * (Pm + KN);
    const int64_t r0 = (int64_t)blockIdx.x * rpb, r1 = min(r0 + rpb, R);
    const int64_t nst = r1 > r0 ? ceil_div_dev(r1 - r0, (int64_t)CH) : 0;
    // U copies of a chunk: q = threadIdx.x + 256 u < nr * KN / 4 (row q / (KN / 4));
    // their row ids are loaded one iteration before the copies are issued, so
    // the issue does not wait on them (chunks hold at most 256 rows: KN / 4 per thread)
    constexpr int UPT = KN / 4;
    int rid[UPT];
    auto load_rids = [&](int64_t s) {
        const int64_t rb = r0 + s * CH;
        const int nq = s < nst ? (int)min((int64_t)CH, r1 - rb) * (KN / 4) : 0;
#pragma unroll
        for (int u = 0; u < UPT; ++u) {
            const int q = threadIdx.x + 256 * u;
            rid[u] = q < nq ? row_id[rb + q / (KN / 4)] : 0;
        }
    };
    auto issue = [&](int64_t s) {
        if (s < nst) {
            const int64_t rb = r0 + s * CH;
            const int nr = (int)min((int64_t)CH, r1 - rb);
            float *ys = csm + (size_t)(s % CY_NS) * stage_f;
            float *us = ys + (size_t)CH * Pm;
            const float *src = Y + (size_t)rb * Pm;
            for (int q = threadIdx.x; q < nr * tpr; q += blockDim.x) cp16(ys + 4 * q, src + 4 * q);
#pragma unroll
            for (int u = 0; u < UPT; ++u) {
                const int q = threadIdx.x + 256 * u;
                if (q < nr * (KN / 4)) {
                    const int rr = q / (KN / 4), c = q - rr * (KN / 4);
                    cp16(us + rr * KN + 4 * c, Un + (size_t)rid[u] * KN + 4 * c);
                }
            }
        }
        cp_commit();
    };
#pragma unroll
    for (int s = 0; s < CY_NS - 1; ++s) {
        load_rids(s);
        issue(s);
    }
    load_rids(CY_NS - 1);
    float2 acc[KN][2];  // acc[k] = G(k, 4 eq .. 4 eq + 3) as two pairs
#pragma unroll
    for (int k = 0; k < KN; ++k) acc[k][0] = acc[k][1] = make_float2(0.f, 0.f);
    for (int64_t s = 0; s < nst; ++s) {
        issue(s + CY_NS - 1);
        load_rids(s + CY_NS);
        cp_wait<CY_NS - 1>();
        __syncthreads();
        const int nr = (int)min((int64_t)CH, r1 - (r0 + s * CH));
        const float *ys = csm + (size_t)(s % CY_NS) * stage_f;
        const float4 *us = reinterpret_cast<const float4 *>(ys + (size_t)CH * Pm);
        if (gi < ng) {
            for (int j = gi; j < nr; j += ng) {
                const float4 y = reinterpret_cast<const float4 *>(ys + (size_t)j * Pm)[eq];
                const float2 ylo = make_float2(y.x, y.y), yhi = make_float2(y.z, y.w);
#pragma unroll
                for (int kq = 0; kq < KN / 4; ++kq) {
                    const float4 uq = us[j * (KN / 4) + kq];
                    const float uu[4] = {uq.x, uq.y, uq.z, uq.w};
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float2 u2 = make_float2(uu[c], uu[c]);
                        acc[4 * kq + c][0] = __ffma2_rn(u2, ylo, acc[4 * kq + c][0]);
                        acc[4 * kq + c][1] = __ffma2_rn(u2, yhi, acc[4 * kq + c][1]);
                    }
                }
            }
        }
        __syncthreads();
    }
    cp_wait<0>();
    __syncthreads();
    float *red = csm;
    if (gi < ng) {
#pragma unroll
        for (int k = 0; k < KN; ++k)
            reinterpret_cast<float4 *>(red + (size_t)gi * KnPm + (size_t)k * Pm)[eq] =
                make_float4(acc[k][0].x, acc[k][0].y, acc[k][1].x, acc[k][1].y);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < KnPm; p += blockDim.x) {
        float s = 0.f;
        for (int q = 0; q < ng; ++q) s += red[(size_t)q * KnPm + p];
        cpart[(size_t)blockIdx.x * KnPm + p] = s;
    }
}

}  // namespace

// A_n = Y_(n) G_(n)^T from the stored rows (Gn: G_(n) as [Kn][Pm] on the device,
// over the padded columns when the mode's plan is padded).
hoqri_status hyb_a_from_y(hoqri_ctx *c, int n, const float *Gn, float *A_out) {
    const ModeStore &M = c->ms[n];
    const int Kn = c->K[n];
    FastTile pl;
    const int Pm = hyb_tile(c, n, &pl) ? pl.Pm : (int)(c->P / Kn);
    const int Knp = (Kn + 3) & ~3;
    const int RT = std::min(256, 4 * (256 / (Knp / 4)));
    const int EC = Pm < 32 ? Pm : 32;
    const size_t smem = ((size_t)EC * (RT + 4) + (size_t)EC * Knp) * sizeof(float);
    HQ_CUDA(cudaMemsetAsync(A_out, 0, (size_t)c->dims[n] * Kn * sizeof(float), c->stream));
    if (M.R > 0 && (Kn == 4 || Kn == 8 || Kn == 16 || Kn == 32) && Pm % AY_EC == 0 &&
        (size_t)Pm * Kn * 4 <= 96 * 1024) {
        // one wave of CTAs (as many as are resident at once) with equal row ranges
#define HQ_AY(KV)                                                                                              \
    if (Kn == KV) {                                                                                            \
        const size_t sm2 = ((size_t)Pm * KV + (size_t)AY_NS * ay_rb<KV>() * AY_LD) * sizeof(float);            \
        HQ_CUDA(smem_limit(k_a_from_y2<KV>, sm2)); \
        int per_sm = 1;                                                                                        \
        HQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_a_from_y2<KV>, 256, sm2));            \
        const int g2 = (int)std::max<int64_t>(                                                                 \
            1, std::min<int64_t>(ceil_div(M.R, 256), (int64_t)c->num_sms * std::max(1, per_sm)));              \
        const int64_t rpb2 = ceil_div(M.R, g2);                                                                \
        k_a_from_y2<KV><<<g2, 256, sm2, c->stream>>>(c->Y, Gn, M.row_id, M.R, rpb2, Pm, A_out);              \
    }
        HQ_AY(4)
        HQ_AY(8)
        HQ_AY(16)
        HQ_AY(32)
#undef HQ_AY
        c->nlaunch++;
    } else if (M.R > 0) {
        HQ_CUDA(smem_limit(k_a_from_y, smem));
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
    FastTile pl;
    const int Pm = hyb_tile(c, n, &pl) ? pl.Pm : (int)(c->P / Kn);
    const int Knp = (Kn + 3) & ~3;
    const int64_t R = M.R;
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(R, 1), 256),
                                                          (int64_t)c->num_sms * 2));
    int64_t rpb = ceil_div(std::max<int64_t>(R, 1), grid);
    const size_t cy_smem = (Pm >= 4 && Pm <= 1024)
                               ? std::max((size_t)CY_NS * cy_rows(Pm) * (Pm + Kn), (size_t)(1024 / Pm) * Kn * Pm) *
                                     sizeof(float)
                               : 0;
    if ((Kn == 4 || Kn == 8 || Kn == 16 || Kn == 32) && Pm % 4 == 0 && Pm <= 1024 && 1024 % Pm == 0 &&
        cy_smem <= 200 * 1024) {
        // one wave: as many CTAs as are resident at once (at most 2 per SM)
#define HQ_CY(KV)                                                                                                    \
    if (Kn == KV) {                                                                                                  \
        HQ_CUDA(smem_limit(k_core_from_y2<KV>, cy_smem)); \
        int per_sm = 1;                                                                                              \
        HQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_core_from_y2<KV>, 256, cy_smem));           \
        grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(R, 1), 256),                  \
                                                           (int64_t)c->num_sms * std::min(2, std::max(1, per_sm))));     \
        rpb = ceil_div(std::max<int64_t>(R, 1), grid);                                                               \
        k_core_from_y2<KV><<<grid, 256, cy_smem, c->stream>>>(c->Y, (const float *)c->U[n], M.row_id, R, Pm, rpb,    \
                                                              (float *)c->core_part);                                \
    }
        HQ_CY(4)
        HQ_CY(8)
        HQ_CY(16)
        HQ_CY(32)
#undef HQ_CY
    } else {
        const size_t smem = (size_t)64 * Knp * sizeof(float);
        k_core_from_y<<<grid, 256, smem, c->stream>>>(c->Y, (const float *)c->U[n], M.row_id, R, Kn, Knp, Pm, rpb,
                                                      (float *)c->core_part);
    }
    c->nlaunch++;
    HQ_CUDA(cudaGetLastError());
    *nblk = grid;
    return HOQRI_OK;
}

}  // namespace hoqri
