// Orthonormalisation U_n <- orthonormal basis of A_n (Alg. 2, the QR step).
//
// CholeskyQR2: W = A^T A (Gram, FP64 sums in a fixed order; for an FP32 A
// double-float sums on the FP32 pipes, see k_gram_df), W = R^T R (Cholesky in
// one CTA, FP64 for an FP64 A, double-float for an FP32 A: k_chol_df),
// A <- A R^{-1} (row-wise substitution); then once more on the result.
// Both R factors have a positive diagonal, so the result is the Q of the thin
// QR with diag(R) > 0.  A_n = Y_(n) G_(n)^T with G_(n) = U_n^T Y_(n) squares
// the conditioning of Y_(n), so a first pivot that is not clearly positive is
// common on skewed data: then the first Cholesky is taken of W + s I instead
// (shifted CholeskyQR3, Fukaya, Kannan, Nakatsukasa, Yamamoto and Yanagisawa,
// SIAM J. Sci. Comput. 42(1), 2020: s = 11 (m n + n (n + 1)) u ||A||^2, with
// ||A||_F^2 = trace(W) for ||A||_2^2), which leaves A R^{-1} well enough
// conditioned for the two unshifted passes that follow.  When a pivot of a
// later pass is not clearly positive (A is rank deficient), a one-CTA
// Householder QR in FP64 produces Q instead (columns signed so diag(R) >= 0;
// zero pivot columns are completed by the accumulated reflectors).  The
// decisions are taken on the device through flags, so the sequence needs no
// host round trip and can be captured in a CUDA graph:
//   flag[0] = 0  -> the CholeskyQR kernels run;
//   flag[0] = 1  -> breakdown seen; the Householder kernel runs and sets 2;
//   flag[0] = 2  -> U is written; every later kernel of this QR returns at once;
//   flag[1]      -> breakdowns counted over the context's life;
//   flag[3] = 1  -> the first pass was shifted: the third pass runs (else its
//                   kernels return at once).
#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace hoqri {

namespace {

constexpr int GRAM_TPB = 256;
constexpr int GRAM_ROWS = 32;   // rows staged per step
constexpr int MAX_GRAM_BLOCKS = 304;
constexpr int HH_TPB = 1024;
constexpr int QR_PASSES = 3;  // the third runs only after a shifted first pass

// true when the kernels of this pass have nothing to do (see the flag states)
__device__ __forceinline__ bool qr_skip(const int32_t *flag, int pass) {
    return flag[0] != 0 || (pass == 2 && flag[3] == 0);
}

template <typename T>
__global__ void __launch_bounds__(GRAM_TPB) k_gram_partial(const T *A, int64_t I, int K, int64_t rows_per_block,
                                                           double *part, const int32_t *flag, int pass) {
    if (qr_skip(flag, pass)) return;
    __shared__ double tile[GRAM_ROWS * HOQRI_MAXK];
    const int npairs = K * (K + 1) / 2;
    constexpr int MAXP = (HOQRI_MAXK * (HOQRI_MAXK + 1) / 2 + GRAM_TPB - 1) / GRAM_TPB;
    double acc[MAXP];
    int pi[MAXP], pj[MAXP];
#pragma unroll
    for (int q = 0; q < MAXP; ++q) {
        acc[q] = 0.0;
        int p = threadIdx.x + q * GRAM_TPB;
        int i = 0, j = 0;
        if (p < npairs) {
            // pair p -> (i, j), i <= j, row-major over the upper triangle
            int rem = p;
            i = 0;
            while (rem >= K - i) {
                rem -= K - i;
                ++i;
            }
            j = i + rem;
        }
        pi[q] = i;
        pj[q] = j;
    }
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(r0 + rows_per_block, I);
    for (int64_t rb = r0; rb < r1; rb += GRAM_ROWS) {
        const int nr = (int)min((int64_t)GRAM_ROWS, r1 - rb);
        __syncthreads();
        for (int t = threadIdx.x; t < nr * K; t += GRAM_TPB) tile[t] = (double)A[rb * K + t];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < MAXP; ++q) {
            if (threadIdx.x + q * GRAM_TPB < npairs) {
                double s = acc[q];
                for (int r = 0; r < nr; ++r) s += tile[r * K + pi[q]] * tile[r * K + pj[q]];
                acc[q] = s;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < MAXP; ++q) {
        int p = threadIdx.x + q * GRAM_TPB;
        if (p < npairs) part[(size_t)blockIdx.x * npairs + p] = acc[q];
    }
}

// ---- double-float arithmetic (a value is hi + lo, two FP32 numbers): the
// Gram of an FP32 A on the FP32 pipes, which run 64 times as many
// multiply-adds per clock as the FP64 pipe of this GPU.  Intrinsics with
// explicit rounding keep the compiler from fusing the error terms away.
// TwoSum (Knuth, TAOCP vol. 2, 4.2.2): a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

// (hi, lo) += a b: the product split exactly by an FMA (TwoProduct), its high
// part added to hi by TwoSum, both error terms to lo (the Dot2 step of Ogita,
// Rump and Oishi, SIAM J. Sci. Comput. 26(6), 2005)
__device__ __forceinline__ void df_fma(float a, float b, float &hi, float &lo) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    float s, q;
    two_sum(hi, p, s, q);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(q, e));
}

// (hi, lo) += (bh, bl), renormalised so that lo is below half an ulp of hi
__device__ __forceinline__ void df_add(float &hi, float &lo, float bh, float bl) {
    float s, q;
    two_sum(hi, bh, s, q);
    q = __fadd_rn(q, __fadd_rn(lo, bl));
    two_sum(s, q, hi, lo);
}

constexpr int DF_ROWS = 256;  // rows staged per step; each row stream's level-1 sum spans one step

template <int KC, int TS>
struct DfShape {
    static constexpr int NTB = KC / TS;                // tile rows and columns
    static constexpr int NT = NTB * (NTB + 1) / 2;     // tiles on and above the diagonal
    static constexpr int S = GRAM_TPB / NT;            // row streams per tile
    static constexpr int NP = KC * (KC + 1) / 2;       // Gram entries i <= j
    static constexpr int TILE_B = DF_ROWS * KC * 4;
    static constexpr int RED_B = S * NT * TS * TS * 8;
    static constexpr int SMEM_B = TILE_B > RED_B ? TILE_B : RED_B;
};

// Gram partials W(i, j) = sum over the CTA's rows of A(r, i) A(r, j), i <= j,
// for an FP32 A with KC in {4, 8, 16, 32} columns (16-byte aligned rows), in
// double-float: thread = (TS x TS tile of W on or above the diagonal, row
// stream); a stream's products over one staged step of DF_ROWS rows are summed
// in a level-1 pair (Dot2), which is then added to a level-2 pair, so no
// running sum spans more than about 40 products; the streams are added in
// stream order at the end.  part: [block][pair] as (hi, lo).
template <int KC, int TS>
__global__ void __launch_bounds__(GRAM_TPB) k_gram_df(const float *A, int64_t I, int64_t rows_per_block,
                                                      float2 *part, const int32_t *flag, int pass) {
    using D = DfShape<KC, TS>;
    if (qr_skip(flag, pass)) return;
    __shared__ __align__(16) unsigned char smem[D::SMEM_B];
    float *tile = reinterpret_cast<float *>(smem);
    const int t = threadIdx.x, tid = t % D::NT, st = t / D::NT;
    const bool active = st < D::S;
    int ti = 0, rem = tid;
    while (rem >= D::NTB - ti) {
        rem -= D::NTB - ti;
        ++ti;
    }
    const int tj = ti + rem;
    float h2[TS][TS], l2[TS][TS];
#pragma unroll
    for (int u = 0; u < TS; ++u)
#pragma unroll
        for (int v = 0; v < TS; ++v) h2[u][v] = l2[u][v] = 0.f;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(r0 + rows_per_block, I);
    // the rows of the next step are loaded into registers while this step's
    // products run (LPT 16-byte vectors per thread)
    constexpr int LPT = DF_ROWS * KC / 4 / GRAM_TPB;
    float4 pf[LPT];
    auto load_step = [&](int64_t rb) {
        const int nq = rb < r1 ? (int)min((int64_t)DF_ROWS, r1 - rb) * (KC / 4) : 0;
        const float4 *src = reinterpret_cast<const float4 *>(A + rb * KC);
#pragma unroll
        for (int u = 0; u < LPT; ++u) {
            const int q = t + u * GRAM_TPB;
            pf[u] = q < nq ? __ldg(src + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    load_step(r0);
    for (int64_t rb = r0; rb < r1; rb += DF_ROWS) {
        const int nr = (int)min((int64_t)DF_ROWS, r1 - rb);
        __syncthreads();
#pragma unroll
        for (int u = 0; u < LPT; ++u) {
            const int q = t + u * GRAM_TPB;
            if (q < nr * (KC / 4)) reinterpret_cast<float4 *>(tile)[q] = pf[u];
        }
        load_step(rb + DF_ROWS);
        __syncthreads();
        if (active) {
            float h1[TS][TS], l1[TS][TS];
#pragma unroll
            for (int u = 0; u < TS; ++u)
#pragma unroll
                for (int v = 0; v < TS; ++v) h1[u][v] = l1[u][v] = 0.f;
            for (int r = st; r < nr; r += D::S) {
                float a[TS], b[TS];
                if constexpr (TS == 2) {
                    const float2 x = *reinterpret_cast<const float2 *>(tile + r * KC + ti * TS);
                    const float2 y = *reinterpret_cast<const float2 *>(tile + r * KC + tj * TS);
                    a[0] = x.x, a[1] = x.y, b[0] = y.x, b[1] = y.y;
                } else {
                    const float4 x = *reinterpret_cast<const float4 *>(tile + r * KC + ti * TS);
                    const float4 y = *reinterpret_cast<const float4 *>(tile + r * KC + tj * TS);
                    a[0] = x.x, a[1] = x.y, a[2] = x.z, a[3] = x.w;
                    b[0] = y.x, b[1] = y.y, b[2] = y.z, b[3] = y.w;
                }
#pragma unroll
                for (int u = 0; u < TS; ++u)
#pragma unroll
                    for (int v = 0; v < TS; ++v) df_fma(a[u], b[v], h1[u][v], l1[u][v]);
            }
#pragma unroll
            for (int u = 0; u < TS; ++u)
#pragma unroll
                for (int v = 0; v < TS; ++v) df_add(h2[u][v], l2[u][v], h1[u][v], l1[u][v]);
        }
    }
    __syncthreads();
    float2 *red = reinterpret_cast<float2 *>(smem);  // [S][NT][TS][TS]
    if (active)
#pragma unroll
        for (int u = 0; u < TS; ++u)
#pragma unroll
            for (int v = 0; v < TS; ++v) red[(st * D::NT + tid) * TS * TS + u * TS + v] = make_float2(h2[u][v], l2[u][v]);
    __syncthreads();
    for (int p = t; p < D::NP; p += GRAM_TPB) {
        int i = 0, rm = p;
        while (rm >= KC - i) {
            rm -= KC - i;
            ++i;
        }
        const int j = i + rm;
        const int a = i / TS, b = j / TS;  // a <= b
        const int tile_idx = a * D::NTB - a * (a - 1) / 2 + (b - a);
        const int e = (tile_idx * TS + i % TS) * TS + j % TS;
        float hi = 0.f, lo = 0.f;
        for (int q = 0; q < D::S; ++q) {
            const float2 x = red[q * D::NT * TS * TS + e];
            df_add(hi, lo, x.x, x.y);
        }
        part[(size_t)blockIdx.x * D::NP + p] = make_float2(hi, lo);
    }
}

constexpr int CHOL_TPB = 1024;

// Sum of the partials b0 <= b < b1 of pair p: four interleaved sums, combined
// in a fixed order.  DF: double-float partials summed in double-float.
template <bool DF>
struct PartSum {
    float hi = 0.f, lo = 0.f;
    double d = 0.0;
};

template <bool DF>
__device__ PartSum<DF> sum_range(const void *part_v, int npairs, int p, int b0, int b1) {
    PartSum<DF> r;
    if constexpr (DF) {
        const float2 *part = static_cast<const float2 *>(part_v);
        float h4[4] = {0.f, 0.f, 0.f, 0.f}, l4[4] = {0.f, 0.f, 0.f, 0.f};
        int b = b0;
        // eight loads in flight; partial b still goes to sum (b - b0) % 4
        for (; b + 8 <= b1; b += 8) {
            float2 x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = part[(size_t)(b + u) * npairs + p];
#pragma unroll
            for (int u = 0; u < 8; ++u) df_add(h4[u & 3], l4[u & 3], x[u].x, x[u].y);
        }
        for (; b + 4 <= b1; b += 4) {
            float2 x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = part[(size_t)(b + u) * npairs + p];
#pragma unroll
            for (int u = 0; u < 4; ++u) df_add(h4[u], l4[u], x[u].x, x[u].y);
        }
        for (int u = 0; b < b1; ++b, ++u) {
            const float2 x = part[(size_t)b * npairs + p];
            df_add(h4[u], l4[u], x.x, x.y);
        }
        df_add(h4[0], l4[0], h4[1], l4[1]);
        df_add(h4[2], l4[2], h4[3], l4[3]);
        df_add(h4[0], l4[0], h4[2], l4[2]);
        r.hi = h4[0];
        r.lo = l4[0];
    } else {
        const double *part = static_cast<const double *>(part_v);
        double s4[4] = {0, 0, 0, 0};
        int b = b0;
        for (; b + 4 <= b1; b += 4)
#pragma unroll
            for (int u = 0; u < 4; ++u) s4[u] += part[(size_t)(b + u) * npairs + p];
        for (int u = 0; b < b1; ++b, ++u) s4[u] += part[(size_t)b * npairs + p];
        r.d = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    }
    return r;
}

__device__ __forceinline__ void put_pair(double *W, int K, int p, double s, double shift) {
    int rem = p, i = 0;
    while (rem >= K - i) {
        rem -= K - i;
        ++i;
    }
    W[i * K + i + rem] = rem == 0 ? s + shift : s;
}

// W(i, j) for i <= j = the sum of the FP64 block partials (+ shift on the
// diagonal).  When the pairs are fewer than the threads, the nblk partials of
// each pair are split into nsub = blockDim / npairs contiguous block ranges,
// one thread per (pair, range), and the nsub sums of a pair are added in range
// order afterwards; otherwise a thread sums all partials of its pairs.  Either
// way the order is fixed (same result every run).  sub: shared scratch of
// blockDim doubles.
__device__ void gram_sum(const double *part, int nblk, int K, double shift, double *W, double *sub) {
    const int npairs = K * (K + 1) / 2;
    const int nsub = (int)blockDim.x / npairs;
    const int t = threadIdx.x;
    if (nsub <= 1) {
        for (int p = t; p < npairs; p += blockDim.x)
            put_pair(W, K, p, sum_range<false>(part, npairs, p, 0, nblk).d, shift);
        return;
    }
    if (t < nsub * npairs) {
        const int p = t % npairs, q = t / npairs;
        const int b0 = (int)((int64_t)nblk * q / nsub), b1 = (int)((int64_t)nblk * (q + 1) / nsub);
        sub[t] = sum_range<false>(part, npairs, p, b0, b1).d;
    }
    __syncthreads();
    for (int p = t; p < npairs; p += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < nsub; ++q) s += sub[q * npairs + p];
        put_pair(W, K, p, s, shift);
    }
}

// W = R^T R in place (R in the upper triangle), inv(j) = 1 / R(j, j); one warp,
// right-looking: step j scales row j by 1 / sqrt(pivot) and subtracts its
// outer product from the trailing triangle, whose entries the lanes share
// (pairs[] lists the upper triangle by row k from K-1 down, so the trailing
// triangle of step j is its first (K-j-1)(K-j)/2 entries, packed k * 64 + l).
// 1 / sqrt(pivot) for 1e-30 < pivot < 1e30 is the FP32 estimate refined by NR
// Newton-Raphson steps y <- y (3 - d y^2) / 2, each of which doubles the
// number of correct bits (about 22 -> 44 -> full FP64): FP64 divisions and
// square roots are long instruction sequences on this GPU, and the pivots are
// sequential.  Returns 1 when a pivot is not above tiny_rel max_j W(j, j).
template <int NR>
__device__ int chol_warp(double *W, double *inv, const uint16_t *pairs, int K, int lane, double tiny_rel) {
    double dmax = 0.0;
    for (int i = 0; i < K; ++i) dmax = fmax(dmax, W[i * K + i]);
    const double tiny = tiny_rel * dmax;
    if (!(dmax > 0.0)) return 1;
    for (int j = 0; j < K; ++j) {
        const double d = W[j * K + j];
        if (!(d > tiny)) return 1;
        double y;
        if (d > 1e-30 && d < 1e30) {
            y = (double)rsqrtf((float)d);
#pragma unroll
            for (int it = 0; it < NR; ++it) y = y * (1.5 - 0.5 * d * y * y);
        } else {
            y = 1.0 / sqrt(d);
        }
        for (int k = j + 1 + lane; k < K; k += 32) W[j * K + k] *= y;
        __syncwarp();
        const int nt = (K - j - 1) * (K - j) / 2;
        for (int q = lane; q < nt; q += 32) {
            const int k = pairs[q] >> 6, l = pairs[q] & 63;
            W[k * K + l] = fma(-W[j * K + k], W[j * K + l], W[k * K + l]);
        }
        if (lane == 0) {
            W[j * K + j] = d * y;
            inv[j] = y;
        }
        __syncwarp();
    }
    return 0;
}

// Sum of the FP64 Gram partials, Cholesky W = R^T R in FP64 (of W + s I after
// a breakdown in the first pass).  Rd receives R with 1 / R(j, j) on its
// diagonal and zeros below it, the form the row substitution of the apply step
// reads.  The partial sums use all threads; the factorisation runs in warp 0.
// m = rows of A.  A pivot counts as not clearly positive below 1e-14 of the
// largest diagonal entry; the reciprocal square root takes two Newton-Raphson
// steps from the FP32 estimate.  (Double-float partials of FP32 factors go to
// k_chol_df.)
__global__ void __launch_bounds__(CHOL_TPB) k_chol(const double *part, int nblk, int K, int64_t m, double *Rd,
                                                   int32_t *flag, int pass) {
    if (qr_skip(flag, pass)) return;
    __shared__ double W[HOQRI_MAXK * HOQRI_MAXK];
    __shared__ double inv[HOQRI_MAXK];  // 1 / R(j, j)
    __shared__ double sub[CHOL_TPB];
    __shared__ uint16_t pairs[HOQRI_MAXK * (HOQRI_MAXK + 1) / 2];
    __shared__ int s_bad;
    __shared__ double s_shift;
    constexpr double tiny_rel = 1e-14;
    constexpr int NR = 2;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int npairs = K * (K + 1) / 2;
    for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
        // entry q of the list: rows k = K-1, K-2, ... with K - k entries each
        int k = K - 1, rem = q;
        while (rem >= K - k) {
            rem -= K - k;
            --k;
        }
        pairs[q] = (uint16_t)(k * 64 + k + rem);
    }
    gram_sum(part, nblk, K, 0.0, W, sub);
    __syncthreads();
    if (wid == 0) {
        double tr = 0.0;
        for (int i = 0; i < K; ++i) tr += W[i * K + i];
        const int bad = chol_warp<NR>(W, inv, pairs, K, lane, tiny_rel);
        if (lane == 0) {
            s_bad = bad;
            s_shift = 11.0 * ((double)m * K + (double)K * (K + 1)) * 0x1p-53 * tr;
        }
    }
    __syncthreads();
    if (s_bad && pass == 0 && s_shift > 0.0) {
        gram_sum(part, nblk, K, s_shift, W, sub);
        __syncthreads();
        if (wid == 0) {
            const int bad = chol_warp<NR>(W, inv, pairs, K, lane, tiny_rel);
            if (lane == 0) {
                s_bad = bad;
                if (!bad) flag[3] = 1;
            }
        }
        __syncthreads();
    }
    if (wid != 0) return;
    if (s_bad) {
        if (lane == 0) {
            flag[0] = 1;
            flag[1] += 1;
        }
        return;
    }
    for (int t = lane; t < K * K; t += 32) {
        const int i = t / K, col = t - i * K;
        Rd[t] = i > col ? 0.0 : (i == col ? inv[i] : W[t]);
    }
}

// ---- the Cholesky of an FP32 factor's Gram in double-float.  The Gram is
// summed in double-float (k_gram_df), and the FP64 pipe of this GPU issues a
// warp instruction far more slowly than the FP32 pipes, which the K dependent
// pivot steps feel directly; so the factorisation keeps every entry as a
// double-float pair too.  Its rounding (about 2^-46 relative per operation) is
// below the Gram's own (a few 1e-15), and the factor is stored in FP32.

// s + e = a + b exactly, for |a| >= |b| (Dekker's Fast2Sum)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// (hi, lo) = (ah + al)(bh + bl) to about 2^-46 relative: the exact product
// ah bh = p + e by an FMA (TwoProduct), the cross terms added to e, renormalised
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &hi, float &lo) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    fast_two_sum(p, e, hi, lo);
}

// (yh, yl) = 1 / sqrt(dh + dl): the FP32 estimate y0 refined by one
// Newton-Raphson step y = y0 + y0 r / 2 with r = 1 - d y0^2 formed in
// double-float (y0^2 exact by TwoProduct); the step squares the estimate's
// relative error (about 2^-22 -> 2^-44).  Outside 1e-30 < dh < 1e30 (where the
// FP32 steps could underflow or overflow) the value comes from FP64.
__device__ __forceinline__ void df_rsqrt(float dh, float dl, float &yh, float &yl) {
    if (dh > 1e-30f && dh < 1e30f) {
        const float y0 = rsqrtf(dh);
        const float th = __fmul_rn(y0, y0);
        const float tl = __fmaf_rn(y0, y0, -th);
        float uh, ul;
        df_mul(dh, dl, th, tl, uh, ul);
        const float r = __fsub_rn(__fsub_rn(1.0f, uh), ul);  // 1 - uh is exact: uh is within 2^-21 of 1
        fast_two_sum(y0, __fmul_rn(__fmul_rn(y0, r), 0.5f), yh, yl);
    } else {
        const double y = 1.0 / sqrt((double)dh + (double)dl);
        yh = (float)y;
        yl = (float)(y - (double)yh);
    }
}

// W(i, j) for i <= j = the sum of the block partials (+ shift on the diagonal),
// as double-float pairs, summed in a fixed order.  sub: shared scratch of blockDim pairs.
__device__ void gram_sum_df(const float2 *part, int nblk, int K, float shift, float2 *W, float2 *sub) {
    const int npairs = K * (K + 1) / 2;
    const int nsub = (int)blockDim.x / npairs;
    const int t = threadIdx.x;
    auto put = [&](int p, float hi, float lo) {
        int rem = p, i = 0;
        while (rem >= K - i) {
            rem -= K - i;
            ++i;
        }
        if (rem == 0) df_add(hi, lo, shift, 0.f);
        W[i * K + i + rem] = make_float2(hi, lo);
    };
    if (nsub <= 1) {
        for (int p = t; p < npairs; p += blockDim.x) {
            const PartSum<true> r = sum_range<true>(part, npairs, p, 0, nblk);
            put(p, r.hi, r.lo);
        }
        return;
    }
    if (t < nsub * npairs) {
        const int p = t % npairs, q = t / npairs;
        const int b0 = (int)((int64_t)nblk * q / nsub), b1 = (int)((int64_t)nblk * (q + 1) / nsub);
        const PartSum<true> r = sum_range<true>(part, npairs, p, b0, b1);
        sub[t] = make_float2(r.hi, r.lo);
    }
    __syncthreads();
    for (int p = t; p < npairs; p += blockDim.x) {
        float hi = 0.f, lo = 0.f;
        for (int q = 0; q < nsub; ++q) df_add(hi, lo, sub[q * npairs + p].x, sub[q * npairs + p].y);
        put(p, hi, lo);
    }
}

// chol_warp in double-float: W = R^T R in place (pairs, R in the upper
// triangle), inv(j) = 1 / R(j, j); the same right-looking order and lane split.
// Returns 1 when a pivot is not above tiny_rel max_j W(j, j).
__device__ int chol_warp_df(float2 *W, float2 *inv, const uint16_t *pairs, int K, int lane, float tiny_rel) {
    float dmax = 0.f;
    for (int i = 0; i < K; ++i) dmax = fmaxf(dmax, W[i * K + i].x);
    const float tiny = tiny_rel * dmax;
    if (!(dmax > 0.f)) return 1;
    for (int j = 0; j < K; ++j) {
        const float2 d = W[j * K + j];
        if (!(d.x > tiny)) return 1;
        float yh, yl;
        df_rsqrt(d.x, d.y, yh, yl);
        for (int k = j + 1 + lane; k < K; k += 32) {
            const float2 w = W[j * K + k];
            float h, l;
            df_mul(w.x, w.y, yh, yl, h, l);
            W[j * K + k] = make_float2(h, l);
        }
        __syncwarp();
        const int nt = (K - j - 1) * (K - j) / 2;
        for (int q = lane; q < nt; q += 32) {
            const int k = pairs[q] >> 6, l = pairs[q] & 63;
            const float2 a = W[j * K + k], b = W[j * K + l];
            float ph, pl;
            df_mul(a.x, a.y, b.x, b.y, ph, pl);
            float2 w = W[k * K + l];
            df_add(w.x, w.y, -ph, -pl);
            W[k * K + l] = w;
        }
        if (lane == 0) {
            float h, l;
            df_mul(d.x, d.y, yh, yl, h, l);
            W[j * K + j] = make_float2(h, l);
            inv[j] = make_float2(yh, yl);
        }
        __syncwarp();
    }
    return 0;
}

// k_chol for double-float Gram partials (FP32 factors): the same steps,
// decisions and output (Rd in FP64, 1 / R(j, j) on the diagonal) with the sums
// and the factorisation in double-float.  The pivot threshold is 1e-13 of the
// largest diagonal entry.
__global__ void __launch_bounds__(CHOL_TPB) k_chol_df(const float2 *part, int nblk, int K, int64_t m, double *Rd,
                                                      int32_t *flag, int pass) {
    if (qr_skip(flag, pass)) return;
    __shared__ float2 W[HOQRI_MAXK * HOQRI_MAXK];
    __shared__ float2 inv[HOQRI_MAXK];
    __shared__ float2 sub[CHOL_TPB];
    __shared__ uint16_t pairs[HOQRI_MAXK * (HOQRI_MAXK + 1) / 2];
    __shared__ int s_bad;
    __shared__ float s_shift;
    constexpr float tiny_rel = 1e-13f;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int npairs = K * (K + 1) / 2;
    for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
        int k = K - 1, rem = q;
        while (rem >= K - k) {
            rem -= K - k;
            --k;
        }
        pairs[q] = (uint16_t)(k * 64 + k + rem);
    }
    gram_sum_df(part, nblk, K, 0.f, W, sub);
    __syncthreads();
    if (wid == 0) {
        float tr = 0.f;
        for (int i = 0; i < K; ++i) tr += W[i * K + i].x;
        const int bad = chol_warp_df(W, inv, pairs, K, lane, tiny_rel);
        if (lane == 0) {
            s_bad = bad;
            s_shift = 11.0f * ((float)m * K + (float)(K * (K + 1))) * 0x1p-53f * tr;
        }
    }
    __syncthreads();
    if (s_bad && pass == 0 && s_shift > 0.f) {
        gram_sum_df(part, nblk, K, s_shift, W, sub);
        __syncthreads();
        if (wid == 0) {
            const int bad = chol_warp_df(W, inv, pairs, K, lane, tiny_rel);
            if (lane == 0) {
                s_bad = bad;
                if (!bad) flag[3] = 1;
            }
        }
        __syncthreads();
    }
    if (s_bad) {
        if (threadIdx.x == 0) {
            flag[0] = 1;
            flag[1] += 1;
        }
        return;
    }
    for (int t = threadIdx.x; t < K * K; t += blockDim.x) {
        const int i = t / K, col = t - i * K;
        const float2 v = i == col ? inv[i] : W[t];
        Rd[t] = i > col ? 0.0 : (double)v.x + (double)v.y;
    }
}

// out(r, :) = A(r, :) R^{-1}: each row solves x R = a by forward substitution,
// x(c) = (a(c) - sum_{i<c} x(i) R(i, c)) / R(c, c), with Rd as k_chol writes it
// (1 / R(c, c) on the diagonal); one thread per row, which reads its whole row
// before writing, so out may alias A.  FP32 rows are solved in FP32 (the
// factor is stored in FP32), FP64 rows in FP64.
template <typename T, int KC>
__global__ void __launch_bounds__(256) k_apply_rows(const T *A, int64_t I, const double *Rd, T *out,
                                                    const int32_t *flag, int pass) {
    if (qr_skip(flag, pass)) return;
    __shared__ T Rs[KC * KC];
    for (int t = threadIdx.x; t < KC * KC; t += blockDim.x) Rs[t] = (T)Rd[t];
    __syncthreads();
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < I; r += (int64_t)gridDim.x * blockDim.x) {
        T a[KC];
        if constexpr (sizeof(T) == 4 && KC % 4 == 0) {
            // a row is KC/4 aligned 16-byte vectors
#pragma unroll
            for (int i = 0; i < KC / 4; ++i) {
                const float4 v = reinterpret_cast<const float4 *>(A + r * KC)[i];
                a[4 * i] = v.x;
                a[4 * i + 1] = v.y;
                a[4 * i + 2] = v.z;
                a[4 * i + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < KC; ++i) a[i] = A[r * KC + i];
        }
#pragma unroll
        for (int c = 0; c < KC; ++c) {
            a[c] *= Rs[c * KC + c];
#pragma unroll
            for (int k = c + 1; k < KC; ++k) a[k] = fma(-a[c], Rs[c * KC + k], a[k]);
        }
        if constexpr (sizeof(T) == 4 && KC % 4 == 0) {
#pragma unroll
            for (int i = 0; i < KC / 4; ++i)
                reinterpret_cast<float4 *>(out + r * KC)[i] =
                    make_float4(a[4 * i], a[4 * i + 1], a[4 * i + 2], a[4 * i + 3]);
        } else {
#pragma unroll
            for (int c = 0; c < KC; ++c) out[r * KC + c] = a[c];
        }
    }
}

// any K <= 64: one thread per row, row kept in local memory, solved in FP64
template <typename T>
__global__ void __launch_bounds__(256) k_apply_rows_any(const T *A, int64_t I, int K, const double *Rd, T *out,
                                                        const int32_t *flag, int pass) {
    if (qr_skip(flag, pass)) return;
    __shared__ double Rs[HOQRI_MAXK * HOQRI_MAXK];
    for (int t = threadIdx.x; t < K * K; t += blockDim.x) Rs[t] = Rd[t];
    __syncthreads();
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < I; r += (int64_t)gridDim.x * blockDim.x) {
        double a[HOQRI_MAXK];
        for (int i = 0; i < K; ++i) a[i] = (double)A[r * K + i];
        for (int c = 0; c < K; ++c) {
            a[c] *= Rs[c * K + c];
            for (int k = c + 1; k < K; ++k) a[k] = fma(-a[c], Rs[c * K + k], a[k]);
            out[r * K + c] = (T)a[c];
        }
    }
}

template <typename T>
void launch_apply(cudaStream_t st, const int32_t *flag, int pass, const T *A, int64_t I, int K, const double *Rd,
                  T *out, int grid) {
    // the fixed-width kernels move FP32 rows as 16-byte vectors: both buffers must be 16-byte aligned
    const bool aligned = ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    if (!aligned) {
        k_apply_rows_any<T><<<grid, 256, 0, st>>>(A, I, K, Rd, out, flag, pass);
        return;
    }
    switch (K) {
        case 4: k_apply_rows<T, 4><<<grid, 256, 0, st>>>(A, I, Rd, out, flag, pass); break;
        case 8: k_apply_rows<T, 8><<<grid, 256, 0, st>>>(A, I, Rd, out, flag, pass); break;
        case 16: k_apply_rows<T, 16><<<grid, 256, 0, st>>>(A, I, Rd, out, flag, pass); break;
        case 32: k_apply_rows<T, 32><<<grid, 256, 0, st>>>(A, I, Rd, out, flag, pass); break;
        default: k_apply_rows_any<T><<<grid, 256, 0, st>>>(A, I, K, Rd, out, flag, pass); break;
    }
}

__device__ double block_sum(double v, double *sh) {
    // fixed-shape tree over HH_TPB threads
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = HH_TPB / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// One-CTA Householder thin QR in FP64 (fallback).  W, Q: I x K doubles of workspace.
template <typename T>
__global__ void __launch_bounds__(HH_TPB) k_householder(const T *A, int64_t I, int K, double *W, double *Q, T *U,
                                                        int32_t *flag) {
    if (*flag != 1) return;
    __shared__ double sh[HH_TPB];
    __shared__ double beta[HOQRI_MAXK], diag[HOQRI_MAXK];
    for (int64_t t = threadIdx.x; t < I * K; t += HH_TPB) W[t] = (double)A[t];
    __syncthreads();
    for (int j = 0; j < K; ++j) {
        double s = 0.0;
        for (int64_t i = j + threadIdx.x; i < I; i += HH_TPB) s += W[i * K + j] * W[i * K + j];
        const double nrm = sqrt(block_sum(s, sh));
        if (nrm == 0.0) {
            if (threadIdx.x == 0) {
                beta[j] = 0.0;
                diag[j] = 0.0;
            }
            __syncthreads();
            continue;
        }
        const double wjj = W[(int64_t)j * K + j];
        const double alpha = wjj > 0 ? -nrm : nrm;
        __syncthreads();
        if (threadIdx.x == 0) W[(int64_t)j * K + j] = wjj - alpha;
        __syncthreads();
        s = 0.0;
        for (int64_t i = j + threadIdx.x; i < I; i += HH_TPB) s += W[i * K + j] * W[i * K + j];
        const double vn2 = block_sum(s, sh);
        const double bj = vn2 > 0 ? 2.0 / vn2 : 0.0;
        if (threadIdx.x == 0) {
            beta[j] = bj;
            diag[j] = alpha;
        }
        for (int c = j + 1; c < K; ++c) {
            s = 0.0;
            for (int64_t i = j + threadIdx.x; i < I; i += HH_TPB) s += W[i * K + j] * W[i * K + c];
            const double f = bj * block_sum(s, sh);
            for (int64_t i = j + threadIdx.x; i < I; i += HH_TPB) W[i * K + c] -= f * W[i * K + j];
            __syncthreads();
        }
        __syncthreads();
    }
    // Q = H_0 ... H_{K-1} [I_K; 0]
    for (int64_t t = threadIdx.x; t < I * K; t += HH_TPB) {
        int64_t r = t / K;
        int c = (int)(t - r * K);
        Q[t] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = K - 1; j >= 0; --j) {
        const double bj = beta[j];
        if (bj == 0.0) continue;
        for (int c = 0; c < K; ++c) {
            double s = 0.0;
            for (int64_t i = j + threadIdx.x; i < I; i += HH_TPB) s += W[i * K + j] * Q[i * K + c];
            const double f = bj * block_sum(s, sh);
            for (int64_t i = j + threadIdx.x; i < I; i += HH_TPB) Q[i * K + c] -= f * W[i * K + j];
            __syncthreads();
        }
    }
    for (int64_t t = threadIdx.x; t < I * K; t += HH_TPB) {
        int c = (int)(t % K);
        double v = Q[t];
        U[t] = (T)(diag[c] < 0 ? -v : v);
    }
    __syncthreads();
    if (threadIdx.x == 0) *flag = 2;
}

// ---- seeded Gaussian initial factors: Philox4x32-10 (Salmon et al., SC'11) + Box-Muller

__device__ __forceinline__ void philox_round(uint32_t c[4], uint32_t k[2]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    uint32_t n0 = hi1 ^ c[1] ^ k[0], n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

__device__ void philox4x32_10(uint32_t ctr[4], uint64_t key64) {
    uint32_t k[2] = {(uint32_t)key64, (uint32_t)(key64 >> 32)};
    for (int r = 0; r < 10; ++r) {
        philox_round(ctr, k);
        k[0] += 0x9E3779B9u;
        k[1] += 0xBB67AE85u;
    }
}

template <typename T>
__global__ void k_gauss(T *out, int64_t n, uint64_t seed, uint32_t stream_id) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c[4] = {(uint32_t)t, (uint32_t)(t >> 32), stream_id, 0x484F5152u};
        philox4x32_10(c, seed);
        const double u1 = ((double)c[0] + 1.0) * (1.0 / 4294967296.0);  // (0, 1]
        const double u2 = (double)c[1] * (1.0 / 4294967296.0);
        out[t] = (T)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
    }
}

// Gram partials and Cholesky of one pass: in double-float for an FP32 A with K
// in {4, 8, 16, 32} and 16-byte aligned rows, in FP64 otherwise.
template <typename T>
void launch_gram_chol(cudaStream_t st, const T *src, int64_t I, int K, int nb, int64_t rpb, void *part, double *Rd,
                      int32_t *flag, int pass) {
    bool df = false;
    if constexpr (sizeof(T) == 4) {
        df = (K == 4 || K == 8 || K == 16 || K == 32) && (reinterpret_cast<uintptr_t>(src) & 15) == 0;
        float2 *p2 = static_cast<float2 *>(part);
        if (df) switch (K) {
                case 4: k_gram_df<4, 2><<<nb, GRAM_TPB, 0, st>>>(src, I, rpb, p2, flag, pass); break;
                case 8: k_gram_df<8, 2><<<nb, GRAM_TPB, 0, st>>>(src, I, rpb, p2, flag, pass); break;
                case 16: k_gram_df<16, 2><<<nb, GRAM_TPB, 0, st>>>(src, I, rpb, p2, flag, pass); break;
                default: k_gram_df<32, 4><<<nb, GRAM_TPB, 0, st>>>(src, I, rpb, p2, flag, pass); break;
            }
    }
    if (df) {
        k_chol_df<<<1, CHOL_TPB, 0, st>>>(static_cast<const float2 *>(part), nb, K, I, Rd, flag, pass);
    } else {
        k_gram_partial<T><<<nb, GRAM_TPB, 0, st>>>(src, I, K, rpb, static_cast<double *>(part), flag, pass);
        k_chol<<<1, CHOL_TPB, 0, st>>>(static_cast<const double *>(part), nb, K, I, Rd, flag, pass);
    }
}

__global__ void k_set_flag(int32_t *flag, int32_t v) {
    flag[0] = v;
    flag[3] = 0;
}

// one Gram block per SM at most (the FP64 multiply-adds need every SM; fewer
// partials keep the Cholesky's reduction short)
int gram_blocks(int64_t I, int num_sms) {
    int64_t b = ceil_div(I, 256);
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, std::min(num_sms, MAX_GRAM_BLOCKS)));
}

template <typename T>
hoqri_status orthonormalize_t(hoqri_ctx *c, int n, T *A, T *U) {
    const int64_t I = c->dims[n];
    const int K = c->K[n];
    cudaStream_t st = c->stream;
    const int nb = gram_blocks(I, c->num_sms);
    const int64_t rpb = ceil_div(I, nb);
    double *Rd = c->qr_small;
    const int apply_rows_grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(I, 256), (int64_t)c->num_sms * 8));
    // flag 0: CholeskyQR2; flag 1 (qr_kind 1): Householder from the start; no
    // shift yet.  Set with a kernel, not a copy from host memory, so a captured
    // graph replays it.
    k_set_flag<<<1, 1, 0, st>>>(c->dflag, c->opt.qr_kind == 1 ? 1 : 0);
    c->nlaunch++;
    // pass 0: A <- A R1^{-1}; pass 1: U = A R2^{-1}; pass 2 (after a shift): U <- U R3^{-1}
    for (int pass = 0; pass < QR_PASSES; ++pass) {
        T *src = pass < 2 ? A : U;
        launch_gram_chol<T>(st, src, I, K, nb, rpb, c->qr_part, Rd, c->dflag, pass);
        k_householder<T><<<1, HH_TPB, 0, st>>>(src, I, K, c->qr_work, c->qr_work + I * K, U, c->dflag);
        launch_apply<T>(st, c->dflag, pass, src, I, K, Rd, pass == 0 ? A : U, apply_rows_grid);
        c->nlaunch += 4;
    }
    HQ_CUDA(cudaGetLastError());
    return HOQRI_OK;
}

}  // namespace

hoqri_status qr_init(hoqri_ctx *c) {
    int64_t maxIK = 0;
    for (int n = 0; n < c->N; ++n) maxIK = std::max<int64_t>(maxIK, c->dims[n] * c->K[n]);
    c->qr_part_bytes = (int64_t)MAX_GRAM_BLOCKS * (HOQRI_MAXK * (HOQRI_MAXK + 1) / 2) * sizeof(double);
    HQ_TRY(dalloc(c, (void **)&c->qr_part, c->qr_part_bytes));
    HQ_TRY(dalloc(c, (void **)&c->qr_small, HOQRI_MAXK * HOQRI_MAXK * sizeof(double)));
    HQ_TRY(dalloc(c, (void **)&c->qr_work, 2 * maxIK * sizeof(double)));
    return HOQRI_OK;
}

hoqri_status orthonormalize(hoqri_ctx *c, int n, void *A_inout, void *U_out) {
    cudaEvent_t e0 = nullptr;
    HQ_TRY(prof_begin(c, 2, &e0));
    hoqri_status s = (c->prec == HOQRI_FP64) ? orthonormalize_t<double>(c, n, (double *)A_inout, (double *)U_out)
                                             : orthonormalize_t<float>(c, n, (float *)A_inout, (float *)U_out);
    HQ_TRY(s);
    return prof_end(c, 2, e0);
}

hoqri_status init_factors_seeded(hoqri_ctx *c) {
    for (int n = 0; n < c->N; ++n) {
        const int64_t cnt = c->dims[n] * c->K[n];
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(cnt, 256), 4096));
        if (c->prec == HOQRI_FP64)
            k_gauss<double><<<g, 256, 0, c->stream>>>((double *)c->A, cnt, c->opt.seed, (uint32_t)n);
        else
            k_gauss<float><<<g, 256, 0, c->stream>>>((float *)c->A, cnt, c->opt.seed, (uint32_t)n);
        c->nlaunch++;
        HQ_TRY(orthonormalize(c, n, c->A, c->U[n]));
    }
    HQ_CUDA(cudaGetLastError());
    return HOQRI_OK;
}

// ---- allocation-free CholeskyQR2 (hoqri_orthonormalize_noalloc): the same
// Gram / Cholesky / apply kernels (shifted first pass included), with their
// scratch in one file-scope device array instead of context buffers.  Layout:
// Gram partials of up to NA_BLOCKS blocks | R (diagonal 1 / R(j, j)) | flag[4] (on a 256-byte
// boundary).
namespace {

constexpr int NA_BLOCKS = 160;
constexpr int NA_PAIRS = HOQRI_NOALLOC_MAXK * (HOQRI_NOALLOC_MAXK + 1) / 2;
constexpr size_t NA_PART_BYTES = (size_t)NA_BLOCKS * NA_PAIRS * sizeof(double);
constexpr size_t NA_RINV_BYTES = (size_t)HOQRI_NOALLOC_MAXK * HOQRI_NOALLOC_MAXK * sizeof(double);
static_assert(NA_PART_BYTES + NA_RINV_BYTES + 256 == HOQRI_NOALLOC_SCRATCH_BYTES, "scratch layout");
static_assert(NA_PART_BYTES % 256 == 0 && NA_RINV_BYTES % 256 == 0, "flag alignment");
static_assert(HOQRI_NOALLOC_MAXK <= HOQRI_MAXK, "kernels are sized for HOQRI_MAXK columns");
constexpr int NA_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_na_scratch[HOQRI_NOALLOC_SCRATCH_BYTES];

std::mutex g_na_mu;
int g_na_sms[NA_MAX_DEVICES];

// Address of the scratch on the current device.  It is looked up on every
// call (cheap once the module is loaded): a cached address would go stale if
// the caller reset the device, which reloads the module and may move the array.
// Only the SM count is cached per device.
hoqri_status na_scratch(unsigned char **p, int *sms) {
    int dev = 0;
    HQ_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) {
        set_error("hoqri_orthonormalize_noalloc: device ordinal " + std::to_string(dev) + " above the supported " +
                  std::to_string(NA_MAX_DEVICES - 1));
        return HOQRI_ERR_INVALID;
    }
    void *a = nullptr;
    HQ_CUDA(cudaGetSymbolAddress(&a, g_na_scratch));
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (g_na_sms[dev] == 0) {
            int n = 0;
            HQ_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
            g_na_sms[dev] = std::max(n, 1);
        }
        *sms = g_na_sms[dev];
    }
    *p = static_cast<unsigned char *>(a);
    return HOQRI_OK;
}

template <typename T>
hoqri_status orthonormalize_noalloc_t(int64_t I, int K, const T *A, T *U, cudaStream_t st) {
    unsigned char *base = nullptr;
    int sms = 1;
    HQ_TRY(na_scratch(&base, &sms));
    double *part = reinterpret_cast<double *>(base);
    double *Rd = reinterpret_cast<double *>(base + NA_PART_BYTES);
    int32_t *flag = reinterpret_cast<int32_t *>(base + NA_PART_BYTES + NA_RINV_BYTES);
    const int nb = std::min(gram_blocks(I, sms), NA_BLOCKS);
    const int64_t rpb = ceil_div(I, nb);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(I, 256), (int64_t)sms * 8));
    HQ_CUDA(cudaMemsetAsync(flag, 0, 4 * sizeof(int32_t), st));
    // pass 0: U = A R1^{-1}; passes 1 and 2 (the latter after a shifted first
    // pass only): U = U R^{-1} in place, row by row
    for (int pass = 0; pass < QR_PASSES; ++pass) {
        const T *src = pass == 0 ? A : U;
        launch_gram_chol<T>(st, src, I, K, nb, rpb, part, Rd, flag, pass);
        launch_apply<T>(st, flag, pass, src, I, K, Rd, U, grid);
    }
    HQ_CUDA(cudaGetLastError());
    int32_t f = 0;
    HQ_CUDA(cudaMemcpyAsync(&f, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    HQ_CUDA(cudaStreamSynchronize(st));
    if (f != 0) {
        set_error("hoqri_orthonormalize_noalloc: Cholesky breakdown (A is rank deficient or too ill conditioned "
                  "for shifted CholeskyQR3)");
        return HOQRI_ERR_QR_BREAKDOWN;
    }
    return HOQRI_OK;
}

}  // namespace

hoqri_status orthonormalize_noalloc(int prec, int64_t I, int K, const void *A, void *U, cudaStream_t st) {
    if (prec == HOQRI_FP64)
        return orthonormalize_noalloc_t<double>(I, K, static_cast<const double *>(A), static_cast<double *>(U), st);
    return orthonormalize_noalloc_t<float>(I, K, static_cast<const float *>(A), static_cast<float *>(U), st);
}

}  // namespace hoqri
