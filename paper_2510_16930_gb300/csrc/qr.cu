// Orthonormalisation U_n <- orthonormal basis of A_n (Alg. 2, the QR step).
//
// CholeskyQR2 in FP64: W = A^T A (Gram, FP64 sums in a fixed order),
// W = R^T R (Cholesky, one CTA), A <- A R^{-1}; then once more on the result.
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

// 1 / sqrt(d) in FP64 for 1e-30 < d < 1e30: the FP32 estimate refined by two
// Newton-Raphson steps y <- y (3 - d y^2) / 2, each of which doubles the number
// of correct bits (about 22 -> 44 -> full FP64).  FP64 divisions and square
// roots are long instruction sequences on this GPU; a pivot of the Cholesky
// needs both, and the pivots are sequential.
__device__ __forceinline__ double rsqrt_fp64(double d) {
    if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
    double y = (double)rsqrtf((float)d);
    y = y * (1.5 - 0.5 * d * y * y);
    y = y * (1.5 - 0.5 * d * y * y);
    return y;
}

// W(i, j) for i <= j = the sum of the block partials (+ shift on the diagonal):
// thread per pair (coalesced across the threads for each block), eight
// interleaved partial sums so eight loads are in flight, combined in a fixed
// order (same result every run)
__device__ void gram_sum(const double *part, int nblk, int K, double shift, double *W) {
    const int npairs = K * (K + 1) / 2;
    for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
        double s8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int b = 0;
        for (; b + 8 <= nblk; b += 8)
#pragma unroll
            for (int u = 0; u < 8; ++u) s8[u] += part[(size_t)(b + u) * npairs + p];
        for (int u = 0; b < nblk; ++b, ++u) s8[u] += part[(size_t)b * npairs + p];
        const double s = ((s8[0] + s8[1]) + (s8[2] + s8[3])) + ((s8[4] + s8[5]) + (s8[6] + s8[7]));
        int rem = p, i = 0;
        while (rem >= K - i) {
            rem -= K - i;
            ++i;
        }
        W[i * K + i + rem] = rem == 0 ? s + shift : s;
    }
}

// W = R^T R in place (R in the upper triangle), inv(j) = 1 / R(j, j); one warp,
// lane k holds column k, so the sequential pivots need no block barrier.
// Returns 1 when a pivot is not above 1e-14 max_j W(j, j).
__device__ int chol_warp(double *W, double *inv, int K, int lane) {
    double dmax = 0.0;
    for (int i = 0; i < K; ++i) dmax = fmax(dmax, W[i * K + i]);
    const double tiny = 1e-14 * dmax;
    if (!(dmax > 0.0)) return 1;
    for (int j = 0; j < K; ++j) {
        // pivot: d = W(j,j) - sum_{i<j} R(i,j)^2, a lane-strided sum in fixed order
        double d = 0.0;
        for (int i = lane; i < j; i += 32) d += W[i * K + j] * W[i * K + j];
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        d = W[j * K + j] - d;
        if (!(d > tiny)) return 1;
        const double y = rsqrt_fp64(d);  // 1 / R(j, j)
        // row j of R: R(j,k) = (W(j,k) - sum_{i<j} R(i,j) R(i,k)) / R(j,j), lane per k
        for (int k = j + 1 + lane; k < K; k += 32) {
            double s = W[j * K + k];
            for (int i = 0; i < j; ++i) s -= W[i * K + j] * W[i * K + k];
            W[j * K + k] = s * y;
        }
        __syncwarp();
        if (lane == 0) {
            W[j * K + j] = d * y;
            inv[j] = y;
        }
        __syncwarp();
    }
    return 0;
}

// Sum of the Gram partials, Cholesky W = R^T R (of W + s I after a breakdown in
// the first pass), Rinv = R^{-1}.  The partial sums use all warps; the
// factorisation and the inverse run in warp 0.  m = rows of A.
__global__ void __launch_bounds__(256) k_chol(const double *part, int nblk, int K, int64_t m, double *Rinv,
                                              int32_t *flag, int pass) {
    if (qr_skip(flag, pass)) return;
    __shared__ double W[HOQRI_MAXK * HOQRI_MAXK];
    __shared__ double inv[HOQRI_MAXK];  // 1 / R(j, j)
    __shared__ int s_bad;
    __shared__ double s_shift;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    gram_sum(part, nblk, K, 0.0, W);
    __syncthreads();
    if (wid == 0) {
        double tr = 0.0;
        for (int i = 0; i < K; ++i) tr += W[i * K + i];
        const int bad = chol_warp(W, inv, K, lane);
        if (lane == 0) {
            s_bad = bad;
            s_shift = 11.0 * ((double)m * K + (double)K * (K + 1)) * 0x1p-53 * tr;
        }
    }
    __syncthreads();
    if (s_bad && pass == 0 && s_shift > 0.0) {
        gram_sum(part, nblk, K, s_shift, W);
        __syncthreads();
        if (wid == 0) {
            const int bad = chol_warp(W, inv, K, lane);
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
    // Rinv: lane col solves R x = e_col by back substitution (x upper triangular);
    // x(i) for i < col is kept in the free strictly-lower entry W(col, i)
    for (int col = lane; col < K; col += 32) {
        const double xd = inv[col];
        for (int i = col - 1; i >= 0; --i) {
            double s = -W[i * K + col] * xd;
            for (int k = i + 1; k < col; ++k) s -= W[i * K + k] * W[col * K + k];
            W[col * K + i] = s * inv[i];
        }
        Rinv[col * K + col] = xd;
    }
    __syncwarp();
    for (int t = lane; t < K * K; t += 32) {
        const int i = t / K, col = t - i * K;
        if (i != col) Rinv[t] = i > col ? 0.0 : W[col * K + i];
    }
}

// out(r, :) = A(r, :) Rinv (Rinv upper triangular), one thread per row; the
// thread reads its whole row before writing, so out may alias A.  FP32 rows
// are multiplied in FP32 (the factor is stored in FP32), FP64 rows in FP64.
template <typename T, int KC>
__global__ void __launch_bounds__(256) k_apply_rows(const T *A, int64_t I, const double *Rinv, T *out,
                                                    const int32_t *flag, int pass) {
    if (qr_skip(flag, pass)) return;
    __shared__ T Rs[KC * KC];
    for (int t = threadIdx.x; t < KC * KC; t += blockDim.x) Rs[t] = (T)Rinv[t];
    __syncthreads();
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < I; r += (int64_t)gridDim.x * blockDim.x) {
        T a[KC], o[KC];
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
            T s = T(0);
#pragma unroll
            for (int i = 0; i <= c; ++i) s = fma(a[i], Rs[i * KC + c], s);
            o[c] = s;
        }
        if constexpr (sizeof(T) == 4 && KC % 4 == 0) {
#pragma unroll
            for (int i = 0; i < KC / 4; ++i)
                reinterpret_cast<float4 *>(out + r * KC)[i] =
                    make_float4(o[4 * i], o[4 * i + 1], o[4 * i + 2], o[4 * i + 3]);
        } else {
#pragma unroll
            for (int c = 0; c < KC; ++c) out[r * KC + c] = o[c];
        }
    }
}

// any K <= 64: one thread per row, row kept in local memory
template <typename T>
__global__ void __launch_bounds__(256) k_apply_rows_any(const T *A, int64_t I, int K, const double *Rinv, T *out,
                                                        const int32_t *flag, int pass) {
    if (qr_skip(flag, pass)) return;
    __shared__ double Rs[HOQRI_MAXK * HOQRI_MAXK];
    for (int t = threadIdx.x; t < K * K; t += blockDim.x) Rs[t] = Rinv[t];
    __syncthreads();
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < I; r += (int64_t)gridDim.x * blockDim.x) {
        double a[HOQRI_MAXK];
        for (int i = 0; i < K; ++i) a[i] = (double)A[r * K + i];
        for (int c = 0; c < K; ++c) {
            double s = 0.0;
            for (int i = 0; i <= c; ++i) s += a[i] * Rs[i * K + c];
            out[r * K + c] = (T)s;
        }
    }
}

template <typename T>
void launch_apply(cudaStream_t st, const int32_t *flag, int pass, const T *A, int64_t I, int K, const double *Rinv,
                  T *out, int grid) {
    // the fixed-width kernels move FP32 rows as 16-byte vectors: both buffers must be 16-byte aligned
    const bool aligned = ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    if (!aligned) {
        k_apply_rows_any<T><<<grid, 256, 0, st>>>(A, I, K, Rinv, out, flag, pass);
        return;
    }
    switch (K) {
        case 4: k_apply_rows<T, 4><<<grid, 256, 0, st>>>(A, I, Rinv, out, flag, pass); break;
        case 8: k_apply_rows<T, 8><<<grid, 256, 0, st>>>(A, I, Rinv, out, flag, pass); break;
        case 16: k_apply_rows<T, 16><<<grid, 256, 0, st>>>(A, I, Rinv, out, flag, pass); break;
        case 32: k_apply_rows<T, 32><<<grid, 256, 0, st>>>(A, I, Rinv, out, flag, pass); break;
        default: k_apply_rows_any<T><<<grid, 256, 0, st>>>(A, I, K, Rinv, out, flag, pass); break;
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
    const int npairs = K * (K + 1) / 2;
    double *Rinv = c->qr_small;
    const int apply_rows_grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(I, 256), (int64_t)c->num_sms * 8));
    // flag 0: CholeskyQR2; flag 1 (qr_kind 1): Householder from the start; no
    // shift yet.  Set with a kernel, not a copy from host memory, so a captured
    // graph replays it.
    k_set_flag<<<1, 1, 0, st>>>(c->dflag, c->opt.qr_kind == 1 ? 1 : 0);
    c->nlaunch++;
    // pass 0: A <- A R1^{-1}; pass 1: U = A R2^{-1}; pass 2 (after a shift): U <- U R3^{-1}
    for (int pass = 0; pass < QR_PASSES; ++pass) {
        T *src = pass < 2 ? A : U;
        k_gram_partial<T><<<nb, GRAM_TPB, 0, st>>>(src, I, K, rpb, c->qr_part, c->dflag, pass);
        k_chol<<<1, 256, 0, st>>>(c->qr_part, nb, K, I, Rinv, c->dflag, pass);
        k_householder<T><<<1, HH_TPB, 0, st>>>(src, I, K, c->qr_work, c->qr_work + I * K, U, c->dflag);
        launch_apply<T>(st, c->dflag, pass, src, I, K, Rinv, pass == 0 ? A : U, apply_rows_grid);
        c->nlaunch += 4;
    }
    (void)npairs;
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
// Gram partials of up to NA_BLOCKS blocks | R^{-1} | flag[4] (on a 256-byte
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
unsigned char *g_na_addr[NA_MAX_DEVICES];
int g_na_sms[NA_MAX_DEVICES];

// address of the scratch on the current device: looked up once per device
hoqri_status na_scratch(unsigned char **p, int *sms) {
    int dev = 0;
    HQ_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) {
        set_error("hoqri_orthonormalize_noalloc: device ordinal " + std::to_string(dev) + " above the supported " +
                  std::to_string(NA_MAX_DEVICES - 1));
        return HOQRI_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev]) {
        void *a = nullptr;
        HQ_CUDA(cudaGetSymbolAddress(&a, g_na_scratch));
        int n = 0;
        HQ_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        g_na_sms[dev] = std::max(n, 1);
        g_na_addr[dev] = static_cast<unsigned char *>(a);
    }
    *p = g_na_addr[dev];
    *sms = g_na_sms[dev];
    return HOQRI_OK;
}

template <typename T>
hoqri_status orthonormalize_noalloc_t(int64_t I, int K, const T *A, T *U, cudaStream_t st) {
    unsigned char *base = nullptr;
    int sms = 1;
    HQ_TRY(na_scratch(&base, &sms));
    double *part = reinterpret_cast<double *>(base);
    double *Rinv = reinterpret_cast<double *>(base + NA_PART_BYTES);
    int32_t *flag = reinterpret_cast<int32_t *>(base + NA_PART_BYTES + NA_RINV_BYTES);
    const int nb = std::min(gram_blocks(I, sms), NA_BLOCKS);
    const int64_t rpb = ceil_div(I, nb);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(I, 256), (int64_t)sms * 8));
    HQ_CUDA(cudaMemsetAsync(flag, 0, 4 * sizeof(int32_t), st));
    // pass 0: U = A R1^{-1}; passes 1 and 2 (the latter after a shifted first
    // pass only): U = U R^{-1} in place, row by row
    for (int pass = 0; pass < QR_PASSES; ++pass) {
        const T *src = pass == 0 ? A : U;
        k_gram_partial<T><<<nb, GRAM_TPB, 0, st>>>(src, I, K, rpb, part, flag, pass);
        k_chol<<<1, 256, 0, st>>>(part, nb, K, I, Rinv, flag, pass);
        launch_apply<T>(st, flag, pass, src, I, K, Rinv, U, grid);
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
