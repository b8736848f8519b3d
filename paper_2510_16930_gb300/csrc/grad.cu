// Riemannian-gradient norm at the current factors (Sec. 5, Eq. tucker_grad and
// Eq. grad2): on the product of Stiefel manifolds the gradient of
// f = ||X x {U^T}||^2 with respect to block n is 2 A_n - 2 U_n G_(n) G_(n)^T,
// A_n = TTMcTC(X, {U}, n).  This file computes one mode's term
// ||A_n - U_n G_(n) G_(n)^T||_F^2 in FP64 (the caller multiplies by 4 and sums
// over the modes).  It is written in this direct form, not as
// ||A_n||^2 - ||G_(n) G_(n)^T||^2 (the last line of Eq. grad2), because the two
// norms nearly cancel close to a stationary point.
#include "internal.cuh"

namespace hoqri {

namespace {

constexpr int GR_TPB = 256;
constexpr int GR_MAX_BLOCKS = 304;

// fixed-shape tree over GR_TPB threads; the result is valid in thread 0
__device__ double block_sum256(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = GR_TPB / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    return sh[0];
}

// M = G_(n) G_(n)^T (K_n x K_n, FP64) from the row-major core: G_(n)(a, :)
// holds the entries G[o][a][q] with o over the modes before n (outer) and q
// over the modes after n (inner).  One CTA per entry a <= b, which also
// writes the mirrored entry.
template <typename T>
__global__ void __launch_bounds__(GR_TPB) k_core_gram(const T *G, int Kn, int64_t outer, int64_t inner, double *M) {
    __shared__ double sh[GR_TPB];
    const int a = blockIdx.x / Kn, b = blockIdx.x - a * Kn;
    if (a > b) return;
    const int64_t tot = outer * inner;
    double s = 0.0;
    for (int64_t t = threadIdx.x; t < tot; t += GR_TPB) {
        const int64_t o = t / inner, q = t - o * inner;
        s += (double)G[(o * Kn + a) * inner + q] * (double)G[(o * Kn + b) * inner + q];
    }
    s = block_sum256(s, sh);
    if (threadIdx.x == 0) {
        M[a * Kn + b] = s;
        M[b * Kn + a] = s;
    }
}

// CTA partials of sum_i ||A(i, :) - U(i, :) M||^2 in FP64 (rows strided over
// the grid, a fixed-shape tree per CTA)
template <typename T>
__global__ void __launch_bounds__(GR_TPB) k_grad_rows(const T *A, const T *U, int64_t I, int K, const double *M,
                                                      double *part) {
    __shared__ double Ms[HOQRI_MAXK * HOQRI_MAXK];
    __shared__ double sh[GR_TPB];
    for (int t = threadIdx.x; t < K * K; t += GR_TPB) Ms[t] = M[t];
    __syncthreads();
    double s = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)GR_TPB + threadIdx.x; r < I; r += (int64_t)gridDim.x * GR_TPB) {
        double u[HOQRI_MAXK];
        for (int k = 0; k < K; ++k) u[k] = (double)U[r * K + k];
        for (int c = 0; c < K; ++c) {
            double d = (double)A[r * K + c];
            for (int k = 0; k < K; ++k) d -= u[k] * Ms[k * K + c];
            s += d * d;
        }
    }
    s = block_sum256(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_parts(const double *part, int n, double *out) {
    double s = 0.0;
    for (int b = 0; b < n; ++b) s += part[b];
    *out = s;
}

template <typename T>
hoqri_status grad_term_t(hoqri_ctx *c, int n, const T *A, double *slot) {
    const int Kn = c->K[n];
    int64_t outer = 1, inner = 1;
    for (int m = 0; m < n; ++m) outer *= c->K[m];
    for (int m = n + 1; m < c->N; ++m) inner *= c->K[m];
    double *M = c->qr_small;  // K_n x K_n FP64 (the QR's scratch; same stream)
    double *part = c->qr_part;
    k_core_gram<T><<<Kn * Kn, GR_TPB, 0, c->stream>>>(static_cast<const T *>(c->G), Kn, outer, inner, M);
    const int64_t I = c->dims[n];
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(I, GR_TPB), GR_MAX_BLOCKS));
    k_grad_rows<T><<<grid, GR_TPB, 0, c->stream>>>(A, static_cast<const T *>(c->U[n]), I, Kn, M, part);
    k_sum_parts<<<1, 1, 0, c->stream>>>(part, grid, slot);
    c->nlaunch += 3;
    HQ_CUDA(cudaGetLastError());
    return HOQRI_OK;
}

}  // namespace

hoqri_status grad_term(hoqri_ctx *c, int n, const void *A, double *slot) {
    if (c->prec == HOQRI_FP64) return grad_term_t<double>(c, n, static_cast<const double *>(A), slot);
    return grad_term_t<float>(c, n, static_cast<const float *>(A), slot);
}

}  // namespace hoqri
