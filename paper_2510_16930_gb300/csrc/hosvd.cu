// HOSVD initialisation of the factors (Alg. 2: "initialize all U_n randomly or
// from HOSVD"): U_n <- an orthonormal basis of the leading K_n left singular
// subspace of the unfolding X_(n), computed by orthogonal iteration on
// X_(n) X_(n)^T (Golub and Van Loan, Matrix Computations, 4th ed., Sec. 8.2.4):
// from a seeded Gaussian start V, each step forms Y = X_(n) (X_(n)^T V) from the
// sparse entries and orthonormalises it with the QR of the sweep.
//
// X_(n)^T V has one row per distinct column of X_(n), i.e. per distinct tuple
// of the other modes' indices among the nonzeros.  The mode-n stream is sorted
// by row; a stable sort of its positions by that tuple groups the columns:
//   W(c, :) = sum over the positions q of column c of x_q V(i_n(q), :)   (one thread per column)
//   Y(i, :) = sum over the positions p of row i of x_p W(col(p), :)      (one warp per row)
// Both sums run in a fixed order, so the result is the same on every run.
#include <cub/cub.cuh>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.cuh"

namespace hoqri {

namespace {

constexpr int HS_TPB = 256;
constexpr int HS_KCH = 16;  // columns of V / W handled per pass over a segment

int hs_grid(int64_t n, int num_sms) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), HS_TPB), (int64_t)num_sms * 8));
}

__global__ void k_hs_iota(int32_t *a, int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        a[t] = (int32_t)t;
}

__global__ void k_hs_key(const int32_t *idx, const int32_t *perm, int64_t n, uint32_t *key) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        key[t] = (uint32_t)idx[perm[t]];
}

struct OtherIdx {
    const int32_t *p[HOQRI_MAXN - 1];
};

// head[q] = 1 where column-sorted position q starts a new column
__global__ void k_hs_heads(OtherIdx o, int nm1, const int32_t *perm, int64_t n, int32_t *head) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        int h = q == 0;
        if (!h) {
            const int32_t a = perm[q], b = perm[q - 1];
            for (int j = 0; j < nm1 && !h; ++j) h = o.p[j][a] != o.p[j][b];
        }
        head[q] = h;
    }
}

// column starts (in column-sorted order) and each row-sorted position's column
__global__ void k_hs_cols(const int32_t *head, const int32_t *incl, const int32_t *perm, int64_t n, int64_t *col_start,
                          int32_t *col_of) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = incl[q] - 1;
        if (head[q]) col_start[c] = q;
        col_of[perm[q]] = c;
        if (q == n - 1) col_start[c + 1] = n;
    }
}

// mode-n index of every row-sorted position (binary search in row_ptr)
__global__ void k_hs_rows(const int64_t *row_ptr, const int32_t *row_id, int64_t R, int64_t n, int32_t *in_of) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = R - 1;  // last row with row_ptr <= p
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (row_ptr[mid] <= p) lo = mid;
            else hi = mid - 1;
        }
        in_of[p] = row_id[lo];
    }
}

// W(c, :) = sum_{q in column c} x V(i_n, :), K columns in chunks of HS_KCH
template <typename T>
__global__ void __launch_bounds__(HS_TPB) k_hs_w(const int64_t *col_start, int64_t ncol, const int32_t *perm,
                                                 const T *vals, const int32_t *in_of, const T *V, int K, T *W) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncol; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q0 = col_start[c], q1 = col_start[c + 1];
        for (int kc = 0; kc < K; kc += HS_KCH) {
            T acc[HS_KCH];
#pragma unroll
            for (int k = 0; k < HS_KCH; ++k) acc[k] = T(0);
            for (int64_t q = q0; q < q1; ++q) {
                const int32_t p = perm[q];
                const T x = vals[p];
                const T *v = V + (int64_t)in_of[p] * K + kc;
#pragma unroll
                for (int k = 0; k < HS_KCH; ++k)
                    if (kc + k < K) acc[k] += x * v[k];
            }
#pragma unroll
            for (int k = 0; k < HS_KCH; ++k)
                if (kc + k < K) W[c * K + kc + k] = acc[k];
        }
    }
}

// Y(row_id[r], :) = sum_{p in row r} x W(col(p), :): one warp per row, lanes
// take every 32nd position, then a fixed butterfly over the lanes
template <typename T>
__global__ void __launch_bounds__(HS_TPB) k_hs_y(const int64_t *row_ptr, const int32_t *row_id, int64_t R,
                                                 const T *vals, const int32_t *col_of, const T *W, int K, T *Y) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < R; r += warps) {
        const int64_t p0 = row_ptr[r], p1 = row_ptr[r + 1];
        for (int kc = 0; kc < K; kc += HS_KCH) {
            T acc[HS_KCH];
#pragma unroll
            for (int k = 0; k < HS_KCH; ++k) acc[k] = T(0);
            for (int64_t p = p0 + lane; p < p1; p += 32) {
                const T x = vals[p];
                const T *w = W + (int64_t)col_of[p] * K + kc;
#pragma unroll
                for (int k = 0; k < HS_KCH; ++k)
                    if (kc + k < K) acc[k] += x * w[k];
            }
#pragma unroll
            for (int k = 0; k < HS_KCH; ++k)
                for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
            if (lane == 0) {
                T *y = Y + (int64_t)row_id[r] * K + kc;
#pragma unroll
                for (int k = 0; k < HS_KCH; ++k)
                    if (kc + k < K) y[k] = acc[k];
            }
        }
    }
}

// temporary device buffers of one call, freed in stream order
struct HsTmp {
    cudaStream_t st;
    std::vector<void *> ptrs;
    explicit HsTmp(cudaStream_t s) : st(s) {}
    ~HsTmp() {
        for (void *p : ptrs) raw_free(p, st);
    }
    template <typename U>
    hoqri_status get(U **p, size_t count) {
        void *q = nullptr;
        const cudaError_t e = raw_alloc(&q, std::max<size_t>(count, 1) * sizeof(U), st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error(std::string("hoqri_init_hosvd: device allocation: ") + cudaGetErrorString(e));
            return HOQRI_ERR_OOM;
        }
        ptrs.push_back(q);
        *p = static_cast<U *>(q);
        return HOQRI_OK;
    }
};

template <typename T>
hoqri_status hosvd_mode(hoqri_ctx *c, int n, int power_iters) {
    const ModeStore &M = c->ms[n];
    const int64_t nnz = c->nnz;
    const int K = c->K[n];
    const int64_t I = c->dims[n];
    cudaStream_t st = c->stream;
    const int G = hs_grid(nnz, c->num_sms);
    HsTmp tmp(st);
    int32_t *perm, *perm2, *head, *incl, *col_of, *in_of;
    uint32_t *ka, *kb;
    int64_t *col_start = nullptr;
    HQ_TRY(tmp.get(&perm, nnz));
    HQ_TRY(tmp.get(&perm2, nnz));
    HQ_TRY(tmp.get(&head, nnz));
    HQ_TRY(tmp.get(&incl, nnz));
    HQ_TRY(tmp.get(&col_of, nnz));
    HQ_TRY(tmp.get(&in_of, nnz));
    HQ_TRY(tmp.get(&ka, nnz));
    HQ_TRY(tmp.get(&kb, nnz));
    int64_t ncol = 0;
    const int nn = (int)nnz;
    if (nnz > 0) {
        // stable sort of the row-sorted positions by the other modes' indices,
        // least significant mode first
        k_hs_iota<<<G, HS_TPB, 0, st>>>(perm, nnz);
        size_t tb = 0;
        HQ_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, ka, kb, perm, perm2, nn, 0, 32, st));
        size_t tb2 = 0;
        HQ_CUDA(cub::DeviceScan::InclusiveSum(nullptr, tb2, head, incl, nn, st));
        char *tsort;
        HQ_TRY(tmp.get(&tsort, std::max(tb, tb2)));
        int32_t *src = perm, *dst = perm2;
        for (int j = c->N - 2; j >= 0; --j) {
            int m = j < n ? j : j + 1;  // the other mode stored at oidx[j]
            int bits = 1;
            while (bits < 32 && ((int64_t)1 << bits) < c->dims[m]) ++bits;
            k_hs_key<<<G, HS_TPB, 0, st>>>(M.oidx[j], src, nnz, ka);
            HQ_CUDA(cub::DeviceRadixSort::SortPairs(tsort, tb, ka, kb, src, dst, nn, 0, bits, st));
            std::swap(src, dst);
        }
        OtherIdx o{};
        for (int j = 0; j < c->N - 1; ++j) o.p[j] = M.oidx[j];
        k_hs_heads<<<G, HS_TPB, 0, st>>>(o, c->N - 1, src, nnz, head);
        HQ_CUDA(cub::DeviceScan::InclusiveSum(tsort, tb2, head, incl, nn, st));
        int32_t last = 0;
        HQ_CUDA(cudaMemcpyAsync(&last, incl + nnz - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        HQ_CUDA(cudaStreamSynchronize(st));
        ncol = last;
        HQ_TRY(tmp.get(&col_start, ncol + 1));
        k_hs_cols<<<G, HS_TPB, 0, st>>>(head, incl, src, nnz, col_start, col_of);
        k_hs_rows<<<G, HS_TPB, 0, st>>>(M.row_ptr, M.row_id, M.R, nnz, in_of);
        perm = src;
    }
    T *W;
    HQ_TRY(tmp.get(&W, (size_t)std::max<int64_t>(ncol, 1) * K));
    T *V = static_cast<T *>(c->U[n]);
    T *Y = static_cast<T *>(c->A);
    const int Gw = hs_grid(ncol, c->num_sms);
    const int Gy = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(M.R, 1), HS_TPB / 32),
                                                              (int64_t)c->num_sms * 16));
    for (int it = 0; it < power_iters; ++it) {
        HQ_CUDA(cudaMemsetAsync(Y, 0, (size_t)I * K * sizeof(T), st));
        if (nnz > 0) {
            k_hs_w<T><<<Gw, HS_TPB, 0, st>>>(col_start, ncol, perm, static_cast<const T *>(M.vals), in_of, V, K, W);
            k_hs_y<T><<<Gy, HS_TPB, 0, st>>>(M.row_ptr, M.row_id, M.R, static_cast<const T *>(M.vals), col_of, W, K, Y);
            c->nlaunch += 2;
        }
        HQ_TRY(orthonormalize(c, n, Y, V));
    }
    HQ_CUDA(cudaGetLastError());
    HQ_CUDA(cudaStreamSynchronize(st));
    return HOQRI_OK;
}

}  // namespace

hoqri_status init_hosvd(hoqri_ctx *c, int power_iters) {
    // the seeded Gaussian start of every factor (orthonormalised)
    HQ_TRY(init_factors_seeded(c));
    for (int n = 0; n < c->N; ++n) {
        if (c->prec == HOQRI_FP64)
            HQ_TRY(hosvd_mode<double>(c, n, power_iters));
        else
            HQ_TRY(hosvd_mode<float>(c, n, power_iters));
    }
    return HOQRI_OK;
}

}  // namespace hoqri
