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
//   W(c, :) = sum over the positions q of column c of x_q V(i_n(q), :)
//   Y(i, :) = sum over the positions p of row i of x_p W(col(p), :)
// Both are segmented sums over skewed segments (Zipf rows and columns hold up
// to millions of positions), so each segment is cut into pieces of at most
// HS_PIECE positions: one warp sums a piece (lanes take every 32nd position,
// then a fixed butterfly), and a second kernel adds the pieces of each segment
// in order.  The order is fixed, so the result is the same on every run.
#include <cub/cub.cuh>

#include <algorithm>
#include <string>
#include <vector>

#include "hosvd.cuh"
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

constexpr int64_t HS_PIECE = 4096;  // positions per piece of a segment

// pieces per segment: max(1, ceil(len / HS_PIECE))
__global__ void k_hs_piece_count(const int64_t *off, int64_t nseg, int32_t *cnt) {
    for (int64_t sg = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sg < nseg; sg += (int64_t)gridDim.x * blockDim.x) {
        const int64_t len = off[sg + 1] - off[sg];
        const int64_t np = (len + HS_PIECE - 1) / HS_PIECE;
        cnt[sg] = (int32_t)(np > 1 ? np : 1);
    }
}

// piece -> (segment, index within the segment)
__global__ void k_hs_piece_fill(const int32_t *cnt, const int32_t *poff, int64_t nseg, int32_t *pseg, int32_t *pj) {
    for (int64_t sg = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sg < nseg; sg += (int64_t)gridDim.x * blockDim.x)
        for (int j = 0; j < cnt[sg]; ++j) {
            pseg[poff[sg] + j] = (int32_t)sg;
            pj[poff[sg] + j] = j;
        }
}

// part(piece, :) = sum over the piece's positions q of x_p Gm(gidx(p), :), with
// p = pmap(q) (pmap NULL: p = q); one warp per piece, K in chunks of HS_KCH
template <typename T>
__global__ void __launch_bounds__(HS_TPB) k_hs_pieces(const int64_t *off, const int32_t *pseg, const int32_t *pj,
                                                      int64_t npiece, const int32_t *pmap, const T *vals,
                                                      const int32_t *gidx, const T *Gm, int K, T *part) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < npiece; w += warps) {
        const int64_t sg = pseg[w];
        const int64_t q0 = off[sg] + (int64_t)pj[w] * HS_PIECE;
        const int64_t q1 = min(off[sg + 1], q0 + HS_PIECE);
        for (int kc = 0; kc < K; kc += HS_KCH) {
            T acc[HS_KCH];
#pragma unroll
            for (int k = 0; k < HS_KCH; ++k) acc[k] = T(0);
            for (int64_t q = q0 + lane; q < q1; q += 32) {
                const int64_t p = pmap ? (int64_t)pmap[q] : q;
                const T x = vals[p];
                const T *g = Gm + (int64_t)gidx[p] * K + kc;
#pragma unroll
                for (int k = 0; k < HS_KCH; ++k)
                    if (kc + k < K) acc[k] += x * g[k];
            }
#pragma unroll
            for (int k = 0; k < HS_KCH; ++k)
                for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < HS_KCH; ++k)
                    if (kc + k < K) part[w * K + kc + k] = acc[k];
            }
        }
    }
}

// out(dst(s), :) = sum of the pieces of segment s in order; dst = s when
// dst_id is NULL
template <typename T>
__global__ void k_hs_combine(const int32_t *cnt, const int32_t *poff, int64_t nseg, const T *part, int K,
                             const int32_t *dst_id, T *out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nseg * K; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sg = t / K;
        const int k = (int)(t - sg * K);
        T s = T(0);
        for (int j = 0; j < cnt[sg]; ++j) s += part[(int64_t)(poff[sg] + j) * K + k];
        out[(dst_id ? (int64_t)dst_id[sg] : sg) * K + k] = s;
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
    T *V = static_cast<T *>(c->U[n]);
    T *Y = static_cast<T *>(c->A);
    if (nnz == 0) {
        // X_(n) = 0: the QR of a zero Y completes an orthonormal basis
        for (int it = 0; it < power_iters; ++it) {
            HQ_CUDA(cudaMemsetAsync(Y, 0, (size_t)I * K * sizeof(T), st));
            HQ_TRY(orthonormalize(c, n, Y, V));
        }
        HQ_CUDA(cudaStreamSynchronize(st));
        return HOQRI_OK;
    }
    // pieces of the columns (column-sorted positions) and of the rows
    struct Pieces {
        int32_t *cnt = nullptr, *poff = nullptr, *pseg = nullptr, *pj = nullptr;
        int64_t n = 0;
    };
    auto make_pieces = [&](const int64_t *off, int64_t nseg, Pieces *pc) -> hoqri_status {
        HQ_TRY(tmp.get(&pc->cnt, nseg));
        HQ_TRY(tmp.get(&pc->poff, nseg));
        const int g = hs_grid(nseg, c->num_sms);
        k_hs_piece_count<<<g, HS_TPB, 0, st>>>(off, nseg, pc->cnt);
        size_t tb = 0;
        HQ_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tb, pc->cnt, pc->poff, (int)nseg, st));
        char *t;
        HQ_TRY(tmp.get(&t, tb));
        HQ_CUDA(cub::DeviceScan::ExclusiveSum(t, tb, pc->cnt, pc->poff, (int)nseg, st));
        int32_t h[2] = {0, 0};
        HQ_CUDA(cudaMemcpyAsync(&h[0], pc->poff + nseg - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        HQ_CUDA(cudaMemcpyAsync(&h[1], pc->cnt + nseg - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        HQ_CUDA(cudaStreamSynchronize(st));
        pc->n = (int64_t)h[0] + h[1];
        HQ_TRY(tmp.get(&pc->pseg, pc->n));
        HQ_TRY(tmp.get(&pc->pj, pc->n));
        k_hs_piece_fill<<<g, HS_TPB, 0, st>>>(pc->cnt, pc->poff, nseg, pc->pseg, pc->pj);
        return HOQRI_OK;
    };
    Pieces pcol, prow;
    HQ_TRY(make_pieces(col_start, ncol, &pcol));
    HQ_TRY(make_pieces(M.row_ptr, M.R, &prow));
    T *W, *part;
    HQ_TRY(tmp.get(&W, (size_t)ncol * K));
    HQ_TRY(tmp.get(&part, (size_t)std::max(pcol.n, prow.n) * K));
    auto warp_grid = [&](int64_t pieces) {
        return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(pieces, HS_TPB / 32), (int64_t)c->num_sms * 16));
    };
    const T *vals = static_cast<const T *>(M.vals);
    for (int it = 0; it < power_iters; ++it) {
        // W = X_(n)^T V over the columns, then Y = X_(n) W over the rows
        k_hs_pieces<T><<<warp_grid(pcol.n), HS_TPB, 0, st>>>(col_start, pcol.pseg, pcol.pj, pcol.n, perm, vals, in_of,
                                                             V, K, part);
        k_hs_combine<T><<<hs_grid(ncol * K, c->num_sms), HS_TPB, 0, st>>>(pcol.cnt, pcol.poff, ncol, part, K, nullptr, W);
        HQ_CUDA(cudaMemsetAsync(Y, 0, (size_t)I * K * sizeof(T), st));
        k_hs_pieces<T><<<warp_grid(prow.n), HS_TPB, 0, st>>>(M.row_ptr, prow.pseg, prow.pj, prow.n, nullptr, vals,
                                                             col_of, W, K, part);
        k_hs_combine<T><<<hs_grid(M.R * K, c->num_sms), HS_TPB, 0, st>>>(prow.cnt, prow.poff, M.R, part, K, M.row_id, Y);
        c->nlaunch += 4;
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
