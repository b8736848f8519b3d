// Set-up of the sparse tensor on the device (once per tensor).
//
// 1. Check every index against its mode size.
// 2. Sum repeated coordinates: stable radix sort of the coordinates into
//    lexicographic (i_1, ..., i_N) order, then one FP64 sum per run in input
//    order.  I(X) is a set of positions (Table 1), so repeats denote one entry.
// 3. ||X||^2 in FP64.
// 4. Per mode n: stable radix sort by i_n (ties keep the lexicographic order),
//    the permutation perm_n, the other modes' indices and the values gathered
//    into that order (structure of arrays), and the row descriptors: the
//    non-empty mode-n slices I^(n)_{i_n} of Table 1 as (row_id, row_ptr).
// 5. The partition of each sorted stream into warp tasks: whole rows packed
//    up to C nonzeros per task, rows longer than C cut into pieces.
//
// Sorting and compaction use CUB (CUDA's header library); everything here runs
// once per tensor, outside the iteration.
#include <cub/cub.cuh>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "internal.cuh"

namespace hoqri {

namespace {

constexpr int TPB = 256;

inline int grid_for(int64_t n, int tpb = TPB) {
    int64_t g = (n + tpb - 1) / tpb;
    return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 1 << 30);
}

struct IdxPack {
    const int32_t *p[HOQRI_MAXN];
};
struct IdxPackW {
    int32_t *p[HOQRI_MAXN];
};

__global__ void k_validate(IdxPack idx, int N, int64_t nnz, const int64_t *dims_dev, int32_t *bad) {
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < nnz; z += (int64_t)gridDim.x * blockDim.x) {
        for (int m = 0; m < N; ++m) {
            int32_t v = idx.p[m][z];
            if (v < 0 || (int64_t)v >= dims_dev[m]) atomicExch(bad, 1);
        }
    }
}

__global__ void k_pack_keys(IdxPack idx, int N, int64_t nnz, const int32_t *shift_dev, uint64_t *keys, int32_t *iota) {
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < nnz; z += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = 0;
        for (int m = 0; m < N; ++m) k |= (uint64_t)(uint32_t)idx.p[m][z] << shift_dev[m];
        keys[z] = k;
        iota[z] = (int32_t)z;
    }
}

__global__ void k_iota(int32_t *a, int64_t n) {
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < n; z += (int64_t)gridDim.x * blockDim.x)
        a[z] = (int32_t)z;
}

__global__ void k_gather_key(const int32_t *src, const int32_t *perm, int64_t n, uint32_t *dst) {
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < n; z += (int64_t)gridDim.x * blockDim.x)
        dst[z] = (uint32_t)src[perm[z]];
}

// head[s] = 1 if sorted position s starts a new coordinate
__global__ void k_heads(IdxPack idx, int N, const int32_t *perm, int64_t n, int32_t *head) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        int h = 1;
        if (s > 0) {
            int32_t a = perm[s], b = perm[s - 1];
            h = 0;
            for (int m = 0; m < N; ++m) h |= (idx.p[m][a] != idx.p[m][b]);
        }
        head[s] = h;
    }
}

__global__ void k_run_starts(const int32_t *head, const int32_t *incl, int64_t n, int64_t *run_start) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        if (head[s]) run_start[incl[s] - 1] = s;
}

template <typename T>
__global__ void k_coalesce_values(IdxPack idx, IdxPackW cidx, int N, const int32_t *perm, const int64_t *run_start,
                                  int64_t nu, int64_t n, const T *vals, T *cval) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nu; u += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = run_start[u], b = (u + 1 < nu) ? run_start[u + 1] : n;
        double s = 0.0;
        for (int64_t q = a; q < b; ++q) s += (double)vals[perm[q]];
        cval[u] = (T)s;
        int32_t z = perm[a];
        for (int m = 0; m < N; ++m) cidx.p[m][u] = idx.p[m][z];
    }
}

// bit layout of the packed lexicographic key: mode m at bits [shift[m], shift[m] + bits[m])
struct KeyLayout {
    int32_t shift[HOQRI_MAXN];
    int32_t bits[HOQRI_MAXN];
};

// head[s] = 1 if sorted position s starts a new coordinate (equal packed keys are equal coordinates)
__global__ void k_heads_keys(const uint64_t *keys, int64_t n, int32_t *head) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        head[s] = (s == 0) || (keys[s] != keys[s - 1]);
}

// one coordinate per run of equal sorted keys: its value is the FP64 sum of the
// run's values in sorted (= input, the sort is stable) order, its indices are
// unpacked from the key
template <typename T>
__global__ void k_coalesce_sorted(const uint64_t *keys, const T *svals, KeyLayout kl, IdxPackW cidx, int N,
                                  const int64_t *run_start, int64_t nu, int64_t n, T *cval) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nu; u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = run_start[u], b = (u + 1 < nu) ? run_start[u + 1] : n;
        double s = 0.0;
        for (int64_t q = a; q < b; ++q) s += (double)svals[q];
        cval[u] = (T)s;
        const uint64_t k = keys[a];
        for (int m = 0; m < N; ++m) cidx.p[m][u] = (int32_t)((k >> kl.shift[m]) & ((1ull << kl.bits[m]) - 1));
    }
}

// deterministic FP64 sum of squares: fixed grid, fixed per-thread stride, tree in shared memory
template <typename T>
__global__ void k_sumsq_partial(const T *v, int64_t n, double *part) {
    __shared__ double sh[TPB];
    double s = 0.0;
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < n; z += (int64_t)gridDim.x * blockDim.x) {
        double x = (double)v[z];
        s += x * x;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = TPB / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_small(const double *part, int n, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = s;
    }
}

template <typename T>
__global__ void k_gather_mode(IdxPack cidx, IdxPackW oidx, int N, int n, const int32_t *perm, int64_t nnz,
                              const T *cval, T *vals) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nnz; s += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = perm[s];
        int j = 0;
        for (int m = 0; m < N; ++m) {
            if (m == n) continue;
            oidx.p[j++][s] = cidx.p[m][u];
        }
        vals[s] = cval[u];
    }
}

__global__ void k_row_heads(const uint32_t *keys, int64_t n, int32_t *head) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        head[s] = (s == 0) || (keys[s] != keys[s - 1]);
}

__global__ void k_row_desc(const uint32_t *keys, const int32_t *head, const int32_t *incl, int64_t n, int32_t *row_id,
                           int64_t *row_ptr) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        if (head[s]) {
            int32_t r = incl[s] - 1;
            row_id[r] = (int32_t)keys[s];
            row_ptr[r] = s;
        }
    }
}

__global__ void k_set_last(int64_t *row_ptr, int64_t R, int64_t n) { row_ptr[R] = n; }

// hybrid copy: dst[p] = src[map[p]] (map -1: padding entry, index 0 and value 0)
template <typename T>
__global__ void k_hyb_gather(IdxPack src, IdxPackW dst, int nm1, const int32_t *map, int64_t total, const T *vsrc,
                             T *vdst) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = map[p];
        for (int j = 0; j < nm1; ++j) dst.p[j][p] = q >= 0 ? src.p[j][q] : 0;
        vdst[p] = q >= 0 ? vsrc[q] : T(0);
    }
}

// map of the long part: position lrp[j] + q holds sorted position row_ptr[lrow[j]] + q;
// a thread per position finds its row j by binary search over lrp (Zipf rows
// differ in length by orders of magnitude, so a block per row would leave
// one block with most of the work)
__global__ void k_map_long(const int64_t *lrp, const int32_t *lrow, const int64_t *row_ptr, int64_t nlong,
                           int32_t *map) {
    const int64_t total = lrp[nlong];
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nlong - 1;  // last j with lrp[j] <= p
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (lrp[mid] <= p) lo = mid;
            else hi = mid - 1;
        }
        map[p] = (int32_t)(row_ptr[lrow[lo]] + (p - lrp[lo]));
    }
}

// map of the slices: position sbase[j] + SW*q + g holds sorted position
// row_ptr[r] + q of the slice's row g (r = srow[SW*j + g]) for q < its length
__global__ void k_map_slices(const int64_t *sbase, const int32_t *srow, const int64_t *row_ptr, int64_t nslice, int SW,
                             int32_t *map) {
    for (int64_t j = blockIdx.x; j < nslice; j += gridDim.x) {
        const int64_t b = sbase[j], e = sbase[j + 1];
        for (int64_t p = b + threadIdx.x; p < e; p += blockDim.x) {
            const int64_t off = p - b, q = off / SW;
            const int g = (int)(off - q * SW);
            const int32_t r = srow[SW * j + g];
            if (r >= 0 && q < row_ptr[r + 1] - row_ptr[r]) map[p] = (int32_t)(row_ptr[r] + q);
        }
    }
}

// RAII holder for set-up temporaries
struct Tmp {
    cudaStream_t st;
    std::vector<void *> ptrs;
    explicit Tmp(cudaStream_t s) : st(s) {}
    ~Tmp() {
        for (void *p : ptrs) raw_free(p, st);
    }
    template <typename T>
    hoqri_status get(T **p, size_t count) {
        void *q = nullptr;
        cudaError_t e = raw_alloc(&q, std::max<size_t>(count, 1) * sizeof(T), st);
        if (e != cudaSuccess) {
            set_error(std::string("set-up allocation: ") + cudaGetErrorString(e));
            return HOQRI_ERR_OOM;
        }
        ptrs.push_back(q);
        *p = (T *)q;
        return HOQRI_OK;
    }
};

int bits_for(int64_t dim) {
    int b = 0;
    while (b < 63 && ((int64_t)1 << b) < dim) ++b;
    return std::max(b, 1);
}

}  // namespace

template <typename T>
static hoqri_status build_storage_t(hoqri_ctx *c, const int32_t *const *idx_dev, const void *vals_dev, int64_t nnz_raw) {
    cudaStream_t st = c->stream;
    const int N = c->N;
    Tmp tmp(c->stream);
    const int G = std::min(grid_for(nnz_raw), c->num_sms * 8);
    IdxPack in{};
    for (int m = 0; m < N; ++m) in.p[m] = idx_dev[m];

    // ---- 1. validate
    int64_t *dims_dev;
    int32_t *bad;
    HQ_TRY(tmp.get(&dims_dev, N));
    HQ_TRY(tmp.get(&bad, 1));
    HQ_CUDA(cudaMemcpyAsync(dims_dev, c->dims, N * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    HQ_CUDA(cudaMemsetAsync(bad, 0, sizeof(int32_t), st));
    if (nnz_raw > 0) k_validate<<<G, TPB, 0, st>>>(in, N, nnz_raw, dims_dev, bad);
    int32_t hbad = 0;
    HQ_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    HQ_CUDA(cudaStreamSynchronize(st));
    if (hbad) {
        set_error("hoqri_create: an index is outside [0, dims[m])");
        return HOQRI_ERR_INVALID;
    }

    // ---- 2. lexicographic stable sort of the raw coordinates.  When the packed
    // coordinate fits 64 bits the (key, value) pairs are sorted together: equal
    // coordinates become adjacent with their values in input order, and the
    // coordinates are unpacked from the keys (no gathers through a permutation).
    // Otherwise a permutation is sorted mode by mode (least significant first,
    // stable passes give lexicographic order) and gathered through.
    int total_bits = 0;
    KeyLayout kl{};
    for (int m = N - 1; m >= 0; --m) {
        kl.shift[m] = total_bits;
        kl.bits[m] = bits_for(c->dims[m]);
        total_bits += kl.bits[m];
    }
    const bool packed = total_bits <= 64;
    const int nn = (int)nnz_raw;
    int32_t *perm = nullptr;
    uint64_t *skeys = nullptr;
    T *svals = nullptr;
    if (nnz_raw > 0 && packed) {
        uint64_t *ka;
        int32_t *shift_dev, *unused;
        HQ_TRY(tmp.get(&ka, nnz_raw));
        HQ_TRY(tmp.get(&skeys, nnz_raw));
        HQ_TRY(tmp.get(&svals, nnz_raw));
        HQ_TRY(tmp.get(&unused, nnz_raw));
        HQ_TRY(tmp.get(&shift_dev, N));
        HQ_CUDA(cudaMemcpyAsync(shift_dev, kl.shift, N * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        k_pack_keys<<<G, TPB, 0, st>>>(in, N, nnz_raw, shift_dev, ka, unused);
        size_t tb = 0;
        HQ_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, ka, skeys, (const T *)vals_dev, svals, nn, 0, total_bits,
                                                st));
        char *t;
        HQ_TRY(tmp.get(&t, tb));
        HQ_CUDA(cub::DeviceRadixSort::SortPairs(t, tb, ka, skeys, (const T *)vals_dev, svals, nn, 0, total_bits, st));
    } else if (nnz_raw > 0) {
        int32_t *perm_a, *perm_b;
        HQ_TRY(tmp.get(&perm_a, nnz_raw));
        HQ_TRY(tmp.get(&perm_b, nnz_raw));
        uint32_t *ka, *kb;
        HQ_TRY(tmp.get(&ka, nnz_raw));
        HQ_TRY(tmp.get(&kb, nnz_raw));
        k_iota<<<G, TPB, 0, st>>>(perm_a, nnz_raw);
        size_t tb = 0;
        HQ_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, ka, kb, perm_a, perm_b, nn, 0, 32, st));
        char *t;
        HQ_TRY(tmp.get(&t, tb));
        int32_t *src = perm_a, *dst = perm_b;
        for (int m = N - 1; m >= 0; --m) {
            k_gather_key<<<G, TPB, 0, st>>>(idx_dev[m], src, nnz_raw, ka);
            HQ_CUDA(cub::DeviceRadixSort::SortPairs(t, tb, ka, kb, src, dst, nn, 0, bits_for(c->dims[m]), st));
            std::swap(src, dst);
        }
        perm = src;
    }

    // ---- runs of equal coordinates
    int32_t *head, *incl;
    HQ_TRY(tmp.get(&head, nnz_raw));
    HQ_TRY(tmp.get(&incl, nnz_raw));
    int64_t nu = 0;
    if (nnz_raw > 0) {
        if (packed) k_heads_keys<<<G, TPB, 0, st>>>(skeys, nnz_raw, head);
        else k_heads<<<G, TPB, 0, st>>>(in, N, perm, nnz_raw, head);
        size_t tb = 0;
        HQ_CUDA(cub::DeviceScan::InclusiveSum(nullptr, tb, head, incl, nn, st));
        char *t;
        HQ_TRY(tmp.get(&t, tb));
        HQ_CUDA(cub::DeviceScan::InclusiveSum(t, tb, head, incl, nn, st));
        int32_t last = 0;
        HQ_CUDA(cudaMemcpyAsync(&last, incl + nnz_raw - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        HQ_CUDA(cudaStreamSynchronize(st));
        nu = last;
    }
    c->nnz = nu;

    int64_t *run_start;
    HQ_TRY(tmp.get(&run_start, nu));
    IdxPackW cidx{};
    for (int m = 0; m < N; ++m) HQ_TRY(tmp.get(&cidx.p[m], nu));
    T *cval;
    HQ_TRY(tmp.get(&cval, nu));
    if (nu > 0) {
        k_run_starts<<<G, TPB, 0, st>>>(head, incl, nnz_raw, run_start);
        const int Gc = std::min(grid_for(nu), c->num_sms * 8);
        if (packed)
            k_coalesce_sorted<T><<<Gc, TPB, 0, st>>>(skeys, svals, kl, cidx, N, run_start, nu, nnz_raw, cval);
        else
            k_coalesce_values<T><<<Gc, TPB, 0, st>>>(in, cidx, N, perm, run_start, nu, nnz_raw, (const T *)vals_dev,
                                                     cval);
    }

    // ---- 3. ||X||^2
    {
        const int NB = 1024;
        double *part;
        HQ_TRY(tmp.get(&part, NB));
        HQ_CUDA(cudaMemsetAsync(part, 0, NB * sizeof(double), st));
        if (nu > 0) k_sumsq_partial<T><<<NB, TPB, 0, st>>>(cval, nu, part);
        k_sum_small<<<1, 32, 0, st>>>(part, NB, c->dnorm + 0);
    }

    // ---- 4. per-mode sorted copies
    IdxPack cin{};
    for (int m = 0; m < N; ++m) cin.p[m] = cidx.p[m];
    uint32_t *ka, *kb;
    int32_t *ia;
    HQ_TRY(tmp.get(&ka, nu));
    HQ_TRY(tmp.get(&kb, nu));
    HQ_TRY(tmp.get(&ia, nu));
    int32_t *rhead, *rincl;
    HQ_TRY(tmp.get(&rhead, nu));
    HQ_TRY(tmp.get(&rincl, nu));
    size_t tb_sort = 0, tb_scan = 0;
    const int nun = (int)nu;
    if (nu > 0) {
        HQ_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb_sort, ka, kb, ia, ia, nun, 0, 32, st));
        HQ_CUDA(cub::DeviceScan::InclusiveSum(nullptr, tb_scan, rhead, rincl, nun, st));
    }
    char *tsort, *tscan;
    HQ_TRY(tmp.get(&tsort, tb_sort));
    HQ_TRY(tmp.get(&tscan, tb_scan));
    const int Gu = std::min(grid_for(nu), c->num_sms * 8);
    for (int n = 0; n < N; ++n) {
        ModeStore &M = c->ms[n];
        HQ_TRY(dalloc(c, (void **)&M.perm, std::max<int64_t>(nu, 1) * sizeof(int32_t)));
        HQ_TRY(dalloc(c, &M.vals, (nu + 16) * sizeof(T)));
        IdxPackW ow{};
        for (int j = 0; j < N - 1; ++j) {
            HQ_TRY(dalloc(c, (void **)&M.oidx[j], (nu + 16) * sizeof(int32_t)));
            ow.p[j] = M.oidx[j];
        }
        int64_t R = 0;
        // the coalesced coordinates are in lexicographic order with mode 0 most
        // significant, so the stable sort by i_0 is the identity: mode 0 copies
        const uint32_t *skey = n == 0 ? reinterpret_cast<const uint32_t *>(cidx.p[0]) : kb;
        if (nu > 0 && n == 0) {
            k_iota<<<Gu, TPB, 0, st>>>(M.perm, nu);
            for (int m = 1; m < N; ++m)
                HQ_CUDA(cudaMemcpyAsync(ow.p[m - 1], cidx.p[m], nu * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
            HQ_CUDA(cudaMemcpyAsync(M.vals, cval, nu * sizeof(T), cudaMemcpyDeviceToDevice, st));
        } else if (nu > 0) {
            HQ_CUDA(cudaMemcpyAsync(ka, cidx.p[n], nu * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
            k_iota<<<Gu, TPB, 0, st>>>(ia, nu);
            HQ_CUDA(cub::DeviceRadixSort::SortPairs(tsort, tb_sort, ka, kb, ia, M.perm, nun, 0, bits_for(c->dims[n]), st));
            k_gather_mode<T><<<Gu, TPB, 0, st>>>(cin, ow, N, n, M.perm, nu, cval, (T *)M.vals);
        }
        if (nu > 0) {
            k_row_heads<<<Gu, TPB, 0, st>>>(skey, nu, rhead);
            HQ_CUDA(cub::DeviceScan::InclusiveSum(tscan, tb_scan, rhead, rincl, nun, st));
            int32_t Rh = 0;
            HQ_CUDA(cudaMemcpyAsync(&Rh, rincl + nu - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            HQ_CUDA(cudaStreamSynchronize(st));
            R = Rh;
        }
        M.R = R;
        HQ_TRY(dalloc(c, (void **)&M.row_id, std::max<int64_t>(R, 1) * sizeof(int32_t)));
        HQ_TRY(dalloc(c, (void **)&M.row_ptr, (R + 1) * sizeof(int64_t)));
        if (nu > 0) k_row_desc<<<Gu, TPB, 0, st>>>(skey, rhead, rincl, nu, M.row_id, M.row_ptr);
        k_set_last<<<1, 1, 0, st>>>(M.row_ptr, R, nu);
    }
    HQ_CUDA(cudaGetLastError());
    HQ_CUDA(cudaStreamSynchronize(st));
    return HOQRI_OK;
}

hoqri_status build_storage(hoqri_ctx *c, const int32_t *const *idx_dev, const void *vals_dev, int64_t nnz_raw) {
    if (nnz_raw >= (int64_t)INT32_MAX) {
        set_error("hoqri_create: nnz must be below 2^31");
        return HOQRI_ERR_UNSUPPORTED;
    }
    if (c->prec == HOQRI_FP64) return build_storage_t<double>(c, idx_dev, vals_dev, nnz_raw);
    return build_storage_t<float>(c, idx_dev, vals_dev, nnz_raw);
}

hoqri_status build_partition(hoqri_ctx *c, int n, int32_t C) {
    ModeStore &M = c->ms[n];
    cudaStream_t st = c->stream;
    dfree(M.chunk_start, c->stream);
    dfree(M.chunk_row, c->stream);
    dfree(M.big, c->stream);
    M.chunk_start = nullptr;
    M.chunk_row = nullptr;
    M.big = nullptr;
    M.C = C;
    std::vector<int64_t> rp(M.R + 1);
    HQ_CUDA(cudaMemcpyAsync(rp.data(), M.row_ptr, (M.R + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    HQ_CUDA(cudaStreamSynchronize(st));
    std::vector<int64_t> starts;
    std::vector<int32_t> crow, big;
    int64_t cur_start = 0, cur_len = 0;
    int32_t cur_row = 0;
    auto close = [&]() {
        if (cur_len > 0) {
            starts.push_back(cur_start);
            crow.push_back(cur_row);
            cur_len = 0;
        }
    };
    for (int64_t r = 0; r < M.R; ++r) {
        const int64_t len = rp[r + 1] - rp[r];
        if (len > C) {
            close();
            const int64_t np = (len + C - 1) / C;
            big.push_back((int32_t)r);
            big.push_back((int32_t)starts.size());
            for (int64_t q = 0; q < np; ++q) {
                starts.push_back(rp[r] + (len * q) / np);
                crow.push_back((int32_t)r);
            }
            big.push_back((int32_t)starts.size() - 1);
        } else {
            if (cur_len + len > C) close();
            if (cur_len == 0) {
                cur_start = rp[r];
                cur_row = (int32_t)r;
            }
            cur_len += len;
        }
    }
    close();
    M.nchunks = (int64_t)starts.size();
    starts.push_back(c->nnz);
    M.nbig = (int64_t)big.size() / 3;
    HQ_TRY(dalloc(c, (void **)&M.chunk_start, starts.size() * sizeof(int64_t)));
    HQ_TRY(dalloc(c, (void **)&M.chunk_row, std::max<size_t>(crow.size(), 1) * sizeof(int32_t)));
    HQ_TRY(dalloc(c, (void **)&M.big, std::max<size_t>(big.size(), 1) * sizeof(int32_t)));
    HQ_CUDA(cudaMemcpyAsync(M.chunk_start, starts.data(), starts.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (!crow.empty())
        HQ_CUDA(cudaMemcpyAsync(M.chunk_row, crow.data(), crow.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (!big.empty())
        HQ_CUDA(cudaMemcpyAsync(M.big, big.data(), big.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    HQ_CUDA(cudaStreamSynchronize(st));
    return HOQRI_OK;
}

template <typename T>
static hoqri_status build_hybrid_t(hoqri_ctx *c, int n, int64_t Lshort, int64_t T8, int SW) {
    ModeStore &M = c->ms[n];
    cudaStream_t st = c->stream;
    const int nm1 = c->N - 1;
    std::vector<int64_t> rp(M.R + 1);
    HQ_CUDA(cudaMemcpyAsync(rp.data(), M.row_ptr, (M.R + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    HQ_CUDA(cudaStreamSynchronize(st));
    std::vector<int32_t> lrow, srt;
    // short rows by length, longest first, ties in row order (a counting sort:
    // lengths are at most Lshort)
    std::vector<int64_t> nlen(Lshort + 2, 0);
    for (int64_t r = 0; r < M.R; ++r) {
        const int64_t len = rp[r + 1] - rp[r];
        if (len > Lshort) lrow.push_back((int32_t)r);
        else ++nlen[Lshort - len + 1];
    }
    for (int64_t l = 1; l <= Lshort + 1; ++l) nlen[l] += nlen[l - 1];
    srt.resize((size_t)nlen[Lshort + 1]);
    for (int64_t r = 0; r < M.R; ++r) {
        const int64_t len = rp[r + 1] - rp[r];
        if (len <= Lshort) srt[(size_t)nlen[Lshort - len]++] = (int32_t)r;
    }
    const int64_t nlong = (int64_t)lrow.size();
    std::vector<int64_t> lrp(nlong + 1, 0);
    for (int64_t j = 0; j < nlong; ++j) lrp[j + 1] = lrp[j] + (rp[lrow[j] + 1] - rp[lrow[j]]);
    const int64_t total_long = lrp[nlong];
    M.long_elems = total_long;
    const int64_t nslice = ((int64_t)srt.size() + SW - 1) / SW;
    std::vector<int64_t> sbase(nslice + 1);
    std::vector<int32_t> srow((size_t)SW * nslice, -1);
    sbase[0] = (total_long + 31) & ~(int64_t)31;
    for (int64_t j = 0; j < nslice; ++j) {
        for (int g = 0; g < SW && SW * j + g < (int64_t)srt.size(); ++g) srow[SW * j + g] = srt[SW * j + g];
        const int64_t L = rp[srow[SW * j] + 1] - rp[srow[SW * j]];
        // slice sizes stay multiples of 4 elements so every slice starts 16-byte aligned
        sbase[j + 1] = sbase[j] + ((SW * L + 3) & ~(int64_t)3);
    }
    const int64_t total = sbase[nslice];
    // work items: the long part in items of TL elements (at least T8, and at
    // least an equal share per warp of the pass, so a warp's range is one item
    // and its windows run on across the rows of the range), then runs of slices
    FastTile tile;
    const int bps = hyb_tile(c, n, &tile) ? hyb_blocks_per_sm(tile) : HY_BLOCKS_PER_SM;
    const int64_t W = (int64_t)c->num_sms * bps * 8;
    const int64_t TL = std::max<int64_t>(T8, ((total_long + W - 1) / W + 31) & ~(int64_t)31);
    std::vector<int64_t> is, ie;
    std::vector<int32_t> ia, span;
    {
        int64_t j = 0;
        for (int64_t t0 = 0; t0 < total_long; t0 += TL) {
            while (j + 1 < nlong && lrp[j + 1] <= t0) ++j;
            is.push_back(t0);
            ie.push_back(std::min(t0 + TL, total_long));
            ia.push_back((int32_t)j);
        }
    }
    const int64_t nitem_long = (int64_t)is.size();
    // slice items of about T8/8 cost units: one per stored element plus P_{-n}/8
    // per row (the row of Y it writes), so items of many tiny rows stay small.
    // Slice items are dealt round-robin to the warps; at an eighth of the long
    // item size each warp gets some twenty, which keeps the SMs level.
    int64_t Pm = 1;
    for (int m = 0; m < c->N; ++m)
        if (m != n) Pm *= c->K[m];
    const int64_t row_cost = std::max<int64_t>(1, Pm / 8);
    const int64_t Ts = std::max<int64_t>(256, T8 / 8);
    for (int64_t j = 0; j < nslice;) {
        int64_t k = j, cost = 0;
        while (k < nslice && cost < Ts) {
            cost += (sbase[k + 1] - sbase[k]) + (int64_t)SW * row_cost;
            ++k;
        }
        is.push_back(sbase[j]);
        ie.push_back(sbase[k]);
        ia.push_back((int32_t)j);
        j = k;
    }
    // long items: contiguous ranges, one per warp of the pass's fixed grid,
    // so a long row crossing items inside a range carries its partial sum; a long
    // row crossing a range boundary is completed from per-range pieces.  Slice
    // items are dealt to the warps in turn.
    const int64_t ipw = std::max<int64_t>(1, (nitem_long + W - 1) / W);
    const int64_t nrange = std::max<int64_t>(1, (nitem_long + ipw - 1) / ipw);
    for (int64_t jj = 0; jj < nlong; ++jj) {
        const int64_t ta = lrp[jj] / TL, tb = (lrp[jj + 1] - 1) / TL;
        const int64_t ra = ta / ipw, rb = tb / ipw;
        if (ra != rb) {
            span.push_back((int32_t)jj);
            span.push_back((int32_t)ra);
            span.push_back((int32_t)rb);
        }
    }
    M.ipw = ipw;
    M.nrange = nrange;
    M.hyb = true;
    M.htotal = total;
    M.nlong = nlong;
    M.nslice = nslice;
    M.nitem_long = nitem_long;
    M.nitem = (int64_t)is.size();
    M.nspan = (int64_t)span.size() / 3;
    auto up = [&](auto **d, const auto &v) -> hoqri_status {
        using E = typename std::decay<decltype(v[0])>::type;
        HQ_TRY(dalloc(c, (void **)d, std::max<size_t>(v.size(), 1) * sizeof(E)));
        if (!v.empty()) HQ_CUDA(cudaMemcpyAsync(*d, v.data(), v.size() * sizeof(E), cudaMemcpyHostToDevice, st));
        return HOQRI_OK;
    };
    HQ_TRY(up(&M.lrp, lrp));
    HQ_TRY(up(&M.lrow, lrow));
    HQ_TRY(up(&M.sbase, sbase));
    HQ_TRY(up(&M.srow, srow));
    // hybrid position -> sorted position (-1: padding), built on the device
    Tmp tmp(c->stream);
    int32_t *dmap;
    HQ_TRY(tmp.get(&dmap, total + 16));
    HQ_CUDA(cudaMemsetAsync(dmap, 0xFF, (total + 16) * sizeof(int32_t), st));
    if (nlong > 0)
        k_map_long<<<std::min(grid_for(total_long), c->num_sms * 8), TPB, 0, st>>>(M.lrp, M.lrow, M.row_ptr, nlong,
                                                                                   dmap);
    if (nslice > 0)
        k_map_slices<<<(unsigned)std::min<int64_t>(nslice, 1 << 20), 64, 0, st>>>(M.sbase, M.srow, M.row_ptr, nslice,
                                                                                 SW, dmap);
    IdxPack src{};
    IdxPackW dst{};
    for (int j = 0; j < nm1; ++j) {
        HQ_TRY(dalloc(c, (void **)&M.hidx[j], (total + 16) * sizeof(int32_t)));
        src.p[j] = M.oidx[j];
        dst.p[j] = M.hidx[j];
    }
    HQ_TRY(dalloc(c, &M.hvals, (total + 16) * sizeof(T)));
    k_hyb_gather<T><<<std::min(grid_for(total + 16), c->num_sms * 8), TPB, 0, st>>>(
        src, dst, nm1, dmap, total + 16, (const T *)M.vals, (T *)M.hvals);
    HQ_TRY(up(&M.item_s, is));
    HQ_TRY(up(&M.item_e, ie));
    HQ_TRY(up(&M.item_aux, ia));
    HQ_TRY(up(&M.span, span));
    HQ_CUDA(cudaGetLastError());
    HQ_CUDA(cudaStreamSynchronize(st));
    return HOQRI_OK;
}

hoqri_status build_hybrid(hoqri_ctx *c, int n, int64_t Lshort, int64_t T, int SW) {
    const int64_t T32 = std::max<int64_t>(32, (T + 31) & ~(int64_t)31);
    const int64_t b0 = c->device_bytes;
    hoqri_status s = c->prec == HOQRI_FP64 ? build_hybrid_t<double>(c, n, Lshort, T32, SW)
                                            : build_hybrid_t<float>(c, n, Lshort, T32, SW);
    ModeStore &M = c->ms[n];
    M.tune_Lshort = Lshort;
    M.tune_T = T;
    M.hyb_bytes = c->device_bytes - b0;
    return s;
}

void free_hybrid(hoqri_ctx *c, int n) {
    ModeStore &M = c->ms[n];
    cudaStream_t st = c->stream;
    for (int j = 0; j < HOQRI_MAXN - 1; ++j) {
        dfree(M.hidx[j], st);
        M.hidx[j] = nullptr;
    }
    void **arrs[] = {&M.hvals, (void **)&M.lrp, (void **)&M.lrow, (void **)&M.sbase, (void **)&M.srow,
                     (void **)&M.item_s, (void **)&M.item_e, (void **)&M.item_aux, (void **)&M.span};
    for (void **a : arrs) {
        dfree(*a, st);
        *a = nullptr;
    }
    c->device_bytes -= M.hyb_bytes;
    M.hyb_bytes = 0;
    M.hyb = false;
    M.nitem = M.nitem_long = M.nlong = M.nslice = M.nspan = M.htotal = 0;
}

}  // namespace hoqri
