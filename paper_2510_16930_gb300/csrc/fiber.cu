// Fiber-factored pass: layout (built once per mode on the device), the
// cut-row fix-up and the launch.  The kernel and its algebra are in fiber.cuh.
#include <cub/cub.cuh>

#include <algorithm>
#include <vector>

#include "fiber.cuh"
#include "internal.cuh"

namespace hoqri {

// fiber3.cu / fiber4.cu: k_fib<2 or 3, PP, KL> and its shared memory per warp
// (4-byte words) with zs prefix floats per piece; false if there is no instance
bool fib_kernel3(int PP, int KL, int zs, const void **fn, int *warp_floats);
bool fib_kernel4(int PP, int KL, int zs, const void **fn, int *warp_floats);

__global__ void __launch_bounds__(256) k_fib_span(const int32_t *span, const float *ypart, int Pm, float *Y) {
    const int b = blockIdx.x;
    const int32_t j = span[3 * b], t0 = span[3 * b + 1], t1 = span[3 * b + 2];
    for (int e = threadIdx.x; e < Pm; e += blockDim.x) {
        double s = ypart[((size_t)t0 * 2 + 1) * Pm + e];
        for (int t = t0 + 1; t <= t1; ++t) s += ypart[((size_t)t * 2) * Pm + e];
        Y[(size_t)j * Pm + e] = (float)s;
    }
}

namespace {

constexpr int TPB = 256;

inline int grid_for(int64_t n, int cap) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + TPB - 1) / TPB, cap));
}

struct FTmp {
    cudaStream_t st;
    std::vector<void *> ptrs;
    explicit FTmp(cudaStream_t s) : st(s) {}
    ~FTmp() {
        for (void *p : ptrs) raw_free(p, st);
    }
    template <typename T>
    hoqri_status get(T **p, size_t count) {
        void *q = nullptr;
        cudaError_t e = raw_alloc(&q, std::max<size_t>(count, 1) * sizeof(T), st);
        if (e != cudaSuccess) {
            set_error(std::string("fiber layout allocation: ") + cudaGetErrorString(e));
            return HOQRI_ERR_OOM;
        }
        ptrs.push_back(q);
        *p = (T *)q;
        return HOQRI_OK;
    }
};

struct MaxI32 {
    __device__ __forceinline__ int32_t operator()(int32_t x, int32_t y) const { return x > y ? x : y; }
};

__global__ void k_fb_rowhead(const int64_t *row_ptr, int64_t R, int32_t *rowhead) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x)
        rowhead[row_ptr[r]] = 1;
}

// fs[z] = z where a fiber starts (a row starts, or a prefix index changes), else 0
__global__ void k_fb_fiber_start(const int32_t *pre0, const int32_t *pre1, const int32_t *rowhead, int64_t nnz,
                                 int32_t *fs) {
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < nnz; z += (int64_t)gridDim.x * blockDim.x) {
        bool h = z == 0 || rowhead[z] || pre0[z] != pre0[z - 1];
        if (pre1 && z > 0) h = h || pre1[z] != pre1[z - 1];
        fs[z] = h ? (int32_t)z : 0;
    }
}

// ph[z] = 1 where a piece starts: every FB_LP-th position of a fiber
__global__ void k_fb_piece_head(const int32_t *fstart, int64_t nnz, int32_t *ph) {
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < nnz; z += (int64_t)gridDim.x * blockDim.x)
        ph[z] = ((z - fstart[z]) % FB_LP) == 0;
}

__global__ void k_fb_fill(const int32_t *ph, const int32_t *pinc, const int32_t *rowinc, const int32_t *pre0,
                          const int32_t *pre1, int64_t nnz, int32_t *pst, int32_t *pa, int32_t *pb, int32_t *prow) {
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < nnz; z += (int64_t)gridDim.x * blockDim.x) {
        if (!ph[z]) continue;
        const int32_t p = pinc[z] - 1;
        pst[p] = (int32_t)z;
        pa[p] = pre0[z];
        if (pre1) pb[p] = pre1[z];
        prow[p] = rowinc[z] - 1;
    }
}

// length and first-piece-of-row flag of piece p, its cost for the ranges
__global__ void k_fb_finish(const int32_t *pst, const int32_t *prow, int64_t np, int64_t nnz, uint32_t *plenf,
                            int64_t *cost) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t len = (uint32_t)((p + 1 < np ? (int64_t)pst[p + 1] : nnz) - pst[p]);
        const bool head = p == 0 || prow[p] != prow[p - 1];
        plenf[p] = len | (head ? FB_HEAD : 0u);
        cost[p] = (int64_t)len + FB_PIECE_COST;
    }
}

// range t = [prange[t], prange[t+1]): first piece whose inclusive cost exceeds t*C/W
__global__ void k_fb_ranges(const int64_t *cum, int64_t np, int W, const int32_t *prow, const uint32_t *plenf,
                            int32_t *prange, int32_t *rrow0, int32_t *rhead) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > W) return;
    int64_t b;
    if (t == 0) b = 0;
    else if (t == W) b = np;
    else {
        const int64_t C = cum[np - 1];
        const int64_t target = C * (int64_t)t / W;  // C < 5 * 2^31, t <= W < 2^20: no overflow
        int64_t lo = 0, hi = np;  // first i with cum[i] > target
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cum[mid] > target) hi = mid;
            else lo = mid + 1;
        }
        b = lo;
    }
    prange[t] = (int32_t)b;
    if (t < W) {
        rrow0[t] = b < np ? prow[b] : 0;
        rhead[t] = b < np ? (int32_t)((plenf[b] & FB_HEAD) != 0) : 1;
    }
}

}  // namespace

bool fib_shape(const hoqri_ctx *c, int n, FibShapeSel *sel) {
    if (c->prec != HOQRI_FP32 || c->mix || (c->N != 3 && c->N != 4)) return false;
    int Ko[3], j = 0;
    for (int m = 0; m < c->N; ++m)
        if (m != n) Ko[j++] = c->K[m];
    for (int q = 0; q < j; ++q)
        if (Ko[q] < 4 || (Ko[q] & (Ko[q] - 1)) != 0) return false;
    FibShapeSel s;
    s.nm1 = c->N - 1;
    s.KL = Ko[s.nm1 - 1];
    s.KA = Ko[0];
    s.KB = s.nm1 == 3 ? Ko[1] : 1;
    s.PP = s.KA * s.KB;
    const int zs = s.nm1 == 2 ? s.PP : s.KA + s.KB;
    const bool ok = s.nm1 == 2 ? fib_kernel3(s.PP, s.KL, zs, &s.fn, &s.warp_floats)
                               : fib_kernel4(s.PP, s.KL, zs, &s.fn, &s.warp_floats);
    if (!ok) return false;
    if (sel) *sel = s;
    return true;
}

static size_t fib_smem(const FibShapeSel &s) { return (size_t)FB_WARPS * s.warp_floats * sizeof(float); }

void free_fiber(hoqri_ctx *c, int n) {
    ModeStore &M = c->ms[n];
    cudaStream_t st = c->stream;
    void **arrs[] = {(void **)&M.fb_pstart, (void **)&M.fb_plenf, (void **)&M.fb_pa, (void **)&M.fb_pb,
                     (void **)&M.fb_prange, (void **)&M.fb_rrow0, (void **)&M.fb_span};
    for (void **a : arrs) {
        dfree(*a, st);
        *a = nullptr;
    }
    c->device_bytes -= M.fb_bytes;
    M.fb_bytes = 0;
    M.fib = false;
    M.fb_np = M.fb_nspan = 0;
    M.fb_W = 0;
}

hoqri_status build_fiber(hoqri_ctx *c, int n) {
    ModeStore &M = c->ms[n];
    FibShapeSel s;
    if (!fib_shape(c, n, &s)) {
        set_error("fiber layout: unsupported shape");
        return HOQRI_ERR_UNSUPPORTED;
    }
    const int64_t b0 = c->device_bytes;
    cudaStream_t st = c->stream;
    const int64_t nnz = c->nnz;
    FTmp tmp(st);
    const int G = grid_for(nnz, c->num_sms * 8);
    const int32_t *pre0 = M.oidx[0];
    const int32_t *pre1 = s.nm1 == 3 ? M.oidx[1] : nullptr;
    const int nn = (int)nnz;
    int64_t np = 0;
    int32_t *ph = nullptr, *pinc = nullptr, *rowinc = nullptr;
    if (nnz > 0) {
        int32_t *rowhead, *fs, *fstart;
        HQ_TRY(tmp.get(&rowhead, nnz));
        HQ_TRY(tmp.get(&rowinc, nnz));
        HQ_TRY(tmp.get(&fs, nnz));
        HQ_TRY(tmp.get(&fstart, nnz));
        HQ_CUDA(cudaMemsetAsync(rowhead, 0, nnz * sizeof(int32_t), st));
        k_fb_rowhead<<<grid_for(M.R, c->num_sms * 8), TPB, 0, st>>>(M.row_ptr, M.R, rowhead);
        k_fb_fiber_start<<<G, TPB, 0, st>>>(pre0, pre1, rowhead, nnz, fs);
        size_t tb1 = 0, tb2 = 0;
        HQ_CUDA(cub::DeviceScan::InclusiveScan(nullptr, tb1, fs, fstart, MaxI32(), nn, st));
        HQ_CUDA(cub::DeviceScan::InclusiveSum(nullptr, tb2, rowhead, rowinc, nn, st));
        char *tscan;
        HQ_TRY(tmp.get(&tscan, std::max(tb1, tb2)));
        HQ_CUDA(cub::DeviceScan::InclusiveScan(tscan, tb1, fs, fstart, MaxI32(), nn, st));
        HQ_CUDA(cub::DeviceScan::InclusiveSum(tscan, tb2, rowhead, rowinc, nn, st));
        ph = fs;  // fs is no longer needed
        k_fb_piece_head<<<G, TPB, 0, st>>>(fstart, nnz, ph);
        pinc = fstart;  // nor is fstart once ph is formed
        HQ_CUDA(cub::DeviceScan::InclusiveSum(tscan, tb2, ph, pinc, nn, st));
        int32_t last = 0;
        HQ_CUDA(cudaMemcpyAsync(&last, pinc + nnz - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        HQ_CUDA(cudaStreamSynchronize(st));
        np = last;
    }
    M.fb_np = np;
    // piece arrays, in stream order
    HQ_TRY(dalloc(c, (void **)&M.fb_pstart, std::max<int64_t>(np, 1) * sizeof(int32_t)));
    HQ_TRY(dalloc(c, (void **)&M.fb_plenf, std::max<int64_t>(np, 1) * sizeof(uint32_t)));
    HQ_TRY(dalloc(c, (void **)&M.fb_pa, std::max<int64_t>(np, 1) * sizeof(int32_t)));
    if (s.nm1 == 3) HQ_TRY(dalloc(c, (void **)&M.fb_pb, std::max<int64_t>(np, 1) * sizeof(int32_t)));
    // ranges: as many warps as are resident at once, each with a cost of at least
    // 2 (FB_LP + FB_PIECE_COST), twice the largest piece cost, so every range
    // holds at least one piece
    int per_sm = 1;
    const size_t smem = fib_smem(s);
    HQ_CUDA(smem_limit(s.fn, smem));
    HQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, s.fn, FB_WARPS * 32, smem));
    per_sm = std::max(1, per_sm);
    int W = 0;
    std::vector<int32_t> prange, rrow0, rhead;
    if (np > 0) {
        int32_t *prow;
        int64_t *cost, *cum;
        HQ_TRY(tmp.get(&prow, np));
        HQ_TRY(tmp.get(&cost, np));
        HQ_TRY(tmp.get(&cum, np));
        k_fb_fill<<<G, TPB, 0, st>>>(ph, pinc, rowinc, pre0, pre1, nnz, M.fb_pstart, M.fb_pa,
                                     s.nm1 == 3 ? M.fb_pb : M.fb_pa, prow);
        const int Gp = grid_for(np, c->num_sms * 8);
        k_fb_finish<<<Gp, TPB, 0, st>>>(M.fb_pstart, prow, np, nnz, M.fb_plenf, cost);
        size_t tb = 0;
        HQ_CUDA(cub::DeviceScan::InclusiveSum(nullptr, tb, cost, cum, (int)np, st));
        char *t;
        HQ_TRY(tmp.get(&t, tb));
        HQ_CUDA(cub::DeviceScan::InclusiveSum(t, tb, cost, cum, (int)np, st));
        int64_t C = 0;
        HQ_CUDA(cudaMemcpyAsync(&C, cum + np - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        HQ_CUDA(cudaStreamSynchronize(st));
        const int64_t Wmax = (int64_t)c->num_sms * per_sm * FB_WARPS;
        W = (int)std::max<int64_t>(1, std::min<int64_t>(Wmax, C / (2 * (FB_LP + FB_PIECE_COST))));
        int32_t *dr, *d0, *dh;
        HQ_TRY(tmp.get(&dr, W + 1));
        HQ_TRY(tmp.get(&d0, W));
        HQ_TRY(tmp.get(&dh, W));
        k_fb_ranges<<<(W + 1 + TPB - 1) / TPB, TPB, 0, st>>>(cum, np, W, prow, M.fb_plenf, dr, d0, dh);
        prange.resize(W + 1);
        rrow0.resize(W);
        rhead.resize(W);
        HQ_CUDA(cudaMemcpyAsync(prange.data(), dr, (W + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        HQ_CUDA(cudaMemcpyAsync(rrow0.data(), d0, W * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        HQ_CUDA(cudaMemcpyAsync(rhead.data(), dh, W * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        HQ_CUDA(cudaStreamSynchronize(st));
        for (int q = 0; q < W; ++q)
            if (prange[q] >= prange[q + 1]) {
                set_error("fiber layout: empty work range (internal)");
                return HOQRI_ERR_CUDA;
            }
    }
    // rows cut by range boundaries: (row, first range, last range)
    std::vector<int32_t> span;
    for (int q = 1; q < W;) {
        if (rhead[q]) {
            ++q;
            continue;
        }
        const int32_t jr = rrow0[q];
        int t1 = q;
        while (t1 + 1 < W && !rhead[t1 + 1] && rrow0[t1 + 1] == jr) ++t1;
        span.push_back(jr);
        span.push_back(q - 1);
        span.push_back(t1);
        q = t1 + 1;
    }
    M.fb_W = W;
    M.fb_grid = (W + FB_WARPS - 1) / FB_WARPS;
    M.fb_smem = smem;
    M.fb_nspan = (int64_t)span.size() / 3;
    HQ_TRY(dalloc(c, (void **)&M.fb_prange, (W + 1) * sizeof(int32_t)));
    HQ_TRY(dalloc(c, (void **)&M.fb_rrow0, std::max(W, 1) * sizeof(int32_t)));
    HQ_TRY(dalloc(c, (void **)&M.fb_span, std::max<size_t>(span.size(), 1) * sizeof(int32_t)));
    if (W > 0) {
        HQ_CUDA(cudaMemcpyAsync(M.fb_prange, prange.data(), (W + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        HQ_CUDA(cudaMemcpyAsync(M.fb_rrow0, rrow0.data(), W * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    }
    if (!span.empty())
        HQ_CUDA(cudaMemcpyAsync(M.fb_span, span.data(), span.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    HQ_CUDA(cudaGetLastError());
    HQ_CUDA(cudaStreamSynchronize(st));
    M.fib = true;
    M.fb_sel = s;
    M.fb_bytes = c->device_bytes - b0;
    return HOQRI_OK;
}

int64_t fib_part_bytes(const hoqri_ctx *c, int n) {
    const ModeStore &M = c->ms[n];
    return (int64_t)std::max(M.fb_W, 1) * 2 * (c->P / c->K[n]) * (int64_t)sizeof(float);
}

hoqri_status fib_pass(hoqri_ctx *c, int n) {
    const ModeStore &M = c->ms[n];
    const FibShapeSel &s = M.fb_sel;
    const int Pm = (int)(c->P / c->K[n]);
    if (M.fb_W == 0) return HOQRI_OK;
    if (!c->fpart || fib_part_bytes(c, n) > c->fpart_bytes) {
        set_error("fiber pass: cut-row buffer too small (internal)");
        return HOQRI_ERR_CUDA;
    }
    FibArgs a{};
    a.lidx = M.oidx[s.nm1 - 1];
    a.vals = (const float *)M.vals;
    a.pstart = M.fb_pstart;
    a.plenf = M.fb_plenf;
    a.pa = M.fb_pa;
    a.pb = s.nm1 == 3 ? M.fb_pb : M.fb_pa;
    a.prange = M.fb_prange;
    a.rrow0 = M.fb_rrow0;
    const float *Uo[3] = {nullptr, nullptr, nullptr};
    int j = 0;
    for (int m = 0; m < c->N; ++m)
        if (m != n) Uo[j++] = (const float *)c->U[m];
    a.Ua = Uo[0];
    a.Ub = s.nm1 == 3 ? Uo[1] : nullptr;
    a.Ul = Uo[s.nm1 - 1];
    a.KA = s.KA;
    a.KB = s.KB;
    int lg = 0;
    while ((1 << lg) < s.KB) ++lg;
    a.lgKB = lg;
    a.W = M.fb_W;
    a.zs_floats = s.nm1 == 2 ? s.PP : s.KA + s.KB;
    a.warp_floats = s.warp_floats;
    a.np = M.fb_np;
    a.Y = c->Y;
    a.ypart = c->fpart;
    void *args[] = {&a};
    cudaEvent_t e0 = nullptr;
    HQ_TRY(prof_begin(c, 3, &e0));
    HQ_CUDA(cudaLaunchKernel(s.fn, dim3(M.fb_grid), dim3(FB_WARPS * 32), args, M.fb_smem, c->stream));
    c->nlaunch++;
    HQ_TRY(prof_end(c, 3, e0));
    if (M.fb_nspan > 0) {
        k_fib_span<<<(unsigned)M.fb_nspan, 256, 0, c->stream>>>(M.fb_span, c->fpart, Pm, c->Y);
        c->nlaunch++;
    }
    HQ_CUDA(cudaGetLastError());
    return HOQRI_OK;
}

}  // namespace hoqri
