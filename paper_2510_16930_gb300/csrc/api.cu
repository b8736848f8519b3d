// C ABI of libhoqri: context life cycle and the HOQRI driver (Alg. 2).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "hosvd.cuh"
#include "internal.cuh"

namespace hoqri {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

// Stream-ordered allocations (contexts on a created stream) come from one
// memory pool per device owned by the library, which keeps freed memory
// reserved (release threshold: unlimited), so creating and destroying contexts
// repeatedly does not map and unmap device memory each time (4.5 GB: 4 ms to
// allocate and 6 ms to free through a releasing pool, 0.1 ms each from a
// retaining one).  hoqri_trim_memory hands the reserved memory back.  A pool
// that no longer answers (the device was reset) is replaced.
namespace {
constexpr int POOL_MAX_DEVICES = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[POOL_MAX_DEVICES];

cudaError_t lib_pool(cudaMemPool_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= POOL_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    cuuint64_t thr = 0;
    if (g_pool[dev] && cudaMemPoolGetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &thr) != cudaSuccess) {
        cudaGetLastError();
        g_pool[dev] = nullptr;
    }
    if (!g_pool[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
        cuuint64_t keep = ~(cuuint64_t)0;
        if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}
}  // namespace

cudaError_t raw_alloc(void **p, size_t bytes, cudaStream_t st) {
    if (!st) return cudaMalloc(p, bytes);
    cudaMemPool_t pool = nullptr;
    const cudaError_t e = lib_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

void raw_free(void *p, cudaStream_t st) {
    if (!p) return;
    if (st) cudaFreeAsync(p, st);
    else cudaFree(p);
}

hoqri_status dalloc(hoqri_ctx *c, void **p, size_t bytes) {
    *p = nullptr;
    cudaError_t e = raw_alloc(p, std::max<size_t>(bytes, 16), c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error(std::string("device allocation of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
        return HOQRI_ERR_OOM;
    }
    c->device_bytes += (int64_t)std::max<size_t>(bytes, 16);
    return HOQRI_OK;
}

void dfree(void *p, cudaStream_t st) { raw_free(p, st); }

cudaError_t smem_limit_raw(const void *fn, size_t bytes) {
    // every caller sets the same value, the most the kernel may have, so
    // settings made on several threads at once cannot undercut each other
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    const size_t lim = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    if (bytes > lim) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
}

static bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static cudaMemcpyKind kind_to_device(const void *src) {
    return is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}

// copy `bytes` from a device buffer to a caller buffer (host or device)
static hoqri_status copy_out(hoqri_ctx *c, void *dst, const void *src_dev, size_t bytes) {
    const bool dev = is_device_ptr(dst);
    HQ_CUDA(cudaMemcpyAsync(dst, src_dev, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!dev) HQ_CUDA(cudaStreamSynchronize(c->stream));
    return HOQRI_OK;
}

static hoqri_status ensure_slots(hoqri_ctx *c, int64_t slots) {
    if (c->dnorm_slots >= slots) return HOQRI_OK;
    double *nd = nullptr;
    HQ_TRY(dalloc(c, (void **)&nd, slots * sizeof(double)));
    HQ_CUDA(cudaMemsetAsync(nd, 0, slots * sizeof(double), c->stream));
    if (c->dnorm) {
        HQ_CUDA(cudaMemcpyAsync(nd, c->dnorm, 2 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        HQ_CUDA(cudaStreamSynchronize(c->stream));
        dfree(c->dnorm, c->stream);
    }
    c->dnorm = nd;
    c->dnorm_slots = slots;
    if (c->sweep_exec) {  // the captured sweep writes into the old history array
        cudaGraphExecDestroy(c->sweep_exec);
        c->sweep_exec = nullptr;
    }
    return HOQRI_OK;
}

static void destroy_impl(hoqri_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaStream_t st = c->stream;
    if (c->sweep_exec) cudaGraphExecDestroy(c->sweep_exec);
    for (auto &r : c->ev_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (int n = 0; n < HOQRI_MAXN; ++n) {
        ModeStore &M = c->ms[n];
        for (int j = 0; j < HOQRI_MAXN - 1; ++j) dfree(M.oidx[j], st);
        dfree(M.vals, st);
        dfree(M.perm, st);
        dfree(M.row_id, st);
        dfree(M.row_ptr, st);
        dfree(M.chunk_start, st);
        dfree(M.chunk_row, st);
        dfree(M.big, st);
        for (int j = 0; j < HOQRI_MAXN - 1; ++j) dfree(M.hidx[j], st);
        dfree(M.hvals, st);
        dfree(M.lrp, st);
        dfree(M.lrow, st);
        dfree(M.sbase, st);
        dfree(M.srow, st);
        dfree(M.item_s, st);
        dfree(M.item_e, st);
        dfree(M.item_aux, st);
        dfree(M.span, st);
        dfree(M.fb_pstart, st);
        dfree(M.fb_plenf, st);
        dfree(M.fb_pa, st);
        dfree(M.fb_pb, st);
        dfree(M.fb_prange, st);
        dfree(M.fb_rrow0, st);
        dfree(M.fb_span, st);
        dfree(c->U[n], st);
        dfree(c->Upad[n], st);
    }
    dfree(c->gslot, st);
    dfree(c->gcount, st);
    dfree(c->G, st);
    dfree(c->A, st);
    dfree(c->dnorm, st);
    dfree(c->dflag, st);
    dfree(c->core_part, st);
    dfree(c->a_part, st);
    dfree(c->qr_part, st);
    dfree(c->qr_small, st);
    dfree(c->qr_work, st);
    dfree(c->gnorm_part, st);
    dfree(c->Y, st);
    dfree(c->ypart, st);
    dfree(c->fpart, st);
    dfree(c->usplit, st);
    dfree(c->claim, st);
    cudaGetLastError();
    delete c;
}

static double resid_of(double nx2, double ng2) {
    if (!(nx2 > 0)) return 0.0;
    double r2 = nx2 - ng2;
    return std::sqrt(r2 > 0 ? r2 : 0.0) / std::sqrt(nx2);
}

static hoqri_status ev_get(hoqri_ctx *c, cudaEvent_t *e) {
    if (!c->ev_pool.empty()) {
        *e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return HOQRI_OK;
    }
    HQ_CUDA(cudaEventCreate(e));
    return HOQRI_OK;
}

hoqri_status prof_begin(hoqri_ctx *c, int kind, cudaEvent_t *a) {
    (void)kind;
    *a = nullptr;
    if (!c->profiling) return HOQRI_OK;
    HQ_TRY(ev_get(c, a));
    HQ_CUDA(cudaEventRecord(*a, c->stream));
    return HOQRI_OK;
}

hoqri_status prof_end(hoqri_ctx *c, int kind, cudaEvent_t a) {
    if (!c->profiling || !a) return HOQRI_OK;
    cudaEvent_t b;
    HQ_TRY(ev_get(c, &b));
    HQ_CUDA(cudaEventRecord(b, c->stream));
    c->ev_recs.push_back({kind, a, b});
    return HOQRI_OK;
}

static hoqri_status prof_collect(hoqri_ctx *c) {
    if (c->ev_recs.empty()) return HOQRI_OK;
    HQ_CUDA(cudaStreamSynchronize(c->stream));
    for (auto &r : c->ev_recs) {
        float ms = 0.f;
        HQ_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        c->prof[2 * r.kind] += ms;
        c->prof[2 * r.kind + 1] += 1.0;
        c->ev_pool.push_back(r.a);
        c->ev_pool.push_back(r.b);
    }
    c->ev_recs.clear();
    return HOQRI_OK;
}

// after a stream synchronisation: did a bounded device wait run out?
static hoqri_status check_device_error(hoqri_ctx *c) {
    int32_t e = 0;
    HQ_CUDA(cudaMemcpy(&e, c->dflag + 2, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (e) {
        set_error("a bounded device wait ran out (staged copy never completed)");
        return HOQRI_ERR_TIMEOUT;
    }
    return HOQRI_OK;
}

static hoqri_status check_mode(hoqri_ctx *c, int32_t mode) {
    if (!c) {
        set_error("NULL context");
        return HOQRI_ERR_INVALID;
    }
    if (mode < 0 || mode >= c->N) {
        set_error("mode out of range");
        return HOQRI_ERR_INVALID;
    }
    return HOQRI_OK;
}

// G <- X x {U^T} with the current factors, computed from mode m's stream.  A
// mode on the two-pass kernels computes it from the context's core_mode
// instead: every mode's stream gives the same G (Alg. 3), and the row-grouped
// cost nnz P_{-m} + R_m P (Table 2) differs between modes (R_m P dominates for
// large cores and many short rows).
static hoqri_status refresh_core(hoqri_ctx *c, int m, double *slot) {
    if (!hyb_mode(c, m) && c->core_mode >= 0) m = c->core_mode;
    if (hyb_mode(c, m)) {
        cudaEvent_t e0 = nullptr;
        HQ_TRY(prof_begin(c, 0, &e0));
        HQ_TRY(hyb_pass(c, m));
        int nb = 0;
        HQ_TRY(hyb_core_partials(c, m, &nb));
        HQ_TRY(core_reduce(c, m, nb, c->G, slot));
        return prof_end(c, 0, e0);
    }
    return core_pass(c, m, c->G, slot);
}

// A <- TTMcTC(X, {U}, n) with the current core; in hybrid modes Y_(n) stays in
// c->Y for a following core_from_y.
static hoqri_status ttmctc_block(hoqri_ctx *c, int n, void *A, bool keep_y) {
    (void)keep_y;
    if (hyb_mode(c, n)) {
        cudaEvent_t e0 = nullptr;
        HQ_TRY(prof_begin(c, 1, &e0));
        HQ_TRY(hyb_pass(c, n));
        HQ_TRY(unfold_core(c, n, c->G, c->core_part));
        HQ_TRY(hyb_a_from_y(c, n, (const float *)c->core_part, (float *)A));
        return prof_end(c, 1, e0);
    }
    return ttmctc_pass(c, n, c->G, A);
}

// G <- U_n^T Y_(n) after the QR of mode n (Y_(n) from the preceding ttmctc_block).
static hoqri_status core_from_y(hoqri_ctx *c, int n, double *slot) {
    cudaEvent_t e0 = nullptr;
    HQ_TRY(prof_begin(c, 0, &e0));
    int nb = 0;
    HQ_TRY(hyb_core_partials(c, n, &nb));
    HQ_TRY(core_reduce(c, n, nb, c->G, slot));
    return prof_end(c, 0, e0);
}

}  // namespace hoqri

using namespace hoqri;

extern "C" {

void hoqri_default_options(hoqri_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->prec = HOQRI_FP32;
    opt->qr_kind = 0;
    opt->chunk_nnz = 0;
    opt->autotune = 0;
    opt->use_graphs = 1;
    opt->seed = 0;
    opt->tol = 0.0;
}

const char *hoqri_last_error(void) { return g_last_error.c_str(); }

hoqri_status hoqri_create(hoqri_ctx **out, int32_t N, const int64_t *dims, const int32_t *ranks, int64_t nnz,
                          const int32_t *const *idx, const void *vals, const hoqri_options *opt,
                          const void *const *U0, void *stream) {
    g_last_error.clear();
    if (!out) {
        set_error("hoqri_create: out is NULL");
        return HOQRI_ERR_INVALID;
    }
    *out = nullptr;
    if (N < 2 || N > HOQRI_MAXN || !dims || !ranks || nnz < 0 || (nnz > 0 && (!idx || !vals))) {
        set_error("hoqri_create: need 2 <= N <= 8, dims, ranks, nnz >= 0 and idx/vals when nnz > 0");
        return HOQRI_ERR_INVALID;
    }
    for (int n = 0; n < N; ++n) {
        if (dims[n] < 1 || dims[n] >= (int64_t)INT32_MAX || ranks[n] < 1) {
            set_error("hoqri_create: need 1 <= dims[n] < 2^31 and ranks[n] >= 1");
            return HOQRI_ERR_INVALID;
        }
        if (nnz > 0 && !idx[n]) {
            set_error("hoqri_create: idx[n] is NULL");
            return HOQRI_ERR_INVALID;
        }
    }
    for (int n = 0; n < N; ++n) {
        int64_t pm = 1;
        for (int m = 0; m < N; ++m)
            if (m != n) pm *= ranks[m];
        if (ranks[n] > HOQRI_MAXK) {
            set_error("hoqri_create: ranks above 64 are not supported");
            return HOQRI_ERR_UNSUPPORTED;
        }
        if ((int64_t)ranks[n] > dims[n] || (int64_t)ranks[n] > pm) {
            set_error("hoqri_create: K_n must not exceed I_n nor prod_{m != n} K_m");
            return HOQRI_ERR_RANK;
        }
    }
    {
        int64_t P = 1;
        for (int n = 0; n < N; ++n) P *= ranks[n];
        if (P > ((int64_t)1 << 26)) {
            set_error("hoqri_create: prod K_n above 2^26 core entries is not supported");
            return HOQRI_ERR_UNSUPPORTED;
        }
    }
    hoqri_options o;
    hoqri_default_options(&o);
    if (opt) o = *opt;
    if (o.prec != HOQRI_FP64 && o.prec != HOQRI_FP32 && o.prec != HOQRI_BF16X3) {
        set_error("hoqri_create: unknown precision");
        return HOQRI_ERR_INVALID;
    }
    hoqri_ctx *c = new (std::nothrow) hoqri_ctx();
    if (!c) {
        set_error("hoqri_create: host allocation failed");
        return HOQRI_ERR_OOM;
    }
    c->N = N;
    c->P = 1;
    for (int n = 0; n < N; ++n) {
        c->dims[n] = dims[n];
        c->K[n] = ranks[n];
        c->P *= ranks[n];
    }
    c->opt = o;
    // HOQRI_BF16X3 stores and computes like HOQRI_FP32 except the Kronecker
    // contraction of long rows, which runs on the tensor cores in split BF16
    c->prec = o.prec == HOQRI_BF16X3 ? HOQRI_FP32 : o.prec;
    c->mix = o.prec == HOQRI_BF16X3;
    c->rsize = (o.prec == HOQRI_FP64) ? sizeof(double) : sizeof(float);
    c->stream = (cudaStream_t)stream;
    auto fail = [&](hoqri_status s) {
        std::string msg = g_last_error;
        destroy_impl(c);
        g_last_error = msg;
        return s;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        set_error("hoqri_create: no CUDA device");
        return fail(HOQRI_ERR_CUDA);
    }
    hoqri_status s;
    if ((s = ensure_slots(c, 64)) != HOQRI_OK) return fail(s);
    if ((s = dalloc(c, (void **)&c->dflag, 4 * sizeof(int32_t))) != HOQRI_OK) return fail(s);
    if (cudaMemsetAsync(c->dflag, 0, 4 * sizeof(int32_t), c->stream) != cudaSuccess) return fail(HOQRI_ERR_CUDA);

    // inputs on the device (temporaries released after set-up)
    std::vector<void *> tmp;
    auto free_tmp = [&]() {
        for (void *p : tmp) raw_free(p, c->stream);
        tmp.clear();
    };
    const int32_t *idx_dev[HOQRI_MAXN] = {};
    const void *vals_dev = vals;
    for (int n = 0; n < N && nnz > 0; ++n) {
        if (is_device_ptr(idx[n])) {
            idx_dev[n] = idx[n];
        } else {
            void *p = nullptr;
            if (raw_alloc(&p, nnz * sizeof(int32_t), c->stream) != cudaSuccess) {
                cudaGetLastError();
                free_tmp();
                set_error("hoqri_create: device allocation for the indices failed");
                return fail(HOQRI_ERR_OOM);
            }
            tmp.push_back(p);
            if (cudaMemcpyAsync(p, idx[n], nnz * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
                free_tmp();
                set_error("hoqri_create: copy of the indices failed");
                return fail(HOQRI_ERR_CUDA);
            }
            idx_dev[n] = (const int32_t *)p;
        }
    }
    if (nnz > 0 && !is_device_ptr(vals)) {
        void *p = nullptr;
        if (raw_alloc(&p, nnz * c->rsize, c->stream) != cudaSuccess) {
            cudaGetLastError();
            free_tmp();
            set_error("hoqri_create: device allocation for the values failed");
            return fail(HOQRI_ERR_OOM);
        }
        tmp.push_back(p);
        if (cudaMemcpyAsync(p, vals, nnz * c->rsize, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
            free_tmp();
            set_error("hoqri_create: copy of the values failed");
            return fail(HOQRI_ERR_CUDA);
        }
        vals_dev = p;
    }
    s = build_storage(c, idx_dev, vals_dev, nnz);
    cudaStreamSynchronize(c->stream);
    free_tmp();
    if (s != HOQRI_OK) return fail(s);

    int64_t maxIK = 0;
    for (int n = 0; n < N; ++n) {
        if ((s = dalloc(c, &c->U[n], c->dims[n] * c->K[n] * c->rsize)) != HOQRI_OK) return fail(s);
        maxIK = std::max<int64_t>(maxIK, c->dims[n] * c->K[n]);
    }
    if ((s = dalloc(c, &c->G, c->P * c->rsize)) != HOQRI_OK) return fail(s);
    if ((s = dalloc(c, &c->A, maxIK * c->rsize)) != HOQRI_OK) return fail(s);
    if ((s = qr_init(c)) != HOQRI_OK) return fail(s);
    if (c->opt.tile_rows > 0 || c->opt.tile_cols > 0) {
        const int tl = c->opt.tile_rows, tv = c->opt.tile_cols;
        if ((tl != 4 && tl != 8) || (tv != 4 && tv != 8)) {
            set_error("hoqri_create: tile_rows and tile_cols must be 4 or 8 (or both 0)");
            return fail(HOQRI_ERR_INVALID);
        }
        for (int n = 0; n < N; ++n) {
            c->ms[n].tune_TL = tl;
            c->ms[n].tune_TV = tv;
        }
    }
    if ((s = passes_init(c)) != HOQRI_OK) return fail(s);
    {
        // the two-pass core is computed from the mode of least nnz P_{-m} + R_m P
        double best = 0.0;
        for (int m = 0; m < N; ++m) {
            if (hyb_mode(c, m)) continue;
            const double cost = (double)c->nnz * (double)(c->P / c->K[m]) + (double)c->ms[m].R * (double)c->P;
            if (c->core_mode < 0 || cost < best) {
                best = cost;
                c->core_mode = m;
            }
        }
    }
    if (U0) {
        for (int n = 0; n < N; ++n) {
            if (!U0[n]) {
                set_error("hoqri_create: U0[n] is NULL");
                return fail(HOQRI_ERR_INVALID);
            }
            if (cudaMemcpyAsync(c->U[n], U0[n], c->dims[n] * c->K[n] * c->rsize, kind_to_device(U0[n]), c->stream) !=
                cudaSuccess) {
                set_error("hoqri_create: copy of U0 failed");
                return fail(HOQRI_ERR_CUDA);
            }
        }
    } else {
        if ((s = init_factors_seeded(c)) != HOQRI_OK) return fail(s);
    }
    if (c->opt.autotune && (s = autotune_hybrid(c)) != HOQRI_OK) return fail(s);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        set_error("hoqri_create: CUDA error during set-up");
        return fail(HOQRI_ERR_CUDA);
    }
    *out = c;
    return HOQRI_OK;
}

void hoqri_destroy(hoqri_ctx *ctx) { destroy_impl(ctx); }

hoqri_status hoqri_core(hoqri_ctx *c, void *G_out) {
    g_last_error.clear();
    HQ_TRY(check_mode(c, 0));
    if (!G_out) {
        set_error("hoqri_core: G_out is NULL");
        return HOQRI_ERR_INVALID;
    }
    HQ_TRY(refresh_core(c, 0, nullptr));
    return copy_out(c, G_out, c->G, c->P * c->rsize);
}

hoqri_status hoqri_ttmctc(hoqri_ctx *c, int32_t mode, void *A_out) {
    g_last_error.clear();
    HQ_TRY(check_mode(c, mode));
    if (!A_out) {
        set_error("hoqri_ttmctc: A_out is NULL");
        return HOQRI_ERR_INVALID;
    }
    HQ_TRY(refresh_core(c, mode, nullptr));
    HQ_TRY(ttmctc_block(c, mode, c->A, false));
    return copy_out(c, A_out, c->A, c->dims[mode] * c->K[mode] * c->rsize);
}

hoqri_status hoqri_orthonormalize(hoqri_ctx *c, int32_t mode, const void *A_in, void *U_out) {
    g_last_error.clear();
    HQ_TRY(check_mode(c, mode));
    if (!A_in || !U_out) {
        set_error("hoqri_orthonormalize: NULL buffer");
        return HOQRI_ERR_INVALID;
    }
    const size_t bytes = c->dims[mode] * c->K[mode] * c->rsize;
    HQ_CUDA(cudaMemcpyAsync(c->A, A_in, bytes, kind_to_device(A_in), c->stream));
    if (is_device_ptr(U_out)) {
        HQ_TRY(orthonormalize(c, mode, c->A, U_out));
    } else {
        void *tmp = nullptr;
        HQ_TRY(dalloc(c, &tmp, bytes));
        hoqri_status s = orthonormalize(c, mode, c->A, tmp);
        if (s == HOQRI_OK) s = copy_out(c, U_out, tmp, bytes);
        cudaStreamSynchronize(c->stream);
        dfree(tmp, c->stream);
        c->device_bytes -= (int64_t)std::max<size_t>(bytes, 16);
        if (s != HOQRI_OK) return s;
    }
    if (c->opt.qr_kind == 2) {
        int32_t f[2];
        HQ_CUDA(cudaMemcpyAsync(f, c->dflag, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        HQ_CUDA(cudaStreamSynchronize(c->stream));
        if (f[0] != 0) {
            set_error("hoqri_orthonormalize: Cholesky breakdown");
            return HOQRI_ERR_QR_BREAKDOWN;
        }
    }
    return HOQRI_OK;
}

hoqri_status hoqri_orthonormalize_noalloc(int32_t prec, int64_t I, int32_t K, const void *A_in, void *U_out,
                                          void *stream) {
    g_last_error.clear();
    if (prec != HOQRI_FP64 && prec != HOQRI_FP32) {
        set_error("hoqri_orthonormalize_noalloc: prec must be HOQRI_FP64 or HOQRI_FP32");
        return HOQRI_ERR_INVALID;
    }
    if (K < 1 || K > HOQRI_NOALLOC_MAXK) {
        set_error("hoqri_orthonormalize_noalloc: K = " + std::to_string(K) + " outside 1.." +
                  std::to_string(HOQRI_NOALLOC_MAXK) + " (the static scratch holds at most " +
                  std::to_string(HOQRI_NOALLOC_MAXK) + " columns)");
        return HOQRI_ERR_INVALID;
    }
    if (I < K) {
        set_error("hoqri_orthonormalize_noalloc: I = " + std::to_string(I) + " < K = " + std::to_string(K));
        return HOQRI_ERR_INVALID;
    }
    if (!is_device_ptr(A_in) || !is_device_ptr(U_out)) {
        set_error("hoqri_orthonormalize_noalloc: A_in and U_out must be device buffers");
        return HOQRI_ERR_INVALID;
    }
    const uintptr_t bytes = (uintptr_t)I * (uintptr_t)K * (prec == HOQRI_FP64 ? 8u : 4u);
    const uintptr_t a = reinterpret_cast<uintptr_t>(A_in), u = reinterpret_cast<uintptr_t>(U_out);
    if (a != u && a < u + bytes && u < a + bytes) {
        set_error("hoqri_orthonormalize_noalloc: U_out overlaps A_in without being equal to it");
        return HOQRI_ERR_INVALID;
    }
    return orthonormalize_noalloc(prec, I, K, A_in, U_out, static_cast<cudaStream_t>(stream));
}

namespace hoqri {

// One sweep of Alg. 2 (every block update once); slots[n] receives ||G||^2
// after the update of block n.
static hoqri_status sweep(hoqri_ctx *c, double *slots) {
    for (int n = 0; n < c->N; ++n) {
        const bool one = hyb_mode(c, n);
        HQ_TRY(ttmctc_block(c, n, c->A, one));
        HQ_TRY(orthonormalize(c, n, c->A, c->U[n]));
        if (one) HQ_TRY(core_from_y(c, n, slots + n));
        else HQ_TRY(refresh_core(c, (n + 1) % c->N, slots + n));
    }
    return HOQRI_OK;
}

// appends the N norms of the replayed sweep to the history: sweep t = *count
__global__ void k_hist_push(const double *slots, int N, double *hist, int32_t *count) {
    const int t = *count;
    for (int n = 0; n < N; ++n) hist[(int64_t)t * N + n] = slots[n];
    *count = t + 1;
}

// Captures one sweep (plus the history append) into a CUDA graph; on any
// capture failure the context falls back to plain launches.
static hoqri_status capture_sweep(hoqri_ctx *c) {
    if (!c->gslot) HQ_TRY(dalloc(c, (void **)&c->gslot, c->N * sizeof(double)));
    if (!c->gcount) HQ_TRY(dalloc(c, (void **)&c->gcount, sizeof(int32_t)));
    const int64_t l0 = c->nlaunch;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        c->sweep_graph_off = true;
        return HOQRI_OK;
    }
    hoqri_status s = sweep(c, c->gslot);
    if (s == HOQRI_OK) {
        k_hist_push<<<1, 1, 0, c->stream>>>(c->gslot, c->N, c->dnorm + 3, c->gcount);
        c->nlaunch++;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (s != HOQRI_OK || e != cudaSuccess || !g) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        c->nlaunch = l0;
        c->sweep_graph_off = true;
        g_last_error.clear();
        return HOQRI_OK;
    }
    const cudaError_t ei = cudaGraphInstantiate(&c->sweep_exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        c->sweep_exec = nullptr;
        c->sweep_graph_off = true;
    }
    c->sweep_launches = c->nlaunch - l0;
    c->nlaunch = l0;
    return HOQRI_OK;
}

}  // namespace hoqri

namespace hoqri {

// Up to `iters` sweeps of Alg. 2; with tol > 0 the sweeps stop after the first
// one whose residual differs from the previous residual by less than tol (the
// stopping rule of Sec. 6.1; the residual before the first sweep is that of
// the initial core), which costs one device-to-host read per sweep.
// *done receives the number of sweeps run.
static hoqri_status run_sweeps(hoqri_ctx *c, int32_t iters, double tol, double *resid_hist, int32_t *done,
                               const char *who) {
    const int N = c->N;
    HQ_TRY(ensure_slots(c, 2 + (int64_t)iters * N + 1));
    int32_t before = 0;
    if (c->opt.qr_kind == 2) {
        HQ_CUDA(cudaMemcpyAsync(&before, c->dflag + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        HQ_CUDA(cudaStreamSynchronize(c->stream));
    }
    // slot 2 + k holds ||G||^2 after k block updates (k = 0: the initial core)
    HQ_TRY(refresh_core(c, 0, c->dnorm + 2));
    double h0[3] = {0, 0, 0};
    if (tol > 0.0) {
        HQ_CUDA(cudaMemcpyAsync(h0, c->dnorm, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        HQ_CUDA(cudaStreamSynchronize(c->stream));
    }
    double r_prev = resid_of(h0[0], h0[2]);
    // sweeps replay one captured CUDA graph, unless tracing is on (its events
    // are recorded per call on the host side) or capture is unavailable
    const bool graphs = c->opt.use_graphs && !c->profiling && iters > 0 && !c->sweep_graph_off;
    if (graphs && !c->sweep_exec) HQ_TRY(capture_sweep(c));
    const bool replay = graphs && c->sweep_exec;
    if (replay) HQ_CUDA(cudaMemsetAsync(c->gcount, 0, sizeof(int32_t), c->stream));
    int32_t ran = 0;
    for (int t = 0; t < iters; ++t) {
        if (replay) {
            HQ_CUDA(cudaGraphLaunch(c->sweep_exec, c->stream));
            c->nlaunch += c->sweep_launches;
        } else {
            HQ_TRY(sweep(c, c->dnorm + 2 + (int64_t)t * N + 1));
        }
        ++ran;
        if (tol > 0.0) {
            double g2 = 0.0;
            HQ_CUDA(cudaMemcpyAsync(&g2, c->dnorm + 2 + (size_t)(t + 1) * N, sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream));
            HQ_CUDA(cudaStreamSynchronize(c->stream));
            HQ_TRY(check_device_error(c));
            const double r = resid_of(h0[0], g2);
            if (std::fabs(r - r_prev) < tol) break;
            r_prev = r;
        }
    }
    if (done) *done = ran;
    if (resid_hist || c->opt.qr_kind == 2) {
        std::vector<double> h(2 + (size_t)ran * N + 1);
        HQ_CUDA(cudaMemcpyAsync(h.data(), c->dnorm, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        int32_t after = 0;
        HQ_CUDA(cudaMemcpyAsync(&after, c->dflag + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        HQ_CUDA(cudaStreamSynchronize(c->stream));
        HQ_TRY(check_device_error(c));
        if (resid_hist)
            for (int t = 0; t < ran; ++t) resid_hist[t] = resid_of(h[0], h[2 + (size_t)(t + 1) * N]);
        if (c->opt.qr_kind == 2 && after != before) {
            set_error(std::string(who) + ": Cholesky breakdown in a QR step");
            return HOQRI_ERR_QR_BREAKDOWN;
        }
    }
    HQ_CUDA(cudaGetLastError());
    return HOQRI_OK;
}

}  // namespace hoqri

hoqri_status hoqri_iterate(hoqri_ctx *c, int32_t iters, double *resid_hist) {
    g_last_error.clear();
    HQ_TRY(check_mode(c, 0));
    if (iters < 0) {
        set_error("hoqri_iterate: iters < 0");
        return HOQRI_ERR_INVALID;
    }
    return run_sweeps(c, iters, 0.0, resid_hist, nullptr, "hoqri_iterate");
}

hoqri_status hoqri_run(hoqri_ctx *c, int32_t max_iters, double *resid_hist, int32_t *iters_done) {
    g_last_error.clear();
    HQ_TRY(check_mode(c, 0));
    if (max_iters < 0 || !(c->opt.tol >= 0.0)) {
        set_error("hoqri_run: max_iters < 0 or tol < 0");
        return HOQRI_ERR_INVALID;
    }
    return run_sweeps(c, max_iters, c->opt.tol, resid_hist, iters_done, "hoqri_run");
}

hoqri_status hoqri_init_hosvd(hoqri_ctx *c, int32_t power_iters) {
    g_last_error.clear();
    HQ_TRY(check_mode(c, 0));
    if (power_iters < 1) {
        set_error("hoqri_init_hosvd: power_iters < 1");
        return HOQRI_ERR_INVALID;
    }
    HQ_TRY(init_hosvd(c, power_iters));
    return check_device_error(c);
}

hoqri_status hoqri_grad_norm2(hoqri_ctx *c, double *out) {
    g_last_error.clear();
    HQ_TRY(check_mode(c, 0));
    if (!out) {
        set_error("hoqri_grad_norm2: out is NULL");
        return HOQRI_ERR_INVALID;
    }
    double *slots = nullptr;
    HQ_TRY(dalloc(c, (void **)&slots, c->N * sizeof(double)));
    hoqri_status s = HOQRI_OK;
    for (int n = 0; n < c->N && s == HOQRI_OK; ++n) {
        // A_n and G at the current factors (Alg. 3: the core first), then the
        // mode's term of Eq. grad2
        s = refresh_core(c, n, nullptr);
        if (s == HOQRI_OK) s = ttmctc_block(c, n, c->A, false);
        if (s == HOQRI_OK) s = grad_term(c, n, c->A, slots + n);
    }
    std::vector<double> h(c->N, 0.0);
    if (s == HOQRI_OK) {
        if (cudaMemcpyAsync(h.data(), slots, c->N * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            set_error(std::string("hoqri_grad_norm2: ") + cudaGetErrorString(cudaGetLastError()));
            s = HOQRI_ERR_CUDA;
        }
    }
    cudaStreamSynchronize(c->stream);
    dfree(slots, c->stream);
    c->device_bytes -= (int64_t)std::max<size_t>(c->N * sizeof(double), 16);
    if (s != HOQRI_OK) return s;
    HQ_TRY(check_device_error(c));
    double g = 0.0;
    for (int n = 0; n < c->N; ++n) g += 4.0 * h[n];
    *out = g;
    return HOQRI_OK;
}

hoqri_status hoqri_get_factor(hoqri_ctx *c, int32_t mode, void *U_out) {
    g_last_error.clear();
    HQ_TRY(check_mode(c, mode));
    if (!U_out) {
        set_error("hoqri_get_factor: U_out is NULL");
        return HOQRI_ERR_INVALID;
    }
    return copy_out(c, U_out, c->U[mode], c->dims[mode] * c->K[mode] * c->rsize);
}

hoqri_status hoqri_set_factor(hoqri_ctx *c, int32_t mode, const void *U_in) {
    g_last_error.clear();
    HQ_TRY(check_mode(c, mode));
    if (!U_in) {
        set_error("hoqri_set_factor: U_in is NULL");
        return HOQRI_ERR_INVALID;
    }
    HQ_CUDA(cudaMemcpyAsync(c->U[mode], U_in, c->dims[mode] * c->K[mode] * c->rsize, kind_to_device(U_in), c->stream));
    if (!is_device_ptr(U_in)) HQ_CUDA(cudaStreamSynchronize(c->stream));
    return HOQRI_OK;
}

hoqri_status hoqri_fit(hoqri_ctx *c, double *resid, double *normX2, double *normG2) {
    g_last_error.clear();
    HQ_TRY(check_mode(c, 0));
    double h[2];
    HQ_CUDA(cudaMemcpyAsync(h, c->dnorm, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    HQ_CUDA(cudaStreamSynchronize(c->stream));
    if (resid) *resid = resid_of(h[0], h[1]);
    if (normX2) *normX2 = h[0];
    if (normG2) *normG2 = h[1];
    return HOQRI_OK;
}

hoqri_status hoqri_info(hoqri_ctx *c, int64_t *nnz, int64_t *rows, int64_t *device_bytes) {
    g_last_error.clear();
    HQ_TRY(check_mode(c, 0));
    if (nnz) *nnz = c->nnz;
    if (rows)
        for (int n = 0; n < c->N; ++n) rows[n] = c->ms[n].R;
    if (device_bytes) *device_bytes = c->device_bytes;
    return HOQRI_OK;
}

hoqri_status hoqri_layout(hoqri_ctx *c, int32_t mode, int64_t *out4) {
    g_last_error.clear();
    HQ_TRY(check_mode(c, mode));
    if (!out4) return HOQRI_OK;
    const ModeStore &M = c->ms[mode];
    FastTile p;
    if (!M.hyb || !hyb_mode(c, mode) || !hyb_tile(c, mode, &p)) {
        for (int q = 0; q < 4; ++q) out4[q] = -1;
        return HOQRI_OK;
    }
    out4[0] = M.tune_Lshort;
    out4[1] = M.tune_T;
    out4[2] = p.TL;
    out4[3] = p.TV;
    return HOQRI_OK;
}

hoqri_status hoqri_profile_enable(hoqri_ctx *c, int32_t enable) {
    g_last_error.clear();
    HQ_TRY(check_mode(c, 0));
    HQ_TRY(prof_collect(c));
    if (enable)
        for (double &v : c->prof) v = 0.0;
    c->profiling = enable != 0;
    return HOQRI_OK;
}

hoqri_status hoqri_profile_read(hoqri_ctx *c, double *out, int64_t *kernel_launches) {
    g_last_error.clear();
    HQ_TRY(check_mode(c, 0));
    HQ_TRY(prof_collect(c));
    if (out)
        for (int i = 0; i < 8; ++i) out[i] = c->prof[i];
    if (kernel_launches) *kernel_launches = c->nlaunch;
    return HOQRI_OK;
}

hoqri_status hoqri_trim_memory(void) {
    g_last_error.clear();
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (cudaMemPool_t &pool : g_pool) {
        if (!pool) continue;
        if (cudaMemPoolTrimTo(pool, 0) != cudaSuccess) {
            cudaGetLastError();
            pool = nullptr;  // the device was reset: its pool is gone
        }
    }
    return HOQRI_OK;
}

hoqri_status hoqri_synchronize(hoqri_ctx *c) {
    g_last_error.clear();
    HQ_TRY(check_mode(c, 0));
    HQ_CUDA(cudaStreamSynchronize(c->stream));
    HQ_CUDA(cudaGetLastError());
    return check_device_error(c);
}

}  // extern "C"
