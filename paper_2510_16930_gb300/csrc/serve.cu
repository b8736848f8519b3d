// Serving: many HOQRI decompositions (differing order, nnz and ranks) resident
// on one GPU at once, admitted by device memory (continuous batching).
//
// A request is queued at submit.  hoqri_server_step admits queued requests in
// arrival order while both the device-memory budget and the slot limit allow
// it, and polls the running ones.  An admitted request gets its own CUDA
// stream and context (sorted COO, factors and core resident on the device);
// all its sweeps (Alg. 2) are queued at once, each replaying the context's
// captured sweep graph, and an event marks the end.  Requests on different
// streams overlap on the device; a finished request keeps its results until
// hoqri_server_take copies them out and frees its memory, so a request that
// arrives while others run is admitted as soon as memory and a slot free up.
// Every request's arithmetic is that of a lone context, in the same order, so
// its results do not depend on the mix it ran in.  The set-up of an admitted
// request (sorting, layouts, graph capture: host work between short device
// steps) runs on a worker thread, so several requests are set up at once
// while the scheduler keeps polling.
#include <algorithm>
#include <chrono>
#include <future>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "internal.cuh"

namespace hoqri {

namespace {

double now_s() {
    using clk = std::chrono::steady_clock;
    static const clk::time_point t0 = clk::now();
    return std::chrono::duration<double>(clk::now() - t0).count();
}

struct Req {
    int64_t id = 0;
    int32_t N = 0;
    int64_t dims[HOQRI_MAXN] = {};
    int32_t ranks[HOQRI_MAXN] = {};
    int64_t nnz = 0;
    const int32_t *idx[HOQRI_MAXN] = {};
    const void *vals = nullptr;
    int32_t iters = 0;
    hoqri_options opt{};
    int32_t state = HOQRI_REQ_QUEUED;
    hoqri_status status = HOQRI_OK;
    std::string error;
    int64_t est_bytes = 0, bytes = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    hoqri_ctx *ctx = nullptr;
    std::future<hoqri_status> setup;  // admission in progress on a worker thread
    bool admitting = false;
};

}  // namespace

// Device bytes a context will hold for this problem (its persistent buffers;
// set-up temporaries of the same order are released before it returns).
int64_t estimate_ctx_bytes(int32_t N, const int64_t *dims, const int32_t *ranks, int64_t nnz, int32_t prec) {
    const int64_t rs = prec == HOQRI_FP64 ? 8 : 4;
    int64_t P = 1, maxIK = 0, sumIK = 0, maxR = 0;
    for (int n = 0; n < N; ++n) {
        P *= ranks[n];
        maxIK = std::max<int64_t>(maxIK, dims[n] * ranks[n]);
        sumIK += dims[n] * ranks[n];
        maxR = std::max<int64_t>(maxR, std::min<int64_t>(dims[n], nnz));
    }
    int64_t maxPm = 0;
    for (int n = 0; n < N; ++n) maxPm = std::max<int64_t>(maxPm, P / ranks[n]);
    // per mode: sorted indices, values, permutation and row descriptors, and the
    // hybrid copy of the stream; then factors, core, TTMcTC output, Y, QR work
    const int64_t per_mode = nnz * ((int64_t)(N - 1) * 4 + rs + 8) + nnz * ((int64_t)(N - 1) * 4 + rs) +
                             std::min<int64_t>(nnz, maxR) * 16;
    int64_t b = N * per_mode + sumIK * rs + 4 * P * rs + maxIK * rs + maxR * maxPm * 4 + 2 * maxIK * 8;
    b += (int64_t)64 << 20;  // partial sums, descriptors and slack
    return b;
}

}  // namespace hoqri

using namespace hoqri;

struct hoqri_server {
    int64_t budget = 0;
    int32_t max_active = 0;
    int64_t next_id = 1;
    int64_t in_use = 0;  // device bytes held by admitted requests
    std::deque<int64_t> queue;
    std::map<int64_t, std::unique_ptr<Req>> reqs;
    int32_t active = 0;
};

namespace {

thread_local std::string g_srv_err;

hoqri_status srv_fail(hoqri_status s, const std::string &m) {
    g_srv_err = m;
    set_error(m);
    return s;
}

void release(hoqri_server *s, Req *r) {
    if (r->admitting) {  // a set-up still in flight: let it finish first
        r->setup.wait();
        r->admitting = false;
        s->in_use -= r->est_bytes;
        s->in_use += r->bytes;
    }
    if (r->ctx) {
        hoqri_destroy(r->ctx);
        r->ctx = nullptr;
    }
    if (r->done) cudaEventDestroy(r->done);
    if (r->stream) cudaStreamDestroy(r->stream);
    r->done = nullptr;
    r->stream = nullptr;
    if (r->bytes > 0) s->in_use -= r->bytes;
    r->bytes = 0;
}

// admission work (runs on a worker thread): stream, context (stream-ordered
// allocations), all sweeps queued, end event recorded.  Touches only r.
hoqri_status admit_work(Req *r) {
    if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        r->error = "server: stream or event creation failed";
        return HOQRI_ERR_CUDA;
    }
    const void *idx_ptrs[HOQRI_MAXN];
    for (int n = 0; n < r->N; ++n) idx_ptrs[n] = r->idx[n];
    hoqri_status st = hoqri_create(&r->ctx, r->N, r->dims, r->ranks, r->nnz,
                                   reinterpret_cast<const int32_t *const *>(idx_ptrs), r->vals, &r->opt, nullptr,
                                   r->stream);
    if (st == HOQRI_OK) {
        int64_t nz = 0, db = 0;
        hoqri_info(r->ctx, &nz, nullptr, &db);
        r->bytes = db;
        st = hoqri_iterate(r->ctx, r->iters, nullptr);
    }
    if (st == HOQRI_OK && cudaEventRecord(r->done, r->stream) != cudaSuccess) {
        cudaGetLastError();
        set_error("server: event record failed");
        st = HOQRI_ERR_CUDA;
    }
    if (st != HOQRI_OK) r->error = hoqri_last_error();
    return st;
}

// a finished admission: RUNNING, or FAILED with its memory released
void admit_done(hoqri_server *s, Req *r) {
    const hoqri_status st = r->setup.get();
    r->admitting = false;
    r->t_admit = now_s();
    s->in_use -= r->est_bytes;  // the estimate charged at dispatch ...
    if (st != HOQRI_OK) {
        r->status = st;
        r->state = HOQRI_REQ_FAILED;
        r->t_done = r->t_admit;
        r->bytes = 0;
        release(s, r);
        --s->active;
        return;
    }
    s->in_use += r->bytes;  // ... is replaced by the context's actual bytes
    r->state = HOQRI_REQ_RUNNING;
}

}  // namespace

extern "C" {

hoqri_status hoqri_server_create(hoqri_server **out, int64_t budget_bytes, int32_t max_active) {
    g_srv_err.clear();
    if (!out || budget_bytes <= 0 || max_active <= 0)
        return srv_fail(HOQRI_ERR_INVALID, "hoqri_server_create: need out, budget_bytes > 0, max_active > 0");
    *out = nullptr;
    hoqri_server *s = new (std::nothrow) hoqri_server();
    if (!s) return srv_fail(HOQRI_ERR_OOM, "hoqri_server_create: host allocation failed");
    s->budget = budget_bytes;
    s->max_active = max_active;
    *out = s;
    return HOQRI_OK;
}

hoqri_status hoqri_server_submit(hoqri_server *s, const hoqri_request *q, int64_t *id) {
    if (!s || !q || !id) return srv_fail(HOQRI_ERR_INVALID, "hoqri_server_submit: NULL argument");
    if (q->N < 2 || q->N > HOQRI_MAXN || !q->dims || !q->ranks || q->iters < 0 || q->nnz < 0 ||
        (q->nnz > 0 && (!q->idx || !q->vals)))
        return srv_fail(HOQRI_ERR_INVALID, "hoqri_server_submit: bad request shape");
    auto r = std::make_unique<Req>();
    r->id = s->next_id++;
    r->N = q->N;
    for (int n = 0; n < q->N; ++n) {
        r->dims[n] = q->dims[n];
        r->ranks[n] = q->ranks[n];
        r->idx[n] = q->nnz > 0 ? q->idx[n] : nullptr;
    }
    r->nnz = q->nnz;
    r->vals = q->vals;
    r->iters = q->iters;
    hoqri_default_options(&r->opt);
    r->opt.prec = q->prec;
    r->opt.seed = q->seed;
    r->est_bytes = estimate_ctx_bytes(q->N, q->dims, q->ranks, q->nnz, q->prec);
    if (r->est_bytes > s->budget)
        return srv_fail(HOQRI_ERR_OOM, "hoqri_server_submit: request needs about " + std::to_string(r->est_bytes) +
                                           " device bytes, more than the whole budget");
    r->t_submit = now_s();
    *id = r->id;
    s->queue.push_back(r->id);
    s->reqs[r->id] = std::move(r);
    return HOQRI_OK;
}

hoqri_status hoqri_server_step(hoqri_server *s, int32_t *n_running, int32_t *n_queued) {
    if (!s) return srv_fail(HOQRI_ERR_INVALID, "hoqri_server_step: NULL server");
    // admissions whose set-up finished on their worker thread
    for (auto &kv : s->reqs) {
        Req *r = kv.second.get();
        if (r->admitting && r->setup.wait_for(std::chrono::seconds(0)) == std::future_status::ready) admit_done(s, r);
    }
    // finished requests: their event has completed (non-blocking query)
    for (auto &kv : s->reqs) {
        Req *r = kv.second.get();
        if (r->state != HOQRI_REQ_RUNNING || r->admitting) continue;
        const cudaError_t e = cudaEventQuery(r->done);
        if (e == cudaErrorNotReady) continue;
        r->t_done = now_s();
        --s->active;
        if (e != cudaSuccess) {
            cudaGetLastError();
            r->status = HOQRI_ERR_CUDA;
            r->error = cudaGetErrorString(e);
            r->state = HOQRI_REQ_FAILED;
            release(s, r);
        } else {
            r->state = HOQRI_REQ_DONE;
        }
    }
    // admission in arrival order: the head waits until memory and a slot are free;
    // its set-up starts on a worker thread (the estimate is charged meanwhile)
    while (!s->queue.empty() && s->active < s->max_active) {
        Req *r = s->reqs[s->queue.front()].get();
        if (s->in_use + r->est_bytes > s->budget) break;
        s->queue.pop_front();
        s->in_use += r->est_bytes;
        ++s->active;
        r->admitting = true;
        r->state = HOQRI_REQ_RUNNING;  // reported as running from dispatch on
        r->setup = std::async(std::launch::async, admit_work, r);
    }
    if (n_running) *n_running = s->active;
    if (n_queued) *n_queued = (int32_t)s->queue.size();
    return HOQRI_OK;
}

hoqri_status hoqri_server_poll(hoqri_server *s, int64_t id, int32_t *state, double *times, int64_t *device_bytes) {
    if (!s) return srv_fail(HOQRI_ERR_INVALID, "hoqri_server_poll: NULL server");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return srv_fail(HOQRI_ERR_INVALID, "hoqri_server_poll: unknown request id");
    Req *r = it->second.get();
    if (state) *state = r->state;
    if (times) {
        times[0] = r->t_submit;
        times[1] = r->t_admit;
        times[2] = r->t_done;
    }
    if (device_bytes) *device_bytes = r->state == HOQRI_REQ_QUEUED ? r->est_bytes : r->bytes;
    if (r->state == HOQRI_REQ_FAILED) {
        set_error(r->error);
        return r->status;
    }
    return HOQRI_OK;
}

hoqri_status hoqri_server_take(hoqri_server *s, int64_t id, void *const *U_out, void *G_out, double *resid) {
    if (!s) return srv_fail(HOQRI_ERR_INVALID, "hoqri_server_take: NULL server");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return srv_fail(HOQRI_ERR_INVALID, "hoqri_server_take: unknown request id");
    Req *r = it->second.get();
    if (r->state == HOQRI_REQ_FAILED) {
        const hoqri_status st = r->status;
        const std::string m = r->error;
        s->reqs.erase(it);
        return srv_fail(st, m);
    }
    if (r->state != HOQRI_REQ_DONE) return srv_fail(HOQRI_ERR_INVALID, "hoqri_server_take: request not finished");
    // the fit of the last sweep first: hoqri_core recomputes the core (and its norm)
    hoqri_status st = HOQRI_OK;
    if (resid) st = hoqri_fit(r->ctx, resid, nullptr, nullptr);
    for (int n = 0; n < r->N && st == HOQRI_OK; ++n)
        if (U_out && U_out[n]) st = hoqri_get_factor(r->ctx, n, U_out[n]);
    if (st == HOQRI_OK && G_out) st = hoqri_core(r->ctx, G_out);
    if (st == HOQRI_OK) st = hoqri_synchronize(r->ctx);
    release(s, r);
    s->reqs.erase(it);
    return st;
}

void hoqri_server_destroy(hoqri_server *s) {
    if (!s) return;
    for (auto &kv : s->reqs) release(s, kv.second.get());
    delete s;
}

}  // extern "C"
