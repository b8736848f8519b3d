"""Serving driver: an open-loop stream of decomposition requests against the
library's request server (hoqri_server_*, continuous batching by device memory).

Requests follow the serving mix of ``inputs.serving_mix``: Poisson arrivals,
order 3 or 4, dims uniform in [1e3, 1e6], log10 nnz ~ N(5.5, 0.5) clipped to
[4, 7], Zipf(1.1) indices, ranks from {4, 8, 16, 32}.  Each request's tensor is
drawn (seeded) before the clock starts; it is submitted at its arrival time,
admitted by the server when device memory and a slot are free, and its latency
is completion minus arrival.  Argument marshalling only: every step of every
request runs in the CUDA library.
"""
from __future__ import annotations

import time

import numpy as np

from . import hoqri, inputs


def draw_requests(n_req, seed, rate_hz=1.0, iters=10, only=None, max_pm=None):
    """The request list with its tensors: [(ServeRequest, SparseTensor)]
    (only: indices of the requests to draw tensors for; None: all)."""
    reqs = inputs.serving_mix(n_req, rate_hz, seed, max_pm=max_pm)
    out = []
    for k in (range(len(reqs)) if only is None else only):
        q = reqs[k]
        X = inputs.random_sparse(q.dims, q.nnz, q.seed, dist="zipf", s=1.1, values="lognormal", dtype=np.float32)
        out.append((q, X))
    return out


def _draw_chunk(args):
    n_req, seed, ks, max_pm = args
    return draw_requests(n_req, seed, only=ks, max_pm=max_pm)


def draw_requests_async(pool, n_req, seed, max_pm=None, chunks=32):
    """Starts drawing the request tensors in a process pool (spawn context, so
    it may be created before or after CUDA is initialised); returns a callable
    that waits and gives the list in request order."""
    ks = list(range(n_req))
    parts = [ks[i::chunks] for i in range(chunks)]
    res = pool.map_async(_draw_chunk, [(n_req, seed, part, max_pm) for part in parts if part])

    def get():
        out = [None] * n_req
        for part in res.get():
            for q, X in part:
                out[q.rid] = (q, X)
        return out
    return get


def run_sequential(reqs, prec=hoqri.HOQRI_FP32, iters=10):
    """The plain method on the same requests: one context after another
    (hoqri_create from host arrays, `iters` sweeps, the fit), nothing
    overlapped.  Returns makespan, nnz/s and every residual."""
    t0 = time.perf_counter()
    work = 0.0
    resid = []
    for q, X in reqs:
        opt = hoqri.hoqri_default_options(prec=prec, seed=q.seed)
        c = hoqri.hoqri_create(X.dims, q.ranks, X.nnz, X.idx, X.vals, opt, None, 0)
        try:
            hoqri.hoqri_iterate(c, iters, want_hist=False)
            r, _, _ = hoqri.hoqri_fit(c)
        finally:
            hoqri.hoqri_destroy(c)
        resid.append(r)
        work += X.nnz * X.N * iters
    makespan = time.perf_counter() - t0
    return {"makespan_s": makespan, "nnz_per_s": work / makespan, "resid": resid}


def run_stream(reqs, budget_bytes, max_active, prec=hoqri.HOQRI_FP32, iters=10, arrival_scale=1.0,
               closed=False, poll_s=2e-4):
    """Submits every request at arrival_scale * its arrival time (all at once
    when closed) and drives the server until all are done.

    Returns a dict: per-request latency (s), makespan (s), aggregate nnz/s
    (nnz * N * iters summed over requests / makespan), p50 / p99 latency, the
    most requests running at once, and the residual of each request."""
    srv = hoqri.hoqri_server_create(int(budget_bytes), int(max_active))
    try:
        order = sorted(range(len(reqs)), key=lambda k: reqs[k][0].arrival_s)
        t0 = time.perf_counter()
        nxt = 0
        live = {}
        lat = {}
        resid = {}
        failed = {}
        max_running = 0
        work = 0.0
        while nxt < len(order) or live:
            now = time.perf_counter() - t0
            while nxt < len(order) and (closed or reqs[order[nxt]][0].arrival_s * arrival_scale <= now):
                k = order[nxt]
                q, X = reqs[k]
                rid = hoqri.hoqri_server_submit(srv, X.dims, q.ranks, X.nnz, X.idx, X.vals, iters, prec, q.seed)
                live[rid] = (k, 0.0 if closed else q.arrival_s * arrival_scale)
                nxt += 1
            running, _ = hoqri.hoqri_server_step(srv)
            max_running = max(max_running, running)
            done_any = False
            for rid in list(live):
                try:
                    st, _, _ = hoqri.hoqri_server_poll(srv, rid)
                except hoqri.HoqriError as e:  # failed at admission: reported, not timed
                    k, _ = live.pop(rid)
                    failed[k] = str(e)
                    continue
                if st == hoqri.HOQRI_REQ_DONE:
                    t_done = time.perf_counter() - t0
                    k, t_arr = live.pop(rid)
                    resid[k] = hoqri.hoqri_server_take(srv, rid)
                    lat[k] = t_done - t_arr
                    q, X = reqs[k]
                    work += X.nnz * X.N * iters
                    done_any = True
            if not done_any:
                time.sleep(poll_s)
        makespan = time.perf_counter() - t0
    finally:
        hoqri.hoqri_server_destroy(srv)
    ls = np.array([lat[k] for k in sorted(lat)])
    return {"latency_s": ls.tolist(), "makespan_s": makespan, "nnz_per_s": work / makespan,
            "p50_s": float(np.percentile(ls, 50)), "p99_s": float(np.percentile(ls, 99)),
            "max_running": max_running, "resid": [resid.get(k) for k in range(len(reqs))],
            "failed": {str(k): v for k, v in failed.items()}}


SERVE_SEED = 0x484F5152 + 5


def serve_benchmark(n_req=2000, seed=SERVE_SEED, budget_bytes=200 << 30, max_active=32, iters=10,
                    prec=hoqri.HOQRI_FP32, load=0.8, reqs=None, sequential=True, sweep_loads=(0.5, 1.2),
                    sweep_requests=500):
    """Capacity from a closed batch (all requests at once), then the open-loop
    Poisson stream at `load` x that capacity (p50 / p99 latency, nnz/s), the
    plain method on the same requests one after another, and the latency at
    other loads (`sweep_loads` x capacity) on the first `sweep_requests`
    requests."""
    if reqs is None:
        reqs = draw_requests(n_req, seed, 1.0, iters)
    n_req = len(reqs)
    closed = run_stream(reqs, budget_bytes, max_active, prec, iters, closed=True)
    cap_rps = n_req / closed["makespan_s"]
    rate = load * cap_rps
    # arrivals were drawn at 1 request/s: scale them to the target rate
    open_ = run_stream(reqs, budget_bytes, max_active, prec, iters, arrival_scale=1.0 / rate)
    nnz = [X.nnz for _, X in reqs]
    out = {"requests": n_req, "iters": iters, "load": load, "capacity_req_per_s": cap_rps,
           "arrival_rate_req_per_s": rate, "p50_s": open_["p50_s"], "p99_s": open_["p99_s"],
           "nnz_per_s": open_["nnz_per_s"], "makespan_s": open_["makespan_s"],
           "max_running": open_["max_running"], "closed_nnz_per_s": closed["nnz_per_s"],
           "closed_makespan_s": closed["makespan_s"], "failed": len(open_["failed"]),
           "nnz_total": int(sum(nnz)), "nnz_median": float(np.median(nnz)), "nnz_max": int(max(nnz)),
           "orders": {str(o): sum(1 for q, _ in reqs if len(q.dims) == o) for o in (3, 4)},
           "budget_bytes": budget_bytes, "max_active": max_active}
    if sequential:
        seq = run_sequential(reqs, prec, iters)
        out["sequential"] = {"makespan_s": seq["makespan_s"], "nnz_per_s": seq["nnz_per_s"],
                             "step": "hoqri_create + sweeps + fit per request, one after another"}
        out["served_over_sequential"] = closed["nnz_per_s"] / seq["nnz_per_s"]
        same = [a for a, b in zip(closed["resid"], seq["resid"]) if a is not None and b is not None and a == b]
        out["resid_equal_to_sequential"] = len(same)
        out["resid_differs_from_sequential"] = [
            {"request": k, "served": a, "sequential": b} for k, (a, b) in enumerate(zip(closed["resid"], seq["resid"]))
            if a is not None and a != b][:20]
    sweep = []
    sub = reqs[:min(sweep_requests, n_req)]
    for ld in sweep_loads:
        r = run_stream(sub, budget_bytes, max_active, prec, iters, arrival_scale=1.0 / (ld * cap_rps))
        sweep.append({"load": ld, "requests": len(sub), "arrival_rate_req_per_s": ld * cap_rps, "p50_s": r["p50_s"],
                      "p99_s": r["p99_s"], "nnz_per_s": r["nnz_per_s"], "max_running": r["max_running"],
                      "failed": len(r["failed"])})
    if sweep:
        out["load_sweep"] = sweep
    out["failures"] = dict(list(open_["failed"].items())[:10])
    return out
