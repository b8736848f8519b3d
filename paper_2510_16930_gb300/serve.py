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


def draw_requests(n_req, seed, rate_hz=1.0, iters=10):
    """The request list with its tensors: [(ServeRequest, SparseTensor)]."""
    reqs = inputs.serving_mix(n_req, rate_hz, seed)
    out = []
    for q in reqs:
        X = inputs.random_sparse(q.dims, q.nnz, q.seed, dist="zipf", s=1.1, values="lognormal", dtype=np.float32)
        out.append((q, X))
    return out


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


def serve_benchmark(n_req=120, seed=0x484F5152 + 5, budget_bytes=200 << 30, max_active=32, iters=10,
                    prec=hoqri.HOQRI_FP32, load=0.8):
    """Capacity from a closed batch (all requests at once), then the open-loop
    Poisson stream at `load` x that capacity; p50 / p99 latency and nnz/s."""
    reqs = draw_requests(n_req, seed, 1.0, iters)
    closed = run_stream(reqs, budget_bytes, max_active, prec, iters, closed=True)
    cap_rps = n_req / closed["makespan_s"]
    rate = load * cap_rps
    # arrivals were drawn at 1 request/s: scale them to the target rate
    open_ = run_stream(reqs, budget_bytes, max_active, prec, iters, arrival_scale=1.0 / rate)
    nnz = [X.nnz for _, X in reqs]
    return {"requests": n_req, "iters": iters, "load": load, "capacity_req_per_s": cap_rps,
            "arrival_rate_req_per_s": rate, "p50_s": open_["p50_s"], "p99_s": open_["p99_s"],
            "nnz_per_s": open_["nnz_per_s"], "makespan_s": open_["makespan_s"],
            "max_running": open_["max_running"], "closed_nnz_per_s": closed["nnz_per_s"],
            "failed": len(open_["failed"]),
            "nnz_median": float(np.median(nnz)), "nnz_max": int(max(nnz)),
            "orders": {str(o): sum(1 for q, _ in reqs if len(q.dims) == o) for o in (3, 4)},
            "budget_bytes": budget_bytes, "max_active": max_active}
