"""Serving (hoqri_server_*): requests of differing order, nnz and ranks run
concurrently on one GPU, admitted by device memory.  Each request's results are
bit-identical alone, in the mix, and from a lone context (same kernels, same
order of arithmetic)."""
import numpy as np
import pytest

from paper_2510_16930_gb300 import hoqri, inputs

pytestmark = pytest.mark.gpu

FP32, MIX = hoqri.HOQRI_FP32, hoqri.HOQRI_BF16X3

REQS = [
    # dims, ranks, nnz, prec
    ((3000, 2000, 1000), (16, 16, 16), 200_000, FP32),
    ((500, 400, 300, 200), (8, 8, 8, 8), 150_000, FP32),
    ((20_000, 5_000, 8_000), (4, 8, 4), 50_000, FP32),
    ((2000, 1500, 1000), (32, 32, 32), 100_000, FP32),
    ((3000, 2000, 1000), (16, 16, 16), 200_000, MIX),
    ((1200, 900, 700, 300), (4, 16, 8, 4), 80_000, FP32),
]


def _tensors():
    out = []
    for k, (dims, ranks, nnz, prec) in enumerate(REQS):
        X = inputs.random_sparse(dims, nnz, 700 + k, dist="zipf", s=1.1, values="lognormal", dtype=np.float32)
        out.append((X, ranks, prec, 900 + k))
    return out


def _run(torch, reqs, budget, max_active, iters=4):
    """Submits all requests at once; returns per request (factors, core, resid) and
    the most requests seen running at once."""
    srv = hoqri.hoqri_server_create(budget, max_active)
    try:
        ids = [hoqri.hoqri_server_submit(srv, X.dims, ranks, X.nnz, X.idx, X.vals, iters, prec, seed)
               for X, ranks, prec, seed in reqs]
        res = {}
        max_running = 0
        while len(res) < len(ids):
            running, _ = hoqri.hoqri_server_step(srv)
            max_running = max(max_running, running)
            for k, rid in enumerate(ids):
                if k in res:
                    continue
                st, _, _ = hoqri.hoqri_server_poll(srv, rid)
                if st == hoqri.HOQRI_REQ_DONE:
                    X, ranks, prec, _ = reqs[k]
                    U = [np.zeros((d, r), np.float32) for d, r in zip(X.dims, ranks)]
                    G = np.zeros(ranks, np.float32)
                    r = hoqri.hoqri_server_take(srv, rid, U, G)
                    res[k] = (U, G, r)
        return [res[k] for k in range(len(ids))], max_running
    finally:
        hoqri.hoqri_server_destroy(srv)


def test_each_result_same_alone_and_in_the_mix():
    torch = pytest.importorskip("torch")
    reqs = _tensors()
    mix, max_running = _run(torch, reqs, 64 << 30, 8)
    assert max_running >= 2  # the requests did overlap
    for k, q in enumerate(reqs):
        alone, _ = _run(torch, [q], 64 << 30, 1)
        U0, G0, r0 = alone[0]
        U1, G1, r1 = mix[k]
        assert r0 == r1, k
        assert np.array_equal(G0, G1), k
        for a, b in zip(U0, U1):
            assert np.array_equal(a, b), k


def test_served_request_equals_lone_context():
    torch = pytest.importorskip("torch")
    X, ranks, prec, seed = _tensors()[0]
    (res,), _ = _run(torch, [(X, ranks, prec, seed)], 64 << 30, 1, iters=4)
    st = torch.cuda.Stream()
    opt = hoqri.hoqri_default_options(prec=prec, seed=seed)
    h = hoqri.hoqri_create(X.dims, ranks, X.nnz, X.idx, X.vals, opt, None, st.cuda_stream)
    try:
        hoqri.hoqri_iterate(h, 4, want_hist=False)
        U = [np.zeros((d, r), np.float32) for d, r in zip(X.dims, ranks)]
        for n in range(3):
            hoqri.hoqri_get_factor(h, n, U[n])
        r, _, _ = hoqri.hoqri_fit(h)
    finally:
        hoqri.hoqri_destroy(h)
    assert r == res[2]
    for a, b in zip(U, res[0]):
        assert np.array_equal(a, b)


def test_admission_by_memory_budget():
    """Three requests of one shape and a budget just above one admission estimate:
    they run one after the other, all complete, and give the same results."""
    torch = pytest.importorskip("torch")
    dims, ranks, nnz, prec = REQS[0]
    reqs = []
    for k in range(3):
        X = inputs.random_sparse(dims, nnz, 800 + k, dist="zipf", s=1.1, values="lognormal", dtype=np.float32)
        reqs.append((X, ranks, prec, 50 + k))
    srv = hoqri.hoqri_server_create(64 << 30, 1)
    try:
        X, ranks, prec, seed = reqs[0]
        rid = hoqri.hoqri_server_submit(srv, X.dims, ranks, X.nnz, X.idx, X.vals, 4, prec, seed)
        _, _, est = hoqri.hoqri_server_poll(srv, rid)  # the estimate, while queued
    finally:
        hoqri.hoqri_server_destroy(srv)
    free, _ = _run(torch, reqs, 64 << 30, 8)
    tight, max_running = _run(torch, reqs, int(est * 1.05), 8)
    assert max_running == 1
    for (U0, G0, r0), (U1, G1, r1) in zip(free, tight):
        assert r0 == r1 and np.array_equal(G0, G1)


def test_failed_request_does_not_stop_the_others():
    torch = pytest.importorskip("torch")
    X, ranks, prec, seed = _tensors()[2]
    srv = hoqri.hoqri_server_create(64 << 30, 4)
    try:
        bad = hoqri.hoqri_server_submit(srv, X.dims, (4, 8, 40), X.nnz, X.idx, X.vals, 2, FP32, 1)  # K_2 > K_0 K_1
        good = hoqri.hoqri_server_submit(srv, X.dims, ranks, X.nnz, X.idx, X.vals, 2, FP32, 1)
        state = {}
        while len(state) < 2:
            hoqri.hoqri_server_step(srv)
            for rid in (bad, good):
                try:
                    st, _, _ = hoqri.hoqri_server_poll(srv, rid)
                except hoqri.HoqriError as e:
                    state[rid] = e.code
                    continue
                if st == hoqri.HOQRI_REQ_DONE:
                    state[rid] = hoqri.HOQRI_OK
        assert state[bad] == hoqri.HOQRI_ERR_RANK
        assert state[good] == hoqri.HOQRI_OK
        assert hoqri.hoqri_server_take(srv, good) > 0
    finally:
        hoqri.hoqri_server_destroy(srv)


def test_served_results_match_the_oracle():
    """Small FP64 requests of order 3 and 4 served together: each request's
    residual history end and its factors' subspaces equal the oracle's Alg. 2
    from the same initial factors (those the library draws from the request's
    seed, read from a lone context before any sweep)."""
    torch = pytest.importorskip("torch")
    from oracle import oracle as orc
    orc.build()
    FP64 = hoqri.HOQRI_FP64
    cases = [((40, 30, 20), (4, 3, 5), 3000, 31), ((16, 14, 12, 10), (3, 2, 4, 2), 2500, 32),
             ((60, 50, 40), (8, 8, 4), 5000, 33)]
    reqs = []
    for k, (dims, ranks, nnz, seed) in enumerate(cases):
        X = inputs.random_sparse(dims, nnz, 1100 + k, dist="zipf", s=1.1, values="uniform", dtype=np.float64)
        reqs.append((X, ranks, seed))
    iters = 5
    srv = hoqri.hoqri_server_create(8 << 30, 4)
    try:
        ids = [hoqri.hoqri_server_submit(srv, X.dims, ranks, X.nnz, X.idx, X.vals, iters, FP64, seed)
               for X, ranks, seed in reqs]
        res = {}
        while len(res) < len(ids):
            hoqri.hoqri_server_step(srv)
            for k, rid in enumerate(ids):
                if k not in res and hoqri.hoqri_server_poll(srv, rid)[0] == hoqri.HOQRI_REQ_DONE:
                    X, ranks, _ = reqs[k]
                    U = [np.zeros((d, r), np.float64) for d, r in zip(X.dims, ranks)]
                    res[k] = (U, hoqri.hoqri_server_take(srv, rid, U))
    finally:
        hoqri.hoqri_server_destroy(srv)
    for k, (X, ranks, seed) in enumerate(reqs):
        # the initial factors of the request: a lone context from the same seed
        opt = hoqri.hoqri_default_options(prec=FP64, seed=seed)
        c = hoqri.hoqri_create(X.dims, ranks, X.nnz, X.idx, X.vals, opt, None, 0)
        try:
            U0 = []
            for n, (d, r) in enumerate(zip(X.dims, ranks)):
                u = np.zeros((d, r), np.float64)
                hoqri.hoqri_get_factor(c, n, u)
                U0.append(u)
        finally:
            hoqri.hoqri_destroy(c)
        ref = orc.hoqri(X.dims, X.idx, X.vals, U0, iters)
        U, r = res[k]
        assert abs(r - ref["resid"][-1]) <= 1e-10 * ref["resid"][-1], k
        for a, b in zip(U, ref["U"]):
            assert np.linalg.norm(a @ a.T - b @ b.T) <= 1e-8, k
