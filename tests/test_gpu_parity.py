"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (relative Frobenius error on A_n and G): 1e-10 for the FP64 path and
1e-5 for the FP32 path, the bounds the hot path is held to.  Sizes span
several warp tasks (chunks) and a ragged tail; the chunk size is forced small
in places so that rows cross chunk boundaries and the fix-up path runs.
"""
import numpy as np
import pytest

from paper_2510_16930_gb300 import hoqri, inputs
from tests import dense_ref as D
from tests.gpu_util import TOL, Ctx, rel

pytestmark = pytest.mark.gpu

FP64, FP32 = hoqri.HOQRI_FP64, hoqri.HOQRI_FP32


def _case(dims, ranks, nnz, seed, dist="uniform", s=1.1, values="uniform"):
    X = inputs.random_sparse(dims, nnz, seed, dist=dist, s=s, values=values, dtype=np.float64)
    U0 = inputs.orthonormal_factors(dims, ranks, seed + 1)
    return X, U0


SHAPES = [
    # (dims, ranks, nnz, dist)
    ((40, 30, 20), (5, 4, 3), 3000, "uniform"),
    ((200, 200, 200), (5, 5, 5), 10_000, "uniform"),       # the 200^3 FP64 workload
    ((300, 100, 50), (16, 16, 16), 20_000, "zipf"),        # K = 16, skewed rows
    ((30, 20, 20, 10), (4, 3, 2, 3), 5000, "zipf"),        # order 4
    ((12, 10, 9, 8, 7), (2, 3, 2, 2, 3), 3000, "uniform"), # order 5
    ((500, 400), (7, 7), 4000, "uniform"),                  # order 2 (matrix)
    ((64, 50, 40), (1, 1, 1), 2000, "uniform"),            # rank one
    ((60, 50, 40), (8, 16, 12), 4000, "zipf"),             # P_{-n} up to 192, mixed K
    ((60, 40, 30, 20), (8, 8, 8, 8), 20_000, "zipf"),      # order 4, K = 8 (register tiles)
    ((40, 30, 20, 16), (4, 8, 4, 8), 6000, "uniform"),      # order 4, mixed power-of-two K
    ((500, 300, 200), (32, 32, 32), 8000, "zipf"),         # K = 32: 1024-element y per row
    ((400, 300, 200), (4, 16, 8), 8000, "zipf"),           # small and mixed tiles
]


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("chunk", [0, 32, 96])
@pytest.mark.parametrize("shape", SHAPES, ids=[str(s[0]) for s in SHAPES])
def test_ttmctc_and_core_match_oracle(orc, shape, chunk, prec):
    dims, ranks, nnz, dist = shape
    X, U0 = _case(dims, ranks, nnz, 1234 + nnz, dist=dist)
    npdt = np.float64 if prec == FP64 else np.float32
    vals = X.vals.astype(npdt)
    U0c = [u.astype(npdt) for u in U0]
    # the oracle sees exactly the values the device sees
    U0o = [u.astype(np.float64) for u in U0c]
    vo = vals.astype(np.float64)
    with Ctx(dims, X.idx, vals, U0c, prec, chunk=chunk) as c:
        for n in range(len(dims)):
            A_ref, G_ref = orc.ttmctc(dims, X.idx, vo, U0o, n, return_core=True)
            A = c.ttmctc(n)
            assert rel(A, A_ref) <= TOL[prec], (n, rel(A, A_ref))
        G = c.core()
        assert rel(G, G_ref) <= TOL[prec]


@pytest.mark.parametrize("chunk", [0, 96])
@pytest.mark.parametrize("shape", SHAPES, ids=[str(s[0]) for s in SHAPES])
def test_o_ik_form_matches_oracle(orc, shape, chunk):
    """The O(IK)-memory form of Table 2 (one_stream = 2: a separate core pass
    over the nonzeros, no stored Y_(n)) for FP32, every shape, against Alg. 3."""
    dims, ranks, nnz, dist = shape
    X, U0 = _case(dims, ranks, nnz, 1234 + nnz, dist=dist)
    vals = X.vals.astype(np.float32)
    U0c = [u.astype(np.float32) for u in U0]
    U0o = [u.astype(np.float64) for u in U0c]
    vo = vals.astype(np.float64)
    with Ctx(dims, X.idx, vals, U0c, FP32, chunk=chunk, one_stream=2) as c:
        _, _, dev_bytes = c.info()
        for n in range(len(dims)):
            A_ref, G_ref = orc.ttmctc(dims, X.idx, vo, U0o, n, return_core=True)
            A = c.ttmctc(n)
            assert rel(A, A_ref) <= TOL[FP32], (n, rel(A, A_ref))
        G = c.core()
        assert rel(G, G_ref) <= TOL[FP32]
    # no Y_(n) is held: the context is no larger than the one-stream form's
    with Ctx(dims, X.idx, vals, U0c, FP32, chunk=chunk) as c1:
        assert dev_bytes <= c1.info()[2]


BLOCKED = [
    # P_{-n} above 2048: the generic pass runs one launch per column block
    ((40, 30, 20, 20), (16, 16, 16, 8), 3000, "zipf"),          # mode 3: 4096 = 2 blocks
    ((14, 13, 12, 11, 10), (10, 10, 10, 10, 10), 2000, "uniform"),  # 10^4 = 4 blocks of 2040 + 1840
]


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("shape", BLOCKED, ids=[str(s[0]) for s in BLOCKED])
def test_column_blocked_passes_match_oracle(orc, shape, prec):
    dims, ranks, nnz, dist = shape
    X, U0 = _case(dims, ranks, nnz, 4321 + nnz, dist=dist)
    npdt = np.float64 if prec == FP64 else np.float32
    vals = X.vals.astype(npdt)
    U0c = [u.astype(npdt) for u in U0]
    U0o = [u.astype(np.float64) for u in U0c]
    vo = vals.astype(np.float64)
    with Ctx(dims, X.idx, vals, U0c, prec, chunk=32) as c:
        for n in range(len(dims)):
            A_ref, G_ref = orc.ttmctc(dims, X.idx, vo, U0o, n, return_core=True)
            A = c.ttmctc(n)
            assert rel(A, A_ref) <= TOL[prec], (n, rel(A, A_ref))
        assert rel(c.core(), G_ref) <= TOL[prec]
        h = c.iterate(2)
        assert np.all(np.isfinite(h)) and h[1] <= h[0] * (1 + 1e-12)


def test_fit_and_nnz_after_coalescing(orc):
    dims, ranks = (50, 40, 30), (4, 4, 3)
    X, U0 = _case(dims, ranks, 6000, 77)
    # plant repeats: the last 500 entries repeat the first 500 coordinates
    for a in X.idx:
        a[-500:] = a[:500]
    ci, cv = orc.coalesce(X.idx, X.vals)
    with Ctx(dims, X.idx, X.vals, U0, FP64) as c:
        nnz, rows, _ = c.info()
        assert nnz == len(cv)
        assert rows == [int(np.unique(a).size) for a in ci]
        G = c.core()
        r, nx2, ng2 = hoqri.hoqri_fit(c.h)
        assert abs(nx2 - orc.norm2(cv)) <= 1e-12 * nx2
        G_ref = orc.core(X.idx, X.vals, U0)
        assert abs(ng2 - float((G_ref ** 2).sum())) <= 1e-10 * ng2


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("I,K", [(1000, 5), (257, 16), (64, 64), (5000, 8), (16, 1), (3001, 10), (2000, 12),
                                 (4000, 20), (1500, 24)])
def test_orthonormalize_matches_householder(orc, I, K, prec):
    rng = np.random.default_rng(I + K)
    A = rng.standard_normal((I, K)) * np.logspace(0, -2, K)[None, :]
    npdt = np.float64 if prec == FP64 else np.float32
    A = A.astype(npdt)
    dims = (I, max(2, K), max(2, K))
    X, U0 = _case(dims, (K, K, K) if K > 1 else (1, 1, 1), 100, 5)
    with Ctx(dims, X.idx, X.vals.astype(npdt), [u.astype(npdt) for u in U0], prec) as c:
        Q = c.orthonormalize(0, A)
    Q_ref, R_ref, z = orc.qr(A.astype(np.float64))
    tol = 1e-12 if prec == FP64 else 2e-6
    assert rel(Q, Q_ref) <= tol * K
    assert np.linalg.norm(Q.T @ Q - np.eye(K)) <= (1e-13 if prec == FP64 else 1e-5)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("K", [6, 10])
def test_orthonormalize_rank_deficient_falls_back(orc, prec, K):
    rng = np.random.default_rng(8)
    I = 300
    A = rng.standard_normal((I, K))
    A[:, 3] = 0.0
    A[:, 5] = A[:, 1]
    npdt = np.float64 if prec == FP64 else np.float32
    A = A.astype(npdt)
    X, U0 = _case((I, 10, 10), (K, 4, 4), 200, 9)
    with Ctx((I, 10, 10), X.idx, X.vals.astype(npdt), [u.astype(npdt) for u in U0], prec) as c:
        Q = c.orthonormalize(0, A)
    tol = 1e-12 if prec == FP64 else 1e-5
    assert np.linalg.norm(Q.T @ Q - np.eye(K)) <= tol
    A64 = A.astype(np.float64)
    assert np.linalg.norm(A64 - Q @ (Q.T @ A64)) <= tol * np.linalg.norm(A64)


def _ill_conditioned(kind, I, K, seed):
    """I x K with a Cholesky pivot of its Gram below 1e-14 of the largest
    diagonal entry: column scaling over 7.5 decades (Q itself stays well
    determined), or singular values graded 1 .. 1e-9 in random directions
    (kappa 1e9, beyond what unshifted CholeskyQR2 can take)."""
    rng = np.random.default_rng(seed)
    if kind == "scaled":
        return rng.standard_normal((I, K)) * np.logspace(0, -7.5, K)[None, :]
    sig = np.logspace(0, -9, K)
    Q0, _ = np.linalg.qr(rng.standard_normal((I, K)))
    V, _ = np.linalg.qr(rng.standard_normal((K, K)))
    return (Q0 * sig[None, :]) @ V.T


@pytest.mark.parametrize("prec,kind,K", [(FP64, "scaled", 16), (FP32, "scaled", 16), (FP64, "graded", 16),
                                        (FP32, "scaled", 10), (FP32, "scaled", 20)])
def test_orthonormalize_ill_conditioned_is_shifted_not_broken(orc, prec, kind, K):
    """Unshifted CholeskyQR2 breaks down on these inputs; with qr_kind 2 (a
    breakdown is an error) the call succeeds, so the shifted first pass
    (shifted CholeskyQR3) produced Q.  Q is orthonormal, spans A, and equals the
    oracle's Q to the conditioning of the problem (kappa u ~ 1e-7 for the graded
    case)."""
    I = 5000
    A = _ill_conditioned(kind, I, K, 31)
    npdt = np.float64 if prec == FP64 else np.float32
    A = A.astype(npdt)
    X, U0 = _case((I, K, K), (K, K, K), 100, 5)
    with Ctx((I, K, K), X.idx, X.vals.astype(npdt), [u.astype(npdt) for u in U0], prec, qr_kind=2) as c:
        Q = c.orthonormalize(0, A)
    A64 = A.astype(np.float64)
    Q_ref, _, _ = orc.qr(A64)
    tol_orth = 1e-13 if prec == FP64 else 1e-5
    assert np.linalg.norm(Q.T @ Q - np.eye(K)) <= tol_orth
    assert np.linalg.norm(A64 - Q @ (Q.T @ A64)) <= tol_orth * np.linalg.norm(A64)
    tol_q = {("scaled", FP64): 1e-11, ("scaled", FP32): 2e-6 * K, ("graded", FP64): 1e-6}[(kind, prec)]
    assert rel(Q, Q_ref) <= tol_q


def test_hoqri_200cubed_fp64_matches_oracle(orc):
    """The 200^3, nnz 1e4, K = 5 workload, 10 iterations, FP64 throughout."""
    X, U0, cfg = inputs.make_config("c1")
    ref = orc.hoqri(X.dims, X.idx, X.vals, U0, cfg["iters"])
    with Ctx(X.dims, X.idx, X.vals, U0, FP64) as c:
        hist = c.iterate(cfg["iters"])
        G = c.core()
        for n in range(3):
            assert rel(c.factor(n), ref["U"][n]) <= 1e-10
        assert rel(G, ref["G"]) <= 1e-10
    np.testing.assert_allclose(hist, ref["resid"], rtol=1e-12, atol=0)


def test_hoqri_fp32_tracks_fp64(orc):
    """FP32 path on a scaled-down Zipf K=16 workload: final fit within 1e-6 of FP64."""
    X = inputs.random_sparse((3000, 1500, 800), 40_000, 4242, dist="zipf", s=1.1, values="lognormal",
                             dtype=np.float64, distinct=True)
    U0 = inputs.orthonormal_factors(X.dims, (16, 16, 16), 4243)
    iters = 3
    ref = orc.hoqri(X.dims, X.idx, X.vals.astype(np.float32).astype(np.float64), U0, iters)
    with Ctx(X.dims, X.idx, X.vals.astype(np.float32), [u.astype(np.float32) for u in U0], FP32) as c:
        hist = c.iterate(iters)
        for n in range(3):
            U = c.factor(n)
            assert D.proj_dist(U, ref["U"][n]) <= 1e-3
    assert abs(hist[-1] - ref["resid"][-1]) <= 1e-6 * ref["resid"][-1]


def test_hoqri_monotone_and_orthonormal_on_device():
    X = inputs.random_sparse((800, 600, 400), 30_000, 99, dist="zipf", values="lognormal", distinct=True)
    U0 = inputs.orthonormal_factors(X.dims, (8, 8, 8), 100)
    with Ctx(X.dims, X.idx, X.vals, U0, FP64) as c:
        hist = c.iterate(6)
        assert np.all(np.diff(hist) <= 1e-12)  # Thm. 1: residual never grows
        for n in range(3):
            U = c.factor(n)
            assert np.linalg.norm(U.T @ U - np.eye(8)) <= 1e-13


def test_eq_AU_on_device():
    """Eq. (AU): A_n^T U_n = G_(n) G_(n)^T from device outputs alone (FP32)."""
    X = inputs.random_sparse((5000, 3000, 1000), 200_000, 5, dist="zipf", values="lognormal", distinct=True)
    U0 = inputs.orthonormal_factors(X.dims, (16, 16, 16), 6)
    U0f = [u.astype(np.float32) for u in U0]
    with Ctx(X.dims, X.idx, X.vals.astype(np.float32), U0f, FP32) as c:
        for n in range(3):
            A = c.ttmctc(n)
            G = c.core()
            Gn = D.unfold(G, n)
            assert rel(A.T @ U0f[n].astype(np.float64), Gn @ Gn.T) <= 1e-5


def test_degenerate_inputs(orc):
    # empty tensor
    dims, ranks = (10, 9, 8), (2, 2, 2)
    U0 = inputs.orthonormal_factors(dims, ranks, 3)
    e = [np.zeros(0, dtype=np.int32)] * 3
    with Ctx(dims, e, np.zeros(0), U0, FP64) as c:
        assert np.all(c.ttmctc(0) == 0) and np.all(c.core() == 0)
        assert c.info()[0] == 0
    # a single nonzero
    one = [np.array([3], dtype=np.int32), np.array([4], dtype=np.int32), np.array([5], dtype=np.int32)]
    with Ctx(dims, one, np.array([2.5]), U0, FP64) as c:
        for n in range(3):
            assert rel(c.ttmctc(n), orc.ttmctc(dims, one, [2.5], U0, n)) <= 1e-12
    # every nonzero in one mode-0 row (one row spanning many chunks)
    rng = np.random.default_rng(11)
    nnz = 5000
    idx = [np.full(nnz, 7, dtype=np.int32), rng.integers(0, 9, nnz).astype(np.int32),
           rng.integers(0, 8, nnz).astype(np.int32)]
    v = rng.standard_normal(nnz)
    with Ctx(dims, idx, v, U0, FP64, chunk=32) as c:
        for n in range(3):
            assert rel(c.ttmctc(n), orc.ttmctc(dims, idx, v, U0, n)) <= 1e-11


def test_large_mode_sizes(orc):
    """Indices near the int32 range of the mode sizes."""
    dims, ranks = (3_000_000, 5, 2_000_000), (2, 2, 2)
    rng = np.random.default_rng(12)
    nnz = 3000
    idx = [rng.integers(0, d, nnz).astype(np.int32) for d in dims]
    idx[0][:5] = dims[0] - 1
    idx[2][:5] = dims[2] - 1
    v = rng.random(nnz)
    U0 = [np.linalg.qr(rng.standard_normal((d, k)))[0] for d, k in zip(dims, ranks)]
    with Ctx(dims, idx, v, U0, FP64) as c:
        for n in range(3):
            A = c.ttmctc(n)
            rows = np.unique(idx[n])[:50].astype(np.int32)
            assert rel(A[rows], orc.ttmctc_rows(dims, idx, v, U0, n, rows)) <= 1e-11


def test_host_inputs_equal_device_inputs():
    X, U0 = _case((80, 70, 60), (4, 4, 4), 5000, 13)
    with Ctx(X.dims, X.idx, X.vals, U0, FP64) as a, Ctx(X.dims, X.idx, X.vals, U0, FP64, host_inputs=True) as b:
        for n in range(3):
            np.testing.assert_array_equal(a.ttmctc(n), b.ttmctc(n))


def test_bitwise_deterministic():
    X, U0 = _case((400, 300, 200), (8, 8, 8), 50_000, 14, dist="zipf")
    out = []
    for _ in range(2):
        with Ctx(X.dims, X.idx, X.vals.astype(np.float32), [u.astype(np.float32) for u in U0], FP32) as c:
            h = c.iterate(2)
            out.append((h, c.factor(0), c.core()))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    np.testing.assert_array_equal(out[0][2], out[1][2])


def test_invalid_index_is_rejected():
    dims = (10, 10, 10)
    idx = [np.array([1, 2], dtype=np.int32), np.array([3, 10], dtype=np.int32), np.array([0, 0], dtype=np.int32)]
    U0 = inputs.orthonormal_factors(dims, (2, 2, 2), 1)
    with pytest.raises(hoqri.HoqriError) as ei:
        Ctx(dims, idx, np.ones(2), U0, FP64)
    assert ei.value.code == hoqri.HOQRI_ERR_INVALID


def test_warp_ranges_with_carry_match_oracle(orc):
    """1.5M Zipf nonzeros: several work items per warp range, long rows carried across
    items and completed across ranges; sampled rows of A_n and all of G vs the oracle."""
    X = inputs.random_sparse((20_000, 10_000, 5_000), 1_500_000, 31, dist="zipf", s=1.1, values="lognormal",
                             dtype=np.float32, distinct=True)
    U0 = [u.astype(np.float32) for u in inputs.orthonormal_factors(X.dims, (16, 16, 16), 32)]
    U0o = [u.astype(np.float64) for u in U0]
    vo = X.vals.astype(np.float64)
    with Ctx(X.dims, X.idx, X.vals, U0, FP32) as c:
        for n in range(3):
            A = c.ttmctc(n)
            cnt = np.bincount(X.idx[n], minlength=X.dims[n])
            heavy = np.argsort(cnt)[-8:]
            rng = np.random.default_rng(n)
            rows = np.unique(np.concatenate([heavy, rng.choice(np.flatnonzero(cnt), 24, replace=False)]))
            ref, G_ref = orc.ttmctc_rows(X.dims, X.idx, vo, U0o, n, rows.astype(np.int32), return_core=True)
            assert rel(A[rows], ref) <= 1e-5
        assert rel(c.core(), G_ref) <= 1e-5
