"""HOSVD initialisation (hoqri_init_hosvd: orthogonal iteration on
X_(n) X_(n)^T from the sparse entries) against the oracle's HOSVD, the leading
left singular subspaces of the dense unfoldings by LAPACK's SVD.

Subspaces are compared through projectors (the basis is not unique).  After q
steps the error of orthogonal iteration falls like rho^(2q), rho =
sigma_{K+1} / sigma_K of the unfolding; the bound below allows a start-
dependent constant of 1e3 on top of that, plus the rounding of the path
(FP64 1e-9, FP32 1e-4).
"""
import numpy as np
import pytest

from paper_2510_16930_gb300 import hoqri, inputs
from tests import dense_ref as D
from tests.gpu_util import Ctx

pytestmark = pytest.mark.gpu

FP64, FP32 = hoqri.HOQRI_FP64, hoqri.HOQRI_FP32
ROUND = {FP64: 1e-9, FP32: 1e-4}


def _factors(c, N):
    return [c.factor(n) for n in range(N)]


def _exact_low_rank(dims, ranks, seed):
    rng = np.random.default_rng(seed)
    Ut = [np.linalg.qr(rng.standard_normal((I, K)))[0] for I, K in zip(dims, ranks)]
    Xd = D.reconstruct(rng.standard_normal(ranks) * 2.0, Ut)
    grid = np.meshgrid(*[np.arange(I) for I in dims], indexing="ij")
    return [g.ravel().astype(np.int32) for g in grid], Xd.ravel(), Ut


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_hosvd_of_exact_low_rank_tensor(orc, prec):
    """Unfoldings of exact rank K_n: one step already spans the planted
    subspaces; the residual of the core at those factors is zero."""
    dims, ranks = (30, 25, 20), (3, 3, 2)
    idx, vals, Ut = _exact_low_rank(dims, ranks, 80)
    U0 = inputs.orthonormal_factors(dims, ranks, 81)
    npdt = np.float64 if prec == FP64 else np.float32
    with Ctx(dims, idx, vals.astype(npdt), [u.astype(npdt) for u in U0], prec, seed=5) as c:
        hoqri.hoqri_init_hosvd(c.h, 2)
        U = _factors(c, 3)
        c.iterate(0)
        r, _, _ = hoqri.hoqri_fit(c.h)
    Uo = orc.hosvd(dims, idx, vals, ranks)
    for u, uo, ut, K in zip(U, Uo, Ut, ranks):
        assert np.linalg.norm(u.T @ u - np.eye(K)) <= (1e-12 if prec == FP64 else 1e-5)
        assert D.proj_dist(u, uo) <= ROUND[prec]
        assert D.proj_dist(u, ut) <= ROUND[prec]
    assert r <= (1e-6 if prec == FP64 else 2e-3)


def _sparse_gapped(dims, R, supp, noise_n, seed):
    """R sparse rank-1 terms (random supports of the given sizes, weights 5, 4,
    ...) plus noise_n random entries of size 0.01: every unfolding has a clear
    gap after its R-th singular value (sigma_{R+1} / sigma_R about 1e-3)."""
    rng = np.random.default_rng(seed)
    idx, vals = [[] for _ in dims], []
    for r in range(R):
        S = [np.sort(rng.choice(I, k, replace=False)) for I, k in zip(dims, supp)]
        f = [rng.standard_normal(k) for k in supp]
        prod = f[0]
        for m in range(1, len(dims)):
            prod = np.multiply.outer(prod, f[m])
        for m, g in enumerate(np.meshgrid(*S, indexing="ij")):
            idx[m].append(g.ravel())
        vals.append((5.0 - r) * prod.ravel())
    for m, I in enumerate(dims):
        idx[m].append(rng.integers(0, I, noise_n))
    vals.append(0.01 * rng.standard_normal(noise_n))
    return [np.concatenate(a).astype(np.int32) for a in idx], np.concatenate(vals)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("shape", [
    ((60, 50, 40), 4, (20, 15, 10)),
    ((40, 30, 20, 10), 3, (10, 8, 6, 4)),
], ids=["3way", "4way"])
def test_hosvd_of_sparse_tensor_matches_dense_svd(orc, prec, shape):
    dims, R, supp = shape
    idx, vals = _sparse_gapped(dims, R, supp, 2000, 84)
    ranks = (R,) * len(dims)
    U0 = inputs.orthonormal_factors(dims, ranks, 85)
    q = 4
    npdt = np.float64 if prec == FP64 else np.float32
    with Ctx(dims, idx, vals.astype(npdt), [u.astype(npdt) for u in U0], prec, seed=7) as c:
        hoqri.hoqri_init_hosvd(c.h, q)
        U = _factors(c, len(dims))
    v = vals.astype(npdt).astype(np.float64)
    Uo = orc.hosvd(dims, idx, v, ranks)
    Xd = D.dense(dims, idx, v)
    for n in range(len(dims)):
        s = np.linalg.svd(D.unfold(Xd, n), compute_uv=False)
        rho = s[R] / s[R - 1]
        assert rho < 0.01
        assert D.proj_dist(U[n], Uo[n]) <= 1e3 * rho ** (2 * q) + ROUND[prec], n


def test_hosvd_is_deterministic_and_seeded(orc):
    dims, ranks, nnz = (60, 50, 40), (4, 4, 3), 4000
    X = inputs.random_sparse(dims, nnz, 90, dist="zipf", s=1.1, values="lognormal", dtype=np.float64)
    U0 = inputs.orthonormal_factors(dims, ranks, 91)
    out = []
    for seed in (3, 3, 4):
        with Ctx(dims, X.idx, X.vals, U0, FP64, seed=seed) as c:
            hoqri.hoqri_init_hosvd(c.h, 3)
            out.append(_factors(c, 3))
    assert all(np.array_equal(a, b) for a, b in zip(out[0], out[1]))
    assert any(not np.array_equal(a, b) for a, b in zip(out[0], out[2]))


def test_hosvd_then_iterate_runs():
    dims, ranks, nnz = (300, 100, 50), (16, 16, 16), 20_000
    X = inputs.random_sparse(dims, nnz, 92, dist="zipf", s=1.1, values="uniform", dtype=np.float32)
    U0 = [u.astype(np.float32) for u in inputs.orthonormal_factors(dims, ranks, 93)]
    with Ctx(dims, X.idx, X.vals, U0, FP32) as c:
        hoqri.hoqri_init_hosvd(c.h, 4)
        h = c.iterate(3)
    assert np.all(np.isfinite(h)) and np.all(np.diff(h) <= 1e-6)
