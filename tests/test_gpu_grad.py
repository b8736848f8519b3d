"""The Riemannian-gradient diagnostic (Sec. 5, Eq. grad2) and the stopping rule
of Sec. 6.1 through the C ABI, against the FP64 oracle.

hoqri_grad_norm2 forms each mode's term row by row in FP64 from the path's
A_n, U_n and core, so its error is that of A_n and G: 1e-9 relative for the
FP64 path, 1e-4 for the FP32 path (A_n and G at 1e-5, and the gradient is a
difference of terms of the size of A_n).
"""
import math

import numpy as np
import pytest

from paper_2510_16930_gb300 import hoqri, inputs
from tests.gpu_util import Ctx

pytestmark = pytest.mark.gpu

FP64, FP32 = hoqri.HOQRI_FP64, hoqri.HOQRI_FP32

SHAPES = [
    ((40, 30, 20), (5, 4, 3), 3000, "uniform"),
    ((300, 100, 50), (16, 16, 16), 20_000, "zipf"),
    ((30, 20, 20, 10), (4, 4, 4, 4), 5000, "zipf"),
]


def _case(dims, ranks, nnz, dist, seed):
    X = inputs.random_sparse(dims, nnz, seed, dist=dist, s=1.1, values="uniform", dtype=np.float64)
    U0 = inputs.orthonormal_factors(dims, ranks, seed + 1)
    return X, U0


def _npv(X, prec):
    return X.vals.astype(np.float64 if prec == FP64 else np.float32)


def _Ucast(U, prec):
    return [u.astype(np.float64 if prec == FP64 else np.float32) for u in U]


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("shape", SHAPES, ids=[f"{s[0]}-{s[1]}" for s in SHAPES])
def test_grad_norm2_matches_oracle(orc, shape, prec):
    dims, ranks, nnz, dist = shape
    X, U0 = _case(dims, ranks, nnz, dist, 60 + nnz)
    U0p = _Ucast(U0, prec)
    with Ctx(dims, X.idx, _npv(X, prec), U0p, prec) as c:
        g = hoqri.hoqri_grad_norm2(c.h)
    ref = orc.grad_norm2(dims, X.idx, _npv(X, prec).astype(np.float64), [u.astype(np.float64) for u in U0p])
    assert abs(g - ref) <= (1e-9 if prec == FP64 else 1e-4) * ref


def test_grad_norm2_at_the_library_factors_after_sweeps(orc):
    """After three sweeps: the oracle's gradient at the factors the library
    holds, and the gradient has decreased."""
    dims, ranks, nnz, dist = SHAPES[1]
    X, U0 = _case(dims, ranks, nnz, dist, 71)
    with Ctx(dims, X.idx, X.vals, U0, FP64) as c:
        g0 = hoqri.hoqri_grad_norm2(c.h)
        c.iterate(3)
        g3 = hoqri.hoqri_grad_norm2(c.h)
        U3 = [c.factor(n) for n in range(3)]
    ref = orc.grad_norm2(dims, X.idx, X.vals, U3)
    assert abs(g3 - ref) <= 1e-8 * ref
    assert g3 < g0


def _r0(X, U0, prec):
    """Residual of the core of the initial factors, as the library computes it."""
    with Ctx(X.dims, X.idx, _npv(X, prec), _Ucast(U0, prec), prec) as c:
        c.iterate(0)
        r, _, _ = hoqri.hoqri_fit(c.h)
    return r


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_run_stops_at_the_first_small_change(prec):
    dims, ranks, nnz, dist = SHAPES[1]
    X, U0 = _case(dims, ranks, nnz, dist, 72)
    tol, cap = 1e-4, 60
    with Ctx(dims, X.idx, _npv(X, prec), _Ucast(U0, prec), prec, tol=tol) as c:
        h = hoqri.hoqri_run(c.h, cap)
    assert 1 <= len(h) <= cap
    d = np.abs(np.diff(np.concatenate([[_r0(X, U0, prec)], h])))
    assert np.all(d[:-1] >= tol)
    assert d[-1] < tol or len(h) == cap
    # the sweeps that ran are those of hoqri_iterate with that count
    with Ctx(dims, X.idx, _npv(X, prec), _Ucast(U0, prec), prec) as c:
        hi = c.iterate(len(h))
    assert np.array_equal(h, hi)


def test_run_without_tolerance_runs_every_sweep():
    dims, ranks, nnz, dist = SHAPES[0]
    X, U0 = _case(dims, ranks, nnz, dist, 73)
    with Ctx(dims, X.idx, X.vals, U0, FP64) as c:
        h = hoqri.hoqri_run(c.h, 4)
    with Ctx(dims, X.idx, X.vals, U0, FP64) as c:
        hi = c.iterate(4)
    assert len(h) == 4 and np.array_equal(h, hi)
    assert all(math.isfinite(v) for v in h)
