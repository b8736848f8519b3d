"""The fiber-factored nonzero-stream pass (FP32) against the oracle's Alg. 3.

The pass groups the nonzeros of a row of X_(n) that share their prefix indices
(a fiber) and forms y_i = sum_f z_f (x) w_f (Eq. ttmctc regrouped); long fibers
are cut into pieces, rows are cut across warp ranges and completed afterwards.
These cases push each of those on purpose: very long fibers and rows (a steep
Zipf law on few rows), a single row holding every nonzero, one nonzero, order
4 with every supported prefix split, and the three forms of the one-stream
option (fiber, sliced, O(IK)) on the same input.
"""
import numpy as np
import pytest

from paper_2510_16930_gb300 import hoqri, inputs
from tests.gpu_util import Ctx, rel

pytestmark = pytest.mark.gpu

FP32 = hoqri.HOQRI_FP32
TOL = 1e-5


def _run(orc, dims, ranks, X, one_stream=3, modes=None):
    U0 = [u.astype(np.float32) for u in inputs.orthonormal_factors(dims, ranks, 7)]
    U0o = [u.astype(np.float64) for u in U0]
    vals = X.vals.astype(np.float32)
    vo = vals.astype(np.float64)
    out = {}
    with Ctx(dims, X.idx, vals, U0, FP32, one_stream=one_stream) as c:
        for n in (modes if modes is not None else range(len(dims))):
            A_ref, G_ref = orc.ttmctc(dims, X.idx, vo, U0o, n, return_core=True)
            A = c.ttmctc(n)
            assert rel(A, A_ref) <= TOL, (n, rel(A, A_ref))
            out[n] = A
        G = c.core()
        assert rel(G, G_ref) <= TOL
    return out


def test_long_fibers_and_rows_cut_across_ranges(orc):
    # few rows, steep Zipf on the prefix mode: fibers of hundreds of nonzeros
    # (cut into pieces) and rows spanning many warp ranges
    dims, ranks = (24, 64, 3000), (16, 8, 16)
    X = inputs.random_sparse(dims, 300_000, 41, dist="zipf", s=1.6, values="lognormal", distinct=True)
    _run(orc, dims, ranks, X)


def test_one_row_holds_every_nonzero(orc):
    dims, ranks = (4, 300, 400), (4, 16, 16)
    X = inputs.random_sparse((1, 300, 400), 60_000, 5, values="uniform", distinct=True)
    idx = [np.full_like(X.idx[0], 2), X.idx[1], X.idx[2]]
    _run(orc, dims, ranks, inputs.SparseTensor(dims, idx, X.vals, dict(X.meta)))


def test_single_nonzero(orc):
    dims, ranks = (10, 12, 14), (4, 8, 4)
    X = inputs.random_sparse(dims, 1, 9, values="uniform")
    _run(orc, dims, ranks, X)


@pytest.mark.parametrize("ranks", [(8, 8, 8, 8), (4, 8, 4, 8), (4, 4, 16, 4), (8, 4, 4, 16)],
                         ids=lambda r: "x".join(map(str, r)))
def test_order4_prefix_splits(orc, ranks):
    dims = (40, 30, 25, 900)
    X = inputs.random_sparse(dims, 60_000, 13, dist="zipf", s=1.3, values="lognormal", distinct=True)
    _run(orc, dims, ranks, X)


def test_fiber_sliced_and_o_ik_forms_agree(orc):
    """The three forms of the pass compute the same A_n (each within the FP32
    bound of the oracle), and the fiber form is bitwise reproducible."""
    dims, ranks = (3000, 2000, 1000), (16, 16, 16)
    X = inputs.random_sparse(dims, 400_000, 21, dist="zipf", s=1.1, values="lognormal", distinct=True)
    a = _run(orc, dims, ranks, X, one_stream=3)
    b = _run(orc, dims, ranks, X, one_stream=0)
    cc = _run(orc, dims, ranks, X, one_stream=2)
    for n in range(3):
        assert rel(a[n], b[n]) <= 2 * TOL and rel(a[n], cc[n]) <= 2 * TOL
    again = _run(orc, dims, ranks, X, one_stream=3)
    for n in range(3):
        assert np.array_equal(a[n], again[n])
