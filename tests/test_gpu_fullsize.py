"""Parity at the benchmark's full size, in the launch configuration bench.py times.

The oracle cannot run the whole trajectory at 5e7 nonzeros, so the checks are
(i) core entries G(k) computed one by one by the oracle at sampled k,
(ii) Eq. (AU), A_n^T U_n = G_(n) G_(n)^T, from device outputs alone,
(iii) sampled rows of A_n, long rows included, by the element-wise TTMcTC of
Alg. 3 in the oracle given the library's core (itself checked entry by entry
in (i); the oracle's own core costs O(nnz P N) and is too slow at this size),
(iv) the FP32 and split-BF16 paths' residual histories over the
configuration's 20 sweeps against the FP64 path of the same library (which the
small-size tests pin to the oracle at 1e-10).
"""
import numpy as np
import pytest

from paper_2510_16930_gb300 import hoqri, inputs
from tests import dense_ref as D
from tests.gpu_util import Ctx, rel

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def c2():
    return inputs.make_config("c2")


def test_full_c2_core_entries_and_AU(orc, c2):
    X, U0, cfg = c2
    U0f = [u.astype(np.float32) for u in U0]
    with Ctx(X.dims, X.idx, X.vals, U0f, hoqri.HOQRI_FP32) as c:
        G = c.core()
        rng = np.random.default_rng(7)
        lin = np.sort(rng.choice(G.size, size=16, replace=False)).astype(np.int64)
        ref = orc.core_entries(X.idx, X.vals.astype(np.float64), [u.astype(np.float64) for u in U0f], lin)
        got = G.ravel()[lin]
        assert np.max(np.abs(got - ref)) <= 1e-5 * np.abs(G).max()
        for n in range(3):
            A = c.ttmctc(n)
            Gn = D.unfold(c.core(), n)
            assert rel(A.T @ U0f[n].astype(np.float64), Gn @ Gn.T) <= 1e-5


def test_full_c2_rows_of_A_match_the_oracle(orc, c2):
    X, U0, cfg = c2
    U0f = [u.astype(np.float32) for u in U0]
    U0o = [u.astype(np.float64) for u in U0f]
    vo = X.vals.astype(np.float64)
    with Ctx(X.dims, X.idx, X.vals, U0f, hoqri.HOQRI_FP32) as c:
        G = c.core()
        for n in (0, 2):
            A = c.ttmctc(n)
            cnt = np.bincount(X.idx[n], minlength=X.dims[n])
            nz = np.flatnonzero(cnt)
            order = nz[np.argsort(cnt[nz], kind="stable")]
            rng = np.random.default_rng(n)
            # long rows (the 99.9th percentile of row length) and random rows
            q = int(0.999 * (len(order) - 1))
            rows = np.unique(np.concatenate([order[q - 4:q], rng.choice(nz, 8, replace=False)])).astype(np.int32)
            ref = orc.ttmctc_rows_with_core(X.dims, X.idx, vo, U0o, n, rows, G)
            assert rel(A[rows], ref) <= 1e-5, (n, rel(A[rows], ref))


def test_full_c2_fp32_trajectory_tracks_fp64(c2):
    X, U0, cfg = c2
    iters = int(cfg["iters"])
    with Ctx(X.dims, X.idx, X.vals.astype(np.float64), U0, hoqri.HOQRI_FP64) as c:
        h64 = c.iterate(iters)
    with Ctx(X.dims, X.idx, X.vals, [u.astype(np.float32) for u in U0], hoqri.HOQRI_FP32) as c:
        h32 = c.iterate(iters)
    assert np.max(np.abs(h32 - h64) / h64) <= 1e-6


def test_full_c2_mixed_trajectory_tracks_fp64(c2):
    """The split-BF16 tensor-core path at the full size: final-fit relative error
    against the FP64 path within 1e-6 (the accuracy target of the mixed form)."""
    X, U0, cfg = c2
    iters = int(cfg["iters"])
    with Ctx(X.dims, X.idx, X.vals.astype(np.float64), U0, hoqri.HOQRI_FP64) as c:
        h64 = c.iterate(iters)
    with Ctx(X.dims, X.idx, X.vals, [u.astype(np.float32) for u in U0], hoqri.HOQRI_BF16X3) as c:
        hmix = c.iterate(iters)
    assert np.max(np.abs(hmix - h64) / h64) <= 1e-6
