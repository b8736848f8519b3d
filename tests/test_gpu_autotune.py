"""The autotuner (opt.autotune) times candidate lane tiles and layouts of the
nonzero-stream pass at create and keeps the fastest: results stay within the
FP32 tolerance of the oracle whatever it picks, the choice is readable through
hoqri_layout, every tile the tuner may pick computes the same A_n, and the
choices are cached (in memory and in HOQRI_TUNE_CACHE)."""
import os

import numpy as np
import pytest

from paper_2510_16930_gb300 import hoqri, inputs
from tests.gpu_util import Ctx, rel

pytestmark = pytest.mark.gpu


def test_autotuned_layout_matches_oracle_and_is_cached(orc, tmp_path):
    cache = tmp_path / "tune.txt"
    os.environ["HOQRI_TUNE_CACHE"] = str(cache)
    X = inputs.random_sparse((5_000, 3_000, 2_000), 300_000, 71, dist="zipf", s=1.1, values="lognormal",
                             dtype=np.float32, distinct=True)
    U0 = [u.astype(np.float32) for u in inputs.orthonormal_factors(X.dims, (16, 16, 16), 72)]
    U0o = [u.astype(np.float64) for u in U0]
    vo = X.vals.astype(np.float64)
    with Ctx(X.dims, X.idx, X.vals, U0, hoqri.HOQRI_FP32, autotune=1) as c:
        for n in range(3):
            ls, T, TL, TV = hoqri.hoqri_layout(c.h, n)
            assert ls > 0 and T > 0 and (TL, TV) in ((8, 8), (8, 4), (4, 8))
            A = c.ttmctc(n)
            cnt = np.bincount(X.idx[n], minlength=X.dims[n])
            rows = np.unique(np.concatenate([np.argsort(cnt)[-6:], np.flatnonzero(cnt)[:10]])).astype(np.int32)
            ref, G_ref = orc.ttmctc_rows(X.dims, X.idx, vo, U0o, n, rows, return_core=True)
            assert rel(A[rows], ref) <= 1e-5
        assert rel(c.core(), G_ref) <= 1e-5
        h1 = c.iterate(3)
    lines = cache.read_text().splitlines()
    assert len(lines) == 3 and all(len(l.split()) == 5 for l in lines)
    # a second context of the same kind takes the cached choice: no new timing lines
    with Ctx(X.dims, X.idx, X.vals, U0, hoqri.HOQRI_FP32, autotune=1) as c:
        h2 = c.iterate(3)
    assert cache.read_text().splitlines() == lines
    assert np.array_equal(h1, h2)  # same layout, same arithmetic


@pytest.mark.parametrize("tile", [(8, 4), (4, 8), (8, 8)])
def test_every_tuner_tile_matches_oracle(orc, tile):
    """Each lane tile the tuner may choose (forced through tile_rows/tile_cols),
    orders 3 and 4, against the oracle's Alg. 3; the layout reports the tile."""
    for dims, ranks, nnz in (((3000, 2000, 1000), (16, 16, 16), 200_000),
                             ((300, 200, 100, 60), (8, 8, 8, 8), 150_000)):
        X = inputs.random_sparse(dims, nnz, 81, dist="zipf", s=1.1, values="lognormal", dtype=np.float32,
                                 distinct=True)
        U0 = [u.astype(np.float32) for u in inputs.orthonormal_factors(dims, ranks, 82)]
        U0o = [u.astype(np.float64) for u in U0]
        vo = X.vals.astype(np.float64)
        with Ctx(dims, X.idx, X.vals, U0, hoqri.HOQRI_FP32, tile_rows=tile[0], tile_cols=tile[1]) as c:
            for n in range(len(dims)):
                assert hoqri.hoqri_layout(c.h, n)[2:] == tile
                A_ref, G_ref = orc.ttmctc(dims, X.idx, vo, U0o, n, return_core=True)
                A = c.ttmctc(n)
                assert rel(A, A_ref) <= 1e-5, (n, rel(A, A_ref))
            assert rel(c.core(), G_ref) <= 1e-5
