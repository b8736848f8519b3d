"""Sweeps replayed from one captured CUDA graph (use_graphs) give bit-identical
results to plain launches: same kernels, same order, same reductions.  Capture
needs a stream other than the legacy default stream."""
import numpy as np
import pytest

from paper_2510_16930_gb300 import hoqri, inputs
from tests.gpu_util import Ctx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [hoqri.HOQRI_FP64, hoqri.HOQRI_FP32, hoqri.HOQRI_BF16X3])
@pytest.mark.parametrize("dims,ranks,nnz", [
    ((2000, 1000, 500), (16, 16, 16), 200_000),
    ((200, 100, 100, 40), (8, 8, 8, 8), 100_000),
    ((300, 200, 100), (5, 4, 3), 20_000),
])
def test_graph_replay_equals_plain_launches(prec, dims, ranks, nnz):
    torch = pytest.importorskip("torch")
    X = inputs.random_sparse(dims, nnz, 61, dist="zipf", s=1.1, values="lognormal", dtype=np.float64)
    U0 = inputs.orthonormal_factors(dims, ranks, 62)
    dt = np.float64 if prec == hoqri.HOQRI_FP64 else np.float32
    out = []
    for graphs in (0, 1):
        st = torch.cuda.Stream()
        with Ctx(dims, X.idx, X.vals.astype(dt), [u.astype(dt) for u in U0], prec, stream=st.cuda_stream,
                 use_graphs=graphs) as c:
            # the history array grows between calls, so the graph is captured again
            h = np.concatenate([c.iterate(2), c.iterate(5), c.iterate(1)])
            _, launches = hoqri.hoqri_profile_read(c.h)
            out.append((h, [c.factor(n) for n in range(len(dims))], c.core(), launches))
    assert np.array_equal(out[0][0], out[1][0])
    for a, b in zip(out[0][1], out[1][1]):
        assert np.array_equal(a, b)
    assert np.array_equal(out[0][2], out[1][2])
    # replayed sweeps count their kernels like plain launches, plus the history append
    assert out[1][3] == out[0][3] + 8
