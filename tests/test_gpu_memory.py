"""Contexts on a created stream allocate from the library's retaining memory
pool: creating and destroying contexts one after another (with and without
hoqri_trim_memory in between, which hands the reserved memory back) gives
bit-identical results, and a context built from reused pool memory matches the
oracle."""
import numpy as np
import pytest

from paper_2510_16930_gb300 import hoqri, inputs
from tests.gpu_util import Ctx, rel

pytestmark = pytest.mark.gpu


def test_pool_reuse_and_trim_keep_results(orc):
    torch = pytest.importorskip("torch")
    dims, ranks = (3000, 2000, 1000), (16, 16, 8)
    X = inputs.random_sparse(dims, 200_000, 91, dist="zipf", s=1.1, values="lognormal", dtype=np.float32,
                             distinct=True)
    U0 = [u.astype(np.float32) for u in inputs.orthonormal_factors(dims, ranks, 92)]
    st = torch.cuda.Stream()
    hist = []
    for k in range(3):
        if k == 2:
            hoqri.hoqri_trim_memory()
        with torch.cuda.stream(st):
            c = Ctx(dims, X.idx, X.vals, U0, hoqri.HOQRI_FP32, stream=st.cuda_stream)
            try:
                if k == 0:
                    A = c.ttmctc(1)
                    U0o = [u.astype(np.float64) for u in U0]
                    A_ref = orc.ttmctc(dims, X.idx, X.vals.astype(np.float64), U0o, 1)
                    assert rel(A, A_ref) <= 1e-5
                hist.append(c.iterate(4))
            finally:
                c.close()
        st.synchronize()
    assert np.array_equal(hist[0], hist[1]) and np.array_equal(hist[0], hist[2])
    hoqri.hoqri_trim_memory()
