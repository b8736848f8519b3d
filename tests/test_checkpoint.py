"""Checkpoint and resume: the file round trip (CPU) and resumed sweeps equal to
the original context's, bit for bit (GPU)."""
import numpy as np
import pytest

from paper_2510_16930_gb300 import checkpoint, hoqri, inputs

FP64, FP32 = hoqri.HOQRI_FP64, hoqri.HOQRI_FP32


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_round_trip(tmp_path, dt):
    rng = np.random.default_rng(3)
    dims, ranks = (20, 15, 9, 7), (4, 3, 2, 2)
    U = [rng.standard_normal((I, K)).astype(dt) for I, K in zip(dims, ranks)]
    p = tmp_path / "ck.npz"
    prec = FP64 if dt == np.float64 else FP32
    opt = hoqri.hoqri_default_options(qr_kind=2, chunk_nnz=96, autotune=1, one_stream=3, tol=1e-9)
    checkpoint.save(p, U, dims=dims, ranks=ranks, prec=prec, sweeps=7, resid_hist=[0.9, 0.8], seed=11, options=opt)
    ck = checkpoint.load(p)
    assert ck["dims"] == list(dims) and ck["ranks"] == list(ranks)
    assert ck["prec"] == prec and ck["sweeps"] == 7 and ck["seed"] == 11
    o = ck["options"]
    assert (o["prec"], o["qr_kind"], o["chunk_nnz"], o["autotune"], o["one_stream"], o["seed"]) == (prec, 2, 96, 1, 3, 11)
    assert o["tol"] == 1e-9 and o["use_graphs"] == opt.use_graphs
    assert np.array_equal(ck["resid_hist"], [0.9, 0.8])
    for a, b in zip(U, ck["U"]):
        assert a.dtype == b.dtype and np.array_equal(a, b)


def test_rejects_bad_shapes_and_formats(tmp_path):
    U = [np.zeros((5, 2)), np.zeros((4, 2))]
    with pytest.raises(ValueError):
        checkpoint.save(tmp_path / "a.npz", U, dims=(5, 3), ranks=(2, 2), prec=FP64, sweeps=0)
    p = tmp_path / "b.npz"
    checkpoint.save(p, U, dims=(5, 4), ranks=(2, 2), prec=FP64, sweeps=0)
    z = dict(np.load(p))
    z["format"] = np.int64(checkpoint.FORMAT + 1)
    np.savez(tmp_path / "c.npz", **z)
    with pytest.raises(ValueError):
        checkpoint.load(tmp_path / "c.npz")
    z = dict(np.load(p))
    z["U1"] = np.zeros((4, 3))
    np.savez(tmp_path / "d.npz", **z)
    with pytest.raises(ValueError):
        checkpoint.load(tmp_path / "d.npz")


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_resume_equals_uninterrupted(tmp_path, prec):
    """Two sweeps, checkpoint, a new context from the file, three sweeps: the
    residuals and factors equal those of the original context's next call of
    three sweeps, bit for bit."""
    import torch
    from tests.gpu_util import Ctx

    dims, ranks, nnz = (300, 100, 50), (16, 16, 16), 20_000
    npdt = np.float64 if prec == FP64 else np.float32
    X = inputs.random_sparse(dims, nnz, 101, dist="zipf", s=1.1, values="lognormal", dtype=npdt)
    U0 = [u.astype(npdt) for u in inputs.orthonormal_factors(dims, ranks, 102)]
    with Ctx(dims, X.idx, X.vals, U0, prec) as a:
        a.iterate(2)
        h_ref = a.iterate(3)
        U_ref = [a.factor(n) for n in range(3)]
    with Ctx(dims, X.idx, X.vals, U0, prec) as b:
        h1 = b.iterate(2)
        F = checkpoint.capture(b.h, dims, ranks, prec)
    p = tmp_path / "ck.npz"
    checkpoint.save(p, F, dims=dims, ranks=ranks, prec=prec, sweeps=2, resid_hist=h1)
    ck = checkpoint.load(p)
    idx_d = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda() for a in X.idx]
    vals_d = torch.from_numpy(np.ascontiguousarray(X.vals)).cuda()
    h = checkpoint.resume(ck, idx_d, vals_d)
    try:
        h_res = hoqri.hoqri_iterate(h, 3)
        U_res = checkpoint.capture(h, dims, ranks, prec)
    finally:
        hoqri.hoqri_destroy(h)
    assert np.array_equal(h_res, h_ref)
    for a, b in zip(U_res, U_ref):
        assert np.array_equal(a.astype(np.float64), b)
