"""hoqri_orthonormalize_noalloc (scratch in a static device array, no context,
no allocation) through the C ABI, against hoqri_orthonormalize of a context on
the same input: the QR step of Alg. 2, thin QR with diag(R) > 0.

Kept in a file of its own, collected last, so that it runs both after every
other GPU test (the static scratch has been used before) and alone.
"""
import numpy as np
import pytest

from paper_2510_16930_gb300 import hoqri, inputs
from tests.gpu_util import TOL, Ctx, rel

pytestmark = pytest.mark.gpu


def _context_result(A, prec):
    """U from hoqri_orthonormalize of a small context whose mode 0 is I x K."""
    I, K = A.shape
    dims = (I, K + 1, K + 2)
    X = inputs.random_sparse(dims, 64, seed=11)
    U0 = inputs.orthonormal_factors(dims, (K, K, K), seed=12)
    if prec == hoqri.HOQRI_FP32:
        U0 = [u.astype(np.float32) for u in U0]
    with Ctx(X.dims, X.idx, X.vals, U0, prec) as c:
        return c.orthonormalize(0, A)


def _noalloc(torch, A, prec, in_place=False):
    dt = torch.float64 if prec == hoqri.HOQRI_FP64 else torch.float32
    Ad = torch.from_numpy(np.ascontiguousarray(A)).to(dt).cuda()
    U = Ad if in_place else torch.empty_like(Ad)
    hoqri.hoqri_orthonormalize_noalloc(prec, A.shape[0], A.shape[1], Ad, U)
    torch.cuda.synchronize()
    return U.cpu().double().numpy(), Ad.cpu().double().numpy()


@pytest.mark.parametrize("prec", [hoqri.HOQRI_FP64, hoqri.HOQRI_FP32])
@pytest.mark.parametrize("I,K", [(40, 32), (1000, 16), (5001, 7), (300007, 16)])
def test_noalloc_matches_orthonormalize_two_calls(prec, I, K):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1000 * I + K)
    A = rng.standard_normal((I, K))
    if prec == hoqri.HOQRI_FP32:
        A = A.astype(np.float32)
    ref = _context_result(A, prec)
    U1, A1 = _noalloc(torch, A, prec)
    U2, _ = _noalloc(torch, A, prec)
    tol = TOL[prec]
    assert rel(U1, ref) <= tol
    assert rel(U2, ref) <= tol
    assert np.array_equal(U1, U2)  # same input, same fixed reduction order
    assert np.array_equal(A1, A.astype(np.float64))  # A_in is read only
    # orthonormal columns and diag(R) = diag(U^T A) > 0
    assert np.abs(U1.T @ U1 - np.eye(K)).max() <= (1e-12 if prec == hoqri.HOQRI_FP64 else 1e-5)
    assert np.all(np.diag(U1.T @ A.astype(np.float64)) > 0)


@pytest.mark.parametrize("prec", [hoqri.HOQRI_FP64, hoqri.HOQRI_FP32])
def test_noalloc_in_place_equals_out_of_place(prec):
    torch = pytest.importorskip("torch")
    A = np.random.default_rng(5).standard_normal((2048, 16))
    if prec == hoqri.HOQRI_FP32:
        A = A.astype(np.float32)
    U_out, _ = _noalloc(torch, A, prec)
    U_in, _ = _noalloc(torch, A, prec, in_place=True)
    assert np.array_equal(U_out, U_in)


def test_noalloc_breakdown_then_recovers():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    A = rng.standard_normal((500, 8))
    A[:, 5] = A[:, 2]  # rank deficient: CholeskyQR2 has no valid pivot
    with pytest.raises(hoqri.HoqriError) as e:
        _noalloc(torch, A, hoqri.HOQRI_FP64)
    assert e.value.code == hoqri.HOQRI_ERR_QR_BREAKDOWN
    # the next call starts from zeroed flags
    B = rng.standard_normal((500, 8))
    U, _ = _noalloc(torch, B, hoqri.HOQRI_FP64)
    assert rel(U, _context_result(B, hoqri.HOQRI_FP64)) <= TOL[hoqri.HOQRI_FP64]


@pytest.mark.parametrize("prec", [hoqri.HOQRI_FP64, hoqri.HOQRI_FP32])
def test_noalloc_ill_conditioned_takes_the_shifted_pass(prec):
    """Columns scaled over 7.5 decades: unshifted CholeskyQR2 breaks down, the
    shifted first pass does not; same U as the context's QR on the same input."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(17)
    A = rng.standard_normal((4000, 16)) * np.logspace(0, -7.5, 16)[None, :]
    if prec == hoqri.HOQRI_FP32:
        A = A.astype(np.float32)
    U, _ = _noalloc(torch, A, prec)
    assert np.linalg.norm(U.T @ U - np.eye(16)) <= (1e-13 if prec == hoqri.HOQRI_FP64 else 1e-5)
    assert rel(U, _context_result(A, prec)) <= TOL[prec]


def test_noalloc_rejects_oversize_and_host_buffers():
    torch = pytest.importorskip("torch")
    A = torch.zeros((100, 33), dtype=torch.float64, device="cuda")
    with pytest.raises(hoqri.HoqriError) as e:
        hoqri.hoqri_orthonormalize_noalloc(hoqri.HOQRI_FP64, 100, 33, A, A)
    assert e.value.code == hoqri.HOQRI_ERR_INVALID and "32" in str(e.value)
    h = np.zeros((100, 16))
    with pytest.raises(hoqri.HoqriError) as e:
        hoqri.hoqri_orthonormalize_noalloc(hoqri.HOQRI_FP64, 100, 16, h, h)
    assert e.value.code == hoqri.HOQRI_ERR_INVALID
    B = torch.zeros((100, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(hoqri.HoqriError) as e:  # overlapping but not equal
        hoqri.hoqri_orthonormalize_noalloc(hoqri.HOQRI_FP64, 99, 16, B, B[1:])
    assert e.value.code == hoqri.HOQRI_ERR_INVALID
