"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks an oracle function against something other than itself: a
hand-derived worked example, dense brute force through numpy library routines
(np.kron / einsum / LAPACK), a second independent formula from the paper
(Alg. 3 vs Alg. 4), an identity the paper proves (Eq. AU, Thm. 1, the
interlacing lemma, the fit identity of Sec. 2.2), or a special case with a
textbook answer (N = 2 subspace iteration vs SVD; exact low multilinear rank).
"""
import math
import os

import numpy as np
import pytest

from paper_2510_16930_gb300 import inputs
from tests import dense_ref as D

HERE = os.path.dirname(os.path.abspath(__file__))


def _rand_coo(dims, nnz, seed, dup=True):
    rng = np.random.default_rng(seed)
    idx = [rng.integers(0, I, size=nnz).astype(np.int32) for I in dims]
    if dup and nnz > 4:  # force some repeated coordinates
        for a in idx:
            a[-3:] = a[:3]
    vals = rng.standard_normal(nnz)
    return idx, vals


def _rand_U(dims, ranks, seed, ortho=False):
    rng = np.random.default_rng(seed)
    U = [rng.standard_normal((I, K)) for I, K in zip(dims, ranks)]
    if ortho:
        U = [np.linalg.qr(u)[0] for u in U]
    return U


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# --------------------------------------------------------------- worked example

def _golden():
    d = {}
    with open(os.path.join(HERE, "golden", "tiny_2x2x2.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            d[k] = np.array([float(x) for x in v])
    return d


def test_golden_tiny_example(orc):
    g = _golden()
    dims = tuple(int(x) for x in g["dims"])
    idx = [g["i1"].astype(np.int32), g["i2"].astype(np.int32), g["i3"].astype(np.int32)]
    U = [g["U1"].reshape(2, 1), g["U2"].reshape(2, 1), g["U3"].reshape(2, 1)]
    G = orc.core(idx, g["x"], U)
    assert G.shape == (1, 1, 1)
    assert abs(G.ravel()[0] - g["G"][0]) < 1e-15
    for n, key in enumerate(("A1", "A2", "A3")):
        A = orc.ttmctc(dims, idx, g["x"], U, n)
        np.testing.assert_allclose(A.ravel(), g[key], rtol=0, atol=1e-14)
    Q, R, z = orc.qr(orc.ttmctc(dims, idx, g["x"], U, 0))
    np.testing.assert_allclose(Q.ravel(), g["U1_after_qr"], rtol=0, atol=1e-15)
    ci, cv = orc.coalesce(idx, g["x"])
    assert orc.norm2(cv) == g["normX2"][0]
    r0 = math.sqrt(g["normX2"][0] - G.ravel()[0] ** 2) / math.sqrt(g["normX2"][0])
    assert abs(r0 - g["resid_initial"][0]) < 1e-15


# -------------------------------------------------------- brute force, dense

@pytest.mark.parametrize("dims,ranks", [((5, 4, 6), (2, 3, 2)), ((4, 3, 5, 3), (2, 2, 3, 2)),
                                        ((6, 7), (3, 2)), ((3, 4, 3, 2, 3), (2, 2, 2, 2, 2))])
def test_core_equals_dense_einsum(orc, dims, ranks):
    idx, vals = _rand_coo(dims, 40, 1)
    U = _rand_U(dims, ranks, 2)  # not orthonormal: the definition does not need it
    G = orc.core(idx, vals, U)
    Gd = D.core_dense(D.dense(dims, idx, vals), U)
    assert _rel(G, Gd) < 1e-13


@pytest.mark.parametrize("dims,ranks", [((5, 4, 6), (2, 3, 2)), ((4, 3, 5, 3), (2, 2, 3, 2)),
                                        ((6, 7), (3, 2)), ((3, 4, 3, 2, 3), (2, 2, 2, 2, 2)),
                                        ((7, 5, 6), (3, 4, 2))])
def test_ttmctc_equals_dense_kronecker(orc, dims, ranks):
    """Alg. 3 == X_(n) (kron_{m != n} U_m) G_(n)^T built with np.kron (Eq. 2 + Eq. ttmctc)."""
    idx, vals = _rand_coo(dims, 50, 3)
    U = _rand_U(dims, ranks, 4)
    Xd = D.dense(dims, idx, vals)
    for n in range(len(dims)):
        A, G = orc.ttmctc(dims, idx, vals, U, n, return_core=True)
        assert _rel(A, D.ttmctc_dense(Xd, U, n)) < 1e-12
        assert _rel(G, D.core_dense(Xd, U)) < 1e-13


def test_ttmctc_rows_subset(orc):
    dims, ranks = (9, 6, 7), (3, 2, 3)
    idx, vals = _rand_coo(dims, 80, 5)
    U = _rand_U(dims, ranks, 6)
    for n in range(3):
        A = orc.ttmctc(dims, idx, vals, U, n)
        rows = np.array([dims[n] - 1, 0, 2], dtype=np.int32)
        Ar = orc.ttmctc_rows(dims, idx, vals, U, n, rows)
        np.testing.assert_array_equal(Ar, A[rows])


def test_core_entries_subset(orc):
    dims, ranks = (6, 5, 4), (3, 2, 4)
    idx, vals = _rand_coo(dims, 60, 7)
    U = _rand_U(dims, ranks, 8)
    G = orc.core(idx, vals, U).ravel()
    lin = np.array([0, 5, 23, 7], dtype=np.int64)
    np.testing.assert_array_equal(orc.core_entries(idx, vals, U, lin), G[lin])


def test_alg3_equals_alg4(orc):
    """The two TTMcTC forms of Sec. 3.2 (G first vs Y Y^T U first) agree."""
    for dims, ranks in [((8, 6, 7), (3, 2, 3)), ((5, 4, 4, 3), (2, 3, 2, 2))]:
        idx, vals = _rand_coo(dims, 70, 9)
        U = _rand_U(dims, ranks, 10)
        for n in range(len(dims)):
            A3 = orc.ttmctc(dims, idx, vals, U, n)
            A4 = orc.ttmctc_matrix(dims, idx, vals, U, n)
            assert _rel(A3, A4) < 1e-12


def test_AU_identity(orc):
    """Eq. (AU): A_n^T U_n = U_n^T A_n = G_(n) G_(n)^T."""
    dims, ranks = (9, 8, 7), (3, 3, 2)
    idx, vals = _rand_coo(dims, 90, 11)
    U = _rand_U(dims, ranks, 12, ortho=True)
    for n in range(3):
        A, G = orc.ttmctc(dims, idx, vals, U, n, return_core=True)
        Gn = D.unfold(G, n)
        lhs = A.T @ U[n]
        assert _rel(lhs, Gn @ Gn.T) < 1e-12
        assert _rel(U[n].T @ A, Gn @ Gn.T) < 1e-12


def test_rotation_equivariance(orc):
    """U_m -> U_m Q_m gives A_n -> A_n Q_n and G -> G x {Q^T} (rotational ambiguity, Sec. 2.2)."""
    dims, ranks = (7, 6, 5), (3, 2, 2)
    idx, vals = _rand_coo(dims, 60, 13)
    U = _rand_U(dims, ranks, 14, ortho=True)
    rng = np.random.default_rng(15)
    Q = [np.linalg.qr(rng.standard_normal((k, k)))[0] for k in ranks]
    UQ = [u @ q for u, q in zip(U, Q)]
    for n in range(3):
        A = orc.ttmctc(dims, idx, vals, U, n)
        AQ = orc.ttmctc(dims, idx, vals, UQ, n)
        assert _rel(AQ, A @ Q[n]) < 1e-12
    G = orc.core(idx, vals, U)
    GQ = orc.core(idx, vals, UQ)
    assert _rel(GQ, D.core_dense(G, Q)) < 1e-12


# ---------------------------------------------------------------------- coalescing

def test_coalesce_sums_repeats(orc):
    dims = (4, 5, 3)
    idx, vals = _rand_coo(dims, 60, 16)
    ci, cv = orc.coalesce(idx, vals)
    Xd = D.dense(dims, idx, vals)
    assert _rel(D.dense(dims, ci, cv), Xd) < 1e-15
    keys = np.ravel_multi_index(tuple(ci), dims)
    assert np.all(np.diff(keys) > 0)  # strictly increasing: distinct, lexicographic
    assert abs(orc.norm2(cv) - float((Xd ** 2).sum())) < 1e-12


def test_order_and_split_invariance(orc):
    dims, ranks = (6, 5, 7), (2, 3, 2)
    idx, vals = _rand_coo(dims, 50, 17, dup=False)
    U = _rand_U(dims, ranks, 18)
    A = [orc.ttmctc(dims, idx, vals, U, n) for n in range(3)]
    p = np.random.default_rng(19).permutation(len(vals))
    idx_p = [a[p] for a in idx]
    idx_s = [np.concatenate([a, a[:10]]) for a in idx]  # split first 10 values into two halves
    vals_s = np.concatenate([vals, vals[:10] * 0.25])
    vals_s[:10] *= 0.75
    for n in range(3):
        assert _rel(orc.ttmctc(dims, idx_p, vals[p], U, n), A[n]) < 1e-13
        assert _rel(orc.ttmctc(dims, idx_s, vals_s, U, n), A[n]) < 1e-13


# ----------------------------------------------------------------------------- QR

@pytest.mark.parametrize("I,K", [(50, 5), (7, 7), (300, 16), (33, 1)])
def test_qr_against_lapack(orc, I, K):
    A = np.random.default_rng(I * 31 + K).standard_normal((I, K))
    Q, R, z = orc.qr(A)
    assert z == 0
    assert np.linalg.norm(Q.T @ Q - np.eye(K)) < 1e-13
    assert _rel(Q @ R, A) < 1e-13
    assert np.allclose(np.tril(R, -1), 0.0)
    assert np.all(np.diag(R) > 0)
    q, r = np.linalg.qr(A)
    s = np.sign(np.diag(r))
    assert np.linalg.norm(Q - q * s) < 1e-12
    assert np.linalg.norm(R - r * s[:, None]) < 1e-11 * np.linalg.norm(A)


def test_qr_rank_deficient_completes(orc):
    rng = np.random.default_rng(21)
    A = rng.standard_normal((40, 5))
    A[:, 2] = 0.0
    A[:, 4] = A[:, 0] * 2.0  # dependent column
    Q, R, z = orc.qr(A)
    assert z >= 1
    assert np.linalg.norm(Q.T @ Q - np.eye(5)) < 1e-12
    assert _rel(Q @ R, A) < 1e-12
    # range(A) is inside range(Q)
    assert np.linalg.norm(A - Q @ (Q.T @ A)) < 1e-12 * np.linalg.norm(A)


# ---------------------------------------------------------------------- HOQRI

def test_fit_identity_dense(orc):
    """||X - G x {U}||^2 = ||X||^2 - ||G||^2 for orthonormal U and G = X x {U^T}."""
    dims, ranks = (6, 5, 7), (3, 2, 3)
    idx, vals = _rand_coo(dims, 80, 22)
    U = _rand_U(dims, ranks, 23, ortho=True)
    Xd = D.dense(dims, idx, vals)
    G = orc.core(idx, vals, U)
    lhs = float(((Xd - D.reconstruct(G, U)) ** 2).sum())
    ci, cv = orc.coalesce(idx, vals)
    rhs = orc.norm2(cv) - float((G ** 2).sum())
    assert abs(lhs - rhs) < 1e-12 * orc.norm2(cv)
    out = orc.hoqri(dims, idx, vals, U, 3)
    Xr = D.reconstruct(out["G"], out["U"])
    r_dense = math.sqrt(float(((Xd - Xr) ** 2).sum()) / float((Xd ** 2).sum()))
    assert abs(out["resid"][-1] - r_dense) < 1e-10


def test_monotone_objective_thm1(orc):
    dims, ranks = (12, 10, 9), (3, 3, 2)
    idx, vals = _rand_coo(dims, 200, 24)
    U = _rand_U(dims, ranks, 25, ortho=True)
    out = orc.hoqri(dims, idx, vals, U, 8)
    f = out["fblock"]
    assert np.all(np.diff(f) >= -1e-12 * f.max())
    assert f[-1] > f[0]
    for u in out["U"]:
        assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) < 1e-13


def test_interlacing_lemma(orc):
    """sigma_k(A_n) >= lambda_k(G_(n) G_(n)^T) (appendix lemma)."""
    dims, ranks = (10, 9, 8), (3, 4, 2)
    idx, vals = _rand_coo(dims, 150, 26)
    U = _rand_U(dims, ranks, 27, ortho=True)
    for n in range(3):
        A, G = orc.ttmctc(dims, idx, vals, U, n, return_core=True)
        Gn = D.unfold(G, n)
        s = np.linalg.svd(A, compute_uv=False)
        lam = np.sort(np.linalg.eigvalsh(Gn @ Gn.T))[::-1]
        assert np.all(s >= lam - 1e-12 * s.max())


def test_matrix_case_is_subspace_iteration(orc):
    """N = 2: HOQRI is alternating subspace iteration; it must reach the top-K
    singular subspaces of the (gapped) matrix, compared with LAPACK's SVD."""
    rng = np.random.default_rng(28)
    I, J, K = 30, 20, 3
    P = np.linalg.qr(rng.standard_normal((I, J)))[0]
    Q = np.linalg.qr(rng.standard_normal((J, J)))[0]
    s = np.array([10.0, 7.0, 5.0] + [1.0 / (1 + k) for k in range(J - 3)])
    M = (P * s) @ Q.T
    ii, jj = np.meshgrid(np.arange(I), np.arange(J), indexing="ij")
    idx = [ii.ravel().astype(np.int32), jj.ravel().astype(np.int32)]
    U0 = _rand_U((I, J), (K, K), 29, ortho=True)
    out = orc.hoqri((I, J), idx, M.ravel(), U0, 40)
    u, sv, vt = np.linalg.svd(M)
    assert D.proj_dist(out["U"][0], u[:, :K]) < 1e-10
    assert D.proj_dist(out["U"][1], vt[:K].T) < 1e-10
    r_expect = math.sqrt(float((sv[K:] ** 2).sum()) / float((sv ** 2).sum()))
    assert abs(out["resid"][-1] - r_expect) < 1e-12


def test_exact_low_rank_recovered(orc):
    """A fully observed tensor of exact multilinear rank K: residual -> 0 and
    the planted subspaces are recovered."""
    dims, ranks = (8, 7, 6), (2, 3, 2)
    rng = np.random.default_rng(30)
    Ut = [np.linalg.qr(rng.standard_normal((I, K)))[0] for I, K in zip(dims, ranks)]
    Gt = rng.standard_normal(ranks) * 3.0
    Xd = D.reconstruct(Gt, Ut)
    grid = np.meshgrid(*[np.arange(I) for I in dims], indexing="ij")
    idx = [g.ravel().astype(np.int32) for g in grid]
    U0 = _rand_U(dims, ranks, 31, ortho=True)
    out = orc.hoqri(dims, idx, Xd.ravel(), U0, 30)
    assert out["resid"][-1] < 1e-7
    for u, ut in zip(out["U"], Ut):
        assert D.proj_dist(u, ut) < 1e-7


# ------------------------------------------------ Riemannian gradient (Sec. 5)

def test_grad_two_forms_of_eq_grad2_agree(orc):
    """Eq. grad2: sum_n ||2 A_n - 2 U_n G_(n) G_(n)^T||^2 equals
    sum_n 4 (||A_n||^2 - ||G_(n) G_(n)^T||^2) at orthonormal U (the last line
    follows from Eq. AU); the second form is computed here from the oracle's
    A_n and core, independently of its gradient routine."""
    dims, ranks = (9, 8, 7, 6), (3, 2, 3, 2)
    idx, vals = _rand_coo(dims, 300, 40)
    U = _rand_U(dims, ranks, 41, ortho=True)
    g = orc.grad_norm2(dims, idx, vals, U)
    alt = 0.0
    for n in range(4):
        A, G = orc.ttmctc(dims, idx, vals, U, n, return_core=True)
        Gn = D.unfold(G, n)
        alt += 4.0 * (float((A ** 2).sum()) - float(((Gn @ Gn.T) ** 2).sum()))
    assert g > 0 and abs(g - alt) <= 1e-10 * g


def test_grad_is_projected_euclidean_gradient(orc):
    """Block n of the gradient is tangent (U_n^T grad_n = 0) and its inner
    product with a tangent direction equals the directional derivative of the
    dense objective f(U) = ||X x {U^T}||^2, taken by central differences."""
    dims, ranks = (7, 6, 5), (3, 2, 2)
    idx, vals = _rand_coo(dims, 90, 42)
    U = _rand_U(dims, ranks, 43, ortho=True)
    Xd = D.dense(dims, idx, vals)

    def f(V):
        return float((D.core_dense(Xd, V) ** 2).sum())

    rng = np.random.default_rng(44)
    for n in range(3):
        gn = orc.grad(dims, idx, vals, U, n)
        assert np.linalg.norm(U[n].T @ gn) <= 1e-12 * np.linalg.norm(gn)
        Z = rng.standard_normal(U[n].shape)
        S = rng.standard_normal((ranks[n], ranks[n]))
        xi = Z - U[n] @ (U[n].T @ Z) + U[n] @ (S - S.T)  # tangent to the Stiefel manifold at U_n
        eps = 1e-5
        Up, Um = list(U), list(U)
        Up[n], Um[n] = U[n] + eps * xi, U[n] - eps * xi
        fd = (f(Up) - f(Um)) / (2 * eps)
        assert abs(fd - float((gn * xi).sum())) <= 1e-7 * max(1.0, abs(fd))


def test_grad_vanishes_at_stationary_points(orc):
    """Def. stationary: zero at the planted factors of an exactly rank-K tensor,
    and driven to zero by HOQRI from a random start (Sec. 5.2)."""
    dims, ranks = (8, 7, 6), (2, 3, 2)
    rng = np.random.default_rng(45)
    Ut = [np.linalg.qr(rng.standard_normal((I, K)))[0] for I, K in zip(dims, ranks)]
    Xd = D.reconstruct(rng.standard_normal(ranks) * 3.0, Ut)
    grid = np.meshgrid(*[np.arange(I) for I in dims], indexing="ij")
    idx = [g.ravel().astype(np.int32) for g in grid]
    nx4 = float((Xd ** 2).sum()) ** 2
    assert orc.grad_norm2(dims, idx, Xd.ravel(), Ut) <= 1e-24 * nx4
    U0 = _rand_U(dims, ranks, 46, ortho=True)
    g0 = orc.grad_norm2(dims, idx, Xd.ravel(), U0)
    out = orc.hoqri(dims, idx, Xd.ravel(), U0, 30)
    assert orc.grad_norm2(dims, idx, Xd.ravel(), out["U"]) <= 1e-10 * g0


def test_hosvd_recovers_planted_subspaces(orc):
    """HOSVD of an exactly rank-K tensor: the leading left singular subspaces of
    its unfoldings are the planted factors' ranges (and the unfolding has rank
    K_n), so the oracle's factors span them; with repeated coordinates summed."""
    dims, ranks = (9, 8, 7), (3, 2, 3)
    rng = np.random.default_rng(47)
    Ut = [np.linalg.qr(rng.standard_normal((I, K)))[0] for I, K in zip(dims, ranks)]
    Xd = D.reconstruct(rng.standard_normal(ranks), Ut)
    grid = np.meshgrid(*[np.arange(I) for I in dims], indexing="ij")
    idx = [np.concatenate([g.ravel(), g.ravel()[:5]]).astype(np.int32) for g in grid]
    vals = np.concatenate([Xd.ravel(), np.zeros(5)])
    U = orc.hosvd(dims, idx, vals, ranks)
    for u, ut, K in zip(U, Ut, ranks):
        assert u.shape[1] == K and np.linalg.norm(u.T @ u - np.eye(K)) < 1e-12
        assert D.proj_dist(u, ut) < 1e-10


def test_hosvd_is_the_top_eigenspace_of_the_unfolding_gram(orc):
    """U_n spans the top-K_n eigenvectors of X_(n) X_(n)^T, here formed from
    the sparse entries by brute force and diagonalised by LAPACK's symmetric
    eigensolver, a different routine from the oracle's SVD."""
    dims, ranks = (10, 7, 6), (3, 2, 2)
    idx, vals = _rand_coo(dims, 120, 48)
    U = orc.hosvd(dims, idx, vals, ranks)
    Xd = D.dense(dims, idx, vals)
    for n, K in enumerate(ranks):
        Xn = D.unfold(Xd, n)
        w, v = np.linalg.eigh(Xn @ Xn.T)
        assert w[-K] - w[-K - 1] > 1e-6 * w[-1]  # a gap, so the subspace is unique
        assert D.proj_dist(U[n], v[:, -K:]) < 1e-9


def test_generator_is_seeded_and_shaped():
    X1, U1, c1 = inputs.make_config("c1")
    X2, U2, c2 = inputs.make_config("c1")
    assert X1.nnz == 10_000 and X1.dims == (200, 200, 200)
    for a, b in zip(X1.idx, X2.idx):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(X1.vals, X2.vals)
    assert all(a.min() >= 0 and a.max() < d for a, d in zip(X1.idx, X1.dims))
    assert np.all((X1.vals > 0) & (X1.vals < 1))
    for u in U1:
        assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) < 1e-13
    Xd = inputs.random_sparse((50, 40, 30), 5000, 99, dist="zipf", s=1.1, distinct=True)
    keys = np.ravel_multi_index(tuple(a.astype(np.int64) for a in Xd.idx), Xd.dims)
    assert np.unique(keys).size == 5000


def test_rows_with_a_given_core_equal_the_rows_with_the_oracle_core(orc):
    """ttmctc_rows_with_core (the element-wise step of Alg. 3 with G supplied)
    given the oracle's own core equals ttmctc_rows, and both equal the dense
    matricised product X_(n) (kron of the other factors) G_(n)^T on those rows."""
    rng = np.random.default_rng(3)
    dims, ranks = (9, 8, 7, 6), (3, 2, 4, 2)
    nnz = 400
    idx = [rng.integers(0, d, nnz).astype(np.int32) for d in dims]
    vals = rng.standard_normal(nnz)
    U = [rng.standard_normal((d, k)) for d, k in zip(dims, ranks)]
    for n in range(4):
        rows = np.array([0, 3, 5], dtype=np.int32)
        A1, G = orc.ttmctc_rows(dims, idx, vals, U, n, rows, return_core=True)
        A2 = orc.ttmctc_rows_with_core(dims, idx, vals, U, n, rows, G)
        assert np.array_equal(A1, A2)
        Xd = np.zeros(dims)
        np.add.at(Xd, tuple(idx), vals)
        Gd = np.einsum("ijkl,ip,jq,kr,ls->pqrs", Xd, *U)  # G = X x {U^T}
        others = [m for m in range(4) if m != n]
        Xn = np.moveaxis(Xd, n, 0).reshape(dims[n], -1)
        Kr = U[others[0]]
        for m in others[1:]:
            Kr = np.kron(Kr, U[m])
        Gn = np.moveaxis(Gd, n, 0).reshape(ranks[n], -1)
        assert np.allclose(A2, (Xn @ Kr @ Gn.T)[rows], rtol=1e-12, atol=1e-12)
