"""Dense brute-force statements used to pin the oracle (tests only).

Everything here goes through numpy library routines on a DENSE copy of X:
np.add.at (duplicates summed), np.kron (Eq. (2) Kronecker chain), matmul and
einsum.  None of it is shared with the oracle or the CUDA library.
"""
from functools import reduce

import numpy as np


def dense(dims, idx, vals):
    X = np.zeros(tuple(dims), dtype=np.float64)
    np.add.at(X, tuple(np.asarray(a, dtype=np.int64) for a in idx), np.asarray(vals, dtype=np.float64))
    return X


def unfold(T, n):
    """Mode-n unfolding: rows i_n, columns over the other modes in ascending
    order with the last one fastest (the Kronecker order of Eq. (2))."""
    return np.moveaxis(T, n, 0).reshape(T.shape[n], -1)


def kron_chain(mats, skip):
    return reduce(np.kron, [M for m, M in enumerate(mats) if m != skip])


def ttmc_unfolded(X, U, n):
    """Y_(n) = X_(n) (U_1 (x) ... (x) U_N, mode n skipped): Eq. (2) with B = U^T."""
    return unfold(X, n) @ kron_chain(U, n)


def core_dense(X, U):
    letters = "abcdefgh"[:X.ndim]
    outl = "ijklmnop"[:X.ndim]
    spec = letters + "," + ",".join(l + o for l, o in zip(letters, outl)) + "->" + outl
    return np.einsum(spec, X, *U, optimize=True)


def ttmctc_dense(X, U, n):
    """A_n = Y_(n) G_(n)^T (Eq. ttmctc) with G = X x {U^T} from einsum."""
    G = core_dense(X, U)
    return ttmc_unfolded(X, U, n) @ unfold(G, n).T


def reconstruct(G, U):
    letters = "ijklmnop"[:G.ndim]
    outl = "abcdefgh"[:G.ndim]
    spec = letters + "," + ",".join(o + l for l, o in zip(letters, outl)) + "->" + outl
    return np.einsum(spec, G, *U, optimize=True)


def proj_dist(U, V):
    """|| U U^T - V V^T ||_F (subspace distance; rotation invariant)."""
    return float(np.linalg.norm(U @ U.T - V @ V.T))
