"""Python entry to the FP64 CPU oracle (hoqri_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  Nothing here imports the
CUDA library or its package, and the library never imports this module.

``build()`` compiles ``hoqri_oracle.c`` with gcc (OpenMP when available,
``-ffp-contract=off`` so x86 and Arm round identically) into
``oracle/_build/libhoqri_oracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "hoqri_oracle.c"
_OUT = _HERE / "_build" / "libhoqri_oracle.so"
_lib = None

_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_f64p = C.POINTER(C.c_double)


def build(force: bool = False) -> Path:
    """Compile the oracle shared library (idempotent)."""
    if _OUT.exists() and not force and _OUT.stat().st_mtime >= _SRC.stat().st_mtime:
        return _OUT
    _OUT.parent.mkdir(parents=True, exist_ok=True)
    tmp = _OUT.with_suffix(f".{os.getpid()}.tmp.so")
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", str(_SRC), "-o", str(tmp), "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(str(_OUT))
        L.hoqri_oracle_coalesce.restype = C.c_int64
        L.hoqri_oracle_coalesce.argtypes = [C.c_int, C.c_int64, C.POINTER(_i32p), _f64p, C.POINTER(_i32p), _f64p]
        L.hoqri_oracle_norm2.restype = C.c_double
        L.hoqri_oracle_norm2.argtypes = [C.c_int64, _f64p]
        L.hoqri_oracle_core.restype = None
        L.hoqri_oracle_core.argtypes = [C.c_int, _i32p, C.c_int64, C.POINTER(_i32p), _f64p, C.POINTER(_f64p), _f64p]
        L.hoqri_oracle_core_entries.restype = None
        L.hoqri_oracle_core_entries.argtypes = [C.c_int, _i32p, C.c_int64, C.POINTER(_i32p), _f64p,
                                                C.POINTER(_f64p), C.c_int64, _i64p, _f64p]
        L.hoqri_oracle_ttmctc.restype = None
        L.hoqri_oracle_ttmctc.argtypes = [C.c_int, _i64p, _i32p, C.c_int64, C.POINTER(_i32p), _f64p,
                                          C.POINTER(_f64p), C.c_int, _f64p, _f64p]
        L.hoqri_oracle_ttmctc_rows.restype = None
        L.hoqri_oracle_ttmctc_rows.argtypes = [C.c_int, _i64p, _i32p, C.c_int64, C.POINTER(_i32p), _f64p,
                                               C.POINTER(_f64p), C.c_int, C.c_int64, _i32p, _f64p, _f64p]
        L.hoqri_oracle_ttmctc_rows_with_core.restype = None
        L.hoqri_oracle_ttmctc_rows_with_core.argtypes = [C.c_int, _i64p, _i32p, C.c_int64, C.POINTER(_i32p), _f64p,
                                                         C.POINTER(_f64p), C.c_int, _f64p, C.c_int64, _i32p, _f64p]
        L.hoqri_oracle_ttmctc_matrix.restype = None
        L.hoqri_oracle_ttmctc_matrix.argtypes = [C.c_int, _i64p, _i32p, C.c_int64, C.POINTER(_i32p), _f64p,
                                                 C.POINTER(_f64p), C.c_int, _f64p]
        L.hoqri_oracle_qr.restype = C.c_int
        L.hoqri_oracle_qr.argtypes = [C.c_int64, C.c_int, _f64p, _f64p, _f64p]
        L.hoqri_oracle_hoqri.restype = C.c_int
        L.hoqri_oracle_hoqri.argtypes = [C.c_int, _i64p, _i32p, C.c_int64, C.POINTER(_i32p), _f64p,
                                         C.POINTER(_f64p), C.c_int, _f64p, _f64p, _f64p]
        L.hoqri_oracle_threads.restype = C.c_int
        L.hoqri_oracle_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def threads() -> int:
    return int(lib().hoqri_oracle_threads())


def set_threads(t: int) -> None:
    lib().hoqri_oracle_set_threads(int(t))


# ---------------------------------------------------------------- marshalling

def _p(a, t):
    return a.ctypes.data_as(t)


class _Coo:
    """Keeps contiguous int32/float64 copies alive for one call."""

    def __init__(self, idx, vals):
        self.idx = [np.ascontiguousarray(a, dtype=np.int32) for a in idx]
        self.vals = np.ascontiguousarray(vals, dtype=np.float64)
        self.N = len(self.idx)
        self.nnz = int(self.vals.shape[0])
        self.idx_arr = (_i32p * self.N)(*[_p(a, _i32p) for a in self.idx])


class _Mats:
    def __init__(self, mats):
        self.m = [np.ascontiguousarray(a, dtype=np.float64) for a in mats]
        self.arr = (_f64p * len(self.m))(*[_p(a, _f64p) for a in self.m])


def _dims(d):
    return np.ascontiguousarray(d, dtype=np.int64)


def _ranks(U):
    return np.ascontiguousarray([u.shape[1] for u in U], dtype=np.int32)


def coalesce(idx, vals):
    """Sum repeated coordinates; returns (idx list, vals) in lexicographic order."""
    c = _Coo(idx, vals)
    out = [np.empty(max(c.nnz, 1), dtype=np.int32) for _ in range(c.N)]
    ov = np.empty(max(c.nnz, 1), dtype=np.float64)
    oarr = (_i32p * c.N)(*[_p(a, _i32p) for a in out])
    n = lib().hoqri_oracle_coalesce(c.N, c.nnz, c.idx_arr, _p(c.vals, _f64p), oarr, _p(ov, _f64p))
    return [a[:n].copy() for a in out], ov[:n].copy()


def norm2(vals_coalesced):
    v = np.ascontiguousarray(vals_coalesced, dtype=np.float64)
    return float(lib().hoqri_oracle_norm2(v.shape[0], _p(v, _f64p)))


def core(idx, vals, U):
    """G = X x {U^T} (row-major, last index fastest)."""
    c, M = _Coo(idx, vals), _Mats(U)
    r = _ranks(M.m)
    G = np.empty(int(np.prod(r)), dtype=np.float64)
    lib().hoqri_oracle_core(c.N, _p(r, _i32p), c.nnz, c.idx_arr, _p(c.vals, _f64p), M.arr, _p(G, _f64p))
    return G.reshape(tuple(int(k) for k in r))


def core_entries(idx, vals, U, lin):
    c, M = _Coo(idx, vals), _Mats(U)
    r = _ranks(M.m)
    lin = np.ascontiguousarray(lin, dtype=np.int64)
    out = np.empty(lin.shape[0], dtype=np.float64)
    lib().hoqri_oracle_core_entries(c.N, _p(r, _i32p), c.nnz, c.idx_arr, _p(c.vals, _f64p), M.arr,
                                    lin.shape[0], _p(lin, _i64p), _p(out, _f64p))
    return out


def ttmctc(dims, idx, vals, U, n, return_core=False):
    """A_n by Alg. 3 (element-wise, recomputing G first)."""
    c, M = _Coo(idx, vals), _Mats(U)
    d, r = _dims(dims), _ranks(M.m)
    A = np.empty((int(d[n]), int(r[n])), dtype=np.float64)
    G = np.empty(int(np.prod(r)), dtype=np.float64)
    lib().hoqri_oracle_ttmctc(c.N, _p(d, _i64p), _p(r, _i32p), c.nnz, c.idx_arr, _p(c.vals, _f64p), M.arr,
                              int(n), _p(A, _f64p), _p(G, _f64p))
    if return_core:
        return A, G.reshape(tuple(int(k) for k in r))
    return A


def ttmctc_rows(dims, idx, vals, U, n, rows, return_core=False):
    """Rows `rows` of A_n (Alg. 3), with G computed by the oracle."""
    c, M = _Coo(idx, vals), _Mats(U)
    d, r = _dims(dims), _ranks(M.m)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    out = np.empty((rows.shape[0], int(r[n])), dtype=np.float64)
    G = np.empty(int(np.prod(r)), dtype=np.float64)
    lib().hoqri_oracle_ttmctc_rows(c.N, _p(d, _i64p), _p(r, _i32p), c.nnz, c.idx_arr, _p(c.vals, _f64p),
                                   M.arr, int(n), rows.shape[0], _p(rows, _i32p), _p(out, _f64p), _p(G, _f64p))
    if return_core:
        return out, G.reshape(tuple(int(k) for k in r))
    return out


def ttmctc_rows_with_core(dims, idx, vals, U, n, rows, G):
    """Rows `rows` of A_n by the element-wise step of Alg. 3, with the core G
    given (for sizes where the oracle's own core, O(nnz P N), is too slow: G is
    then checked separately at sampled entries with core_entries)."""
    c, M = _Coo(idx, vals), _Mats(U)
    d, r = _dims(dims), _ranks(M.m)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    Gd = np.ascontiguousarray(np.asarray(G, dtype=np.float64).ravel())
    if Gd.shape[0] != int(np.prod(r)):
        raise ValueError("G has the wrong number of entries")
    out = np.empty((rows.shape[0], int(r[n])), dtype=np.float64)
    lib().hoqri_oracle_ttmctc_rows_with_core(c.N, _p(d, _i64p), _p(r, _i32p), c.nnz, c.idx_arr, _p(c.vals, _f64p),
                                             M.arr, int(n), _p(Gd, _f64p), rows.shape[0], _p(rows, _i32p),
                                             _p(out, _f64p))
    return out


def ttmctc_matrix(dims, idx, vals, U, n):
    """A_n by Alg. 4 (sum over k_{-n} of y y^T U_n)."""
    c, M = _Coo(idx, vals), _Mats(U)
    d, r = _dims(dims), _ranks(M.m)
    A = np.empty((int(d[n]), int(r[n])), dtype=np.float64)
    lib().hoqri_oracle_ttmctc_matrix(c.N, _p(d, _i64p), _p(r, _i32p), c.nnz, c.idx_arr, _p(c.vals, _f64p),
                                     M.arr, int(n), _p(A, _f64p))
    return A


def grad(dims, idx, vals, U, n):
    """Block n of the Riemannian gradient of f = ||X x {U^T}||^2 on the product of
    Stiefel manifolds at {U} (Sec. 5, Eq. tucker_grad): 2 A_n - 2 U_n G_(n) G_(n)^T,
    A_n by Alg. 3 and G = X x {U^T}; G_(n) is the mode-n unfolding of the core
    (the other modes ascending, the last fastest)."""
    A, G = ttmctc(dims, idx, vals, U, n, return_core=True)
    Gn = np.moveaxis(G, n, 0).reshape(G.shape[n], -1)
    return 2.0 * A - 2.0 * (np.asarray(U[n], dtype=np.float64) @ (Gn @ Gn.T))


def grad_norm2(dims, idx, vals, U):
    """||grad f||^2 = sum over n of ||grad block n||_F^2 (Eq. grad2, first line)."""
    return float(sum(np.sum(grad(dims, idx, vals, U, n) ** 2) for n in range(len(U))))


def hosvd(dims, idx, vals, ranks):
    """HOSVD factors (the initialisation that Alg. 2 allows): U_n = the K_n leading
    left singular vectors of the mode-n unfolding of X (repeated coordinates
    summed), by LAPACK's SVD of the dense unfolding; small tensors only."""
    X = np.zeros(tuple(int(d) for d in dims), dtype=np.float64)
    np.add.at(X, tuple(np.asarray(a, dtype=np.int64) for a in idx), np.asarray(vals, dtype=np.float64))
    out = []
    for n, K in enumerate(ranks):
        Xn = np.moveaxis(X, n, 0).reshape(X.shape[n], -1)
        u, s, _ = np.linalg.svd(Xn, full_matrices=False)
        out.append(u[:, :int(K)])
    return out


def qr(A):
    """Householder thin QR with diag(R) >= 0: returns (Q, R, zero_pivots)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    I, K = A.shape
    Q = np.empty_like(A)
    R = np.empty((K, K), dtype=np.float64)
    z = lib().hoqri_oracle_qr(I, K, _p(A, _f64p), _p(Q, _f64p), _p(R, _f64p))
    return Q, R, int(z)


def hoqri(dims, idx, vals, U0, iters):
    """Alg. 2.  Returns dict(U, G, resid[iters], fblock[iters*N], zero_pivots)."""
    c = _Coo(idx, vals)
    U = [np.array(u, dtype=np.float64, order="C") for u in U0]
    M = _Mats(U)  # same buffers, written in place
    d, r = _dims(dims), _ranks(M.m)
    G = np.empty(int(np.prod(r)), dtype=np.float64)
    resid = np.empty(max(iters, 1), dtype=np.float64)
    fblock = np.empty(max(iters * c.N, 1), dtype=np.float64)
    z = lib().hoqri_oracle_hoqri(c.N, _p(d, _i64p), _p(r, _i32p), c.nnz, c.idx_arr, _p(c.vals, _f64p), M.arr,
                                 int(iters), _p(G, _f64p), _p(resid, _f64p), _p(fblock, _f64p))
    return dict(U=M.m, G=G.reshape(tuple(int(k) for k in r)), resid=resid[:iters],
                fblock=fblock[:iters * c.N], zero_pivots=int(z))
