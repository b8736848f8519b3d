"""ctypes binding of libhoqri (include/hoqri.h); argument marshalling only.

Every function keeps the C name.  Buffers are passed as raw addresses: a
``torch.Tensor`` (device or host), a ``numpy.ndarray`` (host) or an ``int``
address.  Every step of the computation runs in the CUDA library; if the
library cannot be loaded the import of this module fails.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

from . import build as _build

HOQRI_OK, HOQRI_ERR_INVALID, HOQRI_ERR_OOM, HOQRI_ERR_CUDA, HOQRI_ERR_QR_BREAKDOWN, HOQRI_ERR_RANK, \
    HOQRI_ERR_TIMEOUT, HOQRI_ERR_UNSUPPORTED = range(8)
HOQRI_FP64, HOQRI_FP32, HOQRI_BF16X3 = range(3)

_STATUS = {0: "HOQRI_OK", 1: "HOQRI_ERR_INVALID", 2: "HOQRI_ERR_OOM", 3: "HOQRI_ERR_CUDA",
           4: "HOQRI_ERR_QR_BREAKDOWN", 5: "HOQRI_ERR_RANK", 6: "HOQRI_ERR_TIMEOUT", 7: "HOQRI_ERR_UNSUPPORTED"}

# every entry point declared in include/hoqri.h
SYMBOLS = ("hoqri_default_options", "hoqri_create", "hoqri_core", "hoqri_ttmctc", "hoqri_orthonormalize",
           "hoqri_iterate", "hoqri_run", "hoqri_grad_norm2", "hoqri_init_hosvd",
           "hoqri_get_factor", "hoqri_set_factor", "hoqri_fit", "hoqri_info", "hoqri_layout",
           "hoqri_profile_enable", "hoqri_profile_read", "hoqri_synchronize", "hoqri_trim_memory",
           "hoqri_last_error", "hoqri_destroy", "hoqri_orthonormalize_noalloc", "hoqri_server_create", "hoqri_server_submit",
           "hoqri_server_step", "hoqri_server_poll", "hoqri_server_take", "hoqri_server_destroy")
HOQRI_REQ_QUEUED, HOQRI_REQ_RUNNING, HOQRI_REQ_DONE, HOQRI_REQ_FAILED = range(4)


class hoqri_options(C.Structure):
    _fields_ = [("prec", C.c_int32), ("qr_kind", C.c_int32), ("chunk_nnz", C.c_int32), ("autotune", C.c_int32),
                ("use_graphs", C.c_int32), ("one_stream", C.c_int32), ("seed", C.c_uint64), ("tol", C.c_double),
                ("tile_rows", C.c_int32), ("tile_cols", C.c_int32)]


class hoqri_request(C.Structure):
    _fields_ = [("N", C.c_int32), ("dims", C.POINTER(C.c_int64)), ("ranks", C.POINTER(C.c_int32)),
                ("nnz", C.c_int64), ("idx", C.POINTER(C.c_void_p)), ("vals", C.c_void_p), ("iters", C.c_int32),
                ("prec", C.c_int32), ("seed", C.c_uint64)]


class HoqriError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library_path() -> Path:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libhoqri.so (building it first when asked and needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not _build.LIB.exists():
        raise RuntimeError(f"libhoqri.so not found at {_build.LIB}; run paper_2510_16930_gb300.build.build()")
    L = C.CDLL(str(_build.LIB))
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    L.hoqri_default_options.argtypes = [C.POINTER(hoqri_options)]
    L.hoqri_default_options.restype = None
    L.hoqri_create.argtypes = [C.POINTER(vp), i32, C.POINTER(i64), C.POINTER(i32), i64, C.POINTER(vp), vp,
                               C.POINTER(hoqri_options), C.POINTER(vp), vp]
    L.hoqri_core.argtypes = [vp, vp]
    L.hoqri_ttmctc.argtypes = [vp, i32, vp]
    L.hoqri_orthonormalize.argtypes = [vp, i32, vp, vp]
    L.hoqri_iterate.argtypes = [vp, i32, C.POINTER(C.c_double)]
    L.hoqri_run.argtypes = [vp, i32, C.POINTER(C.c_double), C.POINTER(i32)]
    L.hoqri_grad_norm2.argtypes = [vp, C.POINTER(C.c_double)]
    L.hoqri_init_hosvd.argtypes = [vp, i32]
    L.hoqri_get_factor.argtypes = [vp, i32, vp]
    L.hoqri_set_factor.argtypes = [vp, i32, vp]
    L.hoqri_fit.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.hoqri_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    L.hoqri_layout.argtypes = [vp, i32, C.POINTER(i64)]
    L.hoqri_profile_enable.argtypes = [vp, i32]
    L.hoqri_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(i64)]
    L.hoqri_synchronize.argtypes = [vp]
    L.hoqri_trim_memory.argtypes = []
    L.hoqri_last_error.restype = C.c_char_p
    L.hoqri_orthonormalize_noalloc.argtypes = [i32, i64, i32, vp, vp, vp]
    L.hoqri_server_create.argtypes = [C.POINTER(vp), i64, i32]
    L.hoqri_server_submit.argtypes = [vp, C.POINTER(hoqri_request), C.POINTER(i64)]
    L.hoqri_server_step.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
    L.hoqri_server_poll.argtypes = [vp, i64, C.POINTER(i32), C.POINTER(C.c_double), C.POINTER(i64)]
    L.hoqri_server_take.argtypes = [vp, i64, C.POINTER(vp), vp, C.POINTER(C.c_double)]
    L.hoqri_server_destroy.argtypes = [vp]
    L.hoqri_server_destroy.restype = None
    L.hoqri_destroy.argtypes = [vp]
    L.hoqri_destroy.restype = None
    for name in ("hoqri_create", "hoqri_core", "hoqri_ttmctc", "hoqri_orthonormalize", "hoqri_iterate", "hoqri_run",
                 "hoqri_grad_norm2", "hoqri_init_hosvd",
                 "hoqri_get_factor", "hoqri_set_factor", "hoqri_fit", "hoqri_info", "hoqri_layout", "hoqri_synchronize",
                 "hoqri_trim_memory", "hoqri_profile_enable", "hoqri_profile_read", "hoqri_orthonormalize_noalloc", "hoqri_server_create",
                 "hoqri_server_submit", "hoqri_server_step", "hoqri_server_poll", "hoqri_server_take"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _addr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy buffers must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return int(x.data_ptr())
    raise TypeError(f"cannot take the address of {type(x)}")


def _check(code: int):
    if code != HOQRI_OK:
        raise HoqriError(code, load().hoqri_last_error().decode())


def hoqri_default_options(**kw) -> hoqri_options:
    o = hoqri_options()
    load().hoqri_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def hoqri_create(dims, ranks, nnz, idx, vals, opt=None, U0=None, stream=0) -> int:
    """Returns the context handle (an int).  idx: N buffers of int32; vals: reals;
    U0: None or N buffers; stream: cudaStream_t as int (0 = default stream)."""
    L = load()
    N = len(dims)
    d = (C.c_int64 * N)(*[int(v) for v in dims])
    r = (C.c_int32 * N)(*[int(v) for v in ranks])
    ia = (C.c_void_p * N)(*[_addr(a) for a in idx])
    ua = None if U0 is None else (C.c_void_p * N)(*[_addr(u) for u in U0])
    if opt is None:
        opt = hoqri_default_options()
    h = C.c_void_p()
    _check(L.hoqri_create(C.byref(h), N, d, r, int(nnz), ia, _addr(vals), C.byref(opt), ua, int(stream)))
    return h.value


def hoqri_core(ctx, G_out):
    _check(load().hoqri_core(ctx, _addr(G_out)))


def hoqri_ttmctc(ctx, mode, A_out):
    _check(load().hoqri_ttmctc(ctx, int(mode), _addr(A_out)))


def hoqri_orthonormalize(ctx, mode, A_in, U_out):
    _check(load().hoqri_orthonormalize(ctx, int(mode), _addr(A_in), _addr(U_out)))


def hoqri_orthonormalize_noalloc(prec, I, K, A_in, U_out, stream=0):
    """No context and no device allocation; A_in and U_out are device buffers."""
    _check(load().hoqri_orthonormalize_noalloc(int(prec), int(I), int(K), _addr(A_in), _addr(U_out), int(stream)))


def hoqri_iterate(ctx, iters, want_hist=True):
    """Returns the residual history (numpy array) when want_hist."""
    h = (C.c_double * max(int(iters), 1))() if want_hist else None
    _check(load().hoqri_iterate(ctx, int(iters), h))
    return np.array(h[:int(iters)]) if want_hist else None


def hoqri_run(ctx, max_iters):
    """Sweeps until the residual changes by less than the context's tol (or
    max_iters sweeps); returns the residual history of the sweeps run."""
    h = (C.c_double * max(int(max_iters), 1))()
    done = C.c_int32(0)
    _check(load().hoqri_run(ctx, int(max_iters), h, C.byref(done)))
    return np.array(h[:done.value])


def hoqri_grad_norm2(ctx):
    """||grad f||^2 at the current factors (FP64)."""
    out = C.c_double(0.0)
    _check(load().hoqri_grad_norm2(ctx, C.byref(out)))
    return out.value


def hoqri_init_hosvd(ctx, power_iters):
    """Factors <- leading left singular subspaces of the unfoldings."""
    _check(load().hoqri_init_hosvd(ctx, int(power_iters)))


def hoqri_get_factor(ctx, mode, U_out):
    _check(load().hoqri_get_factor(ctx, int(mode), _addr(U_out)))


def hoqri_set_factor(ctx, mode, U_in):
    _check(load().hoqri_set_factor(ctx, int(mode), _addr(U_in)))


def hoqri_fit(ctx):
    r, x, g = C.c_double(), C.c_double(), C.c_double()
    _check(load().hoqri_fit(ctx, C.byref(r), C.byref(x), C.byref(g)))
    return r.value, x.value, g.value


def hoqri_info(ctx, N):
    nnz, b = C.c_int64(), C.c_int64()
    rows = (C.c_int64 * N)()
    _check(load().hoqri_info(ctx, C.byref(nnz), rows, C.byref(b)))
    return nnz.value, list(rows), b.value


def hoqri_layout(ctx, mode):
    """(long-row threshold, work-item size, tile rows, tile columns) of the mode's
    sliced pass, or all -1 when the mode does not use it."""
    out = (C.c_int64 * 4)()
    _check(load().hoqri_layout(ctx, int(mode), out))
    return tuple(out)


def hoqri_profile_enable(ctx, enable=True):
    _check(load().hoqri_profile_enable(ctx, 1 if enable else 0))


def hoqri_profile_read(ctx):
    """Returns (dict of per-pass ms/count totals, kernel launches since create)."""
    out = (C.c_double * 8)()
    n = C.c_int64()
    _check(load().hoqri_profile_read(ctx, out, C.byref(n)))
    keys = ("core_ms", "core_n", "ttmctc_ms", "ttmctc_n", "qr_ms", "qr_n", "stream_ms", "stream_n")
    return dict(zip(keys, list(out))), n.value


def hoqri_synchronize(ctx):
    _check(load().hoqri_synchronize(ctx))


def hoqri_trim_memory():
    """Releases the device memory the library's pools keep for new contexts."""
    _check(load().hoqri_trim_memory())


def hoqri_last_error() -> str:
    return load().hoqri_last_error().decode()


def hoqri_destroy(ctx):
    if ctx:
        load().hoqri_destroy(ctx)


# ---- serving

def hoqri_server_create(budget_bytes, max_active):
    h = C.c_void_p()
    _check(load().hoqri_server_create(C.byref(h), int(budget_bytes), int(max_active)))
    return h.value


def hoqri_server_submit(srv, dims, ranks, nnz, idx, vals, iters, prec, seed=0):
    """Queues a request; idx / vals (host or device) must stay alive until it is
    admitted.  Returns the request id."""
    N = len(dims)
    keep = ((C.c_int64 * N)(*[int(v) for v in dims]), (C.c_int32 * N)(*[int(v) for v in ranks]),
            (C.c_void_p * N)(*[_addr(a) for a in idx]))
    q = hoqri_request(N, keep[0], keep[1], int(nnz), keep[2], _addr(vals), int(iters), int(prec), int(seed))
    rid = C.c_int64()
    _check(load().hoqri_server_submit(srv, C.byref(q), C.byref(rid)))
    return rid.value


def hoqri_server_step(srv):
    """One scheduling round; returns (running, queued)."""
    r, q = C.c_int32(), C.c_int32()
    _check(load().hoqri_server_step(srv, C.byref(r), C.byref(q)))
    return r.value, q.value


def hoqri_server_poll(srv, rid):
    """(state, (t_submit, t_admit, t_done), device_bytes); raises for a failed request."""
    st, b = C.c_int32(), C.c_int64()
    t = (C.c_double * 3)()
    _check(load().hoqri_server_poll(srv, int(rid), C.byref(st), t, C.byref(b)))
    return st.value, tuple(t), b.value


def hoqri_server_take(srv, rid, U_out=None, G_out=None):
    """Copies the results of a finished request out (buffers may be None) and
    frees it; returns the residual of the last sweep."""
    ua = None
    if U_out is not None:
        ua = (C.c_void_p * len(U_out))(*[_addr(u) for u in U_out])
    r = C.c_double()
    _check(load().hoqri_server_take(srv, int(rid), ua, _addr(G_out), C.byref(r)))
    return r.value


def hoqri_server_destroy(srv):
    if srv:
        load().hoqri_server_destroy(srv)
