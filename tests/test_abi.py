"""The C-ABI library builds, loads and exports every symbol include/hoqri.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import os
import re

from paper_2510_16930_gb300 import build, hoqri

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hoqri.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hoqri_[a-z_0-9]+)\s*\(", src)))


def test_header_matches_binding():
    assert _declared() == sorted(hoqri.SYMBOLS)


def test_library_exports_all_symbols():
    lib = ctypes.CDLL(str(build.build()))
    for name in _declared():
        assert hasattr(lib, name), name


def test_default_options_and_error_text():
    o = hoqri.hoqri_default_options()
    assert o.prec == hoqri.HOQRI_FP32 and o.qr_kind == 0 and o.use_graphs == 1
    assert ctypes.sizeof(hoqri.hoqri_options) == 48 and o.tile_rows == 0 and o.tile_cols == 0
    assert isinstance(hoqri.hoqri_last_error(), str)


def test_create_rejects_bad_arguments_without_gpu_work():
    import numpy as np
    # argument checks run before any device call: rank above the mode size
    idx = [np.zeros(1, dtype=np.int32)] * 3
    vals = np.ones(1, dtype=np.float32)
    try:
        hoqri.hoqri_create((2, 3, 4), (3, 2, 2), 1, idx, vals)
        raise AssertionError("expected HOQRI_ERR_RANK")
    except hoqri.HoqriError as e:
        assert e.code == hoqri.HOQRI_ERR_RANK
    try:  # order 1 is not a tensor decomposition
        hoqri.hoqri_create((5,), (1,), 1, idx[:1], vals)
        raise AssertionError("expected HOQRI_ERR_INVALID")
    except hoqri.HoqriError as e:
        assert e.code == hoqri.HOQRI_ERR_INVALID
    try:  # K_n > prod_{m != n} K_m
        hoqri.hoqri_create((9, 9, 9), (5, 2, 2), 1, idx, vals)
        raise AssertionError("expected HOQRI_ERR_RANK")
    except hoqri.HoqriError as e:
        assert e.code == hoqri.HOQRI_ERR_RANK


def test_noalloc_rejects_bad_arguments_before_device_work():
    """Size and precision checks of hoqri_orthonormalize_noalloc come before any CUDA call."""
    import pytest
    for prec, I, K, frag in ((hoqri.HOQRI_BF16X3, 10, 4, "prec"), (hoqri.HOQRI_FP64, 100, 33, "32"),
                             (hoqri.HOQRI_FP32, 100, 0, "K = 0"), (hoqri.HOQRI_FP64, 5, 8, "I = 5 < K = 8")):
        with pytest.raises(hoqri.HoqriError) as e:
            hoqri.hoqri_orthonormalize_noalloc(prec, I, K, 0, 0)
        assert e.value.code == hoqri.HOQRI_ERR_INVALID and frag in str(e.value)


def test_server_rejects_bad_requests_without_gpu_work():
    """Server creation and submission validate on the host; nothing runs until a step."""
    import numpy as np
    import pytest
    srv = hoqri.hoqri_server_create(1 << 30, 4)
    try:
        idx = [np.zeros(10, np.int32)] * 3
        vals = np.ones(10, np.float32)
        with pytest.raises(hoqri.HoqriError) as e:
            hoqri.hoqri_server_submit(srv, (10,), (2,), 10, idx[:1], vals, 1, hoqri.HOQRI_FP32)
        assert e.value.code == hoqri.HOQRI_ERR_INVALID
        with pytest.raises(hoqri.HoqriError) as e:  # alone larger than the budget
            hoqri.hoqri_server_submit(srv, (10**6,) * 3, (32,) * 3, 10**9, idx, vals, 1, hoqri.HOQRI_FP32)
        assert e.value.code == hoqri.HOQRI_ERR_OOM
        rid = hoqri.hoqri_server_submit(srv, (10, 10, 10), (2, 2, 2), 10, idx, vals, 1, hoqri.HOQRI_FP32)
        st, t, b = hoqri.hoqri_server_poll(srv, rid)
        assert st == hoqri.HOQRI_REQ_QUEUED and b > 0  # while queued: the admission estimate
    finally:
        hoqri.hoqri_server_destroy(srv)
    with pytest.raises(hoqri.HoqriError):
        hoqri.hoqri_server_create(0, 4)


def test_run_and_grad_reject_a_null_context_without_gpu_work():
    import ctypes as C
    L = hoqri.load()
    done = C.c_int32(-1)
    out = C.c_double(-1.0)
    assert L.hoqri_run(None, 3, None, C.byref(done)) == hoqri.HOQRI_ERR_INVALID
    assert done.value == -1
    assert L.hoqri_grad_norm2(None, C.byref(out)) == hoqri.HOQRI_ERR_INVALID
    assert "NULL context" in hoqri.load().hoqri_last_error().decode()


def test_init_hosvd_rejects_a_null_context_without_gpu_work():
    assert hoqri.load().hoqri_init_hosvd(None, 2) == hoqri.HOQRI_ERR_INVALID
