"""The C-ABI library builds, loads and exports what include/prism_proj.h
declares; host-side argument checks run without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2608_25666_b300 import build, prism_proj

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return prism_proj.lib()


def declared_functions():
    with open(os.path.join(ROOT, "include", "prism_proj.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(prism_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("prism_proj_create", "prism_proj_factor", "prism_proj_solve",
                     "prism_proj_destroy", "prism_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_status_strings(L):
    for code, name in prism_proj.STATUS.items():
        assert L.prism_status_string(code).decode() == name


def _create(L, J, H, dt, bounds):
    rows = [np.ascontiguousarray(bounds[r], dtype=np.float64) for r in range(8)]
    h = ctypes.c_void_p()
    st = L.prism_proj_create(J, H, dt, *[r.ctypes.data_as(ctypes.c_void_p) for r in rows],
                             ctypes.byref(h))
    return st, h


def _bounds(J):
    b = np.zeros((8, J))
    b[:] = np.array([-6.0, 6.0, -3.0, 3.0, -8.0, 8.0, -80.0, 80.0])[:, None]
    return b


def test_create_rejects_bad_arguments_on_host(L):
    assert _create(L, 0, 10, 0.05, _bounds(1))[0] == 1
    assert _create(L, 65, 10, 0.05, _bounds(65))[0] == 1
    assert _create(L, 2, 1, 0.05, _bounds(2))[0] == 1
    assert _create(L, 2, 133, 0.05, _bounds(2))[0] == 1
    assert _create(L, 2, 10, 0.0, _bounds(2))[0] == 1
    assert _create(L, 2, 10, float("nan"), _bounds(2))[0] == 1
    b = _bounds(2)
    b[2, 1], b[3, 1] = 1.0, -1.0          # v_min > v_max
    assert _create(L, 2, 10, 0.05, b)[0] == 1
    b = _bounds(2)
    b[4, 0] = 0.5                          # a_min > 0: first acceleration row is 0
    st, h = _create(L, 2, 10, 0.05, b)
    assert st == 4
    assert "acceleration" in L.prism_last_error().decode()
    b = _bounds(2)
    b[0, 0] = float("inf")
    assert _create(L, 2, 10, 0.05, b)[0] == 1
    h = ctypes.c_void_p()
    assert L.prism_proj_create(2, 10, 0.05, *([None] * 8), ctypes.byref(h)) == 1


def test_null_handle_calls_fail_cleanly(L):
    assert L.prism_proj_destroy(None) == 1
    assert L.prism_proj_factor(None, 1.0, 0, 0, 0, None) == 1
    assert L.prism_proj_solve(None, 1, None, None, None, 10, 1.0, None, None, None, None) == 1


def test_valid_create_without_gpu_reports_cuda_error(L):
    try:
        import torch
        gpu = torch.cuda.is_available()
    except Exception:
        gpu = False
    st, h = _create(L, 3, 10, 0.05, _bounds(3))
    if gpu:
        assert st == 0
        assert L.prism_proj_destroy(h) == 0
    else:
        assert st == 6
        assert h.value is None
