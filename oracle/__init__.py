"""CPU FP64 oracle of the PRISM QP projection (ctypes wrapper over prism_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path never
imports this package, and this package never imports the product (it only
reads the seeded input generator module, which holds no projection arithmetic).

See ``prism_oracle.c`` for what each routine computes and which equation of the
paper (Sec. III-D) it follows.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

MODE_ADMM, MODE_PAPER = 0, 1
SCALE_ROWNORM, SCALE_NONE = 0, 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prism_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libprism_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) into oracle/_build/."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(path: str):
    """Open a compiled oracle library and declare its entry points."""
    lib = ctypes.CDLL(path)
    d, i, ll = ctypes.c_double, ctypes.c_int, ctypes.c_longlong
    P = ctypes.c_void_p
    lib.oracle_build_G_h.argtypes = [i, d, P, d, d, P, P]
    lib.oracle_build_G_h.restype = i
    lib.oracle_kkt_inverse.argtypes = [i, i, i, d, d, P, P]
    lib.oracle_kkt_inverse.restype = i
    lib.oracle_solve_batch.argtypes = [i, i, i, i, i, d, P, P, P, P, i, d, P, P, P, P, P,
                                       P, P, ll, i]
    lib.oracle_solve_batch.restype = i
    lib.oracle_exact_projection.argtypes = [i, d, P, d, d, P, d, d, ll, P, P]
    lib.oracle_exact_projection.restype = ll
    lib.oracle_philox4x32_10.argtypes = [P, P, P]
    lib.oracle_philox4x32_10.restype = None
    lib.oracle_sample_batch.argtypes = [i, i, i, P, P, ctypes.c_ulonglong, ctypes.c_ulonglong, P]
    lib.oracle_sample_batch.restype = i
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = i
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


@contextlib.contextmanager
def swapped_library(path: str):
    """Run the oracle's functions on another build of prism_oracle.c (a copy
    with a planted mistake, compiled by a test) inside the ``with`` block."""
    global _lib
    old = _load()
    new = _bind(path)
    with _lock:
        _lib = new
    try:
        yield
    finally:
        with _lock:
            _lib = old


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def build_G_h(H: int, dt: float, bnd, q0: float, v0: float):
    """Verbatim G ((8H-2) x H) and h (8H-2) of Eq. (G_h_def) for one joint."""
    lib = _load()
    bnd = _f64(bnd)
    assert bnd.shape == (8,)
    G = np.zeros((8 * H - 2, H))
    h = np.zeros(8 * H - 2)
    rc = lib.oracle_build_G_h(H, dt, _p(bnd), q0, v0, _p(G), _p(h))
    if rc:
        raise ValueError(f"oracle_build_G_h failed: {rc}")
    return G, h


def kkt_inverse(H: int, dt: float, rho: float, mode: int = MODE_ADMM, scale: int = SCALE_ROWNORM):
    """K = [M^-1]_{1:H,1:H} and kb = [M^-1]_{1:H,H+1} of the KKT matrix (Eq. admm_primal)."""
    lib = _load()
    K = np.zeros((H, H))
    kb = np.zeros(H)
    rc = lib.oracle_kkt_inverse(mode, scale, H, dt, rho, _p(K), _p(kb))
    if rc:
        raise ValueError(f"oracle_kkt_inverse failed: {rc}")
    return K, kb


def max_threads() -> int:
    return int(_load().oracle_num_threads())


def solve_batch(xi, q0, v0, bounds, dt: float, iters: int, rho: float = 1.0,
                mode: int = MODE_ADMM, scale: int = SCALE_ROWNORM, x_init=None, dual_init=None,
                cols=None, nthreads: int = 1, want_dual_state: bool = False):
    """Project a batch [N][H][J]; returns dict(x, primal, dual[, dual_state]).

    ``cols`` (optional) lists flattened columns n*J + j to solve; the other
    entries of the outputs are NaN.
    """
    lib = _load()
    xi = _f64(xi)
    N, H, J = xi.shape
    q0 = _f64(q0).reshape(J)
    v0 = _f64(v0).reshape(J)
    bounds = _f64(bounds).reshape(8, J)
    D = 4 * H - 1 if mode == MODE_ADMM else H
    x = np.full((N, H, J), np.nan)
    pr = np.full((N, J), np.nan)
    du = np.full((N, J), np.nan)
    dstate = np.full((N, D, J), np.nan) if want_dual_state else None
    xin = None if x_init is None else _f64(x_init).reshape(N, H, J)
    din = None if dual_init is None else _f64(dual_init).reshape(N, D, J)
    carr = None
    ncols = 0
    if cols is not None:
        carr = np.ascontiguousarray(np.asarray(cols, dtype=np.int64))
        ncols = int(carr.size)
    rc = lib.oracle_solve_batch(mode, scale, N, J, H, float(dt), _p(bounds), _p(q0), _p(v0), _p(xi),
                                int(iters), float(rho), _p(xin), _p(din), _p(x), _p(pr), _p(du),
                                _p(dstate), _p(carr), ncols, int(nthreads))
    if rc:
        raise ValueError(f"oracle_solve_batch failed: {rc}")
    out = {"x": x, "primal": pr, "dual": du}
    if want_dual_state:
        out["dual_state"] = dstate
    return out


def exact_projection(xi_col, H: int, dt: float, bnd, q0: float, v0: float,
                     tol_step: float = 1e-14, tol_viol: float = 1e-13, max_iters: int = 2_000_000):
    """Pi(xi) for one column by ADMM run to convergence; returns (x, iters, violation)."""
    lib = _load()
    xi_col = _f64(xi_col).reshape(H)
    bnd = _f64(bnd).reshape(8)
    x = np.zeros(H)
    viol = np.zeros(1)
    it = lib.oracle_exact_projection(H, float(dt), _p(bnd), float(q0), float(v0), _p(xi_col),
                                     tol_step, tol_viol, int(max_iters), _p(x), _p(viol))
    if it < 0:
        raise ValueError("oracle_exact_projection failed")
    return x, int(it), float(viol[0])


def philox4x32_10(counter, key):
    """Philox4x32-10 block: four uint32 words from a 4-word counter and a 2-word key."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(counter, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def sample_batch(N, H, J, mean, std, seed: int, stream: int):
    """xi [N][H][J] = mean + std * z, z from Philox4x32-10 + Box-Muller (see prism_oracle.c)."""
    lib = _load()
    m = _f64(mean).reshape(H, J)
    sd = _f64(std).reshape(H, J)
    xi = np.zeros((N, H, J))
    rc = lib.oracle_sample_batch(int(N), int(H), int(J), _p(m), _p(sd), int(seed), int(stream), _p(xi))
    if rc:
        raise ValueError("oracle_sample_batch failed")
    return xi
