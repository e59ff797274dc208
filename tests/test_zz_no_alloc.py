"""The allocation-free plain solve (prism_proj_solve_plain_noalloc).

It exists for callers that must not allocate device memory when they solve
(real-time controller threads that forbid allocation after start-up, hosts
whose device memory belongs to a pool this library cannot see).  It runs the
plain comparator with its workspace in a fixed device array instead of a
cudaMalloc'd one.  This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2608_25666_b300 import prism_proj as pp
from paper_2608_25666_b300 import workloads
from gpu_helpers import VIOL_TOL, X_TOL

pytestmark = pytest.mark.gpu

MAX_FLOATS = 4194304   # PRISM_NOALLOC_MAX_FLOATS in include/prism_proj.h


def _noalloc_fn():
    L = pp.lib()
    fn = L.prism_proj_solve_plain_noalloc
    P = ctypes.c_void_p
    fn.argtypes = [P, ctypes.c_int, P, P, P, ctypes.c_int, ctypes.c_double, P, P, P, P]
    fn.restype = ctypes.c_int
    return fn


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_plain_on_two_calls_in_a_row():
    import torch
    fn = _noalloc_fn()
    J, H, dt, iters = 12, 30, 0.05, 120
    P = pp.Projector(J, H, dt, workloads.base_bounds(J)).factor(1.0)
    stream = torch.cuda.current_stream()
    for call, (seed, N) in enumerate([(501, 300), (502, 177)]):
        b = workloads.make_custom(seed, N, J, H, dt)
        xi = torch.from_numpy(b["xi"]).cuda()
        q0 = torch.from_numpy(b["q0"]).cuda()
        v0 = torch.from_numpy(b["v0"]).cuda()
        xr, pr, dr = P.solve_plain(q0, v0, xi, iters)
        x = torch.empty_like(xi)
        prim = torch.empty((N, J), device="cuda")
        dual = torch.empty((N, J), device="cuda")
        st = fn(P._h, N, _ptr(q0), _ptr(v0), _ptr(xi), iters, 1.0, _ptr(x), _ptr(prim), _ptr(dual),
                ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, pp.lib().prism_last_error().decode()
        torch.cuda.synchronize()
        dx = float((x - xr).abs().max())
        dv = float((prim - pr).abs().max())
        dd = float((dual - dr).abs().max())
        assert dx <= X_TOL, (call, dx)
        assert dv <= VIOL_TOL, (call, dv)
        assert dd <= 2 * X_TOL, (call, dd)
        assert bool(torch.all(x[:, 0, :] == v0[None, :]))
    P.close()


def test_noalloc_rejects_batches_beyond_the_fixed_array():
    import torch
    fn = _noalloc_fn()
    J, H = 12, 50
    P = pp.Projector(J, H, 0.02, workloads.base_bounds(J)).factor(1.0)
    N = MAX_FLOATS // (J * 6 * H) + 1
    xi = torch.zeros((N, H, J), device="cuda")
    q0 = torch.zeros(J, device="cuda")
    v0 = torch.zeros(J, device="cuda")
    st = fn(P._h, N, _ptr(q0), _ptr(v0), _ptr(xi), 10, 1.0, _ptr(xi), None, None, None)
    assert st == 1
    assert "exceeds" in pp.lib().prism_last_error().decode()
    P.close()
