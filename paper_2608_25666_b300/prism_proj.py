"""Python binding of libprism_proj (argument marshalling only).

Every step of the projection runs in the CUDA library; this module only turns
torch tensors into device pointers and status codes into exceptions.  There is
no CPU fallback: if the compiled library is missing, importing the symbols
fails with an error that says how to build it.

Layouts follow the C ABI (include/prism_proj.h): samples and trajectories are
[N, H, J] float32 (time-major, joint-minor), q0 / v0 are [J] float32,
residuals are [N, J] float32.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

MODE_ADMM, MODE_PAPER = 0, 1
SCALE_ROWNORM, SCALE_NONE = 0, 1
PREC_FP32, PREC_BF16X3, PREC_TF32, PREC_TF32X3 = 0, 1, 2, 3
TC_MAX_H = 116
MAX_H, MAX_J = 132, 64

STATUS = {0: "PRISM_OK", 1: "PRISM_ERR_INVALID_ARG", 2: "PRISM_ERR_NOT_FACTORED",
          3: "PRISM_ERR_RHO_MISMATCH", 4: "PRISM_ERR_INFEASIBLE_BOUNDS", 5: "PRISM_ERR_OOM",
          6: "PRISM_ERR_CUDA", 7: "PRISM_ERR_UNSUPPORTED", 8: "PRISM_ERR_TIMEOUT"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libprism_proj.so")
_lock = threading.Lock()
_lib = None


INIT_SAMPLE_MAJOR, INIT_COLUMN_MAJOR = 0, 1   # warm-start input layouts of prism_proj_solve_ex
HOST_MAX_CHUNKS = 16          # PRISM_HOST_MAX_CHUNKS: most chunks of the host-buffer pipeline


class SolveOpts(ctypes.Structure):
    """prism_solve_opts of the C ABI."""
    _fields_ = [("x_init", ctypes.c_void_p), ("dual_init", ctypes.c_void_p),
                ("dual_out", ctypes.c_void_p), ("polish_iters", ctypes.c_int), ("init_layout", ctypes.c_int)]


class Problem(ctypes.Structure):
    """prism_problem of the C ABI."""
    _fields_ = [("h", ctypes.c_void_p), ("batch", ctypes.c_int),
                ("q0", ctypes.c_void_p), ("v0", ctypes.c_void_p), ("samples", ctypes.c_void_p),
                ("out", ctypes.c_void_p), ("primal_res", ctypes.c_void_p), ("dual_res", ctypes.c_void_p),
                ("x_init", ctypes.c_void_p), ("dual_init", ctypes.c_void_p), ("dual_out", ctypes.c_void_p)]


PLAN_AUTOTUNE, PLAN_GRAPH = 1, 2


class PrismError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def lib() -> ctypes.CDLL:
    """Load the compiled library (build it with ``paper_2608_25666_b300.build.build()``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libprism_proj is not built ({LIB_PATH} missing); run "
                                  "python -c 'import __graft_entry__ as g; g.build()'")
            L = ctypes.CDLL(LIB_PATH)
            P, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
            L.prism_proj_create.argtypes = [i, i, d] + [P] * 8 + [ctypes.POINTER(P)]
            L.prism_proj_factor.argtypes = [P, d, i, i, i, P]
            sig = [P, i, P, P, P, i, d, P, P, P, P]
            L.prism_proj_solve.argtypes = sig
            L.prism_proj_solve_plain.argtypes = sig
            L.prism_proj_solve_host.argtypes = sig
            L.prism_proj_solve_ex.argtypes = [P, i, P, P, P, i, d, P, P, P, P, P]
            L.prism_proj_sample_solve.argtypes = [P, i, P, P, P, P, ctypes.c_ulonglong, ctypes.c_ulonglong,
                                                  i, d, P, P, P, P, P]
            L.prism_proj_sample_solve.restype = i
            L.prism_proj_check_fp64.argtypes = [P, i, P, P, P, P, P]
            L.prism_proj_shift_state.argtypes = [P, i, i, P, P, P]
            L.prism_proj_get_factor.argtypes = [P, P, P]
            L.prism_proj_query.argtypes = [P, i, ctypes.POINTER(ll)]
            L.prism_proj_destroy.argtypes = [P]
            L.prism_proj_device_status.argtypes = [P, P]
            L.prism_diag_wait_timeout.argtypes = [ctypes.c_uint, ctypes.POINTER(i)]
            L.prism_diag_wait_timeout.restype = i
            L.prism_test_fail_allocs.argtypes = [i, i]
            L.prism_test_fail_allocs.restype = None
            L.prism_test_set_device_flag.argtypes = [P, i]
            L.prism_test_set_device_flag.restype = i
            L.prism_proj_set_tiling.argtypes = [P, i]
            L.prism_proj_set_tiling.restype = i
            L.prism_proj_set_host_chunks.argtypes = [P, i]
            L.prism_proj_set_host_chunks.restype = i
            for name in ("create", "factor", "solve", "solve_ex", "solve_plain", "solve_host",
                         "check_fp64", "shift_state", "get_factor", "query", "device_status", "destroy"):
                getattr(L, "prism_proj_" + name).restype = i
            L.prism_plan_create.argtypes = [P, i, i, i, ctypes.POINTER(P)]
            L.prism_plan_launch.argtypes = [P, P]
            L.prism_plan_query.argtypes = [P, i, ctypes.POINTER(ll)]
            L.prism_plan_destroy.argtypes = [P]
            for name in ("create", "launch", "query", "destroy"):
                getattr(L, "prism_plan_" + name).restype = i
            L.prism_proj_describe.argtypes = [P, P, P]
            L.prism_proj_describe.restype = i
            sz = ctypes.c_size_t
            L.prism_server_create.argtypes = [sz, i, d, ctypes.POINTER(P)]
            L.prism_server_create_ex.argtypes = [sz, i, d, i, ctypes.POINTER(P)]
            L.prism_server_create_ex.restype = i
            L.prism_server_add_controller.argtypes = [P, P, i, i, i, ctypes.POINTER(i)]
            L.prism_server_submit.argtypes = [P, i, P, P, P, P, P, ctypes.POINTER(ctypes.c_ulonglong)]
            L.prism_server_wait.argtypes = [P, ctypes.c_ulonglong, d, ctypes.POINTER(i),
                                            ctypes.POINTER(d)]
            L.prism_server_stats.argtypes = [P, P]
            L.prism_server_reset_stats.argtypes = [P]
            L.prism_server_destroy.argtypes = [P]
            for name in ("create", "add_controller", "submit", "wait", "stats", "reset_stats", "destroy"):
                getattr(L, "prism_server_" + name).restype = i
            L.prism_mppi_workspace_bytes.argtypes = [i, i, i]
            L.prism_mppi_workspace_bytes.restype = ctypes.c_size_t
            L.prism_mppi_update.argtypes = [i, i, i, P, d, d, P, P, P, P, P, ctypes.c_size_t, P]
            L.prism_mppi_update.restype = i
            L.prism_ws_create.argtypes = [P, i, P, P, ctypes.POINTER(P)]
            L.prism_ws_accumulate.argtypes = [P, i, P, P, P, P, P, P]
            L.prism_ws_fit.argtypes = [P, d, P]
            L.prism_ws_predict.argtypes = [P, i, P, P, P, P, P, i, P]
            L.prism_ws_get.argtypes = [P, P, P, P, ctypes.POINTER(ll)]
            L.prism_ws_reset.argtypes = [P]
            L.prism_ws_destroy.argtypes = [P]
            for name in ("create", "accumulate", "fit", "predict", "get", "reset", "destroy"):
                getattr(L, "prism_ws_" + name).restype = i
            L.prism_status_string.argtypes = [i]
            L.prism_status_string.restype = ctypes.c_char_p
            L.prism_last_error.argtypes = []
            L.prism_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise PrismError(status, lib().prism_last_error().decode())


def _ptr(t):
    """Device (or host) pointer of a tensor / array, None passes NULL."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _need_cuda_f32(name, t, shape):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError(f"{name} must be a CUDA float32 tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Projector:
    """One projector per (J, H, dt, bounds): prism_proj_create / factor / solve."""

    def __init__(self, J: int, H: int, dt: float, bounds):
        b = np.ascontiguousarray(np.asarray(bounds, dtype=np.float64).reshape(8, J))
        self.J, self.H, self.dt = int(J), int(H), float(dt)
        self.bounds = b
        self._rows = [np.ascontiguousarray(b[r]) for r in range(8)]
        h = ctypes.c_void_p()
        _check(lib().prism_proj_create(self.J, self.H, self.dt,
                                       *[_ptr(r) for r in self._rows], ctypes.byref(h)))
        self._h = h
        self.rho = None
        self.mode = None

    # ------------------------------------------------------------------
    def factor(self, rho: float = 1.0, mode: int = MODE_ADMM, scale: int = SCALE_ROWNORM,
               prec: int = PREC_FP32, stream=None):
        _check(lib().prism_proj_factor(self._h, float(rho), int(mode), int(scale), int(prec),
                                       _stream_ptr(stream)))
        self.rho, self.mode, self.scale = float(rho), int(mode), int(scale)
        return self

    def _outputs(self, N, out, primal, dual, want_res):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        if out is None:
            out = torch.empty((N, self.H, self.J), dtype=torch.float32, device=dev)
        if want_res and primal is None:
            primal = torch.empty((N, self.J), dtype=torch.float32, device=dev)
        if want_res and dual is None:
            dual = torch.empty((N, self.J), dtype=torch.float32, device=dev)
        return out, primal, dual

    def _solve(self, fn, q0, v0, samples, iters, rho, out, primal, dual, stream, want_res):
        N = int(samples.shape[0])
        _need_cuda_f32("samples", samples, (N, self.H, self.J))
        _need_cuda_f32("q0", q0, (self.J,))
        _need_cuda_f32("v0", v0, (self.J,))
        out, primal, dual = self._outputs(N, out, primal, dual, want_res)
        _need_cuda_f32("out", out, (N, self.H, self.J))
        if primal is not None:
            _need_cuda_f32("primal", primal, (N, self.J))
        if dual is not None:
            _need_cuda_f32("dual", dual, (N, self.J))
        rho = self.rho if rho is None else rho
        _check(fn(self._h, N, _ptr(q0), _ptr(v0), _ptr(samples), int(iters), float(rho), _ptr(out),
                  _ptr(primal), _ptr(dual), _stream_ptr(stream)))
        return out, primal, dual

    def solve(self, q0, v0, samples, iters: int, rho: float | None = None, out=None, primal=None,
              dual=None, stream=None, want_res: bool = True):
        """prism_proj_solve: returns (x, primal_res, dual_res) as CUDA tensors."""
        return self._solve(lib().prism_proj_solve, q0, v0, samples, iters, rho, out, primal, dual,
                           stream, want_res)

    def dual_rows(self) -> int:
        """Multiplier rows per column of the factored mode (4H-1 ADMM, H PAPER)."""
        return 4 * self.H - 1 if self.mode == MODE_ADMM else self.H

    def solve_ex(self, q0, v0, samples, iters: int, rho: float | None = None, x_init=None,
                 dual_init=None, dual_out=None, polish_iters: int = 0, out=None, primal=None,
                 dual=None, stream=None, want_res: bool = True, want_dual_out: bool = False,
                 init_layout: int = 0):
        """prism_proj_solve_ex: warm start (x_init, dual_init) and multiplier export.
        init_layout INIT_COLUMN_MAJOR takes x_init [H][N*J] and dual_init [D][N*J]."""
        import torch
        N = int(samples.shape[0])
        D = self.dual_rows()
        cm = init_layout == INIT_COLUMN_MAJOR
        if x_init is not None:
            _need_cuda_f32("x_init", x_init, (self.H, N * self.J) if cm else (N, self.H, self.J))
        if dual_init is not None:
            _need_cuda_f32("dual_init", dual_init, (D, N * self.J) if cm else (N, D, self.J))
        if want_dual_out and dual_out is None:
            dual_out = torch.empty((N, D, self.J), dtype=torch.float32, device=samples.device)
        if dual_out is not None:
            _need_cuda_f32("dual_out", dual_out, (N, D, self.J))
        opts = SolveOpts(None if x_init is None else x_init.data_ptr(),
                         None if dual_init is None else dual_init.data_ptr(),
                         None if dual_out is None else dual_out.data_ptr(), int(polish_iters), int(init_layout))
        L = lib()

        def fn(h, n, a, b_, c, it, r, o, pr, du, st):
            return L.prism_proj_solve_ex(h, n, a, b_, c, it, r, ctypes.byref(opts), o, pr, du, st)

        x, pr, du = self._solve(fn, q0, v0, samples, iters, rho, out, primal, dual, stream, want_res)
        return x, pr, du, dual_out

    def sample_solve(self, q0, v0, mean, std, N: int, iters: int, seed: int, stream_id: int,
                     rho: float | None = None, want_samples: bool = False, stream=None):
        """prism_proj_sample_solve: draw N samples of N(mean, std^2) on the device and project
        them; returns (x, primal, dual, samples or None)."""
        import torch
        _need_cuda_f32("q0", q0, (self.J,))
        _need_cuda_f32("v0", v0, (self.J,))
        _need_cuda_f32("mean", mean, (self.H, self.J))
        _need_cuda_f32("std", std, (self.H, self.J))
        out, primal, dual = self._outputs(N, None, None, None, True)
        xs = torch.empty((N, self.H, self.J), dtype=torch.float32, device=mean.device) if want_samples else None
        rho = self.rho if rho is None else rho
        _check(lib().prism_proj_sample_solve(self._h, int(N), _ptr(q0), _ptr(v0), _ptr(mean), _ptr(std),
                                             int(seed), int(stream_id), int(iters), float(rho), _ptr(out),
                                             _ptr(xs), _ptr(primal), _ptr(dual), _stream_ptr(stream)))
        return out, primal, dual, xs

    def solve_plain(self, q0, v0, samples, iters: int, rho: float | None = None, out=None,
                    primal=None, dual=None, stream=None, want_res: bool = True):
        """prism_proj_solve_plain (the plain FP32 comparator)."""
        return self._solve(lib().prism_proj_solve_plain, q0, v0, samples, iters, rho, out, primal,
                           dual, stream, want_res)

    def solve_host(self, q0, v0, samples, iters: int, rho: float | None = None, out=None,
                   primal=None, dual=None, stream=None, want_res: bool = True):
        """prism_proj_solve_host on host float32 arrays (numpy or pinned CPU tensors)."""
        import torch
        N = int(samples.shape[0])

        def host(a, shape):
            if isinstance(a, torch.Tensor):
                assert a.device.type == "cpu" and a.dtype == torch.float32 and a.is_contiguous()
                assert tuple(a.shape) == tuple(shape)
                return a
            a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
            assert a.shape == tuple(shape)
            return a

        samples = host(samples, (N, self.H, self.J))
        q0 = host(q0, (self.J,))
        v0 = host(v0, (self.J,))
        if out is None:
            out = np.empty((N, self.H, self.J), dtype=np.float32)
        if want_res and primal is None:
            primal = np.empty((N, self.J), dtype=np.float32)
        if want_res and dual is None:
            dual = np.empty((N, self.J), dtype=np.float32)
        rho = self.rho if rho is None else rho
        _check(lib().prism_proj_solve_host(self._h, N, _ptr(q0), _ptr(v0), _ptr(samples), int(iters),
                                           float(rho), _ptr(out), _ptr(primal), _ptr(dual),
                                           _stream_ptr(stream)))
        return out, primal, dual

    def shift_state(self, steps: int, x=None, dual=None, stream=None):
        """prism_proj_shift_state: in-place receding-horizon shift of x and/or dual."""
        N = int((x if x is not None else dual).shape[0])
        if x is not None:
            _need_cuda_f32("x", x, (N, self.H, self.J))
        if dual is not None:
            _need_cuda_f32("dual", dual, (N, self.dual_rows(), self.J))
        _check(lib().prism_proj_shift_state(self._h, N, int(steps), _ptr(x), _ptr(dual),
                                            _stream_ptr(stream)))

    def device_status(self, stream=None):
        """prism_proj_device_status: synchronise ``stream`` and raise PrismError
        (PRISM_ERR_TIMEOUT) if a launch of this handle hit a device-side wait bound."""
        _check(lib().prism_proj_device_status(self._h, _stream_ptr(stream)))

    def check_fp64(self, q0, v0, x, stream=None):
        """prism_proj_check_fp64: FP64 primal residual [N, J] (CUDA float64 tensor)."""
        import torch
        N = int(x.shape[0])
        _need_cuda_f32("x", x, (N, self.H, self.J))
        res = torch.empty((N, self.J), dtype=torch.float64, device=x.device)
        _check(lib().prism_proj_check_fp64(self._h, N, _ptr(q0), _ptr(v0), _ptr(x), _ptr(res),
                                           _stream_ptr(stream)))
        return res

    def get_factor(self):
        """(K [H,H], kb [H]) in float64, copied from the device."""
        K = np.zeros((self.H, self.H))
        kb = np.zeros(self.H)
        _check(lib().prism_proj_get_factor(self._h, _ptr(K), _ptr(kb)))
        return K, kb

    def set_tiling(self, warps: int):
        """prism_proj_set_tiling: 0 default, 4 / 8 (four quarters), 16 (eight quarters)."""
        _check(lib().prism_proj_set_tiling(self._h, int(warps)))
        return self

    def set_host_chunks(self, chunks: int):
        """prism_proj_set_host_chunks: 0 automatic, 1 one solve on the mapped buffers, else chunks."""
        _check(lib().prism_proj_set_host_chunks(self._h, int(chunks)))
        return self

    def query(self, batch: int) -> dict:
        out = (ctypes.c_longlong * 8)()
        _check(lib().prism_proj_query(self._h, int(batch), out))
        keys = ("cols_per_tile", "samples_per_tile", "blocks_per_sm", "grid", "smem_bytes",
                "regs_per_thread", "hq", "num_sms")
        return dict(zip(keys, [int(v) for v in out]))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(lib().prism_proj_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Plan:
    """prism_plan_*: many uneven problems solved by concurrent persistent launches.

    ``items`` is a list of dicts with keys proj (a factored Projector), q0, v0,
    samples, out and optionally primal, dual, x_init, dual_init, dual_out (CUDA
    float32 tensors in the single-solve layouts).  The tensors must stay alive
    and in place while the plan exists.
    """

    def __init__(self, items, iters: int, autotune: bool = False, graph: bool = False):
        self._keep = items
        arr = (Problem * len(items))()
        for k, it in enumerate(items):
            P = it["proj"]
            N = int(it["samples"].shape[0])
            arr[k].h = P._h.value
            arr[k].batch = N
            for name in ("q0", "v0", "samples", "out", "primal", "dual", "x_init", "dual_init",
                         "dual_out"):
                t = it.get(name)
                field = {"primal": "primal_res", "dual": "dual_res"}.get(name, name)
                setattr(arr[k], field, None if t is None else t.data_ptr())
        self._arr = arr
        flags = (PLAN_AUTOTUNE if autotune else 0) | (PLAN_GRAPH if graph else 0)
        h = ctypes.c_void_p()
        _check(lib().prism_plan_create(ctypes.cast(arr, ctypes.c_void_p), len(items), int(iters), flags,
                                       ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(lib().prism_plan_launch(self._h, _stream_ptr(stream)))

    def query(self):
        out = (ctypes.c_longlong * 8)()
        _check(lib().prism_plan_query(self._h, -1, out))
        info = {"groups": [], "graph": bool(out[1]), "num_sms": int(out[2])}
        for g in range(int(out[0])):
            o = (ctypes.c_longlong * 8)()
            _check(lib().prism_plan_query(self._h, g, o))
            info["groups"].append(dict(zip(("hq", "tensor_cores", "problems", "tiles", "grid",
                                            "blocks_per_sm", "smem_bytes", "autotune_us"),
                                           [int(v) for v in o])))
        return info

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(lib().prism_plan_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


REQUEST_STATES = {0: "queued", 1: "running", 2: "done", 3: "dropped", 4: "failed"}


class Server:
    """prism_server_*: continuous-batching request loop over many controllers.

    Host arrays passed to ``submit`` (numpy float32 or pinned CPU tensors) are
    kept referenced here until their ticket has been waited for.
    """

    def __init__(self, mem_budget_bytes: int = 8 << 30, max_inflight: int = 16,
                 deadline_ms: float = 20.0, plain: bool = False):
        h = ctypes.c_void_p()
        _check(lib().prism_server_create_ex(int(mem_budget_bytes), int(max_inflight), float(deadline_ms),
                                            1 if plain else 0, ctypes.byref(h)))
        self._h = h
        self._refs = {}
        self._projs = []

    def add_controller(self, proj: Projector, batch: int, iters: int, warm: bool = True) -> int:
        cid = ctypes.c_int()
        _check(lib().prism_server_add_controller(self._h, proj._h, int(batch), int(iters), int(bool(warm)),
                                                 ctypes.byref(cid)))
        self._projs.append(proj)
        return int(cid.value)

    def submit(self, cid: int, q0, v0, samples, out, primal=None) -> int:
        t = ctypes.c_ulonglong()
        _check(lib().prism_server_submit(self._h, int(cid), _ptr(q0), _ptr(v0), _ptr(samples), _ptr(out),
                                         _ptr(primal), ctypes.byref(t)))
        self._refs[int(t.value)] = (q0, v0, samples, out, primal)
        return int(t.value)

    def wait(self, ticket: int, timeout_ms: float = -1.0):
        st = ctypes.c_int()
        lat = ctypes.c_double()
        _check(lib().prism_server_wait(self._h, int(ticket), float(timeout_ms), ctypes.byref(st),
                                       ctypes.byref(lat)))
        state = REQUEST_STATES.get(int(st.value), int(st.value))
        if state in ("done", "dropped", "failed"):
            self._refs.pop(int(ticket), None)
        return state, float(lat.value)

    def stats(self) -> dict:
        out = (ctypes.c_double * 10)()
        _check(lib().prism_server_stats(self._h, ctypes.cast(out, ctypes.c_void_p)))
        keys = ("completed", "dropped", "failed", "p50_ms", "p99_ms", "max_ms", "deadline_misses",
                "trajectories", "trajectories_per_s", "free_bytes")
        return dict(zip(keys, [float(v) for v in out]))

    def reset_stats(self):
        _check(lib().prism_server_reset_stats(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(lib().prism_server_destroy(self._h))
            self._h = None
            self._refs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class WarmStart:
    """Learned warm start of an ADMM-mode Projector (prism_ws_*): a fixed random
    first layer (W1 [hidden][H+3], b1 [hidden]; drawn here from ``seed`` unless
    given) with a linear skip, output layer fitted by ridge regression on
    converged solves, evaluated on the tensor cores."""

    def __init__(self, proj: "Projector", hidden: int = 64, seed: int = 0, W1=None, b1=None):
        self.proj = proj
        self.J, self.H = proj.J, proj.H
        self.D = 4 * self.H - 1
        self.hidden = int(hidden)
        d = self.H + 3
        if self.hidden > 0 and W1 is None:
            rng = np.random.default_rng(seed)
            W1 = rng.normal(0.0, 1.0 / np.sqrt(d), size=(self.hidden, d))
            b1 = rng.uniform(-1.0, 1.0, size=self.hidden)
        self.W1 = None if W1 is None else np.ascontiguousarray(np.asarray(W1, dtype=np.float64).reshape(self.hidden, d))
        self.b1 = None if b1 is None else np.ascontiguousarray(np.asarray(b1, dtype=np.float64).reshape(self.hidden))
        h = ctypes.c_void_p()
        _check(lib().prism_ws_create(proj._h, self.hidden, _ptr(self.W1), _ptr(self.b1), ctypes.byref(h)))
        self._h = h

    @property
    def K2(self) -> int:
        return self.hidden + self.H + 3

    def accumulate(self, q0, v0, samples, x_star, dual_star, stream=None):
        N = int(samples.shape[0])
        _need_cuda_f32("q0", q0, (self.J,))
        _need_cuda_f32("v0", v0, (self.J,))
        _need_cuda_f32("samples", samples, (N, self.H, self.J))
        _need_cuda_f32("x_star", x_star, (N, self.H, self.J))
        _need_cuda_f32("dual_star", dual_star, (N, self.D, self.J))
        _check(lib().prism_ws_accumulate(self._h, N, _ptr(q0), _ptr(v0), _ptr(samples), _ptr(x_star),
                                         _ptr(dual_star), _stream_ptr(stream)))
        return self

    def fit(self, lam: float = 1e-3, stream=None):
        _check(lib().prism_ws_fit(self._h, float(lam), _stream_ptr(stream)))
        return self

    def predict(self, q0, v0, samples, x_init=None, dual_init=None, layout: int = INIT_SAMPLE_MAJOR,
                stream=None):
        """(x_init, dual_init) on the device: [N][H][J] and [N][D][J], or with
        layout INIT_COLUMN_MAJOR [H][N*J] and [D][N*J] (pass the same layout to
        Projector.solve_ex)."""
        import torch
        N = int(samples.shape[0])
        _need_cuda_f32("q0", q0, (self.J,))
        _need_cuda_f32("v0", v0, (self.J,))
        _need_cuda_f32("samples", samples, (N, self.H, self.J))
        cm = layout == INIT_COLUMN_MAJOR
        xs = (self.H, N * self.J) if cm else (N, self.H, self.J)
        us = (self.D, N * self.J) if cm else (N, self.D, self.J)
        if x_init is None:
            x_init = torch.empty(xs, dtype=torch.float32, device=samples.device)
        if dual_init is None:
            dual_init = torch.empty(us, dtype=torch.float32, device=samples.device)
        _need_cuda_f32("x_init", x_init, xs)
        _need_cuda_f32("dual_init", dual_init, us)
        _check(lib().prism_ws_predict(self._h, N, _ptr(q0), _ptr(v0), _ptr(samples), _ptr(x_init),
                                      _ptr(dual_init), int(layout), _stream_ptr(stream)))
        return x_init, dual_init

    def get(self, want_w2: bool = True):
        """Host copies: dict(S [K2][K2], T [K2][D+H], W2 or None, n)."""
        K2, NO = self.K2, self.D + self.H
        S = np.empty((K2, K2))
        T = np.empty((K2, NO))
        W2 = np.empty((K2, NO)) if want_w2 else None
        n = ctypes.c_longlong()
        _check(lib().prism_ws_get(self._h, _ptr(S), _ptr(T), _ptr(W2), ctypes.byref(n)))
        return {"S": S, "T": T, "W2": W2, "n": int(n.value)}

    def reset(self):
        _check(lib().prism_ws_reset(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().prism_ws_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def test_fail_allocs(skip: int, count: int) -> None:
    """prism_test_fail_allocs: after ``skip`` device allocations of the library, fail
    the next ``count`` as out-of-memory (host-side fault injection; (0, 0) = off)."""
    lib().prism_test_fail_allocs(int(skip), int(count))


def test_set_device_flag(proj: "Projector", value: int = 1) -> None:
    """prism_test_set_device_flag: write the handle's device-side timeout flag from
    the host (what a solve whose bounded wait ran out leaves behind)."""
    _check(lib().prism_test_set_device_flag(proj._h, int(value)))


def diag_wait_timeout(poll_limit: int = 1000) -> bool:
    """prism_diag_wait_timeout: run the bounded device wait on a phase that nothing
    completes; True when the bound ran out (the expected outcome)."""
    flag = ctypes.c_int(-1)
    _check(lib().prism_diag_wait_timeout(int(poll_limit), ctypes.byref(flag)))
    return flag.value == 1


def mppi_update(cost, x, temperature: float, eps: float = 0.0, workspace=None, stream=None):
    """prism_mppi_update: (mean [H,J], var [H,J], weights [N]) from costs [N] and x [N,H,J]."""
    import torch
    N, H, J = (int(v) for v in x.shape)
    _need_cuda_f32("x", x, (N, H, J))
    _need_cuda_f32("cost", cost, (N,))
    nbytes = int(lib().prism_mppi_workspace_bytes(N, H, J))
    if workspace is None:
        workspace = torch.empty(max(1, nbytes // 4 + 1), dtype=torch.float32, device=x.device)
    mean = torch.empty((H, J), dtype=torch.float32, device=x.device)
    var = torch.empty((H, J), dtype=torch.float32, device=x.device)
    w = torch.empty((N,), dtype=torch.float32, device=x.device)
    _check(lib().prism_mppi_update(N, H, J, _ptr(cost), float(temperature), float(eps), _ptr(x), _ptr(mean),
                                   _ptr(var), _ptr(w), _ptr(workspace), workspace.numel() * 4,
                                   _stream_ptr(stream)))
    return mean, var, w
