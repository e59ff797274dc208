"""Batched plans: uneven problems in concurrent persistent launches (one per
kernel variant), optionally autotuned and replayed from a CUDA graph.  Each
problem's result equals its own single solve and the FP64 oracle."""
import numpy as np
import pytest

from paper_2608_25666_b300 import prism_proj as pp
from paper_2608_25666_b300 import workloads
from gpu_helpers import VIOL_TOL, X_TOL, assert_parity, oracle_solve

pytestmark = pytest.mark.gpu

# (J, H, N, dt, scale, precision)
SHAPES = [
    (6, 20, 130, 0.05, 0.6, pp.PREC_FP32),
    (7, 45, 77, 0.01, 1.3, pp.PREC_FP32),
    (12, 50, 300, 0.02, 1.0, pp.PREC_TF32X3),
    (14, 64, 41, 0.02, 0.9, pp.PREC_TF32X3),
    (12, 100, 25, 0.05, 1.4, pp.PREC_FP32),
    (6, 120, 9, 0.01, 0.5, pp.PREC_FP32),
    (14, 33, 1, 0.05, 1.1, pp.PREC_TF32X3),
    (7, 28, 0, 0.02, 0.8, pp.PREC_FP32),        # empty problem
    (12, 50, 64, 0.02, 0.7, pp.PREC_FP32),
    (6, 97, 50, 0.02, 1.2, pp.PREC_TF32X3),
]


def make_items(iters, seed=0):
    import torch
    items, batches = [], []
    for k, (J, H, N, dt, scale, prec) in enumerate(SHAPES):
        b = workloads.make_custom(seed + 31 * k, N, J, H, dt, scale=scale)
        P = pp.Projector(J, H, dt, b["bounds"]).factor(1.0, pp.MODE_ADMM, pp.SCALE_ROWNORM, prec)
        it = {"proj": P, "q0": torch.from_numpy(b["q0"]).cuda(), "v0": torch.from_numpy(b["v0"]).cuda(),
              "samples": torch.from_numpy(b["xi"]).cuda(),
              "out": torch.full((N, H, J), float("nan"), device="cuda"),
              "primal": torch.full((N, J), float("nan"), device="cuda"),
              "dual": torch.full((N, J), float("nan"), device="cuda")}
        items.append(it)
        batches.append(b)
    return items, batches


@pytest.mark.parametrize("autotune,graph", [(False, False), (True, False), (False, True), (True, True)])
def test_plan_matches_single_solves_and_oracle(autotune, graph):
    import torch
    iters = 60
    items, batches = make_items(iters, seed=7)
    plan = pp.Plan(items, iters, autotune=autotune, graph=graph)
    info = plan.query()
    assert info["graph"] == graph
    assert sum(g["problems"] for g in info["groups"]) == sum(1 for s in SHAPES if s[2] > 0)
    for it in items:
        it["out"].fill_(float("nan"))
    plan.launch()
    plan.launch()      # a replay gives the same result
    torch.cuda.synchronize()
    for it, b, shape in zip(items, batches, SHAPES):
        P = it["proj"]
        N = shape[2]
        if N == 0:
            continue
        x, pr, du = P.solve(it["q0"], it["v0"], it["samples"], iters)
        torch.cuda.synchronize()
        # the autotuner may pick the other FP32-accurate K-apply path for a group
        close = X_TOL if autotune else 1e-5
        assert float((it["out"] - x).abs().max()) <= close
        assert float((it["primal"] - pr).abs().max()) <= (VIOL_TOL if autotune else 1e-6)
        g = {"x": it["out"].cpu().numpy().astype(np.float64),
             "primal": it["primal"].cpu().numpy().astype(np.float64),
             "dual": it["dual"].cpu().numpy().astype(np.float64)}
        ncols = N * shape[0]
        cols = np.unique(np.linspace(0, ncols - 1, min(ncols, 24)).astype(np.int64))
        o = oracle_solve(b, iters, 1.0, cols=cols)
        assert_parity(g, o, cols=cols, dual_tol=2e-4)
    plan.close()
    for it in items:
        it["proj"].close()


def test_plan_rejects_bad_problems():
    import torch
    b = workloads.make_custom(1, 4, 6, 20, 0.05)
    P = pp.Projector(6, 20, 0.05, b["bounds"])      # not factored
    item = {"proj": P, "q0": torch.zeros(6, device="cuda"), "v0": torch.zeros(6, device="cuda"),
            "samples": torch.zeros((4, 20, 6), device="cuda"), "out": torch.zeros((4, 20, 6), device="cuda")}
    with pytest.raises(pp.PrismError) as e:
        pp.Plan([item], 10)
    assert e.value.status == 2
    P.close()


def test_autotune_reports_a_flag_raised_on_any_problem():
    """Autotuning reads the timeout flag of every distinct handle (the launches
    write each tile's flag to its own problem's handle).  A flag written from
    the host on the LAST problem's handle fails plan creation with
    PRISM_ERR_TIMEOUT and is cleared; the next creation succeeds."""
    iters = 10
    items, _ = make_items(iters, seed=3)
    pp.test_set_device_flag(items[-1]["proj"], 1)
    with pytest.raises(pp.PrismError) as e:
        pp.Plan(items, iters, autotune=True)
    assert e.value.status == 8
    plan = pp.Plan(items, iters, autotune=True)
    plan.close()
    for it in items:
        it["proj"].device_status()
        it["proj"].close()


def test_plan_with_warm_starts_matches_single_solves():
    """Problems that start from x_init / dual_init (a previous solve's iterate and
    exported multiplier) run the plan group's warm-start kernel; each result
    equals the single warm-started solve, and the cold members of the same plan
    equal their single cold solves."""
    import torch
    iters = 40
    items, batches = make_items(iters, seed=11)
    warm_idx = [2, 3, 5]       # tensor-core and FP32-pipe problems
    for k in warm_idx:
        it = items[k]
        x1, _, _, u1 = it["proj"].solve_ex(it["q0"], it["v0"], it["samples"], 25, want_dual_out=True)
        it["x_init"], it["dual_init"] = x1.clone(), u1.clone()
        # the warm start is applied to fresh samples of the same shape
        it["samples"] = (it["samples"] + 0.3).contiguous()
    torch.cuda.synchronize()
    plan = pp.Plan(items, iters)
    plan.launch()
    torch.cuda.synchronize()
    for k, (it, shape) in enumerate(zip(items, SHAPES)):
        if shape[2] == 0:
            continue
        P = it["proj"]
        if k in warm_idx:
            x, pr, _, _ = P.solve_ex(it["q0"], it["v0"], it["samples"], iters, x_init=it["x_init"],
                                     dual_init=it["dual_init"])
        else:
            x, pr, _ = P.solve(it["q0"], it["v0"], it["samples"], iters)
        torch.cuda.synchronize()
        assert float((it["out"] - x).abs().max()) <= 1e-5, k
        assert float((it["primal"] - pr).abs().max()) <= 1e-6, k
    plan.close()
    for it in items:
        it["proj"].close()
