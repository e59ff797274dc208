"""Three-way bf16 split K-apply (PRISM_PREC_BF16X3) vs the FP64 oracle.

Both operands of the K-apply are carried as three bf16 parts and multiplied on
the tensor cores (kind::f16, FP32 accumulation); every product of the parts
but the one of the two smallest is formed, so the K-apply is FP32-accurate and
the same bar as every other solve path applies: max |x_gpu - x_oracle| <= 1e-4
rad/s and |primal_gpu - primal_oracle| <= 1e-5 after the same iterations.
"""
import numpy as np
import pytest

import oracle
from paper_2608_25666_b300 import prism_proj as pp
from paper_2608_25666_b300 import workloads
from gpu_helpers import TC_MAX_H, assert_parity, gpu_solve, oracle_solve, to_dev

pytestmark = pytest.mark.gpu

BF = pp.PREC_BF16X3


def _host(x, pr, du):
    import torch
    torch.cuda.synchronize()
    return {"x": x.cpu().numpy().astype(np.float64), "primal": pr.cpu().numpy().astype(np.float64),
            "dual": du.cpu().numpy().astype(np.float64)}


@pytest.mark.parametrize("N,J,H,dt,iters", [
    (1, 1, 2, 0.05, 50),
    (3, 1, 3, 0.05, 40),
    (7, 5, 17, 0.02, 60),        # one ragged tile
    (20, 7, 45, 0.01, 80),       # J does not divide 64: 63-column tiles
    (9, 64, 12, 0.05, 30),       # one sample per tile
    (13, 14, 64, 0.02, 50),
    (11, 12, 50, 0.02, 0),       # no iteration: x^0
    (11, 12, 50, 0.02, 1),
    (40, 6, 21, 0.05, 25),
])
def test_bf16x3_edge_shapes(N, J, H, dt, iters):
    b = workloads.make_custom(7 + N + J + H, N, J, H, dt, scale=0.7)
    g = gpu_solve(b, iters, 1.0, prec=BF)
    o = oracle_solve(b, iters, 1.0)
    assert_parity(g, o, dual_tol=2e-4)
    assert np.all(g["x"][:, 0, :] == b["v0"][None, :].astype(np.float64))


@pytest.mark.parametrize("H", [10, 20, 28, 36, 44, 60, 68, 84, 100, TC_MAX_H])
def test_bf16x3_every_variant(H):
    """One horizon per kernel variant (quarters of 3 .. 29 steps), ragged tiles,
    rho != 1."""
    b = workloads.make_custom(500 + H, 11, 6, H, 0.02, scale=0.8)
    g = gpu_solve(b, 40, 1.3, prec=BF)
    o = oracle_solve(b, 40, 1.3)
    assert_parity(g, o, dual_tol=2e-4)


def test_bf16x3_realistic_full_size_sampled():
    """N=4096, J=12, H=50, dt=0.02, 100 iterations; 400 sampled columns (and the
    first and last) against the oracle, properties on all."""
    w = workloads.WORKLOADS["realistic"]
    b = workloads.make_batch(w, step=5)
    g = gpu_solve(b, w.iters, w.rho, prec=BF)
    rng = np.random.default_rng(1)
    cols = np.sort(rng.choice(w.N * w.J, 400, replace=False))
    cols = np.concatenate([cols, [0, w.N * w.J - 1]])
    o = oracle_solve(b, w.iters, w.rho, cols=cols)
    assert_parity(g, o, cols=cols, dual_tol=2e-4)
    assert np.all(np.isfinite(g["x"]))
    assert np.all(g["primal"] >= 0) and np.all(g["dual"] >= 0)


def test_bf16x3_precision_workload_shape():
    """J=14, H=64, dt=0.02, 100 + 20 iterations (the precision workload's shape
    and iteration count) on every column of 256 samples."""
    b = workloads.make_custom(91, 256, 14, 64, 0.02)
    g = gpu_solve(b, 120, 1.0, prec=BF)
    o = oracle_solve(b, 120, 1.0)
    dx, dv = assert_parity(g, o)
    print(f"bf16x3 at J=14 H=64, 120 iterations: max|dx| {dx:.3e}, max|dviol| {dv:.3e}")


def test_bf16x3_warm_start_sampling_and_host_buffers():
    """A warm-started second solve (iterate and multiplier of the first, in the
    oracle's units) against the oracle given the same warm start; the fused
    sampling entry point and the host-buffer entry point equal the device
    solve of the same samples."""
    import torch
    b = workloads.make_custom(77, 23, 12, 30, 0.05)
    P = pp.Projector(12, 30, 0.05, b["bounds"]).factor(1.0, pp.MODE_ADMM, pp.SCALE_ROWNORM, BF)
    xi, q0, v0 = to_dev(b)
    x1, _, _, u1 = P.solve_ex(q0, v0, xi, 40, want_dual_out=True)
    o1 = oracle.solve_batch(b["xi"], b["q0"], b["v0"], b["bounds"], 0.05, 40, 1.0, want_dual_state=True)
    torch.cuda.synchronize()
    assert float(np.max(np.abs(u1.cpu().numpy() - o1["dual_state"]))) <= 1e-3
    b2 = workloads.make_custom(78, 23, 12, 30, 0.05)
    xi2 = torch.from_numpy(b2["xi"]).cuda()
    x2, pr2, du2, _ = P.solve_ex(q0, v0, xi2, 30, x_init=x1, dual_init=u1)
    o2 = oracle.solve_batch(b2["xi"], b["q0"], b["v0"], b["bounds"], 0.05, 30, 1.0,
                            x_init=x1.cpu().numpy().astype(np.float64),
                            dual_init=u1.cpu().numpy().astype(np.float64))
    assert_parity(_host(x2, pr2, du2), o2, dual_tol=2e-4)

    mean = torch.zeros((30, 12), device="cuda")
    std = torch.full((30, 12), 1.5, device="cuda")
    xs_, prs, dus, drawn = P.sample_solve(q0, v0, mean, std, 23, 40, seed=7, stream_id=3, want_samples=True)
    xd, prd, dud = P.solve(q0, v0, drawn, 40)
    torch.cuda.synchronize()
    assert torch.equal(xs_, xd) and torch.equal(prs, prd)

    hx = xi.cpu().contiguous()
    hout = torch.empty_like(hx)
    P.solve_host(q0.cpu().contiguous(), v0.cpu().contiguous(), hx, 40, out=hout)
    assert torch.equal(hout, x1.cpu())
    P.close()


@pytest.mark.parametrize("N,J,H,dt,iters", [(1, 1, 2, 0.05, 50), (7, 5, 17, 0.02, 60), (20, 7, 45, 0.01, 80),
                                         (13, 14, 64, 0.02, 50), (3, 2, 101, 0.02, 40)])
def test_bf16x3_paper_mode(N, J, H, dt, iters):
    """The printed iteration (PAPER mode) with the bf16 split K-apply."""
    b = workloads.make_custom(99 + H, N, J, H, dt, scale=0.8)
    g = gpu_solve(b, iters, 0.7, mode=pp.MODE_PAPER, prec=BF)
    o = oracle_solve(b, iters, 0.7, mode=pp.MODE_PAPER)
    assert_parity(g, o)


def test_bf16x3_horizon_limit():
    """The bf16 split shares the tensor-core kernels' horizon limit."""
    P = pp.Projector(2, TC_MAX_H + 1, 0.02, workloads.base_bounds(2))
    with pytest.raises(pp.PrismError) as e:
        P.factor(1.0, pp.MODE_ADMM, pp.SCALE_ROWNORM, BF)
    assert e.value.status == 7
    P.close()


@pytest.mark.parametrize("autotune,graph", [(False, False), (True, True)])
def test_bf16x3_in_plans(autotune, graph):
    """Plans with bf16-split handles (several kernel variants, both modes, a
    ragged and an empty problem) next to split-TF32 and FP32 ones: each
    problem's result equals its own single solve (the autotuner never moves a
    bf16 group to another K-apply) and the oracle."""
    import torch
    shapes = [  # J, H, N, dt, mode, precision
        (6, 20, 130, 0.05, pp.MODE_ADMM, BF), (7, 45, 77, 0.01, pp.MODE_ADMM, BF),
        (12, 50, 300, 0.02, pp.MODE_ADMM, BF), (14, 64, 41, 0.02, pp.MODE_PAPER, BF),
        (6, 97, 50, 0.02, pp.MODE_ADMM, BF), (7, 28, 0, 0.02, pp.MODE_ADMM, BF),
        (12, 50, 64, 0.02, pp.MODE_ADMM, pp.PREC_TF32X3), (6, 20, 33, 0.05, pp.MODE_ADMM, pp.PREC_FP32)]
    iters = 50
    items, batches = [], []
    for k, (J, H, N, dt, mode, prec) in enumerate(shapes):
        b = workloads.make_custom(600 + 17 * k, N, J, H, dt, scale=0.9)
        P = pp.Projector(J, H, dt, b["bounds"]).factor(1.0, mode, pp.SCALE_ROWNORM, prec)
        items.append({"proj": P, "q0": torch.from_numpy(b["q0"]).cuda(), "v0": torch.from_numpy(b["v0"]).cuda(),
                      "samples": torch.from_numpy(b["xi"]).cuda(),
                      "out": torch.full((N, H, J), float("nan"), device="cuda"),
                      "primal": torch.full((N, J), float("nan"), device="cuda"),
                      "dual": torch.full((N, J), float("nan"), device="cuda")})
        batches.append((b, mode))
    plan = pp.Plan(items, iters, autotune=autotune, graph=graph)
    plan.launch()
    torch.cuda.synchronize()
    for it, (b, mode), shape in zip(items, batches, shapes):
        if shape[2] == 0:
            continue
        P = it["proj"]
        x, pr, du = P.solve(it["q0"], it["v0"], it["samples"], iters)
        torch.cuda.synchronize()
        if shape[5] == BF:
            assert float((it["out"] - x).abs().max()) <= 1e-6
            assert float((it["primal"] - pr).abs().max()) <= 1e-6
        g = _host(it["out"], it["primal"], it["dual"])
        assert_parity(g, oracle_solve(b, iters, 1.0, mode=mode))
    plan.close()
    for it in items:
        it["proj"].close()
