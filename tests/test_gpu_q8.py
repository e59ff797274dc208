"""The eight-quarter solve kernel (ADMM on the tensor cores, 52 < H <= 104,
selected with prism_proj_set_tiling(16)): eight threads per column, every
cross-quarter term through the MMA.  Shapes at its boundaries (first and last
horizon of each chunk, quarters without real rows, ragged column tiles), warm
starts with multiplier export, on-device sampling and the launch facts, all
against the FP64 oracle; the other tilings on the same problems too."""
import numpy as np
import pytest

import oracle
from paper_2608_25666_b300 import prism_proj as pp
from paper_2608_25666_b300 import workloads
from gpu_helpers import assert_parity, oracle_solve, to_dev

pytestmark = pytest.mark.gpu

SHAPES = [
    # N, J, H, dt, iters
    (5, 12, 53, 0.02, 60),       # first horizon of the 9-step chunk; 60 columns (one partial tile)
    (40, 7, 72, 0.02, 50),       # all eight quarters full; 280 columns (4 tiles + 24)
    (9, 14, 73, 0.05, 40),       # 13-step chunk, quarters 6 and 7 without real rows
    (3, 6, 88, 0.01, 45),
    (17, 5, 104, 0.02, 30),      # largest horizon of the kernel
    (1, 1, 64, 0.02, 20),        # one column
]


def solve_tiled(b, iters, warps, rho=1.0):
    import torch
    P = pp.Projector(b["J"], b["H"], b["dt"], b["bounds"]).factor(rho, prec=pp.PREC_TF32X3).set_tiling(warps)
    xi, q0, v0 = to_dev(b)
    x, pr, du = P.solve(q0, v0, xi, iters)
    torch.cuda.synchronize()
    q = P.query(b["xi"].shape[0])
    P.close()
    return {"x": x.cpu().numpy().astype(np.float64), "primal": pr.cpu().numpy().astype(np.float64),
            "dual": du.cpu().numpy().astype(np.float64)}, q


@pytest.mark.parametrize("N,J,H,dt,iters", SHAPES)
def test_q8_matches_oracle(N, J, H, dt, iters):
    b = workloads.make_custom(500 + H, N, J, H, dt, scale=0.8)
    o = oracle_solve(b, iters, 1.0)
    g, q = solve_tiled(b, iters, 16)
    assert q["cols_per_tile"] == 64 and q["hq"] in (9, 13) and 8 * q["hq"] >= H
    assert_parity(g, o, dual_tol=2e-4)
    assert np.all(g["x"][:, 0, :] == b["v0"][None, :].astype(np.float64))
    for warps in (4, 8):   # the four-quarter tilings on the same problem
        g4, q4 = solve_tiled(b, iters, warps)
        assert q4["cols_per_tile"] == 8 * warps
        assert_parity(g4, o, dual_tol=2e-4)


def test_tiling_choices_are_validated():
    P = pp.Projector(3, 40, 0.02, workloads.base_bounds(3))
    with pytest.raises(pp.PrismError) as e:
        P.set_tiling(16)            # H = 40 is below the eight-quarter range
    assert e.value.status == 7
    with pytest.raises(pp.PrismError) as e:
        P.set_tiling(5)
    assert e.value.status == 1
    P.close()


@pytest.mark.parametrize("H", [64, 97])
def test_q8_warm_start_and_multiplier_export(H):
    import torch
    N, J, dt = 23, 12, 0.02
    b = workloads.make_custom(H + 1, N, J, H, dt)
    P = pp.Projector(J, H, dt, b["bounds"]).factor(1.3, pp.MODE_ADMM, pp.SCALE_ROWNORM, pp.PREC_TF32X3)
    P.set_tiling(16)
    xi, q0, v0 = to_dev(b)
    x1, _, _, u1 = P.solve_ex(q0, v0, xi, 40, want_dual_out=True)
    o1 = oracle.solve_batch(b["xi"], b["q0"], b["v0"], b["bounds"], dt, 40, 1.3, want_dual_state=True, nthreads=8)
    torch.cuda.synchronize()
    assert float(np.max(np.abs(u1.cpu().numpy() - o1["dual_state"]))) <= 1e-3
    b2 = workloads.make_custom(H + 2, N, J, H, dt)
    xi2 = torch.from_numpy(b2["xi"]).cuda()
    x2, p2, d2, u2 = P.solve_ex(q0, v0, xi2, 40, x_init=x1, dual_init=u1, want_dual_out=True)
    torch.cuda.synchronize()
    o2 = oracle.solve_batch(b2["xi"], b["q0"], b["v0"], b["bounds"], dt, 40, 1.3, x_init=x1.cpu().numpy(),
                            dual_init=u1.cpu().numpy(), want_dual_state=True, nthreads=8)
    g2 = {"x": x2.cpu().numpy().astype(np.float64), "primal": p2.cpu().numpy().astype(np.float64),
          "dual": d2.cpu().numpy().astype(np.float64)}
    assert_parity(g2, o2, dual_tol=2e-4)
    assert float(np.max(np.abs(u2.cpu().numpy() - o2["dual_state"]))) <= 1e-3
    P.close()


def test_q8_sampling_matches_oracle():
    import torch
    N, J, H, seed, stream = 50, 6, 81, 17, 4
    b = workloads.make_custom(3, 1, J, H, 0.02)
    rng = np.random.default_rng(5)
    mean = rng.normal(0, 0.3, (H, J)).astype(np.float32)
    std = rng.uniform(0.5, 2.0, (H, J)).astype(np.float32)
    P = pp.Projector(J, H, 0.02, b["bounds"]).factor(1.0, prec=pp.PREC_TF32X3).set_tiling(16)
    x, pr, du, xs = P.sample_solve(torch.from_numpy(b["q0"]).cuda(), torch.from_numpy(b["v0"]).cuda(),
                                   torch.from_numpy(mean).cuda(), torch.from_numpy(std).cuda(), N, 50,
                                   seed, stream, want_samples=True)
    torch.cuda.synchronize()
    ref_xi = oracle.sample_batch(N, H, J, mean, std, seed, stream)
    assert np.max(np.abs(xs.cpu().numpy() - ref_xi)) <= 1e-5 * (1 + np.max(np.abs(ref_xi)))
    o = oracle.solve_batch(ref_xi, b["q0"], b["v0"], b["bounds"], 0.02, 50, 1.0, nthreads=8)
    g = {"x": x.cpu().numpy().astype(np.float64), "primal": pr.cpu().numpy().astype(np.float64),
         "dual": du.cpu().numpy().astype(np.float64)}
    assert_parity(g, o)
    P.close()
