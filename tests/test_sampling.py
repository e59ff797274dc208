"""On-device sampling fused with the projection (Alg. 1, sample step):
Philox4x32-10 + Box-Muller, implemented independently by the oracle (C) and
the kernel.  CPU: the oracle generator against the published known-answer
vectors and normal statistics.  GPU: drawn samples and projections against
the oracle."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answer_vectors():
    n = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            assert list(oracle.philox4x32_10(v[:4], v[4:6])) == v[6:]
            n += 1
    assert n == 3


def test_oracle_normals_have_unit_moments_and_streams_differ():
    N, H, J = 2000, 25, 4
    z = oracle.sample_batch(N, H, J, np.zeros((H, J)), np.ones((H, J)), seed=123, stream=7)
    m, v = z.mean(), z.var()
    se = 1.0 / np.sqrt(z.size)
    assert abs(m) < 5 * se and abs(v - 1.0) < 5 * np.sqrt(2.0) * se
    assert abs(np.mean(z ** 3)) < 5 * np.sqrt(15.0) * se       # symmetric
    z2 = oracle.sample_batch(N, H, J, np.zeros((H, J)), np.ones((H, J)), seed=123, stream=8)
    z3 = oracle.sample_batch(N, H, J, np.zeros((H, J)), np.ones((H, J)), seed=123, stream=7)
    assert np.array_equal(z, z3) and not np.allclose(z, z2)
    x = oracle.sample_batch(3, H, J, np.full((H, J), 2.0), np.full((H, J), 0.5), seed=123, stream=7)
    np.testing.assert_allclose(x, 2.0 + 0.5 * z[:3], rtol=1e-15)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 3])    # FP32-pipe K-apply (whole-sample tiles), split TF32 (column tiles)
@pytest.mark.parametrize("N,J,H,seed,stream", [(301, 12, 30, 5, 0), (64, 7, 45, 2 ** 40 + 3, 2 ** 33 + 1),
                                               (1, 1, 2, 0, 0), (77, 5, 50, 11, 3)])
def test_device_sampling_and_projection_match_oracle(N, J, H, seed, stream, prec):
    import torch
    from paper_2608_25666_b300 import prism_proj as pp
    from paper_2608_25666_b300 import workloads
    from gpu_helpers import X_TOL, VIOL_TOL
    b = workloads.make_custom(N + H, 1, J, H, 0.05)
    rng = np.random.default_rng(H)
    mean = rng.normal(0, 0.3, (H, J)).astype(np.float32)
    std = rng.uniform(0.5, 2.0, (H, J)).astype(np.float32)
    P = pp.Projector(J, H, 0.05, b["bounds"]).factor(1.0, prec=prec)
    x, pr, du, xs = P.sample_solve(torch.from_numpy(b["q0"]).cuda(), torch.from_numpy(b["v0"]).cuda(),
                                   torch.from_numpy(mean).cuda(), torch.from_numpy(std).cuda(), N, 60,
                                   seed, stream, want_samples=True)
    torch.cuda.synchronize()
    ref_xi = oracle.sample_batch(N, H, J, mean, std, seed, stream)
    assert np.max(np.abs(xs.cpu().numpy() - ref_xi)) <= 1e-5 * (1 + np.max(np.abs(ref_xi)))
    o = oracle.solve_batch(ref_xi, b["q0"], b["v0"], b["bounds"], 0.05, 60, 1.0)
    assert np.max(np.abs(x.cpu().numpy() - o["x"])) <= X_TOL
    assert np.max(np.abs(pr.cpu().numpy() - o["primal"])) <= VIOL_TOL
    P.close()


SIGMA_BOUNDS = np.array([-1e6, 1e6, -1.0, 1.0, -2.0, 2.0, -4.0, 4.0]).reshape(8, 1)
SIGMA_TOL = 1e-3     # row-normalised violation below which a column counts as projected


def sigma_eff(x, primal, tol=SIGMA_TOL):
    """Pooled standard deviation of the projected velocities x_2..x_H over the
    columns whose violation is below tol; (sigma_eff, fraction of columns used)."""
    ok = primal.reshape(-1) <= tol
    v = x[ok][:, 1:, 0]
    return float(v.std()), float(ok.mean())


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 3])
def test_sigma_eff_diagnostic(prec):
    """Sec. III-C diagnostic on the device: single-joint samples of N(0, 10^2)
    drawn in the solve's prologue and projected under |v| <= 1, |a| <= 2,
    |j| <= 4 with v0 = 0 (no position bound), at rho = 64 (the same projection
    as any rho; it converges fastest for samples this far outside the set).
    Checks: the draw and the projection against the oracle column by column;
    every trajectory starts at v0; sigma_eff, computed on the columns whose
    violation is below SIGMA_TOL, equals the oracle's on the same columns; the
    projected velocities saturate at the bounds (the paper's qualitative
    finding) and sigma_eff is far below the sampling sigma."""
    import torch
    from paper_2608_25666_b300 import prism_proj as pp
    from gpu_helpers import X_TOL, VIOL_TOL
    N, H, dt, rho, iters, sigma = 256, 20, 0.1, 64.0, 3000, 10.0
    P = pp.Projector(1, H, dt, SIGMA_BOUNDS).factor(rho, prec=prec)
    z1 = torch.zeros(1, device="cuda")
    mean = torch.zeros((H, 1), device="cuda")
    std = torch.full((H, 1), sigma, device="cuda")
    x, pr, du, xs = P.sample_solve(z1, z1, mean, std, N, iters, seed=2026, stream_id=7, want_samples=True)
    torch.cuda.synchronize()
    xg, pg, xsg = x.cpu().numpy(), pr.cpu().numpy(), xs.cpu().numpy()
    ref_xi = oracle.sample_batch(N, H, 1, np.zeros((H, 1)), np.full((H, 1), sigma), 2026, 7)
    assert np.max(np.abs(xsg - ref_xi)) <= 1e-5 * (1 + np.max(np.abs(ref_xi)))
    o = oracle.solve_batch(xsg, [0.0], [0.0], SIGMA_BOUNDS, dt, iters, rho, nthreads=8)
    assert np.max(np.abs(xg - o["x"])) <= X_TOL
    assert np.max(np.abs(pg - o["primal"])) <= VIOL_TOL
    assert np.all(xg[:, 0, 0] == 0.0)
    s_gpu, frac = sigma_eff(xg, pg)
    ok = o["primal"].reshape(-1) <= SIGMA_TOL
    s_ora = float(o["x"][ok][:, 1:, 0].std())
    print(f"sigma_eff {s_gpu:.4f} (oracle {s_ora:.4f}) on {frac:.0%} of the columns, "
          f"max violation {pg.max():.2e}")
    assert frac >= 0.9
    assert abs(s_gpu - s_ora) <= 1e-4
    assert 0.05 < s_gpu < 1.0 < sigma
    used = xg[pg.reshape(-1) <= SIGMA_TOL][:, 1:, 0]
    assert np.mean(np.abs(used) >= 1.0 - 1e-3) > 0.05       # saturated at the velocity bounds (13 % in the oracle)
    assert np.max(np.abs(used)) <= 1.0 + 1e-3
    P.close()
