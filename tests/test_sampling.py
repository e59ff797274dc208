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
@pytest.mark.parametrize("N,J,H,seed,stream", [(301, 12, 30, 5, 0), (64, 7, 45, 2 ** 40 + 3, 2 ** 33 + 1),
                                               (1, 1, 2, 0, 0)])
def test_device_sampling_and_projection_match_oracle(N, J, H, seed, stream):
    import torch
    from paper_2608_25666_b300 import prism_proj as pp
    from paper_2608_25666_b300 import workloads
    from gpu_helpers import X_TOL, VIOL_TOL
    b = workloads.make_custom(N + H, 1, J, H, 0.05)
    rng = np.random.default_rng(H)
    mean = rng.normal(0, 0.3, (H, J)).astype(np.float32)
    std = rng.uniform(0.5, 2.0, (H, J)).astype(np.float32)
    P = pp.Projector(J, H, 0.05, b["bounds"]).factor(1.0)
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
