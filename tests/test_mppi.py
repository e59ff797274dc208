"""The distribution update around the projection (Alg. 1, Eqs. weight_update,
mean_update_new, cov_update_new): oracle pins on CPU, CUDA kernel vs oracle
on GPU."""
import numpy as np
import pytest

from oracle.mppi import mppi_update as oracle_update


def test_equal_costs_reduce_to_plain_mean_and_variance():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(37, 5, 3))
    mean, var, w = oracle_update(np.full(37, 4.2), x, temperature=0.7, eps=1e-3)
    np.testing.assert_allclose(w, np.full(37, 1 / 37))
    np.testing.assert_allclose(mean, x.mean(axis=0), rtol=1e-12)
    np.testing.assert_allclose(var, x.var(axis=0) + 1e-3, rtol=1e-12)


def test_weights_are_a_softmax_of_negative_costs():
    rng = np.random.default_rng(1)
    c = rng.uniform(0, 50, 20)
    _, _, w = oracle_update(c, rng.normal(size=(20, 2, 2)), temperature=3.0)
    assert w.sum() == pytest.approx(1.0)
    assert np.all(np.diff(w[np.argsort(c)]) <= 0)          # cheaper -> heavier
    _, _, w2 = oracle_update(c + 1e4, rng.normal(size=(20, 2, 2)), temperature=3.0)
    np.testing.assert_allclose(w, w2, rtol=1e-12)           # shift invariance
    np.testing.assert_allclose(w[0] / w[1], np.exp(-(c[0] - c[1]) / 3.0), rtol=1e-12)


def test_small_temperature_selects_the_best_sample():
    rng = np.random.default_rng(2)
    c = rng.uniform(0, 10, 15)
    x = rng.normal(size=(15, 4, 2))
    mean, var, _ = oracle_update(c, x, temperature=1e-4, eps=0.5)
    np.testing.assert_allclose(mean, x[np.argmin(c)], atol=1e-12)
    np.testing.assert_allclose(var, 0.5, atol=1e-12)


@pytest.mark.gpu
@pytest.mark.parametrize("N,H,J,tau", [(4096, 50, 12, 5.0), (1, 3, 1, 1.0), (777, 64, 14, 0.5),
                                       (2000, 20, 6, 100.0)])
def test_kernel_matches_oracle(N, H, J, tau):
    import torch
    from paper_2608_25666_b300 import prism_proj as pp
    rng = np.random.default_rng(N + H)
    cost = rng.uniform(0, 60, N).astype(np.float32)
    x = rng.normal(0, 1.5, (N, H, J)).astype(np.float32)
    mean, var, w = pp.mppi_update(torch.from_numpy(cost).cuda(), torch.from_numpy(x).cuda(), tau, eps=1e-4)
    torch.cuda.synchronize()
    om, ov, ow = oracle_update(cost, x, tau, eps=1e-4)
    np.testing.assert_allclose(w.cpu().numpy(), ow, rtol=2e-5, atol=1e-9)
    np.testing.assert_allclose(mean.cpu().numpy(), om, rtol=1e-4, atol=2e-6)
    np.testing.assert_allclose(var.cpu().numpy(), ov, rtol=1e-4, atol=2e-6)
