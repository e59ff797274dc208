"""Pins of the learned warm-start oracle (oracle/warmstart.py) against facts
outside its own formulas: exact recovery of a linear map, ridge regression as
least squares on the augmented system (a QR/SVD routine, not the normal
equations), hand-computed features, the identity first layer, the target
layout, the warm start as an exact continuation of the iteration, and the
fitted model beating a cold start on fresh samples."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import warmstart as ws
from paper_2608_25666_b300 import workloads


def test_fit_recovers_an_exact_linear_map():
    rng = np.random.default_rng(1)
    Phi = rng.normal(size=(400, 17))
    M = rng.normal(size=(17, 9))
    S, T, n = ws.normal_equations(Phi, Phi @ M)
    assert n == 400
    assert np.max(np.abs(ws.fit(S, T, n, 0.0) - M)) <= 1e-10


@pytest.mark.parametrize("lam", [1e-4, 0.3, 7.0])
def test_ridge_is_least_squares_on_the_augmented_system(lam):
    rng = np.random.default_rng(2)
    Phi = rng.normal(size=(300, 12)) * rng.uniform(0.1, 3.0, size=12)
    Y = rng.normal(size=(300, 5))
    n = Phi.shape[0]
    S, T, _ = ws.normal_equations(Phi, Y)
    A = np.vstack([Phi / np.sqrt(n), np.sqrt(lam) * np.eye(12)])
    B = np.vstack([Y / np.sqrt(n), np.zeros((12, 5))])
    ref = scipy.linalg.lstsq(A, B)[0]
    assert np.max(np.abs(ws.fit(S, T, n, lam) - ref)) <= 1e-10


def test_features_on_a_hand_computed_case():
    # N = 2 samples, H = 2 steps, J = 2 joints
    xi = np.array([[[1.0, 4.0], [-2.0, 8.0]],
                   [[0.5, -4.0], [3.0, 2.0]]])          # [n][k][j]
    bounds = np.array([[-1.0, 0.0], [3.0, 10.0],        # q min, q max
                       [-2.0, -4.0], [2.0, 4.0],        # v min, v max
                       [-5.0, -5.0], [5.0, 5.0], [-9.0, -9.0], [9.0, 9.0]])
    q0 = np.array([2.0, 0.0])
    v0 = np.array([1.0, -2.0])
    F = ws.features(xi, q0, v0, bounds)
    # column n*J + j: [xi[n][0][j]/vmax_j, xi[n][1][j]/vmax_j, v0_j/vmax_j, (q0_j - mid_j)/half_j, 1]
    expect = np.array([[0.5, -1.0, 0.5, 0.5, 1.0],
                       [1.0, 2.0, -0.5, -1.0, 1.0],
                       [0.25, 1.5, 0.5, 0.5, 1.0],
                       [-1.0, 0.5, -0.5, -1.0, 1.0]])
    assert np.array_equal(F, expect)


def test_identity_first_layer_is_the_positive_part():
    rng = np.random.default_rng(3)
    F = rng.normal(size=(50, 7))
    Phi = ws.design(F, np.eye(7), np.zeros(7))
    assert np.array_equal(Phi[:, :7], np.where(F > 0, F, 0.0))
    assert np.array_equal(Phi[:, 7:], F)


def test_no_hidden_layer_is_the_linear_model():
    rng = np.random.default_rng(8)
    F = rng.normal(size=(20, 6))
    assert np.array_equal(ws.design(F, None, None), F)


def test_target_layout():
    N, H, J = 3, 4, 2
    D = 4 * H - 1
    x = np.arange(N * H * J, dtype=np.float64).reshape(N, H, J)
    u = -np.arange(N * D * J, dtype=np.float64).reshape(N, D, J)
    Y = ws.targets(x, u)
    for n in range(N):
        for j in range(J):
            assert np.array_equal(Y[n * J + j], np.concatenate([u[n, :, j], x[n, :, j]]))


@pytest.mark.parametrize("H,dt,rho", [(12, 0.05, 1.0), (20, 0.02, 2.5)])
def test_warm_start_from_the_iteration_state_continues_it(H, dt, rho):
    """Warm-starting from (x^L, u^L) and running K more iterations equals running
    L + K iterations cold: the warm-start inputs are the iteration state, in the
    units and layout of the exported multiplier."""
    b = workloads.make_custom(21, 5, 3, H, dt)
    L, K = 17, 6
    a = oracle.solve_batch(b["xi"], b["q0"], b["v0"], b["bounds"], dt, L, rho, want_dual_state=True)
    c = oracle.solve_batch(b["xi"], b["q0"], b["v0"], b["bounds"], dt, K, rho,
                           x_init=a["x"], dual_init=a["dual_state"], want_dual_state=True)
    full = oracle.solve_batch(b["xi"], b["q0"], b["v0"], b["bounds"], dt, L + K, rho, want_dual_state=True)
    assert np.max(np.abs(c["x"] - full["x"])) <= 1e-12
    assert np.max(np.abs(c["dual_state"] - full["dual_state"])) <= 1e-12


def test_fitted_model_beats_a_cold_start():
    """Fitted on converged solves of one set of samples, the prediction used as
    the warm start of fresh samples leaves a smaller violation and a smaller
    distance to the converged solution than a cold start after as many
    iterations."""
    H, J, dt = 20, 3, 0.02
    rng = np.random.default_rng(4)
    hidden = 32
    W1 = rng.normal(0.0, 1.0 / np.sqrt(H + 3), size=(hidden, H + 3))
    b1 = rng.uniform(-1.0, 1.0, size=hidden)
    Phis, Ys = [], []
    for step in range(6):
        b = workloads.make_custom(100 + step, 40, J, H, dt, offset_sigma=0.5)
        o = oracle.solve_batch(b["xi"], b["q0"], b["v0"], b["bounds"], dt, 1500, 1.0, nthreads=8,
                               want_dual_state=True)
        Phis.append(ws.design(ws.features(b["xi"], b["q0"], b["v0"], b["bounds"]), W1, b1))
        Ys.append(ws.targets(o["x"], o["dual_state"]))
    S, T, n = ws.normal_equations(np.concatenate(Phis), np.concatenate(Ys))
    W2 = ws.fit(S, T, n, 1e-3)
    t = workloads.make_custom(999, 40, J, H, dt, offset_sigma=0.5)
    ref = oracle.solve_batch(t["xi"], t["q0"], t["v0"], t["bounds"], dt, 1500, 1.0, nthreads=8)
    xw, dw = ws.predict(t["xi"], t["q0"], t["v0"], t["bounds"], W1, b1, W2)
    L = 20
    cold = oracle.solve_batch(t["xi"], t["q0"], t["v0"], t["bounds"], dt, L, 1.0, nthreads=8)
    warm = oracle.solve_batch(t["xi"], t["q0"], t["v0"], t["bounds"], dt, L, 1.0, nthreads=8,
                              x_init=xw, dual_init=dw)
    assert np.max(warm["primal"]) < 0.7 * np.max(cold["primal"])
    assert np.max(np.abs(warm["x"] - ref["x"])) < 0.7 * np.max(np.abs(cold["x"] - ref["x"]))


def test_warm_start_first_step_is_the_boundary_value():
    """x_1 = v0 (Eq. proj_boundary) holds for the starting iterate too: a warm
    start whose first step differs from v0 gives the result of one whose first
    step is v0."""
    H, dt = 15, 0.05
    b = workloads.make_custom(31, 6, 3, H, dt)
    rng = np.random.default_rng(9)
    x0 = rng.normal(size=(6, H, 3))
    u0 = rng.normal(size=(6, 4 * H - 1, 3))
    x0v = x0.copy()
    x0v[:, 0, :] = b["v0"][None, :]
    a = oracle.solve_batch(b["xi"], b["q0"], b["v0"], b["bounds"], dt, 7, 1.0, x_init=x0, dual_init=u0,
                           want_dual_state=True)
    c = oracle.solve_batch(b["xi"], b["q0"], b["v0"], b["bounds"], dt, 7, 1.0, x_init=x0v, dual_init=u0,
                           want_dual_state=True)
    assert np.array_equal(a["x"], c["x"]) and np.array_equal(a["dual_state"], c["dual_state"])


def test_first_layer_bias_and_relu_on_a_hand_computed_case():
    """W1 = 0: every column's hidden layer is max(0, b1), whatever its features."""
    F = np.array([[1.0, -2.0, 3.0], [0.5, 0.0, -1.0]])
    Phi = ws.design(F, np.zeros((3, 3)), np.array([1.5, -0.5, 2.0]))
    assert np.array_equal(Phi, np.array([[1.5, 0.0, 2.0, 1.0, -2.0, 3.0],
                                         [1.5, 0.0, 2.0, 0.5, 0.0, -1.0]]))


def test_predict_layout():
    """A linear model (no hidden layer) whose output layer copies feature k into
    output o (k = o mod H for the multiplier rows, k = step for the iterate)
    returns dual_init[n][o][j] = xi[n][o mod H][j] / vmax_j and
    x_init[n][k][j] = xi[n][k][j] / vmax_j."""
    N, H, J = 3, 4, 2
    D = 4 * H - 1
    rng = np.random.default_rng(12)
    xi = rng.normal(size=(N, H, J))
    bounds = workloads.base_bounds(J)
    bounds[3] = [2.0, 4.0]                                  # vmax per joint
    W2 = np.zeros((H + 3, D + H))
    for o in range(D):
        W2[o % H, o] = 1.0
    for k in range(H):
        W2[k, D + k] = 1.0
    x, u = ws.predict(xi, np.zeros(J), np.zeros(J), bounds, None, None, W2)
    for n in range(N):
        for j in range(J):
            for o in range(D):
                assert u[n, o, j] == xi[n, o % H, j] / bounds[3][j]
            for k in range(H):
                assert x[n, k, j] == xi[n, k, j] / bounds[3][j]
