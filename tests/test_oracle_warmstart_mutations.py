"""Planted mistakes in the learned warm-start oracle must each fail a pin.

Each case replaces one function of ``oracle/warmstart.py`` (in memory, on the
CPU) with a copy that carries one plausible slip -- a wrong bound, a dropped
term, a transposed layout, a missing 1/n -- and runs the pins of
``test_oracle_warmstart``; at least one of the listed pins has to fail.  The
oracle file itself is never modified.
"""
import numpy as np
import pytest

from oracle import warmstart as ws
import test_oracle_warmstart as pins

_features = ws.features          # the unmodified function, for mutants that wrap it


def features_vmin(xi, q0, v0, bounds):
    xi = np.asarray(xi, dtype=np.float64)
    N, H, J = xi.shape
    bnd = np.asarray(bounds, dtype=np.float64).reshape(8, J)
    F = np.empty((N, J, H + 3))
    F[:, :, :H] = xi.transpose(0, 2, 1) / bnd[2][None, :, None]          # v_min instead of v_max
    F[:, :, H] = (np.asarray(v0) / bnd[3])[None, :]
    F[:, :, H + 1] = ((np.asarray(q0) - 0.5 * (bnd[0] + bnd[1])) / (0.5 * (bnd[1] - bnd[0])))[None, :]
    F[:, :, H + 2] = 1.0
    return F.reshape(N * J, H + 3)


def features_joint_major(xi, q0, v0, bounds):
    xi = np.asarray(xi, dtype=np.float64)
    N, H, J = xi.shape
    bnd = np.asarray(bounds, dtype=np.float64).reshape(8, J)
    F = np.empty((J, N, H + 3))                                          # column j*N + n
    F[:, :, :H] = xi.transpose(2, 0, 1) / bnd[3][:, None, None]
    F[:, :, H] = (np.asarray(v0) / bnd[3])[:, None]
    F[:, :, H + 1] = ((np.asarray(q0) - 0.5 * (bnd[0] + bnd[1])) / (0.5 * (bnd[1] - bnd[0])))[:, None]
    F[:, :, H + 2] = 1.0
    return F.reshape(N * J, H + 3)


def features_q0_uncentred(xi, q0, v0, bounds):
    F = _features(xi, q0, v0, bounds)
    xi = np.asarray(xi)
    N, H, J = xi.shape
    bnd = np.asarray(bounds, dtype=np.float64).reshape(8, J)
    F.reshape(N, J, H + 3)[:, :, H + 1] = (np.asarray(q0) / (0.5 * (bnd[1] - bnd[0])))[None, :]
    return F


def design_no_skip(F, W1, b1):
    F = np.asarray(F, dtype=np.float64)
    if W1 is None:
        return F.copy()
    W1 = np.asarray(W1, dtype=np.float64).reshape(-1, F.shape[1])
    return np.maximum(F @ W1.T + np.asarray(b1)[None, :], 0.0)               # phi = h only


def design_no_relu(F, W1, b1):
    F = np.asarray(F, dtype=np.float64)
    if W1 is None:
        return F.copy()
    W1 = np.asarray(W1, dtype=np.float64).reshape(-1, F.shape[1])
    return np.concatenate([F @ W1.T + np.asarray(b1)[None, :], F], axis=1)


def design_no_bias(F, W1, b1):
    F = np.asarray(F, dtype=np.float64)
    if W1 is None:
        return F.copy()
    W1 = np.asarray(W1, dtype=np.float64).reshape(-1, F.shape[1])
    return np.concatenate([np.maximum(F @ W1.T, 0.0), F], axis=1)


def fit_without_mean(S, T, n, lam):
    return np.linalg.solve(S + lam * np.eye(S.shape[0]), T)


def targets_swapped(x, dual_state):
    x = np.asarray(x, dtype=np.float64)
    u = np.asarray(dual_state, dtype=np.float64)
    N, H, J = x.shape
    D = u.shape[1]
    return np.concatenate([x.transpose(0, 2, 1).reshape(N * J, H), u.transpose(0, 2, 1).reshape(N * J, D)], axis=1)


def predict_dual_layout_transposed(xi, q0, v0, bounds, W1, b1, W2):
    xi = np.asarray(xi, dtype=np.float64)
    N, H, J = xi.shape
    Yh = ws.design(ws.features(xi, q0, v0, bounds), W1, b1) @ np.asarray(W2, dtype=np.float64)
    D = Yh.shape[1] - H
    dual = Yh[:, :D].reshape(N, D, J)                                    # rows and joints mixed up
    x = Yh[:, D:].reshape(N, J, H).transpose(0, 2, 1)
    return np.ascontiguousarray(x), np.ascontiguousarray(dual)


MUTATIONS = [
    ("features scaled by the velocity lower bound", "features", features_vmin,
     [pins.test_features_on_a_hand_computed_case]),
    ("joint-major column order", "features", features_joint_major,
     [pins.test_features_on_a_hand_computed_case]),
    ("q0 not centred", "features", features_q0_uncentred,
     [pins.test_features_on_a_hand_computed_case]),
    ("no linear skip", "design", design_no_skip,
     [pins.test_identity_first_layer_is_the_positive_part]),
    ("no ReLU", "design", design_no_relu,
     [pins.test_identity_first_layer_is_the_positive_part]),
    ("no bias", "design", design_no_bias,
     [pins.test_first_layer_bias_and_relu_on_a_hand_computed_case]),
    ("ridge without the mean over columns", "fit", fit_without_mean,
     [lambda: pins.test_ridge_is_least_squares_on_the_augmented_system(0.3)]),
    ("targets with the iterate first", "targets", targets_swapped,
     [pins.test_target_layout]),
    ("dual layout transposed in predict", "predict", predict_dual_layout_transposed,
     [pins.test_predict_layout]),
]


@pytest.mark.parametrize("name,fn,mutant,checks", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(name, fn, mutant, checks, monkeypatch):
    monkeypatch.setattr(ws, fn, mutant)
    failed = 0
    for check in checks:
        try:
            check()
        except AssertionError:
            failed += 1
    assert failed > 0, f"planted mistake '{name}' passed every listed pin"
