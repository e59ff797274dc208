"""FP64 oracle of the learned warm start of the projection (the neural
warm-starting the paper's conclusion names as future work for the projection
QP; the paper gives no model, so the model here is this library's reading).

TEST INFRASTRUCTURE ONLY (tests, smoke check and benchmark baseline).

Per column c = n*J + j (joint j of sample n) the model maps d = H + 3 features
  f_k     = xi[n][k][j] / vmax_j                     (k < H)
  f_H     = v0_j / vmax_j
  f_{H+1} = (q0_j - (qmin_j + qmax_j) / 2) / ((qmax_j - qmin_j) / 2)
  f_{H+2} = 1
through one hidden layer with a fixed first layer (W1 [hidden][d], b1 [hidden],
drawn by the caller) and a linear skip,
  h_i = max(0, sum_k W1[i][k] f_k + b1[i]),     phi = [h | f]  (K2 = hidden + d),
to the NO = D + H targets y = [u' | x] of the converged solve (u' the scaled
multiplier in the oracle's units, D = 4H - 1 rows in the order velocity,
position, acceleration, jerk; x the trajectory):
  y_hat = phi W2.
The output layer is fitted by ridge regression on converged solves,
  W2 = argmin_W (1/n) sum_c ||phi_c W - y_c||^2 + lambda ||W||_F^2,
i.e. (Phi^T Phi / n + lambda I) W2 = Phi^T Y / n, and a prediction is used as
the warm start (x_init, dual_init) of the ADMM projection.
"""
import numpy as np


def n_features(H: int) -> int:
    return H + 3


def features(xi, q0, v0, bounds):
    """F [N*J][H+3] in column order n*J + j."""
    xi = np.asarray(xi, dtype=np.float64)
    N, H, J = xi.shape
    bnd = np.asarray(bounds, dtype=np.float64).reshape(8, J)
    qmin, qmax, vmax = bnd[0], bnd[1], bnd[3]
    q0 = np.asarray(q0, dtype=np.float64).reshape(J)
    v0 = np.asarray(v0, dtype=np.float64).reshape(J)
    F = np.empty((N, J, H + 3))
    F[:, :, :H] = xi.transpose(0, 2, 1) / vmax[None, :, None]
    F[:, :, H] = (v0 / vmax)[None, :]
    F[:, :, H + 1] = ((q0 - 0.5 * (qmin + qmax)) / (0.5 * (qmax - qmin)))[None, :]
    F[:, :, H + 2] = 1.0
    return F.reshape(N * J, H + 3)


def design(F, W1, b1):
    """Phi = [max(0, F W1^T + b1) | F]; Phi = F without a hidden layer (W1 None)."""
    F = np.asarray(F, dtype=np.float64)
    if W1 is None:
        return F.copy()
    W1 = np.asarray(W1, dtype=np.float64).reshape(-1, F.shape[1])
    b1 = np.asarray(b1, dtype=np.float64).reshape(W1.shape[0])
    h = np.maximum(F @ W1.T + b1[None, :], 0.0)
    return np.concatenate([h, F], axis=1)


def targets(x, dual_state):
    """Y [N*J][D+H] = [u' | x] in column order from x [N][H][J], u' [N][D][J]."""
    x = np.asarray(x, dtype=np.float64)
    u = np.asarray(dual_state, dtype=np.float64)
    N, H, J = x.shape
    D = u.shape[1]
    return np.concatenate([u.transpose(0, 2, 1).reshape(N * J, D), x.transpose(0, 2, 1).reshape(N * J, H)], axis=1)


def normal_equations(Phi, Y):
    """(Phi^T Phi, Phi^T Y, n): the sums a fit accumulates."""
    Phi = np.asarray(Phi, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return Phi.T @ Phi, Phi.T @ Y, Phi.shape[0]


def fit(S, T, n, lam):
    """W2 solving (S / n + lam I) W2 = T / n."""
    K2 = S.shape[0]
    return np.linalg.solve(S / n + lam * np.eye(K2), T / n)


def predict(xi, q0, v0, bounds, W1, b1, W2):
    """(x_init [N][H][J], dual_init [N][D][J]) of the fitted model."""
    xi = np.asarray(xi, dtype=np.float64)
    N, H, J = xi.shape
    Yh = design(features(xi, q0, v0, bounds), W1, b1) @ np.asarray(W2, dtype=np.float64)
    D = Yh.shape[1] - H
    dual = Yh[:, :D].reshape(N, J, D).transpose(0, 2, 1)
    x = Yh[:, D:].reshape(N, J, H).transpose(0, 2, 1)
    return np.ascontiguousarray(x), np.ascontiguousarray(dual)
