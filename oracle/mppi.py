"""FP64 oracle of the sampling-distribution update (paper Alg. 1,
Eqs. weight_update, mean_update_new, cov_update_new).

TEST INFRASTRUCTURE ONLY (tests, smoke check and benchmark baseline).  The
equations written out with numpy, in the paper's order:
  w_n  = exp(-c_n / tau) / sum_m exp(-c_m / tau)          (Eq. weight_update)
  nu   = sum_n w_n x_n                                     (Eq. mean_update_new)
  Sigma = diag(sum_n w_n (x_n - nu)^2) + eps I             (Eq. cov_update_new)
The exponent is shifted by min(c) before exponentiating, which leaves w
unchanged and avoids underflow.
"""
import numpy as np


def mppi_update(cost, x, temperature, eps=0.0):
    c = np.asarray(cost, dtype=np.float64)
    X = np.asarray(x, dtype=np.float64)
    e = np.exp(-(c - c.min()) / float(temperature))
    w = e / e.sum()
    mean = np.tensordot(w, X, axes=(0, 0))
    var = np.tensordot(w, (X - mean[None]) ** 2, axes=(0, 0)) + float(eps)
    return mean, var, w
