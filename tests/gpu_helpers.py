"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle on
the same seeded inputs."""
import numpy as np

import oracle
from paper_2608_25666_b300 import prism_proj as pp

# Parity bar (FP32 CUDA path vs FP64 oracle after the same iteration count):
X_TOL = 1e-4          # max |x_gpu - x_oracle|, rad/s
VIOL_TOL = 1e-5       # |primal_res_gpu - primal_res_oracle|, row-normalised units


def to_dev(b):
    import torch
    return (torch.from_numpy(b["xi"]).cuda(), torch.from_numpy(b["q0"]).cuda(),
            torch.from_numpy(b["v0"]).cuda())


TC_MAX_H = 116       # largest horizon of the tensor-core K-apply


def gpu_solve(b, iters, rho=1.0, mode=pp.MODE_ADMM, scale=pp.SCALE_ROWNORM, kernel="persistent",
              prec=pp.PREC_FP32):
    import torch
    P = pp.Projector(b["J"], b["H"], b["dt"], b["bounds"]).factor(rho, mode, scale, prec)
    xi, q0, v0 = to_dev(b)
    fn = P.solve if kernel == "persistent" else P.solve_plain
    x, pr, du = fn(q0, v0, xi, iters)
    torch.cuda.synchronize()
    out = {"x": x.cpu().numpy().astype(np.float64), "primal": pr.cpu().numpy().astype(np.float64),
           "dual": du.cpu().numpy().astype(np.float64)}
    P.close()
    return out


def oracle_solve(b, iters, rho=1.0, mode=pp.MODE_ADMM, scale=pp.SCALE_ROWNORM, cols=None,
                 nthreads=8):
    return oracle.solve_batch(b["xi"], b["q0"], b["v0"], b["bounds"], b["dt"], iters, rho,
                              mode=mode, scale=scale, cols=cols, nthreads=nthreads)


def assert_parity(g, o, x_tol=X_TOL, viol_tol=VIOL_TOL, cols=None, dual_tol=None):
    gx, ox = g["x"], o["x"]
    gp, op = g["primal"], o["primal"]
    gd, od = g["dual"], o["dual"]
    if cols is not None:
        N, H, J = ox.shape
        n, j = np.divmod(np.asarray(cols), J)
        gx, ox = gx[n, :, j], ox[n, :, j]
        gp, op, gd, od = gp[n, j], op[n, j], gd[n, j], od[n, j]
    assert np.all(np.isfinite(gx))
    dx = float(np.max(np.abs(gx - ox))) if gx.size else 0.0
    dv = float(np.max(np.abs(gp - op))) if gp.size else 0.0
    assert dx <= x_tol, f"max |dx| = {dx:.3e} > {x_tol}"
    assert dv <= viol_tol, f"max |d viol| = {dv:.3e} > {viol_tol}"
    if dual_tol is not None and gd.size:
        dd = float(np.max(np.abs(gd - od)))
        assert dd <= dual_tol, f"max |d dual| = {dd:.3e} > {dual_tol}"
    return dx, dv
