"""Learned warm start on the GPU (prism_ws_*) against the FP64 oracle
(oracle/warmstart.py).  Targets are the oracle's own converged solves (rounded
to float32, the precision the device reads), so no expected value comes from
the CUDA path.  The fit's sums and its solution are FP64 on both sides; the
predictor runs on the tensor cores with bf16 operands, so it is checked
against a bound derived from bf16 rounding (unit roundoff 2^-8) of its inputs,
its hidden layer and its weights."""
import numpy as np
import pytest

import oracle
from oracle import warmstart as ows
from paper_2608_25666_b300 import prism_proj as pp
from paper_2608_25666_b300 import workloads
from gpu_helpers import assert_parity

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8


def converged(b, iters=1500, nthreads=16):
    o = oracle.solve_batch(b["xi"], b["q0"], b["v0"], b["bounds"], b["dt"], iters, 1.0, nthreads=nthreads,
                           want_dual_state=True)
    return o["x"].astype(np.float32), o["dual_state"].astype(np.float32)


def dev(*arrs):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def first_layer(hidden, d, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 1.0 / np.sqrt(d), size=(hidden, d)), rng.uniform(-1.0, 1.0, size=hidden)


def oracle_fit(batches, targets, W1, b1, lam):
    Phis, Ys = [], []
    for b, (x, u) in zip(batches, targets):
        F = ows.features(b["xi"], b["q0"], b["v0"], b["bounds"])
        Phis.append(ows.design(F, W1, b1))
        Ys.append(ows.targets(x.astype(np.float64), u.astype(np.float64)))
    Phi, Y = np.concatenate(Phis), np.concatenate(Ys)
    S, T, n = ows.normal_equations(Phi, Y)
    return Phi, Y, S, T, n, ows.fit(S, T, n, lam)


def predict_bound(b, W1, b1, W2):
    """Elementwise bound on |bf16 predictor - FP64 model| in [N*J][NO] order."""
    F = ows.features(b["xi"], b["q0"], b["v0"], b["bounds"])
    hidden = 0 if W1 is None else W1.shape[0]
    aW2 = np.abs(W2)
    bound = 3.0 * U_BF16 * (np.abs(F) @ aW2[hidden:])
    if hidden:
        z = F @ W1.T + b1[None, :]
        dz = 2.01 * U_BF16 * (np.abs(F) @ np.abs(W1).T)
        bound += (1.01 * dz + 3.0 * U_BF16 * np.maximum(z, 0.0)) @ aW2[:hidden]
    return 1.5 * bound + 1e-6


@pytest.mark.parametrize("hidden", [0, 32, 64])
@pytest.mark.parametrize("J,H,N,dt", [(12, 50, 24, 0.02), (7, 33, 19, 0.05)])
def test_sums_fit_and_prediction_match_oracle(hidden, J, H, N, dt):
    import torch
    batches = [workloads.make_custom(40 + s, N, J, H, dt, offset_sigma=0.5) for s in range(2)]
    targets = [converged(b, 400) for b in batches]
    W1, b1 = first_layer(hidden, H + 3, 5) if hidden else (None, None)
    P = pp.Projector(J, H, dt, batches[0]["bounds"]).factor(1.0, pp.MODE_ADMM, pp.SCALE_ROWNORM, pp.PREC_TF32X3)
    ws = pp.WarmStart(P, hidden, W1=W1, b1=b1)
    for b, (x, u) in zip(batches, targets):
        xi, q0, v0, xs, us = dev(b["xi"], b["q0"], b["v0"], x, u)
        ws.accumulate(q0, v0, xi, xs, us)
    lam = 1e-3
    ws.fit(lam)
    g = ws.get()
    Phi, Y, S, T, n, W2 = oracle_fit(batches, targets, W1, b1, lam)
    assert g["n"] == n == 2 * N * J
    aP = np.abs(Phi)
    assert np.all(np.abs(g["S"] - S) <= 1e-11 * (aP.T @ aP) + 1e-300)
    assert np.all(np.abs(g["T"] - T) <= 1e-11 * (aP.T @ np.abs(Y)) + 1e-300)
    assert np.max(np.abs(g["W2"] - W2)) <= 1e-8 * np.max(np.abs(W2))
    # the predictor on a fresh batch (ragged: N*J is not a multiple of the 128-column tile)
    t = workloads.make_custom(77, N + 3, J, H, dt, offset_sigma=0.5)
    xi, q0, v0 = dev(t["xi"], t["q0"], t["v0"])
    xg, ug = ws.predict(q0, v0, xi)
    torch.cuda.synchronize()
    xo, uo = ows.predict(t["xi"], t["q0"], t["v0"], t["bounds"], W1, b1, W2)
    bound = predict_bound(t, W1, b1, W2)
    D = 4 * H - 1
    Ng = N + 3
    bu = bound[:, :D].reshape(Ng, J, D).transpose(0, 2, 1)
    bx = bound[:, D:].reshape(Ng, J, H).transpose(0, 2, 1)
    assert np.all(np.abs(ug.cpu().numpy() - uo) <= bu)
    assert np.all(np.abs(xg.cpu().numpy() - xo) <= bx)
    ws.close()
    P.close()


@pytest.mark.parametrize("H,hidden", [(100, 64), (132, 128), (3, 16)])
def test_predictor_extreme_shapes(H, hidden):
    """Several output chunks (H = 100: 499 outputs; H = 132: 659 outputs, the
    largest operands) and the smallest horizon: the model fitted by the oracle
    on synthetic targets, the predictor against its bound."""
    import torch
    J, N, dt = 3, 50, 0.02
    b = workloads.make_custom(9, N, J, H, dt)
    D = 4 * H - 1
    rng = np.random.default_rng(H)
    x = rng.normal(size=(N, H, J)).astype(np.float32)
    u = rng.normal(size=(N, D, J)).astype(np.float32)
    W1, b1 = first_layer(hidden, H + 3, 6)
    P = pp.Projector(J, H, dt, b["bounds"]).factor(1.0, pp.MODE_ADMM, pp.SCALE_ROWNORM, pp.PREC_FP32)
    ws = pp.WarmStart(P, hidden, W1=W1, b1=b1)
    xi, q0, v0, xs, us = dev(b["xi"], b["q0"], b["v0"], x, u)
    ws.accumulate(q0, v0, xi, xs, us)
    ws.fit(0.5)
    _, _, _, _, _, W2 = oracle_fit([b], [(x, u)], W1, b1, 0.5)
    assert np.max(np.abs(ws.get()["W2"] - W2)) <= 1e-8 * np.max(np.abs(W2))
    xg, ug = ws.predict(q0, v0, xi)
    torch.cuda.synchronize()
    xo, uo = ows.predict(b["xi"], b["q0"], b["v0"], b["bounds"], W1, b1, W2)
    bound = predict_bound(b, W1, b1, W2)
    bu = bound[:, :D].reshape(N, J, D).transpose(0, 2, 1)
    bx = bound[:, D:].reshape(N, J, H).transpose(0, 2, 1)
    assert np.all(np.abs(ug.cpu().numpy() - uo) <= bu)
    assert np.all(np.abs(xg.cpu().numpy() - xo) <= bx)
    ws.close()
    P.close()


def test_learned_warm_start_end_to_end():
    """Fit on the oracle's converged solves; on fresh samples the oracle's
    prediction warm-starts the GPU solve and the oracle alike (parity of the
    warm-started solve), and the GPU's own prediction -> solve leaves a smaller
    violation and distance to the converged solution than a cold start after as
    many iterations."""
    import torch
    J, H, N, dt = 12, 50, 32, 0.02
    hidden = 64
    W1, b1 = first_layer(hidden, H + 3, 7)
    batches = [workloads.make_custom(200 + s, N, J, H, dt, offset_sigma=0.5) for s in range(3)]
    targets = [converged(b, 1500) for b in batches]
    P = pp.Projector(J, H, dt, batches[0]["bounds"]).factor(1.0, pp.MODE_ADMM, pp.SCALE_ROWNORM, pp.PREC_TF32X3)
    ws = pp.WarmStart(P, hidden, W1=W1, b1=b1)
    for b, (x, u) in zip(batches, targets):
        xi, q0, v0, xs, us = dev(b["xi"], b["q0"], b["v0"], x, u)
        ws.accumulate(q0, v0, xi, xs, us)
    ws.fit(1e-3)
    _, _, _, _, _, W2 = oracle_fit(batches, targets, W1, b1, 1e-3)
    t = workloads.make_custom(999, N, J, H, dt, offset_sigma=0.5)
    xi, q0, v0 = dev(t["xi"], t["q0"], t["v0"])
    L = 20
    # parity of the warm-started solve, both sides from the oracle's prediction
    xo, uo = ows.predict(t["xi"], t["q0"], t["v0"], t["bounds"], W1, b1, W2)
    xo32, uo32 = xo.astype(np.float32), uo.astype(np.float32)
    xin, uin = dev(xo32, uo32)
    xg, pg, dg, _ = P.solve_ex(q0, v0, xi, L, x_init=xin, dual_init=uin)
    torch.cuda.synchronize()
    o = oracle.solve_batch(t["xi"], t["q0"], t["v0"], t["bounds"], dt, L, 1.0, nthreads=16,
                           x_init=xo32.astype(np.float64), dual_init=uo32.astype(np.float64))
    g = {"x": xg.cpu().numpy().astype(np.float64), "primal": pg.cpu().numpy().astype(np.float64),
         "dual": dg.cpu().numpy().astype(np.float64)}
    assert_parity(g, o, dual_tol=2e-4)
    # the device's own prediction as the warm start beats a cold start
    ref = oracle.solve_batch(t["xi"], t["q0"], t["v0"], t["bounds"], dt, 1500, 1.0, nthreads=16)
    xp, up = ws.predict(q0, v0, xi)
    xw, pw, _, _ = P.solve_ex(q0, v0, xi, L, x_init=xp, dual_init=up)
    xc, pc, _ = P.solve(q0, v0, xi, L)
    torch.cuda.synchronize()
    warm_viol, cold_viol = float(pw.max()), float(pc.max())
    warm_dx = float(np.max(np.abs(xw.cpu().numpy() - ref["x"])))
    cold_dx = float(np.max(np.abs(xc.cpu().numpy() - ref["x"])))
    assert warm_viol < 0.5 * cold_viol, (warm_viol, cold_viol)
    assert warm_dx < 0.75 * cold_dx, (warm_dx, cold_dx)
    ws.close()
    P.close()


def test_errors():
    import torch
    b = workloads.make_custom(3, 4, 3, 20, 0.05)
    P = pp.Projector(3, 20, 0.05, b["bounds"]).factor(1.0, pp.MODE_ADMM, pp.SCALE_ROWNORM, pp.PREC_FP32)
    with pytest.raises(pp.PrismError) as e:
        pp.WarmStart(P, 17)
    assert e.value.status == 1
    # a first layer whose ReLU is 0 on every input: 16 exactly zero design columns
    ws = pp.WarmStart(P, 16, W1=np.zeros((16, 23)), b1=-np.ones(16))
    xi, q0, v0 = dev(b["xi"], b["q0"], b["v0"])
    with pytest.raises(pp.PrismError) as e:
        ws.predict(q0, v0, xi)
    assert e.value.status == 2
    with pytest.raises(pp.PrismError) as e:
        ws.fit(1e-3)                      # nothing accumulated
    assert e.value.status == 1
    x = torch.zeros((4, 20, 3), device="cuda")
    u = torch.zeros((4, 79, 3), device="cuda")
    ws.accumulate(q0, v0, xi, x, u)
    with pytest.raises(pp.PrismError) as e:
        ws.fit(0.0)                       # zero pivots: singular without ridge
    assert e.value.status == 1
    ws.fit(1e-2)
    ws.close()
    Pp = pp.Projector(3, 20, 0.05, b["bounds"]).factor(1.0, pp.MODE_PAPER, pp.SCALE_ROWNORM, pp.PREC_FP32)
    with pytest.raises(pp.PrismError) as e:
        pp.WarmStart(Pp, 16)
    assert e.value.status == 1
    Pu = pp.Projector(3, 20, 0.05, b["bounds"])
    with pytest.raises(pp.PrismError) as e:
        pp.WarmStart(Pu, 16)
    assert e.value.status == 2
    for p_ in (P, Pp, Pu):
        p_.close()


@pytest.mark.parametrize("prec", [pp.PREC_TF32X3, pp.PREC_FP32], ids=["tc", "simt"])
def test_column_major_layout_equals_sample_major(prec):
    """The predictor's column-major outputs ([H][N*J], [D][N*J]) are its
    sample-major outputs transposed, bit for bit, and a solve warm-started from
    either layout gives identical results (ragged tiles: N*J = 444)."""
    import torch
    J, H, N, dt = 12, 50, 37, 0.02
    b = workloads.make_custom(61, N, J, H, dt, offset_sigma=0.5)
    D = 4 * H - 1
    rng = np.random.default_rng(3)
    x = rng.normal(size=(N, H, J)).astype(np.float32)
    u = (0.1 * rng.normal(size=(N, D, J))).astype(np.float32)
    W1, b1 = first_layer(32, H + 3, 8)
    P = pp.Projector(J, H, dt, b["bounds"]).factor(1.0, pp.MODE_ADMM, pp.SCALE_ROWNORM, prec)
    ws = pp.WarmStart(P, 32, W1=W1, b1=b1)
    xi, q0, v0, xs, us = dev(b["xi"], b["q0"], b["v0"], x, u)
    ws.accumulate(q0, v0, xi, xs, us).fit(0.1)
    xs_, us_ = ws.predict(q0, v0, xi)
    xc, uc = ws.predict(q0, v0, xi, layout=pp.INIT_COLUMN_MAJOR)
    torch.cuda.synchronize()
    assert tuple(xc.shape) == (H, N * J) and tuple(uc.shape) == (D, N * J)
    assert torch.equal(xc, xs_.permute(1, 0, 2).reshape(H, N * J))
    assert torch.equal(uc, us_.permute(1, 0, 2).reshape(D, N * J))
    a = P.solve_ex(q0, v0, xi, 15, x_init=xs_, dual_init=us_, want_dual_out=True)
    c = P.solve_ex(q0, v0, xi, 15, x_init=xc, dual_init=uc, want_dual_out=True, init_layout=pp.INIT_COLUMN_MAJOR)
    torch.cuda.synchronize()
    for ta, tc in zip(a, c):
        assert torch.equal(ta, tc)
    with pytest.raises(pp.PrismError) as e:
        P.solve_ex(q0, v0, xi, 15, x_init=xs_, dual_init=us_, init_layout=2)
    assert e.value.status == 1
    ws.close()
    P.close()
