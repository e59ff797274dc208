"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these tests re-types the oracle's iteration.  Each checks the oracle
against something independent of it:
  * the printed operator matrices instantiated by hand at H=3 (golden file);
  * the constraint set written from its definition (derivatives of the
    velocity sequence, Sec. III-D) and the projection found by brute-force
    active-set enumeration (H <= 5) or by a closed form (H = 2);
  * optimality certificates (KKT with non-negative multipliers from NNLS);
  * properties of a Euclidean projection onto a convex set: idempotence,
    non-expansiveness, invariance to positive row scaling of the constraints;
  * the definition of each splitting step as an argmin, solved by
    numpy's least squares.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy.optimize import nnls

import oracle
from paper_2608_25666_b300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# the feasible set written from its definition (not from G): Sec. III-D
#   vel_k = x_k, pos_k = q0 + dt sum_{i<=k} x_i, acc_k = (x_k - x_{k-1})/dt
#   with x_0 = v0, jerk_k = (acc_k - acc_{k-1})/dt for k = 2..H; x_1 = v0.
# ---------------------------------------------------------------------------
def derivs(x, dt, q0, v0):
    x = np.asarray(x, dtype=np.float64)
    pos = q0 + dt * np.cumsum(x)
    xprev = np.concatenate([[v0], x[:-1]])
    acc = (x - xprev) / dt
    jerk = (acc[1:] - acc[:-1]) / dt
    return np.concatenate([x, pos, acc, jerk])


def bounds_vec(bnd, H):
    qmn, qmx, vmn, vmx, amn, amx, jmn, jmx = bnd
    lo = np.concatenate([np.full(H, vmn), np.full(H, qmn), np.full(H, amn), np.full(H - 1, jmn)])
    hi = np.concatenate([np.full(H, vmx), np.full(H, qmx), np.full(H, amx), np.full(H - 1, jmx)])
    return lo, hi


def affine_rows(H, dt, q0, v0):
    """c(x) = A x + c0 for the derivative map above (A from unit vectors)."""
    c0 = derivs(np.zeros(H), dt, q0, v0)
    A = np.stack([derivs(np.eye(H)[i], dt, q0, v0) - c0 for i in range(H)], axis=1)
    return A, c0


def violation(x, H, dt, bnd, q0, v0):
    c = derivs(x, dt, q0, v0)
    lo, hi = bounds_vec(bnd, H)
    return max(0.0, float(np.max(np.maximum(c - hi, lo - c))), abs(x[0] - v0))


def brute_force_projection(xi, H, dt, bnd, q0, v0, max_active=None):
    """Exact projection by enumerating active sets (rows depending on x_2..x_H)."""
    A, c0 = affine_rows(H, dt, q0, v0)
    lo, hi = bounds_vec(bnd, H)
    free_rows = [r for r in range(A.shape[0]) if np.any(np.abs(A[r, 1:]) > 0)]
    best, best_obj = None, np.inf
    nfree = H - 1
    max_active = nfree if max_active is None else max_active
    for k in range(0, max_active + 1):
        for rows in itertools.combinations(free_rows, k):
            for sides in itertools.product((0, 1), repeat=k):
                if k:
                    C = A[list(rows)][:, 1:]
                    tgt = np.array([(hi if s else lo)[r] for r, s in zip(rows, sides)])
                    d = tgt - c0[list(rows)] - A[list(rows), 0] * v0
                    CC = C @ C.T
                    if np.linalg.matrix_rank(CC) < k:
                        continue
                    mu = np.linalg.solve(CC, C @ xi[1:] - d)
                    y = xi[1:] - C.T @ mu
                else:
                    y = xi[1:].copy()
                x = np.concatenate([[v0], y])
                if violation(x, H, dt, bnd, q0, v0) > 1e-9:
                    continue
                obj = 0.5 * np.sum((x - xi) ** 2)
                if obj < best_obj - 1e-15:
                    best, best_obj = x, obj
    return best


def rand_case(rng, H, dt, tight=1.0):
    bnd = np.array([-2 * math.pi, 2 * math.pi, -math.pi, math.pi, -8.0, 8.0, -80.0, 80.0]) * tight
    q0 = rng.uniform(0.8 * bnd[0], 0.8 * bnd[1])
    v0 = rng.uniform(-0.5 * bnd[3], 0.5 * bnd[3])
    xi = rng.normal(0, 1.5, H)
    return xi, bnd, q0, v0


# ---------------------------------------------------------------------------
def test_G_h_matches_printed_matrices_H3():
    rows = []
    with open(os.path.join(GOLDEN, "G_h_H3.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(t) for t in line.split()])
    ref = np.array(rows)
    G, h = oracle.build_G_h(3, 0.5, [-1, 2, -3, 4, -5, 6, -7, 8], 0.25, 0.5)
    assert G.shape == (22, 3)
    np.testing.assert_array_equal(G, ref[:, :3])
    np.testing.assert_array_equal(h, ref[:, 3])


@pytest.mark.parametrize("H,dt", [(4, 0.05), (7, 0.02), (12, 0.1)])
def test_G_h_is_the_derivative_definition(H, dt):
    """G x <= h is the same set as the derivative bounds (every row pair)."""
    rng = np.random.default_rng(H)
    bnd = np.array([-1.0, 2.0, -3.0, 4.0, -5.0, 6.0, -7.0, 8.0])
    q0, v0 = 0.3, -0.7
    G, h = oracle.build_G_h(H, dt, bnd, q0, v0)
    lo, hi = bounds_vec(bnd, H)
    for _ in range(5):
        x = rng.normal(0, 1, H)
        c = derivs(x, dt, q0, v0)
        Gx = G @ x
        # "+" rows: c <= hi  <=>  Gx <= h ; "-" rows: -c <= -lo
        plus = np.concatenate([Gx[0:H], Gx[2 * H:3 * H], Gx[4 * H:5 * H], Gx[6 * H:7 * H - 1]])
        hp = np.concatenate([h[0:H], h[2 * H:3 * H], h[4 * H:5 * H], h[6 * H:7 * H - 1]])
        minus = np.concatenate([Gx[H:2 * H], Gx[3 * H:4 * H], Gx[5 * H:6 * H], Gx[7 * H - 1:]])
        hm = np.concatenate([h[H:2 * H], h[3 * H:4 * H], h[5 * H:6 * H], h[7 * H - 1:]])
        np.testing.assert_allclose(plus - hp, c - hi, rtol=1e-12, atol=1e-9)
        np.testing.assert_allclose(minus - hm, lo - c, rtol=1e-12, atol=1e-9)


def test_closed_form_H2():
    """H=2: x1 = v0 and x2 = clip(xi2, l, u) over the four interval constraints."""
    rng = np.random.default_rng(2)
    for t in range(40):
        dt = [0.01, 0.05, 0.2][t % 3]
        xi, bnd, q0, v0 = rand_case(rng, 2, dt, tight=rng.uniform(0.3, 1.5))
        qmn, qmx, vmn, vmx, amn, amx, jmn, jmx = bnd
        l = max(vmn, (qmn - q0) / dt - v0, v0 + dt * amn, v0 + dt * dt * jmn)
        u = min(vmx, (qmx - q0) / dt - v0, v0 + dt * amx, v0 + dt * dt * jmx)
        assert l <= u
        ref = np.array([v0, min(max(xi[1], l), u)])
        x, it, viol = oracle.exact_projection(xi, 2, dt, bnd, q0, v0)
        np.testing.assert_allclose(x, ref, atol=1e-10)


@pytest.mark.parametrize("H,ncase", [(3, 12), (4, 8), (5, 2)])
def test_brute_force_active_set(H, ncase):
    rng = np.random.default_rng(100 + H)
    for t in range(ncase):
        dt = [0.05, 0.02, 0.1][t % 3]
        xi, bnd, q0, v0 = rand_case(rng, H, dt, tight=rng.uniform(0.2, 1.0))
        xi = xi * 3.0
        ref = brute_force_projection(xi, H, dt, bnd, q0, v0)
        assert ref is not None
        x, it, viol = oracle.exact_projection(xi, H, dt, bnd, q0, v0)
        np.testing.assert_allclose(x, ref, atol=1e-9)


def kkt_certificate(x, xi, H, dt, bnd, q0, v0, act_tol=1e-8):
    """Residual of stationarity with sign-constrained multipliers (NNLS)."""
    A, c0 = affine_rows(H, dt, q0, v0)
    lo, hi = bounds_vec(bnd, H)
    c = A @ x + c0
    cols = []
    for r in range(A.shape[0]):
        if abs(c[r] - hi[r]) < act_tol:
            cols.append(A[r, 1:])
        if abs(c[r] - lo[r]) < act_tol:
            cols.append(-A[r, 1:])
    g = -(x - xi)[1:]            # need sum mu_r a_r = -(x - xi) on x_2..x_H
    if not cols:
        return float(np.max(np.abs(g)))
    M = np.stack(cols, axis=1)
    mu, res = nnls(M, g)
    return float(np.max(np.abs(M @ mu - g)))


@pytest.mark.parametrize("H,dt", [(10, 0.05), (30, 0.05)])
def test_kkt_certificate_and_feasibility(H, dt):
    rng = np.random.default_rng(7 + H)
    for _ in range(4):
        xi, bnd, q0, v0 = rand_case(rng, H, dt)
        x, it, viol = oracle.exact_projection(xi, H, dt, bnd, q0, v0)
        assert violation(x, H, dt, bnd, q0, v0) < 1e-10
        assert x[0] == pytest.approx(v0, abs=1e-12)
        assert kkt_certificate(x, xi, H, dt, bnd, q0, v0) < 1e-7


def test_projection_idempotent_and_nonexpansive():
    rng = np.random.default_rng(11)
    H, dt = 12, 0.05
    for _ in range(4):
        a, bnd, q0, v0 = rand_case(rng, H, dt)
        b = a + rng.normal(0, 0.3, H)
        pa, _, _ = oracle.exact_projection(a, H, dt, bnd, q0, v0)
        pb, _, _ = oracle.exact_projection(b, H, dt, bnd, q0, v0)
        ppa, _, _ = oracle.exact_projection(pa, H, dt, bnd, q0, v0)
        np.testing.assert_allclose(ppa, pa, atol=1e-10)
        assert np.linalg.norm(pa - pb) <= np.linalg.norm(a - b) + 1e-10


def test_rownorm_and_unscaled_reach_same_projection():
    """Positive row scaling leaves the feasible set, hence Pi, unchanged."""
    rng = np.random.default_rng(5)
    H, dt, J = 8, 0.25, 3
    b = workloads.make_custom(5, N=2, J=J, H=H, dt=dt)
    b["bounds"][6:] *= 0.05    # make jerk rows active
    r1 = oracle.solve_batch(b["xi"], b["q0"], b["v0"], b["bounds"], dt, 40000, 1.0,
                            scale=oracle.SCALE_ROWNORM)
    r2 = oracle.solve_batch(b["xi"], b["q0"], b["v0"], b["bounds"], dt, 40000, 1.0,
                            scale=oracle.SCALE_NONE)
    np.testing.assert_allclose(r1["x"], r2["x"], atol=1e-8)
    for n in range(2):
        for j in range(J):
            xi = b["xi"][n, :, j].astype(np.float64)
            bnd = b["bounds"][:, j]
            ref, _, _ = oracle.exact_projection(xi, H, dt, bnd, float(b["q0"][j]), float(b["v0"][j]))
            np.testing.assert_allclose(r1["x"][n, :, j], ref, atol=1e-8)


@pytest.mark.parametrize("mode", [oracle.MODE_ADMM, oracle.MODE_PAPER])
def test_loose_bounds_and_feasible_inputs_are_fixed_points(mode):
    """Feasible xi with xi_1 = v0 is returned unchanged after one iteration."""
    rng = np.random.default_rng(3)
    N, H, J, dt = 5, 20, 2, 0.05
    bounds = workloads.base_bounds(J, 50.0)           # loose: nothing active
    v0 = np.array([0.3, -0.2])
    q0 = np.array([0.1, 0.0])
    xi = np.stack([workloads.feasible_samples(rng, N, H, v, 0.05) for v in v0], axis=2)
    for iters in (1, 5):
        r = oracle.solve_batch(xi, q0, v0, bounds, dt, iters, 1.0, mode=mode)
        np.testing.assert_allclose(r["x"], xi, atol=1e-11)
        assert np.all(r["primal"] < 1e-12)
    # loose bounds and arbitrary xi: the projection only pins x_1 = v0
    xi2 = rng.normal(0, 1, (N, H, J))
    r = oracle.solve_batch(xi2, q0, v0, bounds, dt, 3, 1.0, mode=mode)
    ref = xi2.copy()
    ref[:, 0, :] = v0
    np.testing.assert_allclose(r["x"], ref, atol=1e-11)


def test_velocity_only_active_is_componentwise_clip():
    rng = np.random.default_rng(4)
    H, dt = 25, 0.05
    bnd = np.array([-1e3, 1e3, -0.5, 0.7, -1e6, 1e6, -1e9, 1e9])
    xi = rng.normal(0, 1.5, H)
    v0 = 0.2
    x, _, _ = oracle.exact_projection(xi, H, dt, bnd, 0.0, v0)
    ref = np.clip(xi, -0.5, 0.7)
    ref[0] = v0
    np.testing.assert_allclose(x, ref, atol=1e-10)


def _scaled_plus_rows(H, dt, bnd, q0, v0, rownorm=True):
    G, h = oracle.build_G_h(H, dt, bnd, q0, v0)
    plus = list(range(0, H)) + list(range(2 * H, 3 * H)) + list(range(4 * H, 5 * H)) + \
        list(range(6 * H, 7 * H - 1))
    minus = list(range(H, 2 * H)) + list(range(3 * H, 4 * H)) + list(range(5 * H, 6 * H)) + \
        list(range(7 * H - 1, 8 * H - 2))
    F = G[plus]
    s = 1.0 / np.linalg.norm(F, axis=1) if rownorm else np.ones(len(plus))
    return F * s[:, None], h[plus] * s, -h[minus] * s, G, h


def test_admm_first_primal_step_is_the_argmin():
    """x^1 = argmin 1/2||x-xi||^2 + rho/2 ||F'x - z^1 + u^0||^2 s.t. x_1 = v0 (lstsq)."""
    rng = np.random.default_rng(8)
    H, dt, rho = 16, 0.05, 1.7
    xi, bnd, q0, v0 = rand_case(rng, H, dt)
    Fs, hi, lo, _, _ = _scaled_plus_rows(H, dt, bnd, q0, v0)
    x0 = xi.copy()
    x0[0] = v0
    z1 = np.clip(Fs @ x0, lo, hi)
    Aop = np.vstack([np.eye(H - 1), math.sqrt(rho) * Fs[:, 1:]])
    rhs = np.concatenate([xi[1:], math.sqrt(rho) * (z1 - Fs[:, 0] * v0)])
    y = np.linalg.lstsq(Aop, rhs, rcond=None)[0]
    ref = np.concatenate([[v0], y])
    r = oracle.solve_batch(xi.reshape(1, H, 1), [q0], [v0], bnd.reshape(8, 1), dt, 1, rho)
    np.testing.assert_allclose(r["x"][0, :, 0], ref, atol=1e-10)


def test_paper_first_primal_step_is_the_argmin_of_aug_lag():
    """Eq. (admm_primal): x^1 minimises Eq. (aug_lag) with lambda^0 = 0 s.t. A x = b."""
    rng = np.random.default_rng(9)
    H, dt, rho = 12, 0.05, 0.8
    xi, bnd, q0, v0 = rand_case(rng, H, dt)
    G, h = oracle.build_G_h(H, dt, bnd, q0, v0)
    for rownorm, scale in ((False, oracle.SCALE_NONE), (True, oracle.SCALE_ROWNORM)):
        s = 1.0 / np.linalg.norm(G, axis=1) if rownorm else np.ones(G.shape[0])
        Gs, hs = G * s[:, None], h * s
        x0 = xi.copy()
        x0[0] = v0
        zeta = np.maximum(0.0, hs - Gs @ x0)
        Aop = np.vstack([np.eye(H - 1), math.sqrt(rho) * Gs[:, 1:]])
        rhs = np.concatenate([xi[1:], math.sqrt(rho) * (hs - zeta - Gs[:, 0] * v0)])
        y = np.linalg.lstsq(Aop, rhs, rcond=None)[0]
        ref = np.concatenate([[v0], y])
        r = oracle.solve_batch(xi.reshape(1, H, 1), [q0], [v0], bnd.reshape(8, 1), dt, 1, rho,
                               mode=oracle.MODE_PAPER, scale=scale)
        np.testing.assert_allclose(r["x"][0, :, 0], ref, rtol=1e-9, atol=1e-9)


def test_paper_mode_fixed_point_relation():
    """At a fixed point of Eqs. (admm_zeta)-(admm_dual): x is feasible and
    x - xi - lambda vanishes off the first component (the x_1 multiplier)."""
    rng = np.random.default_rng(12)
    H, dt = 10, 0.1
    b = workloads.make_custom(12, N=1, J=2, H=H, dt=dt)
    r = oracle.solve_batch(b["xi"], b["q0"], b["v0"], b["bounds"], dt, 60000, 1.0,
                           mode=oracle.MODE_PAPER, want_dual_state=True)
    assert np.all(r["dual"] < 1e-10)
    assert np.all(r["primal"] < 1e-9)
    g = r["x"] - b["xi"].astype(np.float64) - r["dual_state"]
    assert np.max(np.abs(g[:, 1:, :])) < 1e-8


def test_admm_iterates_converge_to_projection():
    """The ADMM reading converges to Pi (the paper's claim for its method)."""
    b = workloads.make_custom(21, N=2, J=2, H=20, dt=0.05)
    r = oracle.solve_batch(b["xi"], b["q0"], b["v0"], b["bounds"], 0.05, 20000, 1.0)
    for n in range(2):
        for j in range(2):
            ref, _, _ = oracle.exact_projection(b["xi"][n, :, j], 20, 0.05, b["bounds"][:, j],
                                                float(b["q0"][j]), float(b["v0"][j]))
            np.testing.assert_allclose(r["x"][n, :, j], ref, atol=1e-9)


def test_batch_layout_and_column_subset():
    """[N][H][J] stacking (time-major, joint-minor) and per-joint bounds."""
    b = workloads.make_custom(31, N=3, J=4, H=9, dt=0.05)
    bounds = b["bounds"].copy()
    bounds *= np.array([0.6, 0.9, 1.2, 1.5])[None, :]
    full = oracle.solve_batch(b["xi"], b["q0"], b["v0"], bounds, 0.05, 30, 1.0)
    for n in range(3):
        for j in range(4):
            one = oracle.solve_batch(b["xi"][n:n + 1, :, j:j + 1], b["q0"][j:j + 1],
                                     b["v0"][j:j + 1], bounds[:, j:j + 1], 0.05, 30, 1.0)
            np.testing.assert_array_equal(one["x"][0, :, 0], full["x"][n, :, j])
    sub = oracle.solve_batch(b["xi"], b["q0"], b["v0"], bounds, 0.05, 30, 1.0, cols=[5, 11],
                             nthreads=2)
    for c in (5, 11):
        n, j = divmod(c, 4)
        np.testing.assert_array_equal(sub["x"][n, :, j], full["x"][n, :, j])
    assert np.isnan(sub["x"][0, 0, 0])


def test_paper_iteration_is_not_the_projection():
    """Documents the measured gap: the printed iteration reaches a feasible
    point that is in general farther from xi than Pi(xi)."""
    b = workloads.make_custom(41, N=2, J=2, H=30, dt=0.05)
    rp = oracle.solve_batch(b["xi"], b["q0"], b["v0"], b["bounds"], 0.05, 20000, 1.0,
                            mode=oracle.MODE_PAPER)
    gaps = []
    for n in range(2):
        for j in range(2):
            xi = b["xi"][n, :, j].astype(np.float64)
            ref, _, _ = oracle.exact_projection(xi, 30, 0.05, b["bounds"][:, j],
                                                float(b["q0"][j]), float(b["v0"][j]))
            d_paper = np.linalg.norm(rp["x"][n, :, j] - xi)
            d_pi = np.linalg.norm(ref - xi)
            assert d_paper >= d_pi - 1e-9
            gaps.append(d_paper - d_pi)
    assert max(gaps) > 1e-3


# ---------------------------------------------------------------------------
# Per-iteration pins of the ADMM reading.  The tests above fix the first primal
# step and the limit; these fix every iteration, so that a changed multiplier
# step or a changed slack step (which have the same limit) is caught after the
# same finite number of iterations that the GPU parity tests compare.
# ---------------------------------------------------------------------------
ADMM_CASES = [(6, 0.05, 1.0, oracle.SCALE_ROWNORM), (12, 0.02, 0.4, oracle.SCALE_ROWNORM),
              (20, 0.1, 2.5, oracle.SCALE_NONE), (30, 0.05, 1.0, oracle.SCALE_ROWNORM)]


def _admm_state(xi, bnd, q0, v0, H, dt, L, rho, scale, x_init=None, dual_init=None):
    r = oracle.solve_batch(xi.reshape(1, H, 1), [q0], [v0], bnd.reshape(8, 1), dt, L, rho,
                           scale=scale, want_dual_state=True,
                           x_init=None if x_init is None else x_init.reshape(1, H, 1),
                           dual_init=None if dual_init is None else dual_init.reshape(1, -1, 1))
    return r["x"][0, :, 0], r["dual_state"][0, :, 0], r


@pytest.mark.parametrize("H,dt,rho,scale", ADMM_CASES)
def test_admm_dual_feasibility_after_every_iteration(H, dt, rho, scale):
    """Scaled ADMM (Boyd et al. 2011, Sec. 3.3): with the multiplier step
    u <- u + F'x - z, the x-step's optimality condition becomes dual
    feasibility of the new pair, x^l - xi + rho F'^T u^l in span(e1) (the
    x_1 = v0 multiplier), after EVERY iteration l.  Any other step size breaks
    it.  F' is built here from the printed G (pinned above) with unit rows."""
    rng = np.random.default_rng(60 + H)
    xi, bnd, q0, v0 = rand_case(rng, H, dt, tight=0.5)
    Fs, _, _, _, _ = _scaled_plus_rows(H, dt, bnd, q0, v0, rownorm=(scale == oracle.SCALE_ROWNORM))
    # rounding bound of one x-step: a few ulps times the condition number of
    # I + rho F'^T F' times the size of the terms (1e-15 with unit rows; the
    # printed rows carry 1/dt^2 and a condition number near 1e6)
    kappa = np.linalg.cond(np.eye(H) + rho * Fs.T @ Fs)
    eps = 16 * np.finfo(float).eps * kappa

    def tol(u):
        return eps * max(1.0, float(np.max(np.abs(rho * Fs.T @ u))), float(np.max(np.abs(xi))))

    seen_active = False
    for L in range(1, 11):
        x, u, _ = _admm_state(xi, bnd, q0, v0, H, dt, L, rho, scale)
        g = x - xi + rho * Fs.T @ u
        assert np.max(np.abs(g[1:])) <= tol(u), (L, np.max(np.abs(g[1:])), tol(u))
        seen_active |= bool(np.max(np.abs(u)) > 1e-3)
    assert seen_active   # the case exercises active constraints
    assert eps < 1e-6    # far below the 1e-2 .. 1 that a wrong step leaves
    # the same holds from a warm start (given iterate and multiplier)
    x5, u5, _ = _admm_state(xi, bnd, q0, v0, H, dt, 5, rho, scale)
    xw, uw, _ = _admm_state(xi, bnd, q0, v0, H, dt, 3, rho, scale, x_init=x5, dual_init=u5)
    g = xw - xi + rho * Fs.T @ uw
    assert np.max(np.abs(g[1:])) <= tol(uw)


PAPER_CASES = [(6, 0.05, 1.0, oracle.SCALE_ROWNORM), (12, 0.02, 0.4, oracle.SCALE_ROWNORM),
               (10, 0.1, 2.5, oracle.SCALE_NONE), (20, 0.05, 0.7, oracle.SCALE_ROWNORM)]


def _paper_state(xi, bnd, q0, v0, H, dt, L, rho, scale):
    r = oracle.solve_batch(xi.reshape(1, H, 1), [q0], [v0], bnd.reshape(8, 1), dt, L, rho,
                           mode=oracle.MODE_PAPER, scale=scale, want_dual_state=True)
    return r["x"][0, :, 0], r["dual_state"][0, :, 0]


@pytest.mark.parametrize("H,dt,rho,scale", PAPER_CASES)
def test_paper_stationarity_after_every_iteration(H, dt, rho, scale):
    """Eq. (admm_primal) makes x^{l+1} the minimiser of Eq. (aug_lag), with
    lambda^l and zeta^{l+1}, subject to A x = b (x_1 = v0): its stationarity is
        x^{l+1} - xi - lambda^l + delta G'^T (G' x^{l+1} - h' + zeta^{l+1}) in span(e1).
    Eq. (admm_dual) moves lambda by -(delta/2) times the same G'^T (...), so the
    last term equals 2 (lambda^l - lambda^{l+1}) and
        x^{l+1} - xi + lambda^l - 2 lambda^{l+1} in span(e1)
    after EVERY iteration, whatever G' is.  A multiplier step c delta with
    c != 1/2 leaves (1/c - 2)(lambda^l - lambda^{l+1}) off e1 instead: this pins
    the factor delta/2 of Eq. (admm_dual)."""
    rng = np.random.default_rng(80 + H)
    xi, bnd, q0, v0 = rand_case(rng, H, dt, tight=0.5)
    G, _ = oracle.build_G_h(H, dt, bnd, q0, v0)
    Gs = G / np.linalg.norm(G, axis=1)[:, None] if scale == oracle.SCALE_ROWNORM else G
    # rounding bound of one x-step: a few ulps times the condition number of the
    # x-step's matrix times the size of the terms
    eps = 16 * np.finfo(float).eps * np.linalg.cond(np.eye(H) + rho * Gs.T @ Gs)
    lam_prev = np.zeros(H)
    moved = 0.0
    for L in range(0, 10):
        x1, lam1 = _paper_state(xi, bnd, q0, v0, H, dt, L + 1, rho, scale)
        g = x1 - xi + lam_prev - 2.0 * lam1
        tol = eps * max(1.0, float(np.max(np.abs(lam_prev))), float(np.max(np.abs(lam1))),
                        float(np.max(np.abs(xi))), float(np.max(np.abs(x1))))
        assert np.max(np.abs(g[1:])) <= tol, (L, np.max(np.abs(g[1:])), tol)
        moved = max(moved, float(np.max(np.abs(lam1 - lam_prev))))
        lam_prev = lam1
    assert eps < 1e-5 and moved > 1e3 * eps   # a wrong factor would be far outside the bound


@pytest.mark.parametrize("H,dt,rho,scale", ADMM_CASES)
def test_admm_slack_step_is_the_box_projection(H, dt, rho, scale):
    """The slack of iteration l is z^l = u^{l-1} + F'x^l - u^l (the multiplier
    step read backwards).  It must be the Euclidean projection of
    w = F'x^{l-1} + u^{l-1} onto the box [lo', hi']: z inside the box and
    w - z in the box's normal cone at z (positive only where z sits on hi',
    negative only where it sits on lo').  This fixes which iterate and which
    multiplier the slack step sees and that it clips before the x-step."""
    rng = np.random.default_rng(70 + H)
    xi, bnd, q0, v0 = rand_case(rng, H, dt, tight=0.5)
    Fs, hi, lo, _, _ = _scaled_plus_rows(H, dt, bnd, q0, v0, rownorm=(scale == oracle.SCALE_ROWNORM))
    x0 = xi.copy()
    x0[0] = v0
    u_prev, x_prev = np.zeros(4 * H - 1), x0
    n_active = 0
    for L in range(1, 9):
        x, u, _ = _admm_state(xi, bnd, q0, v0, H, dt, L, rho, scale)
        z = u_prev + Fs @ x - u
        w = Fs @ x_prev + u_prev
        scl = 1e-11 * max(1.0, float(np.max(np.abs(w))))
        assert np.all(z >= lo - scl) and np.all(z <= hi + scl), L
        r = w - z
        on_hi = np.abs(z - hi) <= scl
        on_lo = np.abs(z - lo) <= scl
        assert np.all((r <= scl) | on_hi), L
        assert np.all((r >= -scl) | on_lo), L
        n_active += int(np.sum(np.abs(r) > 1e-6))
        u_prev, x_prev = u, x
    assert n_active > 0


def test_admm_residuals_are_their_definitions():
    """primal = max(|x_1 - v0|, row-normalised violation of the derivative
    bounds), the rows and their norms taken from the derivative map itself;
    dual = max |x^L - x^{L-1}| from two runs of L-1 and L iterations."""
    rng = np.random.default_rng(81)
    H, dt, rho = 14, 0.05, 1.3
    xi, bnd, q0, v0 = rand_case(rng, H, dt, tight=0.6)
    A, c0 = affine_rows(H, dt, q0, v0)
    lo, hi = bounds_vec(bnd, H)
    nrm = np.linalg.norm(A, axis=1)
    for L in (0, 1, 4, 9):
        x, _, r = _admm_state(xi, bnd, q0, v0, H, dt, L, rho, oracle.SCALE_ROWNORM)
        c = A @ x + c0
        ref = max(abs(x[0] - v0), float(np.max(np.maximum(0.0, np.maximum(c - hi, lo - c)) / nrm)))
        assert r["primal"][0, 0] == pytest.approx(ref, rel=1e-12, abs=1e-14)
        if L == 0:
            assert r["dual"][0, 0] == 0.0
        else:
            xp, _, _ = _admm_state(xi, bnd, q0, v0, H, dt, L - 1, rho, oracle.SCALE_ROWNORM)
            assert r["dual"][0, 0] == pytest.approx(float(np.max(np.abs(x - xp))), rel=1e-12, abs=1e-15)
