"""Seeded synthetic inputs for the projection workloads.

This module only draws random numbers and lays out bounds; it holds none of the
projection's arithmetic.  It is the one module that both the CUDA path and the
CPU oracle take their inputs from, so that both see the same values.

Conventions (Sec. III-D, "From Joint-Velocity Sequences to Derivative Bounds"):
  * samples xi are stacked time-major, joint-minor: ``xi[n, k, j]`` is the
    sampled velocity of joint j at horizon step k+1 of sample n, shape [N, H, J];
  * q0 / v0 are theta_init / thetadot_init per joint, shape [J];
  * bounds are an [8, J] float64 array with rows
    (q_min, q_max, v_min, v_max, a_min, a_max, j_min, j_max).

Every floating-point input that the GPU receives in FP32 (xi, q0, v0) is drawn
in float64 and rounded to float32 here, so the oracle can take the exact same
values widened back to float64.

Workloads (their shapes follow the bimanual setting of the paper: two 6-DOF
arms, N_dof = 12, white-noise velocity samples as in the sigma_eff study of
Sec. III-C):
  * "single"    N=64,    J=12, H=30, dt=0.05, 200 iterations
  * "realistic" N=4096,  J=12, H=50, dt=0.02, 100 iterations, per-(sample,
                joint) mean offset ~ N(0, 0.5^2), 64 independent steps
  * "batched"   512 uneven problems: J in {6,7,12,14}, H ~ U{20..100},
                N log-uniform in [128, 8192], dt in {0.01,0.02,0.05},
                bounds scaled per problem by s ~ U(0.5, 1.5), 150 iterations
  * "precision" N=16384, J=14, H=64, dt=0.02
Base bounds: |q| <= 2*pi, |v| <= pi, |a| <= 8, |j| <= 80 (rad, s).
Samples xi ~ N(0, 1.5^2); q0 ~ U(0.8*[q_min, q_max]); v0 ~ U(+-0.5*v_max).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BOUND_ROWS = ("q_min", "q_max", "v_min", "v_max", "a_min", "a_max", "j_min", "j_max")

BASE_Q = 2.0 * math.pi
BASE_V = math.pi
BASE_A = 8.0
BASE_J = 80.0
SAMPLE_SIGMA = 1.5


@dataclass(frozen=True)
class Workload:
    name: str
    N: int
    J: int
    H: int
    dt: float
    iters: int
    rho: float = 1.0
    offset_sigma: float = 0.0
    steps: int = 1
    seed: int = 1000


WORKLOADS = {
    "single": Workload("single", N=64, J=12, H=30, dt=0.05, iters=200, seed=1000),
    "realistic": Workload("realistic", N=4096, J=12, H=50, dt=0.02, iters=100,
                          offset_sigma=0.5, steps=64, seed=1001),
    "precision": Workload("precision", N=16384, J=14, H=64, dt=0.02, iters=100,
                          seed=1003),
}


def base_bounds(J: int, scale: float = 1.0) -> np.ndarray:
    """[8, J] float64 bounds, identical for all joints, scaled by ``scale``."""
    row = np.array([-BASE_Q, BASE_Q, -BASE_V, BASE_V, -BASE_A, BASE_A, -BASE_J, BASE_J],
                   dtype=np.float64) * float(scale)
    return np.repeat(row[:, None], J, axis=1).copy()


def _rng(seed: int, *stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), *map(int, stream)])))


def draw_batch(rng: np.random.Generator, N: int, J: int, H: int, bounds: np.ndarray,
               offset_sigma: float = 0.0) -> dict:
    """One projection batch: xi [N,H,J], q0 [J], v0 [J], all float32."""
    q_lo, q_hi = bounds[0], bounds[1]
    v_hi = bounds[3]
    q0 = rng.uniform(0.8 * q_lo, 0.8 * q_hi)
    v0 = rng.uniform(-0.5 * v_hi, 0.5 * v_hi)
    xi = rng.normal(0.0, SAMPLE_SIGMA, size=(N, H, J))
    if offset_sigma > 0.0:
        xi = xi + rng.normal(0.0, offset_sigma, size=(N, 1, J))
    return {
        "xi": np.ascontiguousarray(xi.astype(np.float32)),
        "q0": q0.astype(np.float32),
        "v0": v0.astype(np.float32),
    }


def make_batch(w: Workload, step: int = 0, N: int | None = None) -> dict:
    """Inputs of step ``step`` of workload ``w`` (optionally with fewer samples)."""
    rng = _rng(w.seed, step)
    bounds = base_bounds(w.J)
    b = draw_batch(rng, w.N if N is None else N, w.J, w.H, bounds, w.offset_sigma)
    b.update(bounds=bounds, J=w.J, H=w.H, dt=w.dt, iters=w.iters, rho=w.rho)
    return b


def make_custom(seed: int, N: int, J: int, H: int, dt: float, scale: float = 1.0,
                offset_sigma: float = 0.0) -> dict:
    """A batch of arbitrary shape with the base distributions (for edge cases)."""
    rng = _rng(seed, N, J, H)
    bounds = base_bounds(J, scale)
    b = draw_batch(rng, N, J, H, bounds, offset_sigma)
    b.update(bounds=bounds, J=J, H=H, dt=dt)
    return b


@dataclass
class Problem:
    J: int
    H: int
    N: int
    dt: float
    scale: float
    bounds: np.ndarray
    xi: np.ndarray
    q0: np.ndarray
    v0: np.ndarray
    extra: dict = field(default_factory=dict)


def batched_problems(nprob: int = 512, seed: int = 1002, n_lo: int = 128, n_hi: int = 8192,
                     h_lo: int = 20, h_hi: int = 100) -> list[Problem]:
    """The uneven multi-problem workload: one entry per independent projection problem."""
    rng = _rng(seed, 0)
    probs = []
    for p in range(nprob):
        J = int(rng.choice([6, 7, 12, 14]))
        H = int(rng.integers(h_lo, h_hi + 1))
        N = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        dt = float(rng.choice([0.01, 0.02, 0.05]))
        s = float(rng.uniform(0.5, 1.5))
        bounds = base_bounds(J, s)
        b = draw_batch(_rng(seed, 1, p), N, J, H, bounds)
        probs.append(Problem(J=J, H=H, N=N, dt=dt, scale=s, bounds=bounds,
                             xi=b["xi"], q0=b["q0"], v0=b["v0"]))
    return probs


def feasible_samples(rng: np.random.Generator, N: int, H: int, v0: float, v_amp: float) -> np.ndarray:
    """Smooth low-amplitude velocity sequences starting at v0 (float64, [N, H]).

    Used to build inputs that already satisfy loose bounds (idempotence cases):
    a constant v0 plus a small, slowly varying cosine ripple that is zero at k=1.
    """
    k = np.arange(H)
    phase = rng.uniform(0, 2 * math.pi, size=(N, 1))
    ripple = v_amp * (np.cos(0.05 * k[None, :] + phase) - np.cos(phase))
    return v0 + ripple
