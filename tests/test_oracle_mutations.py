"""Planted mistakes in the CPU oracle must each fail a pin.

Each case copies ``oracle/prism_oracle.c``, changes one line the way a
plausible slip would (a dropped term, a wrong sign, a halved step, a wrong
operand), builds the copy with gcc in a temporary directory and runs the pins
of ``test_oracle_pins`` on it.  At least one of the listed pins has to fail.
The oracle in ``oracle/`` itself is never modified; everything runs on the CPU.
"""
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "prism_oracle.c")

# (name, exact text in prism_oracle.c, replacement, pins of which one must fail)
MUTATIONS = [
    ("admm dual step halved",
     "u[k] += g - z[k];", "u[k] += 0.5 * (g - z[k]);",
     [lambda: pins.test_admm_dual_feasibility_after_every_iteration(12, 0.02, 0.4, oracle.SCALE_ROWNORM)]),
    ("admm dual step doubled",
     "u[k] += g - z[k];", "u[k] += 2.0 * (g - z[k]);",
     [lambda: pins.test_admm_dual_feasibility_after_every_iteration(6, 0.05, 1.0, oracle.SCALE_ROWNORM)]),
    ("admm slack step without the multiplier",
     "z[k] = clipd(g + u[k], lo[k], hi[k]);", "z[k] = clipd(g, lo[k], hi[k]);",
     [lambda: pins.test_admm_slack_step_is_the_box_projection(12, 0.02, 0.4, oracle.SCALE_ROWNORM)]),
    ("admm slack step with the multiplier subtracted",
     "z[k] = clipd(g + u[k], lo[k], hi[k]);", "z[k] = clipd(g - u[k], lo[k], hi[k]);",
     [lambda: pins.test_admm_slack_step_is_the_box_projection(6, 0.05, 1.0, oracle.SCALE_ROWNORM)]),
    ("admm right-hand side with the multiplier's sign flipped",
     "s += S->Fs[k * H + i] * (z[k] - u[k]);", "s += S->Fs[k * H + i] * (z[k] + u[k]);",
     [lambda: pins.test_admm_dual_feasibility_after_every_iteration(12, 0.02, 0.4, oracle.SCALE_ROWNORM)]),
    ("admm right-hand side without rho",
     "rhs[i] = xi[i] + rho * s;", "rhs[i] = xi[i] + s;",
     [pins.test_admm_first_primal_step_is_the_argmin]),
    ("rho dropped from the KKT matrix",
     "Mm[i * n + j] = rho * s + (i == j ? 1.0 : 0.0);", "Mm[i * n + j] = s + (i == j ? 1.0 : 0.0);",
     [pins.test_admm_first_primal_step_is_the_argmin, pins.test_paper_first_primal_step_is_the_argmin_of_aug_lag]),
    ("lower bound of the admm rows with the wrong sign",
     "lo[k] = -h[minus_row(H, k)] * S->fs[k];", "lo[k] = h[minus_row(H, k)] * S->fs[k];",
     [lambda: pins.test_brute_force_active_set(3, 12)]),
    ("b_jerk with the wrong sign",
     "bjerk[0] = v0 / (dt * dt);", "bjerk[0] = -v0 / (dt * dt);",
     [pins.test_G_h_matches_printed_matrices_H3]),
    ("exclusive instead of inclusive position sum",
     "for (int j = 0; j <= i; ++j) L[i * H + j] = 1.0;", "for (int j = 0; j < i; ++j) L[i * H + j] = 1.0;",
     [pins.test_G_h_matches_printed_matrices_H3]),
    ("paper slack step with the sign of G x flipped",
     "double v = -g + hs[r];", "double v = g + hs[r];",
     [pins.test_paper_first_primal_step_is_the_argmin_of_aug_lag]),
    ("paper right-hand side with lambda subtracted",
     "rhs[i] = rho * s + lam[i] + xi[i];", "rhs[i] = rho * s - lam[i] + xi[i];",
     [pins.test_paper_mode_fixed_point_relation]),
    ("violation not normalised by the row norm",
     "double v = (g - h[r]) / S->gn[r];", "double v = (g - h[r]);",
     [pins.test_admm_residuals_are_their_definitions]),
    ("last-step size measured against the initial iterate",
     "memcpy(xprev, x, sizeof(double) * H);\n            /* Slack step",
     "if (l == 0) memcpy(xprev, x, sizeof(double) * H);\n            /* Slack step",
     [pins.test_admm_residuals_are_their_definitions]),
    ("paper multiplier step factor delta/2 -> delta (Eq. admm_dual)",
     "lam[i] -= 0.5 * rho * s;", "lam[i] -= rho * s;",
     [lambda: pins.test_paper_stationarity_after_every_iteration(12, 0.02, 0.4, oracle.SCALE_ROWNORM)]),
    ("paper multiplier step factor delta/2 -> delta/4 (Eq. admm_dual)",
     "lam[i] -= 0.5 * rho * s;", "lam[i] -= 0.25 * rho * s;",
     [lambda: pins.test_paper_stationarity_after_every_iteration(6, 0.05, 1.0, oracle.SCALE_ROWNORM)]),
    ("paper multiplier step with the sign flipped (Eq. admm_dual)",
     "lam[i] -= 0.5 * rho * s;", "lam[i] += 0.5 * rho * s;",
     [lambda: pins.test_paper_stationarity_after_every_iteration(10, 0.1, 2.5, oracle.SCALE_NONE)]),
]


def _build_mutant(tmp_path, find, repl):
    src = open(SRC).read()
    assert src.count(find) == 1, f"mutation anchor not unique or missing: {find!r}"
    path = tmp_path / "mut.c"
    path.write_text(src.replace(find, repl))
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(lib),
                           str(path), "-lm"])
    return str(lib)


@pytest.mark.parametrize("name,find,repl,checks", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, name, find, repl, checks):
    for chk in checks:   # the pins pass on the real oracle
        chk()
    lib = _build_mutant(tmp_path, find, repl)
    caught = []
    with oracle.swapped_library(lib):
        for chk in checks:
            try:
                chk()
            except (AssertionError, ValueError):
                caught.append(chk)
    assert caught, f"planted mistake '{name}' passed every listed pin"
