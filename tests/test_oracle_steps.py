"""Step-wise pins of the oracle's local solvers (Sec. 3.1, Eq. 9) over a fixed number of
steps.

tests/golden/local_steps.json holds trajectories written by
tests/golden/make_local_steps.py from oracle/steps_restated.py, a second statement of the
damped Gauss-Newton and L-BFGS solves that shares no code with oracle/dba_oracle.c
(complex-step Jacobians and gradients, numpy LU solves, the dense BFGS product form).
Every GPU parity test compares a few-step trajectory, so the oracle must be right step
by step, not only at convergence: each golden case is replayed through ora_local_solve /
ora_local_solve_lbfgs with 1, 2, ... steps.  The cases include rejected steps, steps
taken by the rounding-noise rule, a binding damping clamp, a trial behind the camera,
both camera-penalty readings and L-BFGS backtracking.

The mutation tests build deliberately wrong oracles on the CPU (each damping or line-search
constant changed once, or the damping start and clamp changed through the configuration)
and check that the same pins reject every one of them.
"""
import ctypes
import json
import os
import subprocess

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "local_steps.json")
ORACLE_DIR = os.path.dirname(os.path.abspath(O.__file__))

# A trajectory point may differ from the golden one by rounding only: relative to the
# distance travelled from the start, plus a few ulps of the coordinates themselves.
REL_TRAVEL, REL_COORD = 1e-9, 1e-14


def _cases():
    with open(GOLDEN) as fh:
        return json.load(fh)["cases"]


def _cfg(case, steps, **over):
    c = dict(case["cfg"])
    c.update(over)
    return O.config(focal=c["focal"], cx=c["cx"], cy=c["cy"], loss=c["loss"], loss_param=c["loss_param"],
                    rho_x=c["rho_x"], rho_y=c["rho_y"], rho_angle=c["rho_angle"], inner_steps=steps,
                    lm_lambda0=c["lm_lambda0"], lm_lambda_min=c["lm_lambda_min"], eps_depth=c["eps_depth"],
                    lm_model_tol=c["lm_model_tol"],
                    local_solver=O.SOLVER_LBFGS if case["solver"] == "lbfgs" else O.SOLVER_GN)


def _solve(lib, case, steps, **over):
    cfg = _cfg(case, steps, **over)
    z = np.array(case["z"])
    vbar = np.array(case["vbar"])
    dual = np.array(case["dual"])
    v = np.array(case["v"][0], dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    args = [ctypes.byref(cfg), z.ctypes.data_as(dp), vbar[:3].copy().ctypes.data_as(dp),
            vbar[3:].copy().ctypes.data_as(dp), dual.ctypes.data_as(dp), v.ctypes.data_as(dp)]
    fn = lib.ora_local_solve_lbfgs if case["solver"] == "lbfgs" else lib.ora_local_solve
    fn(*args)
    return v


def _worst(lib, case, **over):
    """Largest excess over the tolerance along the case's trajectory (<= 1 passes)."""
    v0 = np.array(case["v"][0])
    worst = 0.0
    for k in range(1, len(case["v"])):
        want = np.array(case["v"][k])
        got = _solve(lib, case, k, **over)
        tol = REL_TRAVEL * np.abs(want - v0).max() + REL_COORD * np.abs(want).max()
        err = np.abs(got - want).max() / tol
        worst = max(worst, err if np.isfinite(err) else np.inf)  # a NaN result fails
    return worst


def test_golden_cases_cover_every_rule():
    cases = _cases()
    codes = "".join(c.get("codes", "") for c in cases)
    assert {"A", "R", "T"} <= set(codes)
    names = [c["name"] for c in cases]
    for need in ("clamp", "behind-camera", "at-minimum", "single_rho_y", "rho_angle", "l2", "huber", "student"):
        assert any(need in n for n in names), need
    trials = [int(t) for c in cases if c["solver"] == "lbfgs" for t in c["trials"].split(",")]
    assert max(trials) >= 3  # line searches that backtrack
    assert max(len(c["v"]) for c in cases if c["solver"] == "lbfgs") >= 6  # history beyond the memory


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_oracle_local_solve_follows_golden_steps(case):
    assert _worst(O.lib(), case) <= 1.0


def _mutant(tmp_path, defines):
    """The oracle compiled with some constants changed (a planted mistake, CPU only)."""
    so = tmp_path / ("mut_" + "_".join(d.split("=")[0] for d in defines) + ".so")
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           *[f"-D{d}" for d in defines], "-o", str(so), os.path.join(ORACLE_DIR, "dba_oracle.c"), "-lm"]
    subprocess.run(cmd, check=True, capture_output=True)
    L = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    for fn in (L.ora_local_solve, L.ora_local_solve_lbfgs):
        fn.argtypes = [ctypes.POINTER(O.Config), dp, dp, dp, dp, dp]
    return L


def _rejected(lib, cases, **over):
    return any(_worst(lib, c, **over) > 1.0 for c in cases)


@pytest.mark.parametrize("defines", [["ORA_LM_INCREASE=9.0"], ["ORA_LM_INCREASE=11.0"], ["ORA_LM_DECREASE=9.0"],
                                     ["ORA_LM_DECREASE=11.0"]])
def test_pins_reject_a_changed_damping_schedule(tmp_path, defines):
    cases = [c for c in _cases() if c["solver"] == "gn"]
    assert _rejected(_mutant(tmp_path, defines), cases)


@pytest.mark.parametrize("defines", [["ORA_LBFGS_ARMIJO=0.3"], ["ORA_LBFGS_MEMORY=3"], ["ORA_LBFGS_MEMORY=5"],
                                     ["ORA_LBFGS_HALVINGS=2"]])
def test_pins_reject_a_changed_line_search(tmp_path, defines):
    cases = [c for c in _cases() if c["solver"] == "lbfgs"]
    assert _rejected(_mutant(tmp_path, defines), cases)


def test_pins_reject_a_changed_damping_start_or_clamp():
    """The rounding-noise rule is not among these: it decides only steps that move a copy by
    rounding-level amounts, below any trajectory tolerance.  It is pinned by
    test_local_solve_noise_rule_keeps_the_minimum and
    test_admm_is_insensitive_to_last_bit_perturbations in test_oracle.py."""
    gn = [c for c in _cases() if c["solver"] == "gn"]
    lib = O.lib()
    assert _rejected(lib, gn, lm_lambda0=1.1e-3)
    assert _rejected(lib, gn, lm_lambda0=0.9e-3)
    clamp = [c for c in gn if "clamp" in c["name"]]
    base = clamp[0]["cfg"]["lm_lambda_min"]
    assert _rejected(lib, clamp, lm_lambda_min=1.2 * base)
    assert _rejected(lib, clamp, lm_lambda_min=0.8 * base)


def test_golden_file_is_what_the_restatement_writes():
    """A few stored trajectories recomputed from oracle/steps_restated.py, bit for bit."""
    from oracle import steps_restated as R

    cases = _cases()
    for case in (cases[0], cases[1], next(c for c in cases if "reject" in c["name"])):
        c = {k: np.array(case[k]) for k in ("z", "vbar", "dual")}
        n = len(case["v"]) - 1
        if case["solver"] == "gn":
            traj = R.gauss_newton(case["cfg"], c, np.array(case["v"][0]), n)[0]
        else:
            traj = R.lbfgs(case["cfg"], c, np.array(case["v"][0]), n)[0]
        np.testing.assert_array_equal(np.array(traj), np.array(case["v"]))
