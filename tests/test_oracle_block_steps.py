"""Step-wise pins of the oracle's block solve (Sec. 3.1.4, Eq. 14) over a fixed number of
damped Gauss-Newton steps.

tests/golden/block_steps.json holds trajectories written by tests/golden/make_block_steps.py
from oracle/steps_restated.py, a second statement of the block solve that shares no code
with oracle/dba_oracle.c (the stacked Jacobian of the block's pixels by complex steps of the
whole block vector, dense products with the weights, numpy LU).  Every GPU parity test of
the block path compares a few-step trajectory of every block, so ora_block_solve must be
right step by step: each golden case is replayed with 1, 2, ... steps.  The cases cover
one-point, one-camera and wider blocks, a single-observation block, rejected steps, steps
taken by the rounding-noise rule, a binding damping clamp, a trial behind a camera, a
start with an observation behind its camera, and rejected steps whose predicted decrease is
small but far above the rounding noise (the noise rule must not trust them).

The mutation tests plant mistakes in a copy of the C oracle's block solve (a dropped dual,
a transposed camera index, a wrong penalty, the damping start over 9 unknowns instead of
the block's) and check that the same pins reject every one of them.
"""
import ctypes
import json
import os
import subprocess

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "block_steps.json")
ORACLE_SRC = os.path.join(os.path.dirname(os.path.abspath(O.__file__)), "dba_oracle.c")

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
                    lm_model_tol=c["lm_model_tol"])


def _solve(lib, case, steps, **over):
    cfg = _cfg(case, steps, **over)
    np_, nc = len(case["xbar"]) // 3, len(case["ybar"]) // 6
    v = np.array(case["v"][0], dtype=np.float64)
    X, Y = v[:3 * np_].copy(), v[3 * np_:].copy()
    arr = {k: np.ascontiguousarray(case[k], dtype=np.float64) for k in ("z", "xbar", "ybar", "rx", "sy")}
    opl = np.ascontiguousarray(case["opl"], dtype=np.int32)
    ocl = np.ascontiguousarray(case["ocl"], dtype=np.int32)
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    lib.ora_block_solve(ctypes.byref(cfg), np_, nc, len(opl), opl.ctypes.data_as(ip), ocl.ctypes.data_as(ip),
                        *[arr[k].ctypes.data_as(dp) for k in ("z", "xbar", "ybar", "rx", "sy")],
                        X.ctypes.data_as(dp), Y.ctypes.data_as(dp))
    return np.concatenate([X, Y])


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


def test_golden_cases_cover_every_rule_and_block_shape():
    cases = _cases()
    codes = "".join(c["codes"] for c in cases)
    assert {"A", "R", "T"} <= set(codes)
    names = [c["name"] for c in cases]
    for need in ("1x3", "5x1", "4x2", "8x2", "4x4", "1x1", "clamp", "at-minimum", "behind-camera-trial",
                 "behind-camera-start", "reject", "small-prediction-reject", "single_rho_y", "rho_angle", "l2",
                 "huber", "student"):
        assert any(need in n for n in names), need
    shapes = {(len(c["xbar"]) // 3, len(c["ybar"]) // 6) for c in cases}
    assert {(1, 3), (5, 1), (4, 2), (8, 2), (4, 4), (1, 1)} <= shapes
    # every observation's indices address a copy of its block
    for c in cases:
        assert max(c["opl"]) < len(c["xbar"]) // 3 and max(c["ocl"]) < len(c["ybar"]) // 6
        assert len(c["z"]) == 2 * len(c["opl"])


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_oracle_block_solve_follows_golden_steps(case):
    assert _worst(O.lib(), case) <= 1.0


# Planted mistakes: (name, text of the oracle's block solve, replacement).  Each text occurs
# exactly once in ora_block_solve.
MUTATIONS = [
    ("point dual dropped", "g[u] += rx[u] + rho_of(c, a)", "g[u] += rho_of(c, a)"),
    ("camera dual dropped", "g[u] += sy[6 * q + a] + rho_of(c, 3 + a)", "g[u] += rho_of(c, 3 + a)"),
    ("camera penalty of the angles for every component", "H[(size_t)u * n + u] += rho_of(c, 3 + a);",
     "H[(size_t)u * n + u] += rho_of(c, 3);"),
    ("camera copies in reverse order", "col[3 + a] = 3 * np + 6 * ocl[k] + a;",
     "col[3 + a] = 3 * np + 6 * (nc - 1 - ocl[k]) + a;"),
    ("damping start over 9 unknowns", "lambda = c->lm_lambda0 * tr / (double)n;",
     "lambda = c->lm_lambda0 * tr / 9.0;"),
    ("second pixel coordinate dropped from the gradient", "g[col[a]] += -2.0 * w * (J[a] * e0 + J[9 + a] * e1);",
     "g[col[a]] += -2.0 * w * (J[a] * e0);"),
    ("weights left out of the Gauss-Newton matrix",
     "H[(size_t)col[a] * n + col[b]] += 2.0 * w * (J[a] * J[b] + J[9 + a] * J[9 + b]);",
     "H[(size_t)col[a] * n + col[b]] += 2.0 * (J[a] * J[b] + J[9 + a] * J[9 + b]);"),
    ("point-camera coupling dropped", "for (int b = 0; b < 9; ++b)\n",
     "for (int b = (a < 3 ? 0 : 3); b < (a < 3 ? 3 : 9); ++b)\n"),
    ("predicted decrease shifted by 0.5 (steps that increase Eq. (14) trusted)", "double gd = 0.0, dd = 0.0;",
     "double gd = 1.0, dd = 0.0;"),
    ("misfit kept behind the camera at the linearisation point",
     "if (!(depth > c->eps_depth)) continue; /* no misfit term at this linearisation point */", ""),
]


def _mutant(tmp_path, name, old, new):
    """The oracle compiled with one planted mistake in its block solve (CPU only)."""
    src = open(ORACLE_SRC).read()
    start = src.index("void ora_block_solve(")
    end = src.index("int ora_block_iterate(", start)
    body = src[start:end]
    assert body.count(old) == 1, name
    path = tmp_path / ("mut_" + "".join(ch if ch.isalnum() else "_" for ch in name))
    path.with_suffix(".c").write_text(src[:start] + body.replace(old, new) + src[end:])
    so = path.with_suffix(".so")
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-I", os.path.dirname(ORACLE_SRC), "-o", str(so), str(path.with_suffix(".c")), "-lm"]
    subprocess.run(cmd, check=True, capture_output=True)
    L = ctypes.CDLL(str(so))
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    L.ora_block_solve.argtypes = [ctypes.POINTER(O.Config), ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip,
                                  dp, dp, dp, dp, dp, dp, dp]
    L.ora_block_solve.restype = None
    return L


@pytest.mark.parametrize("mutation", MUTATIONS, ids=lambda m: m[0])
def test_pins_reject_a_planted_mistake_in_the_block_solve(tmp_path, mutation):
    lib = _mutant(tmp_path, *mutation)
    assert any(_worst(lib, c) > 1.0 for c in _cases()), mutation[0]


def test_unmutated_copy_passes_the_pins(tmp_path):
    """The mutation harness itself: the copy compiled without a change follows every case."""
    lib = _mutant(tmp_path, "none", "void ora_block_solve(", "void ora_block_solve(")
    assert all(_worst(lib, c) <= 1.0 for c in _cases())


def test_pins_reject_a_changed_damping_start_or_clamp():
    cases = _cases()
    lib = O.lib()
    assert any(_worst(lib, c, lm_lambda0=1.1e-3) > 1.0 for c in cases if c["cfg"]["lm_lambda0"] == 1e-3)
    assert any(_worst(lib, c, lm_lambda0=0.9e-3) > 1.0 for c in cases if c["cfg"]["lm_lambda0"] == 1e-3)
    clamp = [c for c in cases if "clamp" in c["name"]]
    base = clamp[0]["cfg"]["lm_lambda_min"]
    assert _worst(lib, clamp[0], lm_lambda_min=1.2 * base) > 1.0
    assert _worst(lib, clamp[0], lm_lambda_min=0.8 * base) > 1.0


def test_golden_file_is_what_the_restatement_writes():
    """A few stored trajectories recomputed from oracle/steps_restated.py, bit for bit."""
    from oracle import steps_restated as R

    cases = _cases()
    picks = [cases[0], next(c for c in cases if "reject" in c["name"]),
             next(c for c in cases if c["name"] == "behind-camera-start")]
    for case in picks:
        blk = {k: np.array(case[k]) for k in ("z", "xbar", "ybar", "rx", "sy")}
        blk["opl"], blk["ocl"] = case["opl"], case["ocl"]
        traj = R.block_gauss_newton(case["cfg"], blk, np.array(case["v"][0]), len(case["v"]) - 1)[0]
        np.testing.assert_array_equal(np.array(traj), np.array(case["v"]))


def test_block_objective_matches_the_restatement():
    """The value of Eq. (14), not only its differences (which are all a solve compares), against
    the restated objective at every golden point, +inf where an observation is behind its camera."""
    from oracle import steps_restated as R

    n_inf = 0
    for case in _cases():
        cfg = _cfg(case, 1)
        blk = {k: np.array(case[k]) for k in ("z", "xbar", "ybar", "rx", "sy")}
        blk["opl"], blk["ocl"] = case["opl"], case["ocl"]
        np_ = len(case["xbar"]) // 3
        for v in case["v"]:
            v = np.array(v)
            want = R.block_objective(case["cfg"], blk, v)
            got = O.block_objective(cfg, case["opl"], case["ocl"], blk["z"], blk["xbar"], blk["ybar"], blk["rx"],
                                    blk["sy"], v[:3 * np_], v[3 * np_:])
            if np.isinf(want):
                n_inf += 1
                assert got == np.inf, case["name"]
            else:
                assert abs(got - want) <= 1e-12 * max(abs(want), 1.0), case["name"]
    assert n_inf >= 1


def test_one_observation_block_restates_the_local_solve():
    """The two restatements agree where Eq. (14) is Eq. (9): a block of one point, one camera
    and one observation takes the local solve's steps (to rounding: the two assemble the
    same 9 x 9 system by different products)."""
    from oracle import steps_restated as R

    for case in (c for c in _cases() if (len(c["xbar"]), len(c["ybar"])) == (3, 6)):
        cfg, n = case["cfg"], len(case["v"]) - 1
        blk = {k: np.array(case[k]) for k in ("z", "xbar", "ybar", "rx", "sy")}
        blk["opl"], blk["ocl"] = case["opl"], case["ocl"]
        local = {"z": blk["z"], "vbar": np.r_[blk["xbar"], blk["ybar"]], "dual": np.r_[blk["rx"], blk["sy"]]}
        a, ca, _ = R.gauss_newton(cfg, local, np.array(case["v"][0]), n)
        assert ca == case["codes"], case["name"]
        v0 = np.array(case["v"][0])
        for k in range(1, n + 1):
            tol = REL_TRAVEL * np.abs(a[k] - v0).max() + REL_COORD * np.abs(a[k]).max()
            assert np.abs(np.array(case["v"][k]) - a[k]).max() <= tol, (case["name"], k)
