"""Iteration-wise pins of the oracle's consensus ADMM iteration (Sec. 3.1, Eqs. 9-13), per
observation (ora_admm_iterate) and with block subproblems (Sec. 3.1.4, Eq. 14;
ora_block_iterate).

tests/golden/admm_steps.json holds iterates written by tests/golden/make_admm_steps.py from
oracle/steps_restated.py, a second statement of the iteration that shares no code with
oracle/dba_oracle.c: its local solves are the restated Gauss-Newton solve, its consensus is
the least-squares minimiser of each point's and camera's part of the augmented Lagrangian,
and its duals ascend by rho (copy - new consensus); one case takes the L-BFGS local solve,
whose dispatch the invariants cannot see either.  The block cases solve each block by the
restated block solve over the oracle's block layout (pinned against brute-force grouping)
and take each consensus over the copies, one per block that holds the point or camera.
Both oracle iterations are replayed over every case and compared after each iteration.

The invariants pinned elsewhere (duals summing to zero per point and camera, the noise-free
fixed point, the centralized optimum at convergence) hold for any positive dual step, so a
dual ascent with the wrong penalty or against the old consensus passes them; the mutation
tests plant such mistakes in a copy of the C iteration and check that these pins reject them.
"""
import ctypes
import json
import os
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_1708_07954_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "admm_steps.json")
ORACLE_SRC = os.path.join(os.path.dirname(os.path.abspath(O.__file__)), "dba_oracle.c")

# Per column: parameters and copies within REL of the column's largest magnitude; duals,
# formed as rho (copy - consensus), within REL of rho times the copies' column magnitude.
REL = 1e-12


def _cases():
    with open(GOLDEN) as fh:
        return json.load(fh)["cases"]


def _scene(case):
    z = np.array(case["z"])
    cams0, pts0 = np.array(case["cams0"]), np.array(case["pts0"])
    l = len(case["pt_idx"])
    return S.Scene(n_cams=case["n_cams"], n_pts=case["n_pts"], pt_idx=np.array(case["pt_idx"], dtype=np.int32),
                   cam_idx=np.array(case["cam_idx"], dtype=np.int32), z=z, z_true=z.copy(),
                   outlier=np.zeros(l, dtype=bool), cams_gt=cams0.copy(), pts_gt=pts0.copy(), cams0=cams0,
                   pts0=pts0, focal=case["cfg"]["focal"], cx=case["cfg"]["cx"], cy=case["cfg"]["cy"])


def _cfg(case):
    c = case["cfg"]
    return O.config(focal=c["focal"], cx=c["cx"], cy=c["cy"], loss=c["loss"], loss_param=c["loss_param"],
                    rho_x=c["rho_x"], rho_y=c["rho_y"], rho_angle=c["rho_angle"], inner_steps=case["steps"],
                    lm_lambda0=c["lm_lambda0"], lm_lambda_min=c["lm_lambda_min"], eps_depth=c["eps_depth"],
                    lm_model_tol=c["lm_model_tol"],
                    local_solver=O.SOLVER_LBFGS if case.get("solver") == "lbfgs" else O.SOLVER_GN)


def _rho(case):
    c = case["cfg"]
    ra = c["rho_angle"] if c["rho_angle"] > 0 else c["rho_y"]
    return np.array([c["rho_x"]] * 3 + [ra] * 3 + [c["rho_y"]] * 3)


def _excess(got, want, scale):
    """Largest error in units of the tolerance; +inf for a NaN (which a running max would drop)."""
    err = float((np.abs(got - want) / (REL * np.maximum(scale, 1e-300))).max())
    return err if np.isfinite(err) else np.inf


def _worst(iterate, case):
    """Largest excess over the tolerance along the case (<= 1 passes); iterate(state) runs one
    iteration of the oracle under test on an oracle.State."""
    st = O.State(_scene(case))
    rho = _rho(case)
    worst = 0.0
    for it in range(1, len(case["cams"]) + 1):
        iterate(st)
        cams, pts = np.array(case["cams"][it - 1]), np.array(case["pts"][it - 1])
        worst = max(worst, _excess(st.cams, cams, np.abs(cams).max(axis=0)),
                    _excess(st.pts, pts, np.abs(pts).max(axis=0)))
        if str(it) in case["copies"]:
            copies, duals = np.array(case["copies"][str(it)]), np.array(case["duals"][str(it)])
            worst = max(worst, _excess(st.copies, copies, np.abs(copies).max(axis=0)),
                        _excess(st.duals, duals, rho * np.abs(copies).max(axis=0)))
    return worst


def test_golden_cases_cover_the_readings():
    cases = _cases()
    names = " ".join(c["name"] for c in cases)
    for need in ("rho_angle", "single_rho_y", "rho_x_half", "unobserved", "huber", "l2", "student", "lbfgs"):
        assert need in names, need
    assert any(c.get("solver") == "lbfgs" for c in cases)
    for c in cases:
        assert len(c["cams"]) >= 3 and str(len(c["cams"])) in c["copies"]
    # the unobserved point and camera are the last ones and keep their starting values
    c = next(c for c in cases if "unobserved" in c["name"])
    assert c["n_pts"] - 1 not in c["pt_idx"] and c["n_cams"] - 1 not in c["cam_idx"]
    assert c["pts"][-1][-1] == c["pts0"][-1] and c["cams"][-1][-1] == c["cams0"][-1]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_oracle_admm_iteration_follows_golden_iterates(case):
    cfg = _cfg(case)
    assert _worst(lambda st: st.iterate(cfg, 1), case) <= 1.0


_WARM_FROM_CONSENSUS = (
    "    for (long o = 0; o < n_obs; ++o) {\n"
    "      for (int k = 0; k < 3; ++k) copies[9 * o + k] = pts[3 * (long)pt_idx[o] + k];\n"
    "      for (int k = 0; k < 6; ++k) copies[9 * o + 3 + k] = cams[6 * (long)cam_idx[o] + k];\n"
    "    }\n")

# Planted mistakes: (name, text of ora_admm_iterate, replacement); each text occurs once.
MUTATIONS = [
    ("point duals ascend against the old consensus",
     "duals[9 * o + k] += c->rho_x * (copies[9 * o + k] - pts[3 * i + k]);",
     "duals[9 * o + k] += c->rho_x * (copies[9 * o + k] - pts_prev[3 * i + k]);"),
    ("camera duals ascend by rho_y for every component",
     "duals[9 * o + 3 + k] += rho_of(c, 3 + k) *", "duals[9 * o + 3 + k] += c->rho_y *"),
    ("point duals ascend by the camera penalty", "duals[9 * o + k] += c->rho_x *", "duals[9 * o + k] += c->rho_y *"),
    ("dual ascent reversed", "duals[9 * o + k] += c->rho_x *", "duals[9 * o + k] -= c->rho_x *"),
    ("camera consensus not a mean", "cams[6 * j + k] = sum_y[6 * j + k] / (double)cnt_y[j];",
     "cams[6 * j + k] = sum_y[6 * j + k] / (double)(cnt_y[j] + 1);"),
    ("the L-BFGS local solve ignored", "if (c->local_solver == ORA_SOLVER_LBFGS)", "if (0)"),
    ("local solves warm-started at the consensus",
     "    /* Eq. (9): every observation's local subproblem, warm-started at its copy. */\n",
     _WARM_FROM_CONSENSUS),
]


def _mutant(tmp_path, name, old, new):
    """The oracle compiled with one planted mistake in its ADMM iteration (CPU only)."""
    src = open(ORACLE_SRC).read()
    start = src.index("int ora_admm_iterate(")
    end = src.index("void ora_eval(", start)
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
    L.ora_admm_iterate.argtypes = [ctypes.POINTER(O.Config), ctypes.c_int, ctypes.c_int, ctypes.c_long, ip, ip,
                                   dp, dp, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    L.ora_admm_iterate.restype = ctypes.c_int
    return L


def _iterate_with(lib, case):
    cfg = _cfg(case)
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)

    def step(st):
        s = st.scene
        rc = lib.ora_admm_iterate(ctypes.byref(cfg), s.n_cams, s.n_pts, s.n_obs, s.pt_idx.ctypes.data_as(ip),
                                  s.cam_idx.ctypes.data_as(ip), np.ascontiguousarray(s.z).ctypes.data_as(dp), None,
                                  st.copies.ctypes.data_as(dp), st.duals.ctypes.data_as(dp),
                                  st.cams.ctypes.data_as(dp), st.pts.ctypes.data_as(dp), 1, 1, None)
        assert rc == 0

    return step


@pytest.mark.parametrize("mutation", MUTATIONS, ids=lambda m: m[0])
def test_pins_reject_a_planted_mistake_in_the_iteration(tmp_path, mutation):
    lib = _mutant(tmp_path, *mutation)
    assert any(_worst(_iterate_with(lib, c), c) > 1.0 for c in _cases()), mutation[0]


def test_unmutated_copy_passes_the_pins(tmp_path):
    lib = _mutant(tmp_path, "none", "int ora_admm_iterate(", "int ora_admm_iterate(")
    assert all(_worst(_iterate_with(lib, c), c) <= 1.0 for c in _cases())


# ------------------------------------------------------------ block subproblems (Eq. 14)
def _block_cases():
    with open(GOLDEN) as fh:
        return json.load(fh)["block_cases"]


def _block_worst(iterate, case):
    """As _worst, over an oracle.BlockState of the case's (pi, kappa)."""
    st = O.BlockState(_scene(case), case["pi"], case["kappa"])
    rho = _rho(case)
    worst = 0.0
    for it in range(1, len(case["cams"]) + 1):
        iterate(st)
        cams, pts = np.array(case["cams"][it - 1]), np.array(case["pts"][it - 1])
        worst = max(worst, _excess(st.cams, cams, np.abs(cams).max(axis=0)),
                    _excess(st.pts, pts, np.abs(pts).max(axis=0)))
        if str(it) in case["copies"]:
            cp, du = case["copies"][str(it)], case["duals"][str(it)]
            for got_c, got_d, key, r in ((st.pcopies, st.pduals, "points", rho[:3]),
                                         (st.ccopies, st.cduals, "cameras", rho[3:])):
                want_c, want_d = np.array(cp[key]), np.array(du[key])
                scale = np.abs(want_c).max(axis=0)
                worst = max(worst, _excess(got_c, want_c, scale), _excess(got_d, want_d, r * scale))
    return worst


def test_golden_block_cases_cover_every_block_kind():
    cases = _block_cases()
    shapes = {tuple(s) for c in cases for s in c["block_shapes"]}
    assert {(1, 1), (1, 3), (5, 1), (4, 2), (3, 2)} <= shapes
    names = " ".join(c["name"] for c in cases)
    for need in ("rho_angle", "single_rho_y", "rho_x_half", "unobserved", "huber", "l2", "student"):
        assert need in names, need
    assert any("R" in "".join(c["codes"]) for c in cases)


@pytest.mark.parametrize("case", _block_cases(), ids=lambda c: c["name"])
def test_oracle_block_iteration_follows_golden_iterates(case):
    cfg = _cfg(case)
    assert _block_worst(lambda st: st.iterate(cfg, 1, with_gt=False), case) <= 1.0


_BLOCK_WARM_FROM_CONSENSUS = (
    "      for (int u = 0; u < 3 * np; ++u) pcopies[3 * pc_off[b] + u] = xbar[u];\n"
    "      for (int u = 0; u < 6 * nc; ++u) ccopies[6 * cc_off[b] + u] = ybar[u];\n"
    "      ora_block_solve(c, np, nc, no,")

_CONSENSUS_PER_OBSERVATION = (
    "    for (long b = 0; b < n_blocks; ++b)\n"
    "      for (long q = obs_off[b]; q < obs_off[b + 1]; ++q) {\n"
    "        long k = pc_off[b] + obs_lp[q], i = pc_pt[k];\n"
    "        for (int a = 0; a < 3; ++a) sum_x[3 * i + a] += pcopies[3 * k + a] + pduals[3 * k + a] / rho_of(c, a);\n"
    "        cnt_x[i] += 1;\n"
    "      }\n")

# Planted mistakes in ora_block_iterate (each text occurs once in it).
BLOCK_MUTATIONS = [
    ("point-copy duals ascend against the old consensus",
     "pduals[3 * k + a] += rho_of(c, a) * (pcopies[3 * k + a] - pts[3 * (long)pc_pt[k] + a]);",
     "pduals[3 * k + a] += rho_of(c, a) * (pcopies[3 * k + a] - pts_prev[3 * (long)pc_pt[k] + a]);"),
    ("camera-copy duals ascend by rho_y for every component",
     "cduals[6 * k + a] += rho_of(c, 3 + a) *", "cduals[6 * k + a] += c->rho_y *"),
    ("camera-copy dual ascent reversed", "cduals[6 * k + a] += rho_of(c, 3 + a) *",
     "cduals[6 * k + a] -= rho_of(c, 3 + a) *"),
    ("point consensus weights each copy by its observations",
     "    for (long k = 0; k < n_pc; ++k) {\n"
     "      long i = pc_pt[k];\n"
     "      for (int a = 0; a < 3; ++a) sum_x[3 * i + a] += pcopies[3 * k + a] + pduals[3 * k + a] / rho_of(c, a);\n"
     "      cnt_x[i] += 1;\n"
     "    }\n", _CONSENSUS_PER_OBSERVATION),
    ("block solves warm-started at the consensus", "      ora_block_solve(c, np, nc, no,",
     _BLOCK_WARM_FROM_CONSENSUS),
]


def _block_mutant(tmp_path, name, old, new):
    src = open(ORACLE_SRC).read()
    start = src.index("int ora_block_iterate(")
    body = src[start:]
    assert body.count(old) == 1, name
    path = tmp_path / ("mutb_" + "".join(ch if ch.isalnum() else "_" for ch in name))
    path.with_suffix(".c").write_text(src[:start] + body.replace(old, new))
    so = path.with_suffix(".so")
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-I", os.path.dirname(ORACLE_SRC), "-o", str(so), str(path.with_suffix(".c")), "-lm"]
    subprocess.run(cmd, check=True, capture_output=True)
    L = ctypes.CDLL(str(so))
    L.ora_block_iterate.argtypes = O.lib().ora_block_iterate.argtypes
    L.ora_block_iterate.restype = ctypes.c_int
    return L


def _block_iterate_with(lib, case):
    cfg = _cfg(case)

    def step(st):
        s, B = st.scene, st.layout
        ip, lp = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_long)
        dp = ctypes.POINTER(ctypes.c_double)
        I = lambda a: a.ctypes.data_as(ip)  # noqa: E731
        L = lambda a: a.ctypes.data_as(lp)  # noqa: E731
        D = lambda a: a.ctypes.data_as(dp)  # noqa: E731
        rc = lib.ora_block_iterate(ctypes.byref(cfg), s.n_cams, s.n_pts, s.n_obs, I(s.pt_idx), I(s.cam_idx),
                                   D(np.ascontiguousarray(s.z)), None, B.n_blocks, L(B.obs_off), L(B.blk_obs),
                                   I(B.obs_lp), I(B.obs_lc), L(B.pc_off), I(B.pc_pt), L(B.cc_off), I(B.cc_cam),
                                   D(st.pcopies), D(st.pduals), D(st.ccopies), D(st.cduals), D(st.cams), D(st.pts),
                                   1, 1, None)
        assert rc == 0

    return step


@pytest.mark.parametrize("mutation", BLOCK_MUTATIONS, ids=lambda m: m[0])
def test_pins_reject_a_planted_mistake_in_the_block_iteration(tmp_path, mutation):
    lib = _block_mutant(tmp_path, *mutation)
    assert any(_block_worst(_block_iterate_with(lib, c), c) > 1.0 for c in _block_cases()), mutation[0]


def test_unmutated_block_copy_passes_the_pins(tmp_path):
    lib = _block_mutant(tmp_path, "none", "int ora_block_iterate(", "int ora_block_iterate(")
    assert all(_block_worst(_block_iterate_with(lib, c), c) <= 1.0 for c in _block_cases())


def test_golden_file_is_what_the_restatement_writes():
    """The first case's first two iterations recomputed from oracle/steps_restated.py, bit for bit."""
    from oracle import steps_restated as R

    case = _cases()[0]
    sc = _scene(case)
    cams, pts = sc.cams0.copy(), sc.pts0.copy()
    copies = np.concatenate([pts[sc.pt_idx], cams[sc.cam_idx]], axis=1)
    duals = np.zeros_like(copies)
    for it in (1, 2):
        copies, duals, cams, pts, _, _ = R.admm_iteration(case["cfg"], sc.pt_idx, sc.cam_idx, sc.z, copies, duals,
                                                          cams, pts, case["steps"])
        np.testing.assert_array_equal(cams, np.array(case["cams"][it - 1]))
        np.testing.assert_array_equal(pts, np.array(case["pts"][it - 1]))
        if str(it) in case["duals"]:
            np.testing.assert_array_equal(duals, np.array(case["duals"][str(it)]))
