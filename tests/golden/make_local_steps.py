"""Writes tests/golden/local_steps.json: step-wise golden trajectories of the two local
solvers of Eq. (9) (Sec. 3.1), for the tests that pin the oracle's ora_local_solve and
ora_local_solve_lbfgs over a fixed number of steps.

The values come from oracle/steps_restated.py, a second statement of those solvers that
shares no code with the C oracle (complex-step derivatives, numpy LU, dense BFGS form).
Inputs are seeded draws around the synthetic scenes of paper_1708_07954_gb300.scenes.
Each case keeps the leading steps whose every decision is far from its threshold
(objective comparisons by more than 1e-11 relative, noise-rule ratios outside
[1e-2, 1e2]), so that rounding differences between the two statements (~1e-15) cannot
flip one; a solve that has reached rounding level ends its clean prefix.  The case set covers
rejected steps, steps accepted by the rounding-noise rule, a binding damping clamp, a
trial behind the camera, the paper's single camera penalty (rho_angle 0) and a separate
angle penalty, all three misfits, and L-BFGS line searches that backtrack.

    python tests/golden/make_local_steps.py      # rewrites local_steps.json
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import steps_restated as R  # noqa: E402
from paper_1708_07954_gb300 import scenes as S  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "local_steps.json")
STEPS = 6


def base_cfg(scene, loss, rho_angle_on):
    p = {S.LOSS_L2: 0.0, S.LOSS_HUBER: 2.0, S.LOSS_STUDENT_T: 4.0}[loss]
    return {"focal": scene.focal, "cx": scene.cx, "cy": scene.cy, "loss": loss, "loss_param": p,
            "rho_x": scene.rho_x, "rho_y": scene.rho_y, "rho_angle": scene.rho_angle if rho_angle_on else 0.0,
            "lm_lambda0": 1e-3, "lm_lambda_min": 1e-12, "eps_depth": 1e-6, "lm_model_tol": 16.0}


def draw(scene, cfg, rng, pix_sigma, outlier_px, start_sigma, dual_sigma):
    """One local problem: an observation of the scene, its consensus (the initial estimate),
    a perturbed pixel, duals rho (copy - consensus) for copy offsets of a plausible size, and a
    start displaced from the consensus."""
    o = int(rng.integers(scene.n_obs))
    vbar = np.r_[scene.pts0[scene.pt_idx[o]], scene.cams0[scene.cam_idx[o]]]
    z = scene.z[o] + rng.normal(0, pix_sigma, 2)
    if outlier_px:
        z = z + rng.choice([-1, 1], 2) * outlier_px
    scale = np.r_[np.full(3, scene.depth * 1e-3), np.full(3, 1e-3), np.full(3, scene.depth * 1e-3)]
    dual = R.rho_vec(cfg) * rng.normal(0, dual_sigma, 9) * scale
    v0 = vbar + rng.normal(0, start_sigma, 9) * scale
    return {"z": z, "vbar": vbar, "dual": dual}, v0


def n_clean(margins):
    """Leading steps whose decision is far from its threshold: the noise-rule ratio outside
    [1e-2, 1e2] and, for a compared step, an objective change above 1e-11 relative (the two
    statements' objectives differ by ~1e-15 relative)."""
    k = 0
    for m in margins:
        r = m["pred_over_noise"]
        if np.isfinite(r) and 1e-2 <= r <= 1e2:
            break
        if not (np.isfinite(r) and r < 1e-2) and abs(m["rel_change"]) < 1e-11:
            break
        k += 1
    return k


def gn_case(name, cfg, c, v0, min_clean=3):
    traj, codes, margins = R.gauss_newton(cfg, c, v0, STEPS)
    k = n_clean(margins)
    if k < min_clean:
        return None
    return {"name": name, "solver": "gn", "cfg": cfg, "z": list(c["z"]), "vbar": list(c["vbar"]),
            "dual": list(c["dual"]), "v": [list(v) for v in traj[:k + 1]], "codes": codes[:k]}


def lbfgs_case(name, cfg, c, v0, min_clean=3):
    traj, trials, margins = R.lbfgs(cfg, c, v0, STEPS)
    k = 0
    while k < len(margins) and margins[k] > 1e-11 and trials[k] != "-":
        k += 1
    if k < min_clean:
        return None
    return {"name": name, "solver": "lbfgs", "cfg": cfg, "z": list(c["z"]), "vbar": list(c["vbar"]),
            "dual": list(c["dual"]), "v": [list(v) for v in traj[:k + 1]], "trials": ",".join(trials[:k])}


def search(make, want, rng, tries=4000):
    """First draw whose case is clean and satisfies want(case)."""
    for _ in range(tries):
        case = make(rng)
        if case is not None and want(case):
            return case
    raise RuntimeError("no case found")


def main():
    scenes = {"ring8": S.scene0(), "ring64": S.scene1(n_pts=400, n_cams=16),
              "grid": S.scene2(n_pts=400, lanes=3, stations=10)}
    for sc in scenes.values():
        for y in sc.cams0[:4]:
            R.check_rotation(y)
    rng = np.random.default_rng(20260)
    cases = []
    losses = {"l2": S.LOSS_L2, "huber": S.LOSS_HUBER, "student": S.LOSS_STUDENT_T}
    for sname, sc in scenes.items():
        for lname, loss in losses.items():
            for rho_on in (False, True):
                tag = f"{sname}-{lname}-{'rho_angle' if rho_on else 'single_rho_y'}"

                def make(r, sc=sc, loss=loss, rho_on=rho_on, tag=tag):
                    cfg = base_cfg(sc, loss, rho_on)
                    c, v0 = draw(sc, cfg, r, 2.0, 0.0, 3.0, 3.0)
                    return gn_case(tag, cfg, c, v0)

                cases.append(search(make, lambda k: len(k["codes"]) >= 4, rng))

                def make_rej(r, sc=sc, loss=loss, rho_on=rho_on, tag=tag):
                    cfg = base_cfg(sc, loss, rho_on)
                    c, v0 = draw(sc, cfg, r, 2.0, 60.0, 30.0, 3.0)
                    return gn_case(tag + "-reject", cfg, c, v0)

                try:
                    cases.append(search(make_rej, lambda k: "R" in k["codes"] and "A" in k["codes"]
                                        and len(k["codes"]) >= 4, rng, 1500))
                except RuntimeError:
                    pass

                def make_lb(r, sc=sc, loss=loss, rho_on=rho_on, tag=tag):
                    cfg = base_cfg(sc, loss, rho_on)
                    c, v0 = draw(sc, cfg, r, 2.0, 30.0, 10.0, 3.0)
                    return lbfgs_case(tag + "-lbfgs", cfg, c, v0)

                cases.append(search(make_lb, lambda k: len(k["v"]) >= 5, rng))

    # a damping clamp that binds: lm_lambda_min a quarter of the first damping
    def make_clamp(r):
        sc = scenes["ring8"]
        cfg = base_cfg(sc, S.LOSS_HUBER, True)
        c, v0 = draw(sc, cfg, r, 2.0, 0.0, 3.0, 3.0)
        H0 = np.trace(np.diag(R.rho_vec(cfg))) / 9.0
        cfg["lm_lambda_min"] = 0.25 * cfg["lm_lambda0"] * H0
        return gn_case("ring8-huber-clamp", cfg, c, v0)

    cases.append(search(make_clamp, lambda k: k["codes"].count("A") >= 3, rng))

    # steps accepted by the rounding-noise rule: start at the solve's own limit
    def make_trust(r):
        sc = scenes["ring8"]
        cfg = base_cfg(sc, S.LOSS_HUBER, True)
        c, v0 = draw(sc, cfg, r, 2.0, 0.0, 3.0, 3.0)
        traj, _, _ = R.gauss_newton(dict(cfg, lm_model_tol=0.0), c, v0, 60)
        return gn_case("ring8-huber-at-minimum", cfg, c, traj[-1], min_clean=2)

    cases.append(search(make_trust, lambda k: k["codes"].startswith("TT"), rng, 200))

    # a trial behind the camera: a strong dual pushes the point backwards
    cfg = {"focal": 500.0, "cx": 320.0, "cy": 240.0, "loss": S.LOSS_L2, "loss_param": 0.0, "rho_x": 1.0,
           "rho_y": 1.0, "rho_angle": 0.0, "lm_lambda0": 1e-3, "lm_lambda_min": 1e-12, "eps_depth": 1e-6,
           "lm_model_tol": 16.0}
    c = {"z": np.array([320.0 + 5000.0, 240.0]), "vbar": np.r_[0.0, 0.0, 1.0, np.zeros(6)],
         "dual": np.array([0, 0, 50.0, 0, 0, 0, 0, 0, 0])}
    behind = gn_case("behind-camera", cfg, c, c["vbar"].copy(), min_clean=2)
    assert behind is not None and "R" in behind["codes"]
    cases.append(behind)

    with open(OUT, "w") as fh:
        json.dump({"about": "step-wise trajectories of the local solvers of Eq. (9); written by "
                            "make_local_steps.py from oracle/steps_restated.py",
                   "steps": STEPS, "cases": cases}, fh, indent=0)
    for k in cases:
        print(f"{k['name']:40s} {k.get('codes', k.get('trials'))}")


if __name__ == "__main__":
    main()
