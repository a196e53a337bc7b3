"""Writes tests/golden/admm_steps.json: golden iterates of the consensus ADMM iteration
(Sec. 3.1, Eqs. 9-13) over whole small scenes, for the tests that pin the oracle's
ora_admm_iterate iteration by iteration.

The values come from oracle/steps_restated.py (admm_iteration): the restated local
Gauss-Newton solve per observation, the consensus as the least-squares minimiser of each
point's and camera's part of the augmented Lagrangian, and the dual ascent; it shares no
code with the C oracle.  The scenes are small versions of the synthetic geometries of
paper_1708_07954_gb300.scenes with their own penalties, one of them with a point penalty
different from the camera penalty, the paper's single camera penalty (rho_angle 0), and an
unobserved point and camera appended.  Every case stores the consensus after each iteration
and the copies and duals after the first and the last.

    python tests/golden/make_admm_steps.py      # rewrites admm_steps.json
"""
from __future__ import annotations

import dataclasses
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import steps_restated as R  # noqa: E402
from paper_1708_07954_gb300 import scenes as S  # noqa: E402

OUT = os.path.join(HERE, "admm_steps.json")


def with_unobserved(sc):
    """The scene with one more point and one more camera that no observation sees."""
    return dataclasses.replace(sc, n_pts=sc.n_pts + 1, n_cams=sc.n_cams + 1,
                               pts0=np.vstack([sc.pts0, sc.pts0[:1] + 1.0]),
                               cams0=np.vstack([sc.cams0, sc.cams0[:1] + 0.1]),
                               pts_gt=np.vstack([sc.pts_gt, sc.pts_gt[:1]]),
                               cams_gt=np.vstack([sc.cams_gt, sc.cams_gt[:1]]))


def case(name, sc, loss, loss_param, rho_x, rho_y, rho_angle, steps, iters):
    cfg = {"focal": sc.focal, "cx": sc.cx, "cy": sc.cy, "loss": loss, "loss_param": loss_param,
           "rho_x": rho_x, "rho_y": rho_y, "rho_angle": rho_angle, "lm_lambda0": 1e-3,
           "lm_lambda_min": 1e-12, "eps_depth": 1e-6, "lm_model_tol": 16.0}
    cams, pts = sc.cams0.astype(float).copy(), sc.pts0.astype(float).copy()
    copies = np.concatenate([pts[sc.pt_idx], cams[sc.cam_idx]], axis=1)
    duals = np.zeros_like(copies)
    out = {"name": name, "cfg": cfg, "steps": steps, "n_pts": sc.n_pts, "n_cams": sc.n_cams,
           "pt_idx": sc.pt_idx.tolist(), "cam_idx": sc.cam_idx.tolist(), "z": sc.z.tolist(),
           "cams0": cams.tolist(), "pts0": pts.tolist(), "cams": [], "pts": [], "copies": {}, "duals": {}}
    for it in range(1, iters + 1):
        copies, duals, cams, pts, codes, _ = R.admm_iteration(cfg, sc.pt_idx, sc.cam_idx, sc.z, copies, duals,
                                                              cams, pts, steps)
        out["cams"].append(cams.tolist())
        out["pts"].append(pts.tolist())
        if it in (1, iters):
            out["copies"][str(it)] = copies.tolist()
            out["duals"][str(it)] = duals.tolist()
        out.setdefault("codes", []).append("".join(codes))
    return out


def main():
    ring = S.scene0(n_pts=8, n_cams=4, seed=7)
    ring64 = S.scene1(n_pts=12, n_cams=8, seed=8)
    grid = S.scene2(n_pts=12, lanes=2, stations=4, seed=9)
    for sc in (ring, ring64, grid):
        for y in sc.cams0[:4]:
            R.check_rotation(y)
    cases = [
        case("ring8-huber-rho_angle", ring, S.LOSS_HUBER, 2.0, ring.rho_x, ring.rho_y, ring.rho_angle, 5, 4),
        case("ring8-l2-single_rho_y-rho_x_half", ring, S.LOSS_L2, 0.0, 0.5 * ring.rho_x, ring.rho_y, 0.0, 5, 4),
        case("ring64-student-rho_angle-unobserved", with_unobserved(ring64), S.LOSS_STUDENT_T, 4.0,
             ring64.rho_x, 2.0 * ring64.rho_y, ring64.rho_angle, 5, 3),
        case("grid-huber-single_rho_y", grid, S.LOSS_HUBER, 2.0, grid.rho_x, grid.rho_y, 0.0, 3, 3),
    ]
    with open(OUT, "w") as fh:
        json.dump({"about": "consensus ADMM iterates (Eqs. 9-13); written by make_admm_steps.py from "
                            "oracle/steps_restated.py", "cases": cases}, fh, indent=0)
    for k in cases:
        print(f"{k['name']:40s} obs={len(k['pt_idx']):3d} iters={len(k['cams'])} codes={k['codes'][-1][:30]}")


if __name__ == "__main__":
    main()
