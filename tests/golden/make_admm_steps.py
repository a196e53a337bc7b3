"""Writes tests/golden/admm_steps.json: golden iterates of the consensus ADMM iteration
(Sec. 3.1, Eqs. 9-13) over whole small scenes, per observation and with block subproblems
(Sec. 3.1.4, Eq. 14), for the tests that pin the oracle's ora_admm_iterate and
ora_block_iterate iteration by iteration.

The values come from oracle/steps_restated.py (admm_iteration, block_admm_iteration): the
restated local Gauss-Newton solve per observation or block, the consensus as the least-squares minimiser of each
point's and camera's part of the augmented Lagrangian, and the dual ascent; it shares no
code with the C oracle.  The scenes are small versions of the synthetic geometries of
paper_1708_07954_gb300.scenes with their own penalties, one of them with a point penalty
different from the camera penalty, the paper's single camera penalty (rho_angle 0), and an
unobserved point and camera appended; one case takes the L-BFGS local solve.  Every case stores the consensus after each iteration
and the copies and duals after the last.  Block cases take the oracle's block
layout (oracle.BlockLayout, pinned against brute-force grouping) and cover one-point,
one-camera and two-camera blocks.

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

import oracle as O  # noqa: E402
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


def case(name, sc, loss, loss_param, rho_x, rho_y, rho_angle, steps, iters, solver="gn"):
    cfg = {"focal": sc.focal, "cx": sc.cx, "cy": sc.cy, "loss": loss, "loss_param": loss_param,
           "rho_x": rho_x, "rho_y": rho_y, "rho_angle": rho_angle, "lm_lambda0": 1e-3,
           "lm_lambda_min": 1e-12, "eps_depth": 1e-6, "lm_model_tol": 16.0}
    cams, pts = sc.cams0.astype(float).copy(), sc.pts0.astype(float).copy()
    copies = np.concatenate([pts[sc.pt_idx], cams[sc.cam_idx]], axis=1)
    duals = np.zeros_like(copies)
    out = {"name": name, "cfg": cfg, "steps": steps, "solver": solver, "n_pts": sc.n_pts, "n_cams": sc.n_cams,
           "pt_idx": sc.pt_idx.tolist(), "cam_idx": sc.cam_idx.tolist(), "z": sc.z.tolist(),
           "cams0": cams.tolist(), "pts0": pts.tolist(), "cams": [], "pts": [], "copies": {}, "duals": {}}
    for it in range(1, iters + 1):
        copies, duals, cams, pts, codes, _ = R.admm_iteration(cfg, sc.pt_idx, sc.cam_idx, sc.z, copies, duals,
                                                              cams, pts, steps, solver)
        out["cams"].append(cams.tolist())
        out["pts"].append(pts.tolist())
        if it == iters:
            out["copies"][str(it)] = copies.tolist()
            out["duals"][str(it)] = duals.tolist()
        out.setdefault("codes", []).append("".join(codes))
    return out


def block_case(name, sc, pi, kappa, loss, loss_param, rho_x, rho_y, rho_angle, steps, iters):
    """The same with block subproblems of pi points and kappa cameras (Sec. 3.1.4, Eq. 14);
    the block layout is the oracle's (pinned against brute-force grouping)."""
    cfg = {"focal": sc.focal, "cx": sc.cx, "cy": sc.cy, "loss": loss, "loss_param": loss_param,
           "rho_x": rho_x, "rho_y": rho_y, "rho_angle": rho_angle, "lm_lambda0": 1e-3,
           "lm_lambda_min": 1e-12, "eps_depth": 1e-6, "lm_model_tol": 16.0}
    B = O.BlockLayout(sc, pi, kappa)
    layout = {k: getattr(B, k).tolist() for k in ("obs_off", "blk_obs", "obs_lp", "obs_lc", "pc_off", "pc_pt",
                                                   "cc_off", "cc_cam")}
    cams, pts = sc.cams0.astype(float).copy(), sc.pts0.astype(float).copy()
    pcopies, ccopies = pts[B.pc_pt].copy(), cams[B.cc_cam].copy()
    pduals, cduals = np.zeros_like(pcopies), np.zeros_like(ccopies)
    out = {"name": name, "cfg": cfg, "steps": steps, "pi": pi, "kappa": kappa, "n_pts": sc.n_pts,
           "n_cams": sc.n_cams, "pt_idx": sc.pt_idx.tolist(), "cam_idx": sc.cam_idx.tolist(), "z": sc.z.tolist(),
           "cams0": cams.tolist(), "pts0": pts.tolist(), "cams": [], "pts": [], "copies": {}, "duals": {}}
    shapes = sorted({(int(B.pc_off[b + 1] - B.pc_off[b]), int(B.cc_off[b + 1] - B.cc_off[b]))
                     for b in range(B.n_blocks)})
    out["block_shapes"] = [list(t) for t in shapes]
    for it in range(1, iters + 1):
        pcopies, pduals, ccopies, cduals, cams, pts, codes = R.block_admm_iteration(
            cfg, layout, sc.z, pcopies, pduals, ccopies, cduals, cams, pts, steps)
        out["cams"].append(cams.tolist())
        out["pts"].append(pts.tolist())
        if it == iters:
            out["copies"][str(it)] = {"points": pcopies.tolist(), "cameras": ccopies.tolist()}
            out["duals"][str(it)] = {"points": pduals.tolist(), "cameras": cduals.tolist()}
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
        case("ring8-huber-rho_angle-lbfgs", ring, S.LOSS_HUBER, 2.0, ring.rho_x, ring.rho_y, ring.rho_angle, 2, 4,
             solver="lbfgs"),
    ]
    block_cases = [
        block_case("ring8-4x2-huber-rho_angle", ring, 4, 2, S.LOSS_HUBER, 2.0, ring.rho_x, ring.rho_y,
                   ring.rho_angle, 5, 3),
        block_case("ring64-1x3-student-single_rho_y-rho_x_half", ring64, 1, 3, S.LOSS_STUDENT_T, 4.0,
                   0.5 * ring64.rho_x, ring64.rho_y, 0.0, 5, 3),
        block_case("grid-5x1-l2-rho_angle-unobserved", with_unobserved(grid), 5, 1, S.LOSS_L2, 0.0, grid.rho_x,
                   grid.rho_y, grid.rho_angle, 5, 3),
        block_case("grid-3x2-huber-single_rho_y", grid, 3, 2, S.LOSS_HUBER, 2.0, grid.rho_x, 2.0 * grid.rho_y,
                   0.0, 4, 3),
    ]
    with open(OUT, "w") as fh:
        json.dump({"about": "consensus ADMM iterates (Eqs. 9-13, Eq. 14 for blocks); written by "
                            "make_admm_steps.py from oracle/steps_restated.py",
                   "cases": cases, "block_cases": block_cases}, fh, separators=(",", ":"))
    for k in block_cases:
        print(f"{k['name']:40s} shapes={k['block_shapes']} codes={k['codes'][-1][:30]}")
    for k in cases:
        print(f"{k['name']:40s} obs={len(k['pt_idx']):3d} iters={len(k['cams'])} codes={k['codes'][-1][:30]}")


if __name__ == "__main__":
    main()
