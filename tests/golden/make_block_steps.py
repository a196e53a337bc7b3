"""Writes tests/golden/block_steps.json: step-wise golden trajectories of the block solve
of Eq. (14) (Sec. 3.1.4), for the tests that pin the oracle's ora_block_solve over a fixed
number of damped Gauss-Newton steps.

The values come from oracle/steps_restated.py (block_gauss_newton), a second statement of
the block solve that shares no code with the C oracle: the stacked Jacobian of all the
block's pixels by complex steps of the whole block vector, dense products with the IRLS
weights and a numpy LU solve.  Inputs are blocks cut from the synthetic scenes of
paper_1708_07954_gb300.scenes by the oracle's own block layout (points grouped by first
camera, cameras in runs of kappa): the block's observations with perturbed pixels, the
scene's initial estimates as consensus, duals rho (copy - consensus) for copy offsets of a
plausible size, and a start displaced from the consensus.  As in make_local_steps.py each
case keeps the leading steps whose every decision is far from its threshold.  The case set
covers one-point, one-camera and wider blocks, all three misfits, both camera-penalty
readings, rejected steps, steps accepted by the rounding-noise rule, a binding damping
clamp, a trial behind a camera, a start with an observation behind its camera, and rejected
steps with a small predicted decrease (below 0.5 px^2, far above the rounding noise).

    python tests/golden/make_block_steps.py      # rewrites block_steps.json
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

import oracle as O  # noqa: E402
from oracle import steps_restated as R  # noqa: E402
from paper_1708_07954_gb300 import scenes as S  # noqa: E402
from make_local_steps import base_cfg, n_clean  # noqa: E402

OUT = os.path.join(HERE, "block_steps.json")
STEPS = 6


def blocks_of(scene, pi, kappa, shape):
    """The blocks of the layout (pi, kappa) of the scene with (points, cameras) = shape."""
    B = O.BlockLayout(scene, pi, kappa)
    npc, ncc = np.diff(B.pc_off), np.diff(B.cc_off)
    return B, np.flatnonzero((npc == shape[0]) & (ncc == shape[1]))


def draw(scene, cfg, rng, B, b, pix_sigma, outlier_px, start_sigma, dual_sigma):
    o = B.blk_obs[B.obs_off[b]:B.obs_off[b + 1]]
    xbar = scene.pts0[B.pc_pt[B.pc_off[b]:B.pc_off[b + 1]]].ravel()
    ybar = scene.cams0[B.cc_cam[B.cc_off[b]:B.cc_off[b + 1]]].ravel()
    z = scene.z[o] + rng.normal(0, pix_sigma, (len(o), 2))
    if outlier_px:
        z[0] += rng.choice([-1, 1], 2) * outlier_px
    np_, nc = len(xbar) // 3, len(ybar) // 6
    r = R.rho_vec(cfg)
    sx = np.full(3 * np_, scene.depth * 1e-3)
    sy = np.tile(np.r_[np.full(3, 1e-3), np.full(3, scene.depth * 1e-3)], nc)
    blk = {"opl": B.obs_lp[B.obs_off[b]:B.obs_off[b + 1]].tolist(),
           "ocl": B.obs_lc[B.obs_off[b]:B.obs_off[b + 1]].tolist(),
           "z": z.ravel(), "xbar": xbar, "ybar": ybar,
           "rx": r[0] * rng.normal(0, dual_sigma, 3 * np_) * sx,
           "sy": np.tile(r[3:], nc) * rng.normal(0, dual_sigma, 6 * nc) * sy}
    v0 = np.concatenate([xbar, ybar]) + rng.normal(0, start_sigma, 3 * np_ + 6 * nc) * np.r_[sx, sy]
    return blk, v0


def case_of(name, cfg, blk, v0, min_clean=3, steps=STEPS):
    traj, codes, margins = R.block_gauss_newton(cfg, blk, v0, steps)
    k = n_clean(margins)
    if k < min_clean:
        return None
    out = {"name": name, "cfg": cfg, "codes": codes[:k], "v": [list(v) for v in traj[:k + 1]]}
    for key in ("opl", "ocl"):
        out[key] = [int(i) for i in blk[key]]
    for key in ("z", "xbar", "ybar", "rx", "sy"):
        out[key] = [float(x) for x in blk[key]]
    return out


def first_damping(cfg, blk, v):
    """lm_lambda0 * mean diag H at the start, H the Gauss-Newton matrix of Eq. (14)."""
    zp, _ = R.block_pixels(cfg, blk, v)
    e = np.asarray(blk["z"]).reshape(-1, 2) - zp
    w = np.repeat([R.weight(cfg, ek @ ek) for ek in e], 2)
    J = R.block_jacobian_cs(cfg, blk, v)
    diag = 2 * (w[:, None] * J * J).sum(axis=0) + R.block_rho(cfg, blk)
    return cfg["lm_lambda0"] * diag.mean()


def search(make, want, rng, tries=400):
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
    rng = np.random.default_rng(20261)
    losses = {"l2": S.LOSS_L2, "huber": S.LOSS_HUBER, "student": S.LOSS_STUDENT_T}
    # (scene, layout, block shape): one-point blocks of 3 cameras, one-camera blocks of 5 points,
    # 4 x 2, 8 x 2 and 4 x 4 blocks, and a single-observation block.
    shapes = [("ring64", (1, 3), (1, 3)), ("grid", (5, 1), (5, 1)), ("ring8", (4, 2), (4, 2)),
              ("ring64", (8, 2), (8, 2)), ("grid", (4, 4), (4, 4)), ("ring64", (1, 1), (1, 1))]
    cases = []
    for si, (sname, layout, shape) in enumerate(shapes):
        sc = scenes[sname]
        B, cand = blocks_of(sc, *layout, shape)
        for lname, loss in losses.items():
            rho_on = (si + len(lname)) % 2 == 0
            tag = f"{sname}-{shape[0]}x{shape[1]}-{lname}-{'rho_angle' if rho_on else 'single_rho_y'}"

            def make(r, sc=sc, loss=loss, rho_on=rho_on, tag=tag, B=B, cand=cand):
                cfg = base_cfg(sc, loss, rho_on)
                blk, v0 = draw(sc, cfg, r, B, int(r.choice(cand)), 2.0, 0.0, 3.0, 3.0)
                return case_of(tag, cfg, blk, v0)

            cases.append(search(make, lambda k: len(k["codes"]) >= 4, rng))

            def make_rej(r, sc=sc, loss=loss, rho_on=rho_on, tag=tag, B=B, cand=cand):
                cfg = base_cfg(sc, loss, rho_on)
                blk, v0 = draw(sc, cfg, r, B, int(r.choice(cand)), 2.0, 60.0, 30.0, 3.0)
                return case_of(tag + "-reject", cfg, blk, v0)

            try:
                cases.append(search(make_rej, lambda k: "R" in k["codes"] and "A" in k["codes"]
                                    and len(k["codes"]) >= 4, rng, 150))
            except RuntimeError:
                pass

    # a damping clamp that binds: lm_lambda_min a quarter of the first damping's scale
    sc = scenes["ring8"]
    B, cand = blocks_of(sc, 4, 2, (4, 2))

    def make_clamp(r):
        cfg = base_cfg(sc, S.LOSS_HUBER, True)
        blk, v0 = draw(sc, cfg, r, B, int(r.choice(cand)), 2.0, 0.0, 3.0, 3.0)
        cfg["lm_lambda_min"] = 0.025 * first_damping(cfg, blk, v0)  # binds from the third step on
        return case_of("ring8-4x2-huber-clamp", cfg, blk, v0)

    cases.append(search(make_clamp, lambda k: k["codes"].count("A") >= 3, rng))

    # steps accepted by the rounding-noise rule: start at the solve's own limit
    def make_trust(r):
        cfg = base_cfg(sc, S.LOSS_HUBER, True)
        blk, v0 = draw(sc, cfg, r, B, int(r.choice(cand)), 2.0, 0.0, 3.0, 3.0)
        traj, _, _ = R.block_gauss_newton(dict(cfg, lm_model_tol=0.0), blk, v0, 40)
        return case_of("ring8-4x2-huber-at-minimum", cfg, blk, traj[-1], min_clean=2)

    cases.append(search(make_trust, lambda k: k["codes"].startswith("TT"), rng, 40))

    # a trial behind a camera: a strong dual pushes the second point of a two-point block
    # backwards, and the start of another block has its first point behind the camera
    # (Eq. (14) is +inf there, so any finite trial is a decrease)
    cfg = {"focal": 500.0, "cx": 320.0, "cy": 240.0, "loss": S.LOSS_L2, "loss_param": 0.0, "rho_x": 1.0,
           "rho_y": 1.0, "rho_angle": 0.0, "lm_lambda0": 1e-3, "lm_lambda_min": 1e-12, "eps_depth": 1e-6,
           "lm_model_tol": 16.0}
    blk = {"opl": [0, 1], "ocl": [0, 0], "z": [320.0 + 40.0, 240.0, 320.0 + 5000.0, 240.0],
           "xbar": [0.0, 0.0, 1.0, 0.05, 0.0, 1.0], "ybar": [0.0] * 6,
           "rx": [0.0, 0.0, 0.0, 0.0, 0.0, 50.0], "sy": [0.0] * 6}
    v0 = np.concatenate([blk["xbar"], blk["ybar"]])
    behind = case_of("behind-camera-trial", cfg, blk, v0, min_clean=2)
    assert behind is not None and "R" in behind["codes"]
    cases.append(behind)
    blk = {"opl": [0, 1], "ocl": [0, 0], "z": [330.0, 240.0, 300.0, 250.0],
           "xbar": [0.02, 0.0, 1.0, -0.04, 0.02, 1.0], "ybar": [0.0] * 6,
           "rx": [0.0] * 6, "sy": [0.0] * 6}
    v0 = np.concatenate([[0.02, 0.0, -0.01], blk["xbar"][3:], blk["ybar"]])
    # a small damping start, so that the first step can carry the point to the front
    start = case_of("behind-camera-start", dict(cfg, lm_lambda0=1e-5), blk, v0, min_clean=2)
    assert start is not None and not np.isfinite(R.block_objective(cfg, blk, v0))
    cases.append(start)

    # a rejected step whose predicted decrease is small (below 0.5 px^2) but far above the
    # rounding noise: plain comparison must reject it, the noise rule must not trust it
    rng2 = np.random.default_rng(20262)
    sc = scenes["grid"]
    for layout, shape, loss, lname in (((1, 3), (1, 2), S.LOSS_STUDENT_T, "student"),
                                       ((5, 1), (2, 1), S.LOSS_HUBER, "huber")):
        B, cand = blocks_of(sc, *layout, shape)

        def make_small(r, B=B, cand=cand, loss=loss, lname=lname, shape=shape):
            cfg = base_cfg(sc, loss, False)
            blk, v0 = draw(sc, cfg, r, B, int(r.choice(cand)), 2.0, float(r.choice([0.0, 10.0, 60.0])),
                           float(r.choice([3.0, 10.0, 30.0])), 3.0)
            traj, codes, margins = R.block_gauss_newton(cfg, blk, v0, STEPS)
            k = n_clean(margins)
            if not any(c == "R" and m["pred"] < 0.5 for c, m in zip(codes[:k], margins[:k])):
                return None
            return case_of(f"grid-{shape[0]}x{shape[1]}-{lname}-single_rho_y-small-prediction-reject", cfg, blk, v0)

        cases.append(search(make_small, lambda k: True, rng2, 2000))

    with open(OUT, "w") as fh:
        json.dump({"about": "step-wise trajectories of the block solve of Eq. (14); written by "
                            "make_block_steps.py from oracle/steps_restated.py",
                   "steps": STEPS, "cases": cases}, fh, indent=0)
    for k in cases:
        print(f"{k['name']:44s} n={len(k['v'][0]):3d} {k['codes']}")


if __name__ == "__main__":
    main()
