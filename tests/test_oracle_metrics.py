"""Closed-form pins of the oracle's metrics (ora_eval): the mean re-projection error of
Sec. 4 over observations in front of their cameras, its counterpart against noise-free
projections, the objective of Eq. (2) with the misfit of Sec. 2.2, and the primal and dual
residuals of the consensus iteration (Eqs. 10-13).

The scene is built by hand so that every expected value is arithmetic: two cameras with no
rotation look along +z at a 3 x 3 grid of points at depth 4, and every point is seen by both
cameras.  Moving a camera by delta along x moves each of its pixels by exactly f delta / 4
along u (along y: along v), so the errors, the objective under each misfit and the residuals
have closed forms.
"""
import numpy as np
import pytest

import oracle as O
from paper_1708_07954_gb300 import scenes as S

F, CX, CY, DEPTH = 500.0, 320.0, 240.0, 4.0


def _grid_scene():
    pts = np.array([[i, j, DEPTH] for i in (-1.0, 0.0, 1.0) for j in (-1.0, 0.0, 1.0)])
    cams = np.array([[0.0, 0.0, 0.0, 0.0, 0.0, 0.0], [0.0, 0.0, 0.0, -0.5, 0.0, 0.0]])
    pt_idx = np.repeat(np.arange(9, dtype=np.int32), 2)
    cam_idx = np.tile(np.arange(2, dtype=np.int32), 9)
    # no rotation: the pixel of x seen from a camera at translation t is f (x + t)_{1,2} / (x + t)_3 + c
    q = pts[pt_idx] + cams[cam_idx, 3:]
    z = np.stack([F * q[:, 0] / q[:, 2] + CX, F * q[:, 1] / q[:, 2] + CY], axis=1)
    return S.Scene(n_cams=2, n_pts=9, pt_idx=pt_idx, cam_idx=cam_idx, z=z, z_true=z.copy(),
                   outlier=np.zeros(18, dtype=bool), cams_gt=cams.copy(), pts_gt=pts.copy(),
                   cams0=cams.copy(), pts0=pts.copy(), focal=F, cx=CX, cy=CY, depth=DEPTH)


def _cfg(loss=O.LOSS_L2, p=0.0, rho_x=2.0, rho_y=3.0, rho_angle=5.0):
    return O.config(focal=F, cx=CX, cy=CY, loss=loss, loss_param=p, rho_x=rho_x, rho_y=rho_y,
                    rho_angle=rho_angle)


def test_metrics_vanish_at_the_observed_geometry():
    sc = _grid_scene()
    m = O.State(sc).metrics(_cfg())
    assert m["rmse_obs"] <= 1e-12 and m["rmse_gt"] <= 1e-12 and m["objective"] <= 1e-20
    assert m["primal_res"] == 0.0 and m["n_invalid"] == 0


S2 = 1.25 ** 2 + 1.0 ** 2  # squared pixel error of camera 0 moved by (0.01, 0.008): (1.25, 1.0) px


@pytest.mark.parametrize("loss,p,per_obs", [
    (O.LOSS_L2, 0.0, S2),                                       # s = 2.5625
    (O.LOSS_HUBER, 2.0, S2),                                    # quadratic branch: s <= p^2
    (O.LOSS_HUBER, 1.0, 2 * 1.0 * np.sqrt(S2) - 1.0),           # linear branch: 2 p sqrt(s) - p^2
    (O.LOSS_STUDENT_T, 4.0, 4.0 * np.log(1 + S2 / 4.0)),        # p log(1 + s / p)
])
def test_reprojection_error_and_objective_of_a_shifted_camera(loss, p, per_obs):
    """Camera 0 moved by (0.01, 0.008) along (x, y): its 9 pixels move by 500 * (0.01, 0.008) / 4
    = (1.25, 1.0) px, the 9 pixels of camera 1 stay; mean squared error 9 * 2.5625 / 18."""
    sc = _grid_scene()
    st = O.State(sc)
    st.cams[0, 3:5] += (0.01, 0.008)
    m = st.metrics(_cfg(loss, p))
    assert m["rmse_obs"] == pytest.approx(np.sqrt(S2 / 2.0), rel=1e-12)
    assert m["rmse_gt"] == pytest.approx(np.sqrt(S2 / 2.0), rel=1e-12)
    assert m["objective"] == pytest.approx(9 * per_obs, rel=1e-12)
    assert m["n_invalid"] == 0


def test_ground_truth_error_is_measured_against_the_noise_free_pixels():
    """Noise-free pixels offset by (0.3, 0.4): camera 1's pixels are 0.5 px from them, camera
    0's (moved (1.25, 1.0) px) sqrt(0.95^2 + 0.6^2); the observed pixels are unchanged."""
    sc = _grid_scene()
    sc.z_true = sc.z + np.array([0.3, 0.4])
    st = O.State(sc)
    st.cams[0, 3:5] += (0.01, 0.008)
    m = st.metrics(_cfg())
    assert m["rmse_obs"] == pytest.approx(np.sqrt(S2 / 2.0), rel=1e-12)
    assert m["rmse_gt"] == pytest.approx(np.sqrt((9 * 0.25 + 9 * (0.95 ** 2 + 0.6 ** 2)) / 18), rel=1e-12)
    assert O.State(sc).metrics(_cfg(), with_gt=False)["rmse_gt"] == 0.0


def test_primal_residual_is_the_distance_of_all_copies_from_the_consensus():
    sc = _grid_scene()
    st = O.State(sc)
    off = np.arange(1.0, 10.0) * 1e-3
    st.copies += off
    assert st.metrics(_cfg())["primal_res"] == pytest.approx(np.sqrt(18 * (off @ off)), rel=1e-12)
    st.copies[5] += 0.2  # one copy further off
    want = np.sqrt(17 * (off @ off) + ((off + 0.2) @ (off + 0.2)))
    assert st.metrics(_cfg())["primal_res"] == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("rho_angle", [5.0, 0.5, 0.0])
def test_dual_residual_weights_each_change_by_its_penalty_once_per_observation(rho_angle):
    """Every point moved by delta since the previous consensus and camera 1 by (eta_angles,
    eta_t): each of the 18 observations adds rho_x^2 |delta|^2, and each of camera 1's 9 adds
    rho_a^2 |eta_angles|^2 + rho_y^2 |eta_t|^2, with rho_a = rho_angle when it is positive
    (also below 1) and rho_a = rho_y under the paper's single camera penalty (rho_angle 0)."""
    sc = _grid_scene()
    st = O.State(sc)
    delta = np.array([0.1, 0.2, 0.2])
    eta_a, eta_t = np.array([0.01, 0.0, -0.02]), np.array([0.0, 0.02, 0.0])
    pts_prev = st.pts - delta
    cams_prev = st.cams.copy()
    cams_prev[1] -= np.r_[eta_a, eta_t]
    cfg = _cfg(rho_angle=rho_angle)
    rho_a = rho_angle if rho_angle > 0 else 3.0
    want = np.sqrt(18 * 2.0 ** 2 * (delta @ delta) + 9 * (rho_a ** 2 * (eta_a @ eta_a) + 3.0 ** 2 * (eta_t @ eta_t)))
    m = st.metrics(cfg, cams_prev=np.ascontiguousarray(cams_prev), pts_prev=np.ascontiguousarray(pts_prev))
    assert m["dual_res"] == pytest.approx(want, rel=1e-12)
    assert st.metrics(cfg)["dual_res"] == 0.0


def test_points_behind_the_cameras_are_counted_and_left_out_of_the_means():
    """A point moved to depth -1 is behind both cameras: 2 observations invalid, the error
    mean over the other 16 (camera 0 moved (1.25, 1.0) px as above: 8 of them)."""
    sc = _grid_scene()
    st = O.State(sc)
    st.cams[0, 3:5] += (0.01, 0.008)
    st.pts[4, 2] = -1.0
    m = st.metrics(_cfg())
    assert m["n_invalid"] == 2
    assert m["rmse_obs"] == pytest.approx(np.sqrt(8 * S2 / 16), rel=1e-12)
    assert m["objective"] == pytest.approx(8 * S2, rel=1e-12)


def test_iteration_reports_the_metrics_of_its_new_consensus():
    """The metrics ora_admm_iterate returns are ora_eval's at the consensus it ends with, the
    dual residual measured from the consensus it started from."""
    sc = S.scene0(n_pts=60, n_cams=6, seed=3)
    cfg = O.config_for(sc)
    st = O.State(sc)
    st.iterate(cfg, 2)
    before = st.clone()
    m = st.iterate(cfg, 1)
    want = st.metrics(cfg, cams_prev=before.cams, pts_prev=before.pts)
    for k in ("rmse_obs", "rmse_gt", "objective", "primal_res", "dual_res"):
        assert m[k] == pytest.approx(want[k], rel=1e-12), k
    assert m["n_invalid"] == want["n_invalid"]


@pytest.mark.parametrize("blocks", [None, (4, 2)])
def test_zero_iterations_report_the_metrics_of_the_start(blocks):
    """Asked for no iteration, both iterations leave the state alone and report its metrics:
    no dual residual (there is no previous consensus) and no primal residual (every copy
    starts at its consensus)."""
    sc = S.scene0(n_pts=40, n_cams=6, seed=4)
    cfg = O.config_for(sc)
    st = O.State(sc) if blocks is None else O.BlockState(sc, *blocks)
    cams, pts = st.cams.copy(), st.pts.copy()
    m = st.iterate(cfg, 0)
    want = O.State(sc).metrics(cfg)
    assert m["dual_res"] == 0.0 and m["primal_res"] == 0.0
    for k in ("rmse_obs", "rmse_gt", "objective", "n_invalid"):
        assert m[k] == want[k], k
    assert np.array_equal(st.cams, cams) and np.array_equal(st.pts, pts)


def test_no_observation_in_front_of_a_camera_gives_zero_means():
    """Every point moved behind both cameras: every observation is counted invalid, and the
    means over an empty set are reported as 0 (not 0/0)."""
    sc = _grid_scene()
    st = O.State(sc)
    st.pts[:, 2] = -1.0
    m = st.metrics(_cfg())
    assert m["n_invalid"] == 18
    assert m["rmse_obs"] == 0.0 and m["rmse_gt"] == 0.0 and m["objective"] == 0.0
