"""The paper's convergence findings, re-run on a reduced scene on the GPU and checked
iteration for iteration against the FP64 CPU oracle.

Scene: workload-2 geometry reduced to 60 cameras on the flight grid (5 lanes x 12
stations) and 4,000 ground points (~32k observations), sigma 0.5 px, 5 % outliers
unless stated.  Target: rmse_gt <= 0.5 px, the RMS distance of the consensus
projections from the noise-free projections over observations of outlier-free tracks.
Each case runs the GPU's FP64 path until the target (dba_iterate_until) and the oracle
one iteration at a time with the same metric, and asks for the same iteration count.

- Sec. 4.1: with gross outliers the Huber misfit reaches the target while the squared
  misfit does not (the robust loss is what lets the consensus converge).
- Sec. 4 (the penalty): within the stable range a smaller rho factor reaches the target
  in fewer iterations on these scenes (the paper reports the opposite direction on its
  real data; DESIGN records both).
- Sec. 3.1.4 / Sec. 4 (Eq. 14): more points and cameras per update step need fewer
  iterations.
"""
import dataclasses

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
from paper_1708_07954_gb300 import build, dba
from paper_1708_07954_gb300 import scenes as S

pytestmark = pytest.mark.gpu

TARGET = 0.5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dba.load()


def _scene(outliers=0.05, loss=S.LOSS_HUBER):
    sc = S.scene2(n_pts=4000, lanes=5, stations=12, outlier_frac=outliers)
    return dataclasses.replace(sc, loss=loss)


def _rmse_clean(sc, cams, pts, mask):
    R = Rotation.from_euler("xyz", cams[:, :3]).as_matrix()
    i, j = sc.pt_idx[mask], sc.cam_idx[mask]
    p = np.einsum("nab,nb->na", R[j], pts[i]) + cams[j, 3:]
    zp = sc.focal * p[:, :2] / p[:, 2:3] + np.array([sc.cx, sc.cy])
    return float(np.sqrt(((zp - sc.z_true[mask]) ** 2).sum(1).mean()))


def _oracle_iters(sc, cfg, max_iters, block=None):
    st = O.State(sc) if block is None else O.BlockState(sc, *block)
    mask = sc.clean_mask()
    r = None
    for k in range(1, max_iters + 1):
        st.iterate(cfg, 1, with_gt=False)
        r = _rmse_clean(sc, st.cams, st.pts, mask)
        if r <= TARGET:
            return k, r
    return None, r


def _gpu_iters(sc, max_iters, block=None, **kw):
    if block is None:
        with dba.Solver(sc, precision=dba.DBA_PREC_F64, **kw) as s:
            m = s.iterate_until(max_iters, TARGET)
            c = s.cfg
    else:
        with dba.BlockSolver(sc, *block, precision=dba.DBA_PREC_F64, **kw) as s:
            m = s.iterate_until(max_iters, TARGET)
            c = s.cfg
    cfg = O.config(focal=c.focal, cx=c.cx, cy=c.cy, loss=c.loss, loss_param=c.loss_param, rho_x=c.rho_x,
                   rho_y=c.rho_y, rho_angle=c.rho_angle, inner_steps=c.inner_steps, lm_lambda0=c.lm_lambda0,
                   lm_lambda_min=c.lm_lambda_min, eps_depth=c.eps_depth, lm_model_tol=c.lm_model_tol)
    return (m["iters_done"] if m["rmse_gt"] <= TARGET else None), m["rmse_gt"], cfg


def test_huber_reaches_the_target_with_outliers_where_l2_does_not():
    """Sec. 4.1: squared vs Huber misfit with 5 % gross outliers."""
    hub = _scene(loss=S.LOSS_HUBER)
    k_h, r_h, cfg_h = _gpu_iters(hub, 160)
    assert k_h is not None and k_h < 160
    assert _oracle_iters(hub, cfg_h, 160)[0] == k_h
    l2 = _scene(loss=S.LOSS_L2)
    k_2, r_2, cfg_2 = _gpu_iters(l2, 160)
    assert k_2 is None and r_2 > 10 * TARGET
    # the squared misfit does not converge here, and its divergent run amplifies rounding
    # differences, so only the outcome is compared with the oracle, not the final value
    k_o, r_o = _oracle_iters(l2, cfg_2, 160)
    assert k_o is None and r_o > 10 * TARGET


def test_iterations_to_target_grow_with_the_penalty():
    """Sec. 4 (rho): factors 0.5, 1, 2 of each block's data curvature, outlier-free scene."""
    sc = _scene(outliers=0.0)
    counts = []
    for f in (0.5, 1.0, 2.0):
        rx, ry, ra = S.default_rho(sc, f)
        k, _, cfg = _gpu_iters(sc, 300, rho_x=rx, rho_y=ry, rho_angle=ra)
        assert k is not None
        assert _oracle_iters(sc, cfg, 300)[0] == k
        counts.append(k)
    assert counts[0] < counts[1] < counts[2], counts


def test_larger_blocks_need_fewer_iterations():
    """Sec. 3.1.4, Eq. (14): 1x1 (the per-observation method), 8 points x 1 camera and
    32 points x 2 cameras per update step."""
    sc = _scene()
    counts = []
    for blk in ((1, 1), (8, 1), (32, 2)):
        k, _, cfg = _gpu_iters(sc, 160, block=blk)
        assert k is not None
        assert _oracle_iters(sc, cfg, 160, block=blk)[0] == k
        counts.append(k)
    assert counts[0] > counts[1] > counts[2], counts
