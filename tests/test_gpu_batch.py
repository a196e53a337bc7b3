"""Batches of independent scenes (one concatenated problem, one tile launch per
iteration) against the oracle run scene by scene; per-scene metrics; the
tile-size autotuner."""
import numpy as np
import pytest
from parity import colerr

import oracle as O
from paper_1708_07954_gb300 import build, dba
from paper_1708_07954_gb300 import scenes as S

pytestmark = pytest.mark.gpu

TOL64 = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dba.load()


def part(batch, k):
    """Scene k of a concatenated batch, re-indexed from zero."""
    o0, o1 = batch.scene_off[k], batch.scene_off[k + 1]
    c0, c1 = batch.cam_off[k], batch.cam_off[k + 1]
    p0, p1 = batch.pt_off[k], batch.pt_off[k + 1]
    return S.Scene(n_cams=int(c1 - c0), n_pts=int(p1 - p0), pt_idx=(batch.pt_idx[o0:o1] - p0).astype(np.int32),
                   cam_idx=(batch.cam_idx[o0:o1] - c0).astype(np.int32), z=batch.z[o0:o1],
                   z_true=batch.z_true[o0:o1], outlier=batch.outlier[o0:o1], cams_gt=batch.cams_gt[c0:c1],
                   pts_gt=batch.pts_gt[p0:p1], cams0=batch.cams0[c0:c1], pts0=batch.pts0[p0:p1],
                   focal=batch.focal, cx=batch.cx, cy=batch.cy, loss=batch.loss, loss_param=batch.loss_param,
                   rho_x=batch.rho_x, rho_y=batch.rho_y, rho_angle=batch.rho_angle)


def oracle_cfg(solver):
    c = solver.cfg
    return O.config(focal=c.focal, cx=c.cx, cy=c.cy, loss=c.loss, loss_param=c.loss_param, rho_x=c.rho_x,
                    rho_y=c.rho_y, rho_angle=c.rho_angle, inner_steps=c.inner_steps, lm_lambda0=c.lm_lambda0,
                    lm_lambda_min=c.lm_lambda_min, eps_depth=c.eps_depth, lm_model_tol=c.lm_model_tol,
                    local_solver=c.local_solver)


def relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_batch_fp64_matches_oracle_scene_by_scene():
    batch = S.scene3(n_scenes=9, max_pts=400)
    n = len(batch.scene_off) - 1
    with dba.Solver(batch, precision=dba.DBA_PREC_F64, tile_obs=64) as s:
        cfg = oracle_cfg(s)
        s.iterate(4, stats=False)
        cams, pts = s.params()
        stats = s.scene_stats()
    for k in range(n):
        sc = part(batch, k)
        st = O.State(sc)
        m = st.iterate(cfg, 4)
        c0, c1 = batch.cam_off[k], batch.cam_off[k + 1]
        p0, p1 = batch.pt_off[k], batch.pt_off[k + 1]
        assert colerr(cams[c0:c1], st.cams) <= TOL64 and colerr(pts[p0:p1], st.pts) <= TOL64, k
        assert abs(stats["rmse_obs"][k] - m["rmse_obs"]) <= 1e-8 * m["rmse_obs"]
        assert abs(stats["objective"][k] - m["objective"]) <= 1e-8 * m["objective"]
        assert abs(stats["rmse_gt"][k] - m["rmse_gt"]) <= 1e-8 * max(m["rmse_gt"], 1e-12)


def test_batch_fp32_tracks_fp64():
    batch = S.scene3(n_scenes=16, max_pts=2000)
    with dba.Solver(batch, precision=dba.DBA_PREC_F64) as a, dba.Solver(batch, precision=dba.DBA_PREC_F32_LOCAL) as b:
        a.iterate(20, stats=False)
        b.iterate(20, stats=False)
        ga, gb = a.scene_stats()["rmse_gt"], b.scene_stats()["rmse_gt"]
    assert np.all(np.abs(ga - gb) <= 1e-3)


def test_autotuned_tile_matches_fixed_tile():
    sc = S.scene1(n_pts=3000, n_cams=24, seed=91)
    with dba.Solver(sc, precision=dba.DBA_PREC_F64, tile_obs=-1) as a, \
            dba.Solver(sc, precision=dba.DBA_PREC_F64, tile_obs=128) as b:
        assert a.layout()["tile_obs"] in (64, 128, 256)
        assert a.layout()["finalize_threads"] in (32, 64, 128, 256)
        assert b.layout()["finalize_threads"] == 128
        a.iterate(5, stats=False)
        b.iterate(5, stats=False)
        assert colerr(a.params()[0], b.params()[0]) <= TOL64
        assert colerr(a.params()[1], b.params()[1]) <= TOL64


def test_set_scenes_rejects_an_observation_leaving_its_scene():
    batch = S.scene3(n_scenes=3, max_pts=200)
    with dba.Solver(batch, precision=dba.DBA_PREC_F32_LOCAL) as s:
        bad = batch.cam_off.copy()
        bad[1] -= 1  # the last camera of scene 0 now belongs to scene 1
        with pytest.raises(dba.DbaError) as e:
            dba.dba_set_scenes(s.ctx, batch.scene_off, bad, batch.pt_off)
        assert e.value.status == dba.DBA_EINVAL and "leaves its scene" in str(e.value)
