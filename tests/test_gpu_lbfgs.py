"""The L-BFGS local solver (Sec. 3.1) on the GPU against the oracle's L-BFGS."""
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


def oracle_cfg(solver):
    c = solver.cfg
    return O.config(focal=c.focal, cx=c.cx, cy=c.cy, loss=c.loss, loss_param=c.loss_param, rho_x=c.rho_x,
                    rho_y=c.rho_y, rho_angle=c.rho_angle, inner_steps=c.inner_steps, lm_lambda0=c.lm_lambda0,
                    lm_lambda_min=c.lm_lambda_min, eps_depth=c.eps_depth, lm_model_tol=c.lm_model_tol,
                    local_solver=c.local_solver)


def relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("tile", [64, 256])
@pytest.mark.parametrize("loss", [S.LOSS_HUBER, S.LOSS_L2, S.LOSS_STUDENT_T])
def test_fp64_lbfgs_matches_oracle_per_iteration(tile, loss):
    sc = S.scene1(n_pts=600, n_cams=16, seed=41)
    sc.loss, sc.loss_param = loss, {S.LOSS_HUBER: 2.0, S.LOSS_L2: 0.0, S.LOSS_STUDENT_T: 4.0}[loss]
    with dba.Solver(sc, precision=dba.DBA_PREC_F64, tile_obs=tile, local_solver=dba.DBA_SOLVER_LBFGS) as s:
        cfg = oracle_cfg(s)
        st = O.State(sc)
        for it in range(5):
            mg = s.iterate(1)
            mo = st.iterate(cfg, 1)
            cams, pts = s.params()
            assert colerr(cams, st.cams) <= TOL64, it
            assert colerr(pts, st.pts) <= TOL64, it
            assert abs(mg["objective"] - mo["objective"]) <= 1e-8 * mo["objective"]


def test_fp64_lbfgs_ring_scene_many_iterations():
    sc = S.scene0()
    with dba.Solver(sc, precision=dba.DBA_PREC_F64, local_solver=dba.DBA_SOLVER_LBFGS) as s:
        cfg = oracle_cfg(s)
        st = O.State(sc)
        for chunk in (1, 9, 40):
            s.iterate(chunk, stats=False)
            st.iterate(cfg, chunk)
            cams, pts = s.params()
            assert colerr(cams, st.cams) <= TOL64 and colerr(pts, st.pts) <= TOL64


def test_fp32_lbfgs_tracks_the_fp64_oracle():
    sc = S.scene1(n_pts=3000, n_cams=24, seed=43)
    with dba.Solver(sc, precision=dba.DBA_PREC_F32_LOCAL, local_solver=dba.DBA_SOLVER_LBFGS) as s:
        cfg = oracle_cfg(s)
        st = O.State(sc)
        mg = s.iterate(60)
        mo = st.iterate(cfg, 60)
        assert abs(mg["rmse_gt"] - mo["rmse_gt"]) <= 1e-3
        assert abs(mg["rmse_obs"] - mo["rmse_obs"]) <= 1e-3


def test_lbfgs_and_gauss_newton_reach_the_target_alike():
    """Both local solvers converge to the same ADMM limit; on workload-2 geometry they
    reach 0.5 px within a few iterations of each other."""
    sc = S.scene2(n_pts=30000)
    its = {}
    for solver in (dba.DBA_SOLVER_GN, dba.DBA_SOLVER_LBFGS):
        with dba.Solver(sc, local_solver=solver) as s:
            m = s.iterate_until(400, 0.5)
            assert m["rmse_gt"] <= 0.5
            its[solver] = m["iters_done"]
    assert abs(its[0] - its[1]) <= 0.25 * its[0] + 2, its


def test_lbfgs_with_an_untrained_warm_start_keeps_the_limit():
    """The L-BFGS solve also starts from the better of the plain and the learned start, so
    a random network leaves the ADMM result within the FP32 tolerance."""
    from paper_1708_07954_gb300 import dba as D

    sc = S.scene1(n_pts=2000, n_cams=32, seed=79)
    mlp = D.Mlp(11)
    with D.Solver(sc, local_solver=D.DBA_SOLVER_LBFGS) as a, D.Solver(sc, local_solver=D.DBA_SOLVER_LBFGS) as b:
        b.set_warm_start(mlp)
        ma = a.iterate(120)
        mb = b.iterate(120)
        assert abs(ma["rmse_obs"] - mb["rmse_obs"]) <= 1e-3
        assert abs(ma["rmse_gt"] - mb["rmse_gt"]) <= 1e-3
