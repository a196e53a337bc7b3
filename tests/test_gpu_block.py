"""Block subproblems (Sec. 3.1.4, Eq. 14) on the GPU against the block oracle."""
import numpy as np
import pytest
from parity import BLOCK_SETTINGS, colerr

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


def size_classes(layout):
    """Blocks per size class of the solve kernel, recounted from the oracle's layout:
    one camera and <= 8 points, <= 2 cameras and <= 16 points, <= 32 points, the rest."""
    npb, ncb = np.diff(layout.pc_off), np.diff(layout.cc_off)
    c8 = (ncb == 1) & (npb <= 8)
    c16 = ~c8 & (ncb <= 2) & (npb <= 16)
    c32 = ~c8 & ~c16 & (npb <= 32)
    return [int(c8.sum()), int(c16.sum()), int(c32.sum()), int((~c8 & ~c16 & ~c32).sum())]


# BLOCK_SETTINGS put blocks in every kernel variant (tests/test_block_variants.py checks it)
@pytest.mark.parametrize("pi,kappa", BLOCK_SETTINGS)
def test_fp64_matches_block_oracle_per_iteration(pi, kappa):
    sc = S.scene1(n_pts=400, n_cams=16, seed=17)
    with dba.BlockSolver(sc, pi, kappa, precision=dba.DBA_PREC_F64) as s:
        cfg = oracle_cfg(s)
        st = O.BlockState(sc, pi, kappa)
        lay = s.layout()
        assert lay == {"n_blocks": st.layout.n_blocks, "n_point_copies": st.layout.n_pc,
                       "n_camera_copies": st.layout.n_cc}
        assert s.size_classes() == size_classes(st.layout)
        for it in range(6):
            mg = s.iterate(1)
            mo = st.iterate(cfg, 1)
            cams, pts = s.params()
            assert colerr(cams, st.cams) <= TOL64, it
            assert colerr(pts, st.pts) <= TOL64, it
            for k in ("rmse_obs", "objective", "primal_res", "dual_res"):
                assert abs(mg[k] - mo[k]) <= 1e-8 * max(abs(mo[k]), 1e-12), (it, k)
            assert abs(mg["rmse_gt"] - mo["rmse_gt"]) <= 1e-8 * max(mo["rmse_gt"], 1e-12)


def test_fp64_ring_scene_many_iterations():
    """Workload-0 geometry (every point in every view): blocks of 8 points x 2 cameras
    for 30 iterations stay with the oracle."""
    sc = S.scene0()
    with dba.BlockSolver(sc, 8, 2, precision=dba.DBA_PREC_F64) as s:
        cfg = oracle_cfg(s)
        st = O.BlockState(sc, 8, 2)
        for chunk in (1, 9, 20):
            s.iterate(chunk, stats=False)
            st.iterate(cfg, chunk)
            cams, pts = s.params()
            assert colerr(cams, st.cams) <= TOL64 and colerr(pts, st.pts) <= TOL64


def test_one_point_one_camera_blocks_equal_the_per_observation_path():
    sc = S.scene1(n_pts=500, n_cams=16, seed=23)
    with dba.BlockSolver(sc, 1, 1, precision=dba.DBA_PREC_F64) as a, \
            dba.Solver(sc, precision=dba.DBA_PREC_F64) as b:
        a.iterate(10, stats=False)
        b.iterate(10, stats=False)
        ca, pa = a.params()
        cb, pb = b.params()
        assert colerr(ca, cb) <= TOL64 and colerr(pa, pb) <= TOL64


# every FP32 solve kernel: one camera in groups of 1 to 32 lanes (32 x 1), two and four
# camera slots, and two point copies a lane
@pytest.mark.parametrize("pi,kappa", [(8, 2), (32, 1), (32, 4), (64, 2)])
def test_fp32_tracks_the_fp64_oracle(pi, kappa):
    sc = S.scene1(n_pts=1500, n_cams=24, seed=29)
    with dba.BlockSolver(sc, pi, kappa, precision=dba.DBA_PREC_F32_LOCAL) as s:
        cfg = oracle_cfg(s)
        st = O.BlockState(sc, pi, kappa)
        mg = s.iterate(40)
        mo = st.iterate(cfg, 40)
        assert abs(mg["rmse_gt"] - mo["rmse_gt"]) <= 1e-3
        assert abs(mg["rmse_obs"] - mo["rmse_obs"]) <= 1e-3
        cams, _ = s.params()
        assert relerr(cams, st.cams) <= 1e-4


def test_edge_cases_single_observation_points_and_unobserved_points():
    """Tracks of length one, a point with no observation (keeps its value), one camera
    per block and one point per block in the same problem."""
    sc = S.scene1(n_pts=200, n_cams=12, seed=31)
    keep = np.ones(sc.n_obs, bool)
    first = np.searchsorted(sc.pt_idx, np.arange(sc.n_pts))
    # point 0: no observation; points 1..20: only their first observation
    keep[sc.pt_idx == 0] = False
    for i in range(1, 21):
        idx = np.nonzero(sc.pt_idx == i)[0]
        keep[idx[1:]] = False
    del first
    sub = S.Scene(n_cams=sc.n_cams, n_pts=sc.n_pts, pt_idx=sc.pt_idx[keep], cam_idx=sc.cam_idx[keep],
                  z=sc.z[keep], z_true=sc.z_true[keep], outlier=sc.outlier[keep], cams_gt=sc.cams_gt,
                  pts_gt=sc.pts_gt, cams0=sc.cams0, pts0=sc.pts0, focal=sc.focal, cx=sc.cx, cy=sc.cy,
                  loss=sc.loss, loss_param=sc.loss_param, rho_x=sc.rho_x, rho_y=sc.rho_y,
                  rho_angle=sc.rho_angle)
    for pi, kappa in ((1, 1), (7, 3), (64, 2)):
        with dba.BlockSolver(sub, pi, kappa, precision=dba.DBA_PREC_F64) as s:
            cfg = oracle_cfg(s)
            st = O.BlockState(sub, pi, kappa)
            s.iterate(5, stats=False)
            st.iterate(cfg, 5)
            cams, pts = s.params()
            assert colerr(cams, st.cams) <= TOL64 and colerr(pts, st.pts) <= TOL64
            assert np.array_equal(pts[0], sub.pts0[0])


def test_larger_blocks_reach_the_target_in_fewer_iterations():
    """Sec. 4: more points and cameras per update lower the error faster per iteration."""
    sc = S.scene2(n_pts=20000)
    its = {}
    for pi, kappa in ((1, 1), (8, 2), (32, 4)):
        with dba.BlockSolver(sc, pi, kappa) as s:
            its[(pi, kappa)] = s.iterate_until(400, 0.5)["iters_done"]
    assert its[(32, 4)] < its[(8, 2)] < its[(1, 1)], its


def test_errors():
    sc = S.scene0(n_pts=10, n_cams=3)
    with pytest.raises(dba.DbaError) as e:
        dba.BlockSolver(sc, 65, 1)
    assert e.value.status == dba.DBA_EINVAL
    with pytest.raises(dba.DbaError) as e:
        dba.BlockSolver(sc, 4, 5)
    assert e.value.status == dba.DBA_EINVAL
    with dba.BlockSolver(sc, 4, 2, ground_truth=False) as s:
        with pytest.raises(dba.DbaError) as e:
            s.iterate_until(5, 0.5)
        assert e.value.status == dba.DBA_ESTATE


def test_full_size_workload2_blocks_fp64_sampled():
    """Blocks of 32 points x 2 cameras on the full workload 2 (~4M observations), FP64:
    after one iteration from the initial state (zero duals) each point is the mean of its
    block copies (Eqs. 10-11 over copies); for sampled points every block holding the point
    is re-solved by the oracle (Eq. 14) and the mean compared, <= 1e-9."""
    sc = S.scene2()
    with dba.BlockSolver(sc, 32, 2, precision=dba.DBA_PREC_F64) as s:
        s.iterate(1, stats=False)
        _, pts = s.params()
        cfg = oracle_cfg(s)
    B = O.BlockLayout(sc, 32, 2)
    blk_of_pc = np.repeat(np.arange(B.n_blocks), np.diff(B.pc_off))
    order = np.argsort(B.pc_pt, kind="stable")
    off = np.searchsorted(B.pc_pt[order], np.arange(sc.n_pts + 1))
    rng = np.random.default_rng(5)
    zero3 = lambda n: np.zeros(3 * n)
    got, want = [], []
    for i in rng.choice(sc.n_pts, 60, replace=False):
        copies = []
        for k in order[off[i]:off[i + 1]]:
            b = blk_of_pc[k]
            o0, o1 = B.obs_off[b], B.obs_off[b + 1]
            obs = B.blk_obs[o0:o1]
            pcs = B.pc_pt[B.pc_off[b]:B.pc_off[b + 1]]
            ccs = B.cc_cam[B.cc_off[b]:B.cc_off[b + 1]]
            xbar, ybar = sc.pts0[pcs].ravel(), sc.cams0[ccs].ravel()
            X, _ = O.block_solve(cfg, B.obs_lp[o0:o1], B.obs_lc[o0:o1], sc.z[obs].ravel(), xbar, ybar,
                                 zero3(len(pcs)), np.zeros(6 * len(ccs)), xbar, ybar)
            copies.append(X.reshape(-1, 3)[int(k - B.pc_off[b])])
        if copies:
            got.append(pts[i])
            want.append(np.mean(copies, axis=0))
    assert colerr(np.array(got), np.array(want)) <= TOL64


def test_a_repeated_point_camera_pair_is_rejected():
    sc = S.scene0(n_pts=10, n_cams=3)
    dup = S.Scene(n_cams=sc.n_cams, n_pts=sc.n_pts, pt_idx=np.r_[sc.pt_idx, sc.pt_idx[:1]].astype(np.int32),
                  cam_idx=np.r_[sc.cam_idx, sc.cam_idx[:1]].astype(np.int32), z=np.r_[sc.z, sc.z[:1]],
                  z_true=np.r_[sc.z_true, sc.z_true[:1]], outlier=np.r_[sc.outlier, sc.outlier[:1]],
                  cams_gt=sc.cams_gt, pts_gt=sc.pts_gt, cams0=sc.cams0, pts0=sc.pts0, focal=sc.focal,
                  cx=sc.cx, cy=sc.cy, loss=sc.loss, loss_param=sc.loss_param, rho_x=sc.rho_x, rho_y=sc.rho_y,
                  rho_angle=sc.rho_angle)
    with pytest.raises(dba.DbaError) as e:
        dba.BlockSolver(dup, 4, 2)
    assert e.value.status == dba.DBA_EINVAL and "observed twice" in str(e.value)


def expected_launches(layout, kappa):
    """Kernel launches of one block iteration, recounted from the oracle's layout by the
    library's documented dispatch: one block-solve launch per nonempty range of blocks
    sharing a kernel and lane-group width, then the point and camera consensus."""
    npb, ncb = np.diff(layout.pc_off), np.diff(layout.cc_off)
    c0 = (ncb == 1) & (npb <= 8)
    c1 = ~c0 & (ncb <= 2) & (npb <= 16)
    c2 = ~c0 & ~c1 & (npb <= 32)
    c3 = ~c0 & ~c1 & ~c2
    ranges = [c0 & (npb == 1), c0 & (npb == 2), c0 & (npb > 2) & (npb <= 4), c0 & (npb > 4)]
    if kappa == 1:
        ranges += [c1, c2]
    else:
        ranges += [c1 & (npb == 1), c1 & (npb > 1) & (npb <= 4), c1 & (npb > 4) & (npb <= 8), c1 & (npb > 8),
                   c2 & (npb == 1), c2 & (npb > 1)]
    ranges += [c3]
    return sum(1 for r in ranges if r.any()) + 2


@pytest.mark.parametrize("pi,kappa", BLOCK_SETTINGS)
def test_launches_per_iteration_match_the_layout(pi, kappa):
    sc = S.scene1(n_pts=400, n_cams=16, seed=17)
    with dba.BlockSolver(sc, pi, kappa, precision=dba.DBA_PREC_F32_LOCAL) as s:
        assert s.launches_per_iteration() == expected_launches(O.BlockLayout(sc, pi, kappa), kappa)
