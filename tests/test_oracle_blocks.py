"""Pins of the block-subproblem oracle (generalized step, Sec. 3.1.4, Eq. 14).

Each test ties the oracle to something other than itself: the per-observation
method it must reduce to, brute force, an independent minimiser, the
centralized LM optimum, or the zero-sum dual invariant of Eqs. (10)-(13)."""
import numpy as np
import pytest

import oracle as O
from paper_1708_07954_gb300 import scenes as S


def test_layout_matches_brute_force_grouping():
    """Every observation lands in the block of (its point's group, its camera's group), in
    (point rank, camera) order inside it; copies are the distinct points/cameras of each
    block, in rank / index order."""
    sc = S.scene1(n_pts=300, n_cams=24, seed=5)
    for pi, kappa in ((1, 1), (8, 2), (32, 4), (7, 3)):
        B = O.BlockLayout(sc, pi, kappa)
        first = {}
        for o in range(sc.n_obs):
            i, j = int(sc.pt_idx[o]), int(sc.cam_idx[o])
            first[i] = min(first.get(i, 10 ** 9), j)
        ranked = sorted(first, key=lambda i: (first[i], i))
        rank = {i: r for r, i in enumerate(ranked)}
        blocks = {}
        for o in range(sc.n_obs):
            i, j = int(sc.pt_idx[o]), int(sc.cam_idx[o])
            blocks.setdefault((rank[i] // pi, j // kappa), []).append(o)
        keys = sorted(blocks)
        assert B.n_blocks == len(keys)
        for b, key in enumerate(keys):
            obs = B.blk_obs[B.obs_off[b]:B.obs_off[b + 1]]
            # inside a block: by point rank, then camera
            assert obs.tolist() == sorted(blocks[key], key=lambda o: (rank[int(sc.pt_idx[o])], int(sc.cam_idx[o])))
            pts = sorted({int(sc.pt_idx[o]) for o in blocks[key]}, key=lambda i: rank[i])
            cams = sorted({int(sc.cam_idx[o]) for o in blocks[key]})
            assert B.pc_pt[B.pc_off[b]:B.pc_off[b + 1]].tolist() == pts
            assert B.cc_cam[B.cc_off[b]:B.cc_off[b + 1]].tolist() == cams
            assert len(pts) <= pi and len(cams) <= kappa
            for k, o in enumerate(obs):
                assert pts[B.obs_lp[B.obs_off[b] + k]] == sc.pt_idx[o]
                assert cams[B.obs_lc[B.obs_off[b] + k]] == sc.cam_idx[o]


def test_one_point_one_camera_blocks_are_the_per_observation_method():
    """pi = kappa = 1: each block is one observation, so Eq. (14) is Eq. (9)."""
    sc = S.scene1(n_pts=400, n_cams=16, seed=9)
    cfg = O.config_for(sc)
    a, b = O.State(sc), O.BlockState(sc, 1, 1)
    ma, mb = a.iterate(cfg, 8), b.iterate(cfg, 8)
    assert np.abs(a.cams - b.cams).max() <= 1e-12 * np.abs(a.cams).max()
    assert np.abs(a.pts - b.pts).max() <= 1e-12 * np.abs(a.pts).max()
    for k in ("rmse_obs", "objective", "primal_res", "dual_res"):
        assert abs(ma[k] - mb[k]) <= 1e-9 * max(abs(ma[k]), 1e-300), k


def _tiny_block(seed):
    """3 points seen by 2 cameras (5 observations), consensus near the truth."""
    rng = np.random.default_rng(seed)
    sc = S.scene0(n_pts=3, n_cams=2, seed=seed)
    cfg = O.config_for(sc, loss=O.LOSS_HUBER, inner_steps=200)
    keep = np.array([0, 1, 2, 3, 4])
    opl = sc.pt_idx[keep].astype(np.int32)
    ocl = sc.cam_idx[keep].astype(np.int32)
    z = sc.z[keep].ravel()
    xbar, ybar = sc.pts0.ravel(), sc.cams0.ravel()
    rx = rng.normal(0, 0.1 * sc.rho_x * 1e-2, 9)
    sy = rng.normal(0, 0.1 * sc.rho_y * 1e-2, 12)
    return cfg, opl, ocl, z, xbar, ybar, rx, sy


@pytest.mark.parametrize("seed", [3, 4])
def test_block_solve_reaches_the_block_argmin(seed):
    """200 damped GN steps end at a stationary point of Eq. (14) (central differences of
    the objective, no Jacobian code) that an independent quasi-Newton minimiser agrees with."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    cfg, opl, ocl, z, xbar, ybar, rx, sy = _tiny_block(seed)
    X, Y = O.block_solve(cfg, opl, ocl, z, xbar, ybar, rx, sy, xbar, ybar)
    f = lambda v: O.block_objective(cfg, opl, ocl, z, xbar, ybar, rx, sy, v[:9], v[9:])
    v = np.concatenate([X, Y])
    g = np.zeros_like(v)
    for k in range(len(v)):
        h = 1e-6 * max(1.0, abs(v[k]))
        vp, vm = v.copy(), v.copy()
        vp[k] += h
        vm[k] -= h
        g[k] = (f(vp) - f(vm)) / (2 * h)
    v0 = np.concatenate([xbar, ybar])
    g0 = np.zeros_like(v0)
    for k in range(len(v0)):
        h = 1e-6 * max(1.0, abs(v0[k]))
        vp, vm = v0.copy(), v0.copy()
        vp[k] += h
        vm[k] -= h
        g0[k] = (f(vp) - f(vm)) / (2 * h)
    assert np.linalg.norm(g) <= 1e-6 * np.linalg.norm(g0)
    res = scipy_opt.minimize(f, v0, method="BFGS", options={"gtol": 1e-10, "maxiter": 20000})
    assert f(v) <= res.fun + 1e-9 * abs(res.fun)
    assert np.abs(res.x - v).max() <= 1e-4 * np.abs(v).max()


def test_single_block_is_a_proximal_iteration_that_reaches_the_dense_lm_optimum():
    """With every point and camera in one block, each point and camera has one copy, the
    dual ascent leaves the duals at zero, and the iteration is a proximal point method on
    the BA objective: it converges to the centralized LM optimum.  The optimum is a
    7-dimensional similarity orbit, so gauge-free quantities are compared: the objective
    and every observation's predicted pixel."""
    sc = S.scene0(n_pts=20, n_cams=4, seed=12)
    cfg = O.config_for(sc, loss=O.LOSS_L2, rho_x=0.1 * sc.rho_x, rho_y=0.1 * sc.rho_y,
                       rho_angle=0.1 * sc.rho_angle)
    st = O.BlockState(sc, 10 ** 6, 10 ** 6)
    assert st.layout.n_blocks == 1
    for _ in range(4):
        st.iterate(cfg, 25)
        assert np.abs(st.pduals).max() <= 1e-9 * cfg.rho_x
        assert np.abs(st.cduals).max() <= 1e-9 * cfg.rho_angle
    cams, pts, obj, _ = O.dense_lm(cfg, sc, max_iters=300)
    m = st.iterate(cfg, 1)
    assert abs(m["objective"] - obj) <= 1e-10 * obj
    for o in range(sc.n_obs):
        i, j = sc.pt_idx[o], sc.cam_idx[o]
        za, _ = O.project(cfg, st.pts[i], st.cams[j])
        zb, _ = O.project(cfg, pts[i], cams[j])
        assert np.abs(za - zb).max() <= 1e-6


@pytest.mark.parametrize("pi,kappa", [(8, 2), (32, 4)])
def test_block_duals_sum_to_zero_per_point_and_camera(pi, kappa):
    """Eqs. (10)-(13) over copies: after any iteration the duals of each point's copies sum
    to zero (likewise per camera)."""
    sc = S.scene1(n_pts=500, n_cams=24, seed=21)
    cfg = O.config_for(sc)
    st = O.BlockState(sc, pi, kappa)
    st.iterate(cfg, 5)
    B = st.layout
    sx = np.zeros((sc.n_pts, 3))
    np.add.at(sx, B.pc_pt, st.pduals)
    sy = np.zeros((sc.n_cams, 6))
    np.add.at(sy, B.cc_cam, st.cduals)
    assert np.abs(sx).max() <= 1e-9 * np.abs(st.pduals).max()
    assert np.abs(sy).max() <= 1e-9 * np.abs(st.cduals).max()


def test_larger_blocks_converge_in_fewer_iterations():
    """The paper's observation (Sec. 4): more points and cameras per update step lower the
    reprojection error faster per iteration."""
    sc = S.scene1(n_pts=600, n_cams=24, seed=33)
    cfg = O.config_for(sc)
    gt = {}
    for pi, kappa in ((1, 1), (8, 2), (32, 4)):
        st = O.BlockState(sc, pi, kappa)
        gt[(pi, kappa)] = st.iterate(cfg, 15)["rmse_gt"]
    assert gt[(32, 4)] < gt[(8, 2)] < gt[(1, 1)], gt


@pytest.mark.parametrize("seed", [3, 4])
def test_block_noise_rule_keeps_the_minimum(seed):
    """Trusting block steps whose predicted decrease is below the rounding noise of Eq. (14)
    converges to the same minimiser as plain comparisons."""
    cfg, opl, ocl, z, xbar, ybar, rx, sy = _tiny_block(seed)
    cfg.lm_model_tol = 0.0
    X0, Y0 = O.block_solve(cfg, opl, ocl, z, xbar, ybar, rx, sy, xbar, ybar)
    cfg.lm_model_tol = 16.0
    X1, Y1 = O.block_solve(cfg, opl, ocl, z, xbar, ybar, rx, sy, xbar, ybar)
    v0, v1 = np.r_[X0, Y0], np.r_[X1, Y1]
    assert np.all(np.abs(v1 - v0) <= 1e-9 * (1 + np.abs(v0)))


def test_block_admm_is_insensitive_to_last_bit_perturbations():
    """With the noise rule a one-ulp difference in the state stays at the rounding level over
    block iterations; with plain comparisons alone the same difference grows by orders of
    magnitude (steps at the rounding level are accepted or rejected by the rounding)."""
    sc = S.scene0()

    def spread(tol):
        cfg = O.config_for(sc, lm_model_tol=tol)
        a, b = O.BlockState(sc, 4, 2), O.BlockState(sc, 4, 2)
        b.pts = b.pts * (1 + 2.2e-16)
        b.pcopies = b.pcopies * (1 + 2.2e-16)
        for _ in range(6):
            a.iterate(cfg, 1, with_gt=False)
            b.iterate(cfg, 1, with_gt=False)
        return np.max([np.abs(a.pts - b.pts).max() / np.abs(a.pts).max(),
                       np.abs(a.cams - b.cams).max() / np.abs(a.cams).max()])

    with_rule = spread(16.0)
    assert with_rule < 1e-13
    assert spread(0.0) > 100 * with_rule
