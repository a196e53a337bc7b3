"""Pins for the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: hand-derived
values (tests/golden), textbook matrices, a library rotation routine, finite
differences, brute-force minimisation with an independent objective, derived
ADMM invariants, the noise-free fixed point (Thm. 1) and a centralized LM.
"""
import os

import numpy as np
import pytest
from scipy.optimize import minimize
from scipy.spatial.transform import Rotation

import oracle as O
from paper_1708_07954_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cases():
    rows = []
    with open(os.path.join(GOLDEN, "projection_cases.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(t) for t in line.split()])
    return np.array(rows)


# ---------------------------------------------------------------- Sec. 2.1
def test_projection_golden_cases():
    """Hand-derived pinhole values (Sec. 2.1, Eq. 1)."""
    for row in _cases():
        x, y, (f, cx, cy), want = row[0:3], row[3:9], row[9:12], row[12:15]
        cfg = O.config(focal=f, cx=cx, cy=cy)
        zp, depth = O.project(cfg, x, y)
        np.testing.assert_allclose(zp, want[:2], rtol=0, atol=1e-9)
        assert abs(depth - want[2]) < 1e-12


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_single_axis_rotations_are_textbook(axis):
    a = 0.37
    c, s = np.cos(a), np.sin(a)
    text = [np.array([[1, 0, 0], [0, c, -s], [0, s, c]]),
            np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]]),
            np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])][axis]
    y = np.zeros(6)
    y[axis] = a
    np.testing.assert_allclose(O.rotation(y), text, atol=1e-15)


def test_rotation_composition_matches_library():
    """R = R3(gamma) R2(beta) R1(alpha): extrinsic x-y-z Euler angles in scipy."""
    rng = np.random.default_rng(0)
    for _ in range(50):
        ang = rng.uniform(-np.pi, np.pi, 3)
        ang[1] = rng.uniform(-1.4, 1.4)
        R = O.rotation(np.r_[ang, 0, 0, 0])
        np.testing.assert_allclose(R, Rotation.from_euler("xyz", ang).as_matrix(), atol=1e-14)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-13


def test_projection_matches_generator_sensor():
    """Oracle f(x*, y*) equals the generator's look-at sensor output (independent construction)."""
    for s in (S.scene0(), S.scene1(n_pts=300), S.scene2(n_pts=300, lanes=3, stations=10)):
        cfg = O.config_for(s)
        k = min(200, s.n_obs)
        zp = np.array([O.project(cfg, s.pts_gt[i], s.cams_gt[j])[0]
                       for i, j in zip(s.pt_idx[:k], s.cam_idx[:k])])
        np.testing.assert_allclose(zp, s.z_true[:k], rtol=0, atol=1e-9)


def test_jacobian_matches_central_differences():
    s = S.scene1(n_pts=50)
    cfg = O.config_for(s)
    rng = np.random.default_rng(1)
    for o in rng.choice(s.n_obs, 20, replace=False):
        x = s.pts0[s.pt_idx[o]]
        y = s.cams0[s.cam_idx[o]]
        v = np.r_[x, y]
        J = O.jacobian(cfg, x, y)
        Jfd = np.zeros((2, 9))
        for k in range(9):
            h = 1e-6 * max(1.0, abs(v[k]))
            vp, vm = v.copy(), v.copy()
            vp[k] += h
            vm[k] -= h
            Jfd[:, k] = (O.project(cfg, vp[:3], vp[3:])[0] - O.project(cfg, vm[:3], vm[3:])[0]) / (2 * h)
        assert np.abs(J - Jfd).max() <= 1e-7 * np.abs(J).max()


# -------------------------------------------------------- losses, Sec. 3.1
def test_losses_closed_forms_and_weights():
    d, nu = 2.0, 4.0
    for sq in [0.0, 0.5, 3.9, 4.0, 4.1, 25.0, 400.0]:
        assert O.loss(O.LOSS_L2, 0, sq) == sq
        hub = sq if sq <= d * d else 2 * d * np.sqrt(sq) - d * d
        assert abs(O.loss(O.LOSS_HUBER, d, sq) - hub) < 1e-12
        assert abs(O.loss(O.LOSS_STUDENT_T, nu, sq) - nu * np.log1p(sq / nu)) < 1e-12
        for kind, p in [(O.LOSS_L2, 0), (O.LOSS_HUBER, d), (O.LOSS_STUDENT_T, nu)]:
            if sq > 0 and abs(sq - d * d) > 1e-3:
                h = 1e-6 * max(1, sq)
                fd = (O.loss(kind, p, sq + h) - O.loss(kind, p, sq - h)) / (2 * h)
                assert abs(O.weight(kind, p, sq) - fd) < 1e-6
    # Huber equals squared l2 inside delta and is C1 at the knot
    assert O.loss(O.LOSS_HUBER, d, 3.0) == 3.0
    assert abs(O.weight(O.LOSS_HUBER, d, 4.0 + 1e-12) - 1.0) < 1e-6
    # Student's t approaches squared l2 near zero
    assert abs(O.loss(O.LOSS_STUDENT_T, nu, 1e-6) - 1e-6) < 1e-12


def test_cholesky_matches_numpy():
    rng = np.random.default_rng(2)
    for n in (1, 2, 9, 30):
        A = rng.normal(size=(n, n))
        A = A @ A.T + n * np.eye(n)
        b = rng.normal(size=n)
        np.testing.assert_allclose(O.chol_solve(A, b), np.linalg.solve(A, b), rtol=1e-12, atol=1e-12)
    with pytest.raises(np.linalg.LinAlgError):
        O.chol_solve(-np.eye(3), np.ones(3))
    # every pivot below 1 (a well-posed system at a small scale) still solves ...
    A = rng.normal(size=(9, 9))
    A = 1e-6 * (A @ A.T + 9 * np.eye(9))
    b = rng.normal(size=9)
    np.testing.assert_allclose(O.chol_solve(A, b), np.linalg.solve(A, b), rtol=1e-10)
    # ... and an exactly zero pivot is refused, not divided by
    with pytest.raises(np.linalg.LinAlgError):
        O.chol_solve(np.diag([1.0, 0.0, 1.0]), np.ones(3))


# ------------------------------------------------- local subproblem, Eq. (9)
def _indep_local_objective(kind, p, f, cx, cy, z, xbar, ybar, dual, rho_x, rho_y, v, rho_a=None):
    """Eq. (9) written with a library rotation and numpy only (rho_a: camera-angle penalty)."""
    R = Rotation.from_euler("xyz", v[3:6]).as_matrix()
    q = R @ v[:3] + v[6:9]
    if q[2] <= 1e-6:
        return 1e30
    e = z - (f * q[:2] / q[2] + np.array([cx, cy]))
    sq = e @ e
    if kind == O.LOSS_HUBER:
        phi = sq if sq <= p * p else 2 * p * np.sqrt(sq) - p * p
    elif kind == O.LOSS_STUDENT_T:
        phi = p * np.log1p(sq / p)
    else:
        phi = sq
    dx, dy = v[:3] - xbar, v[3:] - ybar
    ra = rho_y if rho_a is None else rho_a
    return (phi + dual[:3] @ dx + dual[3:] @ dy + 0.5 * rho_x * dx @ dx + 0.5 * ra * dy[:3] @ dy[:3]
            + 0.5 * rho_y * dy[3:] @ dy[3:])


def _local_case(seed, kind):
    s = S.scene0(seed=seed)
    rng = np.random.default_rng(seed)
    o = int(rng.integers(s.n_obs))
    xbar, ybar = s.pts0[s.pt_idx[o]], s.cams0[s.cam_idx[o]]
    dual = rng.normal(0, 5.0, 9)
    z = s.z[o] + rng.normal(0, 3.0, 2)
    p = {O.LOSS_L2: 0.0, O.LOSS_HUBER: 2.0, O.LOSS_STUDENT_T: 4.0}[kind]
    cfg = O.config_for(s, loss=kind, loss_param=p, rho_x=2000.0, rho_y=2000.0, rho_angle=0.0)
    return s, cfg, z, xbar, ybar, dual, p


@pytest.mark.parametrize("kind", [O.LOSS_L2, O.LOSS_HUBER, O.LOSS_STUDENT_T])
def test_local_objective_matches_independent_restatement(kind):
    s, cfg, z, xbar, ybar, dual, p = _local_case(3, kind)
    rng = np.random.default_rng(4)
    for _ in range(10):
        v = np.r_[xbar, ybar] + rng.normal(0, 1e-2, 9)
        a = O.local_objective(cfg, z, xbar, ybar, dual, v)
        b = _indep_local_objective(kind, p, s.focal, s.cx, s.cy, z, xbar, ybar, dual, 2000.0, 2000.0, v)
        assert abs(a - b) <= 1e-10 * max(1.0, abs(b))
        # a separate camera-angle penalty weights only the three Euler angles
        cfg.rho_angle = 9.0e4
        a = O.local_objective(cfg, z, xbar, ybar, dual, v)
        b = _indep_local_objective(kind, p, s.focal, s.cx, s.cy, z, xbar, ybar, dual, 2000.0, 2000.0, v,
                                   rho_a=9.0e4)
        cfg.rho_angle = 0.0
        assert abs(a - b) <= 1e-10 * max(1.0, abs(b))


@pytest.mark.parametrize("rho_a", [None, 5.0e4])
@pytest.mark.parametrize("kind", [O.LOSS_L2, O.LOSS_HUBER, O.LOSS_STUDENT_T])
def test_local_solve_reaches_brute_force_minimum(kind, rho_a):
    """Long damped-GN run equals a BFGS minimisation of the independently written Eq. (9)."""
    for seed in (5, 6, 7):
        s, cfg, z, xbar, ybar, dual, p = _local_case(seed, kind)
        cfg.inner_steps = 200
        cfg.lm_model_tol = 0.0  # plain comparisons on every step: converge to the rounding floor
        cfg.rho_angle = 0.0 if rho_a is None else rho_a
        v0 = np.r_[xbar, ybar]
        v = O.local_solve(cfg, z, xbar, ybar, dual, v0)
        fun = lambda u: _indep_local_objective(kind, p, s.focal, s.cx, s.cy, z, xbar, ybar, dual,
                                               2000.0, 2000.0, v0 + u, rho_a=rho_a)
        res = minimize(fun, np.zeros(9), method="BFGS", options={"gtol": 1e-10, "maxiter": 5000})
        vb = v0 + res.x
        assert O.local_objective(cfg, z, xbar, ybar, dual, v) <= fun(res.x) + 1e-9
        np.testing.assert_allclose(v, vb, rtol=0, atol=2e-6)
        # first-order optimality of Eq. (9) by central differences of the independent objective
        g = np.array([(fun(v - v0 + h) - fun(v - v0 - h)) / 2e-6 for h in np.eye(9) * 1e-6])
        assert np.abs(g).max() < 1e-3


@pytest.mark.parametrize("kind", [O.LOSS_L2, O.LOSS_HUBER, O.LOSS_STUDENT_T])
def test_local_solve_noise_rule_keeps_the_minimum(kind):
    """Trusting model steps below the objective's rounding noise converges to the same
    minimiser as plain comparisons, to well below sqrt(eps)."""
    for seed in (9, 10):
        s, cfg, z, xbar, ybar, dual, p = _local_case(seed, kind)
        v0 = np.r_[xbar, ybar]
        cfg.inner_steps, cfg.lm_model_tol = 300, 0.0
        vinf = O.local_solve(cfg, z, xbar, ybar, dual, v0)
        cfg.lm_model_tol = 16.0
        v1 = O.local_solve(cfg, z, xbar, ybar, dual, v0)
        assert np.all(np.abs(v1 - vinf) <= 1e-9 * (1 + np.abs(vinf)))


def test_admm_is_insensitive_to_last_bit_perturbations():
    """With the noise rule, one ulp of difference in the state stays at the rounding level over
    iterations (plain objective comparisons amplify it ~1e6 in one iteration)."""
    s = S.scene0()
    c = O.config_for(s)
    a, b = O.State(s), O.State(s)
    b.pts = b.pts * (1 + 2.2e-16)
    b.copies[:, :3] *= 1 + 2.2e-16
    for _ in range(6):
        a.iterate(c, 1)
        b.iterate(c, 1)
    err = np.max([np.abs(a.pts - b.pts).max() / np.abs(a.pts).max(), np.abs(a.cams - b.cams).max() / np.abs(a.cams).max()])
    assert err < 1e-13


def test_local_solve_monotone_and_fixed_count():
    """Each accepted step lowers Eq. (9) (up to its rounding noise, where model steps are
    trusted); zero steps leave the copy unchanged."""
    s, cfg, z, xbar, ybar, dual, p = _local_case(8, O.LOSS_HUBER)
    v0 = np.r_[xbar, ybar] + 1e-3
    prev = O.local_objective(cfg, z, xbar, ybar, dual, v0)
    for k in range(1, 8):
        cfg.inner_steps = k
        cur = O.local_objective(cfg, z, xbar, ybar, dual, O.local_solve(cfg, z, xbar, ybar, dual, v0))
        assert cur <= prev + 1e-12 * abs(prev)
        prev = cur
    cfg.inner_steps = 0
    np.testing.assert_array_equal(O.local_solve(cfg, z, xbar, ybar, dual, v0), v0)


def test_local_solve_rejects_points_behind_camera():
    """Copies are never moved to depth <= eps (Thm. 1 proof, A4 reading)."""
    cfg = O.config(rho_x=1.0, rho_y=1.0, loss=O.LOSS_L2)
    xbar, ybar = np.array([0.0, 0.0, 1.0]), np.zeros(6)
    z = np.array([320.0 + 5000.0, 240.0])  # pulls strongly sideways
    dual = np.array([0, 0, 50.0, 0, 0, 0, 0, 0, 0])  # pushes the point backwards
    cfg.inner_steps = 30
    v = O.local_solve(cfg, z, xbar, ybar, dual, np.r_[xbar, ybar])
    assert O.project(cfg, v[:3], v[3:])[1] > cfg.eps_depth


# ------------------------------------------- ADMM iteration, Eqs. (9)-(13)
def test_noise_free_ground_truth_is_a_fixed_point():
    """Thm. 1 stationarity: copies = consensus = ground truth and zero duals stay put."""
    s = S.scene0()
    s.z = s.z_true.copy()
    cfg = O.config_for(s)
    st = O.State(s, cams=s.cams_gt, pts=s.pts_gt)
    m = st.iterate(cfg, 3)
    np.testing.assert_allclose(st.cams, s.cams_gt, rtol=0, atol=1e-12)
    np.testing.assert_allclose(st.pts, s.pts_gt, rtol=0, atol=1e-12)
    assert np.abs(st.duals).max() < 1e-6
    assert m["rmse_obs"] < 1e-9 and m["primal_res"] < 1e-10


def test_duals_sum_to_zero_per_segment():
    """Derived from Eqs. (10)-(13): after every iteration each point's r and each camera's s sum to 0."""
    s = S.scene1(n_pts=400, n_cams=16)
    cfg = O.config_for(s, rho_x=s.rho_x * 0.1, rho_y=s.rho_y * 0.1)
    st = O.State(s)
    for _ in range(4):
        st.iterate(cfg, 1)
        sr = np.zeros((s.n_pts, 3))
        np.add.at(sr, s.pt_idx, st.duals[:, :3])
        ss = np.zeros((s.n_cams, 6))
        np.add.at(ss, s.cam_idx, st.duals[:, 3:])
        assert np.abs(sr).max() < 1e-8 * max(1.0, np.abs(st.duals).max())
        assert np.abs(ss).max() < 1e-8 * max(1.0, np.abs(st.duals).max())
        # hence (derived) the consensus equals the plain mean of the copies
        mx = np.zeros((s.n_pts, 3))
        np.add.at(mx, s.pt_idx, st.copies[:, :3])
        cnt = np.bincount(s.pt_idx, minlength=s.n_pts)[:, None]
        np.testing.assert_allclose(st.pts, mx / cnt, rtol=0, atol=1e-10)


def test_first_iteration_consensus_is_mean_of_copies():
    """With zero initial duals, Eqs. (10)/(11) reduce to the mean of the new copies."""
    s = S.scene0(n_pts=30, n_cams=5)
    cfg = O.config_for(s)
    st = O.State(s)
    st.iterate(cfg, 1)
    my = np.zeros((s.n_cams, 6))
    np.add.at(my, s.cam_idx, st.copies[:, 3:])
    np.testing.assert_allclose(st.cams, my / np.bincount(s.cam_idx)[:, None], rtol=0, atol=1e-12)


def test_unobserved_camera_and_point_keep_their_values():
    s = S.scene0(n_pts=30, n_cams=5)
    keep = (s.cam_idx != 2) & (s.pt_idx != 7)
    s.pt_idx, s.cam_idx, s.z, s.z_true = s.pt_idx[keep], s.cam_idx[keep], s.z[keep], s.z_true[keep]
    cfg = O.config_for(s)
    st = O.State(s)
    st.iterate(cfg, 3)
    np.testing.assert_array_equal(st.cams[2], s.cams0[2])
    np.testing.assert_array_equal(st.pts[7], s.pts0[7])


@pytest.mark.parametrize("kind", [O.LOSS_L2, O.LOSS_HUBER])
def test_converged_admm_matches_centralized_lm(kind):
    """Thm. 1: the ADMM limit is a stationary point of Eq. (2) with phi_m; compare with dense LM
    (Sec. 4 stop rule) on a tiny scene of the Sec. 4.2 size (5 cameras, 10 points, 50 observations)."""
    s = S.scene0(n_pts=10, n_cams=5, seed=11)
    cfg = O.config_for(s, loss=kind, rho_x=2000.0, rho_y=2000.0, rho_angle=0.0)
    st = O.State(s)
    st.iterate(cfg, 4000)
    cams_lm, pts_lm, obj_lm, it = O.dense_lm(cfg, s, max_iters=500)
    m = st.metrics(cfg)
    assert abs(m["objective"] - obj_lm) <= 1e-6 * obj_lm
    # gauge-invariant comparison: predicted pixels of every observation
    pa = np.array([O.project(cfg, st.pts[i], st.cams[j])[0] for i, j in zip(s.pt_idx, s.cam_idx)])
    pb = np.array([O.project(cfg, pts_lm[i], cams_lm[j])[0] for i, j in zip(s.pt_idx, s.cam_idx)])
    assert np.abs(pa - pb).max() < 1e-3


def test_dense_lm_stop_rule_on_noise_free_data():
    """Sec. 4: LM stops once the objective drops below 1e-14."""
    s = S.scene0(n_pts=10, n_cams=5, seed=12)
    s.z = s.z_true.copy()
    cfg = O.config_for(s, loss=O.LOSS_L2)
    _, _, obj, it = O.dense_lm(cfg, s, max_iters=1000)
    assert obj < 1e-14 and it < 1000


# --------------------------------------------- warm-start network reference
def test_mlp_reference_gradient_matches_finite_differences():
    import oracle.mlp as OM

    rng = np.random.default_rng(21)
    p = rng.normal(0, 0.3, OM.N_PARAMS)
    p[OM.N_TRAINABLE + OM.N_IN:OM.N_TRAINABLE + 2 * OM.N_IN] = rng.uniform(0.5, 2, OM.N_IN)
    p[OM.N_TRAINABLE + 2 * OM.N_IN:] = rng.uniform(0.5, 2, OM.N_OUT)
    f = rng.normal(0, 1, (7, OM.N_IN))
    t = rng.normal(0, 1, (7, OM.N_OUT))
    loss, g = OM.loss_and_grad(p, f, t)
    for k in rng.choice(OM.N_TRAINABLE, 40, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (OM.loss_and_grad(pp, f, t)[0] - OM.loss_and_grad(pm, f, t)[0]) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * max(1.0, abs(fd))
    # the unused outputs 9..15 and the normaliser get no gradient
    assert np.all(g[OM.N_TRAINABLE:] == 0)


def test_mlp_reference_forward_loss_and_gradient_match_torch():
    """The network as the layout documents it, stated with torch's own modules in float64 (the
    tanh-form GELU, linear layers, standardised inputs, the mean squared error over the first 9
    outputs against scaled targets), and its gradient by torch's autograd: every output, the
    loss and every trainable parameter's derivative agree with the numpy reference."""
    import torch
    import torch.nn.functional as F

    import oracle.mlp as OM

    rng = np.random.default_rng(22)
    p = rng.normal(0, 0.3, OM.N_PARAMS)
    p[OM.N_TRAINABLE:OM.N_TRAINABLE + OM.N_IN] = rng.normal(0, 1, OM.N_IN)
    p[OM.N_TRAINABLE + OM.N_IN:OM.N_TRAINABLE + 2 * OM.N_IN] = rng.uniform(0.5, 2, OM.N_IN)
    p[OM.N_TRAINABLE + 2 * OM.N_IN:] = rng.uniform(0.5, 2, OM.N_OUT)
    f = rng.normal(0, 1, (11, OM.N_IN))
    t = rng.normal(0, 1, (11, OM.N_OUT))

    q = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in OM.unpack(p).items()}
    x = (torch.tensor(f) - q["in_mean"]) / q["in_std"]
    h = F.gelu(F.linear(x, q["W1"], q["b1"]), approximate="tanh")
    h = F.gelu(F.linear(h, q["W2"], q["b2"]), approximate="tanh")
    h = F.gelu(F.linear(h, q["W3"], q["b3"]), approximate="tanh")
    y = F.linear(h, q["W4"], q["b4"])
    target = torch.tensor(t) / q["out_scale"]
    loss = F.mse_loss(y[:, :OM.N_USED], target[:, :OM.N_USED])
    loss.backward()

    y_ref, _ = OM.forward(p, f)
    np.testing.assert_allclose(y_ref, y.detach().numpy(), rtol=1e-12, atol=1e-12)
    loss_ref, g_ref = OM.loss_and_grad(p, f, t)
    assert abs(loss_ref - loss.item()) <= 1e-12 * loss.item()
    trainable = [name for name, _ in OM.SHAPES][:8]
    g_torch = np.concatenate([q[name].grad.numpy().ravel() for name in trainable])
    assert len(g_torch) == OM.N_TRAINABLE
    np.testing.assert_allclose(g_ref[:OM.N_TRAINABLE], g_torch, rtol=1e-10, atol=1e-13)


def test_mlp_reference_gelu_and_its_derivative():
    """The tanh form of GELU stays within 5e-4 of its definition x Phi(x) (Phi the standard
    normal CDF, here through scipy's erf), has the limits 0 and x, and its derivative matches
    central differences."""
    import oracle.mlp as OM
    from scipy.special import erf

    z = np.linspace(-8.0, 8.0, 4001)
    exact = 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))
    assert np.abs(OM.gelu(z) - exact).max() < 5e-4
    assert OM.gelu(np.array([0.0]))[0] == 0.0
    assert abs(OM.gelu(np.array([30.0]))[0] - 30.0) < 1e-12 and abs(OM.gelu(np.array([-30.0]))[0]) < 1e-12
    h = 1e-6
    fd = (OM.gelu(z + h) - OM.gelu(z - h)) / (2 * h)
    assert np.abs(OM.gelu_grad(z) - fd).max() < 1e-8


# --------------------------------------------- L-BFGS local solver (Sec. 3.1)
@pytest.mark.parametrize("kind", [O.LOSS_HUBER, O.LOSS_L2])
def test_lbfgs_local_solve_reaches_the_argmin(kind):
    """Many L-BFGS iterations end at a stationary point of Eq. (9) (central differences of
    the objective, no Jacobian code), the minimiser a long Gauss-Newton run and an
    independent quasi-Newton routine also find."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    s, cfg, z, xbar, ybar, dual, _ = _local_case(5, kind)
    cfg.inner_steps = 300
    v0 = np.r_[xbar, ybar]
    v = O.local_solve_lbfgs(cfg, z, xbar, ybar, dual, v0)
    f = lambda u: O.local_objective(cfg, z, xbar, ybar, dual, u)
    g = np.zeros(9)
    for k in range(9):
        h = 1e-7 * max(1.0, abs(v[k]))
        vp, vm = v.copy(), v.copy()
        vp[k] += h
        vm[k] -= h
        g[k] = (f(vp) - f(vm)) / (2 * h)
    g0 = np.zeros(9)
    for k in range(9):
        h = 1e-7 * max(1.0, abs(v0[k]))
        vp, vm = v0.copy(), v0.copy()
        vp[k] += h
        vm[k] -= h
        g0[k] = (f(vp) - f(vm)) / (2 * h)
    assert np.linalg.norm(g) <= 1e-5 * np.linalg.norm(g0)
    gn = O.local_solve(cfg, z, xbar, ybar, dual, v0)
    assert np.abs(v - gn).max() <= 1e-6 * np.abs(gn).max()
    res = scipy_opt.minimize(f, v0, method="BFGS", options={"gtol": 1e-10, "maxiter": 20000})
    assert f(v) <= res.fun + 1e-9 * abs(res.fun)


def test_lbfgs_never_increases_the_local_objective():
    """Every accepted step satisfies the Armijo condition (or sits at rounding noise), so
    the objective after k iterations is non-increasing in k."""
    for seed in range(6):
        s, cfg, z, xbar, ybar, dual, _ = _local_case(seed, O.LOSS_HUBER)
        v0 = np.r_[xbar, ybar]
        prev = O.local_objective(cfg, z, xbar, ybar, dual, v0)
        for k in range(1, 12):
            cfg.inner_steps = k
            v = O.local_solve_lbfgs(cfg, z, xbar, ybar, dual, v0)
            cur = O.local_objective(cfg, z, xbar, ybar, dual, v)
            assert cur <= prev + 1e-12 * abs(prev)
            prev = cur


def test_lbfgs_and_gauss_newton_admm_share_the_fixed_point():
    """Both local solvers stop moving only at a stationary point of Eq. (9), so the two ADMM
    runs converge to the same limit (compared on gauge-free projections)."""
    sc = S.scene0(n_pts=40, n_cams=6, seed=8)
    runs = {}
    for solver in (O.SOLVER_GN, O.SOLVER_LBFGS):
        cfg = O.config_for(sc, local_solver=solver)
        st = O.State(sc)
        m = st.iterate(cfg, 1600)
        runs[solver] = (st, m)
    a, b = runs[O.SOLVER_GN][0], runs[O.SOLVER_LBFGS][0]
    assert abs(runs[0][1]["objective"] - runs[1][1]["objective"]) <= 1e-8 * runs[0][1]["objective"]
    cfg = O.config_for(sc)
    for o in range(0, sc.n_obs, 7):
        i, j = sc.pt_idx[o], sc.cam_idx[o]
        za, _ = O.project(cfg, a.pts[i], a.cams[j])
        zb, _ = O.project(cfg, b.pts[i], b.cams[j])
        assert np.abs(za - zb).max() <= 1e-5
