"""Learned warm start: the library's FP32 training kernels and BF16 tensor-core
(tcgen05) inference against the FP64 numpy reference in oracle/mlp.py, and the
warm start inside ADMM iterations."""
import os

import numpy as np
import pytest

import oracle as O
import oracle.mlp as OM
from paper_1708_07954_gb300 import build, dba, warmstart
from paper_1708_07954_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dba.load()


def _dev(torch, a):
    x = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    torch.cuda.synchronize()
    return x


def _random_net(seed=3):
    rng = np.random.default_rng(seed)
    mlp = dba.Mlp(seed)
    p = mlp.get_params().astype(np.float64)
    q = OM.unpack(p)
    p[OM.N_TRAINABLE:OM.N_TRAINABLE + OM.N_IN] = rng.normal(0, 0.5, OM.N_IN)            # input mean
    p[OM.N_TRAINABLE + OM.N_IN:OM.N_TRAINABLE + 2 * OM.N_IN] = rng.uniform(0.5, 2, OM.N_IN)  # input std
    p[OM.N_TRAINABLE + 2 * OM.N_IN:] = rng.uniform(0.5, 2, OM.N_OUT)                        # target scale
    mlp.set_params(p.astype(np.float32))
    del q
    return mlp, mlp.get_params().astype(np.float64)


def test_training_gradient_matches_fp64_reference():
    import torch

    mlp, p = _random_net()
    rng = np.random.default_rng(4)
    f = rng.normal(0, 1.5, (67, OM.N_IN))
    t = rng.normal(0, 1.0, (67, OM.N_OUT))
    fd, td = _dev(torch, f), _dev(torch, t)  # keep the buffers alive across the call
    loss, g = mlp.loss_grad(fd.data_ptr(), td.data_ptr(), 67)
    lo, go = OM.loss_and_grad(p, f.astype(np.float32), t.astype(np.float32))
    assert abs(loss - lo) <= 1e-5 * lo
    assert np.abs(g - go).max() <= 1e-4 * np.abs(go).max()


def _bf16(x):
    """Round to bfloat16 (nearest even), as the tensor-core operands are."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def test_tensor_core_inference_matches_reference():
    """tcgen05 BF16 x BF16 -> FP32: the reference rounds operands and hidden activations to
    BF16 at the same points; 300 rows span three 128-row tiles with a ragged tail."""
    import torch

    mlp, p = _random_net(5)
    rng = np.random.default_rng(6)
    f = rng.normal(0, 1.5, (300, OM.N_IN)).astype(np.float32)
    out = torch.zeros((300, OM.N_OUT), dtype=torch.float32, device="cuda")
    fd = _dev(torch, f)
    mlp.predict(fd.data_ptr(), 300, out.data_ptr())
    y = out.cpu().numpy().astype(np.float64)
    q = OM.unpack(p)
    x = _bf16((f - q["in_mean"]) / q["in_std"])
    h = x
    for k in (1, 2, 3):
        h = _bf16(OM.gelu(h @ _bf16(q[f"W{k}"]).T + q[f"b{k}"]))
    ref = h @ _bf16(q["W4"]).T + q["b4"]
    assert np.abs(y - ref).max() <= 2e-2 * max(1.0, np.abs(ref).max())
    # and close to the unrounded FP64 network
    full, _ = OM.forward(p, f)
    assert np.abs(y - full).max() <= 0.1 * max(1.0, np.abs(full).max())


def test_harvest_and_training_reduce_the_loss():
    import torch

    sc = S.scene1(n_pts=3000, n_cams=32, seed=2009)
    feats, targs = warmstart.harvest(sc, samples=20000, target_steps=10, iters=(0, 2, 8))
    assert feats.shape[1] == OM.N_IN and targs.shape[1] == OM.N_OUT and feats.shape[0] > 10000
    assert torch.isfinite(feats).all() and torch.isfinite(targs).all()
    mlp, hist = warmstart.train(feats, targs, epochs=6, batch=1024)
    assert hist[-1] < 0.8 * hist[0], hist


def test_warm_start_keeps_the_method_correct():
    """The local solve keeps a learned start only when it lowers Eq. (9), so any network
    leaves the ADMM limit unchanged: an untrained one ends within the FP32 tolerance."""
    sc = S.scene1(n_pts=2000, n_cams=32, seed=77)
    mlp, _ = _random_net(8)
    with dba.Solver(sc) as a, dba.Solver(sc) as b:
        b.set_warm_start(mlp)
        ma = a.iterate(120)
        mb = b.iterate(120)
        assert abs(ma["rmse_obs"] - mb["rmse_obs"]) <= 1e-3
        assert abs(ma["rmse_gt"] - mb["rmse_gt"]) <= 1e-3
        prof = b.profile(3)
        assert "mlp_warm_start" in prof


@pytest.mark.skipif(not os.path.exists(warmstart.WEIGHTS), reason="trained weights not present")
def test_trained_warm_start_gain_is_reported():
    """Held-out scene (workload-2 geometry, evaluation seed): iterations to 0.5 px with one
    Gauss-Newton step per local solve, plain vs learned start, beside five plain steps."""
    sc = S.scene2(n_pts=60000)
    mlp = warmstart.load()
    res = {}
    for name, steps, warm in (("plain1", 1, False), ("learned1", 1, True), ("plain5", 5, False)):
        with dba.Solver(sc, inner_steps=steps) as s:
            if warm:
                s.set_warm_start(mlp)
            m = s.iterate_until(400, 0.5)
            res[name] = (m["iters_done"], m["seconds"], m["rmse_gt"])
    print("time to 0.5 px (iterations, device s, rmse):", res)
    # the learned start reaches the target in well under the iterations of the plain one, and
    # one Gauss-Newton step from it needs nearly as few iterations as five plain steps (the
    # ADMM consensus, not the local accuracy, then bounds the count)
    assert res["plain1"][2] <= 0.5 and res["learned1"][2] <= 0.5 and res["plain5"][2] <= 0.5
    assert res["learned1"][0] <= 0.6 * res["plain1"][0]
    assert res["learned1"][0] <= 1.2 * res["plain5"][0]


def test_harvested_features_and_targets_match_a_cpu_restatement():
    """dba_mlp_harvest against a restatement from the paper's state (dba_get_state,
    dba_get_params) with the oracle: for sampled observations (internal order, every 7th)
    the features are the local problem of Eq. (9) at the current copy v (residual z - f(v),
    the square root of the IRLS weight, the Jacobian rows over r = sqrt(rho), r (v - vbar +
    dual / rho), two zeros), and the target is r (v* - v) for v* the oracle's local solve of
    20 damped Gauss-Newton steps from v.  FP64 context; features and targets are FP32."""
    import torch

    sc = S.scene1(n_pts=1500, n_cams=24, seed=81)
    stride, steps = 7, 20
    with dba.Solver(sc, precision=dba.DBA_PREC_F64) as s:
        s.iterate(3, stats=False)
        copies, duals = s.state()
        cams, pts = s.params()
        cap = (sc.n_obs + stride - 1) // stride
        f = torch.zeros((cap, OM.N_IN), dtype=torch.float32, device="cuda")
        t = torch.zeros((cap, OM.N_OUT), dtype=torch.float32, device="cuda")
        n = s.harvest(stride, steps, f.data_ptr(), t.data_ptr(), cap)
        torch.cuda.synchronize()
        c = s.cfg
        tile = s.layout()["tile_obs"]
    assert n == cap
    feats, targs = f.cpu().numpy().astype(np.float64), t.cpu().numpy().astype(np.float64)
    perm = dba.dba_build_layout(sc.n_cams, sc.n_pts, sc.pt_idx, sc.cam_idx, tile)["perm"]
    cfg = O.config(focal=c.focal, cx=c.cx, cy=c.cy, loss=c.loss, loss_param=c.loss_param, rho_x=c.rho_x,
                   rho_y=c.rho_y, rho_angle=c.rho_angle, inner_steps=steps, lm_lambda0=c.lm_lambda0,
                   lm_lambda_min=c.lm_lambda_min, eps_depth=c.eps_depth, lm_model_tol=c.lm_model_tol)
    rho = np.r_[[c.rho_x] * 3, [c.rho_angle if c.rho_angle > 0 else c.rho_y] * 3, [c.rho_y] * 3]
    r = np.sqrt(rho)
    want_f = np.zeros((n, OM.N_IN))
    want_t = np.zeros((n, OM.N_OUT))
    for k in range(n):
        o = perm[k * stride]
        i, j = sc.pt_idx[o], sc.cam_idx[o]
        v, vbar = copies[o], np.r_[pts[i], cams[j]]
        zp, depth = O.project(cfg, v[:3], v[3:])
        assert depth > cfg.eps_depth
        e = sc.z[o] - zp
        J = O.jacobian(cfg, v[:3], v[3:])
        want_f[k, :2] = e
        want_f[k, 2] = np.sqrt(O.weight(cfg.loss, cfg.loss_param, e @ e))
        want_f[k, 3:12] = J[0] / r
        want_f[k, 12:21] = J[1] / r
        want_f[k, 21:30] = r * (v - vbar + duals[o] / rho)
        vs = O.local_solve(cfg, sc.z[o], vbar[:3], vbar[3:], duals[o], v)
        want_t[k, :9] = r * (vs - v)
    # FP32 outputs: per column, a few FP32 ulps of the column's scale
    fscale = np.maximum(np.abs(want_f).max(axis=0), 1e-30)
    assert np.all(np.abs(feats - want_f).max(axis=0) <= 1e-6 * fscale)
    tscale = np.maximum(np.abs(want_t).max(axis=0), 1e-30)
    assert np.all(np.abs(targs - want_t).max(axis=0) <= 1e-5 * tscale)
    assert np.all(targs[:, 9:] == 0) and np.all(feats[:, 30:] == 0)
