"""Second, independent statement of the two local solvers of Eq. (9) and of the block
solve of Eq. (14), step by step.

TEST INFRASTRUCTURE ONLY: used by ``tests/golden/make_local_steps.py`` and
``tests/golden/make_block_steps.py`` to write the step-wise golden vectors that pin
``ora_local_solve``, ``ora_local_solve_lbfgs`` and ``ora_block_solve`` over a fixed
number of steps.  It shares no code with ``dba_oracle.c`` and reaches
each quantity by another route:

- rotation (Sec. 2.1): built here as R3(gamma) R2(beta) R1(alpha) from the textbook
  single-axis matrices and checked against scipy's extrinsic "xyz" Euler angles;
- Jacobian of the pixel model (Eq. 1) and gradient of Eq. (9): complex-step
  differentiation (Squire and Trapp, SIAM Review 40, 1998), exact to rounding, instead
  of the oracle's chain rule;
- the damped Gauss-Newton system: numpy's LU solve instead of a Cholesky factorisation;
- L-BFGS (Nocedal and Wright, Numerical Optimization, Ch. 7): the inverse-Hessian
  approximation formed as a dense matrix by the BFGS product update
  H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T over the stored pairs, instead of
  the two-loop recursion;
- the block system of Eq. (14): the stacked Jacobian of all the block's pixels by complex
  steps of the whole block vector and dense products with the weights, instead of the
  oracle's per-observation 9 x 9 scatter into the block system.

The rules restated (the readings the oracle documents): Levenberg damping
lambda_0 = lm_lambda0 * mean diag H at the first step, divided by 10 after an accepted
step (clamped at lm_lambda_min) and multiplied by 10 after a rejected one; a step is
accepted when the trial point is in front of the camera and lowers Eq. (9), or when its
predicted decrease (lambda |d|^2 - g.d) / 2 is below kappa 2^-53 (|L| + 2 w |e| (|z1| + |z2|));
a linearisation point behind the camera contributes no misfit term.  L-BFGS runs in
u = sqrt(rho) (v - vbar), memory 4, H0 = (s.y / y.y) I (I before the first pair), steepest
descent when -H g is not a descent direction, backtracking from t = 1 with at most 10
halvings and Armijo constant 1e-4 (or the same rounding-noise rule on -t g.p), a pair kept
only when s.y > 0, and a failed line search ends the solve.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial.transform import Rotation

L2, HUBER, STUDENT_T = 0, 1, 2
U64 = 2.0 ** -53
H_CS = 1e-30  # complex-step size


def _rot(a, b, g):
    ca, sa, cb, sb, cg, sg = np.cos(a), np.sin(a), np.cos(b), np.sin(b), np.cos(g), np.sin(g)
    one, zero = ca ** 0, 0 * ca
    R1 = np.array([[one, zero, zero], [zero, ca, -sa], [zero, sa, ca]])
    R2 = np.array([[cb, zero, sb], [zero, one, zero], [-sb, zero, cb]])
    R3 = np.array([[cg, -sg, zero], [sg, cg, zero], [zero, zero, one]])
    return R3 @ R2 @ R1


def check_rotation(y):
    """The rotation above equals scipy's extrinsic x-y-z Euler angles (raises otherwise)."""
    R = _rot(*np.asarray(y[:3], float))
    Rs = Rotation.from_euler("xyz", np.asarray(y[:3], float)).as_matrix()
    if np.abs(R - Rs).max() > 1e-14:
        raise AssertionError("rotation convention mismatch")


def pixel(cfg, v):
    """z = f (R x + t)_{1,2} / (R x + t)_3 + (cx, cy) and the depth; v = (x, angles, t).
    Works on complex v (for the complex step)."""
    R = _rot(v[3], v[4], v[5])
    q = R @ v[:3] + v[6:9]
    return np.array([cfg["focal"] * q[0] / q[2] + cfg["cx"], cfg["focal"] * q[1] / q[2] + cfg["cy"]]), q[2]


def rho_vec(cfg):
    ra = cfg["rho_angle"] if cfg["rho_angle"] > 0 else cfg["rho_y"]
    return np.array([cfg["rho_x"]] * 3 + [ra] * 3 + [cfg["rho_y"]] * 3)


def misfit(cfg, s):
    p = cfg["loss_param"]
    if cfg["loss"] == HUBER:
        return s if np.real(s) <= p * p else 2 * p * np.sqrt(s) - p * p
    if cfg["loss"] == STUDENT_T:
        return p * np.log(1 + s / p)
    return s


def weight(cfg, s):
    """d misfit / d s, the IRLS weight."""
    p = cfg["loss_param"]
    if cfg["loss"] == HUBER:
        return 1.0 if s <= p * p else p / np.sqrt(s)
    if cfg["loss"] == STUDENT_T:
        return p / (p + s)
    return 1.0


def objective(cfg, c, v):
    """Eq. (9) at v: misfit + dual^T (v - vbar) + rho/2 |v - vbar|^2; +inf behind the camera."""
    zp, depth = pixel(cfg, v)
    if not np.real(depth) > cfg["eps_depth"]:
        return np.inf
    e = c["z"] - zp
    dv = v - c["vbar"]
    return misfit(cfg, e @ e) + c["dual"] @ dv + 0.5 * (rho_vec(cfg) * dv) @ dv


def jacobian_cs(cfg, v):
    J = np.zeros((2, 9))
    for k in range(9):
        vc = v.astype(complex)
        vc[k] += 1j * H_CS
        J[:, k] = np.imag(pixel(cfg, vc)[0]) / H_CS
    return J


def gradient_cs(cfg, c, v):
    g = np.zeros(9)
    for k in range(9):
        vc = v.astype(complex)
        vc[k] += 1j * H_CS
        g[k] = np.imag(objective(cfg, c, vc)) / H_CS
    return g


def _linearise(cfg, c, v):
    """Residual, weight, Jacobian at v; zero misfit terms behind the camera."""
    zp, depth = pixel(cfg, v)
    if not depth > cfg["eps_depth"]:
        return np.zeros(2), 0.0, np.zeros((2, 9))
    e = c["z"] - zp
    return e, weight(cfg, e @ e), jacobian_cs(cfg, v)


def gauss_newton(cfg, c, v0, steps):
    """The damped Gauss-Newton (Levenberg) local solve; returns the iterates v_0..v_steps and
    per step a code: 'A' accepted by comparison, 'T' accepted by the noise rule, 'R' rejected,
    with the margins of every decision."""
    rho = rho_vec(cfg)
    v = np.array(v0, float)
    L = objective(cfg, c, v)
    lam = None
    traj, codes, margins = [v.copy()], [], []
    for _ in range(steps):
        e, w, J = _linearise(cfg, c, v)
        g = -2 * w * J.T @ e + c["dual"] + rho * (v - c["vbar"])
        H = 2 * w * J.T @ J + np.diag(rho)
        if lam is None:
            lam = cfg["lm_lambda0"] * np.trace(H) / 9.0
        d = np.linalg.solve(H + lam * np.eye(9), -g)
        pred = 0.5 * (lam * d @ d - g @ d)
        noise = cfg["lm_model_tol"] * U64 * (abs(L) + 2 * w * np.sqrt(e @ e) * (abs(c["z"][0]) + abs(c["z"][1])))
        trust = np.isfinite(L) and cfg["lm_model_tol"] > 0 and pred <= noise
        Lt = objective(cfg, c, v + d)
        ok = np.isfinite(Lt) and (trust or Lt < L)
        margins.append({"pred_over_noise": float(pred / noise) if noise > 0 else np.inf,
                        "rel_change": float((Lt - L) / abs(L)) if np.isfinite(Lt) and np.isfinite(L) else np.inf})
        if ok:
            v = v + d
            L = Lt
            lam = max(lam / 10.0, cfg["lm_lambda_min"])
            codes.append("T" if trust else "A")
        else:
            lam = lam * 10.0
            codes.append("R")
        traj.append(v.copy())
    return traj, "".join(codes), margins


def lbfgs(cfg, c, v0, iters, memory=4, halvings=10, armijo=1e-4):
    """The L-BFGS local solve; returns the iterates, per iteration the number of line-search
    trials ('-' once a line search failed and the solve ended), and per iteration the smallest
    distance of its decisions from their thresholds (an Armijo comparison: relative to |L|; the
    noise rule: 1e-9 times the decimal log of the ratio)."""
    r = np.sqrt(rho_vec(cfg))
    v = np.array(v0, float)
    L = objective(cfg, c, v)

    def grad_u(vv):
        return gradient_cs(cfg, c, vv) / r

    def noise_at(vv):
        zp, depth = pixel(cfg, vv)
        if not depth > cfg["eps_depth"]:
            return 0.0
        e = c["z"] - zp
        return 2 * weight(cfg, e @ e) * np.sqrt(e @ e) * (abs(c["z"][0]) + abs(c["z"][1]))

    gu, noise = grad_u(v), noise_at(v)
    pairs = []
    traj, trials = [v.copy()], []
    margins = []  # per iteration: smallest relative distance of a line-search decision from its threshold
    done = False
    for _ in range(iters):
        if done:
            traj.append(v.copy())
            trials.append("-")
            continue
        if pairs:
            s_new, y_new = pairs[-1]
            Hinv = (s_new @ y_new) / (y_new @ y_new) * np.eye(9)
        else:
            Hinv = np.eye(9)
        for s, y in pairs:  # oldest to newest
            p_ = 1.0 / (s @ y)
            V = np.eye(9) - p_ * np.outer(y, s)
            Hinv = V.T @ Hinv @ V + p_ * np.outer(s, s)
        p = -Hinv @ gu
        gp = gu @ p
        if not gp < 0:
            p = -gu
            gp = -(gu @ gu)
        t, accepted, n_trials, margin = 1.0, False, 0, np.inf
        for _h in range(halvings + 1):
            n_trials += 1
            vt = v + t * p / r
            Lt = objective(cfg, c, vt)
            if np.isfinite(Lt):
                tol = cfg["lm_model_tol"] * U64 * (abs(L) + noise)
                trust = np.isfinite(L) and cfg["lm_model_tol"] > 0 and -t * gp <= tol
                margin = min(margin, abs(Lt - (L + armijo * t * gp)) / abs(L))
                if tol > 0:
                    margin = min(margin, abs(np.log10(-t * gp / tol)) * 1e-9)
                if trust or Lt <= L + armijo * t * gp:
                    accepted = True
                    break
            t *= 0.5
        margins.append(margin)
        if not accepted:
            done = True
            traj.append(v.copy())
            trials.append("-")
            continue
        gut = grad_u(vt)
        s, y = t * p, gut - gu
        if s @ y > 0:
            pairs.append((s, y))
            if len(pairs) > memory:
                pairs.pop(0)
        v, gu, L, noise = vt, gut, Lt, noise_at(vt)
        traj.append(v.copy())
        trials.append(str(n_trials))
    return traj, trials, margins


# ---------------------------------------------------------------------------------------
# The block subproblem of Eq. (14) (Sec. 3.1.4), step by step.
#
# A block holds np point copies X and nc camera copies Y; its parameter vector is
# v = (X_1 .. X_np, Y_1 .. Y_nc) of length n = 3 np + 6 nc.  The second statement reaches
# the damped Gauss-Newton system by another route than the oracle's per-observation
# scatter: the stacked pixel residual of all the block's observations is differentiated
# column by column with complex steps of the WHOLE vector v (an observation that does not
# depend on a column gets an exactly zero derivative), H and g are dense products of that
# stacked Jacobian with the IRLS weights, and (H + lambda I) d = -g is solved by numpy LU.
# The rules are those of the local solve above, over the block: lambda_0 = lm_lambda0 *
# mean diag H over all n unknowns, the noise bound summed over the observations in front
# of their cameras, and Eq. (14) +inf when any observation of a trial is behind its camera.
# ---------------------------------------------------------------------------------------


def _block_unpack(blk, v):
    np_ = len(blk["xbar"]) // 3
    return v[:3 * np_].reshape(np_, 3), v[3 * np_:].reshape(-1, 6)


def block_pixels(cfg, blk, v):
    """Predicted pixels [no, 2] and depths [no] of the block's observations at v."""
    X, Y = _block_unpack(blk, v)
    zs, ds = [], []
    for lp, lc in zip(blk["opl"], blk["ocl"]):
        zp, depth = pixel(cfg, np.concatenate([X[lp], Y[lc]]))
        zs.append(zp)
        ds.append(depth)
    return np.array(zs), np.array(ds)


def block_rho(cfg, blk):
    """The penalty of every unknown of v: rho_x for point coordinates, the camera penalty
    (angles, translation) for camera components."""
    np_, nc = len(blk["xbar"]) // 3, len(blk["ybar"]) // 6
    r = rho_vec(cfg)
    return np.concatenate([np.tile(r[:3], np_), np.tile(r[3:], nc)])


def block_objective(cfg, blk, v):
    """Eq. (14) at v: the misfits of the block's observations plus, per copy, dual^T (copy -
    consensus) + rho/2 |copy - consensus|^2; +inf when any observation is behind its camera."""
    zp, depth = block_pixels(cfg, blk, v)
    if not np.all(np.real(depth) > cfg["eps_depth"]):
        return np.inf
    e = np.asarray(blk["z"]).reshape(-1, 2) - zp
    vbar = np.concatenate([blk["xbar"], blk["ybar"]])
    dual = np.concatenate([blk["rx"], blk["sy"]])
    dv = v - vbar
    return sum(misfit(cfg, ek @ ek) for ek in e) + dual @ dv + 0.5 * (block_rho(cfg, blk) * dv) @ dv


def block_jacobian_cs(cfg, blk, v):
    """d (stacked predicted pixels) / d v, [2 no, n], by complex steps of the whole vector."""
    n = len(v)
    J = np.zeros((2 * len(blk["opl"]), n))
    for k in range(n):
        vc = v.astype(complex)
        vc[k] += 1j * H_CS
        J[:, k] = np.imag(block_pixels(cfg, blk, vc)[0]).ravel() / H_CS
    return J


def block_gauss_newton(cfg, blk, v0, steps):
    """The damped Gauss-Newton (Levenberg) solve of Eq. (14); returns the iterates, the step
    codes ('A', 'T', 'R' as in gauss_newton) and the margins of every decision."""
    rho = block_rho(cfg, blk)
    vbar = np.concatenate([blk["xbar"], blk["ybar"]])
    dual = np.concatenate([blk["rx"], blk["sy"]])
    z = np.asarray(blk["z"], float).reshape(-1, 2)
    n = len(vbar)
    v = np.array(v0, float)
    L = block_objective(cfg, blk, v)
    lam = None
    traj, codes, margins = [v.copy()], [], []
    for _ in range(steps):
        zp, depth = block_pixels(cfg, blk, v)
        front = depth > cfg["eps_depth"]  # a linearisation point behind its camera adds no misfit term
        e = np.where(front[:, None], z - zp, 0.0)
        s = np.sum(e * e, axis=1)
        w = np.array([weight(cfg, sk) if f else 0.0 for sk, f in zip(s, front)])
        J = block_jacobian_cs(cfg, blk, v)
        w2 = np.repeat(2.0 * w, 2)
        g = -J.T @ (w2 * e.ravel()) + dual + rho * (v - vbar)
        H = J.T @ (w2[:, None] * J) + np.diag(rho)
        if lam is None:
            lam = cfg["lm_lambda0"] * np.trace(H) / n
        d = np.linalg.solve(H + lam * np.eye(n), -g)
        pred = 0.5 * (lam * d @ d - g @ d)
        noise = cfg["lm_model_tol"] * U64 * (abs(L) + np.sum(2 * w * np.sqrt(s) * np.abs(z).sum(axis=1)))
        trust = np.isfinite(L) and cfg["lm_model_tol"] > 0 and pred <= noise
        Lt = block_objective(cfg, blk, v + d)
        ok = np.isfinite(Lt) and (trust or Lt < L)
        margins.append({"pred_over_noise": float(pred / noise) if noise > 0 else np.inf,
                        "rel_change": float((Lt - L) / abs(L)) if np.isfinite(Lt) and np.isfinite(L) else np.inf,
                        "pred": float(pred)})
        if ok:
            v = v + d
            L = Lt
            lam = max(lam / 10.0, cfg["lm_lambda_min"])
            codes.append("T" if trust else "A")
        else:
            lam = lam * 10.0
            codes.append("R")
        traj.append(v.copy())
    return traj, "".join(codes), margins


# ---------------------------------------------------------------------------------------
# One consensus ADMM iteration (Sec. 3.1, Eqs. 9-13) over all observations.
#
# The local solves are gauss_newton above, one per observation, each warm-started at its
# copy with the consensus and dual of the previous iteration.  The consensus of a point
# (likewise a camera) is reached as the minimiser of its part of the augmented Lagrangian,
#   sum_j  r_ij^T (x_ij - x) + rho/2 |x_ij - x|^2,
# by a least-squares solve over the stacked rows sqrt(rho) (x - (x_ij + r_ij / rho)) of all
# its copies, not by averaging; an unobserved point or camera keeps its value.  The duals
# then ascend by rho (copy - new consensus).
# ---------------------------------------------------------------------------------------


def _consensus(idx, count, values, weights, old):
    out = np.array(old, float)
    for i in range(count):
        rows = np.flatnonzero(idx == i)
        if len(rows) == 0:
            continue
        k = values.shape[1]
        A = np.kron(np.ones((len(rows), 1)), np.diag(np.sqrt(weights)))
        b = (values[rows] * np.sqrt(weights)).ravel()
        out[i] = np.linalg.lstsq(A, b, rcond=None)[0].reshape(k)
    return out


def admm_iteration(cfg, pt_idx, cam_idx, z, copies, duals, cams, pts, steps, solver="gn"):
    """One iteration with the Gauss-Newton ("gn") or L-BFGS ("lbfgs") local solve of `steps`
    steps / iterations; returns the new (copies, duals, cams, pts) and the codes of every
    local solve with their margins (for the golden writer's cleanliness check)."""
    rho = rho_vec(cfg)
    copies, duals = np.array(copies, float), np.array(duals, float)
    codes, margins = [], []
    for o in range(len(pt_idx)):
        c = {"z": np.asarray(z[o], float), "vbar": np.r_[pts[pt_idx[o]], cams[cam_idx[o]]], "dual": duals[o]}
        if solver == "lbfgs":
            traj, trials, marg = lbfgs(cfg, c, copies[o], steps)
            code = ",".join(trials)
        else:
            traj, code, marg = gauss_newton(cfg, c, copies[o], steps)
        copies[o] = traj[-1]
        codes.append(code)
        margins.append(marg)
    target = copies + duals / rho
    pts_new = _consensus(np.asarray(pt_idx), len(pts), target[:, :3], rho[:3], pts)
    cams_new = _consensus(np.asarray(cam_idx), len(cams), target[:, 3:], rho[3:], cams)
    consensus = np.concatenate([pts_new[pt_idx], cams_new[cam_idx]], axis=1)
    duals = duals + rho * (copies - consensus)
    return copies, duals, cams_new, pts_new, codes, margins


def block_admm_iteration(cfg, layout, z, pcopies, pduals, ccopies, cduals, cams, pts, steps):
    """One consensus ADMM iteration with block subproblems (Sec. 3.1.4, Eq. 14): every block
    solved by block_gauss_newton from its copies, each point's (camera's) consensus the
    least-squares minimiser over its copies, one per block that holds it, then the duals of
    every copy ascend by rho (copy - new consensus).  layout carries the block arrays
    (obs_off, blk_obs, obs_lp, obs_lc, pc_off, pc_pt, cc_off, cc_cam); returns the new
    (pcopies, pduals, ccopies, cduals, cams, pts) and every block's step codes."""
    rho = rho_vec(cfg)
    pcopies, pduals = np.array(pcopies, float), np.array(pduals, float)
    ccopies, cduals = np.array(ccopies, float), np.array(cduals, float)
    z = np.asarray(z, float)
    codes = []
    for b in range(len(layout["obs_off"]) - 1):
        o0, o1 = layout["obs_off"][b], layout["obs_off"][b + 1]
        p0, p1 = layout["pc_off"][b], layout["pc_off"][b + 1]
        c0, c1 = layout["cc_off"][b], layout["cc_off"][b + 1]
        blk = {"opl": list(layout["obs_lp"][o0:o1]), "ocl": list(layout["obs_lc"][o0:o1]),
               "z": z[np.asarray(layout["blk_obs"][o0:o1])].ravel(),
               "xbar": pts[np.asarray(layout["pc_pt"][p0:p1])].ravel(),
               "ybar": cams[np.asarray(layout["cc_cam"][c0:c1])].ravel(),
               "rx": pduals[p0:p1].ravel(), "sy": cduals[c0:c1].ravel()}
        v0 = np.concatenate([pcopies[p0:p1].ravel(), ccopies[c0:c1].ravel()])
        traj, code, _ = block_gauss_newton(cfg, blk, v0, steps)
        pcopies[p0:p1] = traj[-1][:3 * (p1 - p0)].reshape(-1, 3)
        ccopies[c0:c1] = traj[-1][3 * (p1 - p0):].reshape(-1, 6)
        codes.append(code)
    pc_pt, cc_cam = np.asarray(layout["pc_pt"]), np.asarray(layout["cc_cam"])
    pts_new = _consensus(pc_pt, len(pts), pcopies + pduals / rho[:3], rho[:3], pts)
    cams_new = _consensus(cc_cam, len(cams), ccopies + cduals / rho[3:], rho[3:], cams)
    pduals = pduals + rho[:3] * (pcopies - pts_new[pc_pt])
    cduals = cduals + rho[3:] * (ccopies - cams_new[cc_cam])
    return pcopies, pduals, ccopies, cduals, cams_new, pts_new, codes
