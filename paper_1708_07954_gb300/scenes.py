"""Seeded synthetic bundle-adjustment scenes (inputs only).

The paper evaluates on synthetic scenes (Sec. 4.1: cameras on an orbit aimed
at an area, random pose jitter, each point seen on a few consecutive frames)
and on real datasets that are not available here.  This module simulates such
scenes: ground-truth cameras and points, which camera sees which point, pixel
noise, outliers and a perturbed initial estimate.

It is the one module that both the CUDA path's tests/benchmarks and the CPU
oracle take inputs from, so it holds none of the method's arithmetic: no loss,
no local solve, no consensus, no dual update.  Cameras are built as look-at
rotation matrices and observations are made by projecting through those
matrices (a pinhole sensor simulation); the Euler angles
(alpha, beta, gamma) of the camera parameter vector are read off each matrix
assuming R = Rz(gamma) Ry(beta) Rx(alpha) (Sec. 2.1).

Camera parameter vector y_j = (alpha, beta, gamma, tx, ty, tz), point x_i in
R^3, pixel z = f * (Rx+t)_{1,2} / (Rx+t)_3 + (cx, cy).

Workloads (sizes, distributions):
  0  8 cameras on a radius-5 circle looking at the origin, 200 points in
     [-1,1]^3, all seen by all cameras (1,600 observations), sigma 1 px,
     Huber delta 2 px, FP64, 50 iterations.
  1  64 cameras on a ring (radius 15, heights jittered), 20,000 points in a
     10x10x2 slab, track lengths truncated-geometric on [2,20] with mean 8
     (~160k observations), sigma 0.5 px, Student's t nu 4, FP32 local solves.
  2  1,000 nadir cameras on a serpentine 25x40 flight grid at 150 m over
     500,000 points on a perturbed ground plane plus box structures, track
     lengths power-law on [2,50] with mean 8 (~4M observations), sigma 0.5 px,
     5% outliers uniform over the image, Huber delta 2 px, FP32 local solves.
  3  a batch of 256 independent scenes: cameras U{4..128}, points
     log-uniform on [100, 20000], tracks U{2..min(30,m)} consecutive ring
     cameras, workload-0 geometry and noise.
Initial estimates: Euler angles + N(0, 0.01^2) rad, each translation
component + N(0, (0.01 |t|)^2), each point component + N(0, (0.01 R)^2) with R
the radius of the point cloud's bounding sphere.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FOCAL, CX, CY, WIDTH, HEIGHT = 500.0, 320.0, 240.0, 640.0, 480.0

LOSS_L2, LOSS_HUBER, LOSS_STUDENT_T = 0, 1, 2
PREC_F64, PREC_F32 = 0, 1


@dataclasses.dataclass
class Scene:
    """One bundle-adjustment problem in caller order (observations unsorted)."""

    n_cams: int
    n_pts: int
    pt_idx: np.ndarray      # int32 [l]
    cam_idx: np.ndarray     # int32 [l]
    z: np.ndarray           # float64 [l, 2] observed pixels
    z_true: np.ndarray      # float64 [l, 2] noise-free projections of ground truth
    outlier: np.ndarray     # bool [l]
    cams_gt: np.ndarray     # float64 [m, 6]
    pts_gt: np.ndarray      # float64 [n, 3]
    cams0: np.ndarray       # float64 [m, 6] initial estimate
    pts0: np.ndarray        # float64 [n, 3] initial estimate
    focal: float = FOCAL
    cx: float = CX
    cy: float = CY
    loss: int = LOSS_HUBER
    loss_param: float = 2.0
    rho_x: float = 1.0
    rho_y: float = 1.0
    rho_angle: float = 0.0
    iters: int = 50
    precision: int = PREC_F64
    name: str = ""
    depth: float = 1.0      # median depth of the observations (ground truth)
    scene_off: np.ndarray | None = None  # batches: int64 [S+1] observation offsets
    cam_off: np.ndarray | None = None    # batches: int32 [S+1] camera offsets
    pt_off: np.ndarray | None = None     # batches: int32 [S+1] point offsets

    @property
    def n_obs(self) -> int:
        return int(self.pt_idx.shape[0])

    def clean_mask(self) -> np.ndarray:
        """Observations of points none of whose observations is an outlier."""
        bad = np.zeros(self.n_pts, dtype=bool)
        bad[self.pt_idx[self.outlier]] = True
        return ~bad[self.pt_idx]


# ---------------------------------------------------------------- sensor model
def look_at(centers: np.ndarray, targets: np.ndarray, up: np.ndarray) -> np.ndarray:
    """World-to-camera rotations with rows (right, down, forward); det = +1."""
    fwd = targets - centers
    fwd /= np.linalg.norm(fwd, axis=-1, keepdims=True)
    right = np.cross(fwd, np.broadcast_to(up, fwd.shape))
    right /= np.linalg.norm(right, axis=-1, keepdims=True)
    down = np.cross(fwd, right)
    return np.stack([right, down, fwd], axis=-2)


def euler_from_matrix(rot: np.ndarray) -> np.ndarray:
    """(alpha, beta, gamma) with rot = Rz(gamma) Ry(beta) Rx(alpha)."""
    beta = -np.arcsin(np.clip(rot[..., 2, 0], -1.0, 1.0))
    alpha = np.arctan2(rot[..., 2, 1], rot[..., 2, 2])
    gamma = np.arctan2(rot[..., 1, 0], rot[..., 0, 0])
    return np.stack([alpha, beta, gamma], axis=-1)


def _sense(rot, trans, pts, pt_idx, cam_idx, focal, cx, cy):
    pc = np.einsum("lab,lb->la", rot[cam_idx], pts[pt_idx]) + trans[cam_idx]
    if np.any(pc[:, 2] <= 0):
        raise RuntimeError("generator produced a point behind a camera")
    z = np.stack([focal * pc[:, 0] / pc[:, 2] + cx, focal * pc[:, 1] / pc[:, 2] + cy], axis=1)
    return z, float(np.median(pc[:, 2]))


def _finish(rng, rot, centers, pts, pt_idx, cam_idx, sigma, outlier_frac, name, shuffle=True):
    trans = -np.einsum("mab,mb->ma", rot, centers)
    cams_gt = np.concatenate([euler_from_matrix(rot), trans], axis=1)
    z_true, depth = _sense(rot, trans, pts, pt_idx, cam_idx, FOCAL, CX, CY)
    l = pt_idx.shape[0]
    z = z_true + rng.normal(0.0, sigma, size=(l, 2))
    outlier = np.zeros(l, dtype=bool)
    if outlier_frac > 0:
        outlier = rng.random(l) < outlier_frac
        k = int(outlier.sum())
        z[outlier] = np.stack([rng.uniform(0, WIDTH, k), rng.uniform(0, HEIGHT, k)], axis=1)
    if shuffle:
        perm = rng.permutation(l)
        pt_idx, cam_idx, z, z_true, outlier = pt_idx[perm], cam_idx[perm], z[perm], z_true[perm], outlier[perm]
    # initial estimate (perturbation scheme of workload 0)
    m, n = cams_gt.shape[0], pts.shape[0]
    cams0 = cams_gt.copy()
    cams0[:, :3] += rng.normal(0.0, 0.01, size=(m, 3))
    tn = np.linalg.norm(trans, axis=1, keepdims=True)
    cams0[:, 3:] += rng.normal(0.0, 1.0, size=(m, 3)) * (0.01 * tn)
    radius = float(np.max(np.linalg.norm(pts - pts.mean(axis=0), axis=1)))
    pts0 = pts + rng.normal(0.0, 0.01 * radius, size=(n, 3))
    return Scene(
        n_cams=m, n_pts=n,
        pt_idx=np.ascontiguousarray(pt_idx, dtype=np.int32),
        cam_idx=np.ascontiguousarray(cam_idx, dtype=np.int32),
        z=np.ascontiguousarray(z), z_true=np.ascontiguousarray(z_true), outlier=outlier,
        cams_gt=cams_gt, pts_gt=pts.copy(), cams0=cams0, pts0=pts0, name=name, depth=depth)


def _ring(rng, m, radius, height_sigma):
    theta = 2.0 * np.pi * np.arange(m) / m
    x = rng.normal(0.0, height_sigma, size=m) if height_sigma > 0 else np.zeros(m)
    centers = np.stack([x, radius * np.cos(theta), radius * np.sin(theta)], axis=1)
    rot = look_at(centers, np.zeros_like(centers), np.array([1.0, 0.0, 0.0]))
    return centers, rot


def _truncated_pmf_mean(kmin, kmax, weight_fn, target):
    """Bisection on the shape parameter so the pmf on [kmin,kmax] has the target mean."""
    ks = np.arange(kmin, kmax + 1, dtype=np.float64)
    lo, hi = 1e-6, 20.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        w = weight_fn(ks, mid)
        mean = float((ks * w).sum() / w.sum())
        if mean > target:
            lo = mid
        else:
            hi = mid
    w = weight_fn(ks, 0.5 * (lo + hi))
    return ks.astype(np.int64), w / w.sum()


def _consecutive_tracks(rng, m, lengths, wrap):
    """Each point is seen on L consecutive cameras (Sec. 4.1)."""
    n = lengths.shape[0]
    if wrap:
        start = rng.integers(0, m, size=n)
    else:
        start = rng.integers(0, m - lengths + 1)
    pt_idx = np.repeat(np.arange(n, dtype=np.int64), lengths)
    offs = np.arange(pt_idx.shape[0]) - np.repeat(np.cumsum(lengths) - lengths, lengths)
    cam = np.repeat(start, lengths) + offs
    if wrap:
        cam %= m
    return pt_idx, cam


# ---------------------------------------------------------------- workloads
def scene0(seed: int = 1000, n_pts: int = 200, n_cams: int = 8) -> Scene:
    rng = np.random.default_rng(seed)
    centers, rot = _ring(rng, n_cams, 5.0, 0.0)
    pts = rng.uniform(-1.0, 1.0, size=(n_pts, 3))
    pt_idx, cam_idx = np.meshgrid(np.arange(n_pts), np.arange(n_cams), indexing="ij")
    s = _finish(rng, rot, centers, pts, pt_idx.ravel(), cam_idx.ravel(), 1.0, 0.0, "ring8-cube200-dense")
    s.loss, s.loss_param, s.iters, s.precision = LOSS_HUBER, 2.0, 50, PREC_F64
    s.rho_x, s.rho_y, s.rho_angle = default_rho(s)
    return s


def scene1(seed: int = 1001, n_pts: int = 20000, n_cams: int = 64) -> Scene:
    rng = np.random.default_rng(seed)
    centers, rot = _ring(rng, n_cams, 15.0, 1.5)
    pts = np.stack([rng.uniform(-1, 1, n_pts), rng.uniform(-5, 5, n_pts), rng.uniform(-5, 5, n_pts)], axis=1)
    kmax = min(20, n_cams)
    ks, p = _truncated_pmf_mean(2, kmax, lambda k, a: np.exp(-a * (k - 2)), min(8.0, 0.5 * (2 + kmax)))
    lengths = rng.choice(ks, size=n_pts, p=p)
    pt_idx, cam_idx = _consecutive_tracks(rng, n_cams, lengths, wrap=True)
    s = _finish(rng, rot, centers, pts, pt_idx, cam_idx, 0.5, 0.0, f"ring{n_cams}-slab{n_pts}-geom")
    s.loss, s.loss_param, s.iters, s.precision = LOSS_STUDENT_T, 4.0, 200, PREC_F32
    s.rho_x, s.rho_y, s.rho_angle = default_rho(s)
    return s


def scene2(seed: int = 1002, n_pts: int = 500000, lanes: int = 25, stations: int = 40,
           outlier_frac: float = 0.05) -> Scene:
    rng = np.random.default_rng(seed)
    alt, step = 150.0, 2.5
    m = lanes * stations
    # serpentine flight path: lane k runs along +x or -x
    st = np.arange(stations, dtype=np.float64) * step
    xs = np.concatenate([st if k % 2 == 0 else st[::-1] for k in range(lanes)])
    ys = np.repeat(np.arange(lanes, dtype=np.float64) * step, stations)
    centers = np.stack([xs, ys, np.full(m, alt)], axis=1)
    centers[:, :2] += rng.normal(0.0, 0.2, size=(m, 2))
    centers[:, 2] += rng.normal(0.0, 1.0, size=m)
    # nadir-looking with small tilt jitter
    targets = centers.copy()
    targets[:, 2] = 0.0
    targets[:, :2] += rng.normal(0.0, 0.02 * alt, size=(m, 2))
    rot = look_at(centers, targets, np.array([0.0, 1.0, 0.0]))
    # track lengths: power law on [2,50], mean 8; consecutive cameras on the path
    ks, p = _truncated_pmf_mean(2, min(50, m), lambda k, a: k ** (-a), 8.0)
    lengths = rng.choice(ks, size=n_pts, p=p)
    pt_idx, cam_idx = _consecutive_tracks(rng, m, lengths, wrap=False)
    # point near the ground footprint of its track: a perturbed ground plane plus boxes
    first = np.cumsum(lengths) - lengths
    mid = cam_idx[first + lengths // 2]
    xy = centers[mid, :2] + rng.uniform(-30.0, 30.0, size=(n_pts, 2))
    zg = 1.5 * np.sin(xy[:, 0] / 17.0) * np.cos(xy[:, 1] / 23.0) + rng.normal(0.0, 0.2, n_pts)
    n_box = 60
    bc = np.stack([rng.uniform(xs.min(), xs.max(), n_box), rng.uniform(ys.min(), ys.max(), n_box)], axis=1)
    bh = rng.uniform(3.0, 25.0, n_box)
    bs = rng.uniform(4.0, 12.0, n_box)
    inside = np.abs(xy[:, None, :] - bc[None, :, :]).max(axis=2) < bs[None, :]
    roof = np.where(inside, bh[None, :], 0.0).max(axis=1)
    pts = np.concatenate([xy, (zg + roof)[:, None]], axis=1)
    s = _finish(rng, rot, centers, pts, pt_idx, cam_idx, 0.5, outlier_frac, f"grid{m}-ground{n_pts}-pow")
    s.loss, s.loss_param, s.iters, s.precision = LOSS_HUBER, 2.0, 300, PREC_F32
    s.rho_x, s.rho_y, s.rho_angle = default_rho(s)
    return s


def scene3(n_scenes: int = 256, seed0: int = 10000, max_pts: int = 20000) -> Scene:
    """Batch of independent uneven scenes, concatenated with offsets."""
    parts = []
    for k in range(n_scenes):
        rng = np.random.default_rng(seed0 + k)
        m = int(rng.integers(4, 129))
        n = int(round(math.exp(rng.uniform(math.log(100.0), math.log(max_pts)))))
        centers, rot = _ring(rng, m, 5.0, 0.0)
        pts = rng.uniform(-1.0, 1.0, size=(n, 3))
        lengths = rng.integers(2, min(30, m) + 1, size=n)
        pt_idx, cam_idx = _consecutive_tracks(rng, m, lengths, wrap=True)
        parts.append(_finish(rng, rot, centers, pts, pt_idx, cam_idx, 1.0, 0.0, f"batch{k}"))
    return concat_scenes(parts, name=f"batch{n_scenes}-ring-cube")


def concat_scenes(parts: list[Scene], name: str = "batch") -> Scene:
    co = np.cumsum([0] + [p.n_cams for p in parts]).astype(np.int32)
    po = np.cumsum([0] + [p.n_pts for p in parts]).astype(np.int32)
    oo = np.cumsum([0] + [p.n_obs for p in parts]).astype(np.int64)
    cat = lambda attr: np.concatenate([getattr(p, attr) for p in parts])
    s = Scene(
        n_cams=int(co[-1]), n_pts=int(po[-1]),
        pt_idx=np.concatenate([p.pt_idx + po[k] for k, p in enumerate(parts)]).astype(np.int32),
        cam_idx=np.concatenate([p.cam_idx + co[k] for k, p in enumerate(parts)]).astype(np.int32),
        z=cat("z"), z_true=cat("z_true"), outlier=cat("outlier"),
        cams_gt=cat("cams_gt"), pts_gt=cat("pts_gt"), cams0=cat("cams0"), pts0=cat("pts0"),
        name=name, scene_off=oo, cam_off=co, pt_off=po,
        depth=float(np.median([p.depth for p in parts])))
    s.loss, s.loss_param, s.iters, s.precision = LOSS_HUBER, 2.0, 50, PREC_F32
    s.rho_x, s.rho_y, s.rho_angle = default_rho(parts[0])
    return s


def default_rho(s: Scene, factor: float = 1.0) -> tuple[float, float, float]:
    """Penalties (rho_x, rho_y, rho_angle) scaled to the data term's curvature.

    The paper prints no penalty value (Thm. 1 asks for it to be large enough).
    One observation's misfit Hessian is ~2 (f/depth)^2 per unit of point
    coordinate or camera translation and ~2 f^2 per radian of camera angle;
    each penalty is `factor` times its block's curvature.  Factor 1 stays
    stable over 3,000 iterations of workload 2; 0.25 converges faster at first
    but diverges after ~1,000 iterations (in FP64 and FP32 alike).
    """
    lin = factor * 2.0 * (s.focal / max(s.depth, 1e-9)) ** 2
    ang = factor * 2.0 * s.focal ** 2
    return lin, lin, ang


WORKLOADS = {0: scene0, 1: scene1, 2: scene2, 3: scene3}


def make(workload: int, **kw) -> Scene:
    return WORKLOADS[workload](**kw)
