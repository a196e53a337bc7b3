"""Python access to the plain FP64 CPU oracle (``dba_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the product path never
does.  The oracle shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dba_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libdba_oracle.so")
_lock = threading.Lock()
_lib = None

LOSS_L2, LOSS_HUBER, LOSS_STUDENT_T = 0, 1, 2


class Config(ctypes.Structure):
    _fields_ = [
        ("focal", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
        ("loss", ctypes.c_int), ("loss_param", ctypes.c_double),
        ("rho_x", ctypes.c_double), ("rho_y", ctypes.c_double), ("rho_angle", ctypes.c_double),
        ("inner_steps", ctypes.c_int), ("lm_lambda0", ctypes.c_double),
        ("lm_lambda_min", ctypes.c_double), ("eps_depth", ctypes.c_double),
        ("lm_model_tol", ctypes.c_double), ("local_solver", ctypes.c_int),
    ]


class Metrics(ctypes.Structure):
    _fields_ = [
        ("rmse_obs", ctypes.c_double), ("rmse_gt", ctypes.c_double),
        ("objective", ctypes.c_double), ("primal_res", ctypes.c_double),
        ("dual_res", ctypes.c_double), ("n_invalid", ctypes.c_long),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available, no fast-math, no FP contraction)."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "dba_oracle.h"))
        ):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        cfgp = ctypes.POINTER(Config)
        L.ora_rotation.argtypes = [dp, dp]
        L.ora_project.argtypes = [cfgp, dp, dp, dp]
        L.ora_project.restype = ctypes.c_double
        L.ora_jacobian.argtypes = [cfgp, dp, dp, dp]
        L.ora_loss.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.ora_loss.restype = ctypes.c_double
        L.ora_weight.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.ora_weight.restype = ctypes.c_double
        L.ora_local_objective.argtypes = [cfgp, dp, dp, dp, dp, dp]
        L.ora_local_objective.restype = ctypes.c_double
        L.ora_local_solve.argtypes = [cfgp, dp, dp, dp, dp, dp]
        L.ora_local_solve_lbfgs.argtypes = [cfgp, dp, dp, dp, dp, dp]
        L.ora_chol_solve.argtypes = [ctypes.c_int, dp, dp, dp]
        L.ora_chol_solve.restype = ctypes.c_int
        L.ora_admm_init.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_long, ip, ip, dp, dp, dp, dp]
        L.ora_admm_iterate.argtypes = [cfgp, ctypes.c_int, ctypes.c_int, ctypes.c_long, ip, ip, dp, dp,
                                       dp, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(Metrics)]
        L.ora_admm_iterate.restype = ctypes.c_int
        L.ora_eval.argtypes = [cfgp, ctypes.c_int, ctypes.c_int, ctypes.c_long, ip, ip, dp, dp, dp, dp,
                               dp, dp, dp, ctypes.POINTER(Metrics)]
        L.ora_dense_lm.argtypes = [cfgp, ctypes.c_int, ctypes.c_int, ctypes.c_long, ip, ip, dp, dp, dp,
                                   ctypes.c_int, dp]
        L.ora_dense_lm.restype = ctypes.c_int
        lp = ctypes.POINTER(ctypes.c_long)
        L.ora_block_objective.argtypes = [cfgp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip, dp, dp, dp,
                                          dp, dp, dp, dp]
        L.ora_block_objective.restype = ctypes.c_double
        L.ora_block_solve.argtypes = [cfgp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip, dp, dp, dp, dp,
                                      dp, dp, dp]
        L.ora_block_iterate.argtypes = [cfgp, ctypes.c_int, ctypes.c_int, ctypes.c_long, ip, ip, dp, dp,
                                        ctypes.c_long, lp, lp, ip, ip, lp, ip, lp, ip, dp, dp, dp, dp, dp, dp,
                                        ctypes.c_int, ctypes.c_int, ctypes.POINTER(Metrics)]
        L.ora_block_iterate.restype = ctypes.c_int
        _lib = L
    return _lib


def _d(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _l(a):
    assert a.dtype == np.int64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_long))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


SOLVER_GN, SOLVER_LBFGS = 0, 1


def config(focal=500.0, cx=320.0, cy=240.0, loss=LOSS_HUBER, loss_param=2.0, rho_x=1.0, rho_y=1.0,
           rho_angle=0.0, inner_steps=5, lm_lambda0=1e-3, lm_lambda_min=1e-12, eps_depth=1e-6,
           lm_model_tol=16.0, local_solver=SOLVER_GN) -> Config:
    return Config(focal, cx, cy, loss, loss_param, rho_x, rho_y, rho_angle, inner_steps, lm_lambda0,
                  lm_lambda_min, eps_depth, lm_model_tol, local_solver)


def config_for(scene, **overrides) -> Config:
    kw = dict(focal=scene.focal, cx=scene.cx, cy=scene.cy, loss=scene.loss, loss_param=scene.loss_param,
              rho_x=scene.rho_x, rho_y=scene.rho_y, rho_angle=getattr(scene, "rho_angle", 0.0))
    kw.update(overrides)
    return config(**kw)


def rotation(y):
    R = np.zeros(9)
    lib().ora_rotation(_d(_f64(y)), _d(R))
    return R.reshape(3, 3)


def project(cfg, x, y):
    zp = np.zeros(2)
    depth = lib().ora_project(ctypes.byref(cfg), _d(_f64(x)), _d(_f64(y)), _d(zp))
    return zp, depth


def jacobian(cfg, x, y):
    J = np.zeros(18)
    lib().ora_jacobian(ctypes.byref(cfg), _d(_f64(x)), _d(_f64(y)), _d(J))
    return J.reshape(2, 9)


def loss(kind, param, s):
    return lib().ora_loss(kind, param, float(s))


def weight(kind, param, s):
    return lib().ora_weight(kind, param, float(s))


def local_objective(cfg, z, xbar, ybar, dual, v):
    return lib().ora_local_objective(ctypes.byref(cfg), _d(_f64(z)), _d(_f64(xbar)), _d(_f64(ybar)),
                                     _d(_f64(dual)), _d(_f64(v)))


def local_solve(cfg, z, xbar, ybar, dual, v0):
    v = _f64(v0).copy()
    lib().ora_local_solve(ctypes.byref(cfg), _d(_f64(z)), _d(_f64(xbar)), _d(_f64(ybar)),
                          _d(_f64(dual)), _d(v))
    return v


def local_solve_lbfgs(cfg, z, xbar, ybar, dual, v0):
    v = _f64(v0).copy()
    lib().ora_local_solve_lbfgs(ctypes.byref(cfg), _d(_f64(z)), _d(_f64(xbar)), _d(_f64(ybar)),
                                _d(_f64(dual)), _d(v))
    return v


def chol_solve(A, b):
    A = _f64(A)
    n = A.shape[0]
    x = np.zeros(n)
    rc = lib().ora_chol_solve(n, _d(A), _d(_f64(b)), _d(x))
    if rc != 0:
        raise np.linalg.LinAlgError("not positive definite")
    return x


class State:
    """ADMM state in caller order: copies/duals [l, 9], cams [m, 6], pts [n, 3]."""

    def __init__(self, scene, cams=None, pts=None):
        self.scene = scene
        self.cams = _f64(scene.cams0 if cams is None else cams).copy()
        self.pts = _f64(scene.pts0 if pts is None else pts).copy()
        l = scene.n_obs
        self.copies = np.zeros((l, 9))
        self.duals = np.zeros((l, 9))
        lib().ora_admm_init(scene.n_cams, scene.n_pts, l, _i(scene.pt_idx), _i(scene.cam_idx),
                            _d(self.cams), _d(self.pts), _d(self.copies), _d(self.duals))
        self.k = 0

    def clone(self):
        o = object.__new__(State)
        o.scene = self.scene
        o.cams, o.pts = self.cams.copy(), self.pts.copy()
        o.copies, o.duals, o.k = self.copies.copy(), self.duals.copy(), self.k
        return o

    def iterate(self, cfg, iters, nthreads=0, with_gt=True):
        s = self.scene
        m = Metrics()
        zt = _f64(s.z_true) if with_gt else None
        rc = lib().ora_admm_iterate(ctypes.byref(cfg), s.n_cams, s.n_pts, s.n_obs, _i(s.pt_idx),
                                    _i(s.cam_idx), _d(_f64(s.z)), _d(zt), _d(self.copies),
                                    _d(self.duals), _d(self.cams), _d(self.pts), iters, nthreads,
                                    ctypes.byref(m))
        if rc != 0:
            raise ValueError("oracle rejected the scene")
        self.k += iters
        return m.as_dict()

    def metrics(self, cfg, cams_prev=None, pts_prev=None, with_gt=True):
        s = self.scene
        m = Metrics()
        zt = _f64(s.z_true) if with_gt else None
        lib().ora_eval(ctypes.byref(cfg), s.n_cams, s.n_pts, s.n_obs, _i(s.pt_idx), _i(s.cam_idx),
                       _d(_f64(s.z)), _d(zt), _d(self.copies), _d(self.cams), _d(self.pts),
                       _d(cams_prev), _d(pts_prev), ctypes.byref(m))
        return m.as_dict()


def dense_lm(cfg, scene, cams=None, pts=None, max_iters=200):
    cams = _f64(scene.cams0 if cams is None else cams).copy()
    pts = _f64(scene.pts0 if pts is None else pts).copy()
    obj = ctypes.c_double(0.0)
    it = lib().ora_dense_lm(ctypes.byref(cfg), scene.n_cams, scene.n_pts, scene.n_obs, _i(scene.pt_idx),
                            _i(scene.cam_idx), _d(_f64(scene.z)), _d(cams), _d(pts), max_iters,
                            ctypes.byref(obj))
    if it < 0:
        raise ValueError("dense LM failed")
    return cams, pts, obj.value, it


# ------------------------------------------------ generalized block step, Eq. (14)
class BlockLayout:
    """Blocks of the generalized step (Sec. 3.1.4, Eq. 14) under this reading: points
    ranked by (smallest observing camera index, point index) and cut into groups of
    `pi` consecutive ranks; cameras cut into groups of `kappa` consecutive indices; one
    block per (point group, camera group) pair holding at least one observation.
    Blocks run in (point group, camera group) order; inside a block the point copies
    follow rank, the camera copies index, the observations (local point, local camera).
    """

    def __init__(self, scene, pi, kappa):
        if pi < 1 or kappa < 1:
            raise ValueError("pi and kappa must be >= 1")
        pt = np.asarray(scene.pt_idx, np.int64)
        cam = np.asarray(scene.cam_idx, np.int64)
        n, m = scene.n_pts, scene.n_cams
        first = np.full(n, np.iinfo(np.int64).max)
        np.minimum.at(first, pt, cam)
        order = np.lexsort((np.arange(n), first))
        rank = np.empty(n, np.int64)
        rank[order] = np.arange(n)
        pg, cg = rank[pt] // pi, cam // kappa
        n_cg = (m + kappa - 1) // kappa
        bkey = pg * n_cg + cg
        uniq_b, blk = np.unique(bkey, return_inverse=True)
        self.n_blocks = len(uniq_b)
        # observations in block order, then (point rank, camera)
        self.blk_obs = np.lexsort((cam, rank[pt], blk)).astype(np.int64)
        b_sorted = blk[self.blk_obs]
        self.obs_off = np.searchsorted(b_sorted, np.arange(self.n_blocks + 1)).astype(np.int64)
        # point copies: distinct (block, point rank) pairs
        pkey = blk * n + rank[pt]
        upk, pinv = np.unique(pkey, return_inverse=True)
        self.pc_pt = order[upk % n].astype(np.int32)
        self.pc_off = np.searchsorted(upk // n, np.arange(self.n_blocks + 1)).astype(np.int64)
        # camera copies: distinct (block, camera) pairs
        ckey = blk * m + cam
        uck, cinv = np.unique(ckey, return_inverse=True)
        self.cc_cam = (uck % m).astype(np.int32)
        self.cc_off = np.searchsorted(uck // m, np.arange(self.n_blocks + 1)).astype(np.int64)
        o = self.blk_obs
        self.obs_lp = (pinv[o] - self.pc_off[blk[o]]).astype(np.int32)
        self.obs_lc = (cinv[o] - self.cc_off[blk[o]]).astype(np.int32)
        self.n_pc, self.n_cc = len(self.pc_pt), len(self.cc_cam)


def block_objective(cfg, opl, ocl, z, xbar, ybar, rx, sy, X, Y):
    np_, nc, no = len(xbar) // 3, len(ybar) // 6, len(opl)
    return lib().ora_block_objective(ctypes.byref(cfg), np_, nc, no, _i(np.asarray(opl, np.int32)),
                                     _i(np.asarray(ocl, np.int32)), _d(_f64(z)), _d(_f64(xbar)),
                                     _d(_f64(ybar)), _d(_f64(rx)), _d(_f64(sy)), _d(_f64(X)), _d(_f64(Y)))


def block_solve(cfg, opl, ocl, z, xbar, ybar, rx, sy, X0, Y0):
    X, Y = _f64(X0).copy(), _f64(Y0).copy()
    np_, nc, no = len(xbar) // 3, len(ybar) // 6, len(opl)
    lib().ora_block_solve(ctypes.byref(cfg), np_, nc, no, _i(np.asarray(opl, np.int32)),
                          _i(np.asarray(ocl, np.int32)), _d(_f64(z)), _d(_f64(xbar)), _d(_f64(ybar)),
                          _d(_f64(rx)), _d(_f64(sy)), _d(X), _d(Y))
    return X, Y


class BlockState:
    """ADMM state with block subproblems: point copies/duals [n_pc, 3] and camera
    copies/duals [n_cc, 6] in layout order, cams [m, 6], pts [n, 3]."""

    def __init__(self, scene, pi, kappa, cams=None, pts=None):
        self.scene = scene
        self.layout = BlockLayout(scene, pi, kappa)
        B = self.layout
        self.cams = _f64(scene.cams0 if cams is None else cams).copy()
        self.pts = _f64(scene.pts0 if pts is None else pts).copy()
        self.pcopies = self.pts[B.pc_pt].copy()
        self.ccopies = self.cams[B.cc_cam].copy()
        self.pduals = np.zeros((B.n_pc, 3))
        self.cduals = np.zeros((B.n_cc, 6))
        self.k = 0

    def iterate(self, cfg, iters, nthreads=0, with_gt=True):
        s, B = self.scene, self.layout
        m = Metrics()
        zt = _f64(s.z_true) if with_gt else None
        rc = lib().ora_block_iterate(ctypes.byref(cfg), s.n_cams, s.n_pts, s.n_obs, _i(s.pt_idx),
                                     _i(s.cam_idx), _d(_f64(s.z)), _d(zt), B.n_blocks, _l(B.obs_off),
                                     _l(B.blk_obs), _i(B.obs_lp), _i(B.obs_lc), _l(B.pc_off), _i(B.pc_pt),
                                     _l(B.cc_off), _i(B.cc_cam), _d(self.pcopies), _d(self.pduals),
                                     _d(self.ccopies), _d(self.cduals), _d(self.cams), _d(self.pts), iters,
                                     nthreads, ctypes.byref(m))
        if rc != 0:
            raise ValueError("oracle rejected the block problem")
        self.k += iters
        return m.as_dict()
