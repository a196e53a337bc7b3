"""Thin Python binding of the C ABI in include/dba.h (argument marshalling only).

Every function has the name and meaning of its C counterpart; failures raise
DbaError carrying the status and dba_last_error().  The library is the
in-tree ``_build/libdba.so`` compiled by ``build.build()``; nothing here falls
back to any other implementation: if the library or a GPU is missing the
calls fail loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

DBA_OK, DBA_EINVAL, DBA_ENOMEM, DBA_ECUDA, DBA_ESTATE, DBA_ENUMERIC, DBA_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
DBA_LOSS_L2, DBA_LOSS_HUBER, DBA_LOSS_STUDENT_T = 0, 1, 2
DBA_PREC_F64, DBA_PREC_F32_LOCAL = 0, 1
DBA_SOLVER_GN, DBA_SOLVER_LBFGS = 0, 1

EXPORTED = [
    "dba_config_default", "dba_create", "dba_set_observations", "dba_set_ground_truth", "dba_iterate",
    "dba_iterate_until", "dba_evaluate", "dba_get_params", "dba_get_state", "dba_set_state",
    "dba_profile", "dba_inject_copy_stall", "dba_inject_host_alloc_failure", "dba_build_layout", "dba_layout", "dba_evaluate_noalloc", "dba_set_scenes", "dba_scene_stats",
    "dba_last_error", "dba_destroy", "dba_mlp_create", "dba_mlp_destroy", "dba_mlp_last_error",
    "dba_mlp_get_params", "dba_mlp_set_params", "dba_mlp_harvest", "dba_mlp_fit_normalizer",
    "dba_mlp_loss_grad", "dba_mlp_train", "dba_mlp_predict", "dba_set_warm_start",
    "dba_block_create", "dba_block_set_observations", "dba_block_set_reference_pixels", "dba_block_iterate",
    "dba_block_iterate_until", "dba_block_profile", "dba_block_get_params", "dba_block_layout",
    "dba_block_size_classes", "dba_block_launches_per_iteration", "dba_block_build_layout",
    "dba_block_algorithmic_flops", "dba_block_last_error",
    "dba_block_destroy",
]
DBA_BLOCK_MAX_POINTS, DBA_BLOCK_MAX_CAMERAS, DBA_BLOCK_SIZE_CLASSES = 64, 4, 4
DBA_MLP_N_PARAMS, DBA_MLP_N_FEATURES, DBA_MLP_N_TARGETS = 11552, 32, 16
DBA_NOALLOC_MAX_OBS = 16777216


class DbaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"dba status {status}: {message}")
        self.status = status


class dba_config(ctypes.Structure):
    _fields_ = [
        ("focal", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
        ("loss", ctypes.c_int), ("loss_param", ctypes.c_double),
        ("rho_x", ctypes.c_double), ("rho_y", ctypes.c_double), ("rho_angle", ctypes.c_double),
        ("inner_steps", ctypes.c_int), ("lm_lambda0", ctypes.c_double),
        ("lm_lambda_min", ctypes.c_double), ("eps_depth", ctypes.c_double),
        ("lm_model_tol", ctypes.c_double), ("precision", ctypes.c_int), ("tile_obs", ctypes.c_int), ("use_graph", ctypes.c_int),
        ("cuda_stream", ctypes.c_void_p), ("local_solver", ctypes.c_int), ("finalize_threads", ctypes.c_int),
    ]


class dba_stats(ctypes.Structure):
    _fields_ = [
        ("iters_done", ctypes.c_longlong), ("rmse_obs", ctypes.c_double), ("rmse_gt", ctypes.c_double),
        ("objective", ctypes.c_double), ("primal_res", ctypes.c_double), ("dual_res", ctypes.c_double),
        ("n_invalid", ctypes.c_longlong), ("seconds", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Loads the in-tree library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise ImportError(f"{_build.LIB} is missing: run paper_1708_07954_gb300.build.build() first")
    L = ctypes.CDLL(_build.LIB)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    dp = P(ctypes.c_double)
    ip = P(ctypes.c_int32)
    L.dba_config_default.argtypes = [P(dba_config)]
    L.dba_config_default.restype = None
    L.dba_create.argtypes = [P(dba_config), P(vp)]
    L.dba_set_observations.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ip, ip, dp, dp, dp]
    L.dba_set_ground_truth.argtypes = [vp, dp, dp, P(ctypes.c_uint8)]
    L.dba_iterate.argtypes = [vp, ctypes.c_int, P(dba_stats)]
    L.dba_iterate_until.argtypes = [vp, ctypes.c_int, ctypes.c_double, P(dba_stats)]
    L.dba_evaluate.argtypes = [vp, P(dba_stats)]
    L.dba_get_params.argtypes = [vp, dp, dp]
    L.dba_get_state.argtypes = [vp, dp, dp]
    L.dba_set_state.argtypes = [vp, dp, dp, dp, dp, ctypes.c_int64]
    L.dba_inject_host_alloc_failure.argtypes = [ctypes.c_int]
    L.dba_build_layout.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ip, ip, ctypes.c_int,
                                   P(ctypes.c_int64), ip, ip, ip, P(ctypes.c_int64), P(ctypes.c_int64)]
    L.dba_inject_copy_stall.argtypes = [vp, ctypes.c_int]
    L.dba_profile.argtypes = [vp, ctypes.c_int, P(ctypes.c_char_p), dp, P(ctypes.c_int)]
    L.dba_layout.argtypes = [vp, P(ctypes.c_int64), P(ctypes.c_int)]
    L.dba_set_scenes.argtypes = [vp, ctypes.c_int32, P(ctypes.c_int64), ip, ip]
    L.dba_scene_stats.argtypes = [vp, dp, dp, dp]
    L.dba_evaluate_noalloc.argtypes = [P(dba_config), ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, vp, vp, vp,
                                       vp, vp, vp, vp]
    fp = P(ctypes.c_float)
    L.dba_mlp_create.argtypes = [ctypes.c_uint64, P(vp)]
    L.dba_mlp_destroy.argtypes = [vp]
    L.dba_mlp_destroy.restype = None
    L.dba_mlp_last_error.argtypes = [vp]
    L.dba_mlp_last_error.restype = ctypes.c_char_p
    L.dba_mlp_get_params.argtypes = [vp, fp]
    L.dba_mlp_set_params.argtypes = [vp, fp]
    L.dba_mlp_harvest.argtypes = [vp, ctypes.c_int64, ctypes.c_int, vp, vp, ctypes.c_int64, P(ctypes.c_int64)]
    L.dba_mlp_fit_normalizer.argtypes = [vp, vp, vp, ctypes.c_int64]
    L.dba_mlp_loss_grad.argtypes = [vp, vp, vp, ctypes.c_int64, P(ctypes.c_double), fp]
    L.dba_mlp_train.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                ctypes.c_uint64, P(ctypes.c_double)]
    L.dba_mlp_predict.argtypes = [vp, vp, ctypes.c_int64, vp]
    L.dba_set_warm_start.argtypes = [vp, vp]
    L.dba_last_error.argtypes = [vp]
    L.dba_last_error.restype = ctypes.c_char_p
    L.dba_destroy.argtypes = [vp]
    L.dba_destroy.restype = None
    L.dba_block_create.argtypes = [P(dba_config), ctypes.c_int, ctypes.c_int, P(vp)]
    L.dba_block_set_observations.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ip, ip, dp, dp,
                                             dp]
    L.dba_block_set_reference_pixels.argtypes = [vp, dp, P(ctypes.c_uint8)]
    L.dba_block_iterate.argtypes = [vp, ctypes.c_int, P(dba_stats)]
    L.dba_block_iterate_until.argtypes = [vp, ctypes.c_int, ctypes.c_double, P(dba_stats)]
    L.dba_block_profile.argtypes = [vp, ctypes.c_int, dp]
    L.dba_block_get_params.argtypes = [vp, dp, dp]
    L.dba_block_layout.argtypes = [vp, P(ctypes.c_int64), P(ctypes.c_int64), P(ctypes.c_int64)]
    L.dba_block_size_classes.argtypes = [vp, P(ctypes.c_int64)]
    L.dba_block_build_layout.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ip, ip, ctypes.c_int,
                                         ctypes.c_int, P(ctypes.c_int64), ip, ip, ip, P(ctypes.c_int64),
                                         P(ctypes.c_int64)]
    L.dba_block_algorithmic_flops.argtypes = [vp, dp]
    L.dba_block_launches_per_iteration.argtypes = [vp, P(ctypes.c_int32)]
    L.dba_block_last_error.argtypes = [vp]
    L.dba_block_last_error.restype = ctypes.c_char_p
    L.dba_block_destroy.argtypes = [vp]
    L.dba_block_destroy.restype = None
    for name in EXPORTED:
        if name not in ("dba_config_default", "dba_last_error", "dba_destroy", "dba_mlp_destroy",
                        "dba_mlp_last_error", "dba_block_last_error", "dba_block_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status, ctx=None):
    if status != DBA_OK:
        msg = load().dba_last_error(ctx).decode()
        raise DbaError(status, msg)


def _d(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        a = a.reshape(shape)
    return a


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double if a.dtype == np.float64 else ctypes.c_int32))


def dba_config_default(**overrides) -> dba_config:
    cfg = dba_config()
    load().dba_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def dba_create(cfg: dba_config) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(load().dba_create(ctypes.byref(cfg), ctypes.byref(ctx)))
    return ctx


def dba_set_observations(ctx, n_cams, n_pts, pt_idx, cam_idx, z, cams0, pts0):
    pt_idx = np.ascontiguousarray(pt_idx, dtype=np.int32)
    cam_idx = np.ascontiguousarray(cam_idx, dtype=np.int32)
    l = pt_idx.shape[0]
    if cam_idx.shape[0] != l:
        raise ValueError("pt_idx and cam_idx differ in length")
    z = _d(z, (l, 2))
    cams0 = _d(cams0, (n_cams, 6))
    pts0 = _d(pts0, (n_pts, 3))
    _check(load().dba_set_observations(ctx, n_cams, n_pts, l, _ptr(pt_idx), _ptr(cam_idx), _ptr(z),
                                       _ptr(cams0), _ptr(pts0)), ctx)


def dba_build_layout(n_cams, n_pts, pt_idx, cam_idx, tile_obs):
    """The internal order and tile table of dba_set_observations, built on the host:
    dict of perm, point, point_perm, cam_rank (numpy arrays) and tile_start."""
    pt_idx = np.ascontiguousarray(pt_idx, dtype=np.int32)
    cam_idx = np.ascontiguousarray(cam_idx, dtype=np.int32)
    l = pt_idx.shape[0]
    if cam_idx.shape[0] != l:
        raise ValueError("pt_idx and cam_idx differ in length")
    perm = np.zeros(l, np.int64)
    point = np.zeros(l, np.int32)
    point_perm = np.zeros(n_pts, np.int32)
    cam_rank = np.zeros(l, np.int32)
    tile_start = np.zeros(l + 1, np.int64)
    nt = ctypes.c_int64()
    i64 = ctypes.POINTER(ctypes.c_int64)
    _check(load().dba_build_layout(n_cams, n_pts, l, _ptr(pt_idx), _ptr(cam_idx), tile_obs,
                                   perm.ctypes.data_as(i64), _ptr(point), _ptr(point_perm), _ptr(cam_rank),
                                   tile_start.ctypes.data_as(i64), ctypes.byref(nt)))
    return {"perm": perm, "point": point, "point_perm": point_perm, "cam_rank": cam_rank,
            "tile_start": tile_start[: nt.value + 1]}


def dba_set_ground_truth(ctx, cams_gt, pts_gt, inlier=None):
    cams_gt = np.ascontiguousarray(cams_gt, dtype=np.float64)
    pts_gt = np.ascontiguousarray(pts_gt, dtype=np.float64)
    mask = None
    if inlier is not None:
        inlier = np.ascontiguousarray(inlier, dtype=np.uint8)
        mask = inlier.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    _check(load().dba_set_ground_truth(ctx, _ptr(cams_gt), _ptr(pts_gt), mask), ctx)


def dba_iterate(ctx, n_iters, stats=True):
    st = dba_stats()
    _check(load().dba_iterate(ctx, int(n_iters), ctypes.byref(st) if stats else None), ctx)
    return st.as_dict() if stats else None


def dba_iterate_until(ctx, max_iters, target_rmse_gt):
    st = dba_stats()
    _check(load().dba_iterate_until(ctx, int(max_iters), float(target_rmse_gt), ctypes.byref(st)), ctx)
    return st.as_dict()


def dba_evaluate(ctx):
    st = dba_stats()
    _check(load().dba_evaluate(ctx, ctypes.byref(st)), ctx)
    return st.as_dict()


def dba_get_params(ctx, n_cams, n_pts):
    cams = np.zeros((n_cams, 6))
    pts = np.zeros((n_pts, 3))
    _check(load().dba_get_params(ctx, _ptr(cams), _ptr(pts)), ctx)
    return cams, pts


def dba_get_state(ctx, n_obs):
    copies = np.zeros((n_obs, 9))
    duals = np.zeros((n_obs, 9))
    _check(load().dba_get_state(ctx, _ptr(copies), _ptr(duals)), ctx)
    return copies, duals


def dba_set_state(ctx, copies, duals, cams, pts, k=0):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (copies, duals, cams, pts)]
    _check(load().dba_set_state(ctx, *[_ptr(a) for a in arrs], int(k)), ctx)


def dba_inject_host_alloc_failure(n):
    """Fault injection (tests): the next n entry points on this thread fail with DBA_ENOMEM."""
    _check(load().dba_inject_host_alloc_failure(int(n)), None)


def dba_profile(ctx, n_iters):
    cap = 16
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_double * cap)()
    count = ctypes.c_int(cap)
    _check(load().dba_profile(ctx, int(n_iters), names, ms, ctypes.byref(count)), ctx)
    return {names[k].decode(): ms[k] for k in range(count.value)}


def dba_layout(ctx):
    out = (ctypes.c_int64 * 7)()
    count = ctypes.c_int(7)
    _check(load().dba_layout(ctx, out, ctypes.byref(count)), ctx)
    keys = ["tiles", "tile_obs", "point_runs", "camera_runs", "split_points", "point_slots", "finalize_threads"]
    return {keys[k]: int(out[k]) for k in range(count.value)}


def dba_evaluate_noalloc(cfg, n_cams, n_pts, n_obs, pt_idx_ptr, cam_idx_ptr, z_ptr, cams_ptr, pts_ptr,
                         out_ptr, stream=None):
    """Device pointers (ints) in, device pointer out; see include/dba.h."""
    _check(load().dba_evaluate_noalloc(ctypes.byref(cfg), int(n_cams), int(n_pts), int(n_obs), pt_idx_ptr,
                                       cam_idx_ptr, z_ptr, cams_ptr, pts_ptr, out_ptr, stream))


def dba_set_scenes(ctx, obs_off, cam_off, pt_off):
    obs_off = np.ascontiguousarray(obs_off, dtype=np.int64)
    cam_off = np.ascontiguousarray(cam_off, dtype=np.int32)
    pt_off = np.ascontiguousarray(pt_off, dtype=np.int32)
    _check(load().dba_set_scenes(ctx, len(obs_off) - 1, obs_off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 _ptr(cam_off), _ptr(pt_off)), ctx)


def dba_scene_stats(ctx, n_scenes):
    out = [np.zeros(n_scenes) for _ in range(3)]
    _check(load().dba_scene_stats(ctx, *[_ptr(a) for a in out]), ctx)
    return {"rmse_obs": out[0], "rmse_gt": out[1], "objective": out[2]}


def dba_last_error(ctx=None) -> str:
    return load().dba_last_error(ctx).decode()


def dba_destroy(ctx):
    if ctx:
        load().dba_destroy(ctx)


class Mlp:
    """The warm-start network (C object dba_mlp).  Feature/target buffers are device pointers
    (e.g. torch CUDA tensors' data_ptr())."""

    def __init__(self, seed=0):
        L = load()
        self.h = ctypes.c_void_p()
        st = L.dba_mlp_create(ctypes.c_uint64(seed), ctypes.byref(self.h))
        if st != DBA_OK:
            raise DbaError(st, L.dba_mlp_last_error(None).decode())

    def _check(self, st):
        if st != DBA_OK:
            raise DbaError(st, load().dba_mlp_last_error(self.h).decode())

    def get_params(self):
        out = np.zeros(DBA_MLP_N_PARAMS, dtype=np.float32)
        self._check(load().dba_mlp_get_params(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.shape == (DBA_MLP_N_PARAMS,)
        self._check(load().dba_mlp_set_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def fit_normalizer(self, feats_ptr, targs_ptr, n):
        self._check(load().dba_mlp_fit_normalizer(self.h, feats_ptr, targs_ptr, int(n)))

    def loss_grad(self, feats_ptr, targs_ptr, n):
        loss = ctypes.c_double()
        g = np.zeros(DBA_MLP_N_PARAMS, dtype=np.float32)
        self._check(load().dba_mlp_loss_grad(self.h, feats_ptr, targs_ptr, int(n), ctypes.byref(loss),
                                             g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return loss.value, g

    def train(self, feats_ptr, targs_ptr, n, epochs, batch, lr, seed=0):
        loss = ctypes.c_double()
        self._check(load().dba_mlp_train(self.h, feats_ptr, targs_ptr, int(n), int(epochs), int(batch),
                                         ctypes.c_float(lr), ctypes.c_uint64(seed), ctypes.byref(loss)))
        return loss.value

    def predict(self, feats_ptr, n, out_ptr):
        self._check(load().dba_mlp_predict(self.h, feats_ptr, int(n), out_ptr))

    def close(self):
        if self.h:
            load().dba_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dba_mlp_harvest(ctx, stride, target_steps, feats_ptr, targs_ptr, cap):
    n = ctypes.c_int64()
    _check(load().dba_mlp_harvest(ctx, int(stride), int(target_steps), feats_ptr, targs_ptr, int(cap),
                                  ctypes.byref(n)), ctx)
    return n.value


def dba_set_warm_start(ctx, mlp):
    _check(load().dba_set_warm_start(ctx, mlp.h if mlp is not None else None), ctx)


def dba_block_build_layout(n_cams, n_pts, pt_idx, cam_idx, block_points, block_cams):
    """The block layout of dba_block_set_observations, built on the host: dict of
    obs_order, blocks (n_blocks x 6: first observation, count, first point copy, count,
    first camera copy, count; launch order), pc_point, cc_camera, size_classes."""
    pt_idx = np.ascontiguousarray(pt_idx, dtype=np.int32)
    cam_idx = np.ascontiguousarray(cam_idx, dtype=np.int32)
    l = pt_idx.shape[0]
    if cam_idx.shape[0] != l:
        raise ValueError("pt_idx and cam_idx differ in length")
    order = np.zeros(l, np.int64)
    blocks = np.zeros(6 * l, np.int32)
    pc = np.zeros(l, np.int32)
    cc = np.zeros(l, np.int32)
    counts = np.zeros(3, np.int64)
    cls = np.zeros(DBA_BLOCK_SIZE_CLASSES, np.int64)
    i64 = ctypes.POINTER(ctypes.c_int64)
    st = load().dba_block_build_layout(n_cams, n_pts, l, _ptr(pt_idx), _ptr(cam_idx), block_points, block_cams,
                                       order.ctypes.data_as(i64), _ptr(blocks), _ptr(pc), _ptr(cc),
                                       counts.ctypes.data_as(i64), cls.ctypes.data_as(i64))
    if st != DBA_OK:
        raise DbaError(st, load().dba_block_last_error(None).decode())
    nb, npc, ncc = (int(x) for x in counts)
    return {"obs_order": order, "blocks": blocks[: 6 * nb].reshape(nb, 6), "pc_point": pc[:npc],
            "cc_camera": cc[:ncc], "size_classes": cls}


class Solver:
    """Owns one context for one scene (a scenes.Scene or anything with its fields)."""

    def __init__(self, scene, precision=None, inner_steps=5, rho_x=None, rho_y=None, rho_angle=None,
                 tile_obs=0, use_graph=1, stream=None, ground_truth=True, **cfg_overrides):
        self.scene = scene
        prec = scene.precision if precision is None else precision
        self.cfg = dba_config_default(
            focal=scene.focal, cx=scene.cx, cy=scene.cy, loss=scene.loss, loss_param=scene.loss_param,
            rho_x=scene.rho_x if rho_x is None else rho_x, rho_y=scene.rho_y if rho_y is None else rho_y,
            rho_angle=getattr(scene, "rho_angle", 0.0) if rho_angle is None else rho_angle,
            inner_steps=inner_steps, precision=prec, tile_obs=tile_obs, use_graph=use_graph,
            cuda_stream=stream, **cfg_overrides)
        self.ctx = dba_create(self.cfg)
        try:
            dba_set_observations(self.ctx, scene.n_cams, scene.n_pts, scene.pt_idx, scene.cam_idx, scene.z,
                                 scene.cams0, scene.pts0)
            if getattr(scene, "scene_off", None) is not None:
                dba_set_scenes(self.ctx, scene.scene_off, scene.cam_off, scene.pt_off)
            if ground_truth:
                # rmse_gt over observations of outlier-free tracks
                mask = scene.clean_mask() if hasattr(scene, "clean_mask") else None
                dba_set_ground_truth(self.ctx, scene.cams_gt, scene.pts_gt, mask)
        except Exception:
            self.close()
            raise

    def iterate(self, n, stats=True):
        return dba_iterate(self.ctx, n, stats)

    def iterate_until(self, max_iters, target):
        return dba_iterate_until(self.ctx, max_iters, target)

    def evaluate(self):
        return dba_evaluate(self.ctx)

    def params(self):
        return dba_get_params(self.ctx, self.scene.n_cams, self.scene.n_pts)

    def state(self):
        return dba_get_state(self.ctx, self.scene.n_obs)

    def set_state(self, copies, duals, cams, pts, k=0):
        dba_set_state(self.ctx, copies, duals, cams, pts, k)

    def profile(self, n):
        return dba_profile(self.ctx, n)

    def inject_copy_stall(self, on):
        """Fault injection (tests): the tile kernel's wait for its tensor copies runs out."""
        _check(load().dba_inject_copy_stall(self.ctx, 1 if on else 0), self.ctx)

    def layout(self):
        return dba_layout(self.ctx)

    def set_warm_start(self, mlp):
        dba_set_warm_start(self.ctx, mlp)

    def harvest(self, stride, target_steps, feats_ptr, targs_ptr, cap):
        return dba_mlp_harvest(self.ctx, stride, target_steps, feats_ptr, targs_ptr, cap)

    def scene_stats(self):
        return dba_scene_stats(self.ctx, len(self.scene.scene_off) - 1)

    def close(self):
        if self.ctx:
            dba_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BlockSolver:
    """Block subproblems of pi points x kappa cameras (Sec. 3.1.4, Eq. 14) for one scene:
    the context dba_block_ctx."""

    def __init__(self, scene, block_points, block_cams, precision=None, inner_steps=5, rho_x=None, rho_y=None,
                 rho_angle=None, stream=None, ground_truth=True, **cfg_overrides):
        self.scene = scene
        prec = scene.precision if precision is None else precision
        self.cfg = dba_config_default(
            focal=scene.focal, cx=scene.cx, cy=scene.cy, loss=scene.loss, loss_param=scene.loss_param,
            rho_x=scene.rho_x if rho_x is None else rho_x, rho_y=scene.rho_y if rho_y is None else rho_y,
            rho_angle=getattr(scene, "rho_angle", 0.0) if rho_angle is None else rho_angle,
            inner_steps=inner_steps, precision=prec, cuda_stream=stream, **cfg_overrides)
        L = load()
        self.ctx = ctypes.c_void_p()
        st = L.dba_block_create(ctypes.byref(self.cfg), int(block_points), int(block_cams), ctypes.byref(self.ctx))
        if st != DBA_OK:
            raise DbaError(st, L.dba_block_last_error(None).decode())
        try:
            pt_idx = np.ascontiguousarray(scene.pt_idx, dtype=np.int32)
            cam_idx = np.ascontiguousarray(scene.cam_idx, dtype=np.int32)
            l = pt_idx.shape[0]
            z = _d(scene.z, (l, 2))
            cams0 = _d(scene.cams0, (scene.n_cams, 6))
            pts0 = _d(scene.pts0, (scene.n_pts, 3))
            self._check(L.dba_block_set_observations(self.ctx, scene.n_cams, scene.n_pts, l, _ptr(pt_idx),
                                                     _ptr(cam_idx), _ptr(z), _ptr(cams0), _ptr(pts0)))
            if ground_truth:
                zt = _d(scene.z_true, (l, 2))
                mask = scene.clean_mask() if hasattr(scene, "clean_mask") else None
                mp = None
                if mask is not None:
                    mask = np.ascontiguousarray(mask, dtype=np.uint8)
                    mp = mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
                self._check(L.dba_block_set_reference_pixels(self.ctx, _ptr(zt), mp))
        except Exception:
            self.close()
            raise

    def _check(self, st):
        if st != DBA_OK:
            raise DbaError(st, load().dba_block_last_error(self.ctx).decode())

    def iterate(self, n, stats=True):
        st = dba_stats()
        self._check(load().dba_block_iterate(self.ctx, int(n), ctypes.byref(st) if stats else None))
        return st.as_dict() if stats else None

    def iterate_until(self, max_iters, target):
        st = dba_stats()
        self._check(load().dba_block_iterate_until(self.ctx, int(max_iters), float(target), ctypes.byref(st)))
        return st.as_dict()

    def profile(self, n):
        ms = np.zeros(3)
        self._check(load().dba_block_profile(self.ctx, int(n), _ptr(ms)))
        return {"block_solve": ms[0], "block_point_consensus": ms[1], "block_camera_consensus": ms[2]}

    def params(self):
        cams = np.zeros((self.scene.n_cams, 6))
        pts = np.zeros((self.scene.n_pts, 3))
        self._check(load().dba_block_get_params(self.ctx, _ptr(cams), _ptr(pts)))
        return cams, pts

    def layout(self):
        nb, npc, ncc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._check(load().dba_block_layout(self.ctx, ctypes.byref(nb), ctypes.byref(npc), ctypes.byref(ncc)))
        return {"n_blocks": nb.value, "n_point_copies": npc.value, "n_camera_copies": ncc.value}

    def size_classes(self):
        """Blocks per size class of the solve kernels: one camera and at most 8 points, at most
        2 cameras and 16 points, at most 32 points, the rest (see dba_block_size_classes in
        include/dba.h for the lane groups of each)."""
        c = (ctypes.c_int64 * DBA_BLOCK_SIZE_CLASSES)()
        self._check(load().dba_block_size_classes(self.ctx, c))
        return list(c)

    def algorithmic_flops(self):
        f = ctypes.c_double()
        self._check(load().dba_block_algorithmic_flops(self.ctx, ctypes.byref(f)))
        return f.value

    def launches_per_iteration(self):
        """Kernel launches of one block iteration (block solves by range, consensus)."""
        n = ctypes.c_int32()
        self._check(load().dba_block_launches_per_iteration(self.ctx, ctypes.byref(n)))
        return n.value

    def close(self):
        if self.ctx:
            load().dba_block_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
