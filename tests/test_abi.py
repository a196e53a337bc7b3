"""C ABI checks that need no GPU: the library builds, loads and exports every
entry point include/dba.h declares; configuration validation runs on the host."""
import ctypes
import os
import re

import pytest

from paper_1708_07954_gb300 import build, dba

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return dba.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "dba.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dba_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("dba_create", "dba_set_observations", "dba_iterate", "dba_get_params"):
        assert required in names
    assert set(names) == set(dba.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    out = os.popen(f"nm -D --defined-only {build.LIB}").read()
    for name in _declared():
        assert re.search(rf"\bT {name}\b", out), name


def test_config_defaults(lib):
    cfg = dba.dba_config_default()
    assert cfg.focal == 500.0 and cfg.cx == 320.0 and cfg.cy == 240.0
    assert cfg.loss == dba.DBA_LOSS_HUBER and cfg.loss_param == 2.0
    assert cfg.inner_steps == 5 and cfg.precision == dba.DBA_PREC_F32_LOCAL and cfg.use_graph == 1
    assert cfg.tile_obs == 0 and cfg.finalize_threads == 0


@pytest.mark.parametrize("field,value", [("focal", -1.0), ("rho_x", 0.0), ("rho_y", float("nan")),
                                         ("loss", 7), ("inner_steps", -1), ("precision", 3),
                                         ("tile_obs", 100), ("loss_param", 0.0), ("local_solver", 2),
                                         ("finalize_threads", 48)])
def test_invalid_config_is_rejected_before_any_device_work(lib, field, value):
    cfg = dba.dba_config_default(**{field: value})
    with pytest.raises(dba.DbaError) as ei:
        dba.dba_create(cfg)
    assert ei.value.status == dba.DBA_EINVAL
    assert "invalid configuration" in dba.dba_last_error(None)


def test_null_arguments(lib):
    assert lib.dba_create(None, None) == dba.DBA_EINVAL
    assert lib.dba_iterate(None, 1, None) == dba.DBA_EINVAL
    assert lib.dba_get_params(None, None, None) == dba.DBA_EINVAL
    lib.dba_destroy(None)
    assert isinstance(lib.dba_last_error(None), bytes)


@pytest.mark.parametrize("pi,kappa", [(0, 1), (65, 1), (4, 0), (4, 5)])
def test_block_sizes_are_validated_before_any_device_work(lib, pi, kappa):
    cfg = dba.dba_config_default()
    ctx = ctypes.c_void_p()
    assert lib.dba_block_create(ctypes.byref(cfg), pi, kappa, ctypes.byref(ctx)) == dba.DBA_EINVAL
    assert "block_points" in lib.dba_block_last_error(None).decode()


def test_block_null_arguments(lib):
    assert lib.dba_block_create(None, 1, 1, None) == dba.DBA_EINVAL
    assert lib.dba_block_iterate(None, 1, None) == dba.DBA_EINVAL
    assert lib.dba_block_get_params(None, None, None) == dba.DBA_EINVAL
    assert lib.dba_inject_copy_stall(None, 1) == dba.DBA_EINVAL
    counts = (ctypes.c_int64 * dba.DBA_BLOCK_SIZE_CLASSES)()
    assert lib.dba_block_size_classes(None, counts) == dba.DBA_EINVAL
    lib.dba_block_destroy(None)


def test_block_path_takes_only_the_gauss_newton_solver(lib):
    cfg = dba.dba_config_default(local_solver=dba.DBA_SOLVER_LBFGS)
    ctx = ctypes.c_void_p()
    assert lib.dba_block_create(ctypes.byref(cfg), 8, 2, ctypes.byref(ctx)) == dba.DBA_EINVAL


def test_binding_constants_match_the_header():
    """The numeric #defines and enum values of include/dba.h and the binding's constants agree."""
    text = open(os.path.join(ROOT, "include", "dba.h")).read()
    defines = {k: int(v) for k, v in re.findall(r"#define\s+(DBA_[A-Z_0-9]+)\s+(\d+)", text)}
    defines.update({k: int(v) for k, v in re.findall(r"\b(DBA_[A-Z_0-9]+)\s*=\s*(-?\d+)", text)})
    assert defines, "no numeric defines found"
    for name, value in defines.items():
        if hasattr(dba, name):
            assert getattr(dba, name) == value, name
    for name in ("DBA_BLOCK_MAX_POINTS", "DBA_BLOCK_MAX_CAMERAS", "DBA_BLOCK_SIZE_CLASSES", "DBA_MLP_N_PARAMS",
                 "DBA_ETIMEOUT", "DBA_SOLVER_LBFGS", "DBA_PREC_F32_LOCAL", "DBA_LOSS_STUDENT_T"):
        assert name in defines and hasattr(dba, name), name


def _status_entry_points():
    """(name, ctypes argument list of zeros/NULLs) of every dba_status function in dba.h."""
    text = open(os.path.join(ROOT, "include", "dba.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = []
    for name, params in re.findall(r"dba_status\s+(dba_[a-z_]+)\s*\(([^)]*)\)\s*;", text):
        args = []
        for p in [q.strip() for q in params.split(",") if q.strip()]:
            if "*" in p:
                args.append(ctypes.c_void_p(None))
            elif p.startswith("double"):
                args.append(ctypes.c_double(0.0))
            elif p.startswith("float"):
                args.append(ctypes.c_float(0.0))
            elif p.startswith("int64_t"):
                args.append(ctypes.c_int64(0))
            elif p.startswith("uint64_t"):
                args.append(ctypes.c_uint64(0))
            else:
                args.append(ctypes.c_int32(0))
        out.append((name, args))
    return out


def test_every_entry_point_turns_a_host_allocation_failure_into_enomem(lib):
    """An injected failed host allocation (std::bad_alloc) in each entry point comes back as
    DBA_ENOMEM with no abort: every dba_status entry point runs its whole body under the
    guard, before touching any argument (the calls pass NULL and zero for everything)."""
    raw = ctypes.CDLL(build.LIB)  # a handle without the binding's argument types
    raw.dba_last_error.restype = ctypes.c_char_p
    raw.dba_block_last_error.restype = ctypes.c_char_p
    raw.dba_mlp_last_error.restype = ctypes.c_char_p
    entries = [e for e in _status_entry_points() if e[0] != "dba_inject_host_alloc_failure"]
    assert len(entries) >= 30
    for name, args in entries:
        assert raw.dba_inject_host_alloc_failure(1) == dba.DBA_OK
        assert getattr(raw, name)(*args) == dba.DBA_ENOMEM, name
        # the injection is used up: the same call now fails on its NULL arguments instead
        assert getattr(raw, name)(*args) != dba.DBA_ENOMEM, name
    assert raw.dba_inject_host_alloc_failure(1) == dba.DBA_OK
    assert raw.dba_create(None, None) == dba.DBA_ENOMEM
    assert raw.dba_last_error(None) == b"out of host memory"
    assert raw.dba_inject_host_alloc_failure(1) == dba.DBA_OK
    assert raw.dba_block_create(None, 1, 1, None) == dba.DBA_ENOMEM
    assert raw.dba_block_last_error(None) == b"out of host memory"
    assert raw.dba_inject_host_alloc_failure(-1) == dba.DBA_EINVAL
    assert raw.dba_inject_host_alloc_failure(0) == dba.DBA_OK


def test_host_layout_reports_enomem_and_recovers(lib):
    """A host-only entry point with real work: injected failure, then the same call succeeds."""
    import numpy as np

    pt = np.array([0, 0, 1, 1], np.int32)
    cam = np.array([0, 1, 0, 1], np.int32)
    n_tiles = ctypes.c_int64(0)
    i32 = ctypes.POINTER(ctypes.c_int32)
    raw = ctypes.CDLL(build.LIB)
    raw.dba_inject_host_alloc_failure(1)
    args = (2, 2, ctypes.c_int64(4), pt.ctypes.data_as(i32), cam.ctypes.data_as(i32), 64, None, None, None, None,
            None, ctypes.byref(n_tiles))
    assert raw.dba_build_layout(*args) == dba.DBA_ENOMEM
    assert raw.dba_build_layout(*args) == dba.DBA_OK and n_tiles.value == 1
