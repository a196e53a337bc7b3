"""dba_evaluate_noalloc: reprojection statistics without any device allocation.

Some callers cannot let a library call cudaMalloc -- their device memory is
owned by another allocator (a framework's caching allocator or a pool reserved
up front), or they run inside graph-replayed or real-time loops where an
allocation would stall or fail.  This entry point takes the caller's device
buffers and keeps its partial sums in a fixed file-scope device array.  These
tests call it through the C ABI on device buffers the test owns and compare
it with the context-based dba_evaluate and with the FP64 CPU oracle on the same
parameters, twice in a row (the scratch array is shared by all calls and reused).  The file is named so
that pytest collects it last.
"""
import numpy as np
import pytest

import oracle as O
from paper_1708_07954_gb300 import build, dba
from paper_1708_07954_gb300 import scenes as S

pytestmark = pytest.mark.gpu

TOL = 1e-9  # FP64 on both sides; only the summation order differs


def _device(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to("cuda")


def test_evaluate_noalloc_matches_context_evaluation_twice():
    import torch

    build.build()
    dba.load()
    sc = S.scene1(n_pts=3000, n_cams=32, seed=61)
    with dba.Solver(sc, precision=dba.DBA_PREC_F64, ground_truth=False) as s:
        refs = [(sc.cams0, sc.pts0, s.evaluate())]
        s.iterate(3, stats=False)
        cams1, pts1 = s.params()
        refs.append((cams1, pts1, s.evaluate()))
        cfg = s.cfg
    pt = _device(torch, sc.pt_idx, np.int32)
    cm = _device(torch, sc.cam_idx, np.int32)
    z = _device(torch, sc.z, np.float64)
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for cams, pts, ref in refs:
        c = _device(torch, cams, np.float64)
        p = _device(torch, pts, np.float64)
        dba.dba_evaluate_noalloc(cfg, sc.n_cams, sc.n_pts, sc.n_obs, pt.data_ptr(), cm.data_ptr(), z.data_ptr(),
                                 c.data_ptr(), p.data_ptr(), out.data_ptr(), stream)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert o[2] + o[3] == sc.n_obs and o[3] == ref["n_invalid"]
        assert abs(np.sqrt(o[0] / o[2]) - ref["rmse_obs"]) <= TOL * ref["rmse_obs"]
        assert abs(o[1] - ref["objective"]) <= TOL * ref["objective"]
        # and, independently of the library, against the FP64 CPU oracle at the same parameters
        ora = O.State(sc, cams=cams, pts=pts).metrics(O.config_for(sc), with_gt=False)
        assert o[3] == ora["n_invalid"]
        assert abs(np.sqrt(o[0] / o[2]) - ora["rmse_obs"]) <= TOL * ora["rmse_obs"]
        assert abs(o[1] - ora["objective"]) <= TOL * ora["objective"]


def test_evaluate_noalloc_rejects_sizes_beyond_its_scratch():
    build.build()
    cfg = dba.dba_config_default()
    with pytest.raises(dba.DbaError) as e:
        dba.dba_evaluate_noalloc(cfg, 1, 1, dba.DBA_NOALLOC_MAX_OBS + 1, 1, 1, 1, 1, 1, 1, None)
    assert e.value.status == dba.DBA_EINVAL and "scratch" in str(e.value)
