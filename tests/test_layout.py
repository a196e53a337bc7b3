"""Host logic without a GPU: the internal observation order and tile table that
dba_set_observations builds (dba_build_layout), checked against their definition with
numpy on inputs with unobserved points, repeated (point, camera) pairs and tracks
longer than a tile."""
import numpy as np
import pytest

from paper_1708_07954_gb300 import build, dba
from paper_1708_07954_gb300 import scenes as S


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dba.load()


def _inputs(seed):
    rng = np.random.default_rng(seed)
    n_cams, n_pts = 40, 700
    pt, cam = [], []
    for i in range(n_pts):
        if i % 53 == 7:
            continue  # unobserved point
        length = int(rng.integers(1, 12)) if i % 97 else int(rng.integers(200, 600))  # some longer than a tile
        c0 = int(rng.integers(0, n_cams))
        for _ in range(length):
            pt.append(i)
            cam.append((c0 + int(rng.integers(0, 6))) % n_cams)  # repeats of a pair occur
    order = rng.permutation(len(pt))
    return n_cams, n_pts, np.array(pt, np.int32)[order], np.array(cam, np.int32)[order]


def _check(n_cams, n_pts, pt, cam, tile):
    L = dba.dba_build_layout(n_cams, n_pts, pt, cam, tile)
    perm, point, point_perm, rank, ts = L["perm"], L["point"], L["point_perm"], L["cam_rank"], L["tile_start"]
    n = len(pt)
    # a permutation of the observations, grouped by internal point
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert np.array_equal(np.sort(point_perm), np.arange(n_pts))
    assert np.all(np.diff(point) >= 0)
    assert np.array_equal(pt[perm], point_perm[point])
    # points ordered by (smallest observing camera, caller id), unobserved points last
    first = np.full(n_pts, n_cams)
    np.minimum.at(first, pt, cam)
    expect = np.lexsort((np.arange(n_pts), first))
    assert np.array_equal(point_perm, expect)
    # inside a point: by camera, then caller index
    c = cam[perm]
    same = point[1:] == point[:-1]
    assert np.all(~same | (c[1:] > c[:-1]) | ((c[1:] == c[:-1]) & (perm[1:] > perm[:-1])))
    # tiles: consecutive and at most `tile` observations; a track of at most `tile`
    # observations lies in one tile; a longer one is cut into pieces of `tile`
    # observations from its start (the last piece may share its tile with whole tracks)
    assert ts[0] == 0 and ts[-1] == n and np.all(np.diff(ts) > 0) and np.all(np.diff(ts) <= tile)
    starts = np.flatnonzero(np.r_[True, point[1:] != point[:-1]])
    ends = np.r_[starts[1:], n]
    tile_of = np.searchsorted(ts, np.arange(n), side="right") - 1
    for s0, e0 in zip(starts, ends):
        if e0 - s0 <= tile:
            assert tile_of[s0] == tile_of[e0 - 1]
        else:
            cuts = [x for x in ts if s0 < x < e0]
            assert cuts == list(range(s0 + tile, e0, tile))
            assert s0 in set(ts.tolist())
    # camera ranks: inside each tile, the order of (camera, position)
    for a, b in zip(ts[:-1], ts[1:]):
        key = np.lexsort((np.arange(b - a), c[a:b]))
        assert np.array_equal(rank[a:b][key], np.arange(b - a))
    return L


@pytest.mark.parametrize("tile", [64, 128, 256])
def test_layout_matches_its_definition(tile):
    n_cams, n_pts, pt, cam = _inputs(5)
    L = _check(n_cams, n_pts, pt, cam, tile)
    assert len(L["tile_start"]) > 3


def test_layout_of_a_generated_workload_and_determinism():
    sc = S.scene1(n_pts=3000, n_cams=32, seed=3)
    a = _check(sc.n_cams, sc.n_pts, sc.pt_idx, sc.cam_idx, 256)
    b = dba.dba_build_layout(sc.n_cams, sc.n_pts, sc.pt_idx, sc.cam_idx, 256)
    for k in a:
        assert np.array_equal(a[k], b[k])


def test_layout_rejects_bad_input():
    pt = np.array([0, 1, 2], np.int32)
    cam = np.array([0, 1, 5], np.int32)
    with pytest.raises(dba.DbaError) as e:
        dba.dba_build_layout(3, 3, pt, cam, 256)
    assert e.value.status == dba.DBA_EINVAL and "observation 2" in str(e.value)
    with pytest.raises(dba.DbaError):
        dba.dba_build_layout(6, 3, pt, cam, 100)


@pytest.mark.parametrize("pi,kappa", [(1, 1), (8, 2), (32, 4), (5, 3), (64, 2)])
def test_block_layout_matches_the_oracle(pi, kappa):
    """The library's block layout (Eq. 14 under the block reading) equals the oracle's,
    which is built independently with numpy: observation order, block boundaries, point
    and camera copies; blocks are launched grouped by size class."""
    import oracle as O

    sc = S.scene1(n_pts=1200, n_cams=24, seed=41)
    ref = O.BlockLayout(sc, pi, kappa)
    L = dba.dba_block_build_layout(sc.n_cams, sc.n_pts, sc.pt_idx, sc.cam_idx, pi, kappa)
    assert np.array_equal(L["obs_order"], ref.blk_obs)
    b = L["blocks"][np.argsort(L["blocks"][:, 0], kind="stable")]
    assert len(b) == ref.n_blocks
    assert np.array_equal(b[:, 0], ref.obs_off[:-1]) and np.array_equal(b[:, 1], np.diff(ref.obs_off))
    assert np.array_equal(b[:, 2], ref.pc_off[:-1]) and np.array_equal(b[:, 3], np.diff(ref.pc_off))
    assert np.array_equal(b[:, 4], ref.cc_off[:-1]) and np.array_equal(b[:, 5], np.diff(ref.cc_off))
    assert np.array_equal(L["pc_point"], ref.pc_pt) and np.array_equal(L["cc_camera"], ref.cc_cam)
    # launch order: size classes one after another (8, 16, 32 lanes; 32 lanes x 2 copies),
    # each ordered by point count (the kernels take its small blocks in narrower lane
    # groups), equal counts in layout order
    npb, ncb = L["blocks"][:, 3], L["blocks"][:, 5]
    cls = np.where((ncb == 1) & (npb <= 8), 0, np.where((ncb <= 2) & (npb <= 16), 1, np.where(npb <= 32, 2, 3)))
    assert np.all(np.diff(cls) >= 0)
    assert np.array_equal(L["size_classes"], np.bincount(cls, minlength=4))
    key = cls.astype(np.int64) * 1000 + npb
    assert np.all(np.diff(key) >= 0)
    same = np.diff(key) == 0
    assert np.all(np.diff(L["blocks"][:, 0])[same] > 0)


def test_block_layout_rejects_a_repeated_pair():
    pt = np.array([0, 1, 0], np.int32)
    cam = np.array([2, 0, 2], np.int32)
    with pytest.raises(dba.DbaError) as e:
        dba.dba_block_build_layout(3, 2, pt, cam, 4, 2)
    assert e.value.status == dba.DBA_EINVAL and "observed twice" in str(e.value)


def test_layout_size_limits():
    """The camera word holds 24 bits of camera index; more cameras, or no observations,
    are rejected before any work."""
    pt = np.array([0, 1], np.int32)
    cam = np.array([0, 1], np.int32)
    with pytest.raises(dba.DbaError):
        dba.dba_build_layout(1 << 24, 2, pt, cam, 256)
    L = dba.dba_build_layout((1 << 24) - 1, 2, pt, cam, 256)
    assert list(L["tile_start"]) == [0, 2]
    with pytest.raises(dba.DbaError):
        dba.dba_build_layout(2, 2, np.zeros(0, np.int32), np.zeros(0, np.int32), 256)
