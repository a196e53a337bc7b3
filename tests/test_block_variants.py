"""The block parity test reaches every kernel variant of the block solve.

The library orders each size class of the block list by point count and solves a block
with the kernel chosen by its cameras and points: one camera and at most 8 points in a
group of 1, 2, 4 or 8 lanes (the smallest that holds its points); otherwise, at most 2
cameras and 16 points in a group of 4, 8 or 16 lanes (two cameras: the register
reduce-scatter solve; one camera when every block has one: the one-camera solve); at most
32 points in 32 lanes (the two-camera solve when block_cams = 2, the same register solve
with four camera slots when block_cams >= 3); above that two point copies a lane, in the
shared-memory solve.  Blocks of one point and two to four cameras eliminate their cameras
instead, a thread per block.  This recounts, from the
oracle's block layout of the parity test's scene, which variants its settings reach."""
import numpy as np

import oracle as O
from parity import BLOCK_SETTINGS
from paper_1708_07954_gb300 import scenes as S


def variant(n_pts, n_cams, kappa):
    width = 1
    while width < n_pts:
        width *= 2
    if n_cams == 1 and n_pts <= 8:
        return ("one camera", width)
    if n_pts == 1:
        return ("one point", 1)
    if n_cams <= 2 and n_pts <= 16:
        return ("one camera" if kappa == 1 else "two cameras", max(width, 4 if kappa > 1 else 16))
    if n_pts <= 32:
        return ("one camera" if kappa == 1 else "two cameras" if kappa == 2 else "four cameras", 32)
    return ("shared memory, two copies a lane", 32)


def test_block_parity_settings_reach_every_kernel_variant():
    sc = S.scene1(n_pts=400, n_cams=16, seed=17)  # the scene of the block parity test
    seen = set()
    for pi, kappa in BLOCK_SETTINGS:
        L = O.BlockLayout(sc, pi, kappa)
        for n_p, n_c in zip(np.diff(L.pc_off), np.diff(L.cc_off)):
            seen.add(variant(int(n_p), int(n_c), kappa))
    want = {("one camera", w) for w in (1, 2, 4, 8, 16, 32)}
    want |= {("two cameras", w) for w in (4, 8, 16, 32)}
    want |= {("four cameras", 32), ("shared memory, two copies a lane", 32), ("one point", 1)}
    assert want <= seen, sorted(want - seen)


def test_block_parity_settings_reach_one_camera_blocks_in_the_two_camera_solve():
    """With block_cams >= 2, a block of one camera and more than 8 points takes the
    two-camera solve, its 12 x 12 system padded by identity rows: the parity settings
    put such blocks in both the 16- and the 32-lane groups."""
    sc = S.scene1(n_pts=400, n_cams=16, seed=17)
    seen = set()
    for pi, kappa in BLOCK_SETTINGS:
        L = O.BlockLayout(sc, pi, kappa)
        for n_p, n_c in zip(np.diff(L.pc_off), np.diff(L.cc_off)):
            v = variant(int(n_p), int(n_c), kappa)
            if v[0] == "two cameras" and n_c == 1:
                seen.add(v[1])
    assert {16, 32} <= seen, sorted(seen)
