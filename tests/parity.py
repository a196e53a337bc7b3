"""Error measures and block settings shared by the GPU parity tests."""
import numpy as np


def colerr(a, b):
    """Largest per-coordinate relative error of a parameter array against the oracle's b:
    every column (a point coordinate, one Euler angle, one translation component, one slot
    of a copy) is measured against that column's own largest oracle magnitude, so small
    angles are not judged on the scale of large translations."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if b.ndim == 1:
        a, b = a[:, None], b[:, None]
    scale = np.maximum(np.abs(b).max(axis=0), 1e-300)
    err = float((np.abs(a - b).max(axis=0) / scale).max())
    # a NaN anywhere is an infinite error, so that a running max over checks cannot drop it
    return err if np.isfinite(err) else float("inf")


# Block sizes (points, cameras) of the block parity test.  Together they put blocks in every
# kernel variant of the block solve: one-camera blocks in groups of 1, 2, 4, 8, 16 and 32
# lanes; two-camera blocks in groups of 4, 8, 16 and 32 lanes; blocks of up to 4 cameras in
# 32 lanes (the register solve with four camera slots); one-point blocks of two to four
# cameras (cameras eliminated, a thread per block); above 32 points (two point copies a lane,
# the shared-memory kernel).
BLOCK_SETTINGS = [(1, 1), (8, 2), (32, 4), (5, 3), (32, 1), (32, 2), (64, 1), (48, 2), (64, 4), (1, 4)]
