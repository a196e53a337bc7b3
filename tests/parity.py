"""Error measures shared by the GPU parity tests."""
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
    return float((np.abs(a - b).max(axis=0) / scale).max())
