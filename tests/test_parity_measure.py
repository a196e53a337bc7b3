"""The error measure of the GPU parity tests (tests/parity.py), on the CPU."""
import numpy as np

from parity import colerr


def test_columns_are_measured_on_their_own_scale():
    b = np.array([[1e-2, 100.0], [-2e-2, 50.0]])
    a = b + np.array([[1e-12, 0.0], [0.0, 1e-9]])
    # 1e-12 against the angle column's 2e-2, 1e-9 against the translation column's 100
    assert np.isclose(colerr(a, b), max(1e-12 / 2e-2, 1e-9 / 100.0), rtol=1e-6)
    assert colerr(b[:, 0], b[:, 0]) == 0.0


def test_a_nan_is_an_infinite_error_that_a_running_max_keeps():
    b = np.ones((3, 2))
    a = b.copy()
    a[1, 0] = np.nan
    assert colerr(a, b) == np.inf
    assert colerr(b, a) == np.inf
    assert max(0.0, colerr(a, b), colerr(b, b)) == np.inf
