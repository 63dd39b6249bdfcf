"""The parity rules every GPU test applies (tests/_gpu_helpers.py) accept what
they should and reject what they should, checked on the CPU with planted
differences: a changed cell outside a near-tie, a near-tie row whose choice is
not within the tolerance of the minimum, codebook and distortion errors just
past their tolerances."""
import numpy as np
import pytest

import oracle
from _gpu_helpers import C_TOL, D_TOL, GAP_TOL, check_assign, check_codebook, check_D


def _problem():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((400, 3)).astype(np.float32)
    C = rng.standard_normal((12, 3)).astype(np.float32)
    a, e, gap = oracle.assign(X, C.astype(np.float64))
    return X, C, a, e, gap


def test_identical_assignments_pass():
    X, C, a, e, gap = _problem()
    assert check_assign(X, C, a.copy(), a, e, gap) == 0


def test_changed_cell_outside_a_near_tie_fails():
    X, C, a, e, gap = _problem()
    m = int(np.flatnonzero(gap > GAP_TOL)[0])
    bad = a.copy()
    bad[m] = (a[m] + 1) % C.shape[0]
    with pytest.raises(AssertionError):
        check_assign(X, C, bad, a, e, gap)


def test_near_tie_rows_may_take_either_member():
    """Row 0 equidistant from codevectors 0 and 1 (gap 0): either choice passes;
    a third, farther codevector does not."""
    X = np.array([[0.0, 0.0], [5.0, 5.0]], np.float32)
    C = np.array([[1.0, 0.0], [0.0, 1.0], [3.0, 3.0]], np.float32)
    a, e, gap = oracle.assign(X, C.astype(np.float64))
    assert a[0] == 0 and gap[0] == 0.0
    assert check_assign(X, C, np.array([1, a[1]]), a, e, gap) == 1
    with pytest.raises(AssertionError):
        check_assign(X, C, np.array([2, a[1]]), a, e, gap)


def test_codebook_and_distortion_tolerances():
    C = np.array([[100.0, -3.0], [0.5, 0.25]])
    check_codebook(C * (1 + 0.5 * C_TOL), C)
    with pytest.raises(AssertionError):
        check_codebook(C + np.array([[0.0, 0.0], [2 * C_TOL, 0.0]]), C)   # |c| < 1: absolute
    check_D(1.0 + 0.5 * D_TOL, 1.0)
    with pytest.raises(AssertionError):
        check_D(1.0 + 2 * D_TOL, 1.0)
    check_D(0.0, 0.0)
    with pytest.raises(AssertionError):
        check_D(1e-30, 0.0)
