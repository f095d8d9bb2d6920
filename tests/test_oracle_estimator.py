"""Pins for the oracle's norm estimator (Section 3.1), by exhaustive enumeration of sign vectors.

The paper shows E[(b^T s)^2] = sum_i b_i^2 for IID Rademacher s.  Enumerating
every s in {-1,+1}^n on a tiny matrix gives the expectation exactly, so the
oracle's estimator is checked against dense NumPy row and column sums of
|DAE|^2 -- a different computation -- to rounding error.
"""
import itertools

import numpy as np
import pytest

import oracle as O


def _all_signs(n):
    return np.array(list(itertools.product([1.0, -1.0], repeat=n)))


def _tiny(m, n, seed, density=0.8):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < density)
    A[0, 0] = 1.5  # never an all-zero matrix
    u = rng.normal(0, 0.5, m)
    v = rng.normal(0, 0.5, n)
    return A, u, v


def test_row_estimator_is_unbiased_by_enumeration():
    A, u, v = _tiny(3, 10, 0)
    B = np.exp(u)[:, None] * A * np.exp(v)[None, :]
    S = _all_signs(10)
    zs = np.array([O.row_estimate(A, u, v, s[:, None]) for s in S])
    np.testing.assert_allclose(zs.mean(axis=0), (B ** 2).sum(axis=1), rtol=1e-12)


def test_col_estimator_is_unbiased_by_enumeration():
    A, u, v = _tiny(10, 4, 1)
    B = np.exp(u)[:, None] * A * np.exp(v)[None, :]
    W = _all_signs(10)
    zs = np.array([O.col_estimate(A, u, v, w[:, None]) for w in W])
    np.testing.assert_allclose(zs.mean(axis=0), (B ** 2).sum(axis=0), rtol=1e-12)


def test_estimator_variance_closed_form():
    """Var((b^T s)^2) = 2 (sum b^2)^2 - 2 sum b^4, derived directly from the Rademacher moments."""
    A, u, v = _tiny(3, 9, 2)
    B = np.exp(u)[:, None] * A * np.exp(v)[None, :]
    S = _all_signs(9)
    zs = np.array([O.row_estimate(A, u, v, s[:, None]) for s in S])
    r2 = (B ** 2).sum(axis=1)
    np.testing.assert_allclose(zs.var(axis=0), 2 * r2 ** 2 - 2 * (B ** 4).sum(axis=1), rtol=1e-10)


def test_second_moment_identity_of_the_gradient_estimate():
    """E||g~||^2 = ||grad f||^2 + 2 1^T|[r2; c2]|^2 - 4 1^T|DAE|^4 1 by enumeration over (s, w).

    Section 3.2 prints the coefficient 3 on the middle term; the enumeration fixes it at 2
    (the printed 3 is checked to disagree, documenting that reading).
    """
    m, n = 5, 6
    A, u, v = _tiny(m, n, 3)
    alpha, beta, gamma = 0.9, 1.1, 0.1
    B = np.exp(u)[:, None] * A * np.exp(v)[None, :]
    r2, c2 = (B ** 2).sum(1), (B ** 2).sum(0)
    gu = r2 - alpha ** 2 + gamma * u
    gv = c2 - beta ** 2 + gamma * v
    S, W = _all_signs(n), _all_signs(m)
    zu = np.array([O.row_estimate(A, u, v, s[:, None]) for s in S])
    zv = np.array([O.col_estimate(A, u, v, w[:, None]) for w in W])
    e_u = np.mean(np.sum((zu - alpha ** 2 + gamma * u) ** 2, axis=1))
    e_v = np.mean(np.sum((zv - beta ** 2 + gamma * v) ** 2, axis=1))
    lhs = e_u + e_v
    quart = (B ** 4).sum()
    derived = gu @ gu + gv @ gv + 2 * (r2 @ r2 + c2 @ c2) - 4 * quart
    printed = gu @ gu + gv @ gv + 3 * (r2 @ r2 + c2 @ c2) - 4 * quart
    assert lhs == pytest.approx(derived, rel=1e-10)
    assert abs(lhs - printed) > 1e-3 * abs(lhs)


def test_k_probe_estimate_is_the_mean_of_single_probe_estimates():
    A, u, v = _tiny(6, 8, 4)
    rng = np.random.default_rng(5)
    s = rng.choice([-1.0, 1.0], size=(8, 7))
    z = O.row_estimate(A, u, v, s)
    singles = np.array([O.row_estimate(A, u, v, s[:, [p]]) for p in range(7)])
    np.testing.assert_allclose(z, singles.mean(axis=0), rtol=1e-13)
