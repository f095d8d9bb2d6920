"""Pins for the oracle's Chambolle-Cremers-Pock Lasso solver (Section 5.2).

The two proximal maps are checked against direct numerical minimisation of their definitions; the solver's
fixed point against the closed-form Lasso solution of a diagonal matrix, the Lasso optimality (KKT)
conditions, scikit-learn's coordinate-descent Lasso, and its invariance under the diagonal scaling (the
minimiser of the original problem does not depend on D, E); the power iteration against the SVD.
"""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import oracle as O
from oracle import ccp as C
from paper_1602_06621_gb300 import inputs as I


def test_prox_maps_minimise_their_definitions():
    rng = np.random.default_rng(0)
    lam, sigma, tau = 0.37, 0.8, 0.6
    for _ in range(20):
        w, d, b = rng.normal(0, 2), np.exp(rng.normal(0, 1)), rng.normal(0, 2)
        # prox_{F/sigma}(w/sigma) by direct minimisation, then Moreau's identity.
        p = w / sigma
        y = minimize_scalar(lambda t: (t / d - b) ** 2 / np.sqrt(lam) + 0.5 * sigma * (t - p) ** 2,
                            bracket=(-1e3, 1e3), tol=1e-14).x
        assert C.prox_f_conj(np.array([w]), np.array([d]), np.array([b]), sigma, lam)[0] == \
            pytest.approx(w - sigma * y, rel=1e-6, abs=1e-8)
        z, e = rng.normal(0, 1), np.exp(rng.normal(0, 1))
        t = tau * np.sqrt(lam) * e
        xs = minimize_scalar(lambda q: t * abs(q) + 0.5 * (q - z) ** 2, bounds=(-10, 10), method="bounded",
                             options={"xatol": 1e-12}).x
        assert C.prox_g(np.array([z]), np.array([t]))[0] == pytest.approx(xs, abs=1e-6)


def test_power_norm_is_the_largest_singular_value():
    A = I.sparse_uniform_density(60, 40, 0.2, seed=1)
    K, _, _ = C.scaled_operator(A, np.random.default_rng(1).normal(0, 0.3, 60),
                                np.random.default_rng(2).normal(0, 0.3, 40))
    assert C.power_norm(K, 2000) == pytest.approx(np.linalg.norm(K.toarray(), 2), rel=1e-9)


def test_diagonal_lasso_closed_form():
    """A = diag(a): minimise sum (a_j x_j - b_j)^2 + lam |x_j| -> x_j = soft(b_j / a_j, lam / (2 a_j^2))."""
    rng = np.random.default_rng(3)
    n = 12
    a = np.exp(rng.normal(0, 0.5, n))
    b = rng.normal(0, 1, n)
    lam = 0.3
    c = b / a
    exact = np.sign(c) * np.maximum(np.abs(c) - lam / (2 * a * a), 0)
    assert np.count_nonzero(exact) not in (0, n)
    x, _, _ = C.ccp_lasso(np.diag(a), b, lam, iters=4000)
    np.testing.assert_allclose(x, exact, atol=1e-9)


def _problem(seed, m=80, n=160):
    """Section 5.2's recipe at small size: A as in Section 4, x_hat with n/10 nonzeros, b = A x_hat + noise."""
    A = I.sparse_uniform_density(m, n, 0.1, seed, mean=1.0, var=1.0)
    rng = np.random.default_rng(seed + 100)
    xh = np.zeros(n)
    idx = rng.choice(n, n // 10, replace=False)
    xh[idx] = rng.standard_normal(idx.size)
    S = C._matrix(A)
    b = S @ xh + rng.standard_normal(m)
    return A, b, C.default_lambda(A, b)


def test_fixed_point_satisfies_kkt_and_matches_sklearn():
    A, b, lam = _problem(4)
    x, hist, _ = C.ccp_lasso(A, b, lam, iters=60000, check_every=1000)
    assert C.lasso_kkt_residual(A, x, b, lam) < 1e-6
    assert all(h1 <= h0 * (1 + 1e-12) for h0, h1 in zip(hist[-10:], hist[-9:]))
    sk = pytest.importorskip("sklearn.linear_model")
    ref = sk.Lasso(alpha=lam / (2 * A.m), fit_intercept=False, tol=1e-14, max_iter=1000000).fit(
        C._matrix(A).toarray(), b).coef_
    np.testing.assert_allclose(x, ref, atol=1e-6 * max(1.0, np.abs(ref).max()))


def test_scaling_leaves_the_minimiser_unchanged():
    A, b, lam = _problem(5)
    rng = np.random.default_rng(6)
    u, v = rng.normal(0, 0.3, A.m), rng.normal(0, 0.3, A.n)
    x0, _, _ = C.ccp_lasso(A, b, lam, iters=100000)
    x1, _, _ = C.ccp_lasso(A, b, lam, iters=100000, u=u, v=v)
    assert C.lasso_kkt_residual(A, x1, b, lam) < 1e-6
    np.testing.assert_allclose(x1, x0, atol=1e-6 * max(1.0, np.abs(x0).max()))


def test_equilibration_speeds_up_ccp():
    """Section 5.2's trend at reduced size: with the scalings of 100 iterations of Algorithm 1, CCP reaches a
    relative gap of 1e-6 in fewer iterations than without (here 180 against 700; the paper reports more than
    4x at 1e4 x 2e4)."""
    A, b, lam = _problem(7, m=200, n=400)
    d = O.default_params(A.m, A.n)
    _, _, ub, vb = O.equilibrate(A, T=100, k=1, seed=0, **d)
    xs, _, _ = C.ccp_lasso(A, b, lam, iters=100000, u=ub, v=vb)
    pstar = C.lasso_objective(A, xs, b, lam)

    def iters_to(h, f0, tol=1e-6):
        for i, f in enumerate(h):
            if (f - pstar) / f0 <= tol:
                return i * 10
        return None

    _, h0, _ = C.ccp_lasso(A, b, lam, iters=20000, check_every=10)
    _, h1, _ = C.ccp_lasso(A, b, lam, iters=20000, check_every=10, u=ub, v=vb)
    n0, n1 = iters_to(h0, h0[0]), iters_to(h1, h1[0])
    assert n1 is not None and (n0 is None or 2 * n1 < n0), (n0, n1)
