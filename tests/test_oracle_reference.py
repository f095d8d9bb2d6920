"""Pins for the oracle's exact tools: objective/gradient, the regularised optimum, the
Lambert-W block minimiser, Sinkhorn-Knopp and the condition-number theorems."""
import numpy as np
import pytest

import oracle as O
from paper_1602_06621_gb300 import inputs as I


def test_gradient_matches_finite_differences_of_the_objective():
    A = I.sparse_uniform_density(12, 9, 0.4, seed=2, var=1.0)
    rng = np.random.default_rng(0)
    u, v = rng.normal(0, 0.4, 12), rng.normal(0, 0.4, 9)
    kw = dict(alpha=0.9, beta=1.1, gamma=0.2)
    gu, gv = O.gradient(A, u, v, **kw)
    h = 1e-6
    for i in range(12):
        e = np.zeros(12)
        e[i] = h
        fd = (O.objective(A, u + e, v, **kw) - O.objective(A, u - e, v, **kw)) / (2 * h)
        assert fd == pytest.approx(gu[i], rel=1e-6, abs=1e-7)
    for j in range(9):
        e = np.zeros(9)
        e[j] = h
        fd = (O.objective(A, u, v + e, **kw) - O.objective(A, u, v - e, **kw)) / (2 * h)
        assert fd == pytest.approx(gv[j], rel=1e-6, abs=1e-7)


def test_regularized_optimum_is_stationary_with_equal_scales():
    """Box inactive: grad f = 0 and 1^T u* = 1^T v* (Section 2.3)."""
    A = I.workload_small(1)
    d = O.default_params(A.m, A.n)
    u, v = O.regularized_optimum(A, **d)
    assert max(np.abs(u).max(), np.abs(v).max()) < d["M"]
    gu, gv = O.gradient(A, u, v, alpha=d["alpha"], beta=d["beta"], gamma=d["gamma"])
    assert np.abs(gu).max() < 1e-9 and np.abs(gv).max() < 1e-9
    assert u.sum() == pytest.approx(v.sum(), abs=1e-8)


def test_lambert_w_block_minimiser_zeroes_the_block_gradient():
    A = I.sparse_uniform_density(40, 30, 0.2, seed=8)
    d = O.default_params(40, 30)
    v = np.random.default_rng(1).normal(0, 0.5, 30)
    u = O.block_minimize_u(A, v, alpha=d["alpha"], gamma=d["gamma"], M=np.inf)
    gu, _ = O.gradient(A, u, v, alpha=d["alpha"], beta=d["beta"], gamma=d["gamma"])
    assert np.abs(gu).max() < 1e-10
    u2 = O.block_minimize_u(A, v, alpha=d["alpha"], gamma=d["gamma"], M=d["M"])
    np.testing.assert_allclose(u2, np.clip(u, -d["M"], d["M"]))
    # Tiny gamma: the log-space Lambert W keeps e^{2 alpha^2/gamma} from overflowing.
    u3 = O.block_minimize_u(A, v, alpha=d["alpha"], gamma=1e-4, M=np.inf)
    gu3, _ = O.gradient(A, u3, v, alpha=d["alpha"], beta=d["beta"], gamma=1e-4)
    assert np.all(np.isfinite(u3)) and np.abs(gu3).max() < 1e-9


def test_block_descent_and_newton_agree():
    A = I.sparse_uniform_density(50, 30, 0.2, seed=9, var=1.0)
    d = O.default_params(50, 30)
    un, vn = O.regularized_optimum(A, **d)
    u, v = np.zeros(50), np.zeros(30)
    for _ in range(3000):
        u = O.block_minimize_u(A, v, alpha=d["alpha"], gamma=d["gamma"], M=d["M"])
        v = O.block_minimize_v(A, u, beta=d["beta"], gamma=d["gamma"], M=d["M"])
    np.testing.assert_allclose(u, un, atol=1e-7)
    np.testing.assert_allclose(v, vn, atol=1e-7)


def test_sinkhorn_knopp_equilibrates():
    A = I.small_dense_positive(8, 8, 3)
    d, e = O.sinkhorn_knopp(A)
    B2 = (d[:, None] * A * e[None, :]) ** 2
    np.testing.assert_allclose(B2.sum(1), 1.0, rtol=1e-10)
    np.testing.assert_allclose(B2.sum(0), 1.0, rtol=1e-10)


def test_vanishing_regularisation_reaches_sinkhorn_knopp():
    """M = inf, m = n, alpha = beta = 1: the regularised optimum tends to SK as gamma -> 0 (Section 2.3)."""
    A = I.small_dense_positive(6, 6, 4)
    d, e = O.sinkhorn_knopp(A)
    sk = d[:, None] * A * e[None, :]
    errs = []
    for gamma in (1e-2, 1e-4, 1e-6):
        u, v = O.regularized_optimum(A, alpha=1.0, beta=1.0, gamma=gamma, M=np.inf)
        reg = np.exp(u)[:, None] * A * np.exp(v)[None, :]
        errs.append(np.abs(reg - sk).max() / np.abs(sk).max())
    assert errs[2] < 1e-5
    assert errs[0] > errs[1] > errs[2]


@pytest.mark.parametrize("n,seed", [(2, 0), (5, 1), (12, 2), (30, 3)])
def test_condition_bound_theorem(n, seed):
    """kappa(U) <= 2 e^{-n/2} Phi(U) (Theorem 2.2), in logs."""
    rng = np.random.default_rng(seed)
    for _ in range(20):
        U = rng.standard_normal((n, n)) * np.exp(rng.normal(0, 1, (n, 1)))
        assert np.log(O.kappa(U)) <= np.log(2) - n / 2 + O.log_phi(U) + 1e-9


@pytest.mark.parametrize("n,kap", [(3, 10.0), (8, 1e3), (20, 2.5)])
def test_condition_bound_is_tight_at_the_printed_singular_values(n, kap):
    """Phi = (e^{n/2}/2)(kappa + 1/kappa) at sigma_1, sigma_n of Theorem 2.2's proof, sigma_i = 1 else."""
    rng = np.random.default_rng(n)
    sig = np.ones(n)
    sig[0] = np.sqrt(2 * kap ** 2 / (1 + kap ** 2))
    sig[-1] = np.sqrt(2 / (1 + kap ** 2))
    Q1, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
    U = Q1 @ np.diag(sig) @ Q2.T
    assert O.kappa(U) == pytest.approx(kap, rel=1e-8)
    expect = n / 2 - np.log(2) + np.log(kap + 1 / kap)
    assert O.log_phi(U) == pytest.approx(expect, rel=1e-10, abs=1e-10)
    assert 2 * np.exp(-n / 2 + O.log_phi(U)) <= 2 * kap * (1 + 1e-10)


def test_equilibration_minimises_phi():
    """Theorem 2.1: the SK scaling (alpha = beta = 1) minimises Phi(DAE) over diagonal D, E."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((7, 7)) * np.exp(rng.normal(0, 1, (7, 1))) * np.exp(rng.normal(0, 1, (1, 7)))
    d, e = O.sinkhorn_knopp(np.abs(A))
    best = O.log_phi(d[:, None] * A * e[None, :])
    for _ in range(200):
        dp = d * np.exp(rng.normal(0, 0.3, 7))
        ep = e * np.exp(rng.normal(0, 0.3, 7))
        assert O.log_phi(dp[:, None] * A * ep[None, :]) >= best - 1e-10
