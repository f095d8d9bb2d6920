"""Pins for the oracle's variants of Section 6: varying row/column norms, symmetric equilibration
(Algorithm 2) and block equilibration.

Each variant's stochastic step is pinned by enumeration: its expectation over all sign vectors equals the
exact projected gradient step of the variant's regularised objective, whose gradient is in turn checked
by finite differences of that objective.  Each variant also reduces exactly to Algorithm 1 in the case the
paper describes as its starting point (uniform targets, blocks of size one, v = u).
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_1602_06621_gb300 import inputs as I


def _signs(n):
    return np.array(list(itertools.product([1.0, -1.0], repeat=n)))


def _dense_state(m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.8)
    A[0, 0] = 1.7
    return A, rng


def test_varying_norms_expected_step_and_uniform_case():
    m, n = 5, 6
    A, rng = _dense_state(m, n, 0)
    u, v = rng.normal(0, 0.3, m), rng.normal(0, 0.3, n)
    ub, vb = rng.normal(0, 0.3, m), rng.normal(0, 0.3, n)
    rt = np.exp(rng.normal(0, 0.5, m))
    ct = np.exp(rng.normal(0, 0.5, n))
    ct *= rt.sum() / ct.sum()  # r^T 1 = c^T 1
    gamma, M, t = 0.1, 1e9, 4
    eta = 2.0 / (gamma * (t + 1))
    B = np.exp(u)[:, None] * A * np.exp(v)[None, :]
    S, W = _signs(n), _signs(m)
    us = np.mean([O.psgd_step_targets(A, u, v, ub, vb, s[:, None], np.ones((m, 1)), t, rt=rt, ct=ct, gamma=gamma,
                                      M=M)[0] for s in S], axis=0)
    vs = np.mean([O.psgd_step_targets(A, u, v, ub, vb, np.ones((n, 1)), w[:, None], t, rt=rt, ct=ct, gamma=gamma,
                                      M=M)[1] for w in W], axis=0)
    np.testing.assert_allclose(us, u - eta * ((B ** 2).sum(1) - rt + gamma * u), rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(vs, v - eta * ((B ** 2).sum(0) - ct + gamma * v), rtol=1e-11, atol=1e-11)
    # Uniform targets alpha^2, beta^2 reproduce Algorithm 1 exactly.
    s, w = O.probe_signs(1, t, 0, n, 3), O.probe_signs(1, t, 1, m, 3)
    a, b = 0.8, 1.2
    got = O.psgd_step_targets(A, u, v, ub, vb, s, w, t, rt=np.full(m, a * a), ct=np.full(n, b * b), gamma=gamma, M=M)
    ref = O.psgd_step(A, u, v, ub, vb, s, w, t, alpha=a, beta=b, gamma=gamma, M=M)
    for x, y in zip(got, ref):
        np.testing.assert_array_equal(x, y)


def _sym_objective(A, u, alpha, gamma):
    """(1/4) sum_ij A_ij^2 e^{2u_i + 2u_j} - alpha^2 1^T u + (gamma/2) ||u||^2 (the regularised symmetric problem)."""
    return 0.25 * np.sum(A ** 2 * np.exp(2 * u[:, None] + 2 * u[None, :])) - alpha ** 2 * u.sum() + 0.5 * gamma * u @ u


def test_symmetric_expected_step_is_the_gradient_step():
    n = 6
    A0, rng = _dense_state(n, n, 1)
    A = A0 + A0.T
    u, ub = rng.normal(0, 0.3, n), rng.normal(0, 0.3, n)
    alpha, gamma, M, t = 1.0, 0.1, 1e9, 3
    h = 1e-6
    grad = np.array([(_sym_objective(A, u + h * e, alpha, gamma) - _sym_objective(A, u - h * e, alpha, gamma)) / (2 * h)
                     for e in np.eye(n)])
    Bs = np.exp(u)[:, None] * A * np.exp(u)[None, :]
    np.testing.assert_allclose(grad, (Bs ** 2).sum(1) - alpha ** 2 + gamma * u, rtol=1e-6, atol=1e-6)
    us = np.mean([O.psgd_step_symmetric(A, u, ub, s[:, None], t, alpha=alpha, gamma=gamma, M=M)[0]
                  for s in _signs(n)], axis=0)
    eta = 2.0 / (gamma * (t + 1))
    np.testing.assert_allclose(us, u - eta * ((Bs ** 2).sum(1) - alpha ** 2 + gamma * u), rtol=1e-11, atol=1e-11)
    # Algorithm 2 is the u-part of Algorithm 1 evaluated at v = u.
    s = O.probe_signs(2, t, 0, n, 4)
    got = O.psgd_step_symmetric(A, u, ub, s, t, alpha=alpha, gamma=gamma, M=M)
    ref = O.psgd_step(A, u, u, ub, ub, s, np.ones((n, 4)), t, alpha=alpha, beta=alpha, gamma=gamma, M=M)
    np.testing.assert_array_equal(got[0], ref[0])
    np.testing.assert_array_equal(got[1], ref[2])


def _block_objective(A, rb, cb, ubk, vbk, alpha, beta, gamma):
    u = np.repeat(ubk, np.diff(rb))
    v = np.repeat(vbk, np.diff(cb))
    return (0.5 * np.sum(A ** 2 * np.exp(2 * u[:, None] + 2 * v[None, :])) - alpha ** 2 * ubk @ np.diff(rb)
            - beta ** 2 * vbk @ np.diff(cb) + 0.5 * gamma * (ubk @ ubk + vbk @ vbk))


def test_block_expected_step_and_singleton_blocks():
    m, n = 6, 5
    A, rng = _dense_state(m, n, 2)
    rb, cb = np.array([0, 2, 3, 6]), np.array([0, 1, 5])
    ubk, vbk = rng.normal(0, 0.3, 3), rng.normal(0, 0.3, 2)
    ubb, vbb = rng.normal(0, 0.3, 3), rng.normal(0, 0.3, 2)
    alpha, beta, gamma, M, t = 0.9, 1.1, 0.1, 1e9, 2
    h = 1e-6
    gu = np.array([(_block_objective(A, rb, cb, ubk + h * e, vbk, alpha, beta, gamma)
                    - _block_objective(A, rb, cb, ubk - h * e, vbk, alpha, beta, gamma)) / (2 * h) for e in np.eye(3)])
    gv = np.array([(_block_objective(A, rb, cb, ubk, vbk + h * e, alpha, beta, gamma)
                    - _block_objective(A, rb, cb, ubk, vbk - h * e, alpha, beta, gamma)) / (2 * h) for e in np.eye(2)])
    u = np.repeat(ubk, np.diff(rb))
    v = np.repeat(vbk, np.diff(cb))
    B2 = (np.exp(u)[:, None] * A * np.exp(v)[None, :]) ** 2
    r, c = B2.sum(1), B2.sum(0)
    exact_gu = np.add.reduceat(r, rb[:-1]) - alpha ** 2 * np.diff(rb) + gamma * ubk
    exact_gv = np.add.reduceat(c, cb[:-1]) - beta ** 2 * np.diff(cb) + gamma * vbk
    np.testing.assert_allclose(gu, exact_gu, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(gv, exact_gv, rtol=1e-6, atol=1e-6)
    kw = dict(alpha=alpha, beta=beta, gamma=gamma, M=M)
    eta = 2.0 / (gamma * (t + 1))
    us = np.mean([O.block_step(A, rb, cb, ubk, vbk, ubb, vbb, s[:, None], np.ones((m, 1)), t, **kw)[0]
                  for s in _signs(n)], axis=0)
    vs = np.mean([O.block_step(A, rb, cb, ubk, vbk, ubb, vbb, np.ones((n, 1)), w[:, None], t, **kw)[1]
                  for w in _signs(m)], axis=0)
    np.testing.assert_allclose(us, ubk - eta * exact_gu, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(vs, vbk - eta * exact_gv, rtol=1e-11, atol=1e-11)
    # Blocks of one row / one column each: Algorithm 1 itself.
    A2 = I.sparse_uniform_density(30, 20, 0.2, seed=3)
    d = O.default_params(30, 20)
    s, w = O.probe_signs(4, 1, 0, 20, 8), O.probe_signs(4, 1, 1, 30, 8)
    z = lambda k_: np.zeros(k_)
    got = O.block_step(A2, np.arange(31), np.arange(21), z(30), z(20), z(30), z(20), s, w, 1, **d)
    ref = O.psgd_step(A2, z(30), z(20), z(30), z(20), s, w, 1, **d)
    for x, y in zip(got, ref):
        np.testing.assert_array_equal(x, y)
