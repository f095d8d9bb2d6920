"""Pins for the oracle's Algorithm 1 (Section 3.2).

* The expected one-step map equals the exact projected gradient step: averaging
  u^t over every sign vector s gives u^{t-1} - eta_t grad_u f(u^{t-1}, v^{t-1})
  with grad_u f = |DAE|^2 1 - alpha^2 + gamma u (Section 3.1), computed here by
  dense NumPy.  The v-step uses the previous u (D is formed once at the top of
  the iteration), which this also pins.
* Projection, averaging weights, iterate bounds, resume and the
  regularised optimum are pinned by properties the paper states.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_1602_06621_gb300 import inputs as I


def _all_signs(n):
    return np.array(list(itertools.product([1.0, -1.0], repeat=n)))


def _state(m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.8)
    A[0, 0] = 2.0
    return A, rng.normal(0, 0.3, m), rng.normal(0, 0.3, n), rng.normal(0, 0.3, m), rng.normal(0, 0.3, n)


@pytest.mark.parametrize("t,t0", [(1, 0), (3, 0), (7, 5)])
def test_expected_step_is_the_exact_gradient_step(t, t0):
    m, n = 5, 6
    A, u, v, ub, vb = _state(m, n, 10 + t)
    alpha, beta, gamma, M = 0.8, 1.2, 0.1, 1e9
    B = np.exp(u)[:, None] * A * np.exp(v)[None, :]
    grad_u = (B ** 2).sum(1) - alpha ** 2 + gamma * u
    grad_v = (B ** 2).sum(0) - beta ** 2 + gamma * v
    eta = 2.0 / (gamma * (t + t0 + 1))
    kw = dict(alpha=alpha, beta=beta, gamma=gamma, M=M, t0=t0)
    w_fixed = np.ones((m, 1))
    s_fixed = np.ones((n, 1))
    us = np.array([O.psgd_step(A, u, v, ub, vb, s[:, None], w_fixed, t, **kw)[0] for s in _all_signs(n)])
    vs = np.array([O.psgd_step(A, u, v, ub, vb, s_fixed, w[:, None], t, **kw)[1] for w in _all_signs(m)])
    np.testing.assert_allclose(us.mean(0), u - eta * grad_u, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(vs.mean(0), v - eta * grad_v, rtol=1e-11, atol=1e-11)


def test_first_step_from_zero_discards_the_start():
    """At t=1, eta = 1/gamma, so u^1 = Pi((alpha^2 - z)/gamma): u^0 enters only through z."""
    A = I.sparse_uniform_density(30, 20, 0.2, seed=3)
    d = O.default_params(30, 20)
    s = O.probe_signs(0, 1, 0, 20, 4)
    w = O.probe_signs(0, 1, 1, 30, 4)
    z = O.row_estimate(A, np.zeros(30), np.zeros(20), s)
    u1 = O.psgd_step(A, np.zeros(30), np.zeros(20), np.zeros(30), np.zeros(20), s, w, 1, **d)[0]
    np.testing.assert_allclose(u1, np.clip((d["alpha"] ** 2 - z) / d["gamma"], -d["M"], d["M"]), rtol=1e-13)


def test_projection_is_the_clip_of_the_unprojected_step():
    m, n = 7, 9
    A, u, v, ub, vb = _state(m, n, 21)
    A *= 5.0
    s = O.probe_signs(3, 2, 0, n, 2)
    w = O.probe_signs(3, 2, 1, m, 2)
    kw = dict(alpha=1.0, beta=1.0, gamma=0.1, t0=0)
    free = O.psgd_step(A, u, v, ub, vb, s, w, 2, M=1e9, **kw)
    boxed = O.psgd_step(A, u, v, ub, vb, s, w, 2, M=0.5, **kw)
    assert np.any(np.abs(free[0]) > 0.5)  # the box is active somewhere
    np.testing.assert_array_equal(boxed[0], np.clip(free[0], -0.5, 0.5))
    np.testing.assert_array_equal(boxed[1], np.clip(free[1], -0.5, 0.5))


def test_running_average_matches_the_printed_weights():
    """ubar after T steps = sum_t 2(t+1)/((T+1)(T+2)) u^t (Section 3.2; u^0 = 0 adds nothing)."""
    A = I.sparse_uniform_density(40, 25, 0.2, seed=4)
    d = O.default_params(40, 25)
    u, v, ub, vb = np.zeros(40), np.zeros(25), np.zeros(40), np.zeros(25)
    T = 13
    us, vs = [], []
    for t in range(1, T + 1):
        s = O.probe_signs(9, t, 0, 25, 3)
        w = O.probe_signs(9, t, 1, 40, 3)
        u, v, ub, vb = O.psgd_step(A, u, v, ub, vb, s, w, t, **d)
        us.append(u)
        vs.append(v)
    wts = np.array([2.0 * (t + 1) / ((T + 1) * (T + 2)) for t in range(1, T + 1)])
    np.testing.assert_allclose(ub, wts @ np.array(us), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(vb, wts @ np.array(vs), rtol=1e-12, atol=1e-14)
    # Equilibrate() with the same seed reproduces the same loop.
    got = O.equilibrate(A, T=T, k=3, seed=9)
    np.testing.assert_array_equal(got[2], ub)


def test_iterate_upper_bounds():
    """u^t_i <= alpha^2/gamma and v^t_j <= beta^2/gamma for every t (Section 3.2)."""
    A = I.workload_small(1)
    d = O.default_params(A.m, A.n)
    d["M"] = 1e9
    state = None
    for t in range(1, 41):
        state = O.equilibrate(A, T=1, k=1, seed=0, t_begin=t, state=state, **d)
        assert state[0].max() <= d["alpha"] ** 2 / d["gamma"] + 1e-12
        assert state[1].max() <= d["beta"] ** 2 / d["gamma"] + 1e-12


def test_resume_is_bitwise_identical():
    A = I.workload_small(1)
    full = O.equilibrate(A, T=20, k=2, seed=5)
    half = O.equilibrate(A, T=8, k=2, seed=5)
    rest = O.equilibrate(A, T=12, k=2, seed=5, t_begin=9, state=half)
    for a, b in zip(full, rest):
        np.testing.assert_array_equal(a, b)


def test_default_targets_balance():
    """m alpha^2 = n beta^2 (Section 1) holds for the Section 4 defaults."""
    for m, n in [(2000, 1000), (7, 13), (1_000_000, 500_000)]:
        d = O.default_params(m, n)
        assert m * d["alpha"] ** 2 == pytest.approx(n * d["beta"] ** 2, rel=1e-14)
        assert d["M"] == pytest.approx(math.log(1e4))


def test_converges_toward_the_regularized_optimum():
    A = I.sparse_uniform_density(60, 40, 0.3, seed=6, var=1.0)
    d = O.default_params(60, 40)
    us, vs = O.regularized_optimum(A, **d)
    fstar = O.objective(A, us, vs, alpha=d["alpha"], beta=d["beta"], gamma=d["gamma"])
    gaps = []
    for T in (50, 200, 800):
        _, _, ub, vb = O.equilibrate(A, T=T, k=8, seed=1)
        gaps.append(O.objective(A, ub, vb, alpha=d["alpha"], beta=d["beta"], gamma=d["gamma"]) - fstar)
    assert all(g > -1e-9 for g in gaps)
    # O(1/t) or faster: quadrupling T cuts the gap by at least 2x each time.
    assert gaps[1] < gaps[0] / 2 and gaps[2] < gaps[1] / 2
    _, _, ub, vb = O.equilibrate(A, T=3000, k=8, seed=1)
    err = np.linalg.norm(np.concatenate([ub - us, vb - vs])) / np.linalg.norm(np.concatenate([us, vs]))
    assert err < 0.02
