"""Pins for the oracle functions the GPU tests use as checkers.

Each function here is compared with something other than itself, and every
case is chosen so that a plausible slip fails it:

* dense_estimate_sampled (Section 3.1 estimator on dense A) equals the CSR
  estimators -- which are pinned by enumeration of every sign vector -- on the
  same matrix with the row scales folded into A, with signs drawn for the
  stream pair (stream_base, stream_base + 1).  A misplaced row scale, swapped
  s/w streams or an ignored stream_base changes the result.
* psgd_step_sampled (Algorithm 1 at a subset of indices) equals the full step
  psgd_step -- pinned by the exact-gradient and averaging tests -- at the
  sampled indices, with a nonzero stream_base, t0 and running averages.
* exact_norms_sq (Section 2.1) equals dense NumPy row and column sums of
  |DAE|^2 and a 2 x 2 case worked by hand.
* rms_error (the RMS equilibration error printed in Section 4) and spread
  (max/min of the l2 norms over the nonempty rows and columns) are checked on
  cases worked by hand.
"""
import math

import numpy as np
import pytest

import oracle as O


def _rand_dense(m, n, seed, density=0.7):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((m, n)) * (rng.random((m, n)) < density)).astype(np.float32)
    A[0, 0] = np.float32(1.25)
    u = rng.normal(0, 0.4, m)
    v = rng.normal(0, 0.4, n)
    return A, u, v, rng


# ------------------------------------------------------------------ dense_estimate_sampled

@pytest.mark.parametrize("k", [4, 64])
@pytest.mark.parametrize("stream_base", [0, 6])
@pytest.mark.parametrize("scaled", [False, True])
def test_dense_sampled_estimate_equals_csr_estimators(k, stream_base, scaled):
    m, n, seed, t = 40, 24, 11, 5
    A, u, v, rng = _rand_dense(m, n, 100 + k + stream_base)
    c = rng.uniform(0.25, 4.0, m) if scaled else None
    folded = A.astype(np.float64) * (c[:, None] if scaled else 1.0)
    s = O.probe_signs(seed, t, stream_base, n, k)
    w = O.probe_signs(seed, t, stream_base + 1, m, k)
    zu_ref = O.row_estimate(folded, u, v, s)
    zv_ref = O.col_estimate(folded, u, v, w)
    rows = np.array([0, 3, 17, 39])
    cols = np.array([0, 5, 23])
    zu, zv = O.dense_estimate_sampled(A, u, v, rows, cols, t=t, k=k, seed=seed, stream_base=stream_base,
                                      row_scale=c)
    np.testing.assert_allclose(zu, zu_ref[rows], rtol=1e-13, atol=1e-13 * zu_ref.max())
    np.testing.assert_allclose(zv, zv_ref[cols], rtol=1e-13, atol=1e-13 * zv_ref.max())


def test_dense_sampled_estimate_uses_the_probe_streams_it_names():
    """Swapping the s and w streams, or dropping stream_base, gives a different estimate."""
    m, n, seed, t, k = 40, 24, 3, 2, 8
    A, u, v, _ = _rand_dense(m, n, 7)
    Ad = A.astype(np.float64)
    rows, cols = np.arange(m), np.arange(n)
    zu, zv = O.dense_estimate_sampled(A, u, v, rows, cols, t=t, k=k, seed=seed, stream_base=2)
    swapped_u = O.row_estimate(Ad, u, v, O.probe_signs(seed, t, 3, n, k))
    swapped_v = O.col_estimate(Ad, u, v, O.probe_signs(seed, t, 2, m, k))
    base0_u = O.row_estimate(Ad, u, v, O.probe_signs(seed, t, 0, n, k))
    assert np.max(np.abs(zu - swapped_u) / zu) > 1e-3
    assert np.max(np.abs(zv - swapped_v) / zv) > 1e-3
    assert np.max(np.abs(zu - base0_u) / zu) > 1e-3


# ------------------------------------------------------------------ psgd_step_sampled

@pytest.mark.parametrize("stream_base,t,t0,M", [(0, 1, 0, 2.0), (4, 3, 60, 1e3), (10, 6, 200, 1e3)])
def test_sampled_step_equals_full_step(stream_base, t, t0, M):
    """The first case saturates the box (step 1/gamma); the others keep every coordinate inside it."""
    rng = np.random.default_rng(20 + t)
    m, n, k, seed = 30, 22, 5, 99
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.3)
    A[0, :] = 0.0  # an empty row
    A[:, 1] = 0.0  # an empty column
    A[2, 3] = 1.0
    u, v = rng.normal(0, 0.3, m), rng.normal(0, 0.3, n)
    ub, vb = rng.normal(0, 0.5, m), rng.normal(0, 0.5, n)  # nonzero averages: the ubar term is exercised
    kw = dict(alpha=0.9, beta=1.1, gamma=0.1, M=M, t0=t0)
    s = O.probe_signs(seed, t, stream_base, n, k)
    w = O.probe_signs(seed, t, stream_base + 1, m, k)
    u1, v1, ub1, vb1 = O.psgd_step(A, u, v, ub, vb, s, w, t, **kw)
    rows = np.array([0, 2, 5, 29])
    cols = np.array([1, 3, 4, 21])
    uo, ubo, vo, vbo = O.psgd_step_sampled(A, u, v, ub, vb, rows, cols, t, k=k, seed=seed,
                                           stream_base=stream_base, **kw)
    np.testing.assert_allclose(uo, u1[rows], rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(ubo, ub1[rows], rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(vo, v1[cols], rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(vbo, vb1[cols], rtol=1e-13, atol=1e-14)


def test_sampled_step_follows_equilibrate_from_a_resumed_state():
    """Two iterations of equilibrate with stream_base 8, then the third sampled == the third run in full."""
    rng = np.random.default_rng(5)
    m, n, k, seed = 25, 18, 3, 4
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.4)
    A[0, 0] = 1.0
    kw = dict(alpha=0.8, beta=1.2, gamma=0.1, M=1e3, t0=100)
    st = O.equilibrate(A, T=2, k=k, seed=seed, stream_base=8, **kw)
    full = O.equilibrate(A, T=1, k=k, seed=seed, stream_base=8, t_begin=3, state=st, **kw)
    rows, cols = np.arange(m), np.arange(n)
    uo, ubo, vo, vbo = O.psgd_step_sampled(A, *st, rows, cols, 3, k=k, seed=seed, stream_base=8, **kw)
    assert np.all(np.abs(full[0]) < 10) and np.all(np.abs(full[1]) < 10)  # box inactive
    for a, b in ((uo, full[0]), (vo, full[1]), (ubo, full[2]), (vbo, full[3])):
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-14)


# ------------------------------------------------------------------ exact_norms_sq

def test_exact_norms_hand_computed_2x2():
    # D = diag(2, 1), E = diag(1, 3): DAE = [[2, 12], [0, 9]].
    A = np.array([[1.0, 2.0], [0.0, 3.0]])
    u = np.array([math.log(2.0), 0.0])
    v = np.array([0.0, math.log(3.0)])
    r2, c2 = O.exact_norms_sq(A, u, v)
    np.testing.assert_allclose(r2, [148.0, 81.0], rtol=1e-14)
    np.testing.assert_allclose(c2, [4.0, 225.0], rtol=1e-14)


def test_exact_norms_equal_dense_sums():
    rng = np.random.default_rng(8)
    m, n = 37, 23
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.3)
    A[4, :] = 0.0
    u, v = rng.normal(0, 0.7, m), rng.normal(0, 0.7, n)
    B = np.exp(u)[:, None] * A * np.exp(v)[None, :]
    r2, c2 = O.exact_norms_sq(A, u, v)
    np.testing.assert_allclose(r2, (B * B).sum(axis=1), rtol=1e-13)
    np.testing.assert_allclose(c2, (B * B).sum(axis=0), rtol=1e-13)
    assert r2[4] == 0.0


# ------------------------------------------------------------------ rms_error, spread

def test_rms_error_hand_computed():
    # norms: rows 2, 1 (targets alpha = 1), column 3 (target beta = 2):
    # ((2-1)^2 + (1-1)^2 + (3-2)^2)^(1/2) / (m+n)^(1/2) = sqrt(2) / sqrt(3).
    assert O.rms_error(np.array([4.0, 1.0]), np.array([9.0]), 1.0, 2.0) == pytest.approx(math.sqrt(2.0 / 3.0),
                                                                                         rel=1e-15)
    # equilibrated: every row norm alpha, every column norm beta.
    assert O.rms_error(np.full(5, 0.49), np.full(3, 1.44), 0.7, 1.2) == pytest.approx(0.0, abs=1e-15)


def test_spread_excludes_empty_rows_and_columns():
    r2 = np.array([4.0, 0.0, 16.0])        # row norms 2, (empty), 4
    c2 = np.array([1.0, 9.0, 0.0, 0.25])   # column norms 1, 3, (empty), 0.5
    rs, cs = O.spread(r2, c2)
    assert rs == pytest.approx(2.0, rel=1e-15)
    assert cs == pytest.approx(6.0, rel=1e-15)


def test_spread_of_equilibrated_matrix_is_one():
    # A permutation matrix times 3: every row and column norm is 3.
    A = 3.0 * np.eye(6)[[2, 0, 5, 1, 4, 3]]
    r2, c2 = O.exact_norms_sq(A, np.zeros(6), np.zeros(6))
    assert O.spread(r2, c2) == (1.0, 1.0)


# ------------------------------------------------------------------ the OpenMP build of the same source

def test_openmp_build_gives_the_checker_bits():
    """The timed CPU baseline runs an OpenMP build of the oracle; it must compute exactly what the checker does."""
    import os
    import subprocess
    import sys

    code = r"""
import numpy as np, oracle as O
from paper_1602_06621_gb300 import inputs as I
A = O.OracleCSR.from_any(I.workload_large(scale=0.003, seed=9))
out = []
for par in (False, True):
    O.set_parallel(par)
    st = O.equilibrate(A, T=3, k=8, seed=2)
    out.append(np.concatenate(st))
print(O.threads(), int(np.array_equal(out[0], out[1])))
"""
    env = dict(os.environ, OMP_NUM_THREADS="4")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    nthreads, same = map(int, r.stdout.split())
    assert nthreads == 4
    assert same == 1
