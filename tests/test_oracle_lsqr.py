"""Pins for the oracle's LSQR (Paige & Saunders 1982; used as in Section 5.1)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from paper_1602_06621_gb300 import inputs as I


def _system(m, n, seed, density=0.05):
    A = I.sparse_uniform_density(m, n, density, seed=seed, var=0.5)
    S = sp.csr_matrix((A.vals, A.col_idx, A.row_ptr), shape=(m, n))
    return A, S


@pytest.mark.parametrize("iters", [1, 4, 8])
def test_iterates_match_scipy_lsqr(iters):
    """Early iterates agree to rounding; later ones drift apart as Lanczos amplifies rounding order."""
    A, S = _system(120, 40, 3, density=0.3)
    b = I.normal_vector(120, 4)
    ours = O.lsqr(lambda x: S @ x, lambda y: S.T @ y, b, 40, max_iters=iters)
    ref = spla.lsqr(S, b, atol=0.0, btol=0.0, conlim=0.0, iter_lim=iters)[0]
    np.testing.assert_allclose(ours.x, ref, rtol=1e-9, atol=1e-12)


def test_converges_to_the_least_squares_solution():
    A, S = _system(150, 60, 5)
    b = I.normal_vector(150, 6)
    D = S.toarray()
    xls = np.linalg.lstsq(D, b, rcond=None)[0]
    normal = lambda x: np.linalg.norm(D.T @ (D @ x - b)) / (np.linalg.norm(D) * np.linalg.norm(D @ x - b))
    r = O.lsqr(lambda x: S @ x, lambda y: S.T @ y, b, 60, max_iters=5000, residual=normal, tol=1e-12)
    assert r.converged
    np.testing.assert_allclose(r.x, xls, rtol=1e-8, atol=1e-10)


def test_preconditioned_solve_recovers_the_original_solution():
    """Solve (DAE) xbar = D b, x = E xbar (Section 5.1) for a consistent square system."""
    n = 200
    A = I.sparse_uniform_density(n, n, 0.05, seed=7, var=1.0)
    S = sp.csr_matrix((A.vals, A.col_idx, A.row_ptr), shape=(n, n))
    xs = I.normal_vector(n, 8)
    b = S @ xs
    _, _, ub, vb = O.equilibrate(A, T=50, k=1, seed=0)
    d, e = np.exp(ub), np.exp(vb)
    K = sp.diags(d) @ S @ sp.diags(e)
    res = lambda xb: np.linalg.norm(S @ (e * xb) - b) / np.linalg.norm(b)
    r = O.lsqr(lambda x: K @ x, lambda y: K.T @ y, d * b, n, max_iters=20000, residual=res, tol=1e-10)
    assert r.converged and r.rel_residual <= 1e-10
    # The oracle's own FP64 matvec agrees with SciPy's.
    np.testing.assert_allclose(O.csr_matvec(A, xs), b, rtol=1e-12, atol=1e-12)
