"""The paper's printed trends, reproduced by the oracle on reduced-size problems shaped
like its experiments (Section 4: uniform sparsity, N(0,1) values, row and column
factors e^{N(1,1)}).  The paper's sizes (2e4 x 1e4; n = 1e4 for LSQR) are scaled
down so the CPU suite stays fast; thresholds are set for the reduced sizes."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_1602_06621_gb300 import inputs as I


@pytest.mark.slow
def test_condition_number_falls_by_two_orders_after_100_iterations():
    """Section 4: kappa(DAE) 200x below kappa(A) after 100 iterations (at 2e4 x 1e4)."""
    A = I.sparse_uniform_density(1000, 500, 0.02, seed=3, mean=1.0, var=1.0)
    Ad = A.to_dense()
    k0 = O.kappa(Ad)
    _, _, ub, vb = O.equilibrate(A, T=100, k=1, seed=0)
    k100 = O.kappa(np.exp(ub)[:, None] * Ad * np.exp(vb)[None, :])
    assert k0 / k100 > 100
    # Early iterations oscillate: after 4 iterations kappa is not yet below kappa(A) by much.
    _, _, ub4, vb4 = O.equilibrate(A, T=4, k=1, seed=0)
    k4 = O.kappa(np.exp(ub4)[:, None] * Ad * np.exp(vb4)[None, :])
    assert k4 > k0 / 10


def test_optimality_gap_decays_faster_than_one_over_t():
    """Section 4: least-squares slope of log gap vs log t is -2.0 (theory: -1)."""
    A = I.sparse_uniform_density(400, 200, 0.05, seed=3, mean=1.0, var=1.0)
    d = O.default_params(400, 200)
    kw = dict(alpha=d["alpha"], beta=d["beta"], gamma=d["gamma"])
    us, vs = O.regularized_optimum(A, **d)
    fs = O.objective(A, us, vs, **kw)
    f0 = O.objective(A, np.zeros(400), np.zeros(200), **kw)
    Ts = [80, 160, 320, 640, 1000]
    gaps = [(O.objective(A, *O.equilibrate(A, T=T, k=1, seed=0)[2:], **kw) - fs) / f0 for T in Ts]
    slope = np.polyfit(np.log(Ts), np.log(gaps), 1)[0]
    assert slope < -1.5


@pytest.mark.slow
def test_equilibration_cuts_lsqr_iterations():
    """Section 5.1: with >= 30 equilibration iterations LSQR needs far fewer iterations to 1e-4
    (equilibration iterations counted); 10 iterations help only a little."""
    n = 1000
    A = I.sparse_uniform_density(n, n, 0.01, seed=5, mean=1.0, var=1.0)
    S = sp.csr_matrix((A.vals, A.col_idx, A.row_ptr), shape=(n, n))
    b = S @ I.normal_vector(n, 11)
    res = lambda x: np.linalg.norm(S @ x - b) / np.linalg.norm(b)
    plain = O.lsqr(lambda x: S @ x, lambda y: S.T @ y, b, n, max_iters=100000, residual=res, tol=1e-4)
    assert plain.converged
    totals = {}
    for T in (10, 30, 100):
        _, _, ub, vb = O.equilibrate(A, T=T, k=1, seed=0)
        d, e = np.exp(ub), np.exp(vb)
        K = sp.diags(d) @ S @ sp.diags(e)
        r = O.lsqr(lambda x: K @ x, lambda y: K.T @ y, d * b, n, max_iters=100000,
                   residual=lambda xb: res(e * xb), tol=1e-4)
        assert r.converged
        totals[T] = r.iters + T
    assert plain.iters / totals[30] > 3
    assert plain.iters / totals[100] > 5
    assert totals[10] > totals[30] > totals[100]
