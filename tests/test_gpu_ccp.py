"""The Chambolle-Cremers-Pock Lasso solver (Section 5.2) on the GPU against the oracle's (oracle/ccp.py)."""
import numpy as np
import pytest

import oracle as O
from oracle import ccp as C
from paper_1602_06621_gb300 import inputs as I
from paper_1602_06621_gb300 import sme

pytestmark = pytest.mark.gpu


def _problem(seed, m, n, density, dtype):
    A = I.sparse_uniform_density(m, n, density, seed, mean=1.0, var=1.0, dtype=dtype)
    rng = np.random.default_rng(seed + 100)
    xh = np.zeros(n)
    idx = rng.choice(n, n // 10, replace=False)
    xh[idx] = rng.standard_normal(idx.size)
    b = C._matrix(A) @ xh + rng.standard_normal(m)
    return A, b, C.default_lambda(A, b)


def _t(x, dtype):
    import torch
    return torch.tensor(np.asarray(x), dtype=torch.float64 if dtype == np.float64 else torch.float32, device="cuda")


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_operator_norm_matches_oracle_power_iteration(dtype):
    A, _, _ = _problem(1, 300, 500, 0.03, dtype)
    rng = np.random.default_rng(2)
    u, v = rng.normal(0, 0.5, A.m), rng.normal(0, 0.5, A.n)
    op = sme.sme_op_create_csr(A.m, A.n, A.row_ptr, A.col_idx, A.vals)
    try:
        got = sme.sme_op_norm2(op, _t(u, dtype), _t(v, dtype), iters=60)
        plain = sme.sme_op_norm2(op, None, None, iters=60)
    finally:
        sme.sme_op_destroy(op)
    K, _, _ = C.scaled_operator(A, u, v)
    tol = 1e-12 if dtype == np.float64 else 2e-5
    assert got == pytest.approx(C.power_norm(K, 60), rel=tol)
    K0, _, _ = C.scaled_operator(A)
    assert plain == pytest.approx(C.power_norm(K0, 60), rel=tol)


@pytest.mark.parametrize("dtype,shape", [(np.float64, (400, 700, 0.02)), (np.float32, (400, 700, 0.02)),
                                         (np.float64, (96, 2400, 0.15)), (np.float32, (1500, 200, 0.4))])
def test_iterates_and_objective_history_match_oracle(dtype, shape):
    """Same iteration on both sides (same steps, same order): x after 60 iterations and f(x) every 10.  The
    wide shapes (360 and 80 nonzeros per row or column) run the passes with several warps per slice; 60
    iterations with checks every 10 replay the captured chunk graph."""
    import torch
    m, n, density = shape
    A, b, lam = _problem(3, m, n, density, dtype)
    d = O.default_params(A.m, A.n)
    _, _, ub, vb = O.equilibrate(A, T=30, k=1, seed=0, **d)
    op = sme.sme_op_create_csr(A.m, A.n, A.row_ptr, A.col_idx, A.vals)
    try:
        x = torch.zeros(A.n, dtype=_t([0.0], dtype).dtype, device="cuda")
        res, hist = sme.sme_ccp_lasso(op, _t(ub, dtype), _t(vb, dtype), _t(b, dtype), x, lam=lam, max_iters=60,
                                      check_every=10, norm_iters=100)
        xg = x.cpu().double().numpy()
    finally:
        sme.sme_op_destroy(op)
    xo, ho, nrm = C.ccp_lasso(A, b, lam, iters=60, u=ub, v=vb, norm_iters=100, check_every=10)
    assert res["iters"] == 60 and res["history_count"] == 6
    tol = 1e-10 if dtype == np.float64 else 2e-4
    assert res["op_norm"] == pytest.approx(nrm, rel=1e-12 if dtype == np.float64 else 2e-5)
    assert np.linalg.norm(xg - xo) <= tol * np.linalg.norm(xo)
    np.testing.assert_allclose(hist, ho[1:], rtol=tol)
    assert res["objective0"] == pytest.approx(ho[0], rel=1e-12 if dtype == np.float64 else 1e-6)
    # The library's f(x) is FP64 arithmetic on its inputs as given (b in the operator's type).
    b_in = np.asarray(b, dtype).astype(np.float64)
    assert res["objective"] == pytest.approx(C.lasso_objective(A, xg, b_in, lam), rel=1e-9)


def test_stops_at_the_relative_gap_of_the_oracle_optimum():
    """FP32 solve with p* from a long FP64 oracle run: stops at (f - p*)/f(0) <= 1e-6, within a few checks of
    the iteration at which the oracle's own history first crosses it."""
    import torch
    A, b, lam = _problem(4, 300, 600, 0.03, np.float32)
    d = O.default_params(A.m, A.n)
    _, _, ub, vb = O.equilibrate(A, T=100, k=1, seed=0, **d)
    xs, _, _ = C.ccp_lasso(A, b, lam, iters=60000, u=ub, v=vb)
    assert C.lasso_kkt_residual(A, xs, b, lam) < 1e-6
    pstar = C.lasso_objective(A, xs, b, lam)
    _, ho, _ = C.ccp_lasso(A, b, lam, iters=5000, u=ub, v=vb, check_every=10)
    n_oracle = next(i * 10 for i, f in enumerate(ho) if (f - pstar) / ho[0] <= 1e-6)
    op = sme.sme_op_create_csr(A.m, A.n, A.row_ptr, A.col_idx, A.vals)
    try:
        x = torch.zeros(A.n, device="cuda")
        res, _ = sme.sme_ccp_lasso(op, _t(ub, np.float32), _t(vb, np.float32), _t(b, np.float32), x, lam=lam,
                                   max_iters=5000, check_every=10, p_star=pstar, tol=1e-6)
    finally:
        sme.sme_op_destroy(op)
    assert res["converged"] == 1 and res["rel_gap"] <= 1e-6
    assert abs(res["iters"] - n_oracle) <= max(30, n_oracle // 10), (res["iters"], n_oracle)


def test_given_steps_and_argument_errors():
    import torch
    A, b, lam = _problem(5, 64, 96, 0.1, np.float32)
    op = sme.sme_op_create_csr(A.m, A.n, A.row_ptr, A.col_idx, A.vals)
    try:
        x = torch.zeros(A.n, device="cuda")
        bt = _t(b, np.float32)
        res, _ = sme.sme_ccp_lasso(op, None, None, bt, x, lam=lam, max_iters=20, check_every=5, tau=1e-3, sigma=1e-3)
        assert res["op_norm"] == 0.0 and res["tau"] == 1e-3 and res["iters"] == 20
        xo, _, _ = C.ccp_lasso(A, b, lam, iters=20, tau=1e-3, sigma=1e-3)
        assert np.linalg.norm(x.cpu().double().numpy() - xo) <= 1e-5 * max(1.0, np.linalg.norm(xo))
        with pytest.raises(sme.SmeError):
            sme.sme_ccp_lasso(op, None, None, bt, x, lam=0.0, max_iters=5)
        with pytest.raises(sme.SmeError):
            sme.sme_op_norm2(op, None, None, iters=0)
    finally:
        sme.sme_op_destroy(op)
    b2 = sme.sme_batch_create([A, A])
    try:
        with pytest.raises(sme.SmeError):
            sme.sme_ccp_lasso(sme.sme_batch_op(b2), None, None, bt, x, lam=lam, max_iters=5)
    finally:
        sme.sme_batch_destroy(b2)
