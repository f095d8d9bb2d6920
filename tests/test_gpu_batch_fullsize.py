"""The batched workload at full size (512 matrices, m log-uniform in [1e3, 2e5], n = m U[0.3, 1], 5-50 nonzeros
per row, 5.1e8 nonzeros in all, FP32, k = 16), in the launch configuration the bench times (the autotuned
shape of the batch's block-diagonal operator).

The oracle cannot run the whole batch, so it checks iteration t = 3 of Algorithm 1 at sampled rows and columns
of six matrices (the largest, the smallest and four drawn at random), from the GPU's own state after two
iterations: each matrix with its own alpha, beta and its own probe streams (2b for s, 2b + 1 for w).  The
tolerance is a bound on FP32 rounding, not a fitted constant.  For a row of L nonzeros with c_j = |a_ij| e^{v_j},
the kernel forms y_p = C - 2 P_p from two FP32 sums (C over all terms, P_p over the terms whose probe bit is
set), so y_p carries an error of at most (3 L + 18) 2^-24 sum_j c_j: the accumulations, the subtraction, the
products a_ij e^{v_j} and the FP32 table value e^{v_j} (expf, within 2 ulp).  Then
|dz| <= (6 L + 80) 2^-24 S1 with S1 = e^{2 u_i} (sum_j c_j)^2, which also bounds z itself (the squares, their
mean over k = 16 probes and e^{2 u_i} add the rest); the step multiplies that by eta and the projection does
not enlarge it.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1602_06621_gb300 import inputs as I
from paper_1602_06621_gb300 import sme

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


@pytest.fixture(scope="module")
def family():
    mats = I.batched_family(512, 1000, 200000, seed=40, workers=min(16, os.cpu_count() or 1))
    yield mats


def _side_bounds(indptr, idx, vals, x_own, x_other, picks):
    """Row length L and S1 = e^{2 x_i} (sum_j |a_ij| e^{x_j})^2 for the picked rows of a CSR (or columns of
    the CSC)."""
    L = np.zeros(picks.size)
    S1 = np.zeros(picks.size)
    for q, i in enumerate(picks):
        a, b = indptr[i], indptr[i + 1]
        L[q] = b - a
        S1[q] = np.exp(2.0 * x_own[i]) * np.sum(np.abs(vals[a:b].astype(np.float64)) * np.exp(x_other[idx[a:b]])) ** 2
    return L, S1


def test_full_batch_sampled_step_matches_oracle(family):
    import scipy.sparse as sps
    import torch

    mats = family
    b = sme.sme_batch_create(mats)
    try:
        _, ro, co = sme.sme_batch_get_info(b)
        M, N = int(ro[-1]), int(co[-1])
        assert sum(A.nnz for A in mats) > 5e8
        sme.sme_op_autotune(sme.sme_batch_op(b), 16)
        z = [torch.zeros(x, dtype=torch.float32, device="cuda") for x in (M, N, M, N)]
        sme.sme_batch_equilibrate(b, *z, T=2, k=16, seed=0)
        s2 = [x.cpu().double().numpy() for x in z]
        sme.sme_batch_equilibrate(b, *z, T=1, k=16, seed=0, t_begin=3)
        s3 = [x.cpu().double().numpy() for x in z]
    finally:
        sme.sme_batch_destroy(b)

    rng = np.random.default_rng(5)
    sizes = np.array([A.m for A in mats])
    pick = [int(sizes.argmax()), int(sizes.argmin())]
    pick += [int(i) for i in rng.choice(np.setdiff1d(np.arange(len(mats)), pick), 4, replace=False)]
    t, eta = 3, 2.0 / (0.1 * 4.0)
    for bi in pick:
        A = mats[bi]
        d = O.default_params(A.m, A.n)
        rs, cs = slice(ro[bi], ro[bi + 1]), slice(co[bi], co[bi + 1])
        u, v, ub, vb = s2[0][rs], s2[1][cs], s2[2][rs], s2[3][cs]
        rows = np.sort(rng.choice(A.m, min(A.m, 48), replace=False))
        cols = np.sort(rng.choice(A.n, min(A.n, 48), replace=False))
        uo, ubo, vo, vbo = O.psgd_step_sampled(O.OracleCSR.from_any(A), u, v, ub, vb, rows, cols, t, k=16, seed=0,
                                               stream_base=2 * bi, **d)
        C = sps.csr_matrix((A.vals, A.col_idx, A.row_ptr), shape=(A.m, A.n)).tocsc()
        Lr, S1r = _side_bounds(A.row_ptr, A.col_idx, A.vals, u, v, rows)
        Lc, S1c = _side_bounds(C.indptr, C.indices, C.data, v, u, cols)
        for got_x, got_xb, ref_x, ref_xb, old_x, L, S1, tgt in (
                (s3[0][rs][rows], s3[2][rs][rows], uo, ubo, u[rows], Lr, S1r, d["alpha"] ** 2),
                (s3[1][cs][cols], s3[3][cs][cols], vo, vbo, v[cols], Lc, S1c, d["beta"] ** 2)):
            tol_z = (6.0 * L + 80.0) * U * S1
            tol_x = eta * tol_z + 4 * U * (np.abs(ref_x) + eta * (S1 + tgt + 0.1 * np.abs(old_x))) + 1e-7
            assert np.all(np.abs(got_x - ref_x) <= tol_x), (bi, np.max(np.abs(got_x - ref_x) / tol_x))
            tol_xb = 0.4 * tol_x + 4 * U * np.abs(ref_xb) + 1e-7
            assert np.all(np.abs(got_xb - ref_xb) <= tol_xb), (bi, np.max(np.abs(got_xb - ref_xb) / tol_xb))
