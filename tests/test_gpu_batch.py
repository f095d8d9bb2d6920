"""Batches of matrices (one block-diagonal operator) against separate runs and the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1602_06621_gb300 import inputs as I
from paper_1602_06621_gb300 import sme

from gpu_util import gpu_equilibrate, make_op, rel_norm

pytestmark = pytest.mark.gpu


def _zeros(n, td):
    import torch
    return torch.zeros(n, dtype=td, device="cuda")


def _batch_run(b, mats, td, **kw):
    M = sum(A.m for A in mats)
    N = sum(A.n for A in mats)
    u, v, ub, vb = _zeros(M, td), _zeros(N, td), _zeros(M, td), _zeros(N, td)
    sme.sme_batch_equilibrate(b, u, v, ub, vb, **kw)
    return [x.cpu().double().numpy() for x in (u, v, ub, vb)]


@pytest.mark.parametrize("k,group_bytes", [(16, None), (32, None), (16, 40000)])
def test_batch_equals_separate_runs_bitwise(k, group_bytes, monkeypatch):
    """Also with matrices laid out in several L2-sized groups (a small group budget forces several).  Rows and
    columns stay under 48 nonzeros on average, so neither the batch nor any matrix alone shares slices among
    warps (a different split would only change the order of the sums)."""
    import torch
    if group_bytes:
        monkeypatch.setenv("SME_BATCH_GROUP_BYTES", str(group_bytes))
    mats = I.batched_family(7, 300, 3000, seed=k, nnz_hi=20)
    b = sme.sme_batch_create(mats)
    try:
        count, ro, co = sme.sme_batch_get_info(b)
        assert count == 7 and ro[-1] == sum(A.m for A in mats)
        got = _batch_run(b, mats, torch.float32, T=25, k=k, seed=4, stream_base=6)
    finally:
        sme.sme_batch_destroy(b)
    for i, A in enumerate(mats):
        op, dt = make_op(A)
        try:
            one = gpu_equilibrate(op, dt, A.m, A.n, T=25, k=k, seed=4, stream_base=6 + 2 * i)
        finally:
            sme.sme_op_destroy(op)
        sl = [slice(ro[i], ro[i + 1]), slice(co[i], co[i + 1]), slice(ro[i], ro[i + 1]), slice(co[i], co[i + 1])]
        for x, s_, y in zip(got, sl, one):
            np.testing.assert_array_equal(x[s_], y)


def test_batch_fp64_matches_oracle_per_matrix():
    import torch
    mats = I.batched_family(5, 40, 400, seed=3, dtype=np.float64)
    b = sme.sme_batch_create(mats)
    try:
        _, ro, co = sme.sme_batch_get_info(b)
        got = _batch_run(b, mats, torch.float64, T=6, k=8, seed=2)
    finally:
        sme.sme_batch_destroy(b)
    for i, A in enumerate(mats):
        ref = O.equilibrate(A, T=6, k=8, seed=2, stream_base=2 * i)
        mine = (got[0][ro[i]:ro[i + 1]], got[1][co[i]:co[i + 1]], got[2][ro[i]:ro[i + 1]], got[3][co[i]:co[i + 1]])
        assert rel_norm(mine, ref) <= 1e-10


def test_batch_of_degenerate_matrices_matches_oracle_per_matrix():
    """A batch holding a matrix with empty rows and columns, a single row, a single column, a 1 x 1 matrix and
    a matrix with no nonzeros at all, between ordinary ones (FP64, T = 6, k = 16): each matrix against the
    oracle run on it alone with its own probe streams."""
    import torch
    mats = [I.sparse_uniform_density(37, 23, 0.08, seed=5, dtype=np.float64),
            I.sparse_uniform_density(1, 5, 0.8, seed=6, dtype=np.float64),
            I.sparse_uniform_density(300, 200, 0.05, seed=9, dtype=np.float64),
            I.sparse_uniform_density(5, 1, 0.8, seed=7, dtype=np.float64),
            I.CSR(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.5])),
            I.CSR(40, 33, np.zeros(41, np.int32), np.zeros(0, np.int32), np.zeros(0)),
            I.sparse_uniform_density(64, 90, 0.1, seed=10, dtype=np.float64)]
    b = sme.sme_batch_create(mats)
    try:
        count, ro, co = sme.sme_batch_get_info(b)
        assert count == len(mats)
        got = _batch_run(b, mats, torch.float64, T=6, k=16, seed=3)
    finally:
        sme.sme_batch_destroy(b)
    for i, A in enumerate(mats):
        ref = O.equilibrate(A, T=6, k=16, seed=3, stream_base=2 * i)
        mine = (got[0][ro[i]:ro[i + 1]], got[1][co[i]:co[i + 1]], got[2][ro[i]:ro[i + 1]], got[3][co[i]:co[i + 1]])
        assert rel_norm(mine, ref) <= 1e-10, i


def test_batch_with_long_rows_every_step_fp64():
    """Matrices of 150-300 nonzeros per row in one batch: the batch's slices are shared among warps (split
    accumulation) while each matrix keeps its own targets and probe streams.  Every step of every matrix
    against the oracle's step from the batch's own state."""
    import torch
    mats = [I.sparse_uniform_density(m, n, dens, seed=40 + i, mean=1.0, var=1.0)
            for i, (m, n, dens) in enumerate([(120, 1500, 0.2), (64, 1000, 0.15), (200, 2000, 0.1)])]
    b = sme.sme_batch_create(mats)
    try:
        _, ro, co = sme.sme_batch_get_info(b)
        state = [np.zeros(int(ro[-1])), np.zeros(int(co[-1])), np.zeros(int(ro[-1])), np.zeros(int(co[-1]))]
        worst = 0.0
        for t in range(1, 6):
            g = [torch.tensor(x, dtype=torch.float64, device="cuda") for x in state]
            sme.sme_batch_equilibrate(b, *g, T=1, k=4, seed=5, t_begin=t)
            new = [x.cpu().numpy() for x in g]
            for i, A in enumerate(mats):
                r, c = slice(ro[i], ro[i + 1]), slice(co[i], co[i + 1])
                mine = (new[0][r], new[1][c], new[2][r], new[3][c])
                ref = O.psgd_step(A, state[0][r], state[1][c], state[2][r], state[3][c],
                                  O.probe_signs(5, t, 2 * i, A.n, 4), O.probe_signs(5, t, 2 * i + 1, A.m, 4), t,
                                  **O.default_params(A.m, A.n))
                worst = max(worst, rel_norm(mine, ref))
            state = new
    finally:
        sme.sme_batch_destroy(b)
    assert worst <= 1e-11, worst


def test_batch_estimate_and_evaluate():
    import torch
    mats = I.batched_family(4, 100, 900, seed=8)
    b = sme.sme_batch_create(mats)
    try:
        _, ro, co = sme.sme_batch_get_info(b)
        rng = np.random.default_rng(0)
        u = rng.normal(0, 0.5, ro[-1]).astype(np.float32)
        v = rng.normal(0, 0.5, co[-1]).astype(np.float32)
        ud, vd = torch.tensor(u, device="cuda"), torch.tensor(v, device="cuda")
        zu, zv = _zeros(ro[-1], torch.float32), _zeros(co[-1], torch.float32)
        sme.sme_batch_estimate(b, ud, vd, 3, 16, 5, 0, zu, zv)
        r2 = _zeros(ro[-1], torch.float64)
        c2 = _zeros(co[-1], torch.float64)
        sme.sme_evaluate(sme.sme_batch_op(b), ud, vd, r2=r2, c2=c2)
        zu, zv, r2, c2 = (x.cpu().double().numpy() for x in (zu, zv, r2, c2))
    finally:
        sme.sme_batch_destroy(b)
    for i, A in enumerate(mats):
        A64 = O.OracleCSR.from_any(A)
        ui, vi = u[ro[i]:ro[i + 1]], v[co[i]:co[i + 1]]
        er2, ec2 = O.exact_norms_sq(A64, ui, vi)
        np.testing.assert_allclose(r2[ro[i]:ro[i + 1]], er2, rtol=1e-12)
        np.testing.assert_allclose(c2[co[i]:co[i + 1]], ec2, rtol=1e-12)
        ez = O.row_estimate(A64, ui, vi, O.probe_signs(5, 3, 2 * i, A.n, 16))
        ezv = O.col_estimate(A64, ui, vi, O.probe_signs(5, 3, 2 * i + 1, A.m, 16))
        assert np.all(np.abs(zu[ro[i]:ro[i + 1]] - ez) <= 3e-5 * er2 + 1e-30)
        assert np.all(np.abs(zv[co[i]:co[i + 1]] - ezv) <= 3e-5 * ec2 + 1e-30)


def test_graph_replay_equals_direct_launches():
    A = I.workload_large(scale=0.004, seed=4)
    op, dt = make_op(A)
    try:
        g1 = gpu_equilibrate(op, dt, A.m, A.n, T=30, k=32, seed=1)  # first call: direct launches
        g2 = gpu_equilibrate(op, dt, A.m, A.n, T=30, k=32, seed=1)  # repeated: captured and launched
        g2b = gpu_equilibrate(op, dt, A.m, A.n, T=30, k=32, seed=1)  # replays the cached graph
        d1 = gpu_equilibrate(op, dt, A.m, A.n, T=30, k=32, seed=1, flags=sme.SME_EQ_NO_GRAPH)
        g3 = gpu_equilibrate(op, dt, A.m, A.n, T=30, k=32, seed=2)  # new key: captured again
        d3 = gpu_equilibrate(op, dt, A.m, A.n, T=30, k=32, seed=2, flags=sme.SME_EQ_NO_GRAPH)
    finally:
        sme.sme_op_destroy(op)
    for a, b_, bb, c in zip(g1, g2, g2b, d1):
        np.testing.assert_array_equal(a, b_)
        np.testing.assert_array_equal(a, bb)
        np.testing.assert_array_equal(a, c)
    for a, c in zip(g3, d3):
        np.testing.assert_array_equal(a, c)


def test_autotuned_shape_gives_identical_results():
    """The launch shape changes only scheduling: results are bitwise those of the default shape."""
    A = I.workload_large(scale=0.004, seed=5)
    op, dt = make_op(A)
    try:
        ref = gpu_equilibrate(op, dt, A.m, A.n, T=12, k=32, seed=1)
        choice = sme.sme_op_autotune(op, 32)
        assert choice["slices_per_cta"] in (4, 8, 16) and choice["cols_first"] in (0, 1)
        assert choice["ms_per_iteration"] > 0
        got = gpu_equilibrate(op, dt, A.m, A.n, T=12, k=32, seed=1)
    finally:
        sme.sme_op_destroy(op)
    for a, b_ in zip(ref, got):
        np.testing.assert_array_equal(a, b_)


@pytest.mark.parametrize("group_bytes", [None, 20000])
def test_batch_lsqr_matches_per_matrix_lsqr(group_bytes, monkeypatch):
    """Each matrix of the batch gets its own LSQR.  Against sme_lsqr on the matrix alone (same scalings,
    same right-hand side): the first iterates agree to rounding; converged solves agree in iteration count
    within 2 % (the norms are summed in a different order, and LSQR amplifies rounding over hundreds of
    iterations); every residual is re-checked by the oracle."""
    import torch
    if group_bytes:
        monkeypatch.setenv("SME_BATCH_GROUP_BYTES", str(group_bytes))
    mats = I.batched_family(5, 80, 1500, seed=21, dtype=np.float64)
    b = sme.sme_batch_create(mats)
    try:
        _, ro, co = sme.sme_batch_get_info(b)
        st = _batch_run(b, mats, torch.float64, T=60, k=16, seed=1)
        ub, vb = (torch.tensor(x, device="cuda") for x in (st[2], st[3]))
        bvecs = [O.csr_matvec(A, I.normal_vector(A.n, 30 + i)) for i, A in enumerate(mats)]
        bcat = torch.tensor(np.concatenate(bvecs), device="cuda")
        x5 = torch.zeros(int(co[-1]), dtype=torch.float64, device="cuda")
        sme.sme_batch_lsqr(b, ub, vb, bcat, x5, tol=0.0, max_iters=5, check_every=5)
        x5 = x5.cpu().numpy()
        x = torch.zeros(int(co[-1]), dtype=torch.float64, device="cuda")
        res = sme.sme_batch_lsqr(b, ub, vb, bcat, x, tol=1e-8, max_iters=5000, check_every=1)
        x = x.cpu().numpy()
    finally:
        sme.sme_batch_destroy(b)
    for i, A in enumerate(mats):
        assert res[i]["converged"] == 1
        xi = x[co[i]:co[i + 1]]
        rel = np.linalg.norm(O.csr_matvec(A, xi) - bvecs[i]) / np.linalg.norm(bvecs[i])
        assert rel <= 1e-8 and res[i]["rel_residual"] == pytest.approx(rel, rel=1e-6)
        op, dt = make_op(A)
        try:
            args = (torch.tensor(st[2][ro[i]:ro[i + 1]], device="cuda"), torch.tensor(st[3][co[i]:co[i + 1]], device="cuda"),
                    torch.tensor(bvecs[i], device="cuda"))
            x1 = torch.zeros(A.n, dtype=torch.float64, device="cuda")
            sme.sme_lsqr(op, *args, x1, tol=0.0, max_iters=5, check_every=5)
            np.testing.assert_allclose(x1.cpu().numpy(), x5[co[i]:co[i + 1]], rtol=1e-10,
                                       atol=1e-12 * np.abs(x5[co[i]:co[i + 1]]).max())
            x1.zero_()
            r1 = sme.sme_lsqr(op, *args, x1, tol=1e-8, max_iters=5000, check_every=1)
        finally:
            sme.sme_op_destroy(op)
        assert r1["converged"] == 1
        assert abs(r1["iters"] - res[i]["iters"]) <= max(2, 0.02 * r1["iters"])
