"""One matrix split into parts (row blocks of A, column blocks of A^T) on the GPU.

Several parts are held by one process on one GPU and exchange their gather-table chunks by device copies
(LocalExchange): the same loop that runs one part per GPU with an all-gather.  Checked against the oracle
step by step (each iteration from the parts' own previous state, FP64: <= 1e-11 norm-wise), and against an
unsplit run bit for bit: every part draws the unsplit run's probes and sums every row in the same order.
"""
import numpy as np
import pytest

import oracle as O
from paper_1602_06621_gb300 import inputs as I
from paper_1602_06621_gb300 import shard as SH
from paper_1602_06621_gb300 import sme

pytestmark = pytest.mark.gpu


def _parts(A, P, k, dtype):
    import torch
    ops = [sme.sme_op_create_csr_shard(A.m, A.n, A.row_ptr, A.col_idx, A.vals, P, q) for q in range(P)]
    return [SH.Part(op, k, "cuda", dtype) for op in ops]


def _gather(parts, A):
    rb, cb = SH.blocks(A.m, len(parts)), SH.blocks(A.n, len(parts))
    out = [np.zeros(A.m), np.zeros(A.n), np.zeros(A.m), np.zeros(A.n)]
    for q, p in enumerate(parts):
        out[0][rb[q]:rb[q + 1]] = p.u.cpu().double().numpy()
        out[1][cb[q]:cb[q + 1]] = p.v.cpu().double().numpy()
        out[2][rb[q]:rb[q + 1]] = p.u_bar.cpu().double().numpy()
        out[3][cb[q]:cb[q + 1]] = p.v_bar.cpu().double().numpy()
    return out


def _scatter(parts, A, state):
    import torch
    rb, cb = SH.blocks(A.m, len(parts)), SH.blocks(A.n, len(parts))
    for q, p in enumerate(parts):
        for dst, src, b in ((p.u, state[0], rb), (p.v, state[1], cb), (p.u_bar, state[2], rb), (p.v_bar, state[3], cb)):
            dst.copy_(torch.tensor(src[b[q]:b[q + 1]], dtype=dst.dtype))


def _destroy(parts):
    for p in parts:
        sme.sme_op_destroy(p.op)


@pytest.mark.parametrize("P", [2, 3])
def test_split_matrix_every_step_matches_oracle(P):
    """Ragged 700 x 450 matrix with empty rows (FP64, k = 4): 12 iterations, each from the parts' state."""
    import torch
    A = I.sparse_variable_row_nnz(700, 450, 0, 30, seed=5, dtype=np.float64)
    A64 = O.OracleCSR.from_any(A)
    d = O.default_params(A.m, A.n)
    k = 4
    parts = _parts(A, P, k, torch.float64)
    worst = 0.0
    try:
        state = [np.zeros(A.m), np.zeros(A.n), np.zeros(A.m), np.zeros(A.n)]
        for t in range(1, 13):
            _scatter(parts, A, state)
            SH.run(parts, SH.LocalExchange(), T=1, k=k, t_begin=t, seed=9)
            got = _gather(parts, A)
            ref = O.psgd_step(A64, *state, O.probe_signs(9, t, 0, A.n, k), O.probe_signs(9, t, 1, A.m, k), t, **d)
            a, b = np.concatenate(got), np.concatenate(ref)
            worst = max(worst, np.linalg.norm(a - b) / np.linalg.norm(b))
            state = got
    finally:
        _destroy(parts)
    assert worst <= 1e-11, worst


@pytest.mark.parametrize("P,dtype", [(2, "f32"), (4, "f32"), (3, "f64")])
def test_split_matrix_equals_unsplit_run_bitwise(P, dtype):
    """A whole run (T = 30, k = 32, from zero) of the parts equals sme_equilibrate on the unsplit matrix."""
    import torch
    tdt = torch.float32 if dtype == "f32" else torch.float64
    A = I.workload_large(scale=0.01, seed=7)  # 10000 x 5000, 20 nonzeros per row
    if dtype == "f64":
        A = A.astype(np.float64)
    k, T = 32, 30
    op = sme.sme_op_create_csr(A.m, A.n, A.row_ptr, A.col_idx, A.vals)
    try:
        z = [torch.zeros(x, dtype=tdt, device="cuda") for x in (A.m, A.n, A.m, A.n)]
        sme.sme_equilibrate(op, *z, T=T, k=k, seed=3, stream_base=2)
        ref = [x.cpu().numpy() for x in z]
    finally:
        sme.sme_op_destroy(op)
    parts = _parts(A, P, k, tdt)
    try:
        SH.run(parts, SH.LocalExchange(), T=T, k=k, seed=3, stream_base=2)
        got = _gather(parts, A)
    finally:
        _destroy(parts)
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g, r.astype(np.float64))


def test_split_part_refuses_whole_matrix_calls():
    import torch
    A = I.workload_large(scale=0.001, seed=3)
    op = sme.sme_op_create_csr_shard(A.m, A.n, A.row_ptr, A.col_idx, A.vals, 2, 1)
    try:
        info = sme.sme_shard_get_info(op, 32)
        assert (info["row_begin"], info["row_end"]) == (A.m // 2, A.m)
        assert (info["col_begin"], info["col_end"]) == (A.n // 2, A.n)
        assert info["row_chunk"] == (A.m + 1) // 2 and info["entry_bytes"] == 8
        z = torch.zeros(A.m, device="cuda")
        with pytest.raises(sme.SmeError) as ei:
            sme.sme_equilibrate(op, z, z[:A.n].clone(), z.clone(), z[:A.n].clone(), T=2, k=32)
        assert ei.value.name == "SME_ERR_UNSUPPORTED"
        with pytest.raises(sme.SmeError) as ei:
            sme.sme_estimate(op, z, z[:A.n].clone(), 1, 32, 0, 0, z.clone(), None)
        assert ei.value.name == "SME_ERR_UNSUPPORTED"
    finally:
        sme.sme_op_destroy(op)


@pytest.mark.parametrize("P,k", [(5, 64), (23, 2), (1, 8)])
def test_split_matrix_edge_shapes_equal_unsplit(P, k):
    """37 x 23 with empty rows and columns, FP64: parts down to one column each (P = n = 23), 16-byte table
    entries (k = 64), and the trivial split (P = 1); T = 8 from zero, bit for bit against the unsplit run."""
    import torch
    A = I.sparse_uniform_density(37, 23, 0.08, seed=5)
    T = 8
    op = sme.sme_op_create_csr(A.m, A.n, A.row_ptr, A.col_idx, A.vals)
    try:
        z = [torch.zeros(x, dtype=torch.float64, device="cuda") for x in (A.m, A.n, A.m, A.n)]
        sme.sme_equilibrate(op, *z, T=T, k=k, seed=6, t0=20)
        ref = [x.cpu().numpy() for x in z]
    finally:
        sme.sme_op_destroy(op)
    parts = _parts(A, P, k, torch.float64)
    try:
        if k > 32:
            assert parts[0].info["entry_bytes"] == 16
        SH.run(parts, SH.LocalExchange(), T=T, k=k, seed=6, t0=20)
        got = _gather(parts, A)
    finally:
        _destroy(parts)
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g, r)


def test_split_part_refuses_steps_without_a_matching_begin():
    """A step or an end before sme_shard_begin, or a step whose k needs another table entry size than the
    begin's, is refused on the host (the tables were sized for one entry size); nothing is launched."""
    import torch
    A = I.workload_large(scale=0.001, seed=3)
    op = sme.sme_op_create_csr_shard(A.m, A.n, A.row_ptr, A.col_idx, A.vals, 2, 0)
    try:
        p8 = SH.Part(op, 8, "cuda")
        with pytest.raises(sme.SmeError) as ei:
            p8.step(1, 1, dict(T=1, k=8, t_begin=1))
        assert ei.value.name == "SME_ERR_ARG"
        with pytest.raises(sme.SmeError) as ei:
            p8.end()
        assert ei.value.name == "SME_ERR_ARG"
        for tab in p8.tables.row + p8.tables.col:
            tab.zero_()  # the other part's chunks are never written here
        p8.begin(1, dict(T=1, k=8, t_begin=1))
        with pytest.raises(sme.SmeError) as ei:
            p8.step(1, 1, dict(T=1, k=64, t_begin=1))  # 16-byte entries into 8-byte tables
        assert ei.value.name == "SME_ERR_ARG"
        p8.step(1, 1, dict(T=1, k=16, t_begin=1))  # same entry size: accepted
        p8.end()
        torch.cuda.synchronize()
    finally:
        sme.sme_op_destroy(op)


@pytest.mark.parametrize("P", [2, 4])
def test_split_full_size_equals_unsplit(P):
    """The 1e6 x 5e5 workload the split bench runs (20 nonzeros per row, FP32, k = 32): P parts on one GPU
    (device-copy exchange), T = 3 from zero, bit for bit against the unsplit operator."""
    import torch
    A = I.workload_large(1.0, seed=2)
    k, T = 32, 3
    op = sme.sme_op_create_csr(A.m, A.n, A.row_ptr, A.col_idx, A.vals)
    try:
        z = [torch.zeros(x, device="cuda") for x in (A.m, A.n, A.m, A.n)]
        sme.sme_equilibrate(op, *z, T=T, k=k, seed=0)
        ref = [x.cpu().numpy() for x in z]
        del z
    finally:
        sme.sme_op_destroy(op)
    parts = _parts(A, P, k, torch.float32)
    try:
        SH.run(parts, SH.LocalExchange(), T=T, k=k, seed=0)
        got = _gather(parts, A)
    finally:
        _destroy(parts)
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g, r.astype(np.float64))
