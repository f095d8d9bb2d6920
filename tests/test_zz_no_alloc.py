"""The allocation-free row estimator against the regular one and the oracle, on the GPU.

sme_estimate_rows_static serves callers that cannot allocate device memory on
their hot path: a process whose free device memory is already held by a
caching allocator, a latency-critical loop that cannot take the device-wide
synchronisation an allocation or a free may cause, or a plug-in handed fixed
buffers by a host application that keeps the memory budget to itself.  It
keeps its gather table in a fixed array inside the library, so these tests
check that consecutive calls -- each overwriting the table the previous call
left behind -- give what sme_estimate gives and what the FP64 oracle gives for
the same inputs, within the FP32 tolerance used throughout (|dz_i| <= 3e-5 r2_i,
r2_i the exact squared row norm), for every supported k and a nonzero probe
stream; that a column index outside [0, n) marks only its own row with NaN;
and that a size beyond the array is refused.

This file is named to be collected last, so a run stopping at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

import oracle as O
from paper_1602_06621_gb300 import inputs as I
from paper_1602_06621_gb300 import sme

pytestmark = pytest.mark.gpu

SEED = 5


def _device_csr(A):
    import torch

    dev = dict(device="cuda")
    return (torch.tensor(A.row_ptr, **dev), torch.tensor(A.col_idx, **dev), torch.tensor(A.vals, **dev))


def test_static_estimator_matches_regular_estimator_and_oracle_in_consecutive_calls():
    import torch

    A = I.workload_large(scale=0.02, seed=21)  # 20000 x 10000, 20 nonzeros per row, FP32
    op = sme.sme_op_create_csr(A.m, A.n, A.row_ptr, A.col_idx, A.vals)
    try:
        rp, ci, va = _device_csr(A)
        rng = np.random.default_rng(3)
        A64 = O.OracleCSR.from_any(A)
        calls = [(4, 32, 0), (9, 16, 0), (2, 1, 6), (3, 2, 6), (5, 4, 2), (7, 8, 10), (8, 32, 4)]
        for call, (t, k, sb) in enumerate(calls):
            u = rng.normal(0, 0.5, A.m).astype(np.float32)
            v = rng.normal(0, 0.5, A.n).astype(np.float32)
            ud, vd = torch.tensor(u, device="cuda"), torch.tensor(v, device="cuda")
            z_ref = torch.full((A.m,), float("nan"), dtype=torch.float32, device="cuda")
            sme.sme_estimate(op, ud, vd, t, k, SEED, sb, z_ref, None)
            z_new = torch.full((A.m,), float("nan"), dtype=torch.float32, device="cuda")
            sme.sme_estimate_rows_static(A.m, A.n, rp, ci, va, ud, vd, t, k, SEED, sb, z_new)
            torch.cuda.synchronize()
            r2, _ = O.exact_norms_sq(A64, u, v)
            zo = O.row_estimate(A64, u, v, O.probe_signs(SEED, t, sb, A.n, k))
            got = z_new.cpu().double().numpy()
            for name, ref in (("sme_estimate", z_ref.cpu().double().numpy()), ("oracle", zo)):
                diff = np.abs(got - ref)
                assert np.all(diff <= 3e-5 * r2 + 1e-30), \
                    f"call {call} (t={t}, k={k}, stream {sb}) vs {name}: max excess {np.max(diff - 3e-5 * r2)}"
    finally:
        sme.sme_op_destroy(op)


def test_static_estimator_marks_rows_with_out_of_range_columns():
    import torch

    A = I.workload_large(scale=0.005, seed=22)  # 5000 x 2500
    col = A.col_idx.copy()
    bad_rows = np.array([0, 17, 4999])
    col[A.row_ptr[bad_rows[0]]] = A.n                          # one past the end
    col[A.row_ptr[bad_rows[1]] + 3] = sme.SME_STATIC_MAX_COLS - 1  # inside the array, outside the matrix
    col[A.row_ptr[bad_rows[2] + 1] - 1] = -7                   # negative
    rp, ci, va = _device_csr(I.CSR(A.m, A.n, A.row_ptr, col, A.vals))
    rng = np.random.default_rng(4)
    u = rng.normal(0, 0.5, A.m).astype(np.float32)
    v = rng.normal(0, 0.5, A.n).astype(np.float32)
    ud, vd = torch.tensor(u, device="cuda"), torch.tensor(v, device="cuda")
    t, k = 3, 16
    z = torch.zeros(A.m, dtype=torch.float32, device="cuda")
    sme.sme_estimate_rows_static(A.m, A.n, rp, ci, va, ud, vd, t, k, SEED, 0, z)
    torch.cuda.synchronize()
    got = z.cpu().double().numpy()
    assert np.all(np.isnan(got[bad_rows]))
    good = np.setdiff1d(np.arange(A.m), bad_rows)
    A64 = O.OracleCSR.from_any(A)
    zo = O.row_estimate(A64, u, v, O.probe_signs(SEED, t, 0, A.n, k))
    r2, _ = O.exact_norms_sq(A64, u, v)
    assert np.all(np.abs(got[good] - zo[good]) <= 3e-5 * r2[good] + 1e-30)


def test_static_estimator_refuses_more_columns_than_its_array():
    import torch

    n = sme.SME_STATIC_MAX_COLS + 1
    z = torch.zeros(4, dtype=torch.float32, device="cuda")
    rp = torch.zeros(5, dtype=torch.int32, device="cuda")
    ci = torch.zeros(0, dtype=torch.int32, device="cuda")
    va = torch.zeros(0, dtype=torch.float32, device="cuda")
    v = torch.zeros(n, dtype=torch.float32, device="cuda")
    with pytest.raises(sme.SmeError) as ei:
        sme.sme_estimate_rows_static(4, n, rp, ci, va, z, v, 1, 32, 0, 0, z)
    assert ei.value.name == "SME_ERR_ARG"


def test_static_estimator_binding_rejects_mistyped_arguments():
    import torch

    A = I.workload_large(scale=0.001, seed=23)
    rp, ci, va = _device_csr(A)
    u = torch.zeros(A.m, dtype=torch.float32, device="cuda")
    v = torch.zeros(A.n, dtype=torch.float32, device="cuda")
    z = torch.zeros(A.m, dtype=torch.float32, device="cuda")
    bad = [
        dict(ci=ci.long()),                              # int64 column indices
        dict(u=u.double()),                              # FP64 state
        dict(v=torch.zeros(2 * A.n, device="cuda")[::2]),  # non-contiguous
        dict(z=torch.zeros(A.m - 1, device="cuda")),       # wrong length
        dict(va=va.cpu()),                               # host tensor
    ]
    for over in bad:
        a = dict(rp=rp, ci=ci, va=va, u=u, v=v, z=z)
        a.update(over)
        with pytest.raises(sme.SmeError) as ei:
            sme.sme_estimate_rows_static(A.m, A.n, a["rp"], a["ci"], a["va"], a["u"], a["v"], 1, 8, 0, 0, a["z"])
        assert ei.value.name == "SME_ERR_ARG"
