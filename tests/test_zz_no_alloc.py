"""The allocation-free row estimator against the regular one, on the GPU.

sme_estimate_rows_static serves callers that cannot allocate device memory on
their hot path (work being recorded into a CUDA graph, a process whose device
memory is held by a caching allocator, latency-critical loops).  It keeps its
gather table in a fixed array inside the library, so this test checks that two
calls in a row -- the second overwriting the table the first left behind --
each give what sme_estimate gives for the same inputs, within the FP32
tolerance used throughout (|dz_i| <= 3e-5 r2_i, r2_i the exact squared row
norm), and that a size beyond the array is refused.

This file is named to be collected last, so a run stopping at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

import oracle as O
from paper_1602_06621_gb300 import inputs as I
from paper_1602_06621_gb300 import sme

pytestmark = pytest.mark.gpu


def test_static_estimator_matches_regular_estimator_twice_in_a_row():
    import torch

    A = I.workload_large(scale=0.02, seed=21)  # 20000 x 10000, 20 nonzeros per row, FP32
    op = sme.sme_op_create_csr(A.m, A.n, A.row_ptr, A.col_idx, A.vals)
    try:
        dev = dict(device="cuda")
        rp = torch.tensor(A.row_ptr, **dev)
        ci = torch.tensor(A.col_idx, **dev)
        va = torch.tensor(A.vals, **dev)
        rng = np.random.default_rng(3)
        A64 = O.OracleCSR.from_any(A)
        for call, (t, k) in enumerate([(4, 32), (9, 16)]):
            u = rng.normal(0, 0.5, A.m).astype(np.float32)
            v = rng.normal(0, 0.5, A.n).astype(np.float32)
            ud, vd = torch.tensor(u, **dev), torch.tensor(v, **dev)
            z_ref = torch.full((A.m,), float("nan"), dtype=torch.float32, **dev)
            sme.sme_estimate(op, ud, vd, t, k, 5, 0, z_ref, None)
            z_new = torch.full((A.m,), float("nan"), dtype=torch.float32, **dev)
            sme.sme_estimate_rows_static(A.m, A.n, rp, ci, va, ud, vd, t, k, 5, 0, z_new)
            torch.cuda.synchronize()
            r2, _ = O.exact_norms_sq(A64, u, v)
            diff = np.abs(z_new.cpu().double().numpy() - z_ref.cpu().double().numpy())
            assert np.all(diff <= 3e-5 * r2 + 1e-30), f"call {call}: max excess {np.max(diff - 3e-5 * r2)}"
    finally:
        sme.sme_op_destroy(op)


def test_static_estimator_refuses_more_columns_than_its_array():
    import torch

    n = sme.SME_STATIC_MAX_COLS + 1
    z = torch.zeros(4, dtype=torch.float32, device="cuda")
    rp = torch.zeros(5, dtype=torch.int32, device="cuda")
    with pytest.raises(sme.SmeError) as ei:
        sme.sme_estimate_rows_static(4, n, rp, rp, z, z, z, 1, 32, 0, 0, z)
    assert ei.value.name == "SME_ERR_ARG"
