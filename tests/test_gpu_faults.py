"""Failure injection on the host: device allocations that fail (SME_FAIL_DEV_ALLOC) at every point of an
operator's life must come back as SME_ERR_OOM, leave nothing allocated, and leave the library usable -
including the operator itself, on which the same call succeeds once allocations succeed again."""
import numpy as np
import pytest

from paper_1602_06621_gb300 import inputs as I
from paper_1602_06621_gb300 import sme

pytestmark = pytest.mark.gpu


def _life(A, torch, heal=None):
    """Create, equilibrate, solve, evaluate, destroy.  heal(): called after a failed phase, before the phase
    is retried once on the same operator."""
    op = sme.sme_op_create_csr(A.m, A.n, A.row_ptr, A.col_idx, A.vals)
    failed = 0
    try:
        z = [torch.zeros(x, device="cuda") for x in (A.m, A.n, A.m, A.n)]
        b = torch.ones(A.m, device="cuda")
        x = torch.zeros(A.n, device="cuda")
        phases = [lambda: sme.sme_equilibrate(op, *[t.zero_() for t in z], T=5, k=32, seed=0),
                  lambda: sme.sme_lsqr(op, z[2], z[3], b, x, tol=0.0, max_iters=5, check_every=5),
                  lambda: sme.sme_evaluate(op, z[2], z[3])]
        for phase in phases:
            try:
                out = phase()
            except sme.SmeError as e:
                if heal is None or e.name != "SME_ERR_OOM":
                    raise
                failed += 1
                heal()
                out = phase()
        return out["rms"], failed
    finally:
        sme.sme_op_destroy(op)


def test_every_failed_allocation_is_reported_and_cleaned_up(monkeypatch):
    import torch
    A = I.workload_large(scale=0.002, seed=7)
    ref, _ = _life(A, torch)
    sme.sme_release_cached_memory()  # blocks of destroyed operators are kept for reuse; measure without them
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    in_create = in_calls = 0
    for k in range(60):
        monkeypatch.setenv("SME_FAIL_DEV_ALLOC", str(k))
        try:
            rms, failed = _life(A, torch, heal=lambda: monkeypatch.delenv("SME_FAIL_DEV_ALLOC"))
            in_calls += failed
            assert rms == ref, k  # the retried call on the same operator gives the undisturbed result
        except sme.SmeError as e:
            assert e.name == "SME_ERR_OOM", (k, e.name)  # failed while creating the operator
            in_create += 1
        monkeypatch.delenv("SME_FAIL_DEV_ALLOC", raising=False)
        assert _life(A, torch)[0] == ref  # nothing left in a bad state
    assert in_create >= 5 and in_calls >= 5, (in_create, in_calls)  # both kinds of allocation were reached
    sme.sme_release_cached_memory()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 >= free0 - (64 << 20), (free0, free1)  # no device memory leaked across 60 lives


def test_destroyed_operator_memory_is_reused_and_released():
    """A second operator of the same shape takes the first one's blocks (same results, same device bytes);
    sme_release_cached_memory returns them to the device."""
    import torch
    A = I.workload_large(scale=0.01, seed=9)
    outs, sizes = [], []
    for _ in range(2):
        op = sme.sme_op_create_csr(A.m, A.n, A.row_ptr, A.col_idx, A.vals)
        try:
            z = [torch.zeros(x, device="cuda") for x in (A.m, A.n, A.m, A.n)]
            sme.sme_equilibrate(op, *z, T=10, k=32, seed=1)
            outs.append([t.cpu().numpy() for t in z])
            sizes.append(sme.sme_op_get_info(op)["device_bytes"])
        finally:
            sme.sme_op_destroy(op)
    assert sizes[0] == sizes[1]
    for x, y in zip(*outs):
        np.testing.assert_array_equal(x, y)
    torch.cuda.synchronize()
    held = torch.cuda.mem_get_info()[0]
    sme.sme_release_cached_memory()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= held + sizes[0] // 2  # the idle blocks went back to the device
