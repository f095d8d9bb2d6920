"""Shared helpers for the GPU tests: run the library through its C ABI and fetch results."""
import numpy as np

from paper_1602_06621_gb300 import sme


def torch_dtype(dtype_code):
    import torch
    return torch.float64 if dtype_code == sme.SME_F64 else torch.float32


def make_op(A, dtype_code=None):
    if dtype_code is None:
        dtype_code = sme.SME_F64 if A.vals.dtype == np.float64 else sme.SME_F32
    vals = A.vals.astype(np.float64 if dtype_code == sme.SME_F64 else np.float32)
    return sme.sme_op_create_csr(A.m, A.n, A.row_ptr, A.col_idx, vals, dtype=dtype_code), dtype_code


def gpu_equilibrate(op, dtype_code, m, n, *, T, k, seed=0, state=None, **kw):
    import torch
    td = torch_dtype(dtype_code)
    if state is None:
        u, v = torch.zeros(m, dtype=td, device="cuda"), torch.zeros(n, dtype=td, device="cuda")
        ub, vb = torch.zeros(m, dtype=td, device="cuda"), torch.zeros(n, dtype=td, device="cuda")
    else:
        u, v, ub, vb = (torch.as_tensor(np.asarray(x), device="cuda").to(td) for x in state)
    sme.sme_equilibrate(op, u, v, ub, vb, T=T, k=k, seed=seed, **kw)
    torch.cuda.synchronize()
    return tuple(x.cpu().double().numpy() for x in (u, v, ub, vb))


def gpu_estimate(op, dtype_code, u, v, *, t, k, seed, stream_base=0):
    import torch
    td = torch_dtype(dtype_code)
    ud = torch.as_tensor(np.asarray(u), device="cuda").to(td)
    vd = torch.as_tensor(np.asarray(v), device="cuda").to(td)
    zu = torch.full((len(u),), float("nan"), dtype=td, device="cuda")
    zv = torch.full((len(v),), float("nan"), dtype=td, device="cuda")
    sme.sme_estimate(op, ud, vd, t, k, seed, stream_base, zu, zv)
    torch.cuda.synchronize()
    return zu.cpu().double().numpy(), zv.cpu().double().numpy()


def rel_norm(a, b):
    a = np.concatenate([np.ravel(x) for x in a])
    b = np.concatenate([np.ravel(x) for x in b])
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
