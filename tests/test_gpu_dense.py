"""GPU parity of the dense tensor-core path (BF16 and FP8-E4M3 operands, FP32 accumulation).

The oracle sees the same matrix the tensor cores see (the BF16- or E4M3-rounded values, widened to
FP64), so what is measured is the arithmetic of the path:
  * the two-term BF16 split of the scalings (relative error <= 2^-17 per scaling), and
  * FP32 accumulation in the tensor cores, which aligns and truncates (rounds toward zero) when it adds
    each block of products to the accumulator, so its error is one-sided and grows with the number of
    16-term MMAs, K/16: on average about 2^-24 of the accumulator per MMA.
Bound used: |dz_i| <= (2e-5 + (K/16) 2^-24) r2_i, with r2_i the exact squared norm of row i of DAE and K the
reduction length (n for rows, m for columns).  At K = 16384 that is 8.1e-5; the measured error there is
about 3e-5, biased low.
"""
import numpy as np
import pytest

import oracle as O
from paper_1602_06621_gb300 import inputs as I
from paper_1602_06621_gb300 import sme

pytestmark = pytest.mark.gpu


def _bf16_matrix(m, n, seed):
    import torch
    A = torch.tensor(I.dense_badly_scaled(m, n, seed), dtype=torch.float32)
    Ab = A.to(torch.bfloat16)
    return Ab.cuda(), Ab.float().numpy()


def _exact_sq(Af, u, v, row_scale=None):
    B = np.exp(u)[:, None] * Af.astype(np.float64) * np.exp(v)[None, :]
    if row_scale is not None:
        B = B * np.asarray(row_scale, np.float64)[:, None]
    return (B ** 2).sum(1), (B ** 2).sum(0)


def _tol(K):
    return 2e-5 + (K / 16) * 2.0 ** -24


def _gpu_estimate(op, m, n, u, v, t, k, seed):
    import torch
    zu = torch.full((m,), float("nan"), device="cuda")
    zv = torch.full((n,), float("nan"), device="cuda")
    sme.sme_estimate(op, torch.tensor(u, dtype=torch.float32, device="cuda"),
                     torch.tensor(v, dtype=torch.float32, device="cuda"), t, k, seed, 0, zu, zv)
    torch.cuda.synchronize()
    return zu.cpu().double().numpy(), zv.cpu().double().numpy()


@pytest.mark.parametrize("m,n", [(256, 256), (384, 256), (256, 512), (1280, 384), (384, 2560)])
@pytest.mark.parametrize("k", [128, 256])
def test_dense_estimate_matches_oracle(m, n, k):
    """Shapes with an odd number of 128-row tiles (384, 1280) exercise the spare CTA of the last cluster;
    384 x 2560 runs more clusters than one per product."""
    Ad, Af = _bf16_matrix(m, n, seed=m + n + k)
    op = sme.sme_op_create_dense(m, n, Ad, dtype=sme.SME_BF16)
    try:
        rng = np.random.default_rng(k)
        u = rng.normal(0, 0.5, m).astype(np.float32)
        v = rng.normal(0, 0.5, n).astype(np.float32)
        zu, zv = _gpu_estimate(op, m, n, u, v, t=3, k=k, seed=7)
    finally:
        sme.sme_op_destroy(op)
    ezu, ezv = O.dense_estimate_sampled(Af, u, v, np.arange(m), np.arange(n), t=3, k=k, seed=7)
    r2, c2 = _exact_sq(Af, u.astype(np.float64), v.astype(np.float64))
    assert np.all(np.abs(zu - ezu) <= _tol(n) * r2), np.max(np.abs(zu - ezu) / r2)
    assert np.all(np.abs(zv - ezv) <= _tol(m) * c2), np.max(np.abs(zv - ezv) / c2)


@pytest.mark.parametrize("m,n", [(256, 384), (1280, 384)])
def test_dense_every_step_matches_oracle(m, n):
    """20 iterations of Algorithm 1 on a dense matrix, k = 256, each step checked against the oracle's step
    from the GPU's own state (norm-wise relative error of [u; v; ubar; vbar] <= 1e-4)."""
    import torch
    k = 256
    Ad, Af = _bf16_matrix(m, n, seed=5)
    A64 = O.OracleCSR.from_any(Af.astype(np.float64))
    d = O.default_params(m, n)
    op = sme.sme_op_create_dense(m, n, Ad, dtype=sme.SME_BF16)
    worst = 0.0
    state = (np.zeros(m), np.zeros(n), np.zeros(m), np.zeros(n))
    try:
        for t in range(1, 21):
            g = [torch.tensor(x, dtype=torch.float32, device="cuda") for x in state]
            sme.sme_equilibrate(op, *g, T=1, k=k, seed=3, t_begin=t)
            got = [x.cpu().double().numpy() for x in g]
            ref = O.psgd_step(A64, *state, O.probe_signs(3, t, 0, n, k), O.probe_signs(3, t, 1, m, k), t, **d)
            a = np.concatenate(got)
            b = np.concatenate(ref)
            worst = max(worst, np.linalg.norm(a - b) / np.linalg.norm(b))
            state = tuple(got)
        # One 20-iteration call equals the step-by-step run (resume is exact on the dense path too).
        g = [torch.zeros(x, device="cuda") for x in (m, n, m, n)]
        sme.sme_equilibrate(op, *g, T=20, k=k, seed=3)
        for x, y in zip(g, state):
            np.testing.assert_array_equal(x.cpu().double().numpy(), y)
    finally:
        sme.sme_op_destroy(op)
    assert worst <= 1e-4, worst


def _e4m3_values():
    """The 256 E4M3 code points (1 sign, 4 exponent bits with bias 7, 3 mantissa bits; codes 0x7f and 0xff
    are NaN, there is no infinity)."""
    vals = np.zeros(256)
    for b in range(256):
        s, e, f = b >> 7, (b >> 3) & 15, b & 7
        if (b & 0x7F) == 0x7F:
            vals[b] = np.nan
            continue
        v = f * 2.0 ** -9 if e == 0 else (8 + f) * 2.0 ** (e - 10)
        vals[b] = -v if s else v
    return vals


def test_dense_fp8_with_row_scales_matches_oracle():
    import torch
    m, n, k = 256, 256, 256
    rng = np.random.default_rng(11)
    codes = rng.integers(0, 256, size=(m, n)).astype(np.uint8)
    codes[(codes & 0x7F) == 0x7F] = 0x38  # no NaN codes (0x38 is 1.0)
    scales = np.exp(rng.normal(0, 1.5, m)).astype(np.float32)
    table = _e4m3_values()
    Af = table[codes].astype(np.float32)  # exact
    op = sme.sme_op_create_dense(m, n, torch.tensor(codes, device="cuda"), dtype=sme.SME_FP8E4M3,
                                 row_scales=torch.tensor(scales, device="cuda"))
    try:
        u = rng.normal(0, 0.5, m).astype(np.float32)
        v = rng.normal(0, 0.5, n).astype(np.float32)
        zu, zv = _gpu_estimate(op, m, n, u, v, t=2, k=k, seed=9)
    finally:
        sme.sme_op_destroy(op)
    ezu, ezv = O.dense_estimate_sampled(Af, u, v, np.arange(m), np.arange(n), t=2, k=k, seed=9, row_scale=scales)
    r2, c2 = _exact_sq(Af, u.astype(np.float64), v.astype(np.float64), row_scale=scales)
    assert np.all(np.abs(zu - ezu) <= _tol(n) * r2)
    assert np.all(np.abs(zv - ezv) <= _tol(m) * c2)


def test_dense_full_size_sampled_estimate():
    """16384 x 16384 BF16 (entries N(0,1) e^{r_i + c_j}, factors of variance 1.5), k = 256: sampled rows and
    columns of one estimate against the oracle."""
    import torch
    m = n = 16384
    A32 = I.dense_badly_scaled(m, n, seed=3)
    Ad = torch.from_numpy(A32).to(torch.bfloat16).cuda()
    Af = Ad.float().cpu().numpy()
    del A32
    op = sme.sme_op_create_dense(m, n, Ad, dtype=sme.SME_BF16)
    try:
        rng = np.random.default_rng(0)
        u = rng.normal(0, 0.5, m).astype(np.float32)
        v = rng.normal(0, 0.5, n).astype(np.float32)
        zu, zv = _gpu_estimate(op, m, n, u, v, t=1, k=256, seed=0)
    finally:
        sme.sme_op_destroy(op)
    rows = np.sort(rng.choice(m, 24, replace=False))
    cols = np.sort(rng.choice(n, 24, replace=False))
    ezu, ezv = O.dense_estimate_sampled(Af, u, v, rows, cols, t=1, k=256, seed=0)
    u64, v64 = u.astype(np.float64), v.astype(np.float64)
    r2 = np.array([np.sum((np.exp(u64[i]) * Af[i].astype(np.float64) * np.exp(v64)) ** 2) for i in rows])
    c2 = np.array([np.sum((np.exp(u64) * Af[:, j].astype(np.float64) * np.exp(v64[j])) ** 2) for j in cols])
    assert np.all(np.abs(zu[rows] - ezu) <= _tol(n) * r2), np.max(np.abs(zu[rows] - ezu) / r2)
    assert np.all(np.abs(zv[cols] - ezv) <= _tol(m) * c2), np.max(np.abs(zv[cols] - ezv) / c2)
    assert np.all(np.isfinite(zu)) and np.all(np.isfinite(zv))


def test_dense_argument_errors():
    import torch
    A = torch.zeros((200, 256), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(sme.SmeError) as ei:
        sme.sme_op_create_dense(200, 256, A, dtype=sme.SME_BF16)
    assert ei.value.name == "SME_ERR_ARG"
    A = torch.zeros((256, 256), dtype=torch.bfloat16, device="cuda")
    op = sme.sme_op_create_dense(256, 256, A, dtype=sme.SME_BF16)
    try:
        z = torch.zeros(256, device="cuda")
        with pytest.raises(sme.SmeError) as ei:
            sme.sme_equilibrate(op, z, z.clone(), z.clone(), z.clone(), T=1, k=32)
        assert ei.value.name == "SME_ERR_UNSUPPORTED"
    finally:
        sme.sme_op_destroy(op)
    A[3, 4] = float("nan")
    with pytest.raises(sme.SmeError) as ei:
        sme.sme_op_create_dense(256, 256, A, dtype=sme.SME_BF16)
    assert ei.value.name == "SME_ERR_NONFINITE"


@pytest.mark.parametrize("fp8", [False, True])
def test_dense_evaluate_matches_oracle(fp8):
    """sme_evaluate on a dense operator: exact norms of D A E (FP64 accumulation) and the metrics built from
    them, against the oracle's exact norms and objective on the dequantised matrix."""
    import torch
    m, n = 384, 256
    rng = np.random.default_rng(21)
    scales = None
    if fp8:
        codes = rng.integers(0, 256, size=(m, n)).astype(np.uint8)
        codes[(codes & 0x7F) == 0x7F] = 0x38
        scales = np.exp(rng.normal(0, 1.0, m)).astype(np.float32)
        Af = _e4m3_values()[codes]
        op = sme.sme_op_create_dense(m, n, torch.tensor(codes, device="cuda"), dtype=sme.SME_FP8E4M3,
                                     row_scales=torch.tensor(scales, device="cuda"))
        Aeff = Af * scales.astype(np.float64)[:, None]
    else:
        Ad, Af = _bf16_matrix(m, n, 22)
        op = sme.sme_op_create_dense(m, n, Ad, dtype=sme.SME_BF16)
        Aeff = Af.astype(np.float64)
    try:
        u = rng.normal(0, 0.5, m).astype(np.float32)
        v = rng.normal(0, 0.5, n).astype(np.float32)
        r2 = torch.zeros(m, dtype=torch.float64, device="cuda")
        c2 = torch.zeros(n, dtype=torch.float64, device="cuda")
        got = sme.sme_evaluate(op, torch.tensor(u, device="cuda"), torch.tensor(v, device="cuda"), gamma=0.05,
                               r2=r2, c2=c2)
        r2, c2 = r2.cpu().numpy(), c2.cpu().numpy()
    finally:
        sme.sme_op_destroy(op)
    er2, ec2 = O.exact_norms_sq(Aeff, u.astype(np.float64), v.astype(np.float64))
    np.testing.assert_allclose(r2, er2, rtol=1e-12)
    np.testing.assert_allclose(c2, ec2, rtol=1e-12)
    d = O.default_params(m, n)
    f = O.objective(Aeff, u.astype(np.float64), v.astype(np.float64), alpha=d["alpha"], beta=d["beta"], gamma=0.05)
    assert got["objective"] == pytest.approx(f, rel=1e-10)
    rn, cn = np.sqrt(er2[er2 > 0]), np.sqrt(ec2[ec2 > 0])
    assert got["row_spread"] == pytest.approx(rn.max() / rn.min(), rel=1e-10)
    assert got["col_spread"] == pytest.approx(cn.max() / cn.min(), rel=1e-10)
    assert got["rms"] == pytest.approx(O.rms_error(er2, ec2, d["alpha"], d["beta"]), rel=1e-10)
