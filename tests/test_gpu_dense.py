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


@pytest.mark.parametrize("m,n", [(128, 128), (128, 1152), (256, 256), (384, 256), (256, 512), (1280, 384),
                                 (384, 2560)])
@pytest.mark.parametrize("k", [128, 256])
def test_dense_estimate_matches_oracle(m, n, k):
    """Shapes with an odd number of 128-row tiles (128, 384, 1280) exercise the spare CTA of the last cluster
    (at 128 one tile per side, a single cluster per product); 384 x 2560 runs more clusters than one per
    product."""
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


# ------------------------------------------------------------------ E4M3 storage and operands
#
# On an E4M3 operator the matrix stays E4M3 (A_ij = c_i q_ij) and each B operand is one E4M3 term,
# e4m3(2^S e^{x_j} c_j) s_jp, with a power-of-two S per operand.  Inside E4M3's normal range rounding
# y 2^S gives 2^S times y rounded to 4 significant bits (round to nearest, ties to even), whatever S is, so
# the scalings the tensor cores see are round4(e^{x_j} c_j).  The oracle is given exactly those (through
# the probe signs s_jp round4(e^{x_j} c_j) / (e^{x_j} c_j)), and then only FP32 accumulation separates the
# two: the bound _tol(K) above applies.  Against the exact scalings each estimate also carries the E4M3
# rounding of the scalings, at most 2^-4 relative per scaling: E_s[dz_i] = sum_j x_ij^2 (2 eps_j + eps_j^2),
# at most (2^-3 + 2^-8) r2_i, plus a zero-mean part whose standard deviation is below sqrt(2/k) times that;
# _F8_ROUNDING_BOUND = 0.19 covers both with five standard deviations at k = 128.

_F8_ROUNDING_BOUND = 0.19


def _round4(x):
    """Round to 4 significant bits, ties to even: E4M3 rounding inside its normal range."""
    x = np.asarray(x, np.float64)
    f, e = np.frexp(x)
    return np.ldexp(np.rint(f * 16.0) / 16.0, e)


def _e4m3_matrix(m, n, seed, var=1.5):
    """A badly scaled matrix quantised as the bench does: row i as E4M3 codes of A_i / c_i, c_i = max|A_i| / 448."""
    import torch
    A = I.dense_badly_scaled(m, n, seed, var=var).astype(np.float32)
    scales = (np.abs(A).max(axis=1) / 448.0).astype(np.float32)
    q = torch.tensor(A / scales[:, None]).to(torch.float8_e4m3fn)
    codes = q.view(torch.uint8).numpy().copy()
    codes[(codes & 0x7F) == 0x7F] = 0x38
    Af = _e4m3_values()[codes]  # exact E4M3 values
    return codes, scales, Af


def _fp8_op(codes, scales):
    import torch
    m, n = codes.shape
    return sme.sme_op_create_dense(m, n, torch.tensor(codes, device="cuda"), dtype=sme.SME_FP8E4M3,
                                   row_scales=torch.tensor(scales, device="cuda"))


def _rounded_signs(seed, t, stream, x, c, k):
    """Probe signs times round4(e^{x} c) / (e^{x} c): the oracle's estimate then sees the rounded scalings."""
    sc = np.exp(np.asarray(x, np.float64)) * (1.0 if c is None else np.asarray(c, np.float64))
    sc32 = np.exp(np.asarray(x, np.float32)).astype(np.float64) * (1.0 if c is None else np.asarray(c, np.float64))
    ratio = _round4(sc32) / sc
    return O.probe_signs(seed, t, stream, len(x), k) * ratio[:, None]


@pytest.mark.parametrize("m,n", [(128, 128), (1152, 128), (256, 256), (384, 256), (1280, 384), (384, 2560)])
@pytest.mark.parametrize("k", [128, 256])
def test_dense_fp8_representable_scalings_match_oracle(m, n, k):
    """Scalings chosen so that e^{v_j} and e^{u_i} c_i are E4M3 values: the operands are exact, so the E4M3
    path must match the oracle on the dequantised matrix within the FP32 accumulation bound."""
    codes, scales, Af = _e4m3_matrix(m, n, seed=m + n + k)
    rng = np.random.default_rng(k + 1)
    grid = _e4m3_values()[0x20:0x58]  # normal values 2^-3 .. 2^3 (codes 0x20 .. 0x57)
    qv = rng.choice(grid, n)
    qu = rng.choice(grid, m)
    v = np.log(qv).astype(np.float32)
    u = np.log(qu / scales.astype(np.float64)).astype(np.float32)
    op = _fp8_op(codes, scales)
    try:
        zu, zv = _gpu_estimate(op, m, n, u, v, t=3, k=k, seed=7)
    finally:
        sme.sme_op_destroy(op)
    ezu, ezv = O.dense_estimate_sampled(Af.astype(np.float32), u, v, np.arange(m), np.arange(n), t=3, k=k, seed=7,
                                        row_scale=scales)
    r2, c2 = _exact_sq(Af, u.astype(np.float64), v.astype(np.float64), row_scale=scales)
    assert np.all(np.abs(zu - ezu) <= _tol(n) * r2), np.max(np.abs(zu - ezu) / r2)
    assert np.all(np.abs(zv - ezv) <= _tol(m) * c2), np.max(np.abs(zv - ezv) / c2)


@pytest.mark.parametrize("m,n,k", [(256, 384, 256), (1280, 384, 128), (1280, 384, 256)])
def test_dense_fp8_estimate_equals_oracle_on_rounded_scalings(m, n, k):
    """Random scalings: equal to the oracle given the E4M3-rounded scalings (FP32 accumulation bound), and
    within _F8_ROUNDING_BOUND r2 of the oracle given the exact ones."""
    codes, scales, Af = _e4m3_matrix(m, n, seed=2 * m + n)
    rng = np.random.default_rng(5)
    u = rng.normal(0, 0.5, m).astype(np.float32)
    v = rng.normal(0, 0.5, n).astype(np.float32)
    t, seed = 4, 11
    op = _fp8_op(codes, scales)
    try:
        zu, zv = _gpu_estimate(op, m, n, u, v, t=t, k=k, seed=seed)
    finally:
        sme.sme_op_destroy(op)
    A64 = O.OracleCSR.from_any(Af * scales.astype(np.float64)[:, None])
    u64, v64 = u.astype(np.float64), v.astype(np.float64)
    r2, c2 = _exact_sq(Af, u64, v64, row_scale=scales)
    s_r = _rounded_signs(seed, t, 0, v, None, k)
    w_r = _rounded_signs(seed, t, 1, u, scales, k)
    rzu = O.row_estimate(A64, u64, v64, s_r)
    rzv = O.col_estimate(A64, u64, v64, w_r)
    assert np.all(np.abs(zu - rzu) <= _tol(n) * r2), np.max(np.abs(zu - rzu) / r2)
    assert np.all(np.abs(zv - rzv) <= _tol(m) * c2), np.max(np.abs(zv - rzv) / c2)
    ezu = O.row_estimate(A64, u64, v64, O.probe_signs(seed, t, 0, n, k))
    ezv = O.col_estimate(A64, u64, v64, O.probe_signs(seed, t, 1, m, k))
    assert np.all(np.abs(zu - ezu) <= _F8_ROUNDING_BOUND * r2), np.max(np.abs(zu - ezu) / r2)
    assert np.all(np.abs(zv - ezv) <= _F8_ROUNDING_BOUND * c2), np.max(np.abs(zv - ezv) / c2)


def test_dense_fp8_every_step_matches_oracle_on_rounded_scalings():
    """20 iterations of Algorithm 1 on an E4M3 operator (k = 256, step offset t0 = 100 so that the scalings
    stay inside E4M3's normal range), each step against the oracle's step from the GPU's own state with the
    E4M3-rounded scalings in its estimates (norm-wise relative error of [u; v; ubar; vbar] <= 1e-4).  This
    covers the operand scale exponents chosen from the step bound and the ring of per-iteration maxima."""
    import torch
    m, n, k, t0 = 1280, 384, 256, 100
    codes, scales, Af = _e4m3_matrix(m, n, seed=8, var=0.5)
    Aeff = Af * scales.astype(np.float64)[:, None]
    A64 = O.OracleCSR.from_any(Aeff)
    d = O.default_params(m, n)
    # Warm start: one sweep of row then column normalisation of |A|^2 towards alpha^2, beta^2 (the averages
    # start at the start point), so that the steps are small from the first one.
    u0 = -0.5 * np.log((Aeff ** 2).sum(1) / d["alpha"] ** 2)
    v0 = -0.5 * np.log(((Aeff ** 2) * np.exp(2 * u0)[:, None]).sum(0) / d["beta"] ** 2)
    u0, v0 = u0.astype(np.float32).astype(np.float64), v0.astype(np.float32).astype(np.float64)
    start = (u0, v0, u0.copy(), v0.copy())
    op = _fp8_op(codes, scales)
    worst = 0.0
    state = start
    try:
        for t in range(1, 21):
            g = [torch.tensor(x, dtype=torch.float32, device="cuda") for x in state]
            sme.sme_equilibrate(op, *g, T=1, k=k, seed=3, t_begin=t, t0=t0)
            got = [x.cpu().double().numpy() for x in g]
            # Each operand (its own scale exponent) stays inside the normal range below its scaled maximum.
            for sc in (np.exp(state[0]) * scales, np.exp(state[1])):
                assert sc.max() / sc.min() < 2.0 ** 12
            s_r = _rounded_signs(3, t, 0, state[1].astype(np.float32), None, k)
            w_r = _rounded_signs(3, t, 1, state[0].astype(np.float32), scales, k)
            ref = O.psgd_step(A64, *state, s_r, w_r, t, t0=t0, **d)
            a = np.concatenate(got)
            b = np.concatenate(ref)
            worst = max(worst, np.linalg.norm(a - b) / np.linalg.norm(b))
            state = tuple(got)
        # One 20-iteration call equals the step-by-step run (the scale exponents follow from the state).
        g = [torch.tensor(x, dtype=torch.float32, device="cuda") for x in start]
        sme.sme_equilibrate(op, *g, T=20, k=k, seed=3, t0=t0)
        for x, y in zip(g, state):
            np.testing.assert_array_equal(x.cpu().double().numpy(), y)
    finally:
        sme.sme_op_destroy(op)
    assert worst <= 1e-4, worst


def test_dense_fp8_whole_run_outcome_close_to_oracle():
    """Whole run from the zero start (paper's step, T = 60, k = 256) on a 256 x 384 E4M3 operator: the
    first steps move the scalings across E4M3's whole range, so the run is compared by its outcome with the
    oracle's run on the dequantised matrix.

    The single E4M3 term biases the fixed point: a row's expected estimate is sum_j x_ij^2 (1 + eps_j)^2 with
    |eps_j| <= 2^-4, so where the exact method settles at r2_i = alpha^2 - gamma u_i the E4M3 path settles at
    r2_i times a factor in [(1 + 2^-4)^-2, (1 - 2^-4)^-2]: each norm moves by at most (1 +- 2^-4)^-1, and the
    spread (a ratio of two norms) by at most (1 + 2^-4) / (1 - 2^-4) = 1.133.  Bound asserted: that factor
    times 1.05 for the finite run; the averaged scalings within 5 % norm-wise."""
    import torch
    m, n, k, T = 256, 384, 256, 60
    codes, scales, Af = _e4m3_matrix(m, n, seed=13)
    A64 = O.OracleCSR.from_any(Af * scales.astype(np.float64)[:, None])
    op = _fp8_op(codes, scales)
    try:
        g = [torch.zeros(x, device="cuda") for x in (m, n, m, n)]
        sme.sme_equilibrate(op, *g, T=T, k=k, seed=1)
        got = [x.cpu().double().numpy() for x in g]
    finally:
        sme.sme_op_destroy(op)
    O.set_parallel(True)  # the OpenMP build of the oracle: the checker's bits on every host core
    try:
        ref = O.equilibrate(A64, T=T, k=k, seed=1)
    finally:
        O.set_parallel(False)
    ub = np.concatenate(got[2:])
    rb = np.concatenate(ref[2:])
    assert np.linalg.norm(ub - rb) / np.linalg.norm(rb) <= 0.05
    sg = max(O.spread(*O.exact_norms_sq(A64, got[2], got[3])))
    so = max(O.spread(*O.exact_norms_sq(A64, ref[2], ref[3])))
    bias = (1 + 2.0 ** -4) / (1 - 2.0 ** -4)
    assert so / (1.05 * bias) <= sg <= so * 1.05 * bias, (sg, so)


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


def test_dense_fp8_full_size_sampled_estimate():
    """16384 x 16384 E4M3 with per-row scales (the dense workload's quantisation), k = 256: 24 sampled rows and
    24 columns of one estimate against the oracle given the E4M3-rounded scalings (rows: u and round4(e^{v});
    columns: round4(e^{u} c) and v), within the FP32 accumulation bound; and within _F8_ROUNDING_BOUND r2 of
    the oracle given the exact scalings."""
    m = n = 16384
    codes, scales, Af = _e4m3_matrix(m, n, seed=3)
    op = _fp8_op(codes, scales)
    try:
        rng = np.random.default_rng(0)
        u = rng.normal(0, 0.5, m).astype(np.float32)
        v = rng.normal(0, 0.5, n).astype(np.float32)
        zu, zv = _gpu_estimate(op, m, n, u, v, t=1, k=256, seed=0)
    finally:
        sme.sme_op_destroy(op)
    assert np.all(np.isfinite(zu)) and np.all(np.isfinite(zv))
    rows = np.sort(rng.choice(m, 24, replace=False))
    cols = np.sort(rng.choice(n, 24, replace=False))
    u64, v64 = u.astype(np.float64), v.astype(np.float64)
    c64 = scales.astype(np.float64)
    v_r = np.log(_round4(np.exp(v).astype(np.float64)))
    u_r = np.log(_round4(np.exp(u).astype(np.float64) * c64) / c64)
    Af32 = Af.astype(np.float32)
    rzu, _ = O.dense_estimate_sampled(Af32, u64, v_r, rows, [], t=1, k=256, seed=0, row_scale=c64)
    _, rzv = O.dense_estimate_sampled(Af32, u_r, v64, [], cols, t=1, k=256, seed=0, row_scale=c64)
    ezu, ezv = O.dense_estimate_sampled(Af32, u64, v64, rows, cols, t=1, k=256, seed=0, row_scale=c64)
    r2 = np.array([np.sum((np.exp(u64[i]) * c64[i] * Af[i] * np.exp(v64)) ** 2) for i in rows])
    c2 = np.array([np.sum((np.exp(u64) * c64 * Af[:, j] * np.exp(v64[j])) ** 2) for j in cols])
    assert np.all(np.abs(zu[rows] - rzu) <= _tol(n) * r2), np.max(np.abs(zu[rows] - rzu) / r2)
    assert np.all(np.abs(zv[cols] - rzv) <= _tol(m) * c2), np.max(np.abs(zv[cols] - rzv) / c2)
    assert np.all(np.abs(zu[rows] - ezu) <= _F8_ROUNDING_BOUND * r2)
    assert np.all(np.abs(zv[cols] - ezv) <= _F8_ROUNDING_BOUND * c2)


@pytest.mark.parametrize("fp8", [False, True])
def test_dense_pipeline_waits_expire_without_writing(fp8):
    """The failure path of the tensor-core kernels, without a GPU fault: with SME_EQ_EXPIRE_PIPELINE_WAITS the
    producer's and the MMA issuer's waits give up at once, so every launch stops before its first MMA.  The
    call must return SME_ERR_TIMEOUT and leave u, v and the averages exactly as passed in; the drain (the
    accumulator barrier, TMEM released only once no MMA is in flight, copies in flight allowed to land) must
    leave the operator usable: the next call on it, and a call on a fresh operator, equal an undisturbed
    run bit for bit.  256 x 256, k = 256."""
    import torch
    m = n = 256
    if fp8:
        codes, scales, _ = _e4m3_matrix(m, n, seed=31)
        make = lambda: _fp8_op(codes, scales)
    else:
        Ad, _ = _bf16_matrix(m, n, seed=31)
        make = lambda: sme.sme_op_create_dense(m, n, Ad, dtype=sme.SME_BF16)

    def run(op, start, flags=0):
        g = [torch.tensor(x, dtype=torch.float32, device="cuda") for x in start]
        sme.sme_equilibrate(op, *g, T=3, k=256, seed=4, flags=flags)
        return [x.cpu().numpy() for x in g]

    zero = [np.zeros(m, np.float32), np.zeros(n, np.float32), np.zeros(m, np.float32), np.zeros(n, np.float32)]
    rng = np.random.default_rng(2)
    start = [rng.normal(0, 0.3, x.size).astype(np.float32) for x in zero]
    op = make()
    try:
        ref = run(op, zero)
        g = [torch.tensor(x, device="cuda") for x in start]
        with pytest.raises(sme.SmeError) as ei:
            sme.sme_equilibrate(op, *g, T=3, k=256, seed=4, flags=sme.SME_EQ_EXPIRE_PIPELINE_WAITS)
        assert ei.value.name == "SME_ERR_TIMEOUT"
        for x, y in zip(g, start):
            np.testing.assert_array_equal(x.cpu().numpy(), y)
        again = run(op, zero)
    finally:
        sme.sme_op_destroy(op)
    op = make()
    try:
        fresh = run(op, zero)
    finally:
        sme.sme_op_destroy(op)
    for a, b, c in zip(ref, again, fresh):
        np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(a, c)


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
