"""The learned warm start on the GPU: the MLP kernels against the FP64 oracle (oracle/mlp.py), the feature
kernel against the oracle's estimator, and the warm start's effect on Algorithm 1."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import mlp as OM
from paper_1602_06621_gb300 import inputs as I
from paper_1602_06621_gb300 import sme as S

pytestmark = pytest.mark.gpu


def _bf16(p):
    """FP32 -> BF16 round to nearest even, as the device's copies (host arithmetic on the bit pattern)."""
    b = np.asarray(p, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _norm(rng):
    return np.concatenate([rng.normal(0, 0.5, OM.IN), np.exp(rng.normal(0, 0.3, OM.IN))]).astype(np.float32)


def _net(seed, rng):
    mlp = S.sme_mlp_create(seed)
    p = S.sme_mlp_get_params(mlp)[0]
    o = np.cumsum([0] + [size for _, size in OM.SIZES])
    for b in (1, 3, 5):  # b1, b2, b3: zero after He initialisation, nonzero here so that every term is exercised
        p[o[b]:o[b + 1]] = rng.normal(0, 0.3, o[b + 1] - o[b]).astype(np.float32)
    S.sme_mlp_set_params(mlp, p, _norm(rng))
    return mlp


def test_bf16_helper_rounds_to_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5 + 2 ** -9, 1.0 + 2 ** -7], np.float32)
    np.testing.assert_array_equal(_bf16(x), [1.0, 1.0, 1.0 + 2 ** -6, -2.5, 1.0 + 2 ** -7])


@pytest.mark.parametrize("N", [1, 31, 1000, 40000])
def test_forward_matches_oracle(N):
    rng = np.random.default_rng(N)
    mlp = _net(7, rng)
    try:
        p, nrm = S.sme_mlp_get_params(mlp)
        X = rng.normal(0, 1.5, (N, OM.IN)).astype(np.float32)
        y = torch.full((N,), np.nan, dtype=torch.float32, device="cuda")
        S.sme_mlp_forward(mlp, torch.from_numpy(X).cuda(), y)
        torch.cuda.synchronize()
        ref, _ = OM.forward(_bf16(p), X, nrm.astype(np.float64))
        got = y.cpu().double().numpy()
        # FP32 accumulation over 128 products per unit: a few ulps of the magnitudes involved.
        scale = 1.0 + np.abs(ref)
        assert np.max(np.abs(got - ref) / scale) < 2e-5
    finally:
        S.sme_mlp_destroy(mlp)


@pytest.mark.parametrize("N", [5, 32 * 152 * 2 + 17])
def test_gradient_matches_oracle_and_is_deterministic(N):
    rng = np.random.default_rng(100 + N)
    mlp = _net(11, rng)
    try:
        p, nrm = S.sme_mlp_get_params(mlp)
        X = rng.normal(0, 1.5, (N, OM.IN)).astype(np.float32)
        tgt = rng.normal(0, 2.0, N).astype(np.float32)
        Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(tgt).cuda()
        g1 = torch.zeros(OM.COUNT, dtype=torch.float32, device="cuda")
        g2 = torch.zeros_like(g1)
        loss = S.sme_mlp_gradient(mlp, Xd, td, g1)
        S.sme_mlp_gradient(mlp, Xd, td, g2)
        assert torch.equal(g1, g2)
        ref_loss, ref_g = OM.loss_and_gradient(_bf16(p), X, tgt, nrm.astype(np.float64))
        assert abs(loss - ref_loss) <= 1e-5 * ref_loss
        g = g1.cpu().double().numpy()
        assert np.linalg.norm(g - ref_g) <= 1e-4 * np.linalg.norm(ref_g)
        # Each block of the layout separately, so that a wrong offset cannot hide in a larger block.
        o = 0
        for name, size in OM.SIZES:
            blk = slice(o, o + size)
            assert np.linalg.norm(g[blk] - ref_g[blk]) <= 1e-4 * np.linalg.norm(ref_g[blk]) + 1e-7, name
            o += size
    finally:
        S.sme_mlp_destroy(mlp)


def test_adam_first_step():
    """First Adam step from zero moments: p - lr * g / (|g| + eps) (bias corrections cancel)."""
    rng = np.random.default_rng(5)
    mlp = _net(13, rng)
    try:
        p, nrm = S.sme_mlp_get_params(mlp)
        N = 3000
        X = rng.normal(0, 1, (N, OM.IN)).astype(np.float32)
        tgt = rng.normal(0, 1, N).astype(np.float32)
        _, g = OM.loss_and_gradient(_bf16(p), X, tgt, nrm.astype(np.float64))
        lr = 1e-3
        S.sme_mlp_train_step(mlp, torch.from_numpy(X).cuda(), torch.from_numpy(tgt).cuda(), lr)
        p1 = S.sme_mlp_get_params(mlp)[0].astype(np.float64)
        big = np.abs(g) > 1e-3 * np.abs(g).max()
        np.testing.assert_allclose(p1[big], (p - lr * np.sign(g))[big], rtol=0, atol=2e-6)
        assert np.all(np.abs(p1 - p) <= lr * 1.0001)
    finally:
        S.sme_mlp_destroy(mlp)


def test_training_fits_a_smooth_function():
    rng = np.random.default_rng(6)
    mlp = S.sme_mlp_create(3)
    try:
        N = 50000
        X = rng.normal(0, 1, (N, OM.IN)).astype(np.float32)
        y = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - 0.3 * X[:, 3]).astype(np.float32)
        S.sme_mlp_set_params(mlp, None, np.concatenate([np.zeros(8), np.ones(8)]).astype(np.float32))
        Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
        first = S.sme_mlp_gradient(mlp, Xd, yd)
        for _ in range(300):
            S.sme_mlp_train_step(mlp, Xd, yd, 3e-3)
        last = S.sme_mlp_gradient(mlp, Xd, yd)
        assert last < 0.05 * first, (first, last)
    finally:
        S.sme_mlp_destroy(mlp)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_features_match_oracle(dtype):
    A = I.sparse_variable_row_nnz(700, 300, 0, 20, 4, var=2.0, dtype=dtype)
    op = S.sme_op_create_csr(A.m, A.n, A.row_ptr, A.col_idx, A.vals)
    try:
        Fr = torch.zeros((A.m, 8), dtype=torch.float32, device="cuda")
        Fc = torch.zeros((A.n, 8), dtype=torch.float32, device="cuda")
        S.sme_op_features(op, 9, Fr, Fc)
        Fr, Fc = Fr.cpu().double().numpy(), Fc.cpu().double().numpy()
    finally:
        S.sme_op_destroy(op)
    z_r = O.row_estimate(A, np.zeros(A.m), np.zeros(A.n), O.probe_signs(9, 1, 0, A.n, 8))
    z_c = O.col_estimate(A, np.zeros(A.m), np.zeros(A.n), O.probe_signs(9, 1, 1, A.m, 8))
    rows = np.repeat(np.arange(A.m), np.diff(A.row_ptr))
    vals = np.asarray(A.vals, np.float64)
    nnz_r = np.bincount(rows[vals != 0], minlength=A.m)
    nnz_c = np.bincount(A.col_idx[vals != 0], minlength=A.n)
    sabs_r = np.bincount(rows, np.abs(vals), minlength=A.m)
    sabs_c = np.bincount(A.col_idx, np.abs(vals), minlength=A.n)
    f0 = lambda z: 0.5 * np.log(np.maximum(z, 1e-30))
    mean_abs = lambda s, c: np.log(np.maximum(np.where(c > 0, s / np.maximum(c, 1), 0.0), 1e-30))
    tol = 1e-4 if dtype == np.float32 else 1e-5
    for F, z, c, s, side in ((Fr, z_r, nnz_r, sabs_r, 0.0), (Fc, z_c, nnz_c, sabs_c, 1.0)):
        nz = z > 0
        np.testing.assert_allclose(F[nz, 0], f0(z[nz]), atol=tol)
        np.testing.assert_allclose(F[:, 1], np.log1p(c), atol=1e-6)
        np.testing.assert_allclose(F[c > 0, 2], mean_abs(s, c)[c > 0], atol=1e-5)
        assert np.all(F[:, 3] == side)
        np.testing.assert_allclose(F[:, 4], f0(z_r).mean(), atol=1e-4)
        np.testing.assert_allclose(F[:, 5], f0(z_c).mean(), atol=1e-4)
        np.testing.assert_allclose(F[:, 6], np.log(A.m), rtol=1e-6)
        np.testing.assert_allclose(F[:, 7], np.log(A.n), rtol=1e-6)
    assert (nnz_r == 0).any()  # the generator's empty rows are covered


def test_warm_start_beats_zero_start_on_held_out_matrices():
    """Train on one family sample, then on unseen matrices of the same family: after the same short run, the
    warm-started average has a lower objective (eq. (3)) than Algorithm 1 from zero."""
    from paper_1602_06621_gb300 import warmstart as W
    mats = I.batched_family(14, 800, 6000, seed=21)
    train, held = mats[:10], mats[10:]
    X, y = W.training_set(train, T=400, k=32, seed=1)
    mlp = S.sme_mlp_create(0)
    try:
        hist = W.train(mlp, X, y, steps=800, batch=8192, lr=2e-3)
        assert hist[-1][1] < 0.5 * hist[0][1], hist
        for i, A in enumerate(held):
            _, _, zero = W.run(A, T=20, k=32, seed=50 + i)
            _, _, warm = W.run(A, T=20, k=32, seed=50 + i, mlp=mlp, t0=W.WARM_T0)
            _, _, long = W.run(A, T=400, k=32, seed=50 + i)
            assert warm["objective"] < zero["objective"], (i, zero, warm)
            # 20 warm-started iterations come close to 400 from zero (RMS within a factor 2; zero-started
            # runs of 20 iterations are still several times worse).
            assert warm["rms"] < 0.3 * zero["rms"], (i, zero, warm)
            assert warm["rms"] < 2.0 * long["rms"], (i, long, warm)
    finally:
        S.sme_mlp_destroy(mlp)


def _batch3():
    return [I.sparse_variable_row_nnz(300, 200, 0, 12, 31, var=2.0),
            I.sparse_variable_row_nnz(450, 120, 1, 20, 32, var=2.0),
            I.sparse_variable_row_nnz(90, 260, 2, 30, 33, var=2.0)]


def test_batch_features_match_the_oracle_per_matrix():
    """Features of a batch: every matrix with its own means and sizes, and matrix b's sketch drawn from its own
    probe streams (2b for s, 2b + 1 for w)."""
    mats = _batch3()
    b = S.sme_batch_create(mats)
    try:
        _, ro, co = S.sme_batch_get_info(b)
        Fr = torch.zeros((int(ro[-1]), 8), dtype=torch.float32, device="cuda")
        Fc = torch.zeros((int(co[-1]), 8), dtype=torch.float32, device="cuda")
        S.sme_batch_features(b, 4, Fr, Fc)
        Fr, Fc = Fr.cpu().double().numpy(), Fc.cpu().double().numpy()
    finally:
        S.sme_batch_destroy(b)
    for i, A in enumerate(mats):
        fr, fc = Fr[ro[i]:ro[i + 1]], Fc[co[i]:co[i + 1]]
        z_r = O.row_estimate(A, np.zeros(A.m), np.zeros(A.n), O.probe_signs(4, 1, 2 * i, A.n, 8))
        z_c = O.col_estimate(A, np.zeros(A.m), np.zeros(A.n), O.probe_signs(4, 1, 2 * i + 1, A.m, 8))
        f0 = lambda z: 0.5 * np.log(np.maximum(z, 1e-30))
        for F, z, side in ((fr, z_r, 0.0), (fc, z_c, 1.0)):
            nz = z > 0
            np.testing.assert_allclose(F[nz, 0], f0(z[nz]), atol=1e-4)
            assert np.all(F[:, 3] == side)
            np.testing.assert_allclose(F[:, 4], f0(z_r).mean(), atol=1e-4)
            np.testing.assert_allclose(F[:, 5], f0(z_c).mean(), atol=1e-4)
            np.testing.assert_allclose(F[:, 6], np.log(A.m), rtol=1e-6)
            np.testing.assert_allclose(F[:, 7], np.log(A.n), rtol=1e-6)
        nnz_r = np.diff(A.row_ptr)
        np.testing.assert_allclose(fr[:, 1], np.log1p(nnz_r), atol=1e-6)


def test_batch_warm_start_is_the_network_on_the_batch_features():
    mats = _batch3()
    b = S.sme_batch_create(mats)
    mlp = _net(17, np.random.default_rng(17))
    try:
        _, ro, co = S.sme_batch_get_info(b)
        M, N = int(ro[-1]), int(co[-1])
        F = torch.zeros((M + N, 8), dtype=torch.float32, device="cuda")
        S.sme_batch_features(b, 6, F[:M], F[M:])
        y = torch.zeros(M + N, dtype=torch.float32, device="cuda")
        S.sme_mlp_forward(mlp, F, y)
        u0 = torch.zeros(M, dtype=torch.float32, device="cuda")
        v0 = torch.zeros(N, dtype=torch.float32, device="cuda")
        S.sme_batch_warm_start(b, mlp, 6, u0, v0)
        assert torch.equal(torch.cat([u0, v0]), y)
    finally:
        S.sme_mlp_destroy(mlp)
        S.sme_batch_destroy(b)


def test_batch_evaluate_matches_single_operators():
    mats = _batch3()
    b = S.sme_batch_create(mats)
    rng = np.random.default_rng(3)
    try:
        _, ro, co = S.sme_batch_get_info(b)
        u = rng.normal(0, 0.5, int(ro[-1])).astype(np.float32)
        v = rng.normal(0, 0.5, int(co[-1])).astype(np.float32)
        got = S.sme_batch_evaluate(b, torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), gamma=0.01)
    finally:
        S.sme_batch_destroy(b)
    for i, A in enumerate(mats):
        op = S.sme_op_create_csr(A.m, A.n, A.row_ptr, A.col_idx, A.vals.astype(np.float32))
        try:
            ref = S.sme_evaluate(op, torch.from_numpy(u[ro[i]:ro[i + 1]]).cuda(),
                                 torch.from_numpy(v[co[i]:co[i + 1]]).cuda(), gamma=0.01)
        finally:
            S.sme_op_destroy(op)
        for key in ("row_spread", "col_spread", "rms", "objective"):
            assert got[i][key] == pytest.approx(ref[key], rel=1e-10), (i, key)
        assert got[i]["empty_rows"] == ref["empty_rows"] and got[i]["empty_cols"] == ref["empty_cols"]
        # The objective of eq. (3) against the oracle's definition (FP64 on both sides).
        d = O.default_params(A.m, A.n)
        f = O.objective(A, u[ro[i]:ro[i + 1]].astype(np.float64), v[co[i]:co[i + 1]].astype(np.float64),
                        alpha=d["alpha"], beta=d["beta"], gamma=0.01)
        assert got[i]["objective"] == pytest.approx(f, rel=1e-9)


def test_fit_normalisation_matches_numpy():
    """Per-feature mean and deviation (N - 1) of the training features, summed on the device in FP64; a constant
    feature keeps scale 1."""
    rng = np.random.default_rng(12)
    N = 100003
    X = rng.normal(0, 1, (N, OM.IN)) * np.exp(rng.normal(0, 2, OM.IN)) + rng.normal(0, 5, OM.IN)
    X[:, 3] = 2.5  # constant
    X = X.astype(np.float32)
    mlp = S.sme_mlp_create(1)
    try:
        S.sme_mlp_fit_normalisation(mlp, torch.tensor(X, device="cuda"))
        nrm = S.sme_mlp_get_params(mlp)[1]
    finally:
        S.sme_mlp_destroy(mlp)
    X64 = X.astype(np.float64)
    mean, std = X64.mean(0), X64.std(0, ddof=1)
    std[3] = 1.0
    np.testing.assert_allclose(nrm[:OM.IN], mean.astype(np.float32), rtol=1e-6, atol=1e-6 * np.abs(mean).max())
    np.testing.assert_allclose(nrm[OM.IN:], std.astype(np.float32), rtol=1e-6)


def test_draw_batch_rows_follow_the_documented_generator():
    """Minibatch rows drawn by the library are the rows the documented Philox counter layout names
    (row floor(r N / 2^32), r = first word at counter (b, b >> 32, step, 0x6D6C7000)), copied exactly."""
    rng = np.random.default_rng(13)
    N, batch, seed = 77777, 5000, 0x1234_5678_9ABC
    X = rng.normal(0, 1, (N, OM.IN)).astype(np.float32)
    y = rng.normal(0, 1, N).astype(np.float32)
    Xd, yd = torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda")
    Xb = torch.zeros((batch, OM.IN), device="cuda")
    yb = torch.zeros(batch, device="cuda")
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for step in (0, 7):
        S.sme_mlp_draw_batch(Xd, yd, batch, seed, step, Xb, yb)
        got_X, got_y = Xb.cpu().numpy(), yb.cpu().numpy()
        for b in (0, 1, 2, 999, 4999):
            r = int(O.philox4x32_10([b, 0, step, 0x6D6C7000], key)[0])
            i = (r * N) >> 32
            np.testing.assert_array_equal(got_X[b], X[i])
            assert got_y[b] == y[i]
        # draws with replacement: about batch^2 / (2 N) = 160 repeats are expected among 5000
        assert np.unique(got_y).size > 0.9 * batch
