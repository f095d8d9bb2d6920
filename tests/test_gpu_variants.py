"""GPU parity of the Section 6 variants (varying norms, symmetric, block) against the oracle, step by step
from the GPU's own state (FP64 operators: <= 1e-11 norm-wise per step)."""
import numpy as np
import pytest

import oracle as O
from paper_1602_06621_gb300 import inputs as I
from paper_1602_06621_gb300 import sme

from gpu_util import gpu_equilibrate, make_op, rel_norm

pytestmark = pytest.mark.gpu


def _t(x, dtype=None):
    import torch
    return torch.tensor(np.asarray(x), dtype=dtype or torch.float64, device="cuda")


def _np(*xs):
    return [x.cpu().double().numpy() for x in xs]


def test_varying_norms_every_step_and_uniform_case():
    A = I.sparse_uniform_density(300, 200, 0.04, seed=11)
    rng = np.random.default_rng(0)
    rt = np.exp(rng.normal(0, 0.4, A.m))
    ct = np.exp(rng.normal(0, 0.4, A.n))
    ct *= rt.sum() / ct.sum()
    d = O.default_params(A.m, A.n)
    op, dt = make_op(A)
    try:
        state = [np.zeros(A.m), np.zeros(A.n), np.zeros(A.m), np.zeros(A.n)]
        worst = 0.0
        for t in range(1, 16):
            g = [_t(x) for x in state]
            sme.sme_equilibrate_targets(op, _t(rt), _t(ct), *g, T=1, k=4, seed=3, t_begin=t)
            got = _np(*g)
            ref = O.psgd_step_targets(A, *state, O.probe_signs(3, t, 0, A.n, 4), O.probe_signs(3, t, 1, A.m, 4), t,
                                      rt=rt, ct=ct, gamma=d["gamma"], M=d["M"])
            worst = max(worst, rel_norm(got, ref))
            state = got
        assert worst <= 1e-11, worst
        # Uniform targets alpha^2, beta^2 give exactly the plain method.
        g = [_t(np.zeros(x)) for x in (A.m, A.n, A.m, A.n)]
        sme.sme_equilibrate_targets(op, _t(np.full(A.m, d["alpha"] ** 2)), _t(np.full(A.n, d["beta"] ** 2)), *g,
                                    T=10, k=4, seed=3)
        plain = gpu_equilibrate(op, dt, A.m, A.n, T=10, k=4, seed=3)
        for x, y in zip(_np(*g), plain):
            np.testing.assert_allclose(x, y, rtol=0, atol=1e-14 * max(1.0, np.abs(y).max()))
    finally:
        sme.sme_op_destroy(op)


@pytest.mark.parametrize("k", [4, 32])
def test_symmetric_every_step(k):
    B = I.sparse_uniform_density(250, 250, 0.02, seed=12).to_dense()
    S = B + B.T
    A = O.OracleCSR.from_any(S)
    from paper_1602_06621_gb300.inputs import CSR
    Ac = CSR(A.m, A.n, A.row_ptr.astype(np.int32), A.col_idx, A.vals)
    op, dt = make_op(Ac, sme.SME_F64)
    try:
        u, ub = np.zeros(A.n), np.zeros(A.n)
        worst = 0.0
        for t in range(1, 21):
            g = [_t(u), _t(ub)]
            sme.sme_equilibrate_symmetric(op, *g, T=1, k=k, seed=5, t_begin=t)
            got = _np(*g)
            ref = O.psgd_step_symmetric(A, u, ub, O.probe_signs(5, t, 0, A.n, k), t, alpha=1.0, gamma=0.1,
                                        M=np.log(1e4))
            worst = max(worst, rel_norm(got, ref))
            u, ub = got
        assert worst <= 1e-11, worst
        g = [_t(np.zeros(A.n)), _t(np.zeros(A.n))]
        sme.sme_equilibrate_symmetric(op, *g, T=20, k=k, seed=5)
        for x, y in zip(_np(*g), (u, ub)):
            np.testing.assert_array_equal(x, y)
    finally:
        sme.sme_op_destroy(op)


def test_block_every_step():
    A = I.sparse_uniform_density(240, 160, 0.05, seed=13)
    rb = np.array([0, 30, 31, 100, 180, 240])
    cb = np.array([0, 40, 41, 160])
    d = O.default_params(A.m, A.n)
    op, dt = make_op(A)
    try:
        state = [np.zeros(5), np.zeros(3), np.zeros(5), np.zeros(3)]
        worst = 0.0
        for t in range(1, 16):
            g = [_t(x) for x in state]
            sme.sme_equilibrate_block(op, rb, cb, *g, T=1, k=8, seed=7, t_begin=t)
            got = _np(*g)
            ref = O.block_step(A, rb, cb, *state, O.probe_signs(7, t, 0, A.n, 8), O.probe_signs(7, t, 1, A.m, 8), t,
                               **d)
            worst = max(worst, rel_norm(got, ref))
            state = got
        assert worst <= 1e-11, worst
    finally:
        sme.sme_op_destroy(op)


def test_variant_argument_errors():
    A = I.sparse_uniform_density(40, 30, 0.1, seed=14)
    op, dt = make_op(A)
    try:
        z = _t(np.zeros(40))
        with pytest.raises(sme.SmeError):
            sme.sme_equilibrate_symmetric(op, z, z, T=1, k=4)  # not square
        with pytest.raises(sme.SmeError):
            sme.sme_equilibrate_block(op, [0, 20, 10, 40], [0, 30], z, z, z, z, T=1, k=4)  # decreasing offsets
    finally:
        sme.sme_op_destroy(op)
