"""The paper's Section 4 experiment at its full size, run by the library on the GPU.

A is 2e4 x 1e4 with 1% of its entries nonzero at uniform-random positions, N(0,1) values, and row and
column factors e^{N(1,1)} (Section 4's recipe); Algorithm 1 runs with one probe pair per iteration and
the paper's parameters.  The optimality gap f(ubar, vbar) - p* (p* from the oracle's Newton solver, run on
the host) is read at log-spaced iterations; the paper reports a least-squares slope of -2.0 for log gap
against log t, against the 1/t of the theory, and an RMS error that falls quickly and then slowly.
"""
import numpy as np
import pytest

import oracle as O
from paper_1602_06621_gb300 import inputs as I
from paper_1602_06621_gb300 import sme

from gpu_util import make_op

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_section4_optimality_gap_and_rms_trend():
    import torch
    A = I.sparse_uniform_density(20000, 10000, 0.01, seed=1, mean=1.0, var=1.0)
    d = O.default_params(A.m, A.n)
    us, vs = O.regularized_optimum(A, **d)
    pstar = O.objective(A, us, vs, alpha=d["alpha"], beta=d["beta"], gamma=d["gamma"])
    op, dt = make_op(A, sme.SME_F64)
    checkpoints = [1, 2, 3, 5, 10, 20, 30, 50, 100, 200, 300, 500, 1000]
    gaps, rms = [], []
    try:
        z = [torch.zeros(x, dtype=torch.float64, device="cuda") for x in (A.m, A.n, A.m, A.n)]
        f0 = sme.sme_evaluate(op, z[0], z[1])["objective"]
        t = 0
        for c in checkpoints:
            sme.sme_equilibrate(op, *z, T=c - t, k=1, seed=0, t_begin=t + 1)
            t = c
            q = sme.sme_evaluate(op, z[2], z[3])
            gaps.append((q["objective"] - pstar) / f0)
            rms.append(q["rms"])
    finally:
        sme.sme_op_destroy(op)
    gaps, rms = np.array(gaps), np.array(rms)
    assert np.all(gaps > 0)
    # Convergence well beyond the 1/t bound over the smooth part: the paper fits -2.0.  Here the gap stays
    # near 3e-5 from t = 3 to t = 20 after the fast first iterations, then falls as about t^-1.8 (t >= 50).
    sel = np.array(checkpoints) >= 50
    slope = np.polyfit(np.log(np.array(checkpoints)[sel]), np.log(gaps[sel]), 1)[0]
    assert slope < -1.5, (slope, gaps)
    # Fast early decrease (gap and RMS), then a smooth decrease.
    assert gaps[-1] < 1e-3 * gaps[0] and rms[-1] < 0.5 * rms[0]
    assert np.all(np.diff(gaps[sel]) < 0)
