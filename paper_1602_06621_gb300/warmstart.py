"""Learned warm start for Algorithm 1 (driver around the library's MLP kernels).

Training data are matrices of the batched family; each is labelled with the scalings the method itself
converges to (a long run of sme_equilibrate), and every row and column becomes one sample: its features
(sme_op_features) and its converged log-scaling.  The network is trained on the device with
sme_mlp_train_step (mean squared error, Adam).

Use: u0, v0 = prediction (sme_warm_start), then sme_equilibrate from (u0, v0) with a step offset t0 > 0 (the
paper's first step, eta_1 = 1/gamma, would otherwise discard the warm start) and with the running averages
starting at (u0, v0) (so the average's t = 0 term is the warm start, as in the printed weights).  Zero
initialisation with t0 = 0 stays the reference method.
"""
from __future__ import annotations

import numpy as np

from . import sme

FEATURES = 8
# Step offset used after a warm start at the default gamma = 0.1: the first step is then
# 2 / (gamma (WARM_T0 + 2)) instead of 1/gamma.
WARM_T0 = 50
# Offset for the small-gamma runs that aim at near-exact equilibration (gamma = 1e-3): there the first
# steps of the plain schedule (1/gamma = 1000) throw any start far out of the box; eta_1 = 2/(gamma 1e4)
# = 0.2 keeps the warm start.
SPREAD_GAMMA = 1e-3
SPREAD_T0 = 10000


def label_matrix(A, *, T=400, k=32, seed=1, gamma=0.0):
    """Features and converged (u, v) of one CSR matrix: X (m+n, 8) float32, y (m+n) float32, on the GPU."""
    import torch
    op = sme.sme_op_create_csr(A.m, A.n, A.row_ptr, A.col_idx, A.vals.astype(np.float32))
    try:
        f32 = dict(dtype=torch.float32, device="cuda")
        u, v = torch.zeros(A.m, **f32), torch.zeros(A.n, **f32)
        ub, vb = torch.zeros(A.m, **f32), torch.zeros(A.n, **f32)
        sme.sme_equilibrate(op, u, v, ub, vb, T=T, k=k, seed=seed, gamma=gamma)
        X = torch.zeros((A.m + A.n, FEATURES), **f32)
        sme.sme_op_features(op, seed + 1, X[:A.m], X[A.m:])
        y = torch.cat([ub, vb])
    finally:
        sme.sme_op_destroy(op)
    return X, y


def batch_training_set(b, *, T=400, k=32, seed=1, gamma=0.0):
    """Features and converged (ubar, vbar) of every row and column of a batch (one batched run)."""
    import torch
    _, ro, co = sme.sme_batch_get_info(b)
    M, N = int(ro[-1]), int(co[-1])
    f32 = dict(dtype=torch.float32, device="cuda")
    z = [torch.zeros(x, **f32) for x in (M, N, M, N)]
    sme.sme_batch_equilibrate(b, *z, T=T, k=k, seed=seed, gamma=gamma)
    X = torch.zeros((M + N, FEATURES), **f32)
    sme.sme_batch_features(b, seed + 1, X[:M], X[M:])
    return X, torch.cat([z[2], z[3]])


def training_set(mats, **kw):
    import torch
    Xs, ys = zip(*(label_matrix(A, **kw) for A in mats))
    return torch.cat(Xs), torch.cat(ys)


def train(mlp, X, y, *, steps=600, batch=8192, lr=2e-3, seed=0):
    """Fit the input normalisation to X, then `steps` minibatch Adam steps (minibatches drawn by the library,
    with replacement); returns the loss history."""
    import torch
    X, y = X.contiguous(), y.contiguous()
    sme.sme_mlp_fit_normalisation(mlp, X)
    N = X.shape[0]
    nb = min(batch, N)
    Xb = torch.empty((nb, FEATURES), dtype=torch.float32, device=X.device)
    yb = torch.empty(nb, dtype=torch.float32, device=X.device)
    hist = []
    for step in range(steps):
        sme.sme_mlp_draw_batch(X, y, nb, seed, step, Xb, yb)
        want = step % 50 == 0 or step == steps - 1
        loss = sme.sme_mlp_train_step(mlp, Xb, yb, lr * (0.5 ** (step / max(1, steps // 3))), want_loss=want)
        if want:
            hist.append((step, loss))
    return hist


def run(A, *, T, k, seed, mlp=None, t0=0, gamma=0.0):
    """Algorithm 1 on one matrix for T iterations, from zero (mlp None) or from the network's prediction."""
    import torch
    op = sme.sme_op_create_csr(A.m, A.n, A.row_ptr, A.col_idx, A.vals.astype(np.float32))
    try:
        f32 = dict(dtype=torch.float32, device="cuda")
        u, v = torch.zeros(A.m, **f32), torch.zeros(A.n, **f32)
        if mlp is not None:
            sme.sme_warm_start(op, mlp, seed + 1, u, v)
        ub, vb = u.clone(), v.clone()
        sme.sme_equilibrate(op, u, v, ub, vb, T=T, k=k, seed=seed, t0=t0, gamma=gamma)
        quality = sme.sme_evaluate(op, ub, vb, gamma=gamma)
        return ub.cpu().double().numpy(), vb.cpu().double().numpy(), quality
    finally:
        sme.sme_op_destroy(op)
