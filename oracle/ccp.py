"""FP64 reference for the Chambolle-Cremers-Pock application (Section 5.2), TEST INFRASTRUCTURE ONLY.

The Lasso problem of Section 5.2,
    minimize  f(x) = ||A x - b||^2 / sqrt(lam) + sqrt(lam) ||x||_1,
is solved by the primal-dual method of Chambolle and Pock on the equilibrated operator K = D A E: with
x = E xs, the problem is  min_xs  F(K xs) + G(xs)  with F(y) = ||D^{-1} y - b||^2 / sqrt(lam) and
G(xs) = sqrt(lam) ||E xs||_1.  One iteration, from y = xs = xbar = 0 (the paper's "all initial iterates 0"):
    y    <- prox_{sigma F*}(y + sigma K xbar)
    xs'  <- prox_{tau G}(xs - tau K^T y)
    xbar <- xs' + theta (xs' - xs),   xs <- xs'
The two proximal maps are closed forms (derived in the comments below).  The step sizes of Section 5.2 are
tau = sigma = 0.9 / ||K||_2, with ||K||_2 from power iteration on K^T K started at the unit vector
1/sqrt(n) (deterministic, so the library and this file start from the same vector).
"""
import numpy as np
import scipy.sparse as sps


def _matrix(A):
    if isinstance(A, np.ndarray):
        return sps.csr_matrix(A.astype(np.float64))
    return sps.csr_matrix((np.asarray(A.vals, np.float64), A.col_idx, A.row_ptr), shape=(A.m, A.n))


def lasso_objective(A, x, b, lam):
    """f(x) of Section 5.2."""
    S = _matrix(A)
    r = S @ np.asarray(x, np.float64) - b
    return float(r @ r / np.sqrt(lam) + np.sqrt(lam) * np.abs(x).sum())


def default_lambda(A, b):
    """lam = 1e-3 ||A^T b||_inf (Section 5.2)."""
    return 1e-3 * float(np.abs(_matrix(A).T @ np.asarray(b, np.float64)).max())


def scaled_operator(A, u=None, v=None):
    S = _matrix(A)
    d = np.exp(np.asarray(u, np.float64)) if u is not None else np.ones(S.shape[0])
    e = np.exp(np.asarray(v, np.float64)) if v is not None else np.ones(S.shape[1])
    return sps.diags(d) @ S @ sps.diags(e), d, e


def power_norm(K, iters):
    """||K||_2 by `iters` steps of power iteration on K^T K from 1/sqrt(n): returns sqrt(||K^T K x||) for the
    last unit iterate x."""
    n = K.shape[1]
    x = np.full(n, 1.0 / np.sqrt(n))
    lam = 0.0
    for _ in range(iters):
        y = K.T @ (K @ x)
        lam = np.linalg.norm(y)
        if lam == 0.0:
            return 0.0
        x = y / lam
    return float(np.sqrt(lam))


def prox_g(z, thresh):
    """prox of t*sqrt(lam)*|e_j xs_j|: soft threshold at thresh_j = tau sqrt(lam) e_j."""
    return np.sign(z) * np.maximum(np.abs(z) - thresh, 0.0)


def prox_f_conj(w, d, b, sigma, lam):
    """prox_{sigma F*}(w) for F(y) = sum_i (y_i/d_i - b_i)^2 / sqrt(lam).

    Moreau: prox_{sigma F*}(w) = w - sigma prox_{F/sigma}(w/sigma).  prox_{F/sigma}(p) minimises
    (y/d - b)^2/sqrt(lam) + (sigma/2)(y - p)^2 elementwise; setting the derivative to zero gives
    y = (a d b + sigma p)/(a + sigma) with a = 2/(d^2 sqrt(lam)).  Substituting p = w/sigma:
    prox_{sigma F*}(w) = a (w - sigma d b) / (a + sigma)."""
    a = 2.0 / (d * d * np.sqrt(lam))
    return a * (w - sigma * d * b) / (a + sigma)


def ccp_lasso(A, b, lam, *, iters, u=None, v=None, tau=None, sigma=None, theta=1.0, norm_iters=100,
              check_every=0):
    """Run `iters` iterations; returns (x in the original variables, history of f(x) every check_every
    iterations (with f(0) first), ||K||_2 estimate)."""
    K, d, e = scaled_operator(A, u, v)
    b = np.asarray(b, np.float64)
    nrm = power_norm(K, norm_iters)
    tau = 0.9 / nrm if tau is None else tau
    sigma = 0.9 / nrm if sigma is None else sigma
    m, n = K.shape
    y = np.zeros(m)
    xs = np.zeros(n)
    xbar = np.zeros(n)
    hist = [lasso_objective(A, np.zeros(n), b, lam)] if check_every else []
    for it in range(1, iters + 1):
        y = prox_f_conj(y + sigma * (K @ xbar), d, b, sigma, lam)
        xn = prox_g(xs - tau * (K.T @ y), tau * np.sqrt(lam) * e)
        xbar = xn + theta * (xn - xs)
        xs = xn
        if check_every and it % check_every == 0:
            hist.append(lasso_objective(A, e * xs, b, lam))
    return e * xs, hist, nrm


def lasso_kkt_residual(A, x, b, lam):
    """Largest violation of the optimality conditions 0 in 2 A^T (A x - b)/sqrt(lam) + sqrt(lam) d||x||_1,
    relative to sqrt(lam): g_j + sqrt(lam) sign(x_j) = 0 where x_j != 0, |g_j| <= sqrt(lam) where x_j = 0."""
    S = _matrix(A)
    g = 2.0 * (S.T @ (S @ x - b)) / np.sqrt(lam)
    s = np.sqrt(lam)
    nz = x != 0
    viol = np.zeros_like(g)
    viol[nz] = np.abs(g[nz] + s * np.sign(x[nz]))
    viol[~nz] = np.maximum(np.abs(g[~nz]) - s, 0.0)
    return float(viol.max() / s)
