"""FP64 oracle: ctypes front end to sme_oracle.c plus plain NumPy reference tools.

TEST INFRASTRUCTURE ONLY (tests, smoke check, bench CPU baseline).

Paper passages followed (Diamond & Boyd, "Stochastic Matrix-Free Equilibration"):
  * objective of the regularised, box-constrained problem: eq. (3), Section 2.3
  * gradient |DAE|^2 1 - alpha^2 + gamma u (and the v analogue): Section 3.1
  * Algorithm 1 (projected stochastic gradient): Section 3.2, in sme_oracle.c
  * RMS equilibration error: Section 4
  * Phi(U) and the condition-number bound: Section 2.2, Theorems 2.1 and 2.2
  * Sinkhorn-Knopp as alternating minimisation of eq. (1): Section 2.1
  * block minimisation of eq. (3) through the Lambert W function: Section 2.3
    (the printed formula drops an exponential; the form used here is derived
    from setting the partial derivative to zero, see block_minimize_u)
  * LSQR with diagonal preconditioning, solve (DAE) xbar = D b, x = E xbar,
    accuracy measured on the original system: Section 5.1.  LSQR itself is
    Paige & Saunders (1982), the bidiagonalisation with plane rotations.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field

import numpy as np

from .build import build_oracle, build_oracle_omp

__all__ = [
    "lib", "philox4x32_10", "probe_signs", "row_estimate", "col_estimate", "psgd_step", "equilibrate",
    "psgd_step_sampled", "exact_norms_sq", "csr_matvec", "dense_estimate_sampled", "psgd_step_targets",
    "psgd_step_symmetric", "block_step", "default_params", "objective", "gradient",
    "rms_error", "spread", "log_phi", "kappa", "sinkhorn_knopp", "block_minimize_u", "block_minimize_v",
    "regularized_optimum", "lsqr", "LsqrResult", "OracleCSR", "set_parallel", "threads",
]

_LIBS = {}
_PARALLEL = False
_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i64, _i32, _u64, _u32, _d = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double


def set_parallel(enabled: bool) -> int:
    """Route later calls to the OpenMP build of the oracle (True: all host cores, or OMP_NUM_THREADS) or to the
    single-threaded checker build (False, the default).  Both give the same bits.  Returns the thread count."""
    global _PARALLEL
    _PARALLEL = bool(enabled)
    return threads()


def threads() -> int:
    """Threads the active build runs its parallel loops on (1 for the checker build)."""
    return int(lib().or_max_threads())


def lib():
    key = "omp" if _PARALLEL else "plain"
    if key not in _LIBS:
        L = ctypes.CDLL(build_oracle_omp() if _PARALLEL else build_oracle())
        L.or_max_threads.restype = ctypes.c_int
        L.or_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.or_probe_sign.argtypes = [_u64, _u32, _u32, _u32, _u32]
        L.or_probe_sign.restype = _d
        L.or_draw_probes.argtypes = [_u64, _i32, _i32, _i64, _i32, _dp]
        est = [_i64, _i64, _i64p, _i32p, _dp, _dp, _dp, _dp, _i32, _dp]
        L.or_row_estimate.argtypes = est
        L.or_col_estimate.argtypes = est
        L.or_psgd_step.argtypes = [_i64, _i64, _i64p, _i32p, _dp, _d, _d, _d, _d, _i32, _i32, _dp, _dp, _i32,
                                   _dp, _dp, _dp, _dp]
        L.or_psgd_step_targets.argtypes = [_i64, _i64, _i64p, _i32p, _dp, _dp, _dp, _d, _d, _d, _d, _i32, _i32, _dp,
                                           _dp, _i32, _dp, _dp, _dp, _dp]
        L.or_psgd_step_symmetric.argtypes = [_i64, _i64p, _i32p, _dp, _d, _d, _d, _i32, _i32, _dp, _i32, _dp, _dp]
        L.or_block_step.argtypes = [_i64, _i64, _i64p, _i32p, _dp, _i64, _i64p, _i64, _i64p, _d, _d, _d, _d, _i32,
                                    _i32, _dp, _dp, _i32, _dp, _dp, _dp, _dp]
        L.or_equilibrate.argtypes = [_i64, _i64, _i64p, _i32p, _dp, _d, _d, _d, _d, _i32, _i32, _i32, _i32, _u64,
                                     _i32, _dp, _dp, _dp, _dp]
        L.or_psgd_step_sampled.argtypes = [_i64, _i64, _i64p, _i32p, _dp, _d, _d, _d, _d, _i32, _i32, _i32, _u64,
                                           _i32, _dp, _dp, _dp, _dp, _i64, _i64p, _i64, _i64p, _dp, _dp, _dp, _dp]
        L.or_exact_norms_sq.argtypes = [_i64, _i64, _i64p, _i32p, _dp, _dp, _dp, _dp, _dp]
        L.or_csr_matvec.argtypes = [_i64, _i64p, _i32p, _dp, _dp, _dp]
        L.or_dense_estimate_sampled.argtypes = [_i64, _i64, ctypes.POINTER(ctypes.c_float), _dp, _dp, _dp, _i32, _i32,
                                                _u64, _i32, _i64, _i64p, _i64, _i64p, _dp, _dp]
        _LIBS[key] = L
    return _LIBS[key]


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class OracleCSR:
    """The oracle's own copy of a CSR matrix: int64 row pointers, int32 columns, FP64 values."""

    m: int
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    vals: np.ndarray

    @staticmethod
    def from_any(A) -> "OracleCSR":
        if isinstance(A, np.ndarray):
            m, n = A.shape
            rows, cols = np.nonzero(A)
            counts = np.bincount(rows, minlength=m)
            rp = np.zeros(m + 1, np.int64)
            np.cumsum(counts, out=rp[1:])
            return OracleCSR(m, n, rp, cols.astype(np.int32), _f64(A[rows, cols]))
        return OracleCSR(int(A.m), int(A.n), np.ascontiguousarray(A.row_ptr, dtype=np.int64),
                         np.ascontiguousarray(A.col_idx, dtype=np.int32), _f64(A.vals))

    @property
    def nnz(self):
        return int(self.row_ptr[-1])

    def rows(self):
        return np.repeat(np.arange(self.m), np.diff(self.row_ptr))

    def dense(self):
        out = np.zeros((self.m, self.n))
        out[self.rows(), self.col_idx] = self.vals
        return out


def _csr(A) -> OracleCSR:
    return A if isinstance(A, OracleCSR) else OracleCSR.from_any(A)


# ------------------------------------------------------------------ Philox / probes

def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(c, _u32p), _p(k, _u32p), _p(out, _u32p))
    return out


def probe_signs(seed: int, t: int, stream: int, length: int, k: int) -> np.ndarray:
    """Signs s[idx, p] in {-1, +1} for idx < length, p < k (the probe contract in sme_oracle.c)."""
    out = np.zeros((length, k))
    lib().or_draw_probes(seed, t, stream, length, k, _p(out, _dp))
    return out


# ------------------------------------------------------------------ estimators / steps

def row_estimate(A, u, v, s) -> np.ndarray:
    A = _csr(A)
    s = _f64(s).reshape(A.n, -1)
    k = s.shape[1]
    z = np.zeros(A.m)
    lib().or_row_estimate(A.m, A.n, _p(A.row_ptr, _i64p), _p(A.col_idx, _i32p), _p(A.vals, _dp),
                          _p(_f64(u), _dp), _p(_f64(v), _dp), _p(s, _dp), k, _p(z, _dp))
    return z


def col_estimate(A, u, v, w) -> np.ndarray:
    A = _csr(A)
    w = _f64(w).reshape(A.m, -1)
    k = w.shape[1]
    z = np.zeros(A.n)
    lib().or_col_estimate(A.m, A.n, _p(A.row_ptr, _i64p), _p(A.col_idx, _i32p), _p(A.vals, _dp),
                          _p(_f64(u), _dp), _p(_f64(v), _dp), _p(w, _dp), k, _p(z, _dp))
    return z


def default_params(m: int, n: int) -> dict:
    """Section 4 parameters: alpha=(n/m)^(1/4), beta=(m/n)^(1/4), gamma=1e-1, M=log(1e4)."""
    return dict(alpha=(n / m) ** 0.25, beta=(m / n) ** 0.25, gamma=0.1, M=math.log(1e4))


def psgd_step(A, u, v, ubar, vbar, s, w, t, *, alpha, beta, gamma, M, t0=0):
    """One iteration t of Algorithm 1 with explicit signs; returns new (u, v, ubar, vbar)."""
    A = _csr(A)
    s = _f64(s).reshape(A.n, -1)
    w = _f64(w).reshape(A.m, -1)
    k = s.shape[1]
    u, v, ubar, vbar = (_f64(x).copy() for x in (u, v, ubar, vbar))
    lib().or_psgd_step(A.m, A.n, _p(A.row_ptr, _i64p), _p(A.col_idx, _i32p), _p(A.vals, _dp),
                       alpha, beta, gamma, M, t, t0, _p(s, _dp), _p(w, _dp), k,
                       _p(u, _dp), _p(v, _dp), _p(ubar, _dp), _p(vbar, _dp))
    return u, v, ubar, vbar


def psgd_step_targets(A, u, v, ubar, vbar, s, w, t, *, rt, ct, gamma, M, t0=0):
    """One iteration t with squared target norms rt (rows) and ct (columns) (Section 6, varying norms)."""
    A = _csr(A)
    s = _f64(s).reshape(A.n, -1)
    w = _f64(w).reshape(A.m, -1)
    k = s.shape[1]
    u, v, ubar, vbar = (_f64(x).copy() for x in (u, v, ubar, vbar))
    rt, ct = _f64(rt), _f64(ct)
    lib().or_psgd_step_targets(A.m, A.n, _p(A.row_ptr, _i64p), _p(A.col_idx, _i32p), _p(A.vals, _dp), _p(rt, _dp),
                               _p(ct, _dp), 0.0, 0.0, gamma, M, t, t0, _p(s, _dp), _p(w, _dp), k,
                               _p(u, _dp), _p(v, _dp), _p(ubar, _dp), _p(vbar, _dp))
    return u, v, ubar, vbar


def psgd_step_symmetric(A, u, ubar, s, t, *, alpha, gamma, M, t0=0):
    """One iteration t of Algorithm 2 (D = E) with explicit signs s (n x k)."""
    A = _csr(A)
    s = _f64(s).reshape(A.n, -1)
    k = s.shape[1]
    u, ubar = _f64(u).copy(), _f64(ubar).copy()
    lib().or_psgd_step_symmetric(A.n, _p(A.row_ptr, _i64p), _p(A.col_idx, _i32p), _p(A.vals, _dp), alpha, gamma, M,
                                 t, t0, _p(s, _dp), k, _p(u, _dp), _p(ubar, _dp))
    return u, ubar


def block_step(A, rb, cb, ub, vb, ubb, vbb, s, w, t, *, alpha, beta, gamma, M, t0=0):
    """One iteration t of block equilibration: row blocks rb (offsets, p+1), column blocks cb (q+1)."""
    A = _csr(A)
    s = _f64(s).reshape(A.n, -1)
    w = _f64(w).reshape(A.m, -1)
    k = s.shape[1]
    rb = np.ascontiguousarray(rb, dtype=np.int64)
    cb = np.ascontiguousarray(cb, dtype=np.int64)
    ub, vb, ubb, vbb = (_f64(x).copy() for x in (ub, vb, ubb, vbb))
    lib().or_block_step(A.m, A.n, _p(A.row_ptr, _i64p), _p(A.col_idx, _i32p), _p(A.vals, _dp), rb.size - 1,
                        _p(rb, _i64p), cb.size - 1, _p(cb, _i64p), alpha, beta, gamma, M, t, t0, _p(s, _dp),
                        _p(w, _dp), k, _p(ub, _dp), _p(vb, _dp), _p(ubb, _dp), _p(vbb, _dp))
    return ub, vb, ubb, vbb


def equilibrate(A, *, T: int, k: int, seed: int = 0, alpha=None, beta=None, gamma=None, M=None,
                t_begin: int = 1, t0: int = 0, stream_base: int = 0, state=None):
    """Algorithm 1 for iterations t_begin..t_begin+T-1 with Philox probes.

    state = (u, v, ubar, vbar) to resume; zeros (the paper's start) when None.
    Returns (u, v, ubar, vbar) after the last iteration.
    """
    A = _csr(A)
    d = default_params(A.m, A.n)
    alpha = d["alpha"] if alpha is None else alpha
    beta = d["beta"] if beta is None else beta
    gamma = d["gamma"] if gamma is None else gamma
    M = d["M"] if M is None else M
    if state is None:
        u, v, ubar, vbar = np.zeros(A.m), np.zeros(A.n), np.zeros(A.m), np.zeros(A.n)
    else:
        u, v, ubar, vbar = (_f64(x).copy() for x in state)
    lib().or_equilibrate(A.m, A.n, _p(A.row_ptr, _i64p), _p(A.col_idx, _i32p), _p(A.vals, _dp),
                         alpha, beta, gamma, M, t_begin, T, t0, k, seed, stream_base,
                         _p(u, _dp), _p(v, _dp), _p(ubar, _dp), _p(vbar, _dp))
    return u, v, ubar, vbar


def psgd_step_sampled(A, u, v, ubar, vbar, rows, cols, t, *, k, seed, alpha, beta, gamma, M, t0=0,
                      stream_base=0):
    """Iteration t of Algorithm 1 evaluated at the listed rows and columns only."""
    A = _csr(A)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    uo, ubo = np.zeros(rows.size), np.zeros(rows.size)
    vo, vbo = np.zeros(cols.size), np.zeros(cols.size)
    lib().or_psgd_step_sampled(A.m, A.n, _p(A.row_ptr, _i64p), _p(A.col_idx, _i32p), _p(A.vals, _dp),
                               alpha, beta, gamma, M, t, t0, k, seed, stream_base,
                               _p(_f64(u), _dp), _p(_f64(v), _dp), _p(_f64(ubar), _dp), _p(_f64(vbar), _dp),
                               rows.size, _p(rows, _i64p), cols.size, _p(cols, _i64p),
                               _p(uo, _dp), _p(ubo, _dp), _p(vo, _dp), _p(vbo, _dp))
    return uo, ubo, vo, vbo


def exact_norms_sq(A, u, v):
    """(|DAE|^2 1, |EA^TD|^2 1): exact squared row and column norms of DAE."""
    A = _csr(A)
    r2, c2 = np.zeros(A.m), np.zeros(A.n)
    lib().or_exact_norms_sq(A.m, A.n, _p(A.row_ptr, _i64p), _p(A.col_idx, _i32p), _p(A.vals, _dp),
                            _p(_f64(u), _dp), _p(_f64(v), _dp), _p(r2, _dp), _p(c2, _dp))
    return r2, c2


def dense_estimate_sampled(A, u, v, rows, cols, *, t, k, seed, stream_base=0, row_scale=None):
    """Estimates of iteration t for dense A at the listed rows and columns (FP64 accumulation)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    m, n = A.shape
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    zu, zv = np.zeros(rows.size), np.zeros(cols.size)
    rs = None if row_scale is None else _f64(row_scale)
    lib().or_dense_estimate_sampled(m, n, A.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                    None if rs is None else _p(rs, _dp), _p(_f64(u), _dp), _p(_f64(v), _dp), t, k, seed,
                                    stream_base, rows.size, _p(rows, _i64p), cols.size, _p(cols, _i64p),
                                    _p(zu, _dp), _p(zv, _dp))
    return zu, zv


def csr_matvec(A, x):
    A = _csr(A)
    y = np.zeros(A.m)
    lib().or_csr_matvec(A.m, _p(A.row_ptr, _i64p), _p(A.col_idx, _i32p), _p(A.vals, _dp), _p(_f64(x), _dp),
                        _p(y, _dp))
    return y


# ------------------------------------------------------------------ objective and metrics

def objective(A, u, v, *, alpha, beta, gamma):
    """f(u, v) of eq. (3) (without the box, which is a constraint, not a term)."""
    A = _csr(A)
    q = A.vals ** 2 * np.exp(2 * u[A.rows()] + 2 * v[A.col_idx])
    return 0.5 * q.sum() - alpha ** 2 * u.sum() - beta ** 2 * v.sum() + 0.5 * gamma * (u @ u + v @ v)


def gradient(A, u, v, *, alpha, beta, gamma):
    """(|DAE|^2 1 - alpha^2 + gamma u,  |EA^TD|^2 1 - beta^2 + gamma v), Section 3.1."""
    A = _csr(A)
    q = A.vals ** 2 * np.exp(2 * u[A.rows()] + 2 * v[A.col_idx])
    r = np.bincount(A.rows(), weights=q, minlength=A.m)
    c = np.bincount(A.col_idx, weights=q, minlength=A.n)
    return r - alpha ** 2 + gamma * u, c - beta ** 2 + gamma * v


def rms_error(r2, c2, alpha, beta):
    """RMS equilibration error of Section 4 from exact squared row/column norms."""
    m, n = len(r2), len(c2)
    tot = np.sum((np.sqrt(r2) - alpha) ** 2) + np.sum((np.sqrt(c2) - beta) ** 2)
    return math.sqrt(tot) / math.sqrt(m + n)


def spread(r2, c2):
    """(row spread, column spread): max/min of the l2 norms over nonempty rows / columns."""
    r = np.sqrt(r2[r2 > 0])
    c = np.sqrt(c2[c2 > 0])
    return float(r.max() / r.min()), float(c.max() / c.min())


def log_phi(U):
    """log Phi(U) = ||U||_F^2 / 2 - sum_i log sigma_i  (Section 2.2)."""
    s = np.linalg.svd(U, compute_uv=False)
    return 0.5 * float(np.sum(s ** 2)) - float(np.sum(np.log(s)))


def kappa(U):
    s = np.linalg.svd(U, compute_uv=False)
    return float(s[0] / s[-1])


# ------------------------------------------------------------------ exact solvers (need entries of A)

def sinkhorn_knopp(A, *, alpha=1.0, beta=1.0, iters=10000, tol=1e-13):
    """Alternating minimisation of eq. (1) (Section 2.1): returns (d, e) with D = diag(d), E = diag(e)."""
    A2 = np.asarray(A, dtype=np.float64) ** 2
    m, n = A2.shape
    d, e = np.ones(m), np.ones(n)
    for _ in range(iters):
        d = alpha / np.sqrt(A2 @ (e ** 2))
        e = beta / np.sqrt(A2.T @ (d ** 2))
        r = (d ** 2) * (A2 @ (e ** 2))
        if np.max(np.abs(r - alpha ** 2)) < tol * alpha ** 2:
            break
    return d, e


def _lambert_w_log(x):
    """w with w + log(w) = x (i.e. w = W(e^x)), elementwise, by Newton in log space."""
    x = np.asarray(x, dtype=np.float64)
    w = np.where(x > 1.0, x - np.log(np.maximum(x, 1.0)), np.exp(np.minimum(x, 1.0)) * 0.5 + 1e-300)
    for _ in range(100):
        f = w + np.log(w) - x
        w_new = w - f / (1.0 + 1.0 / w)
        w_new = np.where(w_new <= 0, w * 0.5, w_new)
        if np.max(np.abs(w_new - w) / np.maximum(w, 1e-300)) < 1e-15:
            w = w_new
            break
        w = w_new
    return w


def block_minimize_u(A, v, *, alpha, gamma, M):
    """Exact minimiser of eq. (3) over u with v fixed (Section 2.3).

    Setting d f / d u_i = a_i e^{2 u_i} - alpha^2 + gamma u_i = 0, a_i = sum_j A_ij^2 e^{2 v_j}, gives
    u_i = alpha^2/gamma - W(2 a_i e^{2 alpha^2/gamma} / gamma) / 2, then projection on [-M, M].
    An empty row (a_i = 0) gives u_i = alpha^2 / gamma before projection.
    """
    A = _csr(A)
    a = np.bincount(A.rows(), weights=A.vals ** 2 * np.exp(2 * v[A.col_idx]), minlength=A.m)
    u = np.full(A.m, alpha ** 2 / gamma)
    nz = a > 0
    x = np.log(2 * a[nz] / gamma) + 2 * alpha ** 2 / gamma
    u[nz] = alpha ** 2 / gamma - 0.5 * _lambert_w_log(x)
    return np.clip(u, -M, M)


def block_minimize_v(A, u, *, beta, gamma, M):
    A = _csr(A)
    a = np.bincount(A.col_idx, weights=A.vals ** 2 * np.exp(2 * u[A.rows()]), minlength=A.n)
    v = np.full(A.n, beta ** 2 / gamma)
    nz = a > 0
    x = np.log(2 * a[nz] / gamma) + 2 * beta ** 2 / gamma
    v[nz] = beta ** 2 / gamma - 0.5 * _lambert_w_log(x)
    return np.clip(v, -M, M)


def regularized_optimum(A, *, alpha, beta, gamma, M, tol=1e-11, max_newton=200, cd_sweeps=200000):
    """Solution (u*, v*) of eq. (3).

    Newton's method with backtracking line search on the unconstrained objective
    (Section 4 obtains p* this way), accepted when the box is inactive; otherwise
    projected block coordinate descent with the Lambert-W block minimisers.
    """
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    A = _csr(A)
    m, n = A.m, A.n
    rows, cols = A.rows(), A.col_idx
    # Start from a few block sweeps: Newton's quadratic phase begins from a sane point.
    u, v = np.zeros(m), np.zeros(n)
    for _ in range(20):
        u = block_minimize_u(A, v, alpha=alpha, gamma=gamma, M=np.inf)
        v = block_minimize_v(A, u, beta=beta, gamma=gamma, M=np.inf)
    f = lambda uu, vv: objective(A, uu, vv, alpha=alpha, beta=beta, gamma=gamma)
    for _ in range(max_newton):
        gu, gv = gradient(A, u, v, alpha=alpha, beta=beta, gamma=gamma)
        g = np.concatenate([gu, gv])
        scale = max(1.0, alpha ** 2 * m + beta ** 2 * n) ** 0.5
        if np.linalg.norm(g) <= tol * scale:
            break
        q = A.vals ** 2 * np.exp(2 * u[rows] + 2 * v[cols])
        r = np.bincount(rows, weights=q, minlength=m)
        c = np.bincount(cols, weights=q, minlength=n)
        off = sp.csr_matrix((2 * q, (rows, cols)), shape=(m, n))
        H = sp.bmat([[sp.diags(2 * r + gamma), off], [off.T, sp.diags(2 * c + gamma)]], format="csc")
        if m + n <= 8000:
            step = -np.linalg.solve(H.toarray(), g)
        else:
            step, _ = spla.cg(H, -g, rtol=1e-13, maxiter=20 * (m + n))
        f0 = f(u, v)
        slope = g @ step
        tstep = 1.0
        while True:
            un, vn = u + tstep * step[:m], v + tstep * step[m:]
            if f(un, vn) <= f0 + 1e-4 * tstep * slope or tstep < 1e-12:
                break
            tstep *= 0.5
        u, v = un, vn
    if max(np.max(np.abs(u)), np.max(np.abs(v))) <= M:
        return u, v
    u, v = np.clip(u, -M, M), np.clip(v, -M, M)
    for _ in range(cd_sweeps):
        un = block_minimize_u(A, v, alpha=alpha, gamma=gamma, M=M)
        vn = block_minimize_v(A, un, beta=beta, gamma=gamma, M=M)
        done = max(np.max(np.abs(un - u)), np.max(np.abs(vn - v))) < tol
        u, v = un, vn
        if done:
            break
    return u, v


# ------------------------------------------------------------------ LSQR (Paige & Saunders 1982)

@dataclass
class LsqrResult:
    x: np.ndarray
    iters: int
    converged: bool
    rel_residual: float
    history: list = field(default_factory=list)


def lsqr(matvec, rmatvec, b, n, *, max_iters, residual=None, tol=0.0, check_every=1, keep_history=False):
    """LSQR on an operator K given by matvec (K x) and rmatvec (K^T y), FP64, x0 = 0.

    residual(x) -> relative residual of the problem the caller cares about; checked every
    check_every iterations against tol.  Returns the iterate xbar of the K-system.
    """
    b = _f64(b)
    x = np.zeros(n)
    beta = float(np.linalg.norm(b))
    hist = []
    if beta == 0.0:
        return LsqrResult(x, 0, True, 0.0, hist)
    u = b / beta
    v = rmatvec(u)
    alpha = float(np.linalg.norm(v))
    if alpha == 0.0:
        return LsqrResult(x, 0, True, 1.0, hist)
    v = v / alpha
    w = v.copy()
    phibar, rhobar = beta, alpha
    it = 0
    rel = float("nan")
    converged = False
    while it < max_iters:
        it += 1
        u = matvec(v) - alpha * u
        beta = float(np.linalg.norm(u))
        if beta > 0.0:
            u = u / beta
        v = rmatvec(u) - beta * v
        alpha = float(np.linalg.norm(v))
        if alpha > 0.0:
            v = v / alpha
        rho = math.hypot(rhobar, beta)
        c, s = rhobar / rho, beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        x = x + (phi / rho) * w
        w = v - (theta / rho) * w
        if residual is not None and (it % check_every == 0 or beta == 0.0 or alpha == 0.0):
            rel = float(residual(x))
            if keep_history:
                hist.append((it, rel))
            if rel <= tol:
                converged = True
                break
        if beta == 0.0 or alpha == 0.0:
            break
    return LsqrResult(x, it, converged, rel, hist)
