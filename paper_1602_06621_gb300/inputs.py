"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module draws matrices and vectors only.  It holds none of the
equilibration arithmetic: no scalings are applied to a matrix here other than
the generative "badly scaled" construction the paper uses for its test
problems, and no probe signs are drawn here (both sides generate those from
the same counter-based Philox definition).

Workloads follow the paper's experiments (Section 4 and Section 5.1): a sparse
matrix with uniform-random sparsity pattern, standard-normal nonzeros, and
log-normal row and column factors,

    A = diag(e^r) * G * diag(e^c),   G_ij ~ N(0, 1),

where the paper draws r, c with mean 1 and variance 1.  The large workloads
stretch the factors to variance 2 ("N(0, 2)" read as mean 0, variance 2) so
that A is badly scaled.  All draws use NumPy's PCG64 with an explicit seed, so
the same seed gives the same matrix on every machine.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "CSR",
    "sparse_uniform_density",
    "sparse_fixed_row_nnz",
    "sparse_variable_row_nnz",
    "dense_badly_scaled",
    "normal_vector",
    "small_dense_positive",
    "workload_small",
    "workload_large",
]


@dataclass
class CSR:
    """A sparse matrix in compressed-row form, columns sorted within each row."""

    m: int
    n: int
    row_ptr: np.ndarray  # int32 [m+1]
    col_idx: np.ndarray  # int32 [nnz]
    vals: np.ndarray  # float32 or float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        out = np.zeros((self.m, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        out[rows, self.col_idx] = self.vals
        return out

    def astype(self, dtype) -> "CSR":
        return CSR(self.m, self.n, self.row_ptr, self.col_idx, self.vals.astype(dtype))


def _log_normal_factors(rng: np.random.Generator, size: int, mean: float, var: float) -> np.ndarray:
    return np.exp(rng.normal(mean, np.sqrt(var), size=size))


def _assemble(m, n, rows, cols, rng, mean, var, dtype) -> CSR:
    order = np.lexsort((cols, rows))
    rows = rows[order]
    cols = cols[order]
    g = rng.standard_normal(rows.size)
    r = _log_normal_factors(rng, m, mean, var)
    c = _log_normal_factors(rng, n, mean, var)
    vals = (g * r[rows] * c[cols]).astype(dtype)
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz exceeds int32 range")
    return CSR(m, n, row_ptr.astype(np.int32), cols.astype(np.int32), vals)


def sparse_uniform_density(m: int, n: int, density: float, seed: int, *, mean: float = 0.0,
                           var: float = 2.0, dtype=np.float64) -> CSR:
    """round(density*m*n) positions drawn uniformly without replacement (Section 4)."""
    rng = np.random.default_rng(seed)
    nnz = int(round(density * m * n))
    flat = rng.choice(m * n, size=nnz, replace=False)
    rows = (flat // n).astype(np.int64)
    cols = (flat % n).astype(np.int64)
    return _assemble(m, n, rows, cols, rng, mean, var, dtype)


def _distinct_columns_per_row(rng: np.random.Generator, m: int, n: int, lens: np.ndarray) -> np.ndarray:
    """For row i draw lens[i] distinct columns uniformly from [0, n); returns the column ids row by row."""
    lmax = int(lens.max()) if lens.size else 0
    if lmax > n:
        raise ValueError("row length exceeds n")
    cols = rng.integers(0, n, size=(m, lmax), dtype=np.int64)
    mask = np.arange(lmax)[None, :] < lens[:, None]
    # Rows long enough that a repeat is likely (lens^2 > n / 4) draw without replacement directly;
    # the others redraw until no column repeats among their first lens[i] slots.
    crowded = np.nonzero(lens * lens * 4 > n)[0]
    for i in crowded:
        cols[i, : lens[i]] = rng.choice(n, size=int(lens[i]), replace=False)
    sparse_rows = np.ones(m, dtype=bool)
    sparse_rows[crowded] = False
    while True:
        masked = np.where(mask, cols, -1 - np.arange(lmax)[None, :])
        s = np.sort(masked, axis=1)
        dup = np.any((s[:, 1:] == s[:, :-1]) & (s[:, 1:] >= 0), axis=1) & sparse_rows
        bad = np.nonzero(dup)[0]
        if bad.size == 0:
            break
        cols[bad] = rng.integers(0, n, size=(bad.size, lmax), dtype=np.int64)
    return cols[mask]


def sparse_fixed_row_nnz(m: int, n: int, row_nnz: int, seed: int, *, mean: float = 0.0,
                         var: float = 2.0, dtype=np.float32) -> CSR:
    """Exactly row_nnz distinct uniform-random columns in every row."""
    rng = np.random.default_rng(seed)
    lens = np.full(m, row_nnz, dtype=np.int64)
    cols = _distinct_columns_per_row(rng, m, n, lens)
    rows = np.repeat(np.arange(m, dtype=np.int64), lens)
    return _assemble(m, n, rows, cols, rng, mean, var, dtype)


def sparse_variable_row_nnz(m: int, n: int, lo: int, hi: int, seed: int, *, mean: float = 0.0,
                            var: float = 2.0, dtype=np.float32) -> CSR:
    """Row lengths uniform integers in [lo, hi], distinct uniform-random columns."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(lo, hi + 1, size=m).astype(np.int64)
    lens = np.minimum(lens, n)
    cols = _distinct_columns_per_row(rng, m, n, lens)
    rows = np.repeat(np.arange(m, dtype=np.int64), lens)
    return _assemble(m, n, rows, cols, rng, mean, var, dtype)


def dense_badly_scaled(m: int, n: int, seed: int, *, mean: float = 0.0, var: float = 1.5,
                       dtype=np.float32) -> np.ndarray:
    """Dense G_ij ~ N(0,1) with log-normal row and column factors, row-major."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((m, n))
    r = _log_normal_factors(rng, m, mean, var)
    c = _log_normal_factors(rng, n, mean, var)
    return (g * r[:, None] * c[None, :]).astype(dtype)


def small_dense_positive(m: int, n: int, seed: int) -> np.ndarray:
    """Small dense matrix with strictly positive entries, spread over a few decades."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.normal(0.0, 1.0, size=(m, n)))


def normal_vector(n: int, seed: int, dtype=np.float64) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(n).astype(dtype)


def workload_small(seed: int = 1) -> CSR:
    """2000 x 1000, 1% density (20,000 nonzeros), factors of variance 2, float64."""
    return sparse_uniform_density(2000, 1000, 0.01, seed, var=2.0, dtype=np.float64)


def workload_large(scale: float = 1.0, seed: int = 2) -> CSR:
    """1e6 x 5e5 (times scale), 20 nonzeros per row, factors of variance 2, float32."""
    m = max(64, int(round(1_000_000 * scale)))
    n = max(32, int(round(500_000 * scale)))
    return sparse_fixed_row_nnz(m, n, 20, seed, var=2.0, dtype=np.float32)


def _family_member(job):
    m, n, lo, hi, s, var, dtype = job
    return sparse_variable_row_nnz(m, n, lo, hi, s, var=var, dtype=dtype)


def batched_family(count: int, m_lo: int, m_hi: int, seed: int, *, nnz_lo: int = 5, nnz_hi: int = 50,
                   var: float = 2.0, dtype=np.float32, workers: int = 0):
    """count matrices: m log-uniform in [m_lo, m_hi], n = round(m * U[0.3, 1.0]), row lengths uniform
    integers in [nnz_lo, nnz_hi] (capped at n), factors of variance `var`.  workers > 1 generates the
    matrices in that many spawned processes (same result; call it before the process touches the GPU)."""
    rng = np.random.default_rng(seed)
    ms = np.exp(rng.uniform(np.log(m_lo), np.log(m_hi), size=count)).round().astype(np.int64)
    ns = np.maximum(1, np.round(ms * rng.uniform(0.3, 1.0, size=count))).astype(np.int64)
    seeds = rng.integers(0, 2 ** 31, size=count)
    jobs = [(int(m), int(n), nnz_lo, nnz_hi, int(s), var, dtype) for m, n, s in zip(ms, ns, seeds)]
    if workers > 1 and count > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, count)) as pool:
            return pool.map(_family_member, jobs, chunksize=max(1, count // (4 * workers)))
    return [_family_member(j) for j in jobs]
