"""One matrix split over several devices: Algorithm 1 with one all-gather of the gather tables per iteration.

Every iteration of Algorithm 1 forms both estimates from the previous iterate: the rows of A need e^{v_j} and
the probe signs s_j of every column, the columns need e^{u_i} and w_i of every row.  A part (one device, one
process) holds only its row block of A and its column block of A^T (sme_op_create_csr_shard) and writes
e^{x} and the probe words of its own rows and columns into its chunk of two gather tables; an all-gather of
equal chunks then gives every part the whole tables for the next iteration.  That is the method's only
exchange: (m + n) table entries per iteration (8 bytes each in FP32 with k <= 32).  Probe signs are
counter-based, so none travel.

The loop (`run`) is written once for any exchange: `CollectiveExchange` all-gathers in place with
torch.distributed (NCCL between GPUs), `LocalExchange` copies chunks between the tables of several parts held
by one process (several parts on one device).  This module only marshals buffers; the iteration itself runs
in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import sme

__all__ = ["blocks", "Part", "CollectiveExchange", "LocalExchange", "run"]


def blocks(length: int, parts: int):
    """Block boundaries: block q = [length q / parts, length (q + 1) / parts) (the library's partition)."""
    return [length * q // parts for q in range(parts + 1)]


@dataclass
class _Tables:
    row: list  # two uint8 tensors: current and next
    col: list


class Part:
    """One part of a split matrix with its state and its two pairs of gather tables (device tensors)."""

    def __init__(self, op, k: int, device, dtype=None):
        import torch

        self.op = op
        self.k = int(k)
        self.info = sme.sme_shard_get_info(op, self.k)
        self.part, self.parts = self.info["part"], self.info["parts"]
        eb = self.info["entry_bytes"]
        self.row_chunk_bytes = self.info["row_chunk"] * eb
        self.col_chunk_bytes = self.info["col_chunk"] * eb
        self.dtype = dtype or torch.float32
        rows = self.info["row_end"] - self.info["row_begin"]
        cols = self.info["col_end"] - self.info["col_begin"]
        z = lambda n: torch.zeros(n, dtype=self.dtype, device=device)
        self.u, self.v, self.u_bar, self.v_bar = z(rows), z(cols), z(rows), z(cols)
        t = lambda b: torch.empty(self.parts * b, dtype=torch.uint8, device=device)
        self.tables = _Tables([t(self.row_chunk_bytes), t(self.row_chunk_bytes)],
                              [t(self.col_chunk_bytes), t(self.col_chunk_bytes)])

    def row_chunk(self, table, q):
        return table[q * self.row_chunk_bytes:(q + 1) * self.row_chunk_bytes]

    def col_chunk(self, table, q):
        return table[q * self.col_chunk_bytes:(q + 1) * self.col_chunk_bytes]

    def begin(self, cur, params):
        sme.sme_shard_begin(self.op, self.u, self.v, self.u_bar, self.v_bar, self.tables.row[cur],
                            self.tables.col[cur], **params)

    def step(self, t, cur, params):
        sme.sme_shard_step(self.op, t, self.tables.row[cur], self.tables.col[cur], self.tables.row[cur ^ 1],
                           self.tables.col[cur ^ 1], **params)

    def end(self):
        sme.sme_shard_end(self.op, self.u, self.v, self.u_bar, self.v_bar)


class CollectiveExchange:
    """All-gather of equal chunks in place, one part per process (torch.distributed, NCCL between GPUs)."""

    def __init__(self, group=None):
        self.group = group

    def __call__(self, parts, cur):
        import torch.distributed as dist

        (p,) = parts
        for table, chunk in ((p.tables.row[cur], p.row_chunk), (p.tables.col[cur], p.col_chunk)):
            dist.all_gather_into_tensor(table, chunk(table, p.part), group=self.group)


class LocalExchange:
    """Several parts held by one process (for instance on one device): every part's chunk is copied into the
    other parts' tables, stream-ordered device copies."""

    def __call__(self, parts, cur):
        for src in parts:
            for dst in parts:
                if dst is not src:
                    dst.row_chunk(dst.tables.row[cur], src.part).copy_(src.row_chunk(src.tables.row[cur], src.part))
                    dst.col_chunk(dst.tables.col[cur], src.part).copy_(src.col_chunk(src.tables.col[cur], src.part))


def run(parts, exchange, *, T, k, t_begin=1, t0=0, seed=0, stream_base=0, alpha=0.0, beta=0.0, gamma=0.0, M=0.0):
    """Iterations t_begin .. t_begin + T - 1 of Algorithm 1 on the parts held here, from their start state
    (u, v, u_bar, v_bar of each part), exchanging the tables after the start and after every iteration."""
    params = dict(T=T, k=k, t_begin=t_begin, t0=t0, seed=seed, stream_base=stream_base, alpha=alpha, beta=beta,
                  gamma=gamma, M=M)
    cur = t_begin & 1
    for p in parts:
        p.begin(cur, params)
    exchange(parts, cur)
    for t in range(t_begin, t_begin + T):
        for p in parts:
            p.step(t, cur, params)
        cur ^= 1
        exchange(parts, cur)
    for p in parts:
        p.end()
