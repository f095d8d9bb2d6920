"""The exchange of a split matrix, on CPU: two ranks over gloo (world size 2).

A part of a split matrix writes only its own chunk of the two gather tables; the loop in
paper_1602_06621_gb300.shard all-gathers the tables after the start and after every iteration, alternating
between the current and the next pair.  Here each rank drives a stand-in part (no GPU) that writes bytes
derived from (iteration, part, table) into its chunk and checks, before every step, that its current tables
hold every part's chunk of the previous iteration at the right offsets.  The partition itself (block q =
[len q / P, len (q + 1) / P)) and the library's argument checks are tested alongside.
"""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _StandInPart:
    """Duck-typed like shard.Part: tables of uneven chunk sizes, bytes marking (iteration, part, table)."""

    def __init__(self, part, parts):
        import torch

        self.part, self.parts = part, parts
        self.row_chunk_bytes, self.col_chunk_bytes = 24, 40

        class _T:
            pass

        self.tables = _T()
        self.tables.row = [torch.zeros(parts * 24, dtype=torch.uint8) for _ in range(2)]
        self.tables.col = [torch.zeros(parts * 40, dtype=torch.uint8) for _ in range(2)]
        self.checked = 0

    def row_chunk(self, table, q):
        return table[q * self.row_chunk_bytes:(q + 1) * self.row_chunk_bytes]

    def col_chunk(self, table, q):
        return table[q * self.col_chunk_bytes:(q + 1) * self.col_chunk_bytes]

    @staticmethod
    def mark(t, q, which):
        return (7 * t + 31 * q + 3 * which + 1) % 251

    def _write(self, t, slot):
        self.row_chunk(self.tables.row[slot], self.part).fill_(self.mark(t, self.part, 0))
        self.col_chunk(self.tables.col[slot], self.part).fill_(self.mark(t, self.part, 1))

    def _check(self, t, slot):
        for q in range(self.parts):
            assert int(self.row_chunk(self.tables.row[slot], q).min()) == self.mark(t, q, 0)
            assert int(self.row_chunk(self.tables.row[slot], q).max()) == self.mark(t, q, 0)
            assert int(self.col_chunk(self.tables.col[slot], q).min()) == self.mark(t, q, 1)
            assert int(self.col_chunk(self.tables.col[slot], q).max()) == self.mark(t, q, 1)
        self.checked += 1

    def begin(self, cur, params):
        self._write(params["t_begin"], cur)

    def step(self, t, cur, params):
        self._check(t, cur)          # every part's tables of iteration t, gathered
        self._write(t + 1, cur ^ 1)  # this part's chunk of iteration t + 1

    def end(self):
        pass


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_1602_06621_gb300 import shard as SH
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        p = _StandInPart(rank, world)
        SH.run([p], SH.CollectiveExchange(), T=6, k=32, t_begin=3)
        p._check(9, (3 + 6) & 1)  # the tables after the last exchange
        dist.destroy_process_group()
        q.put((rank, p.checked, None))
    except Exception as e:
        q.put((rank, None, repr(e)))


def test_split_matrix_exchange_world_size_2():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    for rank, checked, err in out:
        assert err is None, f"rank {rank}: {err}"
        assert checked == 7  # six steps and the final tables


def test_local_exchange_assembles_every_chunk():
    """Several parts held by one process: LocalExchange copies every part's chunk into the others' tables."""
    from paper_1602_06621_gb300 import shard as SH
    parts = [_StandInPart(q, 3) for q in range(3)]
    SH.run(parts, SH.LocalExchange(), T=4, k=8, t_begin=1)
    for p in parts:
        p._check(5, (1 + 4) & 1)
        assert p.checked == 5


@pytest.mark.parametrize("length,parts", [(10, 3), (7, 7), (1000001, 4), (5, 1)])
def test_blocks_partition(length, parts):
    from paper_1602_06621_gb300 import shard as SH
    b = SH.blocks(length, parts)
    assert b[0] == 0 and b[-1] == length and len(b) == parts + 1
    sizes = np.diff(b)
    assert sizes.min() >= 1 and sizes.max() - sizes.min() <= 1
    # block(i) = ((i + 1) parts - 1) // length, the library's formula, agrees with the boundaries
    for q in range(parts):
        for i in (b[q], b[q + 1] - 1):
            assert ((i + 1) * parts - 1) // length == q


@pytest.mark.parametrize("parts,part", [(0, 0), (2, 2), (2, -1), (7, 0)])
def test_split_creation_argument_errors(parts, part):
    """Bad part counts are refused on the host, before any device work."""
    from paper_1602_06621_gb300 import sme
    rp = np.array([0, 2, 3, 5, 6, 6, 7], np.int32)  # 6 x 4
    col = np.array([0, 2, 1, 0, 3, 1, 2], np.int32)
    val = np.ones(7)
    with pytest.raises(sme.SmeError) as ei:
        sme.sme_op_create_csr_shard(6, 4, rp, col, val, parts, part, stream=0)
    assert ei.value.name == "SME_ERR_ARG"
