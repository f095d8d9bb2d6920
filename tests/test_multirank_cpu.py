"""The benchmark's multi-GPU path, on CPU: two ranks over gloo (world size 2).

Each rank equilibrates its own matrix (weak scaling, no data-path collective); the only collectives are the
barrier around the timed region and the maximum of the elapsed times over ranks, which rank 0 reports.
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


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    from paper_1602_06621_gb300 import inputs as I
    try:
        ranks = bench.Ranks(rank, world, 0, backend="gloo")
        ranks.barrier()
        elapsed = 0.25 * (rank + 1)  # rank 1 is the slow one
        got = ranks.max(elapsed)
        A = I.workload_large(0.0005, seed=bench.rank_matrix_seed(rank))
        ranks.barrier()
        ranks.close()
        q.put((rank, got, int(A.col_idx[:50].sum()), None))
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, None, None, repr(e)))


def test_two_ranks_time_by_the_slowest_and_work_on_different_matrices():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(2):
            rank, got, sig, err = q.get(timeout=120)
            assert err is None, err
            out[rank] = (got, sig)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    assert out[0][0] == out[1][0] == 0.5  # both ranks see the slowest rank's time
    assert out[0][1] != out[1][1]  # independent matrices per rank


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks(0, 1, 0, backend="gloo")
    assert r.dist is None and r.max(1.5) == 1.5
    r.close()
    assert np.isfinite(r.max(2.0))


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm (the oracle on the host) runs on rank 0; the other ranks exit at once."""
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        scale, k, T, steps, warmup = 0.001, 32, 500, 1, 0

    assert bench.run_reference(Args, 1, 2) == 0
