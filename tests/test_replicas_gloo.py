"""The N > 1 bench path (replicas only) with two gloo ranks on the CPU.

The data path has no collective: each rank builds its own seeded dataset and
runs the whole step alone. Only the timing is combined: the slowest rank's
step time (max over ranks) and the whole-job throughput = ranks x points per
step / that time. Both are checked here with world size 2, without a GPU.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _Args:
    n, d, nq, components = 400, 8, 16, 5


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        x, q = bench.make_inputs(_Args, rank)
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        out[rank] = (ms, bench.job_value(ws, _Args.n, ms), float(x[0, 0]), float(x.sum()), x.shape, q.shape)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_timing_and_seed_replicas():
    ws = 2
    with mp.Manager() as man:
        out = man.dict()
        mp.start_processes(_rank, args=(ws, _free_port(), out), nprocs=ws, start_method="spawn", join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for r in range(ws):
        ms, val, _, _, xs, qs = res[r]
        assert ms == 15.0  # the slower rank's time, on every rank
        assert val == pytest.approx(ws * _Args.n / 15.0e-3)
        assert xs == (_Args.n, _Args.d) and qs == (_Args.nq, _Args.d)
    # each replica has its own data (seed offset by rank), reproducibly
    assert res[0][3] != res[1][3]
    import bench
    x0, _ = bench.make_inputs(_Args, 0)
    assert np.isclose(float(x0.sum()), res[0][3])


def test_one_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_value(1, 3_000_000, 100.0) == pytest.approx(3e7)
