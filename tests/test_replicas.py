"""The replica (N > 1) host logic of bench.py on CPU: two gloo ranks agree on
the largest per-rank time and the whole-job throughput counts every rank's
points; the reference arm does no work off rank 0."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t = bench.max_over_ranks(10.0 + 5.0 * rank, ws)
    v = bench.aggregate_gpts(100_000, ws, 50, t)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, v))


def test_two_gloo_ranks_agree_on_max_and_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]
    # 2 ranks x 1e5 points x 50 steps in 15 ms
    assert abs(out[0][2] - 2 * 1e5 * 50 / 15e-3 / 1e9) < 1e-9
    assert out[0][2] == out[1][2]


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert abs(bench.aggregate_gpts(1000, 1, 10, 1.0) - 1e-2) < 1e-15


def test_reference_arm_off_rank_zero_does_nothing(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(None) is None     # returns before touching args or the oracle
