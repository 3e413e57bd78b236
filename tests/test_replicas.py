"""The multi-rank (replicas) path of bench.py on CPU: two gloo ranks.

With one process per GPU, every rank solves its own problems (the batched workload is split round robin, no
data exchange) and only the timing is reduced: the slowest rank's time and the sum of all ranks' work.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        mine = bench.shard(range(64), ws, rank)
        all_shards = [None] * ws
        dist.all_gather_object(all_shards, mine)
        t_ms = 100.0 + 50.0 * rank          # ranks finish at different times
        flops = 1e12 * (rank + 1)
        (t_max,) = bench.reduce_over_ranks([t_ms], "max")
        (f_sum,) = bench.reduce_over_ranks([flops], "sum")
        out[rank] = {"shards": all_shards, "t_max": t_max, "f_sum": f_sum,
                     "value": bench.whole_job_tflops(f_sum, t_max)}
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True, start_method="spawn")
        res = dict(out)
    assert set(res) == {0, 1}
    for r in range(ws):
        shards = res[r]["shards"]
        flat = sorted(x for s in shards for x in s)
        assert flat == list(range(64))                       # every problem once
        assert not set(shards[0]) & set(shards[1])           # disjoint
        assert res[r]["t_max"] == 150.0                      # slowest rank's time on every rank
        assert res[r]["f_sum"] == 3e12                       # all ranks' work
        assert abs(res[r]["value"] - 3e12 / 0.150 / 1e12) < 1e-9


def test_single_process_reduction_is_identity():
    import bench
    assert not dist.is_initialized()
    assert bench.reduce_over_ranks([1.5, 2.0], "max") == [1.5, 2.0]
    assert bench.shard(range(5), 1, 0) == [0, 1, 2, 3, 4]
