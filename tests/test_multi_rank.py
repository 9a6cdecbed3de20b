"""Host logic of the N > 1 bench path on CPU: two gloo ranks (no GPU).

Cells and frames are independent, so ranks shard by frame with no data-path
collective; the only collective is the max over ranks of the timed region.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        # slowest rank sets the job time; every rank sees the same max
        t = bench.max_over_ranks(10.0 + 5.0 * rank, ws)
        out[rank] = (t, bench.rank_seed(100, rank, 0), bench.rank_seed(100, rank, 1))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_shard_frames():
    ws, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    seeds = {res[r][1] for r in range(ws)} | {res[r][2] for r in range(ws)}
    assert len(seeds) == 2 * ws                      # no two frames shared between ranks


def test_weak_scaling_value():
    import bench
    # 1M cells per frame, 10 steps per rank, 2 ranks, slowest rank 200 ms
    assert bench.job_value(1 << 20, 10, 2, 200.0) == pytest.approx((1 << 20) * 20 / 0.2)
    assert bench.max_over_ranks(3.5, 1) == 3.5
