"""The multi-GPU host logic on CPU: two gloo ranks split beams, take the
slowest rank's time and sum weight gradients, exactly as bench.py's
torchrun path does on GPUs."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1601_05052_gb300.shard import allreduce_grad_w, beams_for_rank, max_over_ranks


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_beams, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = list(beams_for_rank(n_beams, rank, world))
        got = [None] * world
        dist.all_gather_object(got, mine)
        t = max_over_ranks(1.0 + rank)
        gw = torch.full((5,), float(rank + 1))
        allreduce_grad_w(gw)
        out.put((rank, got, t, gw.tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n_beams", [7, 128, 1])
def test_two_gloo_ranks(n_beams):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_beams, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, t, gw in res:
        flat = [b for share in got for b in share]
        assert sorted(flat) == list(range(n_beams))  # every beam exactly once
        assert max(len(s) for s in got) - min(len(s) for s in got) <= 1
        assert t == 2.0
        assert gw == [3.0] * 5


def test_split_is_contiguous_and_balanced():
    for n in range(0, 40):
        for w in range(1, 9):
            shares = [beams_for_rank(n, r, w) for r in range(w)]
            assert [b for s in shares for b in s] == list(range(n))
    with pytest.raises(ValueError):
        beams_for_rank(4, 2, 2)
