"""The bench's N > 1 path (independent replicas, one per rank) on CPU with two
gloo ranks: barrier, max / sum over ranks, per-rank sources and the whole-job
time per solve."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1010_4782_gb300 import inputs
from paper_1010_4782_gb300.replicas import Replicas, dist_env


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    w, r, local = dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        reps = Replicas(w, r, "cpu")
        reps.barrier()
        elapsed = 1.0 + r  # rank 1 is the slower one
        res = {"max": reps.max(elapsed), "sum": reps.sum(10 * (r + 1)),
               "per_solve": reps.time_per_solve(reps.max(elapsed), steps=3),
               "seed": reps.source_seed()}
        src = inputs.gaussian_even_source((2, 2, 2, 4), res["seed"])
        res["src_norm"] = float(np.linalg.norm(src))
        out[r] = res
        reps.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for r in (0, 1):
        assert res[r]["max"] == 2.0          # the slowest rank's time on every rank
        assert res[r]["sum"] == 30.0
        assert res[r]["per_solve"] == 2.0 / (3 * 2)
    assert res[0]["seed"] != res[1]["seed"]   # independent replicas
    assert res[0]["src_norm"] != res[1]["src_norm"]


def test_single_process_needs_no_process_group():
    reps = Replicas(1, 0)
    reps.barrier()
    assert reps.max(3.5) == 3.5 and reps.sum(2) == 2.0
    assert reps.time_per_solve(6.0, steps=3) == 2.0
