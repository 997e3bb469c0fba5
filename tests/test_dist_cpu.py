"""Host logic of the multi-process benchmark path on CPU (gloo, world size 2):
max-over-ranks timing, the whole-job weak-scaling value and per-rank views."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2509_03775_gb300 import scenes
    secs = 1.0 + rank          # rank 1 is the slow one
    m = bench.max_over_ranks(secs)
    val = bench.whole_job_value(10, world, m)
    _, cams = scenes.config_single(n=10, k=4, width=64, height=48)
    cam = bench.rank_camera(cams, rank)[0]
    out[rank] = (m, val, float(np.linalg.norm(cam.campos)), cam.width, cam.height,
                 tuple(np.round(cam.campos, 4)))
    bench.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_and_views():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 2.0                      # max over ranks
    assert r0[1] == r1[1] == pytest.approx(10 * 2 / 2.0)
    assert r0[2] == pytest.approx(r1[2], rel=1e-5)    # same radius
    assert (r0[3], r0[4]) == (r1[3], r1[4])           # same resolution: same per-rank work
    assert r0[5] != r1[5]                             # different views
