"""The multi-GPU path of the bench is replicas only (independent stereo frames,
no collective on the data path): the host logic that assigns frames to ranks
and turns the ranks' times into the whole-job number, run as two gloo ranks on
the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def test_rank_poses_are_disjoint_per_step():
    poses = list(range(8))
    for world in (1, 2, 4, 8):
        per_rank = [bench.rank_poses(poses, r, world) for r in range(world)]
        for k in range(8):
            step = [p[k] for p in per_rank]
            assert len(set(step)) == world  # no two ranks render one pose at one step
        assert set().union(*map(set, per_rank)) == set(poses)  # together they cover the arc
    assert bench.rank_poses(poses, 0, 1) == poses


def test_job_time_single_rank():
    assert bench.job_ms_per_frame(2.0, 10, 1) == 2.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def reduce_max(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    out[rank] = bench.job_ms_per_frame(ms[rank], 10, world, reduce_max)
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_slowest_rank_over_all_frames():
    world, port = 2, _free_port()
    ms = [1.0, 1.5]  # per-step times of the two ranks
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, ms, out), nprocs=world, join=True)
        got = dict(out)
    # both ranks report the slowest rank's 10 steps over the 20 frames rendered
    assert got[0] == got[1] == pytest.approx(1.5 * 10 / 20)
