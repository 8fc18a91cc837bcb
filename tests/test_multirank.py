"""The multi-GPU path of bench.py on the CPU: two gloo ranks (one process
each, rendezvous on 127.0.0.1) with different step times. Each rank takes a
disjoint seeded batch, the job's time is the slowest rank's, the job's
frames/s counts every rank's frames; the reference arm runs on rank 0 only."""

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


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world)})
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        my_ms = 2.0 + 3.0 * rank                # rank 1 is the slow one
        job_ms = bench.max_over_ranks(my_ms, dist, "cpu")
        value = bench.whole_job_frames_per_s(bench.FRAMES, world, job_ms)
        seed = bench.rank_seed0(rank)
        seeds = [None] * world
        dist.all_gather_object(seeds, seed)
        np.save(os.path.join(out_dir, "rank%d.npy" % rank), np.array([job_ms, value, *seeds], dtype=np.float64))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    r = [np.load(tmp_path / ("rank%d.npy" % i)) for i in range(world)]
    sys.path.insert(0, ROOT)
    import bench
    for v in r:
        assert v[0] == 5.0                                   # the slowest rank's time, on every rank
        assert v[1] == pytest.approx(2 * bench.FRAMES / 5e-3)  # both ranks' frames over that time
        assert list(v[2:]) == [bench.SEED0, bench.SEED0 + bench.FRAMES]
    # the ranks' batches are different seeded frames
    from paper_1705_04298_gb300 import synth
    a, _, _ = synth.batch(8, 2, bench.rank_seed0(0), 0.05)
    b, _, _ = synth.batch(8, 2, bench.rank_seed0(1), 0.05)
    assert not np.allclose(a, b)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.whole_job_frames_per_s(1000, 1, 1.0) == pytest.approx(1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        gpus, steps, warmup = 2, 1, 0
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""
