"""The multi-rank form of bench.py on the CPU (gloo, world size 2): every rank analyses its
own seeded problems (weak scaling, no data-path collective), the job's time is the slowest
rank's (all_reduce MAX), and the reported value is the units of all ranks over that time."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, _ = bench._dist()
        seed = bench._rank_seed(1, got_rank)
        spec = synth.problems.batched_problem_specs(3, seed)
        local_ms = [7.0, 11.5][rank]                      # rank 1 is the slower one
        ms = bench._max_over_ranks(local_ms, torch.device("cpu"), got_ws)
        rate = bench._job_rate(5, ms / 1e3, got_ws)       # 5 analyses per rank
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([got_ws, got_rank, seed, ms, rate] + [s["n"] for s in spec], dtype=np.float64))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_weak_scaling_on_gloo(tmp_path):
    mp.start_processes(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    r0, r1 = (np.load(tmp_path / f"r{k}.npy") for k in range(2))
    assert r0[0] == r1[0] == 2 and (r0[1], r1[1]) == (0, 1)
    assert r0[2] != r1[2]                                 # each rank its own seed ...
    assert not np.array_equal(r0[5:], r1[5:])             # ... and so its own problems
    assert r0[3] == r1[3] == 11.5                         # the slowest rank's time, on both
    assert r0[4] == r1[4] == pytest.approx(2 * 5 / 11.5e-3)   # all ranks' analyses / that time


def test_single_rank_helpers():
    assert bench._rank_seed(3, 0) == 3
    assert bench._max_over_ranks(4.25, None, 1) == 4.25
    assert bench._job_rate(256, 0.5, 1) == 512.0


def test_recorded_traffic_only_for_the_captured_configuration():
    """The DRAM bytes of a capture are reported only for the configuration it measured (CG
    preconditioned by R, atomic step sums) and while the kernel sources keep its hash."""
    for prec, rec in bench.NCU_TRAFFIC.items():
        got = bench._recorded_traffic(prec, 1, 1)
        assert got == (rec["bytes"] if rec["src_sha"] == bench._src_hash(prec) else None)
        assert bench._recorded_traffic(prec, 0, 1) is None
        assert bench._recorded_traffic(prec, 1, 0) is None
    assert bench._recorded_traffic("fp64", 1, 1) is None
    assert bench._recorded_traffic("bf16", 1, 1) is None
