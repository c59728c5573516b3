"""The multi-rank bench path on CPU: two gloo ranks reduce their elapsed
times to the slowest one and report whole-job throughput of independent
replicas (weak scaling), each rank with its own seeded inputs."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
from paper_1801_10187_gb300 import inputs  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = [0.25, 0.40][rank]  # seconds on this rank
    slowest = bench.max_over_ranks(elapsed, dist, "cpu")
    rate = bench.job_rate(1000, world, slowest)
    cfg = bench.workload_cfg("srd-10c-rho5-fp64")
    s, _, _ = bench.make_state(cfg, seed_offset=rank)
    out[rank] = (slowest, rate, float(s.vel[0, 0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_and_replica_seeds():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    assert out[0][0] == out[1][0] == 0.40
    assert out[0][1] == out[1][1] == 1000 * 2 / 0.40
    # replicas draw different inputs (seed + rank)
    assert out[0][2] != out[1][2]
    cfg = bench.workload_cfg("srd-10c-rho5-fp64")
    ref = inputs.solvent(cfg["n"], cfg["density"], seed=cfg["seed"] + 1).vel[0, 0]
    assert out[1][2] == ref


def test_single_rank_helpers():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_rate(10, 1, 2.0) == 5.0
