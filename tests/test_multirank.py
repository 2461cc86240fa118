"""The replicas-only multi-GPU path of bench.py, on CPU: two gloo ranks
aggregate their timings (max over ranks) and unit counts (sum), and every rank
advances its own, different field of the same distribution."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench._rank_info()
        t_local = [0.5, 0.8][rank]
        units = [1000, 3000][rank]
        rate, t_max, total = bench.whole_job_rate(t_local, units, dist, "cpu")
        out[rank] = (r, w, lr, rate, t_max, total, bench.field_seed(rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregate_and_fields():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")  # no fork after the GPU has been used
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for rank in range(world):
        r, w, lr, rate, t_max, total, seed = out[rank]
        assert (r, w, lr) == (rank, world, rank)
        assert t_max == 0.8 and total == 4000.0  # slowest rank's time, all ranks' units
        assert rate == pytest.approx(4000.0 / 0.8)
    assert out[0][6] != out[1][6]
    from paper_2210_07094_gb300 import synth
    mech = synth.h2_air_mechanism()
    f0 = synth.field(1, mech, 64, seed=out[0][6])
    f1 = synth.field(1, mech, 64, seed=out[1][6])
    assert not np.array_equal(f0["T"], f1["T"])
    # same distribution: both bimodal in T
    for f in (f0, f1):
        assert np.all((f["T"] >= 700) & (f["T"] <= 2500))


def test_single_rank_rate_without_a_process_group():
    import bench
    rate, t_max, total = bench.whole_job_rate(2.0, 10, None, "cpu")
    assert (rate, t_max, total) == (5.0, 2.0, 10.0)
