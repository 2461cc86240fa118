"""Sharding of the chemistry substep over ranks, on CPU: the cell partition,
and two gloo ranks running the data-parallel training step's host logic
(gradient share -> in-place sum over the ranks -> Adam) with the CPU oracle as
each rank's compute.  The parameters after two steps equal one rank's on the
union of the rows."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2210_07094_gb300 import shard  # noqa: E402


def test_partition_even_and_balanced():
    assert shard.partition(10, 3) == [(0, 3), (3, 6), (6, 10)]
    assert shard.partition(0, 2) == [(0, 0), (0, 0)]
    assert shard.partition(5, 1) == [(0, 5)]
    rng = np.random.default_rng(1)
    work = np.where(rng.random(10000) < 0.5, 1.0, 12.0)  # bimodal substep counts
    parts = shard.partition(10000, 4, work)
    assert parts[0][0] == 0 and parts[-1][1] == 10000
    assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
    loads = [work[lo:hi].sum() for lo, hi in parts]
    assert max(loads) - min(loads) <= 2 * work.max()
    with pytest.raises(ValueError):
        shard.partition(3, 0)
    with pytest.raises(ValueError):
        shard.partition(3, 2, [1.0, -1.0, 1.0])


class OracleNet:
    """Stand-in for a Dnn handle whose compute is the CPU oracle (exact FP64
    network): grad() leaves this shard's share of the global-mean gradient in
    its buffer, adam_step() applies Adam to it."""

    def __init__(self, params, widths):
        from oracle import mlp
        self.mlp, self.widths = mlp, widths
        self.theta = mlp.pack(params, widths)
        self.m = np.zeros_like(self.theta)
        self.v = np.zeros_like(self.theta)
        self.t = 0
        self.buf = torch.zeros(self.theta.size, dtype=torch.float64)

    def grad(self, X, tgt, n_total, N):
        loss, g, _ = self.mlp.loss_and_grads(self.mlp.unpack(self.theta, self.widths), X, tgt, N, emulate=False)
        share = X.shape[0] / n_total
        self.buf.copy_(torch.from_numpy(self.mlp.pack(g, self.widths) * share))
        return loss * share

    def grad_tensor(self):
        return self.buf

    def adam_step(self, lr):
        self.t += 1
        self.theta, self.m, self.v = self.mlp.adam_step(self.theta, self.m, self.v, self.buf.numpy(), self.t, lr)


def _data(widths, rows, seed=3):
    from oracle import mlp
    rng = np.random.default_rng(seed)
    P = {name: rng.standard_normal(shp) * (0.3 if name.startswith("W") else 0.05)
         for name, shp in mlp.layout(widths)}
    X = np.zeros((rows, mlp.DNN_IN))
    X[:, :5] = rng.standard_normal((rows, 5))
    tgt = np.zeros((rows, mlp.DNN_OUT))
    tgt[:, :3] = rng.standard_normal((rows, 3))
    return P, X, tgt


def _dp_steps(net, X, tgt, n_total, group=None, steps=2):
    class Adapter:  # the call shape shard.dp_train_step expects of a Dnn
        def grad(self, T, p, Y, Y_next, n_total, want_loss):
            return net.grad(X, tgt, n_total, 3)

        def grad_tensor(self):
            return net.grad_tensor()

        def adam_step(self, lr):
            net.adam_step(lr)

    losses = [shard.dp_train_step(Adapter(), None, None, None, None, 1e-2, n_total, group) for _ in range(steps)]
    return net.theta, losses


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        widths = (8, 8, 8)
        P, X, tgt = _data(widths, 37)
        lo, hi = shard.partition(37, world)[rank]
        theta, losses = _dp_steps(OracleNet(P, widths), X[lo:hi], tgt[lo:hi], 37)
        out[rank] = (theta, losses)
    finally:
        dist.destroy_process_group()


def test_two_ranks_train_like_one_rank_on_the_union():
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
    widths = (8, 8, 8)
    P, X, tgt = _data(widths, 37)
    theta1, losses1 = _dp_steps(OracleNet(P, widths), X, tgt, 37)
    for rank in range(world):
        theta, losses = out[rank]
        assert np.allclose(theta, theta1, rtol=0, atol=1e-12), np.abs(theta - theta1).max()
        assert np.allclose(losses, losses1, rtol=1e-12)
    assert np.array_equal(out[0][0], out[1][0])  # every rank holds the same parameters
    assert not np.allclose(theta1, OracleNet(P, widths).theta)  # the steps moved them
