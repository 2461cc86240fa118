"""Two ranks (gloo, both on cuda:0, no kernel of one waits on the other) give
what one rank gives on the union of their cells: the adjoint's ln A gradient
summed over the ranks (one all-reduce of M doubles), and the parameters after
two data-parallel training steps (gradient shares summed in place, then Adam
on every rank)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

NCELLS, NBATCH, LR = 4096, 512, 1e-3


def _setup():
    import paper_2210_07094_gb300 as df
    from paper_2210_07094_gb300 import surrogate, synth
    mech = synth.h2_air_mechanism()
    m = df.Mechanism(mech)
    f = synth.field(0, mech, NCELLS, seed=515)
    T, p, Y = (torch.tensor(np.ascontiguousarray(f[k]), device="cuda:0") for k in ("T", "p", "Y"))
    Ts, pt, Ys = surrogate.trajectories(m, mech, NBATCH // 2, 2, seed=616)
    pairs = surrogate.pairs(Ts, pt, Ys)
    o = df.dnn_default_opts()
    o.width[0], o.width[1], o.width[2] = 64, 32, 16
    o.batch = NBATCH
    dnn = df.Dnn(o, seed=3)
    dnn.fit_norm(pairs[0], pairs[1], pairs[2], pairs[4])
    return df, m, f, (T, p, Y), pairs, dnn


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2210_07094_gb300 import shard
        df, m, f, (T, p, Y), pairs, dnn = _setup()
        lo, hi = shard.partition(NCELLS, world)[rank]
        ones = torch.ones(hi - lo, dtype=torch.float64, device="cuda:0")
        r = shard.adjoint_sharded(m, T[lo:hi].contiguous(), p[lo:hi].contiguous(), Y[:, lo:hi].contiguous(),
                                  f["dt"], gT1=ones, gQ1=ones)
        g_lnA = r["g_lnA"].cpu().numpy()
        blo, bhi = shard.partition(NBATCH, world)[rank]
        T0, P0, Y0, _, Y1 = (a[..., blo:bhi].contiguous() for a in pairs)
        losses = [shard.dp_train_step(dnn, T0, P0, Y0, Y1, LR, NBATCH) for _ in range(2)]
        out[rank] = (g_lnA, dnn.params(), losses, int((r["status"] != 0).sum()))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_match_one_rank_on_the_union():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")  # no fork after the GPU has been used
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(600)
        assert p.exitcode == 0
    df, m, f, (T, p, Y), pairs, dnn = _setup()
    ones = torch.ones(NCELLS, dtype=torch.float64, device="cuda:0")
    ref = df.adjoint(m, T, p, Y, f["dt"], gT1=ones, gQ1=ones)
    g1 = ref["g_lnA"].cpu().numpy()
    T0, P0, Y0, _, Y1 = (a[..., :NBATCH].contiguous() for a in pairs)
    losses1 = [dnn.train_step(T0, P0, Y0, Y1, LR) for _ in range(2)]
    theta1 = dnn.params()
    for rank in range(world):
        g, theta, losses, bad = out[rank]
        assert bad == 0
        # the same terms summed in another order (per rank, then across ranks)
        assert np.allclose(g, g1, rtol=1e-11, atol=1e-11 * np.abs(g1).max()), np.abs(g - g1).max()
        # FP32 gradients summed in another order; Adam's step is ~lr per element
        d = np.abs(theta - theta1)
        assert d.max() <= 2e-2 * LR and np.median(d) <= 1e-4 * LR, (d.max(), np.median(d))
        assert np.allclose(losses, losses1, rtol=1e-5)
    assert np.array_equal(out[0][1], out[1][1])  # every rank holds the same parameters
    assert np.array_equal(out[0][0], out[1][0])
