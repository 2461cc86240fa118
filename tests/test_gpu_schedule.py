"""Scheduling of the persistent integrator launch: the autotuner's choice, the
independence of every cell's result from the launch shape and the work order,
and replay of the whole step from a captured CUDA graph."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2210_07094_gb300 as df  # noqa: E402
from paper_2210_07094_gb300 import synth  # noqa: E402

DEV = "cuda:0"


def _dev(f):
    return (torch.tensor(f["T"], device=DEV), torch.tensor(f["p"], device=DEV),
            torch.tensor(np.ascontiguousarray(f["Y"]), device=DEV))


def _run(m, T0, p, Y0, dt, opts=None):
    T, Y = T0.clone(), Y0.clone()
    st, ns = df.integrate(m, T, p, Y, dt, opts)
    return T, Y, st, ns


def _same(a, b):
    return all(torch.equal(x, y) for x, y in zip(a, b))


def test_autotune_choice_and_shape_independence():
    mech = synth.h2_air_mechanism()
    m = df.Mechanism(mech)
    f = synth.field(1, mech, 12000, seed=31)
    T0, p, Y0 = _dev(f)
    Tc, Yc = T0.clone(), Y0.clone()
    best, ms = m.autotune(T0, p, Y0, f["dt"], sample=8192)
    assert torch.equal(T0, Tc) and torch.equal(Y0, Yc)  # inputs untouched
    assert best.block_threads in (32, 64, 96, 128) and best.blocks_per_sm in (0, 1, 2)
    assert best.order_by_T in (0, 1) and best.path == 1 and ms > 0
    tuned = _run(m, T0, p, Y0, f["dt"], best)
    assert int(tuned[2].abs().sum()) == 0
    # zero shape fields take the cached choice
    assert _same(tuned, _run(m, T0, p, Y0, f["dt"]))
    # the mechanism-independent kernel: explicit shapes (32/64/128 threads with a
    # compile-time stride, 96 with the run-time one) and both work orders give
    # bitwise the same cells
    gen = df.default_opts()
    gen.block_threads, gen.blocks_per_sm, gen.order_by_T, gen.jit = best.block_threads, best.blocks_per_sm, 1, 1
    ref = _run(m, T0, p, Y0, f["dt"], gen)
    for bt, bps, order in ((32, 1, 0), (64, 2, 1), (128, 0, 1), (96, 2, 0)):
        o = df.default_opts()
        o.block_threads, o.blocks_per_sm, o.order_by_T, o.jit = bt, bps, order, 1
        assert _same(ref, _run(m, T0, p, Y0, f["dt"], o)), (bt, bps, order)
    # the kernel generated for the mechanism (the default at 32 and 64 threads)
    # agrees with it to rounding, in either work order
    for bt, order in ((32, 0), (64, 1)):
        o = df.default_opts()
        o.block_threads, o.blocks_per_sm, o.order_by_T = bt, 0, order
        T, Y, st, ns = _run(m, T0, p, Y0, f["dt"], o)
        assert torch.equal(st, ref[2])
        assert (T - ref[0]).abs().max().item() <= 1e-6
        assert ((Y - ref[1]).abs() / ref[1].abs().amax(dim=0)).max().item() <= 1e-9
        assert (ns != ref[3]).float().mean().item() <= 0.01


def test_autotune_warp_path():
    mech = synth.hydrocarbon_mechanism()
    m = df.Mechanism(mech)
    f = synth.field(2, mech, 192, seed=5)
    T0, p, Y0 = _dev(f)
    best, ms = m.autotune(T0, p, Y0, f["dt"])
    assert best.path == 2 and best.block_threads in (64, 128, 256)
    ref = _run(m, T0, p, Y0, f["dt"], best)
    o = df.default_opts()
    o.block_threads = 64 if best.block_threads != 64 else 256
    assert _same(ref, _run(m, T0, p, Y0, f["dt"], o))


def test_cuda_graph_replay_of_the_step():
    mech = synth.h2_air_mechanism()
    m = df.Mechanism(mech)
    f = synth.field(1, mech, 5000, seed=41)
    T0, p, Y0 = _dev(f)
    ref = _run(m, T0, p, Y0, f["dt"])
    T, Y = T0.clone(), Y0.clone()
    st = torch.empty(T.numel(), dtype=torch.int32, device=DEV)
    ns = torch.empty_like(st)

    def step():
        T.copy_(T0)
        Y.copy_(Y0)
        df.integrate(m, T, p, Y, f["dt"], status=st, nsub=ns)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()  # allocations and one-time set-up happen outside the capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for _ in range(3):
        T.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert _same(ref, (T, Y, st, ns))
    acc, rej = m.last_stats()
    assert acc == int(ns.sum())
