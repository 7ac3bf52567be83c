"""Host logic of the multi-GPU path on CPU: two gloo ranks split one photon
budget, each traces its range (with the CPU oracle standing in for the GPU),
and the all-reduced irradiance and gradients equal the single-process run.
Integer texel sums reduce exactly; the rank loop the benchmark runs
(shard.ShardedPass: forward, in-place all-reduce of the int64 texel sums,
objective, adjoint, gradient reduction) reproduces one pass over the whole
budget bit for bit, with a stand-in tracer that keeps its sums the way the
library does."""
import multiprocessing as mp
import os
import socket

import numpy as np

import oracle
from paper_2310_02043_gb300 import scenes, shard

N_PER_RANK, HITS, SEED = 3001, 3, 5


def _setup():
    sc = scenes.cornell_box(res=8)
    L = scenes.make_lights([scenes.point_light((0.5, 0.5, 0.9), 1.0),
                            scenes.spot_light((0.3, 0.4, 0.95), 0.4, -1.3, 1.5, 0.3, 0.7)])
    w = scenes.random_weights(sc.n_texels, seed=2).astype(np.float64)
    return sc, L, w


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc, L, w = _setup()
        n_total, b, e = shard.photon_range(rank, world, N_PER_RANK)
        E = torch.from_numpy(oracle.forward(sc, L, SEED, n_total, HITS, begin=b, end=e, threads=1)["E"])
        shard.allreduce_sum(E)
        G = torch.from_numpy(oracle.adjoint(sc, L, SEED, n_total, HITS, w, begin=b, end=e, threads=1)[0])
        shard.allreduce_sum(G)
        big = torch.full((4,), (1 << 61) + rank * 12345 + 7, dtype=torch.int64)
        shard.allreduce_sum(big)
        if rank == 0:
            out.put((E.numpy(), G.numpy(), big.numpy()))
    finally:
        dist.destroy_process_group()


def _pass_setup():
    sc, L, _ = _setup()
    Lt = scenes.perturb_lights(L, seed=3, pos_sigma=0.05)
    target = oracle.forward(sc, Lt, 9, 4096, HITS, threads=1)["E"]
    return sc, L, target


def _tracer():
    from tests.oracle_tracer import OracleFixedTracer
    sc, L, target = _pass_setup()
    tr = OracleFixedTracer()
    tr.upload_scene(sc)
    tr.set_target(target)
    tr.set_lights(L)
    return tr


def _pass_worker(rank, world, port, exact, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        tr = _tracer()
        sp = shard.ShardedPass(tr, rank, world, N_PER_RANK, HITS, accumulator=torch.from_numpy(tr.q), exact=exact)
        O, g = sp.step(SEED, SEED + 1)
        out.put((rank, tr.q.copy(), O, np.array(g)))
    finally:
        dist.destroy_process_group()


def _run_ranks(target, args, world=2):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, *args, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(res, key=lambda r: r[0])


def test_sharded_pass_reproduces_one_pass_exactly():
    oracle.build()
    one = shard.ShardedPass(_tracer(), 0, 1, 2 * N_PER_RANK, HITS)
    O1, g1 = one.step(SEED, SEED + 1)
    q1 = one.tracer.q.copy()
    for rank, q, O, g in _run_ranks(_pass_worker, (True,)):
        assert np.array_equal(q, q1), rank            # int64 texel sums: exact
        assert O == O1, rank                          # the same integers give the same objective
        assert np.array_equal(g, g1), rank            # exact gradient sums: bit for bit
    # summing the ranks' doubles instead agrees to rounding
    for rank, q, O, g in _run_ranks(_pass_worker, (False,)):
        assert np.array_equal(q, q1) and O == O1
        np.testing.assert_allclose(g, g1, rtol=1e-12, atol=1e-15 * np.abs(g1).max())


def test_sharded_pass_needs_the_accumulator_for_several_ranks():
    import pytest
    with pytest.raises(ValueError):
        shard.ShardedPass(object(), 0, 2, 10, 3)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_reproduce_the_single_run():
    oracle.build()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    E, G, big = out.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sc, L, w = _setup()
    full_E = oracle.forward(sc, L, SEED, 2 * N_PER_RANK, HITS)["E"]
    full_G, _ = oracle.adjoint(sc, L, SEED, 2 * N_PER_RANK, HITS, w)
    np.testing.assert_allclose(E, full_E, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(G, full_G, rtol=1e-10, atol=1e-12 * np.abs(full_G).max())
    assert np.all(big == 2 * (1 << 61) + 12345 + 14)


def test_photon_range_covers_the_budget():
    ranges = [shard.photon_range(r, 4, 1000) for r in range(4)]
    assert all(t == 4000 for t, _, _ in ranges)
    assert [b for _, b, _ in ranges] == [0, 1000, 2000, 3000]
    assert ranges[-1][2] == 4000
