"""Multi-rank host logic on CPU (gloo, world size 2): the one exchange step of
the sharded Count Sketch and the max-over-ranks timing reduction."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import datagen
import oracle
from paper_2008_08654_gb300 import dist as msd


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n, t, m, seed, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        keys = datagen.u64_below(seed, (1 << 61) - 1, n)
        w = datagen.i32_range(seed, -100, 100, n)
        lo, hi = msd.shard_range(n, rank, world)
        coeffs = oracle.sketch_coeffs(61, 1, 4, t, 0, seed)
        part = oracle.cs_update(61, 1, 4, t, m, 0, coeffs, keys[lo:hi], w[lo:hi])
        ct = torch.from_numpy(part.copy())
        msd.merge_counters_(ct)
        slowest = msd.max_over_ranks(1.5 + rank)
        q.put((rank, ct.numpy().copy(), slowest))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_sharded_sketch_merges_to_the_whole_stream(world):
    n, t, m, seed = 30011, 5, 256, 12
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, t, m, seed, q))
             for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    keys = datagen.u64_below(seed, (1 << 61) - 1, n)
    w = datagen.i32_range(seed, -100, 100, n)
    want = oracle.cs_update(61, 1, 4, t, m, 0, oracle.sketch_coeffs(61, 1, 4, t, 0, seed), keys, w)
    for rank, counters, slowest in results:
        assert np.array_equal(counters, want)
        assert slowest == 1.5 + (world - 1)


def _lib_worker(rank, world, port, n, t, m, seed, q):
    """One rank on the library: its shard through cs_update on cuda:0, the
    partial sketch checkpointed (cs_export) and restored (cs_import), its
    counters copied to the host and merged with the others by gloo."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_2008_08654_gb300 as ms
        torch.cuda.set_device(0)
        keys = datagen.u64_below(seed, (1 << 61) - 1, n)
        w = datagen.i32_range(seed, -100, 100, n)
        lo, hi = msd.shard_range(n, rank, world)
        sk = ms.Sketch(t=t, m=m, k=4, seed=seed)
        sk.update(torch.from_numpy(keys[lo:hi].view(np.int64)).cuda(),
                  torch.from_numpy(w[lo:hi]).cuda())
        restored = ms.Sketch.import_(sk.export())
        ct = restored.counters().cpu().clone()
        msd.merge_counters_(ct)
        # the merged counters back into a sketch of this rank: its F2 is the
        # whole stream's
        restored.counters().copy_(ct.cuda())
        q.put((rank, ct.numpy().copy(), restored.f2()))
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
def test_library_partial_sketches_merge_to_the_whole_stream():
    """Two gloo ranks (both on the one GPU; their kernels never wait on each
    other): partial sketches made by the library, exported and imported, merged
    by one int64 sum, equal the oracle's sketch of the whole stream."""
    world, n, t, m, seed = 2, 200003, 5, 1024, 21
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_lib_worker, args=(r, world, port, n, t, m, seed, q))
             for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    keys = datagen.u64_below(seed, (1 << 61) - 1, n)
    w = datagen.i32_range(seed, -100, 100, n)
    want = oracle.cs_update(61, 1, 4, t, m, 0, oracle.sketch_coeffs(61, 1, 4, t, 0, seed), keys, w)
    for rank, counters, f2 in results:
        assert np.array_equal(counters, want)
        assert f2 == oracle.f2_estimate(want)


def test_shard_ranges_cover_the_stream():
    for n in (0, 1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            got = [msd.shard_range(n, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == n
            for (a, b), (c, d) in zip(got, got[1:]):
                assert b == c and a <= b


def test_single_process_merge_is_identity():
    c = torch.arange(10, dtype=torch.int64)
    assert torch.equal(msd.merge_counters_(c.clone()), c)
    with pytest.raises(TypeError):
        msd.merge_counters_(torch.zeros(3, dtype=torch.int32))
