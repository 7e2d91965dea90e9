"""De-duplicating update (unit weights, global placement, one-word keys): a key
held by the block's table is counted and hashed once with its count, the rest
are hashed from per-warp queues.  A sketch is linear in the stream (Sec. 1.3),
so the counters must equal the oracle's key-by-key update exactly, whatever the
table absorbs: ragged queue drains, saturated and colliding tables, the table's
EMPTY word as a key, every block size and grid, every mode and prime."""
import numpy as np
import pytest

import datagen
import oracle
from test_gpu_parity import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2008_08654_gb300 as ms
    assert torch.cuda.is_available()
    ms.lib()
    return torch, ms


def zipf_keys(b, n, seed, ranks=1 << 20):
    z = datagen.zipf(seed, 1.1, ranks, n)
    if b == 31:
        return (z & np.uint64(0x7FFFFFFF)).astype(np.uint32)
    return z


def sketch_and_check(torch, ms, b, c, t, m, k, mode, keys, seed, **launch):
    sk = ms.Sketch(t=t, m=m, k=k, b=b, c=c, seed=seed, mode=mode)
    sk.set_launch(place=launch.pop("place", 2), **launch)
    sk.update(to_dev(torch, keys))
    ll = sk.last_launch()
    C = sk.counters().cpu().numpy()
    want = oracle.cs_update(b, c, k, t, sk.m, mode, oracle.sketch_coeffs(b, c, k, t, mode, seed), keys)
    assert np.array_equal(C, want), "counters differ (%d cells)" % int((C != want).sum())
    return sk, ll, want


# sizes around one warp chunk (128 keys), one block chunk and the table size
SIZES = [1, 3, 127, 128, 129, 255, 2047, 2049, 4097, 65537, 300007]


@pytest.mark.parametrize("n", SIZES)
def test_ragged_sizes(env, n):
    torch, ms = env
    keys = zipf_keys(61, n, 11 + n)
    _, ll, _ = sketch_and_check(torch, ms, 61, 1, 7, 1 << 16, 4, 0, keys, 3)
    assert ll["place"] == 2 and ll["replicas"] > 0


@pytest.mark.parametrize("threads,blocks", [(32, 0), (32, 1), (64, 3), (256, 0), (512, 0),
                                            (512, 1), (128, 7)])
def test_block_shapes(env, threads, blocks):
    """Queue length and table drain depend on the warps per block."""
    torch, ms = env
    keys = zipf_keys(61, 100003, 5)
    _, ll, _ = sketch_and_check(torch, ms, 61, 1, 7, 1 << 15, 4, 0, keys, 9,
                                threads=threads, blocks=blocks)
    assert ll["threads"] == threads and (blocks == 0 or ll["blocks"] == blocks)


def test_saturated_table_and_collisions(env):
    """Many more distinct repeated keys than table slots (every slot taken
    early by a cold key), plus the table's EMPTY word (all ones) repeated."""
    torch, ms = env
    n = 400009
    rng = np.random.default_rng(7)
    warm = datagen.u64_below(21, 0, 20000)           # 20000 keys, each ~10 times
    keys = warm[rng.integers(0, warm.size, n)]
    keys[rng.random(n) < 0.05] = np.uint64((1 << 64) - 1)
    keys[:64] = np.uint64((1 << 64) - 1)
    for blocks in (0, 1):
        for aggregate in (2, 3):
            sketch_and_check(torch, ms, 61, 1, 5, 1 << 15, 4, 0, keys, 13, blocks=blocks,
                             aggregate=aggregate)


def test_all_equal_and_all_distinct(env):
    torch, ms = env
    same = np.full(70001, 12345678901, dtype=np.uint64)
    sketch_and_check(torch, ms, 61, 1, 7, 1 << 15, 4, 0, same, 2)
    distinct = datagen.u64_below(8, 0, 70001)
    sketch_and_check(torch, ms, 61, 1, 7, 1 << 15, 4, 0, distinct, 2)


CASES = [
    # b, c, t, m, k, mode, strategy
    (61, 1, 7, 1 << 16, 4, 0, 1),                      # power sum, two-for-one
    (61, 1, 7, 1 << 16, 4, 0, 0),                      # Horner
    (61, 1, 5, 1 << 15, 4, oracle.TWO_POLY, 1),        # two polynomials
    (61, 1, 5, 50000, 4, oracle.ANY_R, 1),             # any m (Algorithm Mersenne-arb-r)
    # the remaining compile-time shapes of the 2^61-1 second-level drain
    (61, 1, 5, 1 << 14, 4, 0, 1),
    (61, 1, 5, 30000, 4, oracle.ANY_R | oracle.TWO_POLY, 1),
    (61, 1, 7, 1 << 15, 4, oracle.TWO_POLY, 1),
    (61, 1, 7, 40000, 4, oracle.ANY_R, 1),
    (61, 1, 7, 30000, 4, oracle.ANY_R | oracle.TWO_POLY, 1),
    (61, 1, 3, 1 << 17, 2, 0, -1),                     # generic kernel (runtime t, k)
    (61, 1, 9, 1 << 15, 5, oracle.TWO_POLY, -1),       # generic, two polynomials
    (64, 59, 7, 1 << 15, 4, 0, -1),                    # 2^64 - 59
    (64, 59, 5, 40000, 4, oracle.ANY_R | oracle.TWO_POLY, -1),
    (31, 1, 7, 1 << 15, 4, 0, -1),                     # 32-bit keys
    (31, 1, 3, 1 << 16, 2, oracle.TWO_POLY, -1),
]


@pytest.mark.parametrize("aggregate", [2, 3])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(map(str, c)))
def test_modes_and_primes(env, case, aggregate):
    """aggregate 2: the block's table; 3: and the second-level table in global
    memory (forced here on a short stream)."""
    torch, ms = env
    b, c, t, m, k, mode, strategy = case
    keys = zipf_keys(b, 150001, 40 + t + k)
    sk, ll, want = sketch_and_check(torch, ms, b, c, t, m, k, mode, keys, 17 + t, strategy=strategy,
                                    aggregate=aggregate)
    assert sk.f2() == oracle.f2_estimate(want)


@pytest.mark.parametrize("aggregate", [2, 3])
def test_repeated_updates_accumulate(env, aggregate):
    """Three updates into one sketch: each launch drains its own tables (the
    second-level table is empty again after each)."""
    torch, ms = env
    keys = zipf_keys(61, 200003, 77)
    sk = ms.Sketch(t=7, m=1 << 16, k=4, seed=4)
    sk.set_launch(aggregate=aggregate)
    for lo, hi in ((0, 123457), (123457, 150001), (150001, 200003)):
        sk.update(to_dev(torch, keys[lo:hi]))
    C = sk.counters().cpu().numpy()
    want = oracle.cs_update(61, 1, 4, 7, 1 << 16, 0, oracle.sketch_coeffs(61, 1, 4, 7, 0, 4), keys)
    assert np.array_equal(C, want)


def test_second_level_table_saturated(env):
    """A default update of more than 2^22 keys (the second-level table on):
    5 million distinct keys each seen about twice, so the 2^21-slot table
    fills early and most of its lookups find another key; the table's EMPTY
    word (all ones) repeated among them.  Also with the statistics hook: the
    entries hashed stay below the keys."""
    import os
    torch, ms = env
    n = (1 << 23) + 12345
    rng = np.random.default_rng(11)
    pool = datagen.u64_below(41, 0, 5_000_000)
    keys = pool[rng.integers(0, pool.size, n)]
    keys[rng.random(n) < 0.01] = np.uint64((1 << 64) - 1)
    sk = ms.Sketch(t=7, m=1 << 16, k=4, seed=21)
    hashed = torch.zeros(1, dtype=torch.int64, device="cuda")
    sk.set_stats(hashed)
    sk.update(to_dev(torch, keys))
    torch.cuda.synchronize()
    want = oracle.cs_update(61, 1, 4, 7, 1 << 16, 0, oracle.sketch_coeffs(61, 1, 4, 7, 0, 21), keys,
                            nthreads=os.cpu_count() or 1)
    assert np.array_equal(sk.counters().cpu().numpy(), want)
    assert 0 < int(hashed.item()) < n


@pytest.mark.parametrize("aggregate", [0, 1, 2, 3])
def test_aggregation_levels_agree(env, aggregate):
    """Off, warp merging, and the de-duplication table: one result."""
    torch, ms = env
    keys = zipf_keys(61, 250007, 3)
    sketch_and_check(torch, ms, 61, 1, 7, 1 << 16, 4, 0, keys, 6, aggregate=aggregate)


def test_direct_int64_placement(env):
    """Place 3 (int64 atomics, no replicas) also takes the table."""
    torch, ms = env
    keys = zipf_keys(61, 100003, 8)
    _, ll, _ = sketch_and_check(torch, ms, 61, 1, 5, 1 << 14, 4, 0, keys, 8, place=3)
    assert ll["place"] == 3


@pytest.mark.parametrize("threads,blocks", [(32, 1), (64, 2), (512, 3)])
def test_table_switches_off_and_stays_exact(env, threads, blocks):
    """A warp whose table absorbs under 1/8 of the keys of its 17th to 32nd
    chunks hashes the rest of its keys directly; what the queue and table already hold is still
    drained.  Streams: all distinct; distinct then heavy repeats; heavy
    repeats then distinct."""
    torch, ms = env
    chunk = 128 * (threads // 32) * blocks       # keys one round of the grid takes
    n = chunk * 80 + 77
    distinct = datagen.u64_below(31, 0, n)
    hot = datagen.u64_below(32, 0, 50)
    rng = np.random.default_rng(5)
    repeats = hot[rng.integers(0, hot.size, n)]
    cut = chunk * 40
    streams = [distinct, np.concatenate([distinct[:cut], repeats[cut:]]),
               np.concatenate([repeats[:cut], distinct[cut:]])]
    for keys in streams:
        sketch_and_check(torch, ms, 61, 1, 7, 1 << 15, 4, 0, keys, 12, threads=threads, blocks=blocks)
