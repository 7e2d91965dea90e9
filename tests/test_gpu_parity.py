"""GPU parity: every kernel, called through the C ABI, against the CPU oracle.

All results are integers, so every comparison is exact (bit for bit): hash
values, quotients and remainders, every int64 counter, every 128-bit row sum
and the F2 median.  Sizes span several blocks and end in a ragged tail.
"""
import os

import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu

PRIMES = [(31, 1), (61, 1), (89, 1), (64, 59)]
NTHREADS = max(1, min(32, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2008_08654_gb300 as ms
    assert torch.cuda.is_available()
    ms.lib()
    return torch, ms


def to_dev(torch, a: np.ndarray):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    elif a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def make_keys(b, c, n, seed, edges=True):
    """Keys of the prime's key type, with edge values at the front."""
    p = (1 << b) - c
    if b == 31:
        k = datagen.u32_below(seed, 0, n)
        e = [0, 1, p - 1, p, p + 1 if p + 1 < 2 ** 32 else 0, 2 ** 32 - 1, 2 ** 31]
    elif b == 89:
        k = datagen.u128_bits(seed, 128, n, stream=datagen.STREAM_KEYS)
        e = [0, 1, p - 1, p, p + 1, 2 ** 128 - 1, 2 ** 89, 2 ** 64 - 1, 2 ** 64]
        if edges:
            m = min(len(e), n)
            k[:m] = oracle.from_ints(e[:m])
        return k
    else:
        k = datagen.u64_below(seed, 0, n)
        e = [0, 1, p - 1, p, p + 1, 2 ** 64 - 1, 2 ** 63, 2 ** 61]
    if edges:
        m = min(len(e), n)
        k[:m] = e[:m]
    return k


def hash_to_np(torch, t, b):
    a = t.cpu().numpy()
    if b == 31:
        return a.view(np.uint32).astype(np.uint64)
    if b == 89:
        return a.view(np.uint64).reshape(-1, 2)
    return a.view(np.uint64)


# ------------------------------------------------------------------ hashing

@pytest.mark.parametrize("b,c", PRIMES)
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8])
def test_hash_eval(env, b, c, k):
    torch, ms = env
    n = 40009
    keys = make_keys(b, c, n, 100 + k)
    h = ms.Hash(k=k, b=b, c=c, seed=7 * k + b)
    got = hash_to_np(torch, h.eval(to_dev(torch, keys)), b)
    want = oracle.hash_eval(b, c, oracle.from_ints(h.coeffs()), keys)
    if b == 89:
        assert np.array_equal(got, want)
    else:
        assert not want[:, 1].any()
        assert np.array_equal(got, want[:, 0])


@pytest.mark.parametrize("b,c", PRIMES)
def test_hash_eval_unaligned_and_tiny(env, b, c):
    """Slices that break 16-byte alignment take the scalar path; n = 1..5."""
    torch, ms = env
    keys = make_keys(b, c, 1031, 5)
    h = ms.Hash(k=4, b=b, c=c, seed=3)
    dk = to_dev(torch, keys)
    coeffs = oracle.from_ints(h.coeffs())
    for lo, hi in [(1, 1031), (3, 1030), (0, 1), (1, 2), (2, 5), (0, 5)]:
        got = hash_to_np(torch, h.eval(dk[lo:hi]), b)
        want = oracle.hash_eval(b, c, coeffs, keys[lo:hi])
        want = want if b == 89 else want[:, 0]
        assert np.array_equal(got, want), (lo, hi)
    assert h.eval(dk[:0]).numel() == 0


# ------------------------------------------------------------------ division

@pytest.mark.parametrize("b,c", PRIMES)
def test_div_mod(env, b, c):
    torch, ms = env
    p = (1 << b) - c
    edges = [0, 1, p - 1, p, p + 1, 2 * p - 1, 2 * p, p * p - 1, p * p, 2 ** 128 - 1, 2 ** 128 - 2,
             2 ** 127, 2 ** 64 - 1, 2 ** 64, ((1 << 64) - 1) * p]
    edges = [v for v in edges if v < 2 ** 128]
    if 2 * b < 128:
        edges += [2 ** (2 * b) - 1, 2 ** (2 * b) - 2, 2 ** (2 * b)]
    vals = [oracle.from_ints(edges)]
    for bits in (2 * b, 122, 128, 64, 17):
        vals.append(datagen.u128_bits(bits * 31 + b, min(bits, 128), 30011))
    v = np.concatenate(vals)
    qw, rw = oracle.divmod_(b, c, v)
    q, r = ms.div(b, c, to_dev(torch, v))
    q = q.cpu().numpy().view(np.uint64)
    r = r.cpu().numpy().view(np.uint64)
    assert np.array_equal(q, qw)
    if b == 89:
        assert np.array_equal(r, rw)
    else:
        assert np.array_equal(r, rw[:, 0])
    r2 = ms.mod(b, c, to_dev(torch, v)).cpu().numpy().view(np.uint64)
    assert np.array_equal(r2, r)


# ------------------------------------------------------------------ count sketch

def run_sketch(torch, ms, b, c, t, m, k, mode, keys, w, seed, place=-1, strategy=-1, cluster=0,
               threads=0, blocks=0):
    sk = ms.Sketch(t=t, m=m, k=k, b=b, c=c, seed=seed, mode=mode)
    sk.set_launch(place=place, strategy=strategy, threads=threads, blocks=blocks, cluster=cluster)
    sk.update(to_dev(torch, keys), None if w is None else to_dev(torch, w))
    rows = torch.empty((t, 2), dtype=torch.int64, device="cuda")
    f2 = sk.estimate_f2(rows=rows)
    torch.cuda.synchronize()
    return sk, sk.counters().cpu().numpy(), ms.u128_to_int(f2.cpu()), \
        [ms.u128_to_int(r) for r in rows.cpu()]


def check_sketch(sk, C, f2, rows, b, c, k, mode, keys, w, seed, nthreads=1):
    coeffs = oracle.sketch_coeffs(b, c, k, sk.t, mode, seed)
    assert sk.coeffs() == oracle.to_ints(coeffs)
    want = oracle.cs_update(b, c, k, sk.t, sk.m, mode, coeffs, keys, w, nthreads=nthreads)
    assert np.array_equal(C, want), "counters differ (%d cells)" % int((C != want).sum())
    assert rows == oracle.row_sumsq(want)
    assert f2 == oracle.f2_estimate(want)
    return want


CASES = [
    # b, c, t, m, k, mode, place, strategy, weights
    (61, 1, 5, 1024, 4, 0, -1, -1, "pm100"),    # config-1 shape, specialized, auto (smem)
    (61, 1, 5, 1024, 4, 0, 0, 0, "pm100"),      # Horner
    (61, 1, 5, 1024, 4, 0, 0, 1, "unit"),       # power sum (lean tile kernel)
    (61, 1, 5, 1024, 4, 0, 0, 2, "pm100"),      # power sum in the general kernel
    (61, 1, 7, 4096, 4, 1, 0, 2, "unit"),       # two-poly, general kernel
    (61, 1, 7, 4096, 4, 1, 0, 1, "pm100"),      # two-poly, lean kernel, 112 KiB tile
    (61, 1, 5, 2, 4, 0, 0, 1, "pm100"),         # lean kernel, m = 2
    (61, 1, 5, 4096, 4, 0, 0, 1, "unit"),       # lean kernel, unit weights, 80 KiB tile
    (61, 1, 5, 1024, 4, 1, 0, 1, "pm100"),      # two-poly, power sum
    (61, 1, 5, 1024, 4, 1, 0, 0, "pm100"),      # two-poly, Horner
    (61, 1, 7, 4096, 4, 0, -1, -1, "unit"),
    (61, 1, 7, 8192, 4, 1, 1, 1, "unit"),       # DSMEM, auto cluster
    (61, 1, 5, 4096, 4, 0, 1, 0, "pm100"),      # DSMEM
    (61, 1, 5, 256, 4, 0, 3, 1, "pm100"),       # int64 global atomics
    (61, 1, 7, 65536, 4, 0, 2, 1, "pm100"),     # int32 global replicas (large sketch)
    (61, 1, 7, 65536, 4, 1, 2, 0, "unit"),      # replicas, two-poly, Horner
    (61, 1, 3, 1 << 20, 2, 0, -1, -1, "pm100"), # generic kernel, replicas
    (61, 1, 1, 1 << 24, 4, 0, -1, -1, "unit"),  # m = 2^24 (maximum)
    (61, 1, 3, 64, 2, 0, -1, -1, "pm100"),      # generic kernel
    (61, 1, 3, 64, 2, 1, 1, -1, "pm100"),       # generic, DSMEM
    (61, 1, 1, 2, 8, 0, -1, -1, "pm100"),       # m = 2, k = 8
    (61, 1, 15, 128, 1, 0, -1, -1, "pm100"),    # k = 1: constant hash, t = 15
    (31, 1, 5, 4096, 4, 0, -1, -1, "pm100"),
    (31, 1, 5, 1024, 4, 1, 3, -1, "pm100"),
    (31, 1, 5, 1 << 16, 4, 0, 2, -1, "pm100"),
    (31, 1, 3, 32, 3, 0, 1, -1, "unit"),
    (89, 1, 5, 4096, 4, 0, -1, -1, "pm100"),
    (89, 1, 5, 1024, 4, 1, 1, -1, "unit"),
    (89, 1, 3, 16, 5, 0, 3, -1, "pm100"),
    (89, 1, 5, 1 << 15, 4, 1, 2, -1, "pm100"),
    (64, 59, 5, 4096, 4, 0, -1, -1, "pm100"),
    (64, 59, 7, 1024, 4, 1, 1, -1, "unit"),
    (64, 59, 1, 64, 2, 0, 3, -1, "pm100"),
    (64, 59, 7, 1 << 16, 4, 0, 2, -1, "unit"),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(map(str, c)))
def test_cs_update_parity(env, case):
    torch, ms = env
    b, c, t, m, k, mode, place, strategy, wk = case
    n = 65543  # several blocks of 1024 keys, ragged tail
    keys = make_keys(b, c, n, 11 + t + m)
    w = None if wk == "unit" else datagen.i32_range(13 + m, -100, 100, n)
    seed = 1000 + t * 31 + k
    sk, C, f2, rows = run_sketch(torch, ms, b, c, t, m, k, mode, keys, w, seed, place, strategy)
    ll = sk.last_launch()
    small = t * m * 4 <= 112 * 1024  # small sketches own no replicas: place 2 runs as 3
    if place >= 0 and ll["place"] != place and not (place == 2 and small and ll["place"] == 3):
        pytest.fail("launch fell back from place %d to %s" % (place, ll))
    check_sketch(sk, C, f2, rows, b, c, k, mode, keys, w, seed)


@pytest.mark.parametrize("cluster", [2, 4, 8, 16])
def test_dsmem_cluster_sizes(env, cluster):
    torch, ms = env
    n, t, m = 50021, 5, 2048
    keys = make_keys(61, 1, n, 77)
    w = datagen.i32_range(78, -100, 100, n)
    sk, C, f2, rows = run_sketch(torch, ms, 61, 1, t, m, 4, 0, keys, w, 5, place=1, strategy=1,
                                 cluster=cluster)
    assert sk.last_launch()["cluster"] == cluster
    check_sketch(sk, C, f2, rows, 61, 1, 4, 0, keys, w, 5)


@pytest.mark.parametrize("threads,blocks", [(32, 1), (64, 3), (512, 7), (256, 1000)])
def test_launch_shapes(env, threads, blocks):
    torch, ms = env
    n, t, m = 30011, 5, 1024
    keys = make_keys(61, 1, n, 91)
    w = datagen.i32_range(92, -100, 100, n)
    sk, C, f2, rows = run_sketch(torch, ms, 61, 1, t, m, 4, 0, keys, w, 9, place=0, strategy=1,
                                 threads=threads, blocks=blocks)
    check_sketch(sk, C, f2, rows, 61, 1, 4, 0, keys, w, 9)


def test_extreme_weights_take_exact_path(env):
    """Weights near +-2^31 on a stream long enough that an int32 tile counter
    could overflow: they must be routed to the int64 counters and stay exact."""
    torch, ms = env
    n, t, m = 200003, 5, 64
    keys = make_keys(61, 1, n, 41)
    w = datagen.i32_range(42, -2 ** 31, 2 ** 31 - 1, n)
    w[:6] = [-2 ** 31, 2 ** 31 - 1, -2 ** 31, -2 ** 31, 2 ** 31 - 1, 0]
    for place in (0, 1, 2, 3):
        sk, C, f2, rows = run_sketch(torch, ms, 61, 1, t, m, 4, 0, keys, w, 3, place=place,
                                     strategy=1, blocks=4)
        check_sketch(sk, C, f2, rows, 61, 1, 4, 0, keys, w, 3)
    # a sketch with replicas: int32 replica counters must not overflow either
    sk, C, f2, rows = run_sketch(torch, ms, 61, 1, 5, 1 << 15, 4, 0, keys, w, 3, place=2,
                                 strategy=1, blocks=16)
    assert sk.last_launch()["place"] == 2
    check_sketch(sk, C, f2, rows, 61, 1, 4, 0, keys, w, 3)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 7, 1023, 1024, 1025])
def test_tiny_streams(env, n):
    torch, ms = env
    keys = make_keys(61, 1, max(n, 1), 5 + n)[:n]
    w = datagen.i32_range(6 + n, -100, 100, max(n, 1))[:n]
    sk, C, f2, rows = run_sketch(torch, ms, 61, 1, 5, 1024, 4, 0, keys, w, 2)
    check_sketch(sk, C, f2, rows, 61, 1, 4, 0, keys, w, 2)


def test_unaligned_stream(env):
    torch, ms = env
    n = 10007
    keys = make_keys(61, 1, n, 8)
    w = datagen.i32_range(9, -100, 100, n)
    sk = ms.Sketch(t=5, m=1024, k=4, seed=4)
    dk, dw = to_dev(torch, keys), to_dev(torch, w)
    sk.update(dk[1:], dw[1:])
    sk.update(dk[:1], dw[:1])
    C = sk.counters().cpu().numpy()
    coeffs = oracle.sketch_coeffs(61, 1, 4, 5, 0, 4)
    assert np.array_equal(C, oracle.cs_update(61, 1, 4, 5, 1024, 0, coeffs, keys, w))


def test_accumulate_reset_merge_export(env):
    torch, ms = env
    n, t, m, k, seed = 30001, 5, 512, 4, 17
    keys = make_keys(61, 1, n, 12)
    w = datagen.i32_range(13, -100, 100, n)
    dk, dw = to_dev(torch, keys), to_dev(torch, w)
    a = ms.Sketch(t=t, m=m, k=k, seed=seed)
    a.update(dk[:12345], dw[:12345])
    a.update(dk[12345:], dw[12345:])
    coeffs = oracle.sketch_coeffs(61, 1, k, t, 0, seed)
    want = oracle.cs_update(61, 1, k, t, m, 0, coeffs, keys, w)
    assert np.array_equal(a.counters().cpu().numpy(), want)
    # merge = linearity
    b1 = ms.Sketch(t=t, m=m, k=k, seed=seed)
    b2 = ms.Sketch(t=t, m=m, k=k, seed=seed)
    b1.update(dk[:777], dw[:777])
    b2.update(dk[777:], dw[777:])
    b1.merge(b2)
    assert np.array_equal(b1.counters().cpu().numpy(), want)
    with pytest.raises(ms.MSError):
        b1.merge(ms.Sketch(t=t, m=m, k=k, seed=seed + 1))
    # checkpoint round trip
    blob = a.export()
    r = ms.Sketch.import_(blob)
    assert (r.t, r.m, r.k, r.b, r.c, r.mode) == (t, m, k, 61, 1, 0)
    assert r.coeffs() == a.coeffs()
    assert np.array_equal(r.counters().cpu().numpy(), want)
    assert r.f2() == oracle.f2_estimate(want)
    # resume after import: keeps sketching exactly
    r.update(dk[:100], dw[:100])
    want2 = oracle.cs_update(61, 1, k, t, m, 0, coeffs, keys[:100], w[:100], counters=want.copy())
    assert np.array_equal(r.counters().cpu().numpy(), want2)
    a.reset()
    torch.cuda.synchronize()
    assert not a.counters().cpu().numpy().any()
    assert a.f2() == 0


@pytest.mark.parametrize("b,c,mode", [(61, 1, 0), (61, 1, 1), (31, 1, 0), (89, 1, 1), (64, 59, 0)])
def test_point_query(env, b, c, mode):
    torch, ms = env
    n, t, m, k, seed = 20011, 5, 4096, 4, 23
    keys = datagen.zipf(31, 1.1, 1 << 20, n)  # heavy keys repeat
    if b == 31:
        keys = (keys & 0xFFFFFFFF).astype(np.uint32)
    elif b == 89:
        keys = np.stack([keys, keys >> np.uint64(7)], axis=1).astype(np.uint64)
    sk = ms.Sketch(t=t, m=m, k=k, b=b, c=c, seed=seed, mode=mode)
    sk.update(to_dev(torch, keys))
    q = keys[:999]
    got = sk.point_query(to_dev(torch, q)).cpu().numpy()
    coeffs = oracle.sketch_coeffs(b, c, k, t, mode, seed)
    C = oracle.cs_update(b, c, k, t, m, mode, coeffs, keys)
    assert np.array_equal(got, oracle.point_query(b, c, k, mode, coeffs, C, q))


@pytest.mark.parametrize("t,k,mode", [(7, 4, 0), (7, 4, 1), (5, 4, 1), (3, 4, 0), (5, 2, 0)])
def test_point_query_shapes_and_edge_keys(env, t, k, mode):
    """2^61-1 point queries: the signed-digit kernel (k = 4, t = 5 or 7) and the
    generic one (other t and k), with keys at and above p (the hash depends on
    x mod p) among ragged numbers of queries."""
    torch, ms = env
    n, m, seed = 30011, 1 << 12, 41 + t + k
    keys = datagen.zipf(37 + t, 1.1, 1 << 20, n)
    p = (1 << 61) - 1
    edge = np.array([0, 1, p - 1, p, p + 1, (1 << 64) - 1, (1 << 63) + 5], dtype=np.uint64)
    keys = np.concatenate([keys, edge, edge])
    sk = ms.Sketch(t=t, m=m, k=k, seed=seed, mode=mode)
    sk.update(to_dev(torch, keys))
    coeffs = oracle.sketch_coeffs(61, 1, k, t, mode, seed)
    C = oracle.cs_update(61, 1, k, t, m, mode, coeffs, keys)
    for q in (np.concatenate([edge, keys[:1000]]), keys[:1], keys[-3:]):
        got = sk.point_query(to_dev(torch, q)).cpu().numpy()
        assert np.array_equal(got, oracle.point_query(61, 1, k, mode, coeffs, C, q))


def test_many_sketches_same_stream_differ_only_by_seed(env):
    torch, ms = env
    keys = make_keys(61, 1, 5000, 1)
    dk = to_dev(torch, keys)
    vals = set()
    for seed in range(4):
        sk = ms.Sketch(t=5, m=1024, seed=seed)
        sk.update(dk)
        vals.add(sk.f2())
    assert len(vals) > 1


@pytest.mark.parametrize("place,replicas,aggregate", [(2, 1, 1), (2, 4, 0), (2, 32, 1), (3, 0, 1),
                                                      (2, 16, 1), (2, 32, 2), (3, 0, 2), (2, 1, 2)])
@pytest.mark.parametrize("b,c", [(61, 1), (31, 1), (89, 1)])
def test_global_replicas_and_warp_aggregation(env, place, replicas, aggregate, b, c):
    """Zipf keys (many equal keys per warp), unit weights, a sketch too large for
    shared memory: global replicas and warp aggregation must stay exact."""
    torch, ms = env
    n, t, m, k, seed = 100003, 7, 1 << 15, 4, 31
    z = datagen.zipf(5, 1.1, 1 << 20, n)
    if b == 31:
        keys = (z & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    elif b == 89:
        keys = np.stack([z, z ^ np.uint64(0x5555)], axis=1).astype(np.uint64)
    else:
        keys = z
    sk = ms.Sketch(t=t, m=m, k=k, b=b, c=c, seed=seed)
    sk.set_launch(place=place, replicas=replicas, aggregate=aggregate)
    sk.update(to_dev(torch, keys))
    ll = sk.last_launch()
    assert ll["place"] == place and (place == 3 or ll["replicas"] == replicas), ll
    C = sk.counters().cpu().numpy()
    coeffs = oracle.sketch_coeffs(b, c, k, t, 0, seed)
    want = oracle.cs_update(b, c, k, t, m, 0, coeffs, keys)
    assert np.array_equal(C, want)
    assert sk.f2() == oracle.f2_estimate(want)


@pytest.mark.parametrize("b,c", [(61, 1), (64, 59), (31, 1)])
def test_hot_key_table_with_sentinel_and_collisions(env, b, c):
    """Unit weights through the per-block hot-key table: a few very hot keys,
    the table's EMPTY value itself (all ones) as a hot key, and many cold keys
    that collide in the table; counters must be exact."""
    torch, ms = env
    n = 300007
    rng = np.random.default_rng(b)
    if b == 31:
        cold = datagen.u32_below(3, 0, n)
        hot = np.array([0xFFFFFFFF, 1, 2, 7, 1 << 31], dtype=np.uint32)
    else:
        cold = datagen.u64_below(3, 0, n)
        hot = np.array([(1 << 64) - 1, 1, 2, 7, 1 << 63], dtype=np.uint64)
    pick = rng.random(n) < 0.4
    keys = cold.copy()
    keys[pick] = hot[rng.integers(0, len(hot), int(pick.sum()))]
    for blocks in (0, 3):
        sk = ms.Sketch(t=7, m=1 << 15, k=4, b=b, c=c, seed=5)
        sk.set_launch(place=2, aggregate=2, blocks=blocks)
        sk.update(to_dev(torch, keys))
        C = sk.counters().cpu().numpy()
        want = oracle.cs_update(b, c, 4, 7, 1 << 15, 0, oracle.sketch_coeffs(b, c, 4, 7, 0, 5), keys)
        assert np.array_equal(C, want)
