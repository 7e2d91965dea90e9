"""Batched updates (include/ms_batch.h): one persistent, graph-captured launch
over many independent sketches must equal the oracle sketch by sketch."""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2008_08654_gb300 as ms
    ms.lib()
    return torch, ms


def _dev(torch, a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    elif a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def _jobs(torch, ms, nsk, seed, b=61, c=1, k=4, mode=0, ts=(3, 5), ms_=(256, 1024, 4096, 8192),
          nmax=200000):
    rng = np.random.default_rng(seed)
    jobs, host = [], []
    p = (1 << b) - c
    for i in range(nsk):
        t = int(rng.choice(ts))
        m = int(rng.choice(ms_))
        n = int(10 ** rng.uniform(0, np.log10(nmax)))
        if i == 0 or i == nsk // 2:
            n = 0  # empty jobs (the plan orders jobs by length, so these move to its end)
        s = seed * 1000 + i
        if b == 31:
            keys = datagen.u32_below(s, 0, n)
        elif b == 89:
            keys = datagen.u128_bits(s, 100, n)
        else:
            keys = datagen.u64_below(s, p, n)
        w = None if i % 3 == 0 else datagen.i32_range(s, -100, 100, n)
        sk = ms.Sketch(t=t, m=m, k=k, b=b, c=c, seed=s, mode=mode)
        jobs.append((sk, _dev(torch, keys), None if w is None else _dev(torch, w)))
        host.append((sk, keys, w, s))
    return jobs, host


def _check(host, b=61, c=1, k=4, mode=0, times=1, extra=None):
    for idx, (sk, keys, w, s) in enumerate(host):
        coeffs = oracle.sketch_coeffs(b, c, k, sk.t, mode, s)
        want = np.zeros((sk.t, sk.m), dtype=np.int64)
        for _ in range(times):
            want = oracle.cs_update(b, c, k, sk.t, sk.m, mode, coeffs, keys, w, counters=want)
        if extra and idx in extra:
            ek, ew = extra[idx]
            want = oracle.cs_update(b, c, k, sk.t, sk.m, mode, coeffs, ek, ew, counters=want)
        got = sk.counters().cpu().numpy()
        assert np.array_equal(got, want), "sketch %d (t=%d m=%d n=%d)" % (idx, sk.t, sk.m,
                                                                         len(keys))


@pytest.mark.parametrize("tuning", [None,
                                    {"threads": 256, "chunk_keys": 1 << 12, "smem_min_ratio": 1},
                                    {"threads": 128, "chunk_keys": 1 << 14, "smem_min_ratio": 1000,
                                     "rows_per_item": 1, "strategy": 0},
                                    {"threads": 512, "chunk_keys": 1 << 10, "smem_min_ratio": 0,
                                     "rows_per_item": 2, "blocks_per_sm": 1},
                                    {"threads": 1024, "chunk_keys": 1 << 16, "smem_min_ratio": 2}])
def test_batched_matches_oracle(env, tuning):
    torch, ms = env
    jobs, host = _jobs(torch, ms, 40, 5)
    plan = ms.Batch(jobs, tuning)
    info = plan.info()
    assert info["total_keys"] == sum(len(h[1]) for h in host)
    plan.launch()
    torch.cuda.synchronize()
    _check(host)
    # a second replay adds the same updates again; a direct launch a third time
    plan.launch()
    plan.launch_direct()
    torch.cuda.synchronize()
    _check(host, times=3)


def test_batched_two_poly_and_shared_sketch(env):
    torch, ms = env
    jobs, host = _jobs(torch, ms, 12, 9, mode=1)
    # two more jobs on sketch 3
    sk3, k3, w3, s3 = host[3]
    extra_keys = datagen.u64_below(77, (1 << 61) - 1, 5000)
    extra_w = datagen.i32_range(77, -100, 100, 5000)
    jobs.append((sk3, _dev(torch, extra_keys), _dev(torch, extra_w)))
    plan = ms.Batch(jobs, {"chunk_keys": 1 << 11, "smem_min_ratio": 1})
    plan.launch()
    torch.cuda.synchronize()
    _check(host, mode=1, extra={3: (extra_keys, extra_w)})


@pytest.mark.parametrize("b,c", [(31, 1), (89, 1), (64, 59)])
def test_batched_other_primes(env, b, c):
    torch, ms = env
    jobs, host = _jobs(torch, ms, 10, 3, b=b, c=c, nmax=30000)
    plan = ms.Batch(jobs, {"chunk_keys": 1 << 12, "smem_min_ratio": 2})
    plan.launch()
    torch.cuda.synchronize()
    _check(host, b=b, c=c)


def test_batched_equals_plain_launches(env):
    torch, ms = env
    jobs, host = _jobs(torch, ms, 16, 21)
    plan = ms.Batch(jobs)
    plan.launch()
    twins = []
    for sk, keys, w in jobs:
        tw = ms.Sketch(t=sk.t, m=sk.m, k=sk.k, seed=0, coeffs=sk.coeffs())
        tw.update(keys, w)
        twins.append(tw)
    torch.cuda.synchronize()
    for (sk, _, _), tw in zip(jobs, twins):
        assert torch.equal(sk.counters(), tw.counters())


def test_tuner_restores_counters_and_picks_a_candidate(env):
    torch, ms = env
    jobs, host = _jobs(torch, ms, 20, 13)
    before = [sk.counters().clone() for sk, _, _ in jobs]
    cands = [{"threads": 256, "chunk_keys": 1 << 13, "smem_min_ratio": 4},
             {"threads": 512, "chunk_keys": 1 << 15, "smem_min_ratio": 16},
             {"threads": 512, "chunk_keys": 1 << 24, "smem_min_ratio": 16, "rows_per_item": 15}]
    best, times = ms.tune_batched(jobs, cands, reps=2)
    assert len(times) == 3 and min(t for t in times if t >= 0) > 0
    assert best["chunk_keys"] in (1 << 13, 1 << 15, 1 << 24)
    for (sk, _, _), b0 in zip(jobs, before):
        assert torch.equal(sk.counters(), b0)
    plan = ms.Batch(jobs, best)
    plan.launch()
    torch.cuda.synchronize()
    _check(host)


def test_batched_rejects_mixed_primes(env):
    torch, ms = env
    a = ms.Sketch(t=5, m=1024, b=61, c=1, seed=1)
    b = ms.Sketch(t=5, m=1024, b=31, c=1, seed=1)
    keys = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(ms.MSError):
        ms.Batch([(a, keys, None), (b, keys.view(torch.int32), None)])
