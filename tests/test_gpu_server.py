"""The continuous-batching server: every query answer equals the oracle's F2
estimate of its sketch over exactly the updates submitted to that sketch
before the query -- whether requests run one at a time or mixed in batches."""
import os

import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu


def _requests(nsk, count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        s = int(rng.integers(0, nsk))
        if rng.random() < 0.25:
            reqs.append(("q", s, None, None))
        else:
            n = int(rng.integers(0, 5000))
            keys = datagen.zipf(seed * 1000 + i, 1.1, 1 << 16, n)
            w = datagen.i32_range(seed * 1000 + i, -100, 100, n) if rng.random() < 0.5 else None
            reqs.append(("u", s, keys, w))
    return reqs


def _expected(reqs, widths, t, seed_base):
    C = [np.zeros((t, m), dtype=np.int64) for m in widths]
    ans = []
    for kind, s, keys, w in reqs:
        if kind == "u":
            oracle.cs_update(61, 1, 4, t, widths[s], 0,
                             oracle.sketch_coeffs(61, 1, 4, t, 0, seed_base + s), keys, w,
                             counters=C[s])
        else:
            ans.append(oracle.f2_estimate(C[s]))
    return ans, C


def _run(ms, reqs, widths, t, seed_base, alone, **kw):
    srv = ms.Server(widths, t=t, seed_base=seed_base, **kw)
    tickets = []
    for kind, s, keys, w in reqs:
        if kind == "u":
            tk = srv.submit_update(s, keys, w)
        else:
            tk = srv.submit_query(s)
        if alone:
            srv.drain()
        tickets.append((kind, tk))
    srv.drain()
    ans = []
    for kind, tk in tickets:
        r = srv.poll(tk)
        assert r["done"] and r["status"] == 0
        if kind == "q":
            ans.append(r["f2"])
    counters = [srv.counters(i) for i in range(len(widths))]
    stats = srv.stats()
    srv.close()
    return ans, counters, stats


@pytest.mark.parametrize("kw", [{}, {"max_batch_requests": 3},
                                {"staging_bytes": 64 << 10, "max_batch_keys": 7000},
                                {"max_inflight": 2}])
def test_server_answers_equal_oracle_alone_and_mixed(kw):
    import paper_2008_08654_gb300 as ms
    widths, t, seed_base = [64, 128, 1024, 64, 256, 4096], 5, 77
    reqs = _requests(len(widths), 80, 5)
    want, want_c = _expected(reqs, widths, t, seed_base)
    mixed, cm, stats = _run(ms, reqs, widths, t, seed_base, alone=False, **kw)
    alone, ca, _ = _run(ms, reqs, widths, t, seed_base, alone=True, **kw)
    assert mixed == want
    assert alone == want
    for a, b, c in zip(cm, ca, want_c):
        assert np.array_equal(a, c) and np.array_equal(b, c)
    assert stats["requests_done"] == len(reqs)


def test_server_rejects_bad_requests():
    import paper_2008_08654_gb300 as ms
    srv = ms.Server([64, 64], staging_bytes=8192)
    with pytest.raises(ms.MSError) as e:
        srv.submit_query(2)
    assert e.value.status == 1
    with pytest.raises(ms.MSError) as e:  # larger than the whole staging ring
        srv.submit_update(0, np.zeros(4096, dtype=np.uint64))
    assert e.value.status == 3
    srv.close()


def test_server_backpressure_statuses():
    """With one slot and try_only, submissions beyond the slot return BUSY; the
    ones accepted are applied exactly."""
    import paper_2008_08654_gb300 as ms
    srv = ms.Server([1024], max_inflight=1)
    keys = datagen.u64_below(3, (1 << 61) - 1, 1 << 20)
    accepted, busy = 0, 0
    for _ in range(20):
        try:
            srv.submit_update(0, keys, try_only=True)
            accepted += 1
        except ms.MSError as e:
            assert e.status == 7
            busy += 1
    srv.drain()
    C = srv.counters(0)
    want = np.zeros((5, 1024), dtype=np.int64)
    co = oracle.sketch_coeffs(61, 1, 4, 5, 0, 0)
    one = oracle.cs_update(61, 1, 4, 5, 1024, 0, co, keys, nthreads=8)
    assert accepted >= 1 and accepted + busy == 20
    assert np.array_equal(C, one * accepted)
    srv.close()


def test_load_generator_runs():
    import paper_2008_08654_gb300 as ms
    srv = ms.Server([1024, 4096] * 8, staging_bytes=1 << 28)
    pool = datagen.zipf(9, 1.1, 1 << 32, 1 << 18)
    r = srv.run_load(pool, count=300, rate_per_s=2000.0, query_fraction=0.1, min_keys=256,
                     max_keys=1 << 16, seed=4)
    assert r["updates"] + r["queries"] == 300 and r["keys"] > 0
    assert 0 < r["update_p50_ms"] <= r["update_p99_ms"]
    srv.close()


def test_server_page_locked_payloads_read_in_place():
    """Updates from page-locked buffers (read in place by the kernel, no staging
    copy) and from pageable ones (copied), mixed in batches, misaligned slices
    among them; a page-locked update larger than the whole staging ring is
    accepted, a pageable one is not."""
    import torch
    import paper_2008_08654_gb300 as ms
    widths, t, seed_base = [64, 1024, 4096], 5, 91
    reqs = _requests(len(widths), 60, 9)
    pinned = []
    for i, (kind, s, keys, w) in enumerate(reqs):
        if kind == "u" and i % 2 == 0:
            kp = torch.from_numpy(keys.view(np.int64)).pin_memory()
            wp = None if w is None else torch.from_numpy(w).pin_memory()
            if i % 4 == 0 and len(keys) > 1:  # an 8-byte offset: scalar loads
                buf = torch.empty(len(keys) + 1, dtype=torch.int64).pin_memory()
                buf[1:] = kp
                kp = buf[1:]
            pinned.append((kp, wp))
            reqs[i] = (kind, s, keys, w, kp, wp)
    big = datagen.zipf(3, 1.1, 1 << 16, 20000)
    reqs.append(("u", 2, big, None, torch.from_numpy(big.view(np.int64)).pin_memory(), None))
    reqs.append(("q", 2, None, None))
    want, want_c = _expected([r[:4] for r in reqs], widths, t, seed_base)
    srv = ms.Server(widths, t=t, seed_base=seed_base, staging_bytes=64 << 10)
    with pytest.raises(ms.MSError):
        srv.submit_update(2, big)  # pageable and larger than the ring
    tickets = []
    for r in reqs:
        if r[0] == "u":
            keys, w = (r[4], r[5]) if len(r) == 6 else (r[2], r[3])
            tickets.append(("u", srv.submit_update(r[1], keys, w)))
        else:
            tickets.append(("q", srv.submit_query(r[1])))
    srv.drain()
    ans = []
    for kind, tk in tickets:
        res = srv.poll(tk)
        assert res["done"] and res["status"] == 0
        if kind == "q":
            ans.append(res["f2"])
    assert ans == want
    for i, c in enumerate(want_c):
        assert np.array_equal(srv.counters(i), c)
    srv.close()


def test_bounded_waits_time_out_on_the_host_and_the_server_recovers():
    """Every blocking host wait of the server is bounded by timeout_s.  With one
    slot and a 100-microsecond limit, a blocking submission behind a 2^24-key
    update (its pageable copy alone takes milliseconds) and a drain while that
    update is in flight both give up with MS_ERR_TIMEOUT -- no device wait is
    involved.  The in-flight request still completes, and afterwards the server
    answers exactly: counters and F2 equal the oracle over everything accepted."""
    import time

    import paper_2008_08654_gb300 as ms
    widths, t, seed_base = [1024], 5, 313
    srv = ms.Server(widths, t=t, seed_base=seed_base, staging_bytes=1 << 30, max_inflight=1,
                    max_batch_keys=1 << 24, max_batch_requests=1, timeout_s=1e-4)
    big = datagen.zipf(41, 1.1, 1 << 32, 1 << 24)
    small = datagen.zipf(42, 1.1, 1 << 32, 1000)
    t_big = srv.submit_update(0, big)
    with pytest.raises(ms.MSError) as e:
        srv.submit_update(0, small)  # blocks for a slot: the only one is taken
    assert e.value.status == 6  # MS_ERR_TIMEOUT
    with pytest.raises(ms.MSError) as e:
        srv.drain()
    assert e.value.status == 6
    with pytest.raises(ms.MSError) as e:
        srv.submit_query(0, try_only=True)  # the non-blocking form: busy
    assert e.value.status == 7  # MS_ERR_BUSY

    def wait_done(tk):
        deadline = time.monotonic() + 60.0
        while True:
            r = srv.poll(tk)
            if r["done"]:
                return r
            assert time.monotonic() < deadline, "request did not complete"
            time.sleep(1e-3)

    assert wait_done(t_big)["status"] == 0
    t_small = srv.submit_update(0, small)
    assert wait_done(t_small)["status"] == 0
    r = wait_done(srv.submit_query(0))
    C = np.zeros((t, widths[0]), dtype=np.int64)
    coeffs = oracle.sketch_coeffs(61, 1, 4, t, 0, seed_base)
    for keys in (big, small):
        oracle.cs_update(61, 1, 4, t, widths[0], 0, coeffs, keys, None, counters=C,
                         nthreads=os.cpu_count() or 1)
    assert r["status"] == 0 and r["f2"] == oracle.f2_estimate(C)
    assert np.array_equal(srv.counters(0), C)
    srv.close()
