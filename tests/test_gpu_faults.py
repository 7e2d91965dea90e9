"""Host-side fault injection: MS_FAULT_ALLOC=n makes the library's n-th device
allocation report MS_ERR_OOM without calling cudaMalloc.  Each case runs in a
child process (the allocation count is per process) and checks that the failing
call returns OOM, that nothing else breaks, and that the next calls in the same
process work and give the oracle's counters.  No GPU fault is involved."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PRELUDE = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, %r)
    import datagen, oracle
    import paper_2008_08654_gb300 as ms

    def expect_oom(fn):
        try:
            fn()
        except ms.MSError as e:
            assert e.status == 4, e
            return
        raise AssertionError("no OOM")

    def check_sketch(sk, seed):
        keys = datagen.u64_below(seed, (1 << 61) - 1, 5000)
        sk.update(torch.from_numpy(keys.view(np.int64)).cuda())
        torch.cuda.synchronize()
        co = oracle.sketch_coeffs(61, 1, 4, sk.t, 0, seed)
        want = oracle.cs_update(61, 1, 4, sk.t, sk.m, 0, co, keys)
        assert np.array_equal(sk.counters().cpu().numpy(), want)
""" % ROOT)


def _run(body: str, fault: int):
    env = dict(os.environ, MS_FAULT_ALLOC=str(fault))
    r = subprocess.run([sys.executable, "-c", PRELUDE + textwrap.dedent(body) + "\nprint('OK')\n"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout + r.stderr


def test_sketch_create_oom_then_recovers():
    _run("""
        expect_oom(lambda: ms.Sketch(t=5, m=1024, seed=1))
        check_sketch(ms.Sketch(t=5, m=1024, seed=1), 1)
    """, fault=1)


def test_large_sketch_oom_then_recovers():
    # the replicas live in the sketch's single allocation: one failure, no leak
    _run("""
        expect_oom(lambda: ms.Sketch(t=7, m=1 << 16, seed=2))
        check_sketch(ms.Sketch(t=7, m=1 << 16, seed=2), 2)
    """, fault=1)


def test_batch_create_oom_then_recovers():
    _run("""
        sk = ms.Sketch(t=5, m=1024, seed=3)                      # allocation 1
        keys = datagen.u64_below(3, (1 << 61) - 1, 5000)
        kd = torch.from_numpy(keys.view(np.int64)).cuda()
        expect_oom(lambda: ms.Batch([(sk, kd, None)]))           # allocation 2 fails
        b = ms.Batch([(sk, kd, None)])                           # allocation 3
        b.launch()
        torch.cuda.synchronize()
        co = oracle.sketch_coeffs(61, 1, 4, 5, 0, 3)
        assert np.array_equal(sk.counters().cpu().numpy(), oracle.cs_update(61, 1, 4, 5, 1024, 0, co, keys))
    """, fault=2)


@pytest.mark.parametrize("fault", [1, 2, 3])
def test_server_create_oom_each_allocation(fault):
    # allocations of a one-sketch server: 1 the sketch, 2 the staging ring,
    # 3 the job and answer tables
    _run("""
        expect_oom(lambda: ms.Server([1024], staging_bytes=1 << 24))
        srv = ms.Server([1024], staging_bytes=1 << 24)
        keys = datagen.u64_below(4, (1 << 61) - 1, 5000)
        srv.submit_update(0, keys)
        srv.drain()
        co = oracle.sketch_coeffs(61, 1, 4, 5, 0, 0)
        assert np.array_equal(srv.counters(0), oracle.cs_update(61, 1, 4, 5, 1024, 0, co, keys))
        srv.close()
    """, fault=fault)
