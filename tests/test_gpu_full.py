"""Full-size GPU parity in the launch configuration bench.py times.

The large single sketch (2^28 Zipf keys, t=7, m=2^16, unit weights) and the
plain sketch (2^20 uniform keys, weights in [-100, 100], t=5, m=1024) are run
through cs_update with the library's automatic launch choice -- exactly what
bench.py does -- and every counter and the F2 estimate are compared with the
multi-threaded CPU oracle over the whole stream.
"""
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

NTHREADS = max(1, os.cpu_count() or 1)


def _run(workload, seed=2008, n=None):
    import torch

    import bench
    import paper_2008_08654_gb300 as ms
    wl = bench.WORKLOADS[workload]
    keys, w = bench.make_inputs(wl, seed, 0, n)
    sk = ms.Sketch(t=wl["t"], m=wl["m"], k=4, b=61, c=1, seed=seed, mode=wl["mode"])
    sk.update(torch.from_numpy(keys.view(np.int64)).cuda(),
              None if w is None else torch.from_numpy(w).cuda())
    got_c = sk.counters().cpu().numpy()
    got_f2 = sk.f2()
    launch = sk.last_launch()
    coeffs = oracle.sketch_coeffs(61, 1, 4, wl["t"], wl["mode"], seed)
    want_c = oracle.cs_update(61, 1, 4, wl["t"], wl["m"], wl["mode"], coeffs, keys, w,
                              nthreads=NTHREADS)
    assert np.array_equal(got_c, want_c), "%d counters differ" % int((got_c != want_c).sum())
    assert got_f2 == oracle.f2_estimate(want_c)
    return launch


def test_plain_sketch_full_size():
    _run("plain")


@pytest.mark.parametrize("n", [(1 << 20) - 3, 3 * (1 << 19) + 1, (1 << 21) + 5])
def test_plain_sketch_balanced_launch_sizes(n):
    """Streams of two or three rounds of four keys a thread, for which the
    automatic launch sizes its blocks so every thread takes the same number of
    rounds; ragged ends included."""
    launch = _run("plain", n=n)
    assert launch["specialized"] == 2  # the lean shared-memory tile kernel
    assert launch["blocks"] * launch["threads"] * 4 * 3 >= n


def test_plain_any_m_quarter():
    """Any number of buckets (m = 1000, Algorithm Mersenne-arb-r) on the first
    2^26 keys of the 2^28-key stream the bench times, in its launch
    configuration (the lean kernel with the any-m map)."""
    launch = _run("plain-anyr", n=1 << 26)
    assert launch["specialized"] == 2


def test_large_sketch_full_size():
    launch = _run("large")
    print("large sketch launch:", launch)


def test_large_sketch_two_poly_quarter():
    """Two polynomials per row on the first 2^26 keys of the same stream."""
    _run("large-twopoly", n=1 << 26)


@pytest.mark.parametrize("b,c,k", [(61, 1, 4), (31, 1, 4), (89, 1, 4), (89, 1, 8), (64, 59, 4)])
def test_hash_eval_1e7_keys(b, c, k):
    """Every hash value of 10^7 keys (edge keys first, the rest uniform over the
    key type) equals the oracle's, bit for bit."""
    import torch

    import paper_2008_08654_gb300 as ms
    from test_gpu_parity import hash_to_np, make_keys, to_dev
    n = 10 ** 7
    keys = make_keys(b, c, n, 4000 + b + k)
    h = ms.Hash(k=k, b=b, c=c, seed=31 * b + k)
    got = hash_to_np(torch, h.eval(to_dev(torch, keys)), b)
    want = oracle.hash_eval(b, c, oracle.from_ints(h.coeffs()), keys)
    if b == 89:
        assert np.array_equal(got, want)
    else:
        assert not want[:, 1].any()
        assert np.array_equal(got, want[:, 0])
