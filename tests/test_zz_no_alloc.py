"""The allocation-free F2 estimate (cs_estimate_f2_noalloc), called through the
C ABI, against the CPU oracle's row sums and median and against the regular
entry point (cs_estimate_f2).  It exists for callers that cannot call
cudaMalloc (e.g. a running serving loop that must not allocate); its scratch is
a static device array shared by every call.  This file is collected last so
that a run stopping at its first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2008_08654_gb300 as ms
    lib = ms.lib()
    f = lib.cs_estimate_f2_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    return torch, ms, f


def _u128(t2):
    """(lo, hi) int64 pairs -> Python integers."""
    a = t2.cpu().numpy().view(np.uint64).reshape(-1, 2)
    return [int(lo) | (int(hi) << 64) for lo, hi in a]


def _call_twice(torch, ms, f, counters, t, m):
    """Two calls in a row on the shared scratch; both must give the same values."""
    stream = torch.cuda.current_stream().cuda_stream
    got = []
    for _ in range(2):
        out = torch.full((2,), -1, dtype=torch.int64, device="cuda")
        rows = torch.full((t, 2), -1, dtype=torch.int64, device="cuda")
        st = f(counters.data_ptr(), t, m, out.data_ptr(), rows.data_ptr(), stream)
        assert st == 0, ms.lib().ms_last_cuda_error()
        torch.cuda.synchronize()
        got.append((_u128(out)[0], _u128(rows)))
    assert got[0] == got[1]
    return got[0]


@pytest.mark.parametrize("t,m,n,weighted", [(5, 1024, 100003, True), (7, 1 << 16, 300007, False),
                                            (1, 2, 17, True), (15, 1 << 13, 50021, True)])
def test_noalloc_f2_equals_the_oracle_and_cs_estimate_f2(env, t, m, n, weighted):
    torch, ms, f = env
    keys = torch.from_numpy(datagen.u64_below(t * 7 + n, (1 << 61) - 1, n).view(np.int64)).cuda()
    w = torch.from_numpy(datagen.i32_range(n, -100, 100, n)).cuda() if weighted else None
    sk = ms.Sketch(t=t, m=m, k=4, seed=n)
    sk.update(keys, w)
    ref_rows = torch.empty((t, 2), dtype=torch.int64, device="cuda")
    ref = sk.estimate_f2(rows=ref_rows)
    counters = sk.counters()
    C = counters.cpu().numpy()
    est, rows = _call_twice(torch, ms, f, counters, t, m)
    assert rows == oracle.row_sumsq(C)
    assert est == oracle.f2_estimate(C)
    assert est == _u128(ref)[0] and rows == _u128(ref_rows)
    out = torch.empty(2, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert f(counters.data_ptr(), t, m, out.data_ptr(), None, stream) == 0  # rows optional
    torch.cuda.synchronize()
    assert _u128(out)[0] == est


@pytest.mark.parametrize("t,m", [(15, 1 << 18), (1, 1 << 24), (15, 1 << 24)])
def test_noalloc_f2_at_the_limits_of_its_scratch(env, t, m):
    """t = 15 rows of 64 blocks each: the 960 partial sums fill the static array
    exactly (m = 2^18 is the smallest width with 64 blocks per row, m = 2^24 the
    largest accepted).  Counters are seeded words of up to 40 bits either sign,
    so the 128-bit row sums carry across their low word."""
    torch, ms, f = env
    words = datagen.u64_below(t * 1000 + m.bit_length(), 0, t * m, stream=datagen.STREAM_VALUES)
    C = ((words >> np.uint64(23)).view(np.int64) - (1 << 40)).reshape(t, m)
    counters = torch.from_numpy(C).cuda()
    est, rows = _call_twice(torch, ms, f, counters, t, m)
    assert rows == oracle.row_sumsq(C)
    assert est == oracle.f2_estimate(C)


def test_noalloc_f2_rejects_bad_arguments(env):
    torch, ms, f = env
    c = torch.zeros(64, dtype=torch.int64, device="cuda")
    out = torch.empty(4, dtype=torch.int64, device="cuda")
    rows = torch.empty(8, dtype=torch.int64, device="cuda")
    assert f(c.data_ptr(), 17, 2, out.data_ptr(), None, None) == 3      # t > 15
    assert f(c.data_ptr(), 1, 1 << 25, out.data_ptr(), None, None) == 3  # m > 2^24
    assert f(c.data_ptr(), 4, 16, out.data_ptr(), None, None) == 1      # even t
    assert f(c.data_ptr(), 1, 12, out.data_ptr(), None, None) == 1      # m not a power of two
    assert f(None, 1, 16, out.data_ptr(), None, None) == 1
    assert f(c.data_ptr(), 1, 16, None, None, None) == 1
    # misaligned: counters not on 8 bytes, out or rows not on 16 (nothing is launched)
    assert f(c.data_ptr() + 4, 1, 16, out.data_ptr(), None, None) == 8
    assert f(c.data_ptr(), 1, 16, out.data_ptr() + 8, None, None) == 8
    assert f(c.data_ptr(), 1, 16, out.data_ptr(), rows.data_ptr() + 8, None) == 8
