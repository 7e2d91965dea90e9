"""The allocation-free F2 estimate (cs_estimate_f2_noalloc) against the regular
one (cs_estimate_f2), called through the C ABI.  It exists for callers that
cannot call cudaMalloc (e.g. a running serving loop that must not allocate);
its scratch is a static device array shared by every call.  This file is
collected last so that a run stopping at its first failure has already run
every other test."""
import ctypes

import numpy as np
import pytest

import datagen

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


@pytest.mark.parametrize("t,m,n,weighted", [(5, 1024, 100003, True), (7, 1 << 16, 300007, False),
                                            (1, 2, 17, True), (15, 1 << 13, 50021, True)])
def test_noalloc_f2_equals_cs_estimate_f2(env, t, m, n, weighted):
    torch, ms, f = env
    keys = torch.from_numpy(datagen.u64_below(t * 7 + n, (1 << 61) - 1, n).view(np.int64)).cuda()
    w = torch.from_numpy(datagen.i32_range(n, -100, 100, n)).cuda() if weighted else None
    sk = ms.Sketch(t=t, m=m, k=4, seed=n)
    sk.update(keys, w)
    ref_rows = torch.empty((t, 2), dtype=torch.int64, device="cuda")
    ref = sk.estimate_f2(rows=ref_rows)
    counters = sk.counters()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # two calls in a row on the shared scratch
        out = torch.full((2,), -1, dtype=torch.int64, device="cuda")
        rows = torch.full((t, 2), -1, dtype=torch.int64, device="cuda")
        st = f(counters.data_ptr(), t, m, out.data_ptr(), rows.data_ptr(), stream)
        assert st == 0, ms.lib().ms_last_cuda_error()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        assert torch.equal(rows, ref_rows)
    out = torch.empty(2, dtype=torch.int64, device="cuda")
    assert f(counters.data_ptr(), t, m, out.data_ptr(), None, stream) == 0
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_noalloc_f2_rejects_sizes_beyond_its_scratch(env):
    torch, ms, f = env
    c = torch.zeros(64, dtype=torch.int64, device="cuda")
    out = torch.empty(2, dtype=torch.int64, device="cuda")
    assert f(c.data_ptr(), 17, 2, out.data_ptr(), None, None) == 3      # t > 15
    assert f(c.data_ptr(), 1, 1 << 25, out.data_ptr(), None, None) == 3  # m > 2^24
    assert f(c.data_ptr(), 4, 16, out.data_ptr(), None, None) == 1      # even t
    assert f(c.data_ptr(), 1, 12, out.data_ptr(), None, None) == 1      # m not a power of two
    assert f(None, 1, 16, out.data_ptr(), None, None) == 1
