"""Count Sketches with any number of buckets (CS_ANY_R: Algorithm
Mersenne-arb-r, Sec. 3.3; floor(h m / p) for 2^64 - 59, Sec. 1.5) on the GPU,
against the oracle counter for counter, in every placement."""
import numpy as np
import pytest

import datagen
import oracle
from test_gpu_parity import check_sketch, make_keys, run_sketch, to_dev

pytestmark = pytest.mark.gpu

ANY, TP = oracle.ANY_R, oracle.TWO_POLY


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2008_08654_gb300 as ms
    assert torch.cuda.is_available()
    ms.lib()
    return torch, ms


CASES = [
    # b, c, t, m, k, mode, place, weights
    (61, 1, 5, 1000, 4, ANY, -1, "pm100"),        # shared-memory tile (stride 1024)
    (61, 1, 5, 1025, 4, ANY, 0, "unit"),          # stride 2048
    (61, 1, 5, 3, 4, ANY, -1, "pm100"),           # tiny m
    (61, 1, 7, 50000, 4, ANY, 2, "unit"),         # global replicas (stride 65536)
    (61, 1, 7, 50000, 4, ANY, 3, "pm100"),        # direct int64 atomics
    (61, 1, 5, 6000, 4, ANY, 1, "pm100"),         # distributed shared memory
    (61, 1, 5, 1000, 4, ANY | TP, -1, "pm100"),   # two polynomials
    (61, 1, 7, 3000, 4, ANY, 0, "unit"),          # seven rows in the shared-memory tile
    (61, 1, 7, 2000, 4, ANY | TP, 0, "pm100"),
    (61, 1, 3, 12345, 2, ANY | TP, 2, "unit"),
    (61, 1, 1, (1 << 24) - 1, 4, ANY, -1, "unit"),  # largest m
    (61, 1, 15, 7, 1, ANY, -1, "pm100"),          # constant hash
    (31, 1, 5, 1000, 4, ANY, -1, "pm100"),
    (31, 1, 5, 70000, 4, ANY | TP, 2, "pm100"),
    (89, 1, 5, 999, 4, ANY, -1, "pm100"),
    (89, 1, 3, 5000, 3, ANY | TP, 1, "unit"),
    (64, 59, 5, 1000, 4, ANY | TP, -1, "pm100"),  # floor(h m / p)
    (64, 59, 7, 40000, 4, ANY | TP, 2, "unit"),
    (64, 59, 3, 3, 2, ANY | TP, 3, "pm100"),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(map(str, c)))
def test_any_r_parity(env, case):
    torch, ms = env
    b, c, t, m, k, mode, place, wk = case
    n = 40009
    keys = make_keys(b, c, n, 7 + t + m)
    w = None if wk == "unit" else datagen.i32_range(17 + m, -100, 100, n)
    seed = 500 + t * 7 + k + m
    sk, C, f2, rows = run_sketch(torch, ms, b, c, t, m, k, mode, keys, w, seed, place)
    assert sk.m == m and sk.stride >= m and sk.stride & (sk.stride - 1) == 0
    assert C.shape == (t, m)
    full = sk.counters(padded=True).cpu().numpy()
    assert not full[:, m:].any(), "padding columns must stay zero"
    want = check_sketch(sk, C, f2, rows, b, c, k, mode, keys, w, seed)
    # point queries of the stream's first keys
    q = sk.point_query(to_dev(torch, keys[:257]))
    coeffs = oracle.sketch_coeffs(b, c, k, t, mode, seed)
    assert np.array_equal(q.cpu().numpy(), oracle.point_query(b, c, k, mode, coeffs, want,
                                                              keys[:257]))


def test_any_r_big_weights_and_export(env):
    """Weights near +-2^31 take the int64 path with the arb-r map too; export,
    import and merge keep m, the row stride and the counters."""
    torch, ms = env
    b, c, t, m, k = 61, 1, 5, 777, 4
    n = 5003
    keys = make_keys(b, c, n, 3)
    w = datagen.i32_range(5, -2 ** 31, 2 ** 31 - 1, n)
    sk, C, f2, rows = run_sketch(torch, ms, b, c, t, m, k, ANY, keys, w, 9)
    check_sketch(sk, C, f2, rows, b, c, k, ANY, keys, w, 9)
    sk2 = ms.Sketch.import_(sk.export())
    assert (sk2.m, sk2.stride, sk2.mode) == (m, sk.stride, ANY)
    assert np.array_equal(sk2.counters().cpu().numpy(), C)
    sk2.merge(sk)
    torch.cuda.synchronize()
    assert np.array_equal(sk2.counters().cpu().numpy(), 2 * C)


def test_any_r_rejected_where_unsupported(env):
    torch, ms = env
    with pytest.raises(ms.MSError):
        ms.Sketch(t=5, m=1000, b=64, c=59, mode=ANY)      # needs two polynomials
    sk = ms.Sketch(t=5, m=1000, mode=ANY)
    kd = to_dev(torch, make_keys(61, 1, 100, 1))
    with pytest.raises(ms.MSError):
        ms.Batch([(sk, kd, None)])                          # batched plans: powers of two only
    with pytest.raises(ms.MSError):
        ms.Sketch(t=5, m=1024).merge(ms.Sketch(t=5, m=1024, mode=ANY))
