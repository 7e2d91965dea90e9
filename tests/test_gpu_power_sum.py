"""GPU parity of the power-sum row hash for p = 2^31-1, 2^89-1 and 2^64-59
(x, x^2, x^3 once per key, then a0 + a1 x + a2 x^2 + a3 x^3 per row, Sec. 1.2):
every counter and the F2 estimate against the CPU oracle, bit for bit, in every
counter placement, with one and two polynomials per row, t = 5 and 7; and the
power sum against Horner's rule (Algorithm Mersenne) on the same sketch."""
import numpy as np
import pytest

import datagen
import oracle
from test_gpu_parity import check_sketch, make_keys, run_sketch, to_dev

pytestmark = pytest.mark.gpu

OTHER_PRIMES = [(31, 1), (89, 1), (64, 59)]


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2008_08654_gb300 as ms
    assert torch.cuda.is_available()
    ms.lib()
    return torch, ms


@pytest.mark.parametrize("place", [0, 1, 2, 3])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("t", [5, 7])
@pytest.mark.parametrize("b,c", OTHER_PRIMES)
def test_power_sum_every_placement(env, b, c, t, mode, place):
    torch, ms = env
    n = 20011  # several blocks, ragged tail, edge keys first
    m = 1 << 15 if place == 2 else 2048  # place 2 needs a sketch that owns replicas
    keys = make_keys(b, c, n, 300 + b + t + place)
    w = datagen.i32_range(301 + mode + place, -100, 100, n)
    seed = 5000 + 7 * b + t + 3 * mode
    sk, C, f2, rows = run_sketch(torch, ms, b, c, t, m, 4, mode, keys, w, seed, place=place,
                                 strategy=1)
    ll = sk.last_launch()
    # a shared-memory tile runs the lean kernels (specialized == 2)
    lean = place == 0
    assert ll["place"] == place and ll["strategy"] == 1 and ll["specialized"] == (2 if lean else 1), ll
    check_sketch(sk, C, f2, rows, b, c, 4, mode, keys, w, seed)


@pytest.mark.parametrize("b,c", OTHER_PRIMES)
def test_power_sum_unit_weights_and_extreme_weights(env, b, c):
    """Unit weights (the table path where the key type allows it) and weights
    near +-2^31, which leave the power-sum loop for the exact int64 path."""
    torch, ms = env
    n, t, m = 60013, 5, 1024
    keys = make_keys(b, c, n, 77 + b)
    sk, C, f2, rows = run_sketch(torch, ms, b, c, t, m, 4, 0, keys, None, 9, strategy=1)
    check_sketch(sk, C, f2, rows, b, c, 4, 0, keys, None, 9)
    w = datagen.i32_range(78 + b, -2 ** 31, 2 ** 31 - 1, n)
    w[:4] = [-2 ** 31, 2 ** 31 - 1, 0, -1]
    for place in (0, 2, 3):
        sk, C, f2, rows = run_sketch(torch, ms, b, c, t, 1 << 15 if place == 2 else m, 4, 1, keys,
                                     w, 11, place=place, strategy=1, blocks=6)
        check_sketch(sk, C, f2, rows, b, c, 4, 1, keys, w, 11)


@pytest.mark.parametrize("b,c", OTHER_PRIMES)
def test_power_sum_equals_horner(env, b, c):
    torch, ms = env
    n, t, m = 100003, 7, 4096
    keys = to_dev(torch, make_keys(b, c, n, 5 + b))
    w = to_dev(torch, datagen.i32_range(6 + b, -100, 100, n))
    got = []
    for strategy in (0, 1):
        sk = ms.Sketch(t=t, m=m, k=4, b=b, c=c, seed=17, mode=1)
        sk.set_launch(strategy=strategy)
        sk.update(keys, w)
        assert sk.last_launch()["strategy"] == strategy
        got.append(sk.counters().cpu().numpy())
    assert np.array_equal(got[0], got[1])
    assert got[0].any()
