"""Wide division (Table 2 sizes, b up to 1024): the oracle's definition-based
quotient and remainder are pinned by the division identity, and the library's
step count for Algorithm division-generalized is checked against the theorem of
Sec. 4 on Python integers.  CPU only."""
from fractions import Fraction

import numpy as np
import pytest

import oracle

CASES = [(32, 1), (32, 3), (61, 1), (64, 1), (64, 59), (65, 5), (100, 1), (127, 1), (128, 1),
         (128, 159), (129, 1), (256, 189), (521, 1), (777, 12345), (1024, 1), (1024, 105)]


def _edges(b, c):
    p = (1 << b) - c
    top = (1 << (2 * b)) - 1
    e = {0, 1, 2, p - 1, p, p + 1, 2 * p - 1, 2 * p, p * p - 1, p * p, p * p + 1, top, top - 1,
         (1 << b) - 1, 1 << b, (1 << b) + 1, 3 * p + 2, (top // p) * p, (top // p) * p - 1}
    return sorted(v for v in e if 0 <= v <= top)


def _values(b, c, n, seed):
    rng = np.random.default_rng(seed)
    vals = _edges(b, c)
    for _ in range(n):
        bits = int(rng.integers(1, 2 * b + 1))
        vals.append(int.from_bytes(rng.bytes((bits + 7) // 8), "little") % (1 << bits))
    return vals


@pytest.mark.parametrize("b,c", CASES)
def test_divmod_wide_identity(b, c):
    """v = q p + r with 0 <= r < p, on edges and random widths up to 2b bits."""
    p = (1 << b) - c
    vals = _values(b, c, 400, b * 131 + c)
    lv = (2 * b + 63) // 64
    q, r = oracle.divmod_wide(b, c, oracle.ints_to_limbs(vals, lv))
    assert q.shape == (len(vals), (b + 64) // 64) and r.shape == (len(vals), (b + 63) // 64)
    for v, qq, rr in zip(vals, oracle.limbs_to_ints(q), oracle.limbs_to_ints(r)):
        assert 0 <= rr < p and qq * p + rr == v


def test_divmod_wide_ignores_bits_above_2b():
    """The operation is defined on v mod 2^(2b): garbage above bit 2b is dropped."""
    b, c = 100, 3
    v = (1 << 200) - 12345
    junk = v | (0xABCDE << 200)
    q1, r1 = oracle.divmod_wide(b, c, oracle.ints_to_limbs([v], 4))
    q2, r2 = oracle.divmod_wide(b, c, oracle.ints_to_limbs([junk], 4))
    assert np.array_equal(q1, q2) and np.array_equal(r1, r2)


def _paper_division(v, b, c, steps):
    """Algorithm division-generalized (Sec. 1.5) on Python integers."""
    vp = v + c
    z = vp >> b
    for _ in range(steps - 1):
        z = (z * c + vp) >> b
    return z


def _theorem_steps(b, c):
    """Smallest n whose range in the theorem of Sec. 4 contains 2^(2b) - 1."""
    q, x, n = 1 << b, (1 << (2 * b)) - 1, 1
    while True:
        bound = c * (q // c) ** n - c if q % c == 0 else Fraction(q, c) ** (n - 1) * (q - c)
        if x <= bound:
            return n
        n += 1


@pytest.mark.parametrize("b,c", CASES)
def test_library_step_count_covers_theorem_range(b, c):
    """ms_div_wide_steps(b, c) is at least the theorem's step count for all
    v < 2^(2b) (c = 1: exactly 2, Algorithm div-simple), and with it the paper's
    division and modulus give the oracle's quotient and remainder."""
    import paper_2008_08654_gb300 as ms
    steps = ms.div_wide_steps(b, c)
    need = _theorem_steps(b, c)
    assert need <= steps <= need + 1
    if c == 1:
        assert steps == 2
    p = (1 << b) - c
    vals = _values(b, c, 300, b * 7 + c)
    for v in vals:
        z = _paper_division(v, b, c, steps)
        assert (z, (v + z * c) & ((1 << b) - 1)) == divmod(v, p)


def test_one_step_too_few_fails_for_c1():
    """With c = 1 a single step is not enough near 2^(2b) (the theorem's range
    for n = 1 ends at 2^b - 1): v = 2^(2b) - 1 has quotient 2^b + 1."""
    for b in (32, 128, 1024):
        v = (1 << (2 * b)) - 1
        assert _paper_division(v, b, 1, 1) == 1 << b
        assert _paper_division(v, b, 1, 2) == (1 << b) + 1 == v // ((1 << b) - 1)


def test_step_count_rejects_large_c():
    import paper_2008_08654_gb300 as ms
    assert ms.div_wide_steps(64, 1 << 63) == -1
    assert ms.div_wide_steps(64, 59) == 3
