"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: Python's
arbitrary-precision integers, exhaustive enumeration over a small prime field,
closed forms from the paper, or published known-answer vectors.  Each is
chosen so that a plausible slip in the oracle (a dropped term, a wrong index,
a flipped sign, a transposed operand) fails at least one of them.
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import datagen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

PRIMES = [(31, 1), (61, 1), (89, 1), (64, 59)]


def _golden_splitmix():
    out = {}
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            seed, vals = line.split(":")
            out[int(seed)] = [int(v) for v in vals.split()]
    return out


# ---------------------------------------------------------------- SplitMix64

def test_splitmix64_known_answers():
    """Both SplitMix64 implementations (oracle, input generator) reproduce the
    published known-answer sequences."""
    for seed, expect in _golden_splitmix().items():
        assert [int(v) for v in oracle.splitmix64(seed, len(expect))] == expect
        assert [int(v) for v in datagen.splitmix64_sequence(seed, len(expect))] == expect


def test_coefficient_draw_rule():
    """Coefficients are SplitMix64 words, masked to b bits, redrawn while >= p
    (uniform on [0, p), Sec. 1.2); b=89 takes two words, low word first."""
    words = _golden_splitmix()[1234567]
    a = oracle.to_ints(oracle.draw_coeffs(61, 1, 4, 1, 1234567))
    assert a == [w & ((1 << 61) - 1) for w in words[:4]]
    a = oracle.to_ints(oracle.draw_coeffs(31, 1, 2, 1, 1234567))
    assert a == [w & ((1 << 31) - 1) for w in words[:2]]
    a = oracle.to_ints(oracle.draw_coeffs(89, 1, 2, 1, 1234567))
    assert a == [words[0] | ((words[1] & ((1 << 25) - 1)) << 64),
                 words[2] | ((words[3] & ((1 << 25) - 1)) << 64)]
    # 2^64-59: a word >= p must be rejected.  Over many draws every value is < p.
    a = oracle.to_ints(oracle.draw_coeffs(64, 59, 4, 4096, 7))
    assert all(0 <= v < (1 << 64) - 59 for v in a)
    # rejection at a tiny prime: p = 2^3 - 1 = 7 rejects the masked value 7
    seq = [int(w) & 7 for w in oracle.splitmix64(99, 64)]
    expect = [v for v in seq if v < 7][:8]
    assert oracle.to_ints(oracle.draw_coeffs(3, 1, 8, 1, 99)) == expect


# ---------------------------------------------------------------- P1 division

def _edges(b, c):
    p = (1 << b) - c
    e = {0, 1, p - 1, p, p + 1, 2 * p - 1, 2 * p, p * p - 1, p * p, (1 << (2 * b)) - 2,
         (1 << (2 * b)) - 1, (1 << 64) - 1, 1 << 64, (1 << 64) + 1, (1 << 127), (1 << 128) - 1,
         (1 << 128) - 2, (1 << b), (1 << b) - 1, 3 * p + 2}
    return sorted(v for v in e if 0 <= v < (1 << 128))


@pytest.mark.parametrize("b,c", PRIMES)
def test_divmod_matches_bigint(b, c):
    """The oracle's / and % on unsigned __int128 equal Python's exact divmod on
    edge values and on 2e5 random values of every width up to 128 bits."""
    p = (1 << b) - c
    vals = _edges(b, c)
    for bits in (2 * b - 1, 2 * b, 122, 128):
        bits = min(bits, 128)
        vals += oracle.to_ints(datagen.u128_bits(bits + 17 * b, bits, 50000))
    q, r = oracle.divmod_(b, c, oracle.from_ints(vals))
    q, r = oracle.to_ints(q), oracle.to_ints(r)
    for v, qq, rr in zip(vals, q, r):
        assert (qq, rr) == divmod(v, p)


def _paper_division(v, b, c, steps):
    """Algorithm division-generalized (Sec. 1.5) restated on Python integers:
    v' = v + c; z = v' >> b; then steps-1 times z = (z*c + v') >> b."""
    vp = v + c
    z = vp >> b
    for _ in range(steps - 1):
        z = (z * c + vp) >> b
    return z


def _paper_mod(v, z, b, c):
    """Algorithm mod-generalized (Sec. 1.5): y = (v + z*c) & (2^b - 1)."""
    return (v + z * c) & ((1 << b) - 1)


def _steps_needed(b, c, vmax):
    """Smallest n with vmax within the range of the division theorem (Sec. 4)."""
    q = 1 << b
    n = 1
    while True:
        if q % c == 0:
            bound = c * (q // c) ** n - c
        else:
            bound = Fraction(q, c) ** (n - 1) * (q - c)
        if vmax <= bound:
            return n
        n += 1


@pytest.mark.parametrize("b,c", PRIMES)
def test_oracle_agrees_with_paper_division(b, c):
    """Within the range of the division theorem (Sec. 4), the paper's branch-free
    division and modulus equal the oracle's quotient and remainder; one step
    fewer is off by at most 1 (error bound u_1 = 1); extra steps change nothing."""
    vals = _edges(b, c)
    vals += oracle.to_ints(datagen.u128_bits(5, 128, 20000))
    vals += oracle.to_ints(datagen.u128_bits(6, min(2 * b, 128), 20000))
    q, r = oracle.divmod_(b, c, oracle.from_ints(vals))
    q, r = oracle.to_ints(q), oracle.to_ints(r)
    for v, qq, rr in zip(vals, q, r):
        n = _steps_needed(b, c, v)
        z = _paper_division(v, b, c, n)
        assert z == qq
        assert _paper_mod(v, z, b, c) == rr
        assert _paper_division(v, b, c, n + 2) == qq
        if n > 1:
            assert 0 <= qq - _paper_division(v, b, c, n - 1) <= 1


@pytest.mark.parametrize("b", [31, 61])
def test_branch_free_division_on_1e7_random_values(b):
    """Algorithm div-simple (Sec. 1.5) for p = 2^b - 1 and v < 2^(2b), restated
    branch free on 64-bit words (numpy) -- v' = v + 1, z = ((v' >> b) + v') >> b,
    y = (v + z) & p -- equals the oracle's / and % on 10^7 random values."""
    n = 10 ** 7
    p = np.uint64((1 << b) - 1)
    v = datagen.u128_bits(1000 + b, 2 * b, n)
    vl, vh = v[:, 0].copy(), v[:, 1].copy()
    one = np.uint64(1)
    sb, s64b = np.uint64(b), np.uint64(64 - b)
    # v' = v + 1 (with the carry into the high word)
    pl = vl + one
    ph = vh + (pl == 0).astype(np.uint64)
    # v' >> b  (< 2^b + 1 for v < 2^(2b)), then + v'
    z1 = (pl >> sb) | (ph << s64b) if b < 64 else ph
    sl = pl + z1
    sh = ph + (sl < z1).astype(np.uint64)
    z = (sl >> sb) | (sh << s64b)
    y = (vl + z) & p
    q, r = oracle.divmod_(b, 1, v)
    assert not q[:, 1].any() and not r[:, 1].any()
    assert np.array_equal(z, q[:, 0])
    assert np.array_equal(y, r[:, 0])
    # the whole range was reached: the largest inputs are near 2^(2b)
    assert int(vh.max()) >> max(0, 2 * b - 64 - 4) > 0 if 2 * b > 64 else int(vl.max()) >> (2 * b - 4) > 0


def test_division_step_counts():
    """Step counts implied by the division theorem: c=1 needs 2 steps below 2^(2b)
    (Algorithm div-simple); 2^64-59 needs 3 steps for all of [0, 2^128) and 2
    steps fail there; 2^61-1 needs 3 steps beyond 2^122."""
    assert _steps_needed(61, 1, (1 << 122) - 1) == 2
    assert _steps_needed(31, 1, (1 << 62) - 1) == 2
    assert _steps_needed(61, 1, (1 << 128) - 1) == 3
    assert _steps_needed(89, 1, (1 << 128) - 1) == 2
    assert _steps_needed(64, 59, (1 << 128) - 1) == 3
    p = (1 << 64) - 59
    # beyond 2 steps' range, exact multiples of p with a large quotient come
    # out one too small after 2 steps (random 128-bit values almost never do)
    for q in ((1 << 64) - 1, (1 << 64) + 59, 3 << 62):
        v = q * p
        assert v < (1 << 128)
        assert _paper_division(v, 64, 59, 2) == q - 1
        assert _paper_division(v, 64, 59, 3) == q
        assert oracle.to_ints(oracle.divmod_(64, 59, oracle.from_ints([v]))[0]) == [q]


# ---------------------------------------------------------------- P6 hash

def _horner(a, x, p):
    y = 0
    for ai in reversed(a):
        y = (y * x + ai) % p
    return y


@pytest.mark.parametrize("b,c", PRIMES)
@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_hash_matches_bigint_horner(b, c, k):
    """The oracle's sum-of-powers hash equals Horner's rule on exact integers
    (the recurrence of Algorithm Mersenne, Sec. 1.2), keys >= p included."""
    p = (1 << b) - c
    a = oracle.to_ints(oracle.draw_coeffs(b, c, k, 1, 1000 * b + k))
    if b == 31:
        keys = datagen.u32_below(3, 0, 3000)
        keys[:4] = [0, 1, p - 1, 0xFFFFFFFF]
        ints = [int(x) for x in keys]
    elif b == 89:
        keys = datagen.u128_bits(3, 128, 3000)
        special = [0, 1, p - 1, p, p + 1, (1 << 128) - 1, (1 << 89)]
        keys[:len(special)] = oracle.from_ints(special)
        ints = oracle.to_ints(keys)
    else:
        keys = datagen.u64_below(3, 0, 3000)
        keys[:6] = [0, 1, p - 1, p, p + 1, (1 << 64) - 1]
        ints = [int(x) for x in keys]
    h = oracle.to_ints(oracle.hash_eval(b, c, oracle.from_ints(a), keys))
    for x, hx in zip(ints, h):
        assert hx == _horner(a, x % p, p)
        assert hx == _horner(a, x, p)


def test_hash_constant_polynomial():
    """k = 1: h(x) = a_0 for every key."""
    a = oracle.draw_coeffs(61, 1, 1, 1, 5)
    keys = datagen.u64_below(9, 0, 100)
    h = oracle.to_ints(oracle.hash_eval(61, 1, a, keys))
    assert set(h) == {oracle.to_int(a[0])}


# ---------------------------------------------------------------- P2 universality

def _all_tuples(p, k):
    grids = np.meshgrid(*[np.arange(p, dtype=np.uint64)] * k, indexing="ij")
    flat = np.stack([g.reshape(-1) for g in grids], axis=1)  # (p^k, k), a_0 first
    pairs = np.zeros((flat.shape[0] * k, 2), dtype=np.uint64)
    pairs[:, 0] = flat.reshape(-1)
    return pairs


def test_exact_4_universality_p31():
    """Def. of k-universality (Sec. 1.2): over all 31^4 coefficient vectors, the
    hash values of 4 distinct keys hit every 4-tuple in [31]^4 exactly once;
    the first j keys hit every j-tuple exactly 31^(4-j) times."""
    p, k = 31, 4
    coeffs = _all_tuples(p, k)
    keys = oracle.from_ints([3, 7, 19, 30])
    h = oracle.hash_many(5, 1, k, coeffs, keys)[:, :, 0].astype(np.int64)
    assert h.max() < p
    for j in range(1, 5):
        code = np.zeros(h.shape[0], dtype=np.int64)
        for i in range(j):
            code = code * p + h[:, i]
        counts = np.bincount(code, minlength=p ** j)
        assert counts.min() == counts.max() == p ** (k - j)


# ---------------------------------------------------------------- P3 split

def _split_of_value(h, b, m):
    """(bucket, sign) the oracle's sketch assigns to a key whose hash value is h:
    a constant polynomial (k=1, a_0 = h), one row of m counters, weight 1."""
    coeffs = oracle.from_ints([h])
    C = oracle.cs_update(b, 1, 1, 1, m, oracle.TWO_FOR_ONE, coeffs,
                         np.array([12345], dtype=np.uint64))
    nz = np.nonzero(C[0])[0]
    assert len(nz) == 1
    return int(nz[0]), int(C[0, nz[0]])


@pytest.mark.parametrize("ell", [1, 2, 3, 4, 5, 6])
def test_two_for_one_joint_distribution_p127(ell):
    """Algorithm h-and-s at p = 2^7 - 1 with r = 2^ell buckets.  Over h in [p]:
    every (bucket, sign-bit) cell holds 2^(b-1-ell) values except
    (r-1, 1), which holds one fewer (the missing all-ones value p); hence the
    marginals of eqs. coll-ell<r-1 / coll-ell=r-1, the collision probability
    (1 + (r-1)/p^2)/r of eq. coll, and Lemma remove-si:
    sum_h s(h) [i(h) = j] = [j = r-1]."""
    b, p = 7, 127
    r = 1 << ell
    cells = {}
    sign_sum = [0] * r
    for h in range(p):
        i, s = _split_of_value(h, b, r)
        a = (1 - s) // 2
        cells[(i, a)] = cells.get((i, a), 0) + 1
        sign_sum[i] += s
    for i in range(r):
        for a in (0, 1):
            expect = (1 << (b - 1 - ell)) - (1 if (i, a) == (r - 1, 1) else 0)
            assert cells.get((i, a), 0) == expect
    pr = [Fraction(cells.get((i, 0), 0) + cells.get((i, 1), 0), p) for i in range(r)]
    for i in range(r - 1):
        assert pr[i] == (1 + Fraction(1, p)) / r
    assert pr[r - 1] == (1 - Fraction(r - 1, p)) / r
    assert sum(x * x for x in pr) == (1 + Fraction(r - 1, p * p)) / r
    assert sign_sum == [0] * (r - 1) + [1]


# ---------------------------------------------------------------- P4 expectation

STREAMS = [
    # (keys, weights): repeated keys aggregate into f_x; signed weights
    ([3, 9, 3, 17, 22, 5, 9], [2, -1, -5, 4, 1, 7, 3]),
    ([0, 1, 2, 30], [1, 1, 1, 1]),
    ([6, 13, 27], [-3, 2, 5]),
]


def _moments(keys, w):
    f = {}
    for x, d in zip(keys, w):
        f[x] = f.get(x, 0) + d
    f1 = sum(f.values())
    f2 = sum(v * v for v in f.values())
    n = sum(1 for v in f.values() if v != 0)
    return f1, f2, n


@pytest.mark.parametrize("b,k,ell", [(5, 4, 1), (5, 4, 2), (5, 4, 3), (5, 4, 4),
                                     (7, 2, 1), (7, 2, 3), (7, 2, 6)])
@pytest.mark.parametrize("stream", range(len(STREAMS)))
def test_two_for_one_expectation_exact(b, k, ell, stream):
    """Thm h-and-s-p / Lemma count-mersenne (Sec. 2): E[X] = F2 + (F1^2 - F2)/p^2
    for the two-for-one split.  Summed over ALL p^k coefficient vectors this is
    the exact integer identity  sum X = p^k F2 + p^(k-2) (F1^2 - F2);  also
    |E[X] - F2| <= F2 (n-1)/p^2."""
    p = (1 << b) - 1
    keys, w = STREAMS[stream]
    keys = [x % p for x in keys]
    f1, f2, n = _moments(keys, w)
    coeffs = _all_tuples(p, k)
    xs = oracle.cs_x_many(b, 1, k, 1 << ell, oracle.TWO_FOR_ONE, coeffs,
                          np.array(keys, dtype=np.uint64), np.array(w, dtype=np.int32))
    assert not xs[:, 1].any()
    total = int(xs[:, 0].astype(object).sum())
    assert total == p ** k * f2 + p ** (k - 2) * (f1 * f1 - f2)
    ex = Fraction(total, p ** k)
    assert abs(ex - f2) <= Fraction(f2 * (n - 1), p * p)


@pytest.mark.parametrize("b,k,ell", [(5, 2, 1), (5, 2, 2), (5, 2, 4), (3, 2, 1), (3, 2, 2)])
@pytest.mark.parametrize("stream", [0, 2])
def test_two_poly_expectation_exact(b, k, ell, stream):
    """Independent sign polynomial (Algorithm count-sketch with two functions):
    E[s] = 1/p for the top bit of a value uniform in [p], so
    E[X] = F2 + (F1^2 - F2) (1/p^2) (1 + (r-1)/p^2)/r; over all p^(2k) pairs of
    coefficient vectors: sum X = p^(2k) F2 + (F1^2-F2) p^(2k-4) (p^2 + r - 1)/r."""
    p = (1 << b) - 1
    r = 1 << ell
    keys, w = STREAMS[stream]
    keys = [x % p for x in keys]
    f1, f2, _ = _moments(keys, w)
    one = _all_tuples(p, k).reshape(-1, k, 2)  # (p^k, k, 2)
    nb = one.shape[0]
    sets = np.concatenate([np.repeat(one, nb, axis=0), np.tile(one, (nb, 1, 1))], axis=1)
    xs = oracle.cs_x_many(b, 1, k, r, oracle.TWO_POLY, sets.reshape(-1, 2),
                          np.array(keys, dtype=np.uint64), np.array(w, dtype=np.int32))
    total = int(xs[:, 0].astype(object).sum())
    assert (p * p + r - 1) % r == 0
    assert total == p ** (2 * k) * f2 + (f1 * f1 - f2) * p ** (2 * k - 4) * (p * p + r - 1) // r


# ---------------------------------------------------------------- P5 special cases

def test_single_key_estimate_is_w_squared():
    for w in (1, -1, 100, -77, 2 ** 31 - 1, -2 ** 31):
        coeffs = oracle.sketch_coeffs(61, 1, 4, 5, oracle.TWO_FOR_ONE, 11)
        C = oracle.cs_update(61, 1, 4, 5, 1024, oracle.TWO_FOR_ONE, coeffs,
                             np.array([424242], dtype=np.uint64), np.array([w], dtype=np.int32))
        assert oracle.row_sumsq(C) == [w * w] * 5
        assert oracle.f2_estimate(C) == w * w


def test_injective_buckets_give_exact_f2():
    """With h(x) = x (k = 2, a = (0, 1)) and keys 0..n-1 < m, buckets are
    distinct, so X = sum_x f_x^2 = F2 exactly."""
    n, m = 200, 256
    coeffs = oracle.from_ints([0, 1])
    keys = np.arange(n, dtype=np.uint64)
    w = datagen.i32_range(4, -100, 100, n)
    C = oracle.cs_update(61, 1, 2, 1, m, oracle.TWO_FOR_ONE, coeffs, keys, w)
    assert oracle.row_sumsq(C)[0] == int((w.astype(np.int64) ** 2).sum())
    assert oracle.f2_estimate(C) == oracle.exact_f2(keys, w)
    # h(x) = x < 2^60 has sign bit 0, so every counter is +w at bucket x
    assert (C[0, :n] == w).all() and not C[0, n:].any()


def test_sign_bit_is_top_bit():
    """h = 2^60 (top bit of a 61-bit value) gives sign -1; h = 2^60 - 1 gives +1
    in bucket 2^10 - 1 (low 10 bits all ones)."""
    assert _split_of_value(1 << 60, 61, 1024) == (0, -1)
    assert _split_of_value((1 << 60) - 1, 61, 1024) == (1023, 1)
    assert _split_of_value((1 << 61) - 2, 61, 1024) == (1022, -1)


def test_linearity_and_threads():
    """Count Sketch is linear (Sec. 1.3): sketch(A) + sketch(B) = sketch(A ++ B);
    the threaded oracle equals the single-threaded one."""
    coeffs = oracle.sketch_coeffs(61, 1, 4, 3, oracle.TWO_POLY, 21)
    keys = datagen.u64_below(8, (1 << 61) - 1, 5000)
    w = datagen.i32_range(8, -100, 100, 5000)
    whole = oracle.cs_update(61, 1, 4, 3, 64, oracle.TWO_POLY, coeffs, keys, w)
    a = oracle.cs_update(61, 1, 4, 3, 64, oracle.TWO_POLY, coeffs, keys[:1234], w[:1234])
    bb = oracle.cs_update(61, 1, 4, 3, 64, oracle.TWO_POLY, coeffs, keys[1234:], w[1234:])
    assert (a + bb == whole).all()
    mt = oracle.cs_update(61, 1, 4, 3, 64, oracle.TWO_POLY, coeffs, keys, w, nthreads=4)
    assert (mt == whole).all()
    # weights summing to zero on every key leave an all-zero sketch
    keys2 = np.concatenate([keys, keys])
    w2 = np.concatenate([w, -w])
    z = oracle.cs_update(61, 1, 4, 3, 64, oracle.TWO_POLY, coeffs, keys2, w2)
    assert not z.any()


def test_counters_match_direct_definition_small():
    """Counters equal C[r][h_r(x) mod m] += (1 - 2 floor(h_r(x)/2^(b-1))) w,
    recomputed here from the oracle's own hash values with Python integers."""
    for (b, c) in PRIMES:
        t, m, k = 3, 16, 4
        coeffs = oracle.sketch_coeffs(b, c, k, t, oracle.TWO_FOR_ONE, 77)
        if b == 31:
            keys = datagen.u32_below(5, 0, 300)
        elif b == 89:
            keys = datagen.u128_bits(5, 100, 300)
        else:
            keys = datagen.u64_below(5, 0, 300)
        w = datagen.i32_range(5, -100, 100, 300)
        C = oracle.cs_update(b, c, k, t, m, oracle.TWO_FOR_ONE, coeffs, keys, w)
        expect = np.zeros((t, m), dtype=np.int64)
        for r in range(t):
            h = oracle.to_ints(oracle.hash_eval(b, c, coeffs[r * k:(r + 1) * k], keys))
            for hx, wx in zip(h, w):
                expect[r, hx % m] += (1 - 2 * (hx >> (b - 1))) * int(wx)
        assert (C == expect).all()


def test_f2_is_median_of_rows():
    rng = np.random.default_rng(0)
    C = rng.integers(-1000, 1000, size=(7, 50)).astype(np.int64)
    rows = [int((C[r].astype(object) ** 2).sum()) for r in range(7)]
    assert oracle.row_sumsq(C) == rows
    assert oracle.f2_estimate(C) == sorted(rows)[3]
    # 128-bit row sums: 40 counters of magnitude 2^40 sum past 2^64
    C = np.full((3, 40), -(1 << 40), dtype=np.int64)
    assert oracle.row_sumsq(C) == [40 * (1 << 80)] * 3
    # and the sum wraps modulo 2^128: 40 * 2^124 = 8 * 2^124 (mod 2^128)
    C = np.full((3, 40), -(1 << 62), dtype=np.int64)
    assert oracle.row_sumsq(C) == [(40 * (1 << 124)) % (1 << 128)] * 3


def test_exact_f2_small():
    keys = np.array([5, 3, 5, 5, 9, 3], dtype=np.uint64)
    w = np.array([1, 2, -4, 10, -3, -2], dtype=np.int32)
    assert oracle.exact_f2(keys, w) == 7 * 7 + 0 + 9
    assert oracle.exact_f2(keys) == 9 + 4 + 1


def test_point_query_definition():
    """Point query (Sec. 1.3): with h(x) = x in every row (injective buckets for
    keys < m) each row's estimate s(x) C[i(x)] is exactly f_x, so the median is
    f_x; a key sharing its bucket with nothing else reads back its own weight."""
    n, m, t = 100, 128, 3
    coeffs = oracle.from_ints([0, 1] * t)
    keys = np.arange(n, dtype=np.uint64)
    w = datagen.i32_range(3, -100, 100, n)
    C = oracle.cs_update(61, 1, 2, t, m, oracle.TWO_FOR_ONE, coeffs, keys, w)
    assert (oracle.point_query(61, 1, 2, oracle.TWO_FOR_ONE, coeffs, C, keys) == w).all()
    # h(x) = 2^60 + x has sign bit 1: the counters hold -f_x and the query returns f_x
    coeffs = oracle.from_ints([1 << 60, 1] * t)
    C = oracle.cs_update(61, 1, 2, t, m, oracle.TWO_FOR_ONE, coeffs, keys, w)
    assert (C[:, :n] == -w).all()
    assert (oracle.point_query(61, 1, 2, oracle.TWO_FOR_ONE, coeffs, C, keys) == w).all()


def test_point_query_median_of_rows():
    """Rows disagree: the median (not the mean or the first row) is returned."""
    t, m = 3, 8
    # row r hashes every key to the constant bucket r, sign +
    coeffs = oracle.from_ints([0, 0, 1, 0, 2, 0])
    C = np.array([[5, 0, 0, 0, 0, 0, 0, 0], [0, -7, 0, 0, 0, 0, 0, 0], [0, 0, 40, 0, 0, 0, 0, 0]],
                 dtype=np.int64)
    assert list(oracle.point_query(61, 1, 2, oracle.TWO_FOR_ONE, coeffs, C,
                                   np.array([9, 10], dtype=np.uint64))) == [5, 5]
