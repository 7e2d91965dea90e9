"""Any number of buckets (CS_ANY_R): the oracle's bucket/sign maps pinned by
exhaustive enumeration against the paper's statements -- Algorithm
Mersenne-arb-r and Lemmas ix-r-dist / remove-si-r-dist (Sec. 3.3), the
most-uniform map of Lemma most-uniform (Sec. 1.4), floor(h r / p) for a
pseudo-Mersenne prime (Sec. 1.5) -- and the exact expectation of Thm
h-and-s-p-arb-r as an integer identity over all coefficient vectors.  CPU only."""
from fractions import Fraction

import numpy as np
import pytest

import oracle

ANY = oracle.ANY_R


def _split(h, b, c, r, mode=ANY, g=0):
    """(bucket, sign) the oracle assigns to a key whose hash value is h (and
    whose sign polynomial has value g in two-polynomial mode): constant
    polynomials (k = 1), one row of r counters, weight 1."""
    vals = [h, g] if mode & oracle.TWO_POLY else [h]
    C = oracle.cs_update(b, c, 1, 1, r, mode, oracle.from_ints(vals),
                         np.array([12345], dtype=np.uint64))
    nz = np.nonzero(C[0])[0]
    assert len(nz) == 1
    return int(nz[0]), int(C[0, nz[0]])


def _ceil(a, b):
    return -(-a // b)


@pytest.mark.parametrize("b", [5, 7])
def test_mersenne_arb_r_distribution(b):
    """Algorithm Mersenne-arb-r at p = 2^b - 1, every r in [2, 2^(b-2)]:
    eq. prix0: (2 ceil(2^(b-1)/r) - 1) values of h land in bucket 0;
    eq. prixneq0: every other bucket gets 2 floor(2^(b-1)/r) or 2 ceil(2^(b-1)/r);
    eq. ix=iy: the collision probability is at most (1 + (r/2^b)^2)/r;
    eq. ix=0: Pr[i = 0] <= (1 + r/2^b)/r;
    Lemma remove-si-r-dist: sum_h s(h) [i(h) = j] = [j = 0] (this fixes the
    sign s = 2a - 1; the printed 1 - 2a would give -[j = 0])."""
    p, q = (1 << b) - 1, 1 << (b - 1)
    for r in range(2, (1 << (b - 2)) + 1):
        counts = [0] * r
        ssum = [0] * r
        for h in range(p):
            i, s = _split(h, b, 1, r)
            assert 0 <= i < r and s in (-1, 1)
            counts[i] += 1
            ssum[i] += s
        assert sum(counts) == p
        assert counts[0] == 2 * _ceil(q, r) - 1
        for j in range(1, r):
            assert counts[j] in (2 * (q // r), 2 * _ceil(q, r))
        pr = [Fraction(cj, p) for cj in counts]
        assert sum(x * x for x in pr) <= (1 + Fraction(r, 1 << b) ** 2) / r
        assert pr[0] <= (1 + Fraction(r, 1 << b)) / r
        assert ssum == [1] + [0] * (r - 1)


@pytest.mark.parametrize("b", [3, 4, 5, 6, 7, 8])
def test_most_uniform_map_lemma(b):
    """Lemma most-uniform (iii), the fact the arb-r construction builds on:
    v -> ((v + 1) r) >> b maps [2^b - 1] most uniformly onto [r] (every bucket
    gets floor or ceil of (2^b - 1)/r).  A check of the lemma itself by
    enumeration; the oracle's map is pinned by the tests around it."""
    q = (1 << b) - 1
    for r in range(1, q + 1):
        counts = [0] * r
        for v in range(q):
            counts[((v + 1) * r) >> b] += 1
        assert set(counts) <= {q // r, _ceil(q, r)}


@pytest.mark.parametrize("b,c", [(5, 3), (6, 3), (7, 3)])
def test_pseudo_mersenne_floor_map_is_most_uniform(b, c):
    """For p = 2^b - c the bucket floor(h r / p) (Sec. 1.5) is most uniform:
    every bucket gets floor(p/r) or ceil(p/r) values of h in [p]; the sign is
    the top bit of the second polynomial (s = 1 - 2a)."""
    p = (1 << b) - c
    for r in (2, 3, 5, 7, 8):
        counts = [0] * r
        for h in range(p):
            i, s = _split(h, b, c, r, ANY | oracle.TWO_POLY, g=h)
            counts[i] += 1
            assert s == 1 - 2 * (h >> (b - 1))
        assert set(counts) <= {p // r, _ceil(p, r)}
        assert counts == [sum(1 for h in range(p) if h * r // p == j) for j in range(r)]


STREAMS = [
    ([3, 9, 3, 17, 22, 5, 9], [2, -1, -5, 4, 1, 7, 3]),
    ([0, 1, 2, 30], [1, 1, 1, 1]),
    ([6, 13, 27], [-3, 2, 5]),
]


def _moments(keys, w):
    f = {}
    for x, d in zip(keys, w):
        f[x] = f.get(x, 0) + d
    return sum(f.values()), sum(v * v for v in f.values())


def _all_tuples(p, k):
    grids = np.meshgrid(*[np.arange(p, dtype=np.uint64)] * k, indexing="ij")
    flat = np.stack([g.reshape(-1) for g in grids], axis=1)
    pairs = np.zeros((flat.shape[0] * k, 2), dtype=np.uint64)
    pairs[:, 0] = flat.reshape(-1)
    return pairs


@pytest.mark.parametrize("b,k,r", [(5, 4, 3), (5, 4, 5), (5, 4, 6), (5, 4, 7), (7, 2, 3),
                                   (7, 2, 10), (7, 2, 25), (7, 2, 32)])
@pytest.mark.parametrize("stream", range(len(STREAMS)))
def test_arb_r_expectation_exact(b, k, r, stream):
    """Thm h-and-s-p-arb-r (Sec. 3.3): E[X] = F2 + (F1^2 - F2)/p^2 for the
    two-for-one split of Algorithm Mersenne-arb-r with any r; over ALL p^k
    coefficient vectors the integer identity sum X = p^k F2 + p^(k-2)(F1^2 - F2)."""
    p = (1 << b) - 1
    keys, w = STREAMS[stream]
    keys = [x % p for x in keys]
    f1, f2 = _moments(keys, w)
    xs = oracle.cs_x_many(b, 1, k, r, ANY, _all_tuples(p, k), np.array(keys, dtype=np.uint64),
                          np.array(w, dtype=np.int32))
    total = int(xs[:, 0].astype(object).sum())
    assert total == p ** k * f2 + p ** (k - 2) * (f1 * f1 - f2)


@pytest.mark.parametrize("b,c,r", [(5, 1, 3), (5, 1, 6), (5, 3, 3), (5, 3, 7), (4, 3, 5)])
def test_arb_r_two_poly_expectation_exact(b, c, r):
    """Two polynomials with any r: the sign bit a of the second value has
    E[s] = c/p (2^(b-1) - c of the p values have a = 1), independent of the
    bucket, so E[X] = F2 + (F1^2 - F2) (c/p)^2 sum_j (n_j/p)^2 with n_j the
    number of h in [p] landing in bucket j; over all p^(2k) coefficient pairs:
    sum X = p^(2k) F2 + (F1^2 - F2) c^2 p^(2k-4) sum_j n_j^2."""
    p, k = (1 << b) - c, 2
    keys, w = STREAMS[0]
    keys = [x % p for x in keys]
    f1, f2 = _moments(keys, w)
    n = [0] * r
    for h in range(p):
        n[_split(h, b, c, r, ANY | oracle.TWO_POLY, g=0)[0]] += 1
    one = _all_tuples(p, k).reshape(-1, k, 2)
    nb = one.shape[0]
    sets = np.concatenate([np.repeat(one, nb, axis=0), np.tile(one, (nb, 1, 1))], axis=1)
    xs = oracle.cs_x_many(b, c, k, r, ANY | oracle.TWO_POLY, sets.reshape(-1, 2),
                          np.array(keys, dtype=np.uint64), np.array(w, dtype=np.int32))
    total = int(xs[:, 0].astype(object).sum())
    assert total == p ** (2 * k) * f2 + (f1 * f1 - f2) * c * c * p ** (2 * k - 4) * sum(
        x * x for x in n)


def test_arb_r_with_power_of_two_r_differs_from_h_and_s():
    """CS_ANY_R is a different map even when r is a power of two: the bucket is
    taken from the low b-1 bits of h + 1, scaled, not from the low bits of h."""
    b, r = 7, 4
    diffs = sum(1 for h in range(127)
                if _split(h, b, 1, r)[0] != _split(h, b, 1, r, oracle.TWO_FOR_ONE)[0])
    assert diffs > 0
