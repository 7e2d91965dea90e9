"""CPU checks of the update kernels' row arithmetic (paper_2008_08654_gb300/
csrc/ms_field.cuh), emulated operation by operation on Python integers: every
32x32->64 multiply-add gets 32-bit operands and a 64-bit result, every
intermediate stays within the width the kernel gives it, and every row value,
bucket and sign equals the definition h(x) = sum a_i x^i mod p (Sec. 1.2) with
the split of Algorithm h-and-s (Sec. 1.3).  Inputs include the largest limbs
the lazy invariants allow and row sums driven onto p - 1, 0 and 2^88 +- 1.
These pin the bound arguments written beside the kernels; the kernels
themselves are checked bit for bit against the oracle by the GPU tests."""
import random

import pytest

M32 = (1 << 32) - 1
M64 = (1 << 64) - 1
M29 = (1 << 29) - 1
M30 = (1 << 30) - 1


def u32(v):
    assert 0 <= v <= M32, hex(v)
    return v


def s32(v):
    assert -(1 << 31) <= v < (1 << 31), v
    return v


def u64(v):
    assert 0 <= v <= M64, hex(v)
    return v


def madw(a, b, c):
    """mad.wide.u32: the bounds must keep the sum below 2^64."""
    return u64(u32(a) * u32(b) + u64(c))


def madws(a, b, c):
    """mad.wide.s32 into a 64-bit accumulator (wraps modulo 2^64)."""
    return (s32(a) * s32(b) + c) & M64


def h_ref(p, a, key):
    x = key % p
    return sum(a[i] * pow(x, i, p) for i in range(len(a))) % p


# ------------------------------------------------------------------ 2^61-1, signed-digit rows

P61 = (1 << 61) - 1


def s64(v):
    """A 64-bit word read as two's complement."""
    v &= M64
    return v - (1 << 64) if v >> 63 else v


def sext31(w):
    """The low 31 bits of a 32-bit word, sign-extended (the kernels' (int)(lo << 1) >> 1)."""
    w &= 0x7FFFFFFF
    return w - (1 << 31) if w >> 30 else w


D61 = (1 << 60) + (1 << 30)  # the key-side digit offset of row_sd


def p61_sdigits(X):
    """sdigits: X - D = h 2^31 + l with l = (X mod 2^31) - 2^30 and h = (X >> 31) - 2^29."""
    assert 0 <= X < (1 << 61) + 8
    lo, hi = X & M32, X >> 32
    lu = lo & 0x7FFFFFFF
    hu = u32(((hi << 32) | lo) >> 31)
    l, h = s32(lu - (1 << 30)), s32(hu - (1 << 29))
    d = s32(hu - lu + (1 << 30) - (1 << 29))
    assert X - D61 == h * (1 << 31) + l and d == h - l
    assert -(1 << 30) <= l < (1 << 30) and -(1 << 29) <= h <= (1 << 29)
    return l, h, d


def p61_sd_coef(a):
    """sd_coef: signed digits of c_i (a_i or a_i - p in (-2^60, 2^60)), cl - ch, k1."""
    cl, ch, nd, s = [], [], [], 0
    for ai in a[1:]:
        c = ai if ai <= (P61 >> 1) else ai - P61
        lo = sext31(c & M32)
        assert (c - lo) % (1 << 31) == 0
        hi = (c - lo) >> 31
        assert -(1 << 30) <= lo < (1 << 30) and -(1 << 29) <= hi <= (1 << 29)
        cl.append(lo)
        ch.append(hi)
        nd.append(s32(lo - hi))
        s = (s + ai) % P61
    s60 = (s + P61) >> 1 if s & 1 else s >> 1
    assert (2 * s60) % P61 == s  # 2^60 s = s / 2 (mod p)
    s30 = ((s & 0x7FFFFFFF) << 30) + (s >> 31)
    s30 = s30 - P61 if s30 >= P61 else s30
    assert s30 == (s << 30) % P61
    k = (a[0] + s60) % P61
    k = (k + s30) % P61
    k1 = k + 3 * P61 + 1
    assert k1 % P61 == (a[0] + D61 * sum(a[1:]) + 1) % P61
    return cl, ch, nd, k1


def p61_row(xs, a):
    """row_sd on lazy powers xs (< 2^61 + 8) and canonical a[0..3]: returns the
    64-bit word y64 whose low 61 bits are the canonical residue."""
    cl, ch, nd, k1 = p61_sd_coef(a)
    dg = [p61_sdigits(x) for x in xs]
    X1 = 0
    for i in range(3):
        X1 = madws(ch[i], dg[i][1], X1)
    X2 = X1
    for i in range(3):
        X2 = madws(cl[i], dg[i][0], X2)
    X3 = X2
    for i in range(3):
        X3 = madws(nd[i], dg[i][2], X3)
    A = sum(cl[i] * dg[i][0] for i in range(3))
    H = sum(ch[i] * dg[i][1] for i in range(3))
    M = sum(cl[i] * dg[i][1] + ch[i] * dg[i][0] for i in range(3))
    assert (s64(X1), s64(X2), s64(X3)) == (H, A + H, M)
    assert abs(A) <= 3 << 60 and abs(H) <= 3 << 58 and abs(M) <= 3 << 60
    m0, M1 = X3 & 0x3FFFFFFF, s64(X3) >> 30
    assert abs(M1) <= 3 << 30 and M == M1 * (1 << 30) + m0
    T = (u32(m0) * (1 << 31) + X2) & M64
    S1 = (T + X1 + M1 + k1) & M64
    S = A + 2 * H + m0 * (1 << 31) + M1  # the value the words hold, without wrap
    assert -(9 << 59) - (3 << 30) <= S <= (13 << 59) + (3 << 30)
    assert S1 == S + k1 and 0 < S1 < M64 - 16  # no wrap: S1 = v + 1 exactly
    q = S1 >> 61
    W = u64(S1 + q)
    z = W >> 61
    assert z == (S1 - 1) // P61  # Algorithm div-simple: floor(v / p)
    y64 = (S1 + z - 1) & M64
    return y64


def p61_bucket_sign(y64, mask):
    """bucket_sign_sd: the low bits and bit 60 of the canonical residue."""
    return (y64 & M32) & mask, ((y64 >> 32) >> 28) & 1


def p61_powers(key):
    def fold(v):
        return (v & P61) + (v >> 61)
    x = fold(key)
    xl, xh = x & 0x7FFFFFFF, x >> 31
    A = madw(xl, xl, 0)
    A = madw(xh << 1, xh, A)
    Q = madw(xh, xl, 0)
    x2 = fold(u64(A + (Q >> 29) + ((Q & 0x1FFFFFFF) << 32)))
    assert x2 < (1 << 61) + 4
    zl, zh = x2 & 0x7FFFFFFF, x2 >> 31
    A = madw(zl, xl, 0)
    A = madw(zh, xh << 1, A)
    M = madw(zh, xl, 0)
    M = madw(zl, xh, M)
    x3 = fold(u64(A + (M >> 30) + ((M & 0x3FFFFFFF) << 31)))
    return [x, x2, x3]


# ------------------------------------------------------------------ 2^31-1

P31 = (1 << 31) - 1


def p31_row(key, a, mask):
    def mul(z, x):
        v = u64(z * x)
        v = (v & P31) + (v >> 31)
        return (v & P31) + (v >> 31)
    x = (key & P31) + (key >> 31)
    x = x - P31 if x >= P31 else x
    x2 = mul(x, x)
    x3 = mul(x2, x)
    S = madw(a[1], x, a[0])
    S = madw(a[2], x2, S)
    S = madw(a[3], x3, S)
    v = madw(S >> 32, 2, S & M32)
    f = u32((v & P31) + (v >> 31))
    over = u32(f + 1) >> 31
    return (f + over) & mask, 0 if over else (f >> 30) & 1, f - P31 if f >= P31 else f


# ------------------------------------------------------------------ 2^64-59

C64 = 59
P64 = (1 << 64) - C64


def p64_mod3(v):  # Algorithm division-generalized, 3 steps, then mod-generalized
    vp = v + C64
    z = vp >> 64
    z = (z * C64 + vp) >> 64
    z = (z * C64 + vp) >> 64
    return (v + z * C64) & M64


def p64_row(key, a, mask):
    x = key - P64 if key >= P64 else key
    x2 = p64_mod3(x * x)
    x3 = p64_mod3(x2 * x)
    limbs = [[z & M29, (z >> 29) & M29, z >> 58] for z in (x, x2, x3)]
    L0, L1 = a[0] & M32, a[0] >> 32
    for i in range(3):
        for v in range(3):
            b = (a[i + 1] << (29 * v)) % P64
            L0 = madw(limbs[i][v], b & M32, L0)
            L1 = madw(limbs[i][v], b >> 32, L1)
    t = (L0 >> 32) + (L1 & M32)
    vl = (L0 & M32) | ((t & M32) << 32)
    vh = u32((L1 >> 32) + (t >> 32))
    vpl = vl + C64
    vph = u32(vh + (vpl >> 64))
    vpl &= M64
    q = u64(vph * C64)
    z = u32(vph + ((vpl + q) >> 64))
    y = (vl + z * C64) & M64
    return y & mask, y >> 63, y


# ------------------------------------------------------------------ 2^89-1, 30-bit limbs

P89 = (1 << 89) - 1


def val89(l):
    return l[0] + (l[1] << 30) + (l[2] << 60)


def norm3(L0, L1, L2):
    L1 = u64(L1 + (L0 >> 30))
    L2 = u64(L2 + (L1 >> 30))
    s0 = (L0 & M30) + (L2 >> 29)
    s1 = (L1 & M30) + (s0 >> 30)
    r = [s0 & M30, s1 & M30, (L2 & M29) + (s1 >> 30)]
    assert r[2] <= 1 << 29
    return r


def mul3(y, z, a=(0, 0, 0)):
    L0 = madw(y[0], z[0], a[0]); L0 = madw(y[1], z[2] << 1, L0); L0 = madw(y[2], z[1] << 1, L0)
    L1 = madw(y[0], z[1], a[1]); L1 = madw(y[1], z[0], L1); L1 = madw(y[2], z[2] << 1, L1)
    L2 = madw(y[0], z[2], a[2]); L2 = madw(y[1], z[1], L2); L2 = madw(y[2], z[0], L2)
    return norm3(L0, L1, L2)


def limbs89(v):
    return [v & M30, (v >> 30) & M30, v >> 60]


def p89_powers(key):
    x = limbs89((key & P89) + (key >> 89))
    x2 = mul3(x, x)
    return [x, x2, mul3(x2, x)]


def p89_row(xl, a, mask):
    """The Karatsuba row: six products per term, columns rebuilt from sums."""
    c = limbs89(a[0])
    S00 = S11 = S22 = 0
    T01, T02, T12 = c[1], c[2], 0
    for i in range(3):
        l = limbs89(a[i + 1])
        x = xl[i]
        S00 = madw(l[0], x[0], S00)
        S11 = madw(l[1], x[1], S11)
        S22 = madw(l[2], x[2], S22)
        T01 = madws(l[0] - l[1], x[1] - x[0], T01)
        T02 = madws(l[0] - l[2], x[2] - x[0], T02)
        T12 = madws(l[1] - l[2], x[2] - x[1], T12)
    U = (S00 + S11 + S22) & M64
    L2 = (U + T02) & M64
    L1 = (U + S22 + T01) & M64
    L0 = (2 * ((U + T12) & M64) - S00 + c[0]) & M64
    for v in (L0, L1, L2):
        assert v < 12 * (1 << 60) + (1 << 31)
    return p89_output(L0, L1, L2, mask)


def p89_output(L0, L1, L2, mask):
    """Bucket, sign and canonical residue of L0 + L1 2^30 + L2 2^60 (mod p)."""
    L1 = u64(L1 + (L0 >> 30))
    L2 = u64(L2 + (L1 >> 30))
    s0 = (L0 & M30) + (L2 >> 29)
    u1 = (L1 & M30) + (s0 >> 30)
    u2 = (L2 & M29) + (u1 >> 30)
    y = (s0 & M30) + ((u1 & M30) << 30) + (u2 << 60)
    assert y < (1 << 89) + (1 << 36)
    over = (u2 + (1 if (s0 & u1 & M30) == M30 else 0)) >> 29
    assert over == (1 if y >= P89 else 0)
    return (s0 + over) & mask, 0 if over else (u2 >> 28) & 1, y - P89 if y >= P89 else y


# ------------------------------------------------------------------ tests

def _coeffs(rng, p, n):
    edges = [[0, 0, 0, 0], [p - 1] * 4, [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1],
             [p - 2, p - 1, 1, p - 1]]
    return edges + [[rng.randrange(p) for _ in range(4)] for _ in range(n)]


def _keys(rng, p, kbits, n):
    e = [0, 1, p - 1, p, p + 1, 2 * p - 1, (1 << kbits) - 1, 1 << (kbits - 1)]
    return [v for v in e if v < (1 << kbits)] + [rng.randrange(1 << kbits) for _ in range(n)]


@pytest.mark.parametrize("prime", [31, 61, 64, 89])
def test_power_sum_rows_equal_the_definition(prime):
    rng = random.Random(prime)
    p, kbits = {31: (P31, 32), 61: (P61, 64), 64: (P64, 64), 89: (P89, 128)}[prime]
    sign_bit = {31: 30, 61: 60, 64: 63, 89: 88}[prime]
    mask = 4095
    for a in _coeffs(rng, p, 60):
        for key in _keys(rng, p, kbits, 25):
            want = h_ref(p, a, key)
            if prime == 31:
                b, s, y = p31_row(key, a, mask)
            elif prime == 61:
                y64 = p61_row(p61_powers(key), a)
                b, s = p61_bucket_sign(y64, mask)
                y = y64 & P61
            elif prime == 64:
                b, s, y = p64_row(key, a, mask)
            else:
                b, s, y = p89_row(p89_powers(key), a, mask)
            assert y == want
            assert (b, s) == (want & mask, (want >> sign_bit) & 1)


def test_rows_at_the_lazy_extremes():
    """The largest power limbs the lazy invariants allow, with the largest
    coefficients: every intermediate still fits its width."""
    half = P61 >> 1
    digit_edges = [0, 1, half, half + 1, half - (1 << 30), half + (1 << 30), P61 - 1,
                   (1 << 30) - 1, 1 << 30, P61 - (1 << 30), (1 << 61) - (1 << 31)]
    lazy = [0, (1 << 61) + 7, 1 << 61, P61 - 1, 1 << 60, (1 << 60) - 1, (1 << 60) + (1 << 30),
            (1 << 60) - (1 << 30), (1 << 60) + (1 << 30) - 1, (1 << 61) - (1 << 30)]
    for a in ([P61 - 1] * 4, [P61 - 2, P61 - 1, (1 << 61) - (1 << 31), P61 - 1]) + tuple(
            [e, e, e, e] for e in digit_edges):
        for xs in ([(1 << 61) + 7] * 3, [1 << 61] * 3, [P61 - 1, (1 << 61) + 7, 0]) + tuple(
                [v, w, v] for v in lazy for w in lazy):
            y = p61_row(xs, a) & P61
            assert y == (a[0] + sum(a[i + 1] * xs[i] for i in range(3))) % P61
    top = [M30, M30, 1 << 29]
    for a in ([P89 - 1] * 4, [P89 - 2, P89 - 1, 1, P89 - 1], [M30] * 4, [0] * 4):
        for xl in ([top] * 3, [[0, 0, 0], top, [0, M30, 0]], [[M30, 0, 1 << 29]] * 3):
            _, _, y = p89_row(xl, a, 1023)
            assert y == (a[0] + sum(a[i + 1] * val89(xl[i]) for i in range(3))) % P89
            r = mul3(xl[0], xl[1], limbs89(a[0]))
            assert val89(r) % P89 == (val89(xl[0]) * val89(xl[1]) + a[0]) % P89


def test_p89_output_stage_near_p():
    """Columns whose value reduces to p - 1, 0, 1, 2^88 - 1, 2^88, 2^88 + 1: the
    canonical test (y >= p from the carry chain), the bucket and the sign bit."""
    rng = random.Random(5)
    n = 0
    for target in (P89 - 1, 0, 1, (1 << 88) - 1, 1 << 88, (1 << 88) + 1, P89 - (1 << 30)):
        for _ in range(300):
            V = target + rng.randrange(1 << 34) * P89
            L2 = min(V >> 60, 9 * (1 << 60) - 1)
            L1 = min((V - (L2 << 60)) >> 30, 9 * (1 << 60))
            L0 = V - (L2 << 60) - (L1 << 30)
            if not 0 <= L0 < 12 * (1 << 60):
                continue
            b, s, y = p89_output(L0, L1, L2, (1 << 20) - 1)
            want = target % P89
            assert (y, b, s) == (want, want & ((1 << 20) - 1), (want >> 88) & 1)
            n += 1
    assert n > 1000


def test_p64_reduction_edges():
    """2^64-59: row sums near multiples of p reduce to the canonical residue
    with two steps of Algorithm division-generalized (V < 2^96)."""
    rng = random.Random(9)
    for _ in range(3000):
        a = [rng.choice([0, P64 - 1, rng.randrange(P64)]) for _ in range(4)]
        key = rng.choice([0, P64 - 1, P64, (1 << 64) - 1, rng.randrange(1 << 64)])
        _, _, y = p64_row(key, a, 4095)
        assert y == h_ref(P64, a, key)


def test_p61_rows_onto_p_and_at_digit_extremes():
    """2^61-1: rows driven onto the residues p - 1, 0, 1, 2^60 - 1, 2^60, 2^60 + 1
    (the canonical test of Algorithm div-simple and the sign bit), and operands
    whose signed digits sit at their extremes (every 64-bit word of the row stays
    within the bounds written beside row_sd)."""
    rng = random.Random(61)
    for target in (P61 - 1, P61 - 2, 0, 1, (1 << 60) - 1, 1 << 60, (1 << 60) + 1):
        for _ in range(400):
            key = rng.randrange(1 << 64)
            a = [0] + [rng.randrange(P61) for _ in range(3)]
            a[0] = (target - h_ref(P61, a, key)) % P61
            y64 = p61_row(p61_powers(key), a)
            assert y64 & P61 == target
            assert p61_bucket_sign(y64, 1023) == (target & 1023, (target >> 60) & 1)
    lo_e, hi_e = [-(1 << 30), (1 << 30) - 1, 0, 1], [-(1 << 29), 1 << 29, 0, -1]
    for _ in range(4000):
        a, xs = [rng.randrange(P61)], []
        for _ in range(3):
            c = rng.choice(hi_e) * (1 << 31) + rng.choice(lo_e)
            while not -(1 << 60) < c < (1 << 60):
                c = rng.choice(hi_e) * (1 << 31) + rng.choice(lo_e)
            a.append(c % P61)
            X = D61 + rng.choice(hi_e) * (1 << 31) + rng.choice(lo_e)
            while not 0 <= X < (1 << 61) + 8:
                X = D61 + rng.choice(hi_e) * (1 << 31) + rng.choice(lo_e)
            xs.append(X)
        y = p61_row(xs, a) & P61
        assert y == (a[0] + sum(a[i + 1] * xs[i] for i in range(3))) % P61


def test_p61_arb_split_from_row_words():
    """P61::arb_split_sd: the any-m bucket floor(r j / 2^60) of h + 1 = a 2^60 + j
    (Algorithm Mersenne-arb-r, Sec. 3.3), taken from row_sd's two output words
    as floor((j_hi r + floor(j_lo r / 2^32)) / 2^28) with j = j_hi 2^32 + j_lo,
    and a = bit 60 of h + 1: emulated in 32/64-bit words against the definition
    at the extremes of h and r and on random values."""
    import random
    rng = random.Random(3)
    P = (1 << 61) - 1
    hs = [0, 1, P - 1, P - 2, (1 << 60) - 1, 1 << 60, (1 << 60) - 2, (1 << 32) - 1, 1 << 32]
    hs += [rng.randrange(P) for _ in range(2000)]
    rs = [1, 2, 3, 1000, (1 << 24) - 1, 1 << 24, (1 << 32) - 1] + [rng.randrange(1, 1 << 32) for _ in range(20)]
    for h in hs:
        # row_sd's output words: canonical h in (yhi mod 2^29 : ylo); the bits above
        # are whatever the lazy sum left there (the helper masks them off)
        ylo = h & 0xFFFFFFFF
        yhi = (h >> 32) | (rng.randrange(8) << 29)
        hlo = (ylo + 1) & 0xFFFFFFFF
        hhi = (yhi & 0x1FFFFFFF) + (1 if hlo == 0 else 0)
        a = hhi >> 28
        hx = h + 1
        assert a == hx >> 60
        j = hx & ((1 << 60) - 1)
        for r in rs:
            umulhi = (hlo * r) >> 32
            wide = ((hhi & 0x0FFFFFFF) * r + umulhi) & ((1 << 64) - 1)
            assert (hhi & 0x0FFFFFFF) * r + umulhi < 1 << 64
            assert wide >> 28 == (r * j) >> 60, (h, r)
