"""CPU oracle for the Mersenne-hashing Count Sketch -- TEST INFRASTRUCTURE ONLY.

Plain, slow, definition-based reference (ms_oracle.c: unsigned __int128 with
the C `%` and `/` operators, no Mersenne tricks).  Only tests, the smoke check
and the benchmark's CPU-baseline leg may import this package; the library's
product path never does, and the two share no code.

128-bit values cross this interface as (n, 2) uint64 arrays of (lo, hi) limbs;
`to_int`/`from_ints` convert them to and from Python integers.

Parity pins for every function live in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ms_oracle.c")
_LIB = os.path.join(_HERE, "libms_oracle.so")
_lib = None

TWO_FOR_ONE = 0
TWO_POLY = 1
ANY_R = 2  # mode flag: any number of buckets m (not only powers of two)


def build(force: bool = False) -> str:
    """Compile ms_oracle.c into libms_oracle.so (gcc -O2; plain C11 + pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-o", tmp, _SRC,
                               "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u64, c_int, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
        lib.or_valid_prime_params.restype = c_int
        lib.or_valid_prime_params.argtypes = [c_int, u64]
        lib.or_splitmix64.argtypes = [u64, u64, vp]
        lib.or_draw_coeffs.argtypes = [c_int, u64, c_int, u64, u64, vp]
        lib.or_hash_eval.argtypes = [c_int, u64, c_int, vp, vp, c_int, u64, vp]
        lib.or_hash_many.argtypes = [c_int, u64, c_int, vp, u64, vp, u64, vp]
        lib.or_cs_update.argtypes = [c_int, u64, c_int, c_int, u64, c_int, vp, vp, c_int, vp, u64, vp]
        lib.or_cs_update_mt.argtypes = [c_int, u64, c_int, c_int, u64, c_int, vp, vp, c_int, vp, u64,
                                        vp, c_int]
        lib.or_cs_row_sumsq.argtypes = [c_int, u64, vp, vp]
        lib.or_cs_f2.argtypes = [c_int, u64, vp, vp]
        lib.or_cs_x_many.argtypes = [c_int, u64, c_int, u64, c_int, vp, u64, vp, c_int, vp, u64, vp]
        lib.or_cs_point_query.argtypes = [c_int, u64, c_int, c_int, u64, c_int, vp, vp, vp, c_int,
                                          u64, vp]
        lib.or_divmod.argtypes = [c_int, u64, vp, u64, vp, vp]
        lib.or_exact_f2.argtypes = [vp, vp, u64, vp]
        _lib = lib
    return _lib


# ---------------- 128-bit helpers ----------------

def to_int(pair) -> int:
    return int(pair[0]) | (int(pair[1]) << 64)


def to_ints(pairs: np.ndarray) -> list:
    pairs = np.asarray(pairs, dtype=np.uint64).reshape(-1, 2)
    return [int(lo) | (int(hi) << 64) for lo, hi in pairs]


def from_ints(values) -> np.ndarray:
    out = np.empty((len(values), 2), dtype=np.uint64)
    mask = (1 << 64) - 1
    for j, v in enumerate(values):
        out[j, 0] = v & mask
        out[j, 1] = (v >> 64) & mask
    return out


def prime(b: int, c: int) -> int:
    return (1 << b) - c


def _ptr(a):
    return None if a is None else a.ctypes.data


def _keys(keys: np.ndarray):
    """(array, key_kind) for uint32, uint64 or (n, 2) uint64 two-limb keys."""
    keys = np.ascontiguousarray(keys)
    if keys.dtype == np.uint32:
        return keys, 32, keys.shape[0]
    if keys.dtype == np.uint64 and keys.ndim == 1:
        return keys, 64, keys.shape[0]
    if keys.dtype == np.uint64 and keys.ndim == 2 and keys.shape[1] == 2:
        return keys, 128, keys.shape[0]
    raise TypeError("keys must be uint32[n], uint64[n] or uint64[n, 2]")


# ---------------- API ----------------

def splitmix64(seed: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    _load().or_splitmix64(seed, n, out.ctypes.data)
    return out


def draw_coeffs(b: int, c: int, k: int, nfun: int, seed: int) -> np.ndarray:
    """(nfun * k, 2) coefficient limbs, function-major, a_0 first."""
    out = np.empty((nfun * k, 2), dtype=np.uint64)
    _load().or_draw_coeffs(b, c, k, nfun, seed, out.ctypes.data)
    return out


def sketch_coeffs(b: int, c: int, k: int, t: int, mode: int, seed: int) -> np.ndarray:
    """Coefficients of a t-row sketch: t functions (two-for-one) or 2t functions
    ordered (row 0 bucket, row 0 sign, row 1 bucket, ...) in two-poly mode."""
    return draw_coeffs(b, c, k, t * (2 if mode & TWO_POLY else 1), seed)


def hash_eval(b: int, c: int, coeffs: np.ndarray, keys: np.ndarray) -> np.ndarray:
    coeffs = np.ascontiguousarray(coeffs, dtype=np.uint64).reshape(-1, 2)
    k = coeffs.shape[0]
    keys, kind, n = _keys(keys)
    out = np.empty((n, 2), dtype=np.uint64)
    _load().or_hash_eval(b, c, k, coeffs.ctypes.data, keys.ctypes.data, kind, n, out.ctypes.data)
    return out


def hash_many(b: int, c: int, k: int, coeffs: np.ndarray, key_pairs: np.ndarray) -> np.ndarray:
    """(nfun, nkeys, 2): every function applied to every (two-limb) key."""
    coeffs = np.ascontiguousarray(coeffs, dtype=np.uint64).reshape(-1, 2)
    key_pairs = np.ascontiguousarray(key_pairs, dtype=np.uint64).reshape(-1, 2)
    nfun = coeffs.shape[0] // k
    nkeys = key_pairs.shape[0]
    out = np.empty((nfun, nkeys, 2), dtype=np.uint64)
    _load().or_hash_many(b, c, k, coeffs.ctypes.data, nfun, key_pairs.ctypes.data, nkeys,
                         out.ctypes.data)
    return out


def cs_update(b: int, c: int, k: int, t: int, m: int, mode: int, coeffs: np.ndarray,
              keys: np.ndarray, weights=None, counters=None, nthreads: int = 1) -> np.ndarray:
    """counters (t, m) int64 += Count Sketch of the stream; returns counters."""
    coeffs = np.ascontiguousarray(coeffs, dtype=np.uint64).reshape(-1, 2)
    keys, kind, n = _keys(keys)
    if weights is not None:
        weights = np.ascontiguousarray(weights, dtype=np.int32)
        assert weights.shape[0] == n
    if counters is None:
        counters = np.zeros((t, m), dtype=np.int64)
    assert counters.dtype == np.int64 and counters.flags.c_contiguous
    if nthreads > 1:
        _load().or_cs_update_mt(b, c, k, t, m, mode, coeffs.ctypes.data, keys.ctypes.data, kind,
                                _ptr(weights), n, counters.ctypes.data, nthreads)
    else:
        _load().or_cs_update(b, c, k, t, m, mode, coeffs.ctypes.data, keys.ctypes.data, kind,
                             _ptr(weights), n, counters.ctypes.data)
    return counters


def row_sumsq(counters: np.ndarray) -> list:
    counters = np.ascontiguousarray(counters, dtype=np.int64)
    t, m = counters.shape
    out = np.empty((t, 2), dtype=np.uint64)
    _load().or_cs_row_sumsq(t, m, counters.ctypes.data, out.ctypes.data)
    return to_ints(out)


def f2_estimate(counters: np.ndarray) -> int:
    counters = np.ascontiguousarray(counters, dtype=np.int64)
    t, m = counters.shape
    out = np.empty(2, dtype=np.uint64)
    _load().or_cs_f2(t, m, counters.ctypes.data, out.ctypes.data)
    return to_int(out)


def cs_x_many(b: int, c: int, k: int, m: int, mode: int, coeffs: np.ndarray, keys: np.ndarray,
              weights=None) -> list:
    coeffs = np.ascontiguousarray(coeffs, dtype=np.uint64).reshape(-1, 2)
    nf = 2 if mode & TWO_POLY else 1
    nsets = coeffs.shape[0] // (nf * k)
    keys, kind, n = _keys(keys)
    if weights is not None:
        weights = np.ascontiguousarray(weights, dtype=np.int32)
    out = np.empty((nsets, 2), dtype=np.uint64)
    _load().or_cs_x_many(b, c, k, m, mode, coeffs.ctypes.data, nsets, keys.ctypes.data, kind,
                         _ptr(weights), n, out.ctypes.data)
    return out


def point_query(b: int, c: int, k: int, mode: int, coeffs: np.ndarray, counters: np.ndarray,
                keys: np.ndarray) -> np.ndarray:
    """Median over rows of s_r(x) C[r][i_r(x)] for each key (int64)."""
    coeffs = np.ascontiguousarray(coeffs, dtype=np.uint64).reshape(-1, 2)
    counters = np.ascontiguousarray(counters, dtype=np.int64)
    t, m = counters.shape
    keys, kind, n = _keys(keys)
    out = np.empty(n, dtype=np.int64)
    _load().or_cs_point_query(b, c, k, t, m, mode, coeffs.ctypes.data, counters.ctypes.data,
                              keys.ctypes.data, kind, n, out.ctypes.data)
    return out


def divmod_(b: int, c: int, v_pairs: np.ndarray):
    """(q, r) as (n, 2) limb arrays: q = v // p, r = v % p."""
    v_pairs = np.ascontiguousarray(v_pairs, dtype=np.uint64).reshape(-1, 2)
    n = v_pairs.shape[0]
    q = np.empty((n, 2), dtype=np.uint64)
    r = np.empty((n, 2), dtype=np.uint64)
    _load().or_divmod(b, c, v_pairs.ctypes.data, n, q.ctypes.data, r.ctypes.data)
    return q, r


def exact_f2(keys: np.ndarray, weights=None) -> int:
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    if weights is not None:
        weights = np.ascontiguousarray(weights, dtype=np.int32)
    out = np.empty(2, dtype=np.uint64)
    _load().or_exact_f2(keys.ctypes.data, _ptr(weights), keys.shape[0], out.ctypes.data)
    return to_int(out)


# ------------------------------------------------------------ wide division

def limbs_to_ints(a: np.ndarray) -> list[int]:
    """(n, L) little-endian uint64 limbs -> Python integers."""
    a = np.ascontiguousarray(a).view(np.uint64).reshape(a.shape[0], -1)
    out = []
    for row in a:
        v = 0
        for i in range(len(row) - 1, -1, -1):
            v = (v << 64) | int(row[i])
        out.append(v)
    return out


def ints_to_limbs(vals, nlimbs: int) -> np.ndarray:
    """Python integers (each < 2^(64 nlimbs)) -> (n, nlimbs) uint64 limbs."""
    out = np.zeros((len(vals), nlimbs), dtype=np.uint64)
    mask = (1 << 64) - 1
    for j, v in enumerate(vals):
        for i in range(nlimbs):
            out[j, i] = (v >> (64 * i)) & mask
    return out


def divmod_wide(b: int, c: int, v: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Quotient and remainder of wide values by p = 2^b - c, by definition
    (Python's integer floor division and remainder) -- the operation whose
    fast form is Algorithm division-generalized + mod-generalized (Sec. 1.5;
    Table 2 of Sec. 5 times it for 2b-bit values).  v: (n, ceil(2b/64)) limbs;
    the value used is v mod 2^(2b).  Returns (q, r) as (n, ceil((b+1)/64)) and
    (n, ceil(b/64)) limb arrays."""
    p = (1 << b) - c
    lq, lr = (b + 64) // 64, (b + 63) // 64
    qs, rs = [], []
    for x in limbs_to_ints(v):
        q, r = divmod(x % (1 << (2 * b)), p)
        qs.append(q)
        rs.append(r)
    return ints_to_limbs(qs, lq), ints_to_limbs(rs, lr)
