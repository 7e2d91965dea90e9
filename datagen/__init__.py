"""Seeded synthetic inputs for the Mersenne-hashing Count Sketch workloads.

This package only generates key, weight and value streams (see datagen.c for
the exact recipes).  It holds none of the method's arithmetic, and it is the
one module that both the CPU oracle tests and the CUDA path consume.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "datagen.c")
_LIB = os.path.join(_HERE, "libdatagen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile datagen.c into libdatagen.so next to it (gcc, -O2, pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC,
                               "-lpthread", "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u64, i32, c_int, dbl = ctypes.c_uint64, ctypes.c_int32, ctypes.c_int, ctypes.c_double
        vp = ctypes.c_void_p
        lib.dg_word.restype = u64
        lib.dg_word.argtypes = [u64, u64, u64]
        lib.dg_splitmix64_seq.argtypes = [u64, u64, vp]
        lib.dg_u64_below.argtypes = [u64, u64, u64, u64, vp, c_int]
        lib.dg_u32_below.argtypes = [u64, u64, u64, u64, vp, c_int]
        lib.dg_u128_bits.argtypes = [u64, u64, c_int, u64, vp, c_int]
        lib.dg_i32_range.argtypes = [u64, u64, i32, i32, u64, vp, c_int]
        lib.dg_zipf.argtypes = [u64, u64, dbl, dbl, c_int, u64, vp, c_int]
        lib.dg_unit_doubles.argtypes = [u64, u64, u64, vp]
        _lib = lib
    return _lib


def _threads(nthreads):
    if nthreads is None:
        return max(1, min(64, os.cpu_count() or 1))
    return int(nthreads)


# Stream identifiers: one per kind of input, so streams never overlap.
STREAM_KEYS = 1
STREAM_WEIGHTS = 2
STREAM_VALUES = 3
STREAM_ZIPF = 4
STREAM_LENGTHS = 5
STREAM_WIDTHS = 6
STREAM_ARRIVALS = 7
STREAM_KINDS = 8


def word(seed: int, stream: int, i: int) -> int:
    return int(_load().dg_word(seed, stream, i))


def splitmix64_sequence(seed: int, n: int) -> np.ndarray:
    """First n outputs of SplitMix64 started at state `seed`."""
    out = np.empty(n, dtype=np.uint64)
    _load().dg_splitmix64_seq(seed, n, out.ctypes.data)
    return out


def u64_below(seed: int, bound: int, n: int, stream: int = STREAM_KEYS, out=None,
              nthreads=None) -> np.ndarray:
    """n uint64 keys uniform in [0, bound); bound=0 means the full 64-bit range."""
    out = np.empty(n, dtype=np.uint64) if out is None else out
    _load().dg_u64_below(seed, stream, bound, n, out.ctypes.data, _threads(nthreads))
    return out


def u32_below(seed: int, bound: int, n: int, stream: int = STREAM_KEYS, out=None,
              nthreads=None) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32) if out is None else out
    _load().dg_u32_below(seed, stream, bound, n, out.ctypes.data, _threads(nthreads))
    return out


def u128_bits(seed: int, bits: int, n: int, stream: int = STREAM_VALUES, out=None,
              nthreads=None) -> np.ndarray:
    """n values uniform in [0, 2^bits) as an (n, 2) uint64 array of (lo, hi) limbs."""
    out = np.empty((n, 2), dtype=np.uint64) if out is None else out
    _load().dg_u128_bits(seed, stream, bits, n, out.ctypes.data, _threads(nthreads))
    return out


def i32_range(seed: int, lo: int, hi: int, n: int, stream: int = STREAM_WEIGHTS, out=None,
              nthreads=None) -> np.ndarray:
    """n int32 weights uniform in [lo, hi] inclusive."""
    out = np.empty(n, dtype=np.int32) if out is None else out
    _load().dg_i32_range(seed, stream, lo, hi, n, out.ctypes.data, _threads(nthreads))
    return out


def zipf(seed: int, alpha: float, n_ranks: int, n: int, map_to_keys: bool = True,
         stream: int = STREAM_ZIPF, out=None, nthreads=None) -> np.ndarray:
    """n Zipf(alpha) draws over ranks [1, n_ranks]; mapped to 61-bit keys if asked."""
    out = np.empty(n, dtype=np.uint64) if out is None else out
    _load().dg_zipf(seed, stream, float(alpha), float(n_ranks), 1 if map_to_keys else 0, n,
                    out.ctypes.data, _threads(nthreads))
    return out


def unit_doubles(seed: int, n: int, stream: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().dg_unit_doubles(seed, stream, n, out.ctypes.data)
    return out


def p89_keys(seed: int, n: int, stream: int = STREAM_KEYS, nthreads=None) -> np.ndarray:
    """Two-limb keys uniform in [0, 2^89 - 1): 89-bit draws, the single value
    2^89 - 1 (probability 2^-89) folded to 0."""
    v = u128_bits(seed, 89, n, stream=stream, nthreads=nthreads)
    allones = (v[:, 0] == np.uint64(0xFFFFFFFFFFFFFFFF)) & (v[:, 1] == np.uint64((1 << 25) - 1))
    v[allones] = 0
    return v
