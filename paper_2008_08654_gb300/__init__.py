"""Python binding of libms, the GB300 (sm_103a) Mersenne-prime hashing and
Count Sketch library (include/ms.h).

The binding only marshals arguments: every computation runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if libms.so is missing or a call fails, an exception is raised.

Names follow the C ABI: hash_init / Hash.eval (ms_hash_*), div / mod
(ms_div / ms_mod), Sketch (cs_*), probe_mul128 (ms_probe_mul128), probe_red
(ms_probe_red).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libms.so")

TWO_FOR_ONE = 0
TWO_POLY = 1
ANY_R = 2  # mode flag: any number of buckets m

PLACE_SMEM, PLACE_DSMEM, PLACE_GLOBAL = 0, 1, 2
STRAT_HORNER, STRAT_POWER_SUM = 0, 1

PRIMES = ((31, 1), (61, 1), (89, 1), (64, 59))

STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported prime", 3: "value out of range",
          4: "out of memory", 5: "CUDA error", 6: "timeout", 7: "busy", 8: "misaligned pointer"}


class MSError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = "%s failed: %s" % (where, STATUS.get(status, "status %d" % status))
        if detail:
            msg += " (" + detail + ")"
        super().__init__(msg)


class U128(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("hi", ctypes.c_uint64)]


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libms.so is not built (expected at %s); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, u32, u64, sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64,
                           ctypes.c_size_t)
    pp = ctypes.POINTER(ctypes.c_void_p)
    dbl = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    sigs = {
        "ms_status_str": (ctypes.c_char_p, [i]),
        "ms_last_cuda_error": (ctypes.c_char_p, []),
        "ms_version": (ctypes.c_char_p, []),
        "ms_set_tracing": (ctypes.c_int, [ctypes.c_int]),
        "ms_hash_init": (i, [pp, i, i, u64, u64]),
        "ms_hash_init_coeffs": (i, [pp, i, i, u64, vp]),
        "ms_hash_coeffs": (i, [vp, vp]),
        "ms_hash_params": (i, [vp, ip, ip, ctypes.POINTER(u64)]),
        "ms_hash_eval": (i, [vp, vp, vp, sz, vp]),
        "ms_hash_destroy": (i, [vp]),
        "ms_div": (i, [i, u64, vp, vp, vp, sz, vp]),
        "ms_mod": (i, [i, u64, vp, vp, sz, vp]),
        "ms_div_wide": (i, [i, u64, vp, vp, vp, sz, vp]),
        "ms_div_wide_steps": (i, [i, u64]),
        "cs_create": (i, [pp, i, u32, i, i, u64, u64, i]),
        "cs_create_coeffs": (i, [pp, i, u32, i, i, u64, i, vp]),
        "cs_destroy": (i, [vp]),
        "cs_params": (i, [vp, ip, ctypes.POINTER(u32), ip, ip, ctypes.POINTER(u64), ip]),
        "cs_row_stride": (i, [vp, ctypes.POINTER(u32)]),
        "cs_coeffs": (i, [vp, vp]),
        "cs_update": (i, [vp, vp, vp, sz, vp]),
        "cs_update_host": (i, [vp, vp, vp, sz, vp]),
        "cs_estimate_f2": (i, [vp, vp, vp, vp]),
        "cs_point_query": (i, [vp, vp, vp, sz, vp]),
        "cs_counters": (i, [vp, pp]),
        "cs_reset": (i, [vp, vp]),
        "cs_merge": (i, [vp, vp, vp]),
        "cs_export": (i, [vp, vp, ctypes.POINTER(sz), vp]),
        "cs_import": (i, [pp, vp, sz]),
        "cs_set_launch": (i, [vp, i, i, i, i, i, i, i, i]),
        "cs_last_launch": (i, [vp, ip, ip, ip, ip, ip, ip, ip, ip]),
        "ms_probe_mul128": (i, [i, i, vp, dbl, dbl]),
        "ms_probe_red": (i, [vp, sz, i, dbl, dbl]),
        "cs_set_stats": (i, [vp, vp]),
        "cs_batch_default_tuning": (i, [vp]),
        "cs_batch_create": (i, [pp, vp, i, vp, vp]),
        "cs_batch_launch": (i, [vp, vp]),
        "cs_batch_launch_direct": (i, [vp, vp]),
        "cs_batch_destroy": (i, [vp]),
        "cs_batch_info": (i, [vp, ctypes.POINTER(u64), ctypes.POINTER(u32), ip, ip,
                              ctypes.POINTER(sz)]),
        "cs_batch_tune": (i, [vp, i, vp, i, i, vp, ctypes.POINTER(ctypes.c_double), vp]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def lib():
    """The loaded ctypes library (loads it on first use)."""
    return _load()


def _check(st: int, where: str):
    if st != 0:
        detail = ""
        if st == 5:
            detail = _load().ms_last_cuda_error().decode(errors="replace")
        raise MSError(st, where, detail)


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor on a CUDA device")
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def key_dtype_bytes(b: int, c: int) -> int:
    return {(31, 1): 4, (61, 1): 8, (89, 1): 16, (64, 59): 8}[(b, c)]


def _nkeys(keys: torch.Tensor, b: int, c: int) -> int:
    kb = key_dtype_bytes(b, c)
    total = keys.numel() * keys.element_size()
    if total % kb:
        raise ValueError("key tensor size is not a multiple of the %d-byte key type" % kb)
    return total // kb


def _host_buffer(a, kb: int):
    """(pointer, element count of kb bytes) of a contiguous host numpy array or
    CPU tensor."""
    if isinstance(a, torch.Tensor):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("expected a contiguous host tensor")
        total, ptr = a.numel() * a.element_size(), a.data_ptr()
    else:
        a = np.ascontiguousarray(a)
        total, ptr = a.nbytes, a.ctypes.data
    if total % kb:
        raise ValueError("host buffer size is not a multiple of %d bytes" % kb)
    return ptr, total // kb


def _u128_array(values):
    arr = (U128 * len(values))()
    for j, v in enumerate(values):
        v = int(v)
        arr[j].lo = v & ((1 << 64) - 1)
        arr[j].hi = (v >> 64) & ((1 << 64) - 1)
    return arr


def version() -> str:
    return _load().ms_version().decode()


def set_tracing(on: bool) -> bool:
    """NVTX ranges around the library's entry points (ms_set_tracing); returns
    the previous setting."""
    return bool(_load().ms_set_tracing(1 if on else 0))


# ------------------------------------------------------------------ hashing

class Hash:
    """h(x) = sum_{i<k} a_i x^i mod p (ms_hash_*)."""

    def __init__(self, k: int = 4, b: int = 61, c: int = 1, seed: int = 0, coeffs=None):
        lib_ = _load()
        h = ctypes.c_void_p()
        if coeffs is None:
            _check(lib_.ms_hash_init(ctypes.byref(h), k, b, c, seed), "ms_hash_init")
        else:
            arr = _u128_array(coeffs)
            _check(lib_.ms_hash_init_coeffs(ctypes.byref(h), len(coeffs), b, c, arr),
                   "ms_hash_init_coeffs")
            k = len(coeffs)
        self._h = h
        self.k, self.b, self.c = k, b, c

    def coeffs(self) -> list:
        arr = (U128 * self.k)()
        _check(_load().ms_hash_coeffs(self._h, arr), "ms_hash_coeffs")
        return [a.lo | (a.hi << 64) for a in arr]

    def out_tensor(self, n: int, device=None) -> torch.Tensor:
        device = device or torch.device("cuda")
        if (self.b, self.c) == (31, 1):
            return torch.empty(n, dtype=torch.int32, device=device)
        if (self.b, self.c) == (89, 1):
            return torch.empty((n, 2), dtype=torch.int64, device=device)
        return torch.empty(n, dtype=torch.int64, device=device)

    def eval(self, keys: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        n = _nkeys(keys, self.b, self.c)
        if out is None:
            out = self.out_tensor(n, keys.device)
        _check(_load().ms_hash_eval(self._h, _ptr(keys), _ptr(out), n, _stream(stream)),
               "ms_hash_eval")
        return out

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ms_hash_destroy(self._h)
            self._h = None


def hash_init(k: int, b: int = 61, c: int = 1, seed: int = 0) -> Hash:
    return Hash(k, b, c, seed)


# ------------------------------------------------------------------ division

def div(b: int, c: int, v: torch.Tensor, q: torch.Tensor | None = None,
        r: torch.Tensor | None = None, want_q: bool = True, want_r: bool = True, stream=None):
    """q = v // p (as (n,2) limbs), r = v % p ((n,) for b <= 64, (n,2) for b = 89);
    v is an (n, 2) int64/uint64 tensor of (lo, hi) limbs."""
    n = v.numel() // 2
    if want_q and q is None:
        q = torch.empty((n, 2), dtype=torch.int64, device=v.device)
    if want_r and r is None:
        r = torch.empty((n, 2) if b > 64 else (n,), dtype=torch.int64, device=v.device)
    _check(_load().ms_div(b, c, _ptr(v), _ptr(q) if want_q else None,
                          _ptr(r) if want_r else None, n, _stream(stream)), "ms_div")
    return q, r


def mod(b: int, c: int, v: torch.Tensor, r: torch.Tensor | None = None, stream=None):
    n = v.numel() // 2
    if r is None:
        r = torch.empty((n, 2) if b > 64 else (n,), dtype=torch.int64, device=v.device)
    _check(_load().ms_mod(b, c, _ptr(v), _ptr(r), n, _stream(stream)), "ms_mod")
    return r


def div_wide(b: int, c: int, v: torch.Tensor, want_q: bool = True, want_r: bool = True,
             stream=None, q: torch.Tensor | None = None, r: torch.Tensor | None = None):
    """Quotient and remainder of wide values by p = 2^b - c (ms_div_wide).
    v: (n, ceil(2b/64)) int64/uint64 tensor of little-endian limbs.  Returns
    (q, r) as (n, ceil((b+1)/64)) and (n, ceil(b/64)) int64 tensors (or None);
    q and r may be passed in preallocated."""
    lv, lq, lr = (2 * b + 63) // 64, (b + 64) // 64, (b + 63) // 64
    if v.dim() != 2 or v.shape[1] != lv:
        raise ValueError("v must have shape (n, %d)" % lv)
    n = v.shape[0]
    if want_q and q is None:
        q = torch.empty((n, lq), dtype=torch.int64, device=v.device)
    if want_r and r is None:
        r = torch.empty((n, lr), dtype=torch.int64, device=v.device)
    q = q if want_q else None
    r = r if want_r else None
    _check(_load().ms_div_wide(b, c, _ptr(v), _ptr(q) if q is not None else None,
                               _ptr(r) if r is not None else None, n, _stream(stream)),
           "ms_div_wide")
    return q, r


def div_wide_steps(b: int, c: int) -> int:
    return int(_load().ms_div_wide_steps(b, c))


# ------------------------------------------------------------------ sketch

class _CudaView:
    def __init__(self, ptr: int, shape, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}
        self._owner = owner


class Sketch:
    """A t-row Count Sketch with m counters per row (cs_*)."""

    def __init__(self, t: int = 5, m: int = 1024, k: int = 4, b: int = 61, c: int = 1,
                 seed: int = 0, mode: int = TWO_FOR_ONE, coeffs=None, _handle=None):
        lib_ = _load()
        if _handle is not None:
            h = _handle
        else:
            h = ctypes.c_void_p()
            if coeffs is None:
                _check(lib_.cs_create(ctypes.byref(h), t, m, k, b, c, seed, mode), "cs_create")
            else:
                arr = _u128_array(coeffs)
                _check(lib_.cs_create_coeffs(ctypes.byref(h), t, m, k, b, c, mode, arr),
                       "cs_create_coeffs")
        self._h = h
        tt, mm, kk, bb, md = ctypes.c_int(), ctypes.c_uint32(), ctypes.c_int(), ctypes.c_int(), \
            ctypes.c_int()
        cc = ctypes.c_uint64()
        _check(lib_.cs_params(h, ctypes.byref(tt), ctypes.byref(mm), ctypes.byref(kk),
                              ctypes.byref(bb), ctypes.byref(cc), ctypes.byref(md)), "cs_params")
        self.t, self.m, self.k, self.b, self.c, self.mode = (tt.value, mm.value, kk.value,
                                                             bb.value, cc.value, md.value)
        st = ctypes.c_uint32()
        _check(lib_.cs_row_stride(h, ctypes.byref(st)), "cs_row_stride")
        self.stride = st.value  # counters per row in memory (> m only for ANY_R sketches)

    @property
    def handle(self):
        return self._h

    def coeffs(self) -> list:
        n = self.t * self.k * (2 if self.mode & TWO_POLY else 1)
        arr = (U128 * n)()
        _check(_load().cs_coeffs(self._h, arr), "cs_coeffs")
        return [a.lo | (a.hi << 64) for a in arr]

    def update(self, keys: torch.Tensor, weights: torch.Tensor | None = None, stream=None):
        n = _nkeys(keys, self.b, self.c)
        if weights is not None and weights.numel() != n:
            raise ValueError("weights must have one entry per key")
        if weights is not None and weights.dtype != torch.int32:
            raise TypeError("weights must be int32")
        _check(_load().cs_update(self._h, _ptr(keys), _ptr(weights), n, _stream(stream)),
               "cs_update")

    def update_host(self, keys, weights=None, stream=None):
        """cs_update_host: keys (and int32 weights) in host memory -- numpy arrays
        or CPU tensors, pinned for asynchronous copies.  Keep them alive until
        `stream` is synchronized."""
        kp, n = _host_buffer(keys, key_dtype_bytes(self.b, self.c))
        wp = None
        if weights is not None:
            wp, nw = _host_buffer(weights, 4)
            if nw != n:
                raise ValueError("weights must have one entry per key")
            if (weights.dtype != torch.int32) if isinstance(weights, torch.Tensor) else \
                    (np.asarray(weights).dtype != np.int32):
                raise TypeError("weights must be int32")
        _check(_load().cs_update_host(self._h, kp, wp, n, _stream(stream)), "cs_update_host")

    def estimate_f2(self, out: torch.Tensor | None = None, rows: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
        """Device tensor (2,) int64 holding the 128-bit estimate as (lo, hi)."""
        if out is None:
            out = torch.empty(2, dtype=torch.int64, device="cuda")
        _check(_load().cs_estimate_f2(self._h, _ptr(out), _ptr(rows), _stream(stream)),
               "cs_estimate_f2")
        return out

    def f2(self) -> int:
        """The F2 estimate as a Python int (synchronizes)."""
        o = self.estimate_f2().cpu()
        return u128_to_int(o)

    def row_values(self) -> list:
        rows = torch.empty((self.t, 2), dtype=torch.int64, device="cuda")
        self.estimate_f2(rows=rows)
        return [u128_to_int(r) for r in rows.cpu()]

    def point_query(self, keys: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        n = _nkeys(keys, self.b, self.c)
        if out is None:
            out = torch.empty(n, dtype=torch.int64, device=keys.device)
        _check(_load().cs_point_query(self._h, _ptr(keys), _ptr(out), n, _stream(stream)),
               "cs_point_query")
        return out

    def counters(self, padded: bool = False) -> torch.Tensor:
        """Zero-copy (t, m) int64 view of the library-owned counters (rows are
        `stride` apart in memory; padded=True returns the full (t, stride))."""
        p = ctypes.c_void_p()
        _check(_load().cs_counters(self._h, ctypes.byref(p)), "cs_counters")
        full = torch.as_tensor(_CudaView(p.value, (self.t, self.stride), "<i8", self),
                               device="cuda")
        return full if padded or self.stride == self.m else full[:, :self.m]

    def reset(self, stream=None):
        _check(_load().cs_reset(self._h, _stream(stream)), "cs_reset")

    def merge(self, other: "Sketch", stream=None):
        _check(_load().cs_merge(self._h, other._h, _stream(stream)), "cs_merge")

    def export(self, stream=None) -> bytes:
        size = ctypes.c_size_t(0)
        _check(_load().cs_export(self._h, None, ctypes.byref(size), _stream(stream)), "cs_export")
        buf = ctypes.create_string_buffer(size.value)
        _check(_load().cs_export(self._h, buf, ctypes.byref(size), _stream(stream)), "cs_export")
        return buf.raw[:size.value]

    @classmethod
    def import_(cls, data: bytes) -> "Sketch":
        h = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(data, len(data))
        _check(_load().cs_import(ctypes.byref(h), buf, len(data)), "cs_import")
        return cls(_handle=h)

    def set_launch(self, place: int = -1, strategy: int = -1, threads: int = 0, blocks: int = 0,
                   blocks_per_sm: int = 0, cluster: int = 0, replicas: int = 0,
                   aggregate: int = -1):
        _check(_load().cs_set_launch(self._h, place, strategy, threads, blocks, blocks_per_sm,
                                     cluster, replicas, aggregate), "cs_set_launch")

    def set_stats(self, hashed=None):
        """Measurement hook: later updates add the entries they hash (t polynomial
        evaluations and t counter additions each) into `hashed`, a one-element
        int64 CUDA tensor; None turns it off."""
        if hashed is not None and (hashed.dtype != torch.int64 or hashed.numel() < 1):
            raise ValueError("hashed must be a one-element int64 CUDA tensor")
        _check(_load().cs_set_stats(self._h, None if hashed is None else _ptr(hashed)),
               "cs_set_stats")
        self._stats = hashed  # keep the counter alive while the library holds it

    def last_launch(self) -> dict:
        v = [ctypes.c_int() for _ in range(8)]
        _check(_load().cs_last_launch(self._h, *[ctypes.byref(x) for x in v]), "cs_last_launch")
        keys = ("place", "strategy", "threads", "blocks", "cluster", "smem", "specialized",
                "replicas")
        return dict(zip(keys, [x.value for x in v]))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.cs_destroy(self._h)
            self._h = None


# ------------------------------------------------------------------ helpers

def u128_to_int(t) -> int:
    lo, hi = int(t[0]), int(t[1])
    return (lo & ((1 << 64) - 1)) | ((hi & ((1 << 64) - 1)) << 64)


def probe_mul128(variant: int = 0, iters: int = 4096) -> tuple:
    """(products per second, kernel ms) of the integer-multiply probe."""
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    rate, ms = ctypes.c_double(), ctypes.c_double()
    _check(_load().ms_probe_mul128(variant, iters, _ptr(sink), ctypes.byref(rate),
                                   ctypes.byref(ms)), "ms_probe_mul128")
    return rate.value, ms.value


def probe_red(words: int = 1 << 22, iters: int = 256) -> tuple:
    """(scattered int32 atomic additions per second, kernel ms) into a buffer of
    `words` int32 (4 * 2^22 bytes = 16 MiB by default, L2-resident)."""
    buf = torch.zeros(words, dtype=torch.int32, device="cuda")
    rate, ms = ctypes.c_double(), ctypes.c_double()
    _check(_load().ms_probe_red(_ptr(buf), words, iters, ctypes.byref(rate), ctypes.byref(ms)),
           "ms_probe_red")
    return rate.value, ms.value


# ------------------------------------------------------------------ batched

class BatchJob(ctypes.Structure):
    _fields_ = [("sketch", ctypes.c_void_p), ("keys_dev", ctypes.c_void_p),
                ("weights_dev", ctypes.c_void_p), ("n", ctypes.c_uint64)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("chunk_keys", ctypes.c_uint32), ("smem_min_ratio", ctypes.c_uint32),
                ("rows_per_item", ctypes.c_int), ("strategy", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}

    @classmethod
    def from_dict(cls, d: dict) -> "BatchTuning":
        t = default_tuning()
        for k, v in d.items():
            setattr(t, k, v)
        return t


def default_tuning() -> BatchTuning:
    t = BatchTuning()
    _check(_load().cs_batch_default_tuning(ctypes.byref(t)), "cs_batch_default_tuning")
    return t


def _job_array(jobs):
    arr = (BatchJob * len(jobs))()
    keep = []
    for j, (sk, keys, w) in enumerate(jobs):
        n = _nkeys(keys, sk.b, sk.c)
        arr[j].sketch = sk.handle
        arr[j].keys_dev = _ptr(keys) if n else None
        arr[j].weights_dev = _ptr(w) if w is not None else None
        arr[j].n = n
        keep.append((sk, keys, w))
    return arr, keep


class Batch:
    """One persistent, graph-captured launch over many (sketch, keys, weights)
    jobs (cs_batch_*).  The tensors and sketches must outlive the plan."""

    def __init__(self, jobs, tuning: BatchTuning | dict | None = None):
        arr, self._keep = _job_array(jobs)
        if isinstance(tuning, dict):
            tuning = BatchTuning.from_dict(tuning)
        h = ctypes.c_void_p()
        _check(_load().cs_batch_create(ctypes.byref(h), arr, len(jobs),
                                       ctypes.byref(tuning) if tuning is not None else None,
                                       None), "cs_batch_create")
        self._h = h

    def launch(self, stream=None):
        _check(_load().cs_batch_launch(self._h, _stream(stream)), "cs_batch_launch")

    def launch_direct(self, stream=None):
        _check(_load().cs_batch_launch_direct(self._h, _stream(stream)), "cs_batch_launch_direct")

    def info(self) -> dict:
        tk, ti = ctypes.c_uint64(), ctypes.c_uint32()
        bl, th, sm = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        _check(_load().cs_batch_info(self._h, ctypes.byref(tk), ctypes.byref(ti), ctypes.byref(bl),
                                     ctypes.byref(th), ctypes.byref(sm)), "cs_batch_info")
        return {"total_keys": tk.value, "total_items": ti.value, "blocks": bl.value,
                "threads": th.value, "smem": sm.value}

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.cs_batch_destroy(self._h)
            self._h = None


def tune_batched(jobs, candidates, reps: int = 3, stream=None):
    """Times every candidate tuning (dicts or BatchTuning) on the real jobs;
    returns (best tuning as a dict, list of median ms per candidate; -1 when a
    candidate could not launch).  Counters are left as they were."""
    arr, keep = _job_array(jobs)
    cands = (BatchTuning * len(candidates))()
    for i, c in enumerate(candidates):
        cands[i] = BatchTuning.from_dict(c) if isinstance(c, dict) else c
    best = BatchTuning()
    times = (ctypes.c_double * len(candidates))()
    _check(_load().cs_batch_tune(arr, len(jobs), cands, len(candidates), reps, ctypes.byref(best),
                                 times, _stream(stream)), "cs_batch_tune")
    return best.as_dict(), list(times)


# ------------------------------------------------------------------ serving

class ServerConfig(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int), ("k", ctypes.c_int), ("b", ctypes.c_int),
                ("c", ctypes.c_uint64), ("mode", ctypes.c_int), ("seed_base", ctypes.c_uint64),
                ("num_sketches", ctypes.c_int), ("m_per_sketch", ctypes.POINTER(ctypes.c_uint32)),
                ("staging_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_int),
                ("max_batch_keys", ctypes.c_uint64), ("max_batch_requests", ctypes.c_int),
                ("timeout_s", ctypes.c_double)]


class RequestResult(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int), ("status", ctypes.c_int), ("f2", U128),
                ("submit_s", ctypes.c_double), ("done_s", ctypes.c_double)]


class LoadSpec(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("count", ctypes.c_uint64),
                ("rate_per_s", ctypes.c_double), ("query_fraction", ctypes.c_double),
                ("min_keys", ctypes.c_uint64), ("max_keys", ctypes.c_uint64),
                ("key_pool_host", ctypes.c_void_p), ("pool_keys", ctypes.c_uint64)]


class LoadResult(ctypes.Structure):
    _fields_ = [("wall_s", ctypes.c_double), ("keys_per_s", ctypes.c_double),
                ("update_p50_ms", ctypes.c_double), ("update_p99_ms", ctypes.c_double),
                ("query_p50_ms", ctypes.c_double), ("query_p99_ms", ctypes.c_double),
                ("updates", ctypes.c_uint64), ("queries", ctypes.c_uint64),
                ("keys", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("offered_keys_per_s", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_SERVER_SIGS = {
    "ms_server_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]),
    "ms_server_submit_update": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_uint64)]),
    "ms_server_submit_query": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_uint64)]),
    "ms_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
    "ms_server_drain": (ctypes.c_int, [ctypes.c_void_p]),
    "ms_server_sketch_counters": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "ms_server_stats": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_uint64)] * 3),
    "ms_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "ms_server_run_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
}


def _server_lib():
    lib_ = _load()
    if not getattr(lib_, "_ms_server_sigs", False):
        for name, (res, args) in _SERVER_SIGS.items():
            f = getattr(lib_, name)
            f.restype = res
            f.argtypes = args
        lib_._ms_server_sigs = True
    return lib_


class Server:
    """Continuous batching over device-resident sketches (ms_server_*).
    Host buffers passed to submit_update are kept referenced until drain()."""

    def __init__(self, widths, t=5, k=4, b=61, c=1, mode=TWO_FOR_ONE, seed_base=0,
                 staging_bytes=1 << 30, max_inflight=1024, max_batch_keys=1 << 24,
                 max_batch_requests=1024, timeout_s=60.0):
        lib_ = _server_lib()
        self._widths = (ctypes.c_uint32 * len(widths))(*widths)
        cfg = ServerConfig(t, k, b, c, mode, seed_base, len(widths), self._widths, staging_bytes,
                           max_inflight, max_batch_keys, max_batch_requests, timeout_s)
        h = ctypes.c_void_p()
        _check(lib_.ms_server_create(ctypes.byref(h), ctypes.byref(cfg)), "ms_server_create")
        self._h = h
        self.t, self.k, self.b, self.c = t, k, b, c
        self.widths = list(widths)
        self._keep = []

    @staticmethod
    def _host_ptr(a):
        if a is None:
            return None, None
        if isinstance(a, torch.Tensor):
            assert not a.is_cuda and a.is_contiguous()
            return a, a.data_ptr()
        return a, a.ctypes.data

    def submit_update(self, sketch_id: int, keys, weights=None, try_only=False) -> int:
        kobj, kp = self._host_ptr(keys)
        wobj, wp = self._host_ptr(weights)
        n = kobj.numel() if isinstance(kobj, torch.Tensor) else len(kobj)
        if self.b == 89:
            n //= 2 if (isinstance(kobj, torch.Tensor) and kobj.dim() == 1) else 1
        tk = ctypes.c_uint64()
        st = _server_lib().ms_server_submit_update(self._h, sketch_id, kp, wp, n,
                                                   1 if try_only else 0, ctypes.byref(tk))
        _check(st, "ms_server_submit_update")
        self._keep.append((kobj, wobj))
        return tk.value

    def submit_query(self, sketch_id: int, try_only=False) -> int:
        tk = ctypes.c_uint64()
        _check(_server_lib().ms_server_submit_query(self._h, sketch_id, 1 if try_only else 0,
                                                    ctypes.byref(tk)), "ms_server_submit_query")
        return tk.value

    def poll(self, ticket: int) -> dict:
        r = RequestResult()
        _check(_server_lib().ms_server_poll(self._h, ticket, ctypes.byref(r)), "ms_server_poll")
        return {"done": bool(r.done), "status": r.status, "f2": r.f2.lo | (r.f2.hi << 64),
                "submit_s": r.submit_s, "done_s": r.done_s}

    def drain(self):
        _check(_server_lib().ms_server_drain(self._h), "ms_server_drain")
        self._keep.clear()

    def counters(self, sketch_id: int):
        import numpy as np
        out = np.empty((self.t, self.widths[sketch_id]), dtype=np.int64)
        _check(_server_lib().ms_server_sketch_counters(self._h, sketch_id, out.ctypes.data),
               "ms_server_sketch_counters")
        return out

    def stats(self) -> dict:
        v = [ctypes.c_uint64() for _ in range(3)]
        _check(_server_lib().ms_server_stats(self._h, *[ctypes.byref(x) for x in v]),
               "ms_server_stats")
        return {"requests_done": v[0].value, "keys_done": v[1].value, "batches": v[2].value}

    def run_load(self, pool, count, rate_per_s, query_fraction=0.1, min_keys=256,
                 max_keys=1 << 20, seed=0) -> dict:
        pobj, pp = self._host_ptr(pool)
        npool = pobj.numel() if isinstance(pobj, torch.Tensor) else len(pobj)
        spec = LoadSpec(seed, count, rate_per_s, query_fraction, min_keys, max_keys, pp, npool)
        res = LoadResult()
        _check(_server_lib().ms_server_run_load(self._h, ctypes.byref(spec), ctypes.byref(res)),
               "ms_server_run_load")
        return res.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            _check(_server_lib().ms_server_destroy(self._h), "ms_server_destroy")
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
