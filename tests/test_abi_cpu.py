"""CPU-only checks of the C ABI library: it loads, exports every symbol the
public headers declare, validates arguments on the host, and draws the same
coefficients as the oracle.  No compute call reaches a GPU here."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ms():
    from paper_2008_08654_gb300 import _build
    if not _build.up_to_date():
        try:
            _build.build()
        except RuntimeError as e:  # pragma: no cover - no nvcc
            pytest.skip("cannot build libms.so here: %s" % e)
    import paper_2008_08654_gb300 as ms
    ms.lib()
    return ms


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z][a-z0-9_]*)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_headers_declare_the_abi():
    names = _declared_functions()
    for must in ("ms_hash_init", "ms_hash_eval", "ms_mod", "ms_div", "cs_create", "cs_update",
                 "cs_estimate_f2", "cs_point_query", "cs_merge", "cs_export", "cs_import"):
        assert must in names


def test_library_exports_every_declared_symbol(ms):
    lib = ms.lib()
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_does_not_import_oracle():
    src = open(os.path.join(ROOT, "paper_2008_08654_gb300", "__init__.py")).read()
    assert "oracle" not in re.sub(r'""".*?"""', "", src, flags=re.S)
    for f in glob.glob(os.path.join(ROOT, "paper_2008_08654_gb300", "csrc", "*")):
        assert "ms_oracle" not in open(f).read()
        assert "or_" + "hash" not in open(f).read()


def test_status_strings(ms):
    lib = ms.lib()
    assert lib.ms_status_str(0) == b"ok"
    assert lib.ms_status_str(2) == b"unsupported prime"
    assert ms.version() == "1.0.0"


@pytest.mark.parametrize("b,c", [(31, 1), (61, 1), (89, 1), (64, 59)])
@pytest.mark.parametrize("k", [1, 4, 8])
def test_hash_coefficients_match_oracle(ms, b, c, k):
    """ms_hash_init's host-side SplitMix64 draw equals the oracle's."""
    for seed in (0, 1, 1234567, 2 ** 64 - 1):
        h = ms.Hash(k=k, b=b, c=c, seed=seed)
        assert h.coeffs() == oracle.to_ints(oracle.draw_coeffs(b, c, k, 1, seed))


def test_explicit_coefficients_round_trip_and_range(ms):
    p = (1 << 61) - 1
    h = ms.Hash(b=61, c=1, coeffs=[0, 1, p - 1, 12345])
    assert h.coeffs() == [0, 1, p - 1, 12345]
    with pytest.raises(ms.MSError) as e:
        ms.Hash(b=61, c=1, coeffs=[p])
    assert e.value.status == 3
    p89 = (1 << 89) - 1
    assert ms.Hash(b=89, c=1, coeffs=[p89 - 1, 5]).coeffs() == [p89 - 1, 5]
    with pytest.raises(ms.MSError):
        ms.Hash(b=89, c=1, coeffs=[p89])
    with pytest.raises(ms.MSError):
        ms.Hash(b=64, c=59, coeffs=[(1 << 64) - 59])


def test_invalid_arguments_are_rejected_on_the_host(ms):
    lib = ms.lib()
    s = ctypes.c_void_p()
    bad = [
        ((4, 1024, 4, 61, 1, 0, 0), 1),     # even t
        ((17, 1024, 4, 61, 1, 0, 0), 1),    # t too large
        ((5, 1000, 4, 61, 1, 0, 0), 1),     # m not a power of two
        ((5, 1, 4, 61, 1, 0, 0), 1),        # m too small
        ((5, 1 << 25, 4, 61, 1, 0, 0), 1),  # m too large
        ((5, 1 << 20, 4, 31, 1, 0, 0), 0),  # allowed: 2^20 < 2^30
        ((5, 1024, 0, 61, 1, 0, 0), 1),     # k = 0
        ((5, 1024, 9, 61, 1, 0, 0), 1),     # k = 9
        ((5, 1024, 4, 61, 1, 0, 4), 1),     # bad mode
        ((5, 1024, 4, 61, 1, 0, 6), 1),     # bad mode bits with CS_ANY_R
        ((5, 1000, 4, 64, 59, 0, 2), 1),    # any m at 2^64-59 needs two polynomials
        ((5, 1, 4, 61, 1, 0, 2), 1),        # any m: m too small
        ((5, (1 << 24) + 1, 4, 61, 1, 0, 2), 1),  # any m: m too large
        ((5, (1 << 29) + 1, 4, 31, 1, 0, 2), 1),  # any m: m > 2^(b-2)
        ((5, 1024, 4, 62, 1, 0, 0), 2),     # unsupported prime
        ((5, 1024, 4, 64, 1, 0, 0), 2),
        ((5, 1024, 4, 61, 3, 0, 0), 2),
    ]
    for args, want in bad:
        if want == 0:
            continue  # would allocate device memory
        assert lib.cs_create(ctypes.byref(s), *args) == want, args
    assert lib.cs_create(None, 5, 1024, 4, 61, 1, 0, 0) == 1
    assert lib.ms_hash_init(ctypes.byref(s), 0, 61, 1, 0) == 1
    assert lib.ms_hash_init(ctypes.byref(s), 4, 61, 2, 0) == 2
    assert lib.ms_div(61, 1, None, None, None, 5, None) == 1
    assert lib.ms_div(62, 1, None, None, None, 5, None) == 2
    assert lib.ms_div(61, 1, None, None, None, 0, None) == 0   # n == 0: no-op
    assert lib.ms_mod(61, 1, None, None, 3, None) == 1
    assert lib.ms_div_wide(31, 1, None, None, None, 5, None) == 1     # b < 32
    assert lib.ms_div_wide(1025, 1, None, None, None, 5, None) == 1   # b > 1024
    assert lib.ms_div_wide(64, 1 << 32, None, None, None, 5, None) == 1
    assert lib.ms_div_wide(128, 1, None, None, None, 0, None) == 0    # n == 0: no-op
    assert lib.ms_div_wide(128, 1, None, None, None, 5, None) == 1    # null buffers
    assert lib.cs_update(None, None, None, 10, None) == 1
    assert lib.cs_estimate_f2(None, None, None, None) == 1
    assert lib.cs_merge(None, None, None) == 1
    assert lib.cs_import(ctypes.byref(s), b"not a sketch", 12) == 1


def test_hash_eval_rejects_bad_pointers_before_launch(ms):
    lib = ms.lib()
    h = ms.Hash(k=4, b=61, c=1, seed=1)
    assert lib.ms_hash_eval(h._h, None, None, 10, None) == 1
    assert lib.ms_hash_eval(h._h, None, None, 0, None) == 0
    assert lib.ms_hash_eval(h._h, ctypes.c_void_p(0x1003), ctypes.c_void_p(0x2000), 10, None) == 8


def test_probes_and_stats_hook_validate_on_the_host(ms):
    """The peak probes and the measurement hook reject bad arguments before
    touching a device."""
    lib = ms.lib()
    r, t = ctypes.c_double(), ctypes.c_double()
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: every call below fails validation
    assert lib.ms_probe_red(None, 1 << 20, 4, ctypes.byref(r), ctypes.byref(t)) == 1
    assert lib.ms_probe_red(fake, 1000, 4, ctypes.byref(r), ctypes.byref(t)) == 1   # not 2^j
    assert lib.ms_probe_red(fake, 16, 4, ctypes.byref(r), ctypes.byref(t)) == 1     # too small
    assert lib.ms_probe_red(fake, 1 << 32, 4, ctypes.byref(r), ctypes.byref(t)) == 1
    assert lib.ms_probe_red(fake, 1 << 20, 0, ctypes.byref(r), ctypes.byref(t)) == 1
    assert lib.ms_probe_red(fake, 1 << 20, 4, None, ctypes.byref(t)) == 1
    assert lib.ms_probe_red(ctypes.c_void_p((1 << 20) + 2), 1 << 20, 4, ctypes.byref(r),
                            ctypes.byref(t)) == 8                                   # misaligned
    assert lib.ms_probe_mul128(5, 16, fake, ctypes.byref(r), ctypes.byref(t)) == 1  # variant
    assert lib.cs_set_stats(None, None) == 1


def test_tracing_is_off_by_default_and_needs_no_nvtx_library(ms):
    """NVTX ranges are off unless asked for (MS_NVTX=1 or ms_set_tracing); the
    library links no NVTX library (the header-only NVTX v3 calls reach a
    profiler only when one injects itself), and with tracing on, entry points
    still validate and return normally in a process without a GPU."""
    import subprocess
    import sys
    out = subprocess.run(["readelf", "-d", ms.LIB_PATH], capture_output=True, text=True)
    if out.returncode == 0:
        needed = re.findall(r"\(NEEDED\)\s+Shared library: \[([^\]]+)\]", out.stdout)
        assert needed and not any("nvToolsExt" in n or "nvtx" in n.lower() for n in needed), needed
    code = ("import sys, ctypes; sys.path.insert(0, %r); import paper_2008_08654_gb300 as ms; "
            "lib = ms.lib(); on = ms.set_tracing(True); "
            "r = lib.cs_update(None, None, None, 10, None); "
            "again = ms.set_tracing(False); print(int(on), int(again), r)") % ROOT
    for env_val, first in (("", 0), ("1", 1)):
        env = dict(os.environ)
        env.pop("MS_NVTX", None)
        if env_val:
            env["MS_NVTX"] = env_val
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                           timeout=300)
        assert r.returncode == 0, r.stderr
        assert r.stdout.split() == [str(first), "1", "1"], r.stdout
