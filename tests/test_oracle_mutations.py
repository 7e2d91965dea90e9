"""The oracle's pins catch plausible slips.  Each case plants one mistake in a
copy of oracle/ms_oracle.c (a dropped term, a flipped sign, a wrong bit, a
transposed operand, ...) in a temporary directory, builds it, and runs the
committed pin files (test_oracle_pins.py, test_anyr_pins.py) against that copy
in a subprocess: every mutant must make a pin fail, and the unmutated copy
must pass.  Mistakes are planted only in a temporary copy of the oracle, on
the CPU."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, text in ms_oracle.c, replacement): each text occurs exactly once
MUTANTS = [
    ("top term dropped", "for (int i = 0; i < k; ++i) {\n        acc = (acc + or_mulmod",
     "for (int i = 0; i < k - 1; ++i) {\n        acc = (acc + or_mulmod"),
    ("key not reduced mod p", "    x %= p;\n    u128 acc = 0;", "    u128 acc = 0;"),
    ("coefficients reversed", "or_mulmod(a[i] % p, xpow, p)", "or_mulmod(a[k - 1 - i] % p, xpow, p)"),
    ("sign flipped", "*sign = 1 - 2 * (int)bit;", "*sign = 2 * (int)bit - 1;"),
    ("bucket from the wrong bits", "*bucket = (u64)(h % m);", "*bucket = (u64)((h >> 1) % m);"),
    ("sign from the wrong bit", "u128 bit = g / half;", "u128 bit = (g / (half >> 1)) & 1;"),
    ("sign polynomial = bucket polynomial",
     "const u128* as = (mode & 1) ? ab + k : ab;\n            u64 bucket;\n            int sign;\n"
     "            or_split(p, b, c, k, m, mode, ab, as, x, &bucket, &sign);\n            u64* cell",
     "const u128* as = ab;\n            u64 bucket;\n            int sign;\n"
     "            or_split(p, b, c, k, m, mode, ab, as, x, &bucket, &sign);\n            u64* cell"),
    ("counter row shifted", "u64* cell = (u64*)&C[(u64)r * m + bucket];",
     "u64* cell = (u64*)&C[(u64)((r + 1) % t) * m + bucket];"),
    ("weights ignored", "int64_t wj = w ? (int64_t)w[j] : 1;", "int64_t wj = 1;"),
    ("median is the minimum", "unpack(v[t / 2], out_pair);", "unpack(v[0], out_pair);"),
    ("30-bit pieces cut to 29", "u128 piece = (x >> shift) & (((u128)1 << 30) - 1);",
     "u128 piece = (x >> shift) & (((u128)1 << 29) - 1);"),
    ("rejection keeps v = p", "} while (v >= p);", "} while (v > p);"),
    ("any-m map without the + 1", "u128 hx = h + 1;", "u128 hx = h;"),
    ("any-m sign 1 - 2a", "*sign = 2 * (int)(hx / half) - 1;", "*sign = 1 - 2 * (int)(hx / half);"),
]


def _workspace(tmp, source):
    """A minimal tree: the (mutated) oracle, the input generators, the pin files."""
    os.makedirs(os.path.join(tmp, "oracle"))
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), os.path.join(tmp, "oracle"))
    with open(os.path.join(tmp, "oracle", "ms_oracle.c"), "w") as f:
        f.write(source)
    shutil.copytree(os.path.join(ROOT, "datagen"), os.path.join(tmp, "datagen"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(os.path.join(tmp, "tests"))
    for name in ("test_oracle_pins.py", "test_anyr_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", name), os.path.join(tmp, "tests"))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(tmp, "tests", "golden"))
    with open(os.path.join(tmp, "tests", "conftest.py"), "w") as f:
        f.write("import os, sys\n"
                "sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))\n"
                "def pytest_configure(config):\n"
                "    config.addinivalue_line('markers', 'gpu: needs a GPU')\n"
                "    config.addinivalue_line('markers', 'slow: long CPU enumeration')\n")


def _run_pins(tmp):
    env = dict(os.environ)
    env.pop("PYTHONPATH", None)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu", "tests/test_oracle_pins.py", "tests/test_anyr_pins.py"],
                       cwd=tmp, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-3000:] + r.stderr[-2000:]


def test_every_planted_slip_fails_a_pin(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc is needed to build the oracle")
    src = open(os.path.join(ROOT, "oracle", "ms_oracle.c")).read()
    jobs = {"unmutated": src}
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, name
        jobs[name] = src.replace(old, new)
    dirs = {}
    for i, (name, code) in enumerate(jobs.items()):
        d = str(tmp_path / ("m%02d" % i))
        _workspace(d, code)
        dirs[name] = d
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        res = dict(zip(dirs, ex.map(_run_pins, dirs.values())))
    rc, out = res.pop("unmutated")
    assert rc == 0, "the unmutated copy must pass its pins:\n" + out
    survivors = [name for name, (rc, out) in res.items() if rc != 1 or " failed" not in out]
    assert not survivors, "slips no pin caught: %s\n%s" % (
        survivors, "\n".join(res[s][1] for s in survivors))
