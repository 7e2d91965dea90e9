"""Guard bands around caller-owned outputs: each kernel that writes into a
caller's buffer writes exactly its n results.  Every output below is a slice
of a larger device buffer whose 64-element bands before and after it are
filled with a sentinel; after the call the bands must be intact and the slice
must equal the oracle."""
import numpy as np
import pytest

import datagen
import oracle
from test_gpu_parity import PRIMES, hash_to_np, make_keys, to_dev

pytestmark = pytest.mark.gpu

G = 64                      # guard elements (rows) on each side
S64 = 0x5A5A5A5A5A5A5A5A    # sentinel of an int64 element
S32 = 0x5A5A5A5A            # sentinel of an int32 element


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2008_08654_gb300 as ms
    assert torch.cuda.is_available()
    ms.lib()
    return torch, ms


def guarded(torch, rows, tail=(), dtype=None):
    """(full buffer, the slice of `rows` rows between the two bands)."""
    dtype = dtype or torch.int64
    s = S32 if dtype == torch.int32 else S64
    full = torch.full((rows + 2 * G,) + tuple(tail), s, dtype=dtype, device="cuda")
    return full, full[G:G + rows]


def intact(torch, full, rows):
    s = S32 if full.dtype == torch.int32 else S64
    torch.cuda.synchronize()
    return bool((full[:G] == s).all()) and bool((full[G + rows:] == s).all())


@pytest.mark.parametrize("n", [10007, 3])
@pytest.mark.parametrize("b,c", PRIMES)
def test_hash_eval_writes_only_its_outputs(env, b, c, n):
    torch, ms = env
    keys = make_keys(b, c, n, 77 + n)
    h = ms.Hash(k=4, b=b, c=c, seed=5)
    if b == 31:
        full, out = guarded(torch, n, dtype=torch.int32)
    elif b == 89:
        full, out = guarded(torch, n, (2,))
    else:
        full, out = guarded(torch, n)
    h.eval(to_dev(torch, keys), out=out)
    assert intact(torch, full, n)
    want = oracle.hash_eval(b, c, oracle.from_ints(h.coeffs()), keys)
    got = hash_to_np(torch, out, b)
    assert np.array_equal(got, want if b == 89 else want[:, 0])


@pytest.mark.parametrize("b,c", PRIMES)
def test_div_mod_write_only_their_outputs(env, b, c):
    torch, ms = env
    n = 9001
    v = datagen.u128_bits(3 * b, 128, n)
    fq, q = guarded(torch, n, (2,))
    fr, r = guarded(torch, n, (2,) if b > 64 else ())
    ms.div(b, c, to_dev(torch, v), q=q, r=r)
    assert intact(torch, fq, n) and intact(torch, fr, n)
    qw, rw = oracle.divmod_(b, c, v)
    assert np.array_equal(q.cpu().numpy().view(np.uint64), qw)
    got_r = r.cpu().numpy().view(np.uint64)
    assert np.array_equal(got_r, rw if b > 64 else rw[:, 0])
    fm, rm = guarded(torch, n, (2,) if b > 64 else ())
    ms.mod(b, c, to_dev(torch, v), r=rm)
    assert intact(torch, fm, n)
    assert np.array_equal(rm.cpu().numpy().view(np.uint64), got_r)


@pytest.mark.parametrize("b,c", [(61, 1), (89, 1)])
def test_point_query_and_f2_write_only_their_outputs(env, b, c):
    torch, ms = env
    n, t, m, k, seed = 20011, 5, 1024, 4, 19
    keys = make_keys(b, c, n, 8)
    sk = ms.Sketch(t=t, m=m, k=k, b=b, c=c, seed=seed)
    sk.update(to_dev(torch, keys))
    coeffs = oracle.sketch_coeffs(b, c, k, t, 0, seed)
    C = oracle.cs_update(b, c, k, t, m, 0, coeffs, keys)
    nq = 999
    fp, out = guarded(torch, nq)
    sk.point_query(to_dev(torch, keys[:nq]), out=out)
    assert intact(torch, fp, nq)
    assert np.array_equal(out.cpu().numpy(), oracle.point_query(b, c, k, 0, coeffs, C, keys[:nq]))
    fo, o = guarded(torch, 1, (2,))
    frows, rows = guarded(torch, t, (2,))
    sk.estimate_f2(out=o[0], rows=rows)
    assert intact(torch, fo, 1) and intact(torch, frows, t)
    assert ms.u128_to_int(o[0].cpu()) == oracle.f2_estimate(C)
    assert [ms.u128_to_int(x) for x in rows.cpu()] == oracle.row_sumsq(C)
