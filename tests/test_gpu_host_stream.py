"""cs_update_host: a stream in host memory, copied in chunks on the library's
copy stream while earlier chunks update, must give exactly the counters of
cs_update on the whole stream (and of the oracle)."""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2008_08654_gb300 as ms
    ms.lib()
    return torch, ms


@pytest.mark.parametrize("n", [1, 1000, (1 << 24) - 1, (1 << 24) + 7, 3 * (1 << 24) + 5])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_stream_equals_device_update(env, n, pinned):
    torch, ms = env
    keys = datagen.u64_below(n % 97 + 3, (1 << 61) - 1, n)
    w = datagen.i32_range(n % 89 + 5, -100, 100, n)
    kt = torch.from_numpy(keys.view(np.int64))
    wt = torch.from_numpy(w)
    if pinned:
        kt, wt = kt.pin_memory(), wt.pin_memory()
    a = ms.Sketch(t=5, m=1024, seed=21)
    a.update_host(kt if pinned else keys, wt if pinned else w)
    b = ms.Sketch(t=5, m=1024, seed=21)
    b.update(kt.cuda(), wt.cuda())
    torch.cuda.synchronize()
    A, B = a.counters().cpu().numpy(), b.counters().cpu().numpy()
    assert np.array_equal(A, B)
    if n <= 1 << 16:
        co = oracle.sketch_coeffs(61, 1, 4, 5, 0, 21)
        assert np.array_equal(A, oracle.cs_update(61, 1, 4, 5, 1024, 0, co, keys, w))


def test_host_stream_large_sketch_replicas_and_repeat(env):
    """Global replicas accumulate over every chunk and are reduced once; a
    second call adds the stream again (staging buffers reused)."""
    torch, ms = env
    n = 2 * (1 << 24) + 12345
    keys = torch.from_numpy(datagen.zipf(7, 1.1, 1 << 32, n).view(np.int64)).pin_memory()
    a = ms.Sketch(t=7, m=1 << 16, seed=3)
    a.update_host(keys)
    a.update_host(keys)
    b = ms.Sketch(t=7, m=1 << 16, seed=3)
    kd = keys.cuda()
    b.update(kd)
    b.update(kd)
    torch.cuda.synchronize()
    assert a.last_launch()["place"] == 2
    assert np.array_equal(a.counters().cpu().numpy(), b.counters().cpu().numpy())


@pytest.mark.parametrize("b,c", [(31, 1), (89, 1), (64, 59)])
def test_host_stream_other_primes(env, b, c):
    torch, ms = env
    n = (1 << 24) + 333
    p = (1 << b) - c
    if b == 31:
        keys = datagen.u32_below(5, 0, n)
    elif b == 89:
        keys = datagen.u128_bits(5, 128, n)
    else:
        keys = datagen.u64_below(5, 0, n)
    a = ms.Sketch(t=3, m=4096, b=b, c=c, seed=8)
    a.update_host(keys)
    d = ms.Sketch(t=3, m=4096, b=b, c=c, seed=8)
    kd = torch.from_numpy(keys.view(np.int32 if b == 31 else np.int64)).cuda()
    d.update(kd)
    torch.cuda.synchronize()
    assert np.array_equal(a.counters().cpu().numpy(), d.counters().cpu().numpy())
