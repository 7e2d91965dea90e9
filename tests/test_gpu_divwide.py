"""ms_div_wide on the GPU (Table 2 sizes, b up to 1024) against the oracle's
definition, limb for limb."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

CASES = [(32, 1), (32, 3), (33, 1), (61, 1), (64, 1), (64, 59), (65, 1), (100, 1), (127, 1),
         (128, 1), (128, 159), (129, 7), (255, 19), (256, 1), (511, 1), (512, 569), (777, 12345),
         (1000, 1), (1023, 1), (1024, 1), (1024, 105), (1024, (1 << 31) - 1)]


def _inputs(b, c, n, seed):
    p = (1 << b) - c
    top = (1 << (2 * b)) - 1
    lv = (2 * b + 63) // 64
    edges = [0, 1, 2, p - 1, p, p + 1, 2 * p - 1, 2 * p, p * p - 1, p * p, p * p + 1, top, top - 1,
             (top // p) * p, (top // p) * p - 1, (1 << b) - 1, 1 << b, 3 * p + 2]
    edges = [v for v in edges if 0 <= v <= top]
    rng = np.random.default_rng(seed)
    raw = rng.integers(0, 1 << 63, size=(n, lv), dtype=np.uint64) * 2 + \
        rng.integers(0, 2, size=(n, lv), dtype=np.uint64)   # full 64-bit limbs, junk above 2b
    return np.concatenate([oracle.ints_to_limbs(edges, lv), raw])


@pytest.mark.parametrize("b,c", CASES)
def test_div_wide_matches_oracle(b, c):
    import torch
    import paper_2008_08654_gb300 as ms
    v = _inputs(b, c, 3000, b * 1000 + c % 997)
    want_q, want_r = oracle.divmod_wide(b, c, v)
    vd = torch.from_numpy(v.view(np.int64)).cuda()
    q, r = ms.div_wide(b, c, vd)
    torch.cuda.synchronize()
    assert np.array_equal(q.cpu().numpy().view(np.uint64), want_q)
    assert np.array_equal(r.cpu().numpy().view(np.uint64), want_r)
    q2, none = ms.div_wide(b, c, vd, want_r=False)
    none2, r2 = ms.div_wide(b, c, vd, want_q=False)
    torch.cuda.synchronize()
    assert none is None and none2 is None
    assert np.array_equal(q2.cpu().numpy().view(np.uint64), want_q)
    assert np.array_equal(r2.cpu().numpy().view(np.uint64), want_r)


def test_div_wide_ragged_counts():
    """Counts that leave a warp's segments partly empty, and n = 0."""
    import torch
    import paper_2008_08654_gb300 as ms
    for b, n in ((64, 1), (64, 17), (128, 5), (1024, 1), (1024, 3), (200, 33)):
        v = _inputs(b, 1, n, n)[:n]
        want_q, want_r = oracle.divmod_wide(b, 1, v)
        q, r = ms.div_wide(b, 1, torch.from_numpy(v.view(np.int64)).cuda())
        assert np.array_equal(q.cpu().numpy().view(np.uint64), want_q)
        assert np.array_equal(r.cpu().numpy().view(np.uint64), want_r)
    q, r = ms.div_wide(64, 1, torch.zeros((0, 2), dtype=torch.int64, device="cuda"))
    assert q.shape == (0, 2) and r.shape == (0, 1)


def test_div_wide_rejects_bad_args():
    import torch
    import paper_2008_08654_gb300 as ms
    v = torch.zeros((4, 2), dtype=torch.int64, device="cuda")
    for b, c in ((31, 1), (1025, 1), (64, 1 << 33), (40, 1 << 20)):
        lv = (2 * b + 63) // 64
        with pytest.raises(ms.MSError) as e:
            ms.div_wide(b, c, torch.zeros((4, lv), dtype=torch.int64, device="cuda"))
        assert e.value.status == 1
