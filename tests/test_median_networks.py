"""The comparator networks the point-query kernel takes the median of t = 5
and t = 7 row estimates with (k_update.cuh, median_of): read from the source as
written and checked on every 0/1 input -- a network of min/max operations
selects the middle value of every input exactly when it does so on every 0/1
input -- and, as a second check, on every ordering of distinct values and on
inputs with ties."""
import itertools
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2008_08654_gb300", "csrc", "k_update.cuh")


def network(t):
    text = open(SRC).read()
    body = text.split("// median network, t = %d" % t, 1)[1].split("return", 1)[0]
    ops = re.findall(r"med_(ce|lo|hi)\(e\[(\d+)\], e\[(\d+)\]\)", body)
    ret = re.search(r"return e\[(\d+)\];", text.split("// median network, t = %d" % t, 1)[1])
    return [(op, int(a), int(b)) for op, a, b in ops], int(ret.group(1))


def run(ops, out, values):
    v = list(values)
    for op, a, b in ops:
        lo, hi = min(v[a], v[b]), max(v[a], v[b])
        if op == "ce":
            v[a], v[b] = lo, hi
        elif op == "lo":
            v[a] = lo
        else:
            v[b] = hi
    return v[out]


@pytest.mark.parametrize("t", [5, 7])
def test_median_network_on_all_01_inputs(t):
    ops, out = network(t)
    assert ops and all(0 <= a < b < t for _, a, b in ops)
    for bits in itertools.product((0, 1), repeat=t):
        assert run(ops, out, bits) == sorted(bits)[t // 2], bits


@pytest.mark.parametrize("t", [5, 7])
def test_median_network_on_orderings_and_ties(t):
    ops, out = network(t)
    for perm in itertools.permutations(range(t)):
        assert run(ops, out, perm) == t // 2
    for vals in itertools.product((-2, 0, 5), repeat=t):
        assert run(ops, out, vals) == sorted(vals)[t // 2]
