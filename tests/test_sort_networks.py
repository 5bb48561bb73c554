"""The fixed sorting networks of the KSG walk (ksg_dev.cuh) sort every input.

The comparator lists are read from the CUDA source as text and checked on all
0/1 inputs (Knuth's 0-1 principle: a comparator network that sorts every 0/1
sequence sorts every sequence), so a mistyped comparator fails here on the CPU.
"""
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2309_03308_gb300", "csrc",
                   "ksg_dev.cuh")


def networks():
    text = open(SRC).read()
    body = text[text.index("void sort_small("):]
    out = {}
    for m in re.finditer(r"N == (\d+)\) \{(.*?)\}", body, re.S):
        pairs = [(int(a), int(b)) for a, b in re.findall(r"ce\(t\[(\d+)\], t\[(\d+)\]\)",
                                                          m.group(2))]
        out[int(m.group(1))] = pairs
    return out


def sorts_all_binary(net, n):
    for bits in range(1 << n):
        v = [(bits >> i) & 1 for i in range(n)]
        for i, j in net:
            if v[i] > v[j]:
                v[i], v[j] = v[j], v[i]
        if any(v[i] > v[i + 1] for i in range(n - 1)):
            return False
    return True


def test_networks_found():
    nets = networks()
    assert set(nets) == {2, 4, 8, 10}
    assert [len(nets[n]) for n in (2, 4, 8, 10)] == [1, 5, 19, 29]


@pytest.mark.parametrize("n", [2, 4, 8, 10])
def test_network_sorts(n):
    net = networks()[n]
    assert all(0 <= i < j < n for i, j in net)
    assert sorts_all_binary(net, n)


def test_zero_one_check_catches_a_dropped_comparator():
    net = networks()[10]
    for drop in range(len(net)):
        assert not sorts_all_binary(net[:drop] + net[drop + 1:], 10), drop
