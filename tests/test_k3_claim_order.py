"""Host logic of the k = 3 tensor-core scan's dynamic schedule (no GPU): the
order in which CTAs claim tiles is a permutation of all (item, discretisation)
tiles, by descending modelled cost (warps with a valid row times valid
columns, at least 0.75 of a full item), ties in tile order.  The items and
the model are restated here from their definitions."""
import ctypes
import math

import numpy as np
import pytest

from paper_1811_00631_gb300 import mdfs


@pytest.fixture(scope="module")
def lib():
    from paper_1811_00631_gb300 import build
    build.build()
    return mdfs.load()


def _items(M):
    out = []
    for b in range(1, M - 1):
        nta = (b + 127) // 128
        nte = (M - 1 - b + 255) // 256
        for ta in range(nta):
            for te in range(nte):
                out.append((b, ta, te))
    return out


def _cost(M, b, ta, te):
    a0 = b - 128 * (ta + 1) if b & 1 else 128 * ta
    e0 = b + 1 + 256 * te
    warps = sum(1 for q in range(4) if a0 + 32 * q < b and a0 + 32 * q + 31 >= 0)
    return max(0.75, warps * 32.0 * min(256, M - e0) / (128.0 * 256.0))


@pytest.mark.parametrize("M,nd", [(3, 1), (4, 2), (130, 3), (500, 2), (700, 1)])
def test_claim_order_is_a_cost_sorted_permutation(lib, M, nd):
    n = lib.mdfs_testing_k3_claim_order(M, nd, None, 0)
    items = _items(M)
    assert n == len(items) * nd
    order = np.zeros(max(n, 1), dtype=np.int32)
    assert lib.mdfs_testing_k3_claim_order(M, nd, ctypes.c_void_p(order.ctypes.data), n) == n
    order = order[:n]
    assert np.array_equal(np.sort(order), np.arange(n))
    cost = np.array([_cost(M, *items[t % len(items)]) for t in order])
    assert np.all(np.diff(cost) <= 0)
    for i in range(1, n):  # ties keep tile order
        if cost[i] == cost[i - 1]:
            assert order[i] > order[i - 1]
    if n:
        assert math.isclose(cost[0], max(_cost(M, *it) for it in items))


def test_claim_order_arguments(lib):
    assert lib.mdfs_testing_k3_claim_order(2, 1, None, 0) == -1
    assert lib.mdfs_testing_k3_claim_order(10, 0, None, 0) == -1
    assert lib.mdfs_testing_k3_claim_order(10, 1, None, 5) == -1
