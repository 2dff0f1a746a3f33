"""Pins of the oracle's contrast variables, p-value adjustment and selection
pipeline (section "Canonical package usage" of arXiv 1811.00631), CPU only.

Each pin checks a property fixed by the definitions rather than retyping them:
the shuffle is a bijection with uniform images, every contrast row is a
permutation of its source row, BH / BY agree with scipy's implementation,
Holm / Hochberg agree with the sequential rejection procedures they are
defined by, and the pipeline controls false selections on null data while
finding planted signal.
"""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("n", list(range(1, 40)) + [63, 64, 65, 255, 256, 257, 1000, 2000])
def test_shuffle_is_a_bijection(n):
    for stream, seed in [(0, 1), (7, 2**40 + 3), (0xFFFFFFFF, 12345)]:
        img = [oracle.shuffle_index(i, n, stream, seed) for i in range(n)]
        assert sorted(img) == list(range(n))


def test_shuffle_images_are_uniform():
    """pi(0) over 6000 streams is uniform on [0, 6); pairs (pi(0), pi(1)) are
    uniform over the 30 ordered pairs (chi-square tests at 1e-4)."""
    from scipy.stats import chisquare
    n, S = 6, 6000
    first = np.zeros(n)
    pairs = np.zeros((n, n))
    for s in range(S):
        a = oracle.shuffle_index(0, n, s, 77)
        b = oracle.shuffle_index(1, n, s, 77)
        first[a] += 1
        pairs[a, b] += 1
    assert chisquare(first).pvalue > 1e-4
    off = pairs[~np.eye(n, dtype=bool)]
    assert np.all(np.diag(pairs) == 0)
    assert chisquare(off).pvalue > 1e-4


def test_shuffles_differ_between_streams_and_seeds():
    n = 1000
    base = [oracle.shuffle_index(i, n, 0, 5) for i in range(n)]
    other_stream = [oracle.shuffle_index(i, n, 1, 5) for i in range(n)]
    other_seed = [oracle.shuffle_index(i, n, 0, 6) for i in range(n)]
    assert base != other_stream and base != other_seed
    # a random permutation has about one fixed point
    assert sum(int(a == i) for i, a in enumerate(base)) < 8


def test_contrast_rows_are_shuffled_copies():
    rng = np.random.default_rng(3)
    M, N, nc = 9, 257, 20
    x = rng.standard_normal((M, N)).astype(np.float32)
    xe, src = oracle.contrast(x, nc, seed=99)
    assert xe.shape == (M + nc, N)
    assert np.array_equal(xe[:M], x)
    assert np.all((src >= 0) & (src < M))
    # without replacement while j < M: the first M sources are a permutation
    assert sorted(src[:M].tolist()) == list(range(M))
    assert np.array_equal(src[M:], src[: nc - M])  # source of j is the same map at j mod M
    for j in range(nc):
        assert np.array_equal(np.sort(xe[M + j]), np.sort(x[src[j]]))
        assert not np.array_equal(xe[M + j], x[src[j]])


def test_p_adjust_bh_by_match_scipy():
    from scipy.stats import false_discovery_control
    rng = np.random.default_rng(11)
    for m in (1, 2, 7, 100, 1000):
        p = rng.random(m) ** 3
        p[: m // 5] = p[0]  # ties
        assert np.allclose(oracle.p_adjust(p, "BH"), false_discovery_control(p, method="bh"), rtol=1e-12, atol=0)
        assert np.allclose(oracle.p_adjust(p, "BY"), false_discovery_control(p, method="by"), rtol=1e-12, atol=0)


def _holm_rejections(p, alpha):
    order = np.argsort(p, kind="stable")
    m = len(p)
    rej = np.zeros(m, dtype=bool)
    for i, j in enumerate(order):  # step down: stop at the first failure
        if p[j] > alpha / (m - i):
            break
        rej[j] = True
    return rej


def _hochberg_rejections(p, alpha):
    order = np.argsort(p, kind="stable")
    m = len(p)
    rej = np.zeros(m, dtype=bool)
    for i in range(m - 1, -1, -1):  # step up: the largest i that passes
        if p[order[i]] <= alpha / (m - i):
            rej[order[: i + 1]] = True
            break
    return rej


def test_holm_and_hochberg_match_sequential_procedures():
    rng = np.random.default_rng(12)
    for m in (1, 3, 10, 200):
        p = np.concatenate([rng.random(m // 2) * 1e-3, rng.random(m - m // 2)])
        holm = oracle.p_adjust(p, "holm")
        hoch = oracle.p_adjust(p, "hochberg")
        for alpha in (1e-4, 1e-3, 0.01, 0.05, 0.2):
            assert np.array_equal(holm <= alpha, _holm_rejections(p, alpha))
            assert np.array_equal(hoch <= alpha, _hochberg_rejections(p, alpha))
        assert np.all(hoch <= holm + 1e-15)  # Hochberg is uniformly more powerful
        assert np.allclose(oracle.p_adjust(p, "bonferroni"), np.minimum(1, m * p))


def test_p_adjust_worked_example():
    """Five p-values 0.01..0.05 by hand: Holm multiplies by 5,4,3,2,1 and takes
    running maxima; BH multiplies by 5/1..5/5 and takes running minima from
    the largest."""
    p = np.array([0.03, 0.01, 0.05, 0.02, 0.04])
    assert np.allclose(oracle.p_adjust(p, "holm"), [0.09, 0.05, 0.09, 0.08, 0.09])
    assert np.allclose(oracle.p_adjust(p, "BH"), [0.05] * 5)
    assert np.allclose(oracle.p_adjust(p, "hochberg"), [0.05] * 5)
    assert np.allclose(oracle.p_adjust(p, "BY"), np.minimum(1, 0.05 * sum(1 / k for k in range(1, 6))))


def test_select_null_and_planted_signal():
    """Null decision: Holm at 0.05 selects nothing in (almost) every seed.
    Planted pair with a strong XOR effect: both members selected at k = 2."""
    rng = np.random.default_rng(21)
    M, N = 12, 400
    false_sel = 0
    for s in range(6):
        x = rng.standard_normal((M, N)).astype(np.float32)
        y = (rng.random(N) < 0.5).astype(np.uint8)
        r = oracle.select(x, y, 24, 1, 1, 1, 0.0, 0.25, seed=100 + s)
        false_sel += int(r["relevant"].any())
        assert r["n_eff"] > 0
    assert false_sel <= 2
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[2] > 0) ^ (x[7] > 0)).astype(np.uint8)
    flip = rng.random(N) < 0.05
    y[flip] ^= 1
    r = oracle.select(x, y, 24, 2, 1, 1, 0.0, 0.25, seed=7)
    assert r["relevant"][2] and r["relevant"][7]
    assert r["relevant"].sum() <= 3


@pytest.mark.parametrize("k", [1, 2, 3])
def test_interesting_tuples_agree_with_the_max(k):
    """Every variable's IG^k_max record is interesting at a threshold just below
    it, nothing is interesting above the global max, and the records at
    threshold -inf are all (variable, tuple) pairs."""
    rng = np.random.default_rng(50 + k)
    M, N, D = 7, 150, 2
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[0] > 0) ^ (x[3] > 0) ^ (rng.random(N) < 0.1)).astype(np.uint8)
    codes = oracle.discretize(x, 1, D, 0.5, seed=9)
    ref = oracle.max_ig(codes, y, 2, k, 0.25)
    allrec = oracle.interesting_tuples(codes, y, 2, k, 0.25, -np.inf)
    assert len(allrec) == M * math.comb(M - 1, k - 1)
    assert [r[:2] for r in allrec] == sorted(r[:2] for r in allrec)
    for v in range(M):
        mine = [r for r in allrec if r[0] == v]
        best = max(mine, key=lambda r: r[2])
        assert best[2] == pytest.approx(ref["ig"][v], abs=1e-12)
    top = float(np.max(ref["ig"]))
    assert oracle.interesting_tuples(codes, y, 2, k, 0.25, top + 1e-9) == []
    recs = oracle.interesting_tuples(codes, y, 2, k, 0.25, top - 1e-9)
    assert len(recs) >= 1 and all(r[2] >= top - 1e-9 for r in recs)


def test_interesting_tuples_threshold_reached_and_lowest_discretisation():
    """A (variable, tuple) is interesting when its IG reaches the threshold,
    equality included; and with range = 0 every discretisation is the same
    equipotent split, so each record's maximum is reached at every d and the
    lowest, d = 0, is the one reported."""
    rng = np.random.default_rng(61)
    M, N, D = 6, 120, 3
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[1] > 0) ^ (x[4] > 0) ^ (rng.random(N) < 0.1)).astype(np.uint8)
    codes = oracle.discretize(x, 1, D, 0.0, seed=3)
    allrec = oracle.interesting_tuples(codes, y, 2, 2, 0.25, -np.inf)
    assert all(r[3] == 0 for r in allrec)
    top = max(r[2] for r in allrec)
    at_top = oracle.interesting_tuples(codes, y, 2, 2, 0.25, top)
    assert at_top == [r for r in allrec if r[2] >= top] and len(at_top) >= 1
