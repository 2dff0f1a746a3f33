"""GPU (sm_103a) parity of interesting tuples (ComputeInterestingTuples,
section "Examples" of arXiv 1811.00631) against the FP64 CPU oracle, through
the C ABI.

Bars: every oracle record farther than the IG tolerance (1e-4 + 1e-5 |IG|)
above the threshold is found, every GPU record not within that tolerance of
the threshold is an oracle record, IG within the tolerance, and the
discretisation equal unless the oracle's two best discretisations of that
(variable, tuple) lie within it (``argmax_rule``).
"""
import math

import numpy as np
import pytest

import argmax_rule
import oracle

pytestmark = pytest.mark.gpu

ATOL, RTOL = 1e-4, 1e-5


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_00631_gb300 import build
    build.build()
    return torch


def _compare(codes, y, c, k, xi, thr, got, ref):
    var, tu, ig, di = (np.asarray(a.cpu() if hasattr(a, "cpu") else a) for a in got)
    g = {(int(v), tuple(int(p) for p in t)): (float(s), int(d)) for v, t, s, d in zip(var, tu, ig, di)}
    o = {(v, S): (s, d) for v, S, s, d in ref}
    # records sorted by (variable, tuple)
    keys = [(int(v), tuple(int(p) for p in t)) for v, t in zip(var, tu)]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    for key, (s, d) in o.items():
        tol = ATOL + RTOL * abs(s)
        if s >= thr + tol:
            assert key in g, f"oracle record {key} ({s}) missing"
    for key, (s, d) in g.items():
        v, S = key
        assert v not in S and list(S) == sorted(S) and len(S) == k - 1
        if key in o:
            so, do = o[key]
            assert abs(s - so) <= ATOL + RTOL * abs(so), (key, s, so)
            if d != do:  # only where another discretisation lies within the tolerance of the maximum
                per_d = [oracle.ig_one(codes, y, c, xi, dd, v, list(S)) for dd in range(codes.shape[0])]
                second = max(val for dd, val in enumerate(per_d) if dd != do)
                argmax_rule.check_alternative(so, second, per_d[d], f"record {key}")
        else:
            assert s < thr + ATOL + RTOL * abs(s), f"GPU record {key} ({s}) not in the oracle"


@pytest.mark.parametrize("k,div,M,N,D", [(1, 1, 40, 300, 3), (2, 1, 30, 400, 2), (2, 2, 20, 333, 2),
                                         (3, 1, 14, 257, 2), (3, 2, 10, 200, 1), (4, 1, 10, 300, 2),
                                         (5, 1, 9, 300, 2)])
def test_interesting_tuples_match_oracle(cuda, k, div, M, N, D):
    from paper_1811_00631_gb300 import mdfs
    rng = np.random.default_rng(k * 100 + M)
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[1] > 0) ^ (x[M - 2] > 0.3) ^ (rng.random(N) < 0.1)).astype(np.uint8)
    c = div + 1
    codes = oracle.discretize(x, div, D, 0.5, 23)
    # a threshold that keeps roughly the top tenth of all (variable, tuple) maxima
    allrec = oracle.interesting_tuples(codes, y, c, k, 0.25, -np.inf)
    thr = float(np.quantile([r[2] for r in allrec], 0.9))
    ref = [r for r in allrec if r[2] >= thr]
    got = mdfs.interesting_tuples(cuda.from_numpy(x).cuda(), cuda.from_numpy(y).cuda(), k, div, D, 0.5, 0.25, 23,
                                  thr, capacity=4096)
    _compare(codes, y, c, k, 0.25, thr, got, ref)
    got_h = mdfs.interesting_tuples(x, y, k, div, D, 0.5, 0.25, 23, thr, capacity=4096)  # host pointers
    for a, b in zip(got, got_h):
        assert np.array_equal(np.asarray(a.cpu()), b)


def test_interesting_tuples_all_records_and_max_agree(cuda):
    """At a threshold below every IG, the records are all M * C(M-1, k-1)
    (variable, tuple) pairs, and each variable's best record is its IG^k_max."""
    from paper_1811_00631_gb300 import mdfs
    rng = np.random.default_rng(5)
    M, N, k = 12, 300, 3
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[0] > 0) ^ (x[5] > 0)).astype(np.uint8)
    var, tu, ig, di = mdfs.interesting_tuples(x, y, k, 1, 2, 0.5, 0.25, 4, -1e6, capacity=M * math.comb(M - 1, k - 1))
    assert len(var) == M * math.comb(M - 1, k - 1)
    best, _, _ = mdfs.max_ig(x, y, k, 1, 2, 0.5, 0.25, 4)
    for v in range(M):
        mine = ig[var == v]
        assert abs(float(mine.max()) - float(best[v])) <= ATOL + RTOL * abs(float(best[v]))


def test_interesting_tuples_capacity(cuda):
    from paper_1811_00631_gb300 import mdfs
    rng = np.random.default_rng(6)
    M, N = 20, 200
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = (rng.random(N) < 0.5).astype(np.uint8)
    with pytest.raises(mdfs.MdfsError) as e:
        mdfs.interesting_tuples(x, y, 2, 1, 1, 0.0, 0.25, 1, -1e6, capacity=10)  # 380 records qualify
    assert e.value.code == -7 and "380" in str(e.value)
    var, tu, ig, di = mdfs.interesting_tuples(x, y, 2, 1, 1, 0.0, 0.25, 1, 1e6, capacity=10)
    assert len(var) == 0


def _oracle_per_d(codes, y, c, xi, v, S):
    return [oracle.ig_one(codes, y, c, xi, d, v, list(S)) for d in range(codes.shape[0])]


@pytest.mark.parametrize("k,div,M,N,D", [(2, 1, 300, 1200, 2), (2, 2, 200, 1000, 2), (3, 1, 120, 900, 2)])
def test_interesting_tuples_tensor_core_sizes_sampled(cuda, k, div, M, N, D):
    """Sizes that the tensor-core kernels serve (k = 2 with two or three
    classes, k = 3 with two) over several tiles and ragged edges: every record
    of sampled variables against the full oracle enumeration of those
    variables, and sampled records of every variable against the oracle."""
    import itertools
    from paper_1811_00631_gb300 import mdfs
    rng = np.random.default_rng(1000 * k + M)
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[1] > 0) ^ (x[M - 2] > 0.3) ^ (x[M // 2] > -0.2) ^ (rng.random(N) < 0.05)).astype(np.uint8)
    c, xi = div + 1, 0.25
    codes = oracle.discretize(x, div, D, 0.5, 29)
    sampled = [1, M // 2, M - 2, 7]
    ref = {}
    for v in sampled:
        for S in itertools.combinations([m for m in range(M) if m != v], k - 1):
            per_d = _oracle_per_d(codes, y, c, xi, v, S)
            ref[(v, S)] = per_d
    # a threshold that keeps about the top 5 % of the sampled variables' records
    thr = float(np.quantile([max(p) for p in ref.values()], 0.95))
    var, tu, ig, di = mdfs.interesting_tuples(x, y, k, div, D, 0.5, xi, 29, thr,
                                              capacity=M * math.comb(M - 1, k - 1))
    var, tu, ig, di = (np.asarray(a) for a in (var, tu, ig, di))
    keys = [(int(v), tuple(int(p) for p in t)) for v, t in zip(var, tu)]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    got = {key: (float(s), int(d)) for key, s, d in zip(keys, ig, di)}

    def check(key, per_d):
        o = max(per_d)
        t = ATOL + RTOL * abs(o)
        if key in got:
            s, d = got[key]
            assert abs(s - o) <= t, (key, s, o)
            assert o >= thr - t, f"GPU record {key} ({s}) below the threshold in the oracle ({o})"
            do = int(np.argmax(per_d))
            if d != do:
                second = max(val for dd, val in enumerate(per_d) if dd != do)
                argmax_rule.check_alternative(o, second, per_d[d], f"record {key}")
        else:
            assert o < thr + t, f"oracle record {key} ({o}) missing"

    for key, per_d in ref.items():
        check(key, per_d)
    assert any(v in sampled for v, _ in got)
    # records of all variables, sampled
    pick = rng.choice(len(keys), size=min(300, len(keys)), replace=False)
    for j in pick:
        v, S = keys[j]
        assert v not in S and list(S) == sorted(S) and len(S) == k - 1
        check(keys[j], _oracle_per_d(codes, y, c, xi, v, S))
