"""GPU (sm_103a) parity of the MDFS scan against the FP64 CPU oracle.

Every call goes through the C ABI (ctypes binding).  Inputs are seeded and
synthetic; expected values come from the oracle only.  Tolerances follow the
statement of the method's precision target: discretised codes bit-exact,
IG within 1e-4 absolute + 1e-5 relative of the FP64 oracle, argmax tuples
equal except where the oracle's top two differ by less than that tolerance
(``argmax_rule``).
"""
import itertools

import numpy as np
import pytest

import argmax_rule
import oracle
from paper_1811_00631_gb300 import synth

pytestmark = pytest.mark.gpu

@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_00631_gb300 import build
    build.build()
    return torch


def _gpu_max_ig(torch, x, y, k, div, D, rng_, xi, seed, host=False):
    from paper_1811_00631_gb300 import mdfs
    if host:
        ig, tu, di = mdfs.max_ig(x, y, k, div, D, rng_, xi, seed)
        return np.asarray(ig, dtype=np.float64), np.asarray(tu), np.asarray(di)
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yt = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    ig, tu, di = mdfs.max_ig(xt, yt, k, div, D, rng_, xi, seed)
    torch.cuda.synchronize()
    return ig.cpu().numpy().astype(np.float64), tu.cpu().numpy(), di.cpu().numpy()


def _check(codes, y, c, k, xi, g_ig, g_tu, g_di, ref, variables):
    """Compare the GPU result for ``variables`` with the oracle's (ref rows align
    with variables): IG within the tolerance, and the argmax equal unless the
    oracle's top two lie within the tolerance (``argmax_rule``)."""
    for row, i in enumerate(variables):
        o = ref["ig"][row]
        assert abs(g_ig[i] - o) <= argmax_rule.tol(o), f"var {i}: gpu {g_ig[i]!r} oracle {o!r}"
        same = g_di[i] == ref["disc"][row] and (k == 1 or tuple(g_tu[i]) == tuple(ref["tuples"][row]))
        if not same:
            S = list(g_tu[i]) if k > 1 else []
            assert 0 <= g_di[i] < codes.shape[0]
            assert i not in S and len(set(S)) == len(S) and S == sorted(S)
            alt = oracle.ig_one(codes, y, c, xi, int(g_di[i]), int(i), S)
            argmax_rule.check_alternative(o, ref["second"][row], alt, f"var {i} (gpu argmax {g_di[i], S})")


def test_discretize_bit_exact(cuda):
    from paper_1811_00631_gb300 import mdfs
    torch = cuda
    rng = np.random.default_rng(1)
    for (M, N, div, D, r) in [(7, 333, 1, 4, 0.5), (5, 2000, 2, 3, 1.0), (3, 97, 3, 5, 0.0), (2, 4, 3, 2, 0.9)]:
        x = rng.standard_normal((M, N)).astype(np.float32)
        want = oracle.discretize(x, div, D, r, seed=1234567890123)
        got = mdfs.discretize(torch.from_numpy(x).cuda(), div, D, r, seed=1234567890123).cpu().numpy()
        assert np.array_equal(got, want)
        got_h = mdfs.discretize(x, div, D, r, seed=1234567890123)
        assert np.array_equal(got_h, want)


@pytest.mark.parametrize("N", [600, 1000, 1025, 3000, 4096, 8000, 16385, 32768])
def test_discretize_bit_exact_sort_sizes(cuda, N):
    """Codes bit-exact for column lengths that use each in-register sort width
    (padded lengths 1024 .. 8192) and its boundaries, the shared-memory sort of
    longer columns, and the largest N the discretiser takes (32768)."""
    from paper_1811_00631_gb300 import mdfs
    rng = np.random.default_rng(N)
    x = rng.standard_normal((5, N)).astype(np.float32)
    x[1] = np.round(x[1] * 4) / 4  # ties
    for div in (1, 3):
        want = oracle.discretize(x, div, 3, 0.7, seed=99)
        got = mdfs.discretize(cuda.from_numpy(x).cuda(), div, 3, 0.7, seed=99).cpu().numpy()
        assert np.array_equal(got, want)


def test_discretize_int8_and_ties(cuda):
    from paper_1811_00631_gb300 import mdfs
    torch = cuda
    rng = np.random.default_rng(2)
    x = synth.to_int8(rng.standard_normal((9, 501)), scale=3.0)  # heavy ties
    want = oracle.discretize(x.astype(np.float32), 2, 6, 0.7, seed=5)
    got = mdfs.discretize(torch.from_numpy(x).cuda(), 2, 6, 0.7, seed=5).cpu().numpy()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("k,div,M,N,D", [
    (1, 1, 70, 333, 3), (1, 3, 40, 1000, 2),
    (2, 1, 70, 333, 3), (2, 2, 67, 290, 2), (2, 3, 33, 257, 2),
    (3, 1, 150, 200, 2), (3, 2, 45, 161, 2), (3, 3, 36, 130, 1),
])
def test_max_ig_small(cuda, k, div, M, N, D):
    """Several tiles with ragged tails in M and N, all k and class counts."""
    rng = np.random.default_rng(100 * k + 10 * div + D)
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[0] > 0) ^ (x[3] > 0.2) ^ (rng.random(N) < 0.2)).astype(np.uint8)
    xi, r, seed = 0.25, 0.5, 77 + k
    c = div + 1
    codes = oracle.discretize(x, div, D, r, seed)
    ref = oracle.max_ig(codes, y, c, k, xi)
    g = _gpu_max_ig(cuda, x, y, k, div, D, r, xi, seed)
    _check(codes, y, c, k, xi, *g, ref, range(M))


def test_max_ig_host_pointers_match_device(cuda):
    rng = np.random.default_rng(5)
    x = rng.standard_normal((50, 300)).astype(np.float32)
    y = (rng.random(300) < 0.3).astype(np.uint8)
    dev = _gpu_max_ig(cuda, x, y, 2, 2, 3, 0.5, 0.3, 9)
    host = _gpu_max_ig(cuda, x, y, 2, 2, 3, 0.5, 0.3, 9, host=True)
    for a, b in zip(dev, host):
        assert np.array_equal(a, b)


def test_xor_small_config(cuda):
    """N=200, M=50 XOR data, 2 bins, 1 discretisation, range 0.25, xi 0.25, seed 1."""
    ds = synth.xor_small()
    codes = oracle.discretize(ds.x, 1, 1, 0.25, 1)
    ref = oracle.max_ig(codes, ds.y, 2, 2, 0.25)
    g = _gpu_max_ig(cuda, ds.x, ds.y, 2, 1, 1, 0.25, 0.25, 1)
    _check(codes, ds.y, 2, 2, 0.25, *g, ref, range(50))
    assert set(np.argsort(-g[0])[:2].tolist()) == {0, 1}
    assert g[1][0, 0] == 1 and g[1][1, 0] == 0


@pytest.mark.parametrize("k,div", [(1, 1), (1, 2), (2, 1), (2, 2)])
def test_madelon_like_full_size_sampled(cuda, k, div):
    """N=2000, M=500, 30 discretisations, range 0.5, xi 0.25: the full GPU
    scan, compared on every informative variable and a random sample of noise
    variables (the oracle computes those rows one by one)."""
    ds = synth.madelon_like()
    D, r, xi, seed = 30, 0.5, 0.25, 11
    c = div + 1
    codes = oracle.discretize(ds.x, div, D, r, seed)
    g = _gpu_max_ig(cuda, ds.x, ds.y, k, div, D, r, xi, seed)
    rng = np.random.default_rng(3)
    noise = np.setdiff1d(np.arange(500), ds.informative)
    variables = np.concatenate([ds.informative, rng.choice(noise, 20, replace=False)]).astype(np.int32)
    ref = oracle.max_ig(codes, ds.y, c, k, xi, variables=variables)
    _check(codes, ds.y, c, k, xi, *g, ref, variables)


def test_madelon_like_k3_full_size_sampled(cuda):
    """k=3 on the 2000 x 500 parity data, 30 discretisations, 2 bins: the
    full triple scan, compared on a sample of variables."""
    ds = synth.madelon_like()
    D, r, xi, seed = 30, 0.5, 0.25, 11
    codes = oracle.discretize(ds.x, 1, D, r, seed)
    g = _gpu_max_ig(cuda, ds.x, ds.y, 3, 1, D, r, xi, seed)
    variables = np.array([ds.info["base"][0], ds.info["comb"][0], 7, 499], dtype=np.int32)
    ref = oracle.max_ig(codes, ds.y, 2, 3, xi, variables=variables)
    _check(codes, ds.y, 2, 3, xi, *g, ref, variables)


def test_edge_minimal_sizes(cuda):
    rng = np.random.default_rng(8)
    for k, M, N, div in [(1, 1, 2, 1), (2, 2, 3, 2), (3, 3, 4, 3), (3, 4, 33, 1), (2, 5, 32, 1), (2, 5, 64, 1)]:
        x = rng.standard_normal((M, N)).astype(np.float32)
        y = (np.arange(N) % 2).astype(np.uint8)
        codes = oracle.discretize(x, div, 2, 0.3, 3)
        ref = oracle.max_ig(codes, y, div + 1, k, 0.5)
        g = _gpu_max_ig(cuda, x, y, k, div, 2, 0.3, 0.5, 3)
        _check(codes, y, div + 1, k, 0.5, *g, ref, range(M))


def test_edge_maximum_sizes(cuda):
    """The largest sample count (N = 32768, the discretiser's in-CTA sort
    limit) with the most classes per variable (divisions = 3) and with two
    classes, for k = 1..3; every variable against the oracle."""
    rng = np.random.default_rng(41)
    M, N, D = 6, 32768, 2
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[1] > 0) ^ (x[4] > 0) ^ (rng.random(N) < 0.1)).astype(np.uint8)
    for k, div in [(1, 3), (2, 1), (2, 3), (3, 1), (3, 3)]:
        codes = oracle.discretize(x, div, D, 0.5, 17)
        ref = oracle.max_ig(codes, y, div + 1, k, 0.25)
        g = _gpu_max_ig(cuda, x, y, k, div, D, 0.5, 0.25, 17)
        _check(codes, y, div + 1, k, 0.25, *g, ref, range(M))


def test_k3_large_n_uses_global_tables(cuda):
    """N beyond the shared-memory table limit of the two-class triple kernel."""
    rng = np.random.default_rng(19)
    M, N = 14, 9000
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[1] > 0) ^ (x[2] > 0) ^ (x[5] > 0) ^ (rng.random(N) < 0.1)).astype(np.uint8)
    codes = oracle.discretize(x, 1, 2, 0.4, 4)
    ref = oracle.max_ig(codes, y, 2, 3, 0.25)
    g = _gpu_max_ig(cuda, x, y, 3, 1, 2, 0.4, 0.25, 4)
    _check(codes, y, 2, 3, 0.25, *g, ref, range(M))
    assert set(g[1][1].tolist()) == {2, 5}


def test_k3_two_class_beyond_shared_tables(cuda):
    """N too large for the tensor-core triple kernel's shared-memory tables."""
    rng = np.random.default_rng(23)
    M, N = 12, 20000
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[0] > 0) ^ (x[4] > 0) ^ (x[7] > 0) ^ (rng.random(N) < 0.1)).astype(np.uint8)
    codes = oracle.discretize(x, 1, 2, 0.4, 6)
    ref = oracle.max_ig(codes, y, 2, 3, 0.25)
    g = _gpu_max_ig(cuda, x, y, 3, 1, 2, 0.4, 0.25, 6)
    _check(codes, y, 2, 3, 0.25, *g, ref, range(M))
    assert set(g[1][0].tolist()) == {4, 7}


@pytest.mark.parametrize("M,N", [(130, 300), (260, 129), (3, 5)])
def test_k3_tensor_core_tiles(cuda, M, N):
    """Two-class triples across several 128-wide a/e tiles, K blocks with
    padding in both classes, and the smallest sizes."""
    rng = np.random.default_rng(M + N)
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[0] > 0) ^ (x[M // 2] > 0) ^ (x[M - 1] > 0) ^ (rng.random(N) < 0.1)).astype(np.uint8)
    if y.min() == y.max():
        y[0] ^= 1
    D = 2
    codes = oracle.discretize(x, 1, D, 0.5, 8)
    ref = oracle.max_ig(codes, y, 2, 3, 0.25)
    g = _gpu_max_ig(cuda, x, y, 3, 1, D, 0.5, 0.25, 8)
    _check(codes, y, 2, 3, 0.25, *g, ref, range(M))


def test_k3_tensor_core_large_class_counts(cuda):
    """Class sizes close to 4096: the single FP32 accumulator holds
    n0 + 4096 n1 with both counts near their limit (wide e groups, many K
    blocks in both classes)."""
    rng = np.random.default_rng(77)
    M, N = 40, 8150
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = np.zeros(N, dtype=np.uint8)
    y[rng.permutation(N)[:4080]] = 1  # N0 = 4070, N1 = 4080
    codes = oracle.discretize(x, 1, 1, 0.2, 31)
    ref = oracle.max_ig(codes, y, 2, 3, 0.25)
    g = _gpu_max_ig(cuda, x, y, 3, 1, 1, 0.2, 0.25, 31)
    _check(codes, y, 2, 3, 0.25, *g, ref, range(M))


@pytest.mark.parametrize("n1", [4095, 4096])
def test_k2_three_classes_class_size_limit(cuda, n1):
    """k = 2 with three classes per variable: one FP32 accumulator per row bin
    holds n0 + 4096 n1, exact for class sizes below 4096.  At N1 = 4095 the
    tensor-core kernel runs; at N1 = 4096 the scan takes the bit-plane kernel
    instead.  Both match the oracle."""
    rng = np.random.default_rng(n1)
    M, N = 24, 4700
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = np.zeros(N, dtype=np.uint8)
    y[rng.permutation(N)[:n1]] = 1
    codes = oracle.discretize(x, 2, 1, 0.3, 5)
    ref = oracle.max_ig(codes, y, 3, 2, 0.25)
    g = _gpu_max_ig(cuda, x, y, 2, 2, 1, 0.3, 0.25, 5)
    _check(codes, y, 3, 2, 0.25, *g, ref, range(M))


def test_k3_permuted_variable_order_and_repeatability(cuda):
    """The triple kernel relabels variables by marginal count and prunes role-e
    updates with the keys found so far.  The same data in two variable orders
    (two different relabellings) must both match the oracle, and repeated
    calls must return identical IG, tuples and discretisations whatever the
    order in which CTAs raised the keys."""
    rng = np.random.default_rng(5)
    M, N = 300, 700
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[3] > 0) ^ (x[150] > 0) ^ (x[299] > 0.3)).astype(np.uint8)
    perm = rng.permutation(M)
    rows = np.arange(0, M, 37)
    for xx in (x, np.ascontiguousarray(x[perm])):
        g = _gpu_max_ig(cuda, xx, y, 3, 1, 2, 0.5, 0.25, 13)
        codes = oracle.discretize(xx, 1, 2, 0.5, 13)
        ref = oracle.max_ig(codes, y, 2, 3, 0.25, variables=rows)
        _check(codes, y, 2, 3, 0.25, *g, ref, rows)
        for _ in range(2):
            again = _gpu_max_ig(cuda, xx, y, 3, 1, 2, 0.5, 0.25, 13)
            for u, v in zip(g, again):
                assert np.array_equal(u, v)


def test_unbalanced_classes_and_int8(cuda):
    rng = np.random.default_rng(9)
    M, N = 40, 777
    x8 = synth.to_int8(rng.standard_normal((M, N)), scale=4.0)
    y = (rng.random(N) < 0.07).astype(np.uint8)
    for k in (1, 2, 3):
        codes = oracle.discretize(x8.astype(np.float32), 2, 3, 0.8, 21)
        ref = oracle.max_ig(codes, y, 3, k, 0.1)
        g = _gpu_max_ig(cuda, x8, y, k, 2, 3, 0.8, 0.1, 21)
        _check(codes, y, 3, k, 0.1, *g, ref, range(M))


def test_errors(cuda):
    from paper_1811_00631_gb300 import mdfs
    torch = cuda
    x = torch.randn(10, 50, device="cuda")
    with pytest.raises(mdfs.MdfsError) as e:
        mdfs.max_ig(x, torch.zeros(50, dtype=torch.uint8, device="cuda"), 2, 1, 1)
    assert e.value.code == -2
    y = torch.zeros(50, dtype=torch.uint8, device="cuda")
    y[3] = 2
    with pytest.raises(mdfs.MdfsError) as e:
        mdfs.max_ig(x, y, 2, 1, 1)
    assert e.value.code == -1
    x2 = x.clone()
    x2[4, 7] = float("nan")
    y[3] = 1
    with pytest.raises(mdfs.MdfsError) as e:
        mdfs.max_ig(x2, y, 2, 1, 1)
    assert e.value.code == -3
    # the context is still usable after host-detected errors
    ig, _, _ = mdfs.max_ig(x, y, 2, 1, 1)
    torch.cuda.synchronize()
    assert torch.isfinite(ig).all()


def test_ig_lim_matches_oracle(cuda):
    from paper_1811_00631_gb300 import mdfs
    rng = np.random.default_rng(31)
    for df_k, T in [(1, 50), (2, 400), (3, 2000)]:
        c = 2
        df = (c - 1) * c ** (df_k - 1)
        ig = (0.5 * rng.chisquare(df, size=(3000, T)).max(axis=1)).astype(np.float32)
        mask = (rng.random(3000) < 0.8).astype(np.uint8)
        p_o, lim_o, t_o = oracle.ig_lim(ig.astype(np.float64), df_k, 1, mask, alpha=0.01)
        p_g, lim_g, t_g = mdfs.ig_lim(ig, df_k, 1, 1, mask, alpha=0.01)
        assert t_g == pytest.approx(t_o, rel=1e-10)
        assert lim_g == pytest.approx(lim_o, rel=1e-9)
        assert np.allclose(p_g, p_o, rtol=1e-9, atol=1e-14)
        p_d, lim_d, t_d = mdfs.ig_lim(cuda.from_numpy(ig).cuda(), df_k, 1, 1, mask, alpha=0.01)
        assert np.allclose(p_d.cpu().numpy(), p_o, rtol=1e-9, atol=1e-14)


def test_repeatable_and_stream_ordered(cuda):
    """Same inputs, same outputs, bit for bit, on the default and a side stream."""
    torch = cuda
    from paper_1811_00631_gb300 import mdfs
    ds = synth.madelon_like(N=500, M=120, seed=3)
    x = torch.from_numpy(ds.x).cuda()
    y = torch.from_numpy(ds.y).cuda()
    a = mdfs.max_ig(x, y, 3, 1, 4, 0.5, 0.25, 5)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b = mdfs.max_ig(x, y, 3, 1, 4, 0.5, 0.25, 5)
    s.synchronize()
    for u, v in zip(a, b):
        assert torch.equal(u, v)


@pytest.mark.parametrize("M,N,D", [(4, 97, 1), (5, 300, 2), (14, 300, 2), (9, 2100, 1), (8, 4500, 1), (6, 40, 2)])
def test_k4_matches_oracle(cuda, M, N, D):
    """k = 4 (two classes): every variable against the brute-force oracle.
    M = 4 is one quadruple; N = 4500 needs two staged chunks of 128 words;
    N = 40 leaves most of a 32-sample word empty."""
    rng = np.random.default_rng(M * 100 + N)
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[0] > 0) ^ (x[1] > 0) ^ (x[M - 1] > 0.2) ^ (rng.random(N) < 0.1)).astype(np.uint8)
    codes = oracle.discretize(x, 1, D, 0.5, 17)
    ref = oracle.max_ig(codes, y, 2, 4, 0.25)
    g = _gpu_max_ig(cuda, x, y, 4, 1, D, 0.5, 0.25, 17)
    _check(codes, y, 2, 4, 0.25, *g, ref, range(M))


def test_k4_several_tiles_sampled(cuda):
    """M = 70 spans three 32-wide c and e tiles; a sample of variables is checked
    (each oracle row scans all C(69, 3) partner triples)."""
    rng = np.random.default_rng(70)
    M, N, D = 70, 200, 1
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[5] > 0) ^ (x[33] > 0) ^ (x[69] > 0)).astype(np.uint8)
    codes = oracle.discretize(x, 1, D, 0.5, 3)
    rows = np.array([0, 5, 31, 32, 33, 40, 63, 64, 69], dtype=np.int32)
    ref = oracle.max_ig(codes, y, 2, 4, 0.25, variables=rows)
    g = _gpu_max_ig(cuda, x, y, 4, 1, D, 0.5, 0.25, 3)
    _check(codes, y, 2, 4, 0.25, *g, ref, rows)


def test_k4_four_way_parity_found(cuda):
    """y = parity of four variables: each member's best partner triple is the
    other three, and the four are the top four at k = 4."""
    rng = np.random.default_rng(404)
    M, N = 12, 3000
    x = rng.standard_normal((M, N)).astype(np.float32)
    mem = [1, 4, 6, 10]
    y = np.zeros(N, dtype=np.uint8)
    for m in mem:
        y ^= (x[m] > 0).astype(np.uint8)
    ig, tu, di = _gpu_max_ig(cuda, x, y, 4, 1, 1, 0.0, 0.25, 9)
    assert set(np.argsort(-ig)[:4].tolist()) == set(mem)
    for m in mem:
        assert sorted(tu[m].tolist()) == sorted(v for v in mem if v != m)


def test_k4_errors(cuda):
    from paper_1811_00631_gb300 import mdfs
    x = np.random.default_rng(0).standard_normal((6, 50)).astype(np.float32)
    y = (np.arange(50) % 2).astype(np.uint8)
    with pytest.raises(mdfs.MdfsError):
        mdfs.max_ig(x, y, 4, 4, 1)  # five classes: more than any scan supports
    xl = np.random.default_rng(1).standard_normal((1700, 8)).astype(np.float32)
    yl = (np.arange(8) % 2).astype(np.uint8)
    with pytest.raises(mdfs.MdfsError):
        mdfs.max_ig(xl, yl, 4, 1, 1)  # 1700^3 >= 2^32: keys cannot index the triple


def _exact_and_bounded(torch, x, y, k, div, D, r, xi, seed):
    """The tensor-core scan evaluated exactly for every tuple (test hook), then
    the normal scan that skips tuples by the entropy lower bound."""
    from paper_1811_00631_gb300 import mdfs
    xt, yt = torch.from_numpy(np.ascontiguousarray(x)).cuda(), torch.from_numpy(np.ascontiguousarray(y)).cuda()
    mdfs.testing_exact()
    exact = [t.cpu().numpy() for t in mdfs.max_ig(xt, yt, k, div, D, r, xi, seed)]
    fast = [t.cpu().numpy() for t in mdfs.max_ig(xt, yt, k, div, D, r, xi, seed)]
    return exact, fast


@pytest.mark.parametrize("case", ["parity_full", "xor_pairs", "unbalanced", "small_xi", "large_xi"])
def test_k3_bound_changes_no_result(cuda, case):
    """The triples the SH3 lower bound skips can never raise a key: the scan
    with the bound returns the IG, tuples and discretisations of the scan that
    evaluates every triple exactly, bit for bit, for every variable.  Covers
    the bench step's k = 3 launch (2000 x 500, 30 discretisations), strong
    pair signals, unbalanced classes and small and large pseudocounts."""
    rng = np.random.default_rng(hash(case) % 2**32)
    D, r, xi, seed = 4, 0.5, 0.25, 21
    if case == "parity_full":
        ds = synth.madelon_like()
        x, y, D, seed = ds.x, ds.y, 30, 11
    elif case == "xor_pairs":
        ds = synth.xor_pairs(N=1500, M=300, n_pairs=10, flip=0.1, seed=3)
        x, y = ds.x, ds.y
    else:
        M, N = 260, 900
        x = rng.standard_normal((M, N)).astype(np.float32)
        y = ((x[3] > 0) ^ (x[100] > 0) ^ (x[259] > 0.2)).astype(np.uint8)
        if case == "unbalanced":
            y = (rng.random(N) < 0.12).astype(np.uint8) | ((x[5] > 1.2) & (x[7] > 1.0)).astype(np.uint8)
        xi = {"unbalanced": 0.25, "small_xi": 0.002, "large_xi": 0.95}[case]
    exact, fast = _exact_and_bounded(cuda, x, y, 3, 1, D, r, xi, seed)
    for a, b, name in zip(exact, fast, ("ig", "tuples", "disc")):
        assert np.array_equal(a, b), f"{case}: {name} differs in {np.count_nonzero(a != b)} entries"


@pytest.mark.parametrize("case", ["parity_full", "xor_pairs", "unbalanced", "small_xi", "large_xi", "batched_size"])
def test_k2_bound_changes_no_result(cuda, case):
    """k = 2 with three classes per variable: the scan that skips pairs by the
    SH2 lower bound returns the IG, partners and discretisations of the scan
    that evaluates every pair exactly, bit for bit, for every variable.
    Covers the 2000 x 500 parity data with 30 discretisations, strong pair
    signals, unbalanced classes, small and large pseudocounts and one job of
    the batched workload's size (1000 x 20000, 10 discretisations)."""
    rng = np.random.default_rng(hash(case) % 2**32)
    D, r, xi, seed = 4, 0.5, 0.25, 21
    if case == "parity_full":
        ds = synth.madelon_like()
        x, y, D, seed = ds.x, ds.y, 30, 11
    elif case == "xor_pairs":
        ds = synth.xor_pairs(N=1500, M=300, n_pairs=10, flip=0.1, seed=3)
        x, y = ds.x, ds.y
    elif case == "batched_size":
        ds = synth.xor_pairs(N=1000, M=20000, n_pairs=100, seed=4)
        x, y, D = ds.x, ds.y, 10
    else:
        M, N = 260, 900
        x = rng.standard_normal((M, N)).astype(np.float32)
        y = ((x[3] > 0) ^ (x[100] > 0) ^ (rng.random(N) < 0.1)).astype(np.uint8)
        if case == "unbalanced":
            y = (rng.random(N) < 0.12).astype(np.uint8) | ((x[5] > 1.2) & (x[7] > 1.0)).astype(np.uint8)
        xi = {"unbalanced": 0.25, "small_xi": 0.002, "large_xi": 0.95}[case]
    exact, fast = _exact_and_bounded(cuda, x, y, 2, 2, D, r, xi, seed)
    for a, b, name in zip(exact, fast, ("ig", "tuples", "disc")):
        assert np.array_equal(a, b), f"{case}: {name} differs in {np.count_nonzero(a != b)} entries"
