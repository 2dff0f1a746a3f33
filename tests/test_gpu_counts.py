"""Voxel counters of the tensor-core scans, bit for bit.

The paper's scan counts, for every tuple and discretisation, the objects of
each decision class in every voxel of the tuple's discretised subspace
(section "Algorithm and implementation"); IG follows from those counts (Eq. 1,
Eqs. H, p, beta).  The IG parity tests only see the counts through the
entropy, where an off-by-one count moves IG by about beta / n, below the IG
tolerance.  Here the k = 2 and k = 3 tensor-core kernels write the counts they
derive (test hook mdfs_testing_counts: the same launch as the scan, with the
counts also stored) and every one is compared exactly with counts taken
directly from the oracle's codes: one-hot products summed over the samples of
each class for every pair, and np.bincount of the 8 voxel indices for sampled
triples.
"""
import math

import numpy as np
import pytest

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


def _packed(n0, n1):
    return (n0.astype(np.int64) | (n1.astype(np.int64) << 16)).astype(np.int64)


def _pair_counts(codes_d, y, c):
    """[C(M,2), c*c]: class counts of every voxel (u, v) of every pair i < m,
    counted as the sum over each class's samples of [code_i = u][code_m = v]."""
    M = codes_d.shape[0]
    iu, ju = np.triu_indices(M, 1)
    cls = []
    for k in (0, 1):
        cd = codes_d[:, y == k]
        oh = (cd[:, None, :] == np.arange(c, dtype=np.uint8)[None, :, None]).astype(np.float64).reshape(M * c, -1)
        g = (oh @ oh.T).reshape(M, c, M, c).transpose(0, 2, 1, 3)
        cls.append(np.rint(g[iu, ju]).astype(np.int64).reshape(len(iu), c * c))
    return _packed(cls[0], cls[1])


def _triple_counts(codes_d, y, tri):
    """[T, 8]: class counts of the voxels 4 u + 2 v + w of the sorted triples
    tri (T x 3), by np.bincount of each sample's voxel index."""
    T = len(tri)
    cls = []
    for k in (0, 1):
        cd = codes_d[:, y == k].astype(np.int64)
        idx = 4 * cd[tri[:, 0]] + 2 * cd[tri[:, 1]] + cd[tri[:, 2]]
        flat = (np.arange(T, dtype=np.int64)[:, None] * 8 + idx).ravel()
        cls.append(np.bincount(flat, minlength=8 * T).reshape(T, 8))
    return _packed(cls[0], cls[1])


def _triple_rank(M, t):
    """Lexicographic rank of sorted triples among the C(M, 3) triples of [0, M)."""
    c2 = lambda n: np.where(n < 2, 0, n * (n - 1) // 2)
    c3 = lambda n: np.where(n < 3, 0, n * (n - 1) * (n - 2) // 6)
    x, yy, z = (t[:, j].astype(np.int64) for j in range(3))
    return c3(M) - c3(M - x) + c2(M - x - 1) - c2(M - yy) + (z - yy - 1)


def test_triple_rank_enumerates_in_lexicographic_order():
    M = 9
    tri = np.array([t for t in __import__("itertools").combinations(range(M), 3)])
    assert np.array_equal(_triple_rank(M, tri), np.arange(len(tri)))


def _sample_triples(M, n, rng, extra=()):
    t = np.sort(np.stack([rng.choice(M, 3, replace=False) for _ in range(n)]), axis=1)
    extra = [v for v in extra if v < M]
    t = np.concatenate([t, np.array(list(__import__("itertools").combinations(sorted(set(extra)), 3)),
                                    dtype=t.dtype).reshape(-1, 3)])
    return np.unique(t, axis=0)


@pytest.mark.parametrize("M,N,div,D", [(300, 777, 1, 2), (300, 777, 2, 2), (131, 129, 1, 3), (3, 5, 2, 1),
                                       (257, 2048, 2, 1)])
def test_pair_counts_bit_exact(cuda, M, N, div, D):
    """k = 2 tensor-core kernel: every pair and discretisation, several 128-row
    tiles with ragged edges, K padding in both classes, both class counts."""
    torch = cuda
    from paper_1811_00631_gb300 import mdfs
    rng = np.random.default_rng(M * 7 + N + div)
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[0] > 0) ^ (x[M - 1] > 0.3) ^ (rng.random(N) < 0.2)).astype(np.uint8)
    y[:2] = (0, 1)
    c = div + 1
    codes = oracle.discretize(x, div, D, 0.5, 19)
    got = mdfs.testing_counts(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), 2, div, D, 0.5, 19)
    got = got.cpu().numpy().astype(np.int64)
    assert got.shape == (D, math.comb(M, 2), c * c)
    for d in range(D):
        assert np.array_equal(got[d], _pair_counts(codes[d], y, c)), f"discretisation {d}"


def test_pair_counts_bit_exact_class_limit(cuda):
    """Three classes per variable: the k = 2 kernel accumulates n0 + 4096 n1 in
    one FP32 value; with N1 = 4095 (the largest class size it takes; N = 4700
    keeps the entropy tables in shared memory) every partial sum is still below
    2^24 and every count exact."""
    torch = cuda
    from paper_1811_00631_gb300 import mdfs
    rng = np.random.default_rng(4095)
    M, N, div, D = 24, 4700, 2, 1
    x = rng.standard_normal((M, N)).astype(np.float32)
    x[3] = np.abs(x[3])  # one variable with most samples in its top bins
    y = np.zeros(N, dtype=np.uint8)
    y[rng.permutation(N)[:4095]] = 1
    codes = oracle.discretize(x, div, D, 0.3, 5)
    got = mdfs.testing_counts(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), 2, div, D, 0.3, 5)
    got = got.cpu().numpy().astype(np.int64)
    assert np.array_equal(got[0], _pair_counts(codes[0], y, div + 1))


@pytest.mark.parametrize("div", [1, 2])
def test_pair_counts_bit_exact_full_size(cuda, div):
    """The 2000 x 500 parity workload with 30 discretisations (the k = 2 launch
    of the bench step for div = 1): all 124750 pairs x 30 discretisations, and
    a bincount cross-check of a sample."""
    torch = cuda
    from paper_1811_00631_gb300 import mdfs
    ds = synth.madelon_like()
    D, c, seed = 30, div + 1, 11
    codes = oracle.discretize(ds.x, div, D, 0.5, seed)
    got = mdfs.testing_counts(torch.from_numpy(ds.x).cuda(), torch.from_numpy(ds.y).cuda(), 2, div, D, 0.5, seed)
    got = got.cpu().numpy().astype(np.int64)
    for d in range(D):
        assert np.array_equal(got[d], _pair_counts(codes[d], ds.y, c)), f"discretisation {d}"
    # independent count of a sample of pairs by bincount
    rng = np.random.default_rng(2)
    iu, ju = np.triu_indices(500, 1)
    for r in rng.choice(len(iu), 50, replace=False):
        i, m = iu[r], ju[r]
        for d in (0, 17, 29):
            want = [np.bincount(codes[d, i, ds.y == k] * c + codes[d, m, ds.y == k], minlength=c * c)
                    for k in (0, 1)]
            assert np.array_equal(got[d, r], _packed(want[0], want[1]))


@pytest.mark.parametrize("M,N,D", [(300, 777, 2), (40, 8150, 1), (3, 5, 1), (130, 300, 2)])
def test_triple_counts_bit_exact(cuda, M, N, D):
    """k = 3 tensor-core kernel (two classes): sampled triples plus every triple
    of a set of variables, across several a tiles and e groups, ragged K
    blocks, class sizes near the kernel's limit of 4096 (N = 8150) and the
    smallest case."""
    torch = cuda
    from paper_1811_00631_gb300 import mdfs
    rng = np.random.default_rng(M + N)
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[0] > 0) ^ (x[M // 2] > 0) ^ (rng.random(N) < 0.1)).astype(np.uint8)
    if N == 8150:
        y = np.zeros(N, np.uint8)
        y[rng.permutation(N)[:4080]] = 1
    y[:2] = (0, 1)
    codes = oracle.discretize(x, 1, D, 0.5, 23)
    got = mdfs.testing_counts(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), 3, 1, D, 0.5, 23)
    assert tuple(got.shape) == (D, math.comb(M, 3), 8)
    assert int((got < 0).sum()) == 0, "some triple was not visited"
    tri = _sample_triples(M, min(20000, math.comb(M, 3)), rng, extra=(0, 1, 2, 126, 127, 128, 129, 255, 256, 257,
                                                                      M - 2, M - 1))
    ranks = torch.from_numpy(_triple_rank(M, tri)).cuda()
    sel = got[:, ranks, :].cpu().numpy().astype(np.int64)
    for d in range(D):
        assert np.array_equal(sel[d], _triple_counts(codes[d], y, tri)), f"discretisation {d}"


def test_triple_counts_bit_exact_full_size(cuda):
    """The bench step's k = 3 launch: 2000 x 500 parity data, 30
    discretisations (6.2e8 triple x discretisation voxel tables, 20 GB of
    counts on the device); every triple written, and a sample of 6000 triples
    plus all triples of the 20 informative variables compared exactly."""
    torch = cuda
    from paper_1811_00631_gb300 import mdfs
    ds = synth.madelon_like()
    D, seed = 30, 11
    codes = oracle.discretize(ds.x, 1, D, 0.5, seed)
    got = mdfs.testing_counts(torch.from_numpy(ds.x).cuda(), torch.from_numpy(ds.y).cuda(), 3, 1, D, 0.5, seed)
    assert int((got < 0).sum()) == 0, "some triple was not visited"
    rng = np.random.default_rng(7)
    tri = _sample_triples(500, 6000, rng, extra=tuple(int(v) for v in ds.informative))
    ranks = torch.from_numpy(_triple_rank(500, tri)).cuda()
    sel = got[:, ranks, :].cpu().numpy().astype(np.int64)
    del got
    torch.cuda.empty_cache()
    for d in range(D):
        assert np.array_equal(sel[d], _triple_counts(codes[d], ds.y, tri)), f"discretisation {d}"


def test_counts_hook_refuses_other_paths(cuda):
    torch = cuda
    from paper_1811_00631_gb300 import mdfs
    x = torch.randn(20, 300, device="cuda")
    y = (torch.arange(300, device="cuda") % 2).to(torch.uint8)
    with pytest.raises(mdfs.MdfsError) as e:
        mdfs.testing_counts(x, y, 3, 2, 1)  # k = 3 with three classes runs on the popcount kernel
    assert e.value.code == -1
