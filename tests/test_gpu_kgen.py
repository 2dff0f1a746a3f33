"""GPU (sm_103a) parity of the k = 4 and k = 5 scans with three and four
classes per variable (every voxel of every tuple counted from the bit planes)
against the FP64 CPU oracle, through the C ABI.  Same bars as the other scans:
IG within 1e-4 absolute + 1e-5 relative, argmax partner tuple and
discretisation equal unless the GPU's choice is an equally good maximiser."""
import numpy as np
import pytest

import oracle

from test_gpu_interesting import _compare
from test_gpu_parity import _check, _gpu_max_ig

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_00631_gb300 import build
    build.build()
    return torch


def _data(M, N, seed, k):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((M, N)).astype(np.float32)
    # a k-way interaction of three-level variables plus label noise
    y = ((x[0] > 0.4) ^ (x[M // 2] < -0.3) ^ (x[M - 1] > 0) ^ (rng.random(N) < 0.1)).astype(np.uint8)
    return x, y


@pytest.mark.parametrize("k,div,M,N,D", [(4, 2, 4, 97, 1),      # one quadruple, a mostly empty last word
                                         (4, 2, 13, 300, 2),    # several CTAs, warps over c
                                         (4, 2, 8, 2500, 1),    # two 32-word chunks per class
                                         (4, 3, 9, 400, 2),     # four classes
                                         (5, 2, 5, 301, 1),     # one quintuple
                                         (5, 2, 10, 300, 2),    # warps over (c, e) pairs
                                         (5, 3, 7, 200, 1)])    # four classes, 1024 voxels
def test_kgen_matches_oracle(cuda, k, div, M, N, D):
    x, y = _data(M, N, 1000 * k + 10 * div + M, k)
    c = div + 1
    codes = oracle.discretize(x, div, D, 0.5, 23)
    ref = oracle.max_ig(codes, y, c, k, 0.25)
    g = _gpu_max_ig(cuda, x, y, k, div, D, 0.5, 0.25, 23)
    _check(codes, y, c, k, 0.25, *g, ref, range(M))
    gh = _gpu_max_ig(cuda, x, y, k, div, D, 0.5, 0.25, 23, host=True)
    for a, b in zip(g, gh):
        assert np.array_equal(a, b)


def test_kgen_unbalanced_classes(cuda):
    """Class sizes 37 and 263: the class-0 words end inside the first chunk."""
    rng = np.random.default_rng(4)
    M, N, D = 9, 300, 2
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = np.zeros(N, dtype=np.uint8)
    y[rng.choice(N, 37, replace=False)] = 1
    codes = oracle.discretize(x, 2, D, 0.5, 3)
    ref = oracle.max_ig(codes, y, 3, 4, 0.25)
    g = _gpu_max_ig(cuda, x, y, 4, 2, D, 0.5, 0.25, 3)
    _check(codes, y, 3, 4, 0.25, *g, ref, range(M))


@pytest.mark.parametrize("k,div,M,N,D", [(4, 2, 8, 300, 2), (5, 2, 7, 250, 1)])
def test_kgen_interesting_tuples(cuda, k, div, M, N, D):
    from paper_1811_00631_gb300 import mdfs
    x, y = _data(M, N, 77 + k, k)
    c = div + 1
    codes = oracle.discretize(x, div, D, 0.5, 31)
    allrec = oracle.interesting_tuples(codes, y, c, k, 0.25, -np.inf)
    thr = float(np.quantile([r[2] for r in allrec], 0.8))
    ref = [r for r in allrec if r[2] >= thr]
    got = mdfs.interesting_tuples(x, y, k, div, D, 0.5, 0.25, 31, thr, capacity=4096)
    _compare(codes, y, c, k, 0.25, thr, got, ref)


@pytest.mark.parametrize("k", [4, 5])
def test_kgen_shards_merge_to_the_scan(cuda, k):
    """Three shards of the pair items, their keys merged by max, decode to the
    unsharded scan bit for bit."""
    from paper_1811_00631_gb300 import mdfs
    M, N, D = (11, 300, 2) if k == 4 else (8, 250, 1)
    x, y = _data(M, N, 5 + k, k)
    full = _gpu_max_ig(cuda, x, y, k, 2, D, 0.5, 0.25, 9, host=True)
    keys = np.zeros(M, dtype=np.uint64)
    for s in range(3):
        keys = np.maximum(keys, mdfs.max_ig_shard(x, y, k, 2, D, 0.5, 0.25, 9, shard=s, n_shards=3))
    got = mdfs.decode_keys(keys, k)
    assert np.array_equal(np.asarray(got[0], dtype=np.float64), full[0])
    assert np.array_equal(np.asarray(got[1]), full[1]) and np.array_equal(np.asarray(got[2]), full[2])
