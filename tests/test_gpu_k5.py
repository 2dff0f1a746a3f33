"""GPU (sm_103a) parity of the k = 5 scan (two classes per variable) against
the FP64 CPU oracle, through the C ABI.  Same bars as the other scans: IG
within 1e-4 absolute + 1e-5 relative, argmax partner quadruple and
discretisation equal unless the GPU's choice is an equally good maximiser."""
import numpy as np
import pytest

import oracle

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


@pytest.mark.parametrize("M,N,D", [(5, 97, 1), (7, 300, 2), (12, 300, 2), (9, 4500, 1), (6, 40, 3)])
def test_k5_matches_oracle(cuda, M, N, D):
    """Every variable against the brute-force oracle.  M = 5 is one quintuple;
    N = 4500 needs two staged chunks of 128 words; N = 40 leaves most of a
    32-sample word empty."""
    rng = np.random.default_rng(M * 1000 + N)
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[0] > 0) ^ (x[2] > 0) ^ (x[M - 1] > 0.3) ^ (rng.random(N) < 0.1)).astype(np.uint8)
    codes = oracle.discretize(x, 1, D, 0.5, 23)
    ref = oracle.max_ig(codes, y, 2, 5, 0.25)
    g = _gpu_max_ig(cuda, x, y, 5, 1, D, 0.5, 0.25, 23)
    _check(codes, y, 2, 5, 0.25, *g, ref, range(M))
    gh = _gpu_max_ig(cuda, x, y, 5, 1, D, 0.5, 0.25, 23, host=True)
    for a, b in zip(g, gh):
        assert np.array_equal(a, b)


def test_k5_int8_input(cuda):
    """int8 variables (ties at the cut points go to the upper class) give the
    oracle's result on the same int8 values."""
    from paper_1811_00631_gb300 import synth
    rng = np.random.default_rng(8)
    M, N, D = 8, 700, 2
    x8 = synth.to_int8(rng.standard_normal((M, N)), scale=6.0)
    y = ((x8[1] > 0) ^ (x8[4] > 2) ^ (x8[6] > -1) ^ (rng.random(N) < 0.1)).astype(np.uint8)
    codes = oracle.discretize(x8.astype(np.float32), 1, D, 0.5, 41)
    ref = oracle.max_ig(codes, y, 2, 5, 0.25)
    g = _gpu_max_ig(cuda, x8, y, 5, 1, D, 0.5, 0.25, 41)
    _check(codes, y, 2, 5, 0.25, *g, ref, range(M))


def test_k5_several_tiles_sampled(cuda):
    """M = 72: e and f span several 32-wide tiles (and the f-tile boundary
    above the diagonal tile); a sample of variables is checked against the
    oracle, each row scanning all C(71, 4) partner quadruples."""
    rng = np.random.default_rng(72)
    M, N, D = 72, 96, 1
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[3] > 0) ^ (x[36] > 0) ^ (x[71] > 0) ^ (rng.random(N) < 0.05)).astype(np.uint8)
    codes = oracle.discretize(x, 1, D, 0.5, 5)
    rows = np.array([0, 3, 34, 36, 67, 70, 71], dtype=np.int32)
    ref = oracle.max_ig(codes, y, 2, 5, 0.25, variables=rows)
    g = _gpu_max_ig(cuda, x, y, 5, 1, D, 0.5, 0.25, 5)
    _check(codes, y, 2, 5, 0.25, *g, ref, rows)


def test_k5_five_way_parity_found(cuda):
    """y = parity of five variables: invisible to every proper subset, so the
    five are the top five at k = 5 and each one's partners are the other four."""
    rng = np.random.default_rng(505)
    M, N = 14, 4000
    x = rng.standard_normal((M, N)).astype(np.float32)
    mem = [0, 3, 7, 8, 13]
    y = np.zeros(N, dtype=np.uint8)
    for m in mem:
        y ^= (x[m] > 0).astype(np.uint8)
    ig, tu, di = _gpu_max_ig(cuda, x, y, 5, 1, 1, 0.0, 0.25, 9)
    assert set(np.argsort(-ig)[:5].tolist()) == set(mem)
    for m in mem:
        assert tu[m].tolist() == [v for v in mem if v != m]
    ig4, _, _ = _gpu_max_ig(cuda, x, y, 4, 1, 1, 0.0, 0.25, 9)
    assert ig4.max() < 0.02 * ig[mem].min()


def test_k5_errors(cuda):
    from paper_1811_00631_gb300 import mdfs
    x = np.random.default_rng(0).standard_normal((7, 50)).astype(np.float32)
    y = (np.arange(50) % 2).astype(np.uint8)
    with pytest.raises(mdfs.MdfsError):
        mdfs.max_ig(x, y, 5, 4, 1)  # five classes: more than any scan supports
    with pytest.raises(mdfs.MdfsError):
        mdfs.max_ig(x[:4], y, 5, 1, 1)  # fewer variables than k
    with pytest.raises(mdfs.MdfsError):
        mdfs.interesting_tuples(x, y, 5, 4, 1)  # five classes
    xm = np.random.default_rng(2).standard_normal((200, 8)).astype(np.float32)
    ym = (np.arange(8) % 2).astype(np.uint8)
    with pytest.raises(mdfs.MdfsError):
        mdfs.max_ig(xm, ym, 5, 2, 67)  # three classes: 67 C(200, 4) >= 2^32 (one key word)
    xl = np.random.default_rng(1).standard_normal((600, 8)).astype(np.float32)
    yl = (np.arange(8) % 2).astype(np.uint8)
    with pytest.raises(mdfs.MdfsError):
        mdfs.max_ig(xl, yl, 5, 1, 1)  # C(600, 4) >= 2^32: keys cannot index the quadruple


def test_k5_per_discretisation_keys(cuda, monkeypatch):
    """Per-discretisation keys (used when D C(M,4) >= 2^32, forced here with
    MDFS_K5_DISC_KEYS) give exactly the single-key result.  With range 0 every
    discretisation is the same equipotent split, so each maximum is tied
    across all D discretisations and must report the lowest one."""
    from paper_1811_00631_gb300 import mdfs
    rng = np.random.default_rng(77)
    M, N = 11, 600
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[1] > 0) ^ (x[4] > 0) ^ (x[9] > 0) ^ (rng.random(N) < 0.1)).astype(np.uint8)
    for D, r in ((4, 0.5), (3, 0.0)):
        want = _gpu_max_ig(cuda, x, y, 5, 1, D, r, 0.25, 31)
        monkeypatch.setenv("MDFS_K5_DISC_KEYS", "1")
        got = _gpu_max_ig(cuda, x, y, 5, 1, D, r, 0.25, 31)
        monkeypatch.delenv("MDFS_K5_DISC_KEYS")
        for a, b in zip(got, want):
            assert np.array_equal(a, b)
        if r == 0.0:
            assert np.all(got[2] == 0)
        codes = oracle.discretize(x, 1, D, r, 31)
        ref = oracle.max_ig(codes, y, 2, 5, 0.25)
        _check(codes, y, 2, 5, 0.25, *got, ref, range(M))


def test_k5_select_pipeline(cuda):
    """The selection pipeline at k = 5 (contrast variables, fit, Holm)
    against the oracle's."""
    from paper_1811_00631_gb300 import mdfs
    from test_gpu_select import _check_select
    rng = np.random.default_rng(55)
    M, N, nc = 7, 500, 6
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = np.zeros(N, dtype=np.uint8)
    for m in (0, 2, 3, 5, 6):
        y ^= (x[m] > 0).astype(np.uint8)
    ref = oracle.select(x, y, nc, 5, 1, 1, 0.0, 0.25, seed=3)
    g = mdfs.select(x, y, nc, 5, 1, 1, 0.0, 0.25, seed=3)
    _check_select(g, ref, M, 5, 1, 0.05)


@pytest.mark.parametrize("k,M,c", [(3, 40, 3), (4, 20, 2), (5, 12, 2)])
def test_discretisation_chunks_give_the_same_result(cuda, monkeypatch, k, M, c):
    """Table passes over chunks of discretisations (forced to one per chunk
    with MDFS_PAIR_TABLE_BYTES) give exactly the single-chunk result: the
    chunk offsets of the pair, triple and quadruple tables and of the keys."""
    rng = np.random.default_rng(k * 10 + M)
    N, D = 300, 4
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[0] > 0) ^ (x[M // 2] > 0) ^ (rng.random(N) < 0.1)).astype(np.uint8)
    want = _gpu_max_ig(cuda, x, y, k, c - 1, D, 0.5, 0.25, 19)
    monkeypatch.setenv("MDFS_PAIR_TABLE_BYTES", "1")
    got = _gpu_max_ig(cuda, x, y, k, c - 1, D, 0.5, 0.25, 19)
    monkeypatch.delenv("MDFS_PAIR_TABLE_BYTES")
    for a, b in zip(got, want):
        assert np.array_equal(a, b)
