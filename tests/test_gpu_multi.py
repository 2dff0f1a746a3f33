"""mdfs_max_ig_multi: several dimensions k of the same data in one call equal
the mdfs_max_ig of each k bit for bit (so the parity of every single-k scan
against the FP64 oracle carries over), whether the scans share one
discretisation (k = 1, 2, 3 with two classes on the tensor-core kernels) or
run one after another (three classes, k = 4), with device and host buffers."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_00631_gb300 import build
    build.build()
    return torch


def _np(a):
    return np.asarray(a.cpu()) if hasattr(a, "cpu") else np.asarray(a)


def _same(a, b, what):
    for u, v, name in zip(a, b, ("ig", "tuples", "disc")):
        assert np.array_equal(_np(u), _np(v)), f"{what}: {name} differs"


@pytest.mark.parametrize("ks,div,N,M,D", [((1, 2, 3), 1, 2000, 500, 30),   # the bench step's shape, fused
                                          ((3, 2), 1, 700, 150, 3),         # fused, another order
                                          ((3, 1), 1, 600, 90, 2),          # fused without k = 2
                                          ((2, 3), 2, 600, 80, 2),          # three classes: one after another
                                          ((4, 2, 1), 1, 300, 24, 2),       # k = 4 beside k = 1, 2
                                          ((3, 4), 2, 300, 20, 2)])         # three classes, k = 4 generic
def test_multi_equals_single_calls(cuda, ks, div, N, M, D):
    from paper_1811_00631_gb300 import mdfs, synth
    torch = cuda
    ds = synth.madelon_like(N=N, M=M, seed=3)
    x = torch.from_numpy(ds.x).cuda()
    y = torch.from_numpy(ds.y).cuda()
    got = mdfs.max_ig_multi(x, y, ks, div, D, 0.5, 0.25, 11)
    assert sorted(got) == sorted(ks)
    for k in ks:
        _same(got[k], mdfs.max_ig(x, y, k, div, D, 0.5, 0.25, 11), f"k = {k}")
    host = mdfs.max_ig_multi(ds.x, ds.y, ks, div, D, 0.5, 0.25, 11)
    for k in ks:
        _same(got[k], host[k], f"k = {k}, host buffers")


def test_multi_repeated_calls_and_single_k(cuda):
    """Calls of different shapes on one stream: the fused scan's extra keys and
    the claim order of the triple kernel do not leak between calls."""
    from paper_1811_00631_gb300 import mdfs, synth
    torch = cuda
    a = synth.madelon_like(N=800, M=120, seed=5)
    b = synth.madelon_like(N=500, M=60, seed=6)
    xa, ya = torch.from_numpy(a.x).cuda(), torch.from_numpy(a.y).cuda()
    xb, yb = torch.from_numpy(b.x).cuda(), torch.from_numpy(b.y).cuda()
    first = mdfs.max_ig_multi(xa, ya, (2, 3), 1, 4, 0.5, 0.25, 1)
    mdfs.max_ig_multi(xb, yb, (1, 2, 3), 1, 2, 0.5, 0.25, 2)
    again = mdfs.max_ig_multi(xa, ya, (2, 3), 1, 4, 0.5, 0.25, 1)
    for k in (2, 3):
        _same(first[k], again[k], f"k = {k} repeated")
    only = mdfs.max_ig_multi(xb, yb, (3,), 1, 2, 0.5, 0.25, 2)
    _same(only[3], mdfs.max_ig(xb, yb, 3, 1, 2, 0.5, 0.25, 2), "k = 3 alone")
