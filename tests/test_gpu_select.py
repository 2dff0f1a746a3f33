"""GPU (sm_103a) parity of the selection pipeline of section "Canonical package
usage" (arXiv 1811.00631): contrast variables, p-value adjustment and
mdfs_select, against the FP64 CPU oracle.  Every call goes through the C ABI.

Bars: contrast rows and sources bit-exact; adjusted p-values equal to the
oracle's definitions within 1e-12 relative (they are FP64 on both sides); IG
within 1e-4 + 1e-5 |IG|; p-values within 1e-9 of the oracle's formula applied to
the GPU's IG and fitted T; the relevant set equal except where an adjusted
p-value lies within 1e-6 of the level.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

METHODS = ("none", "bonferroni", "holm", "hochberg", "BH", "BY")


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_00631_gb300 import build
    build.build()
    return torch


@pytest.mark.parametrize("M,N,nc", [(7, 333, 20), (50, 2000, 50), (1, 2, 5), (3, 1025, 1), (40, 129, 3)])
def test_contrast_bit_exact(cuda, M, N, nc):
    from paper_1811_00631_gb300 import mdfs
    rng = np.random.default_rng(M * 1000 + N)
    x = rng.standard_normal((M, N)).astype(np.float32)
    want, wsrc = oracle.contrast(x, nc, seed=2**40 + M)
    got, gsrc = mdfs.contrast(cuda.from_numpy(x).cuda(), nc, seed=2**40 + M)
    assert np.array_equal(got.cpu().numpy(), want)
    assert np.array_equal(gsrc.cpu().numpy(), wsrc)
    got_h, gsrc_h = mdfs.contrast(x, nc, seed=2**40 + M)  # host pointers
    assert np.array_equal(got_h, want) and np.array_equal(gsrc_h, wsrc)


def test_contrast_int8(cuda):
    from paper_1811_00631_gb300 import mdfs, synth
    rng = np.random.default_rng(8)
    x8 = synth.to_int8(rng.standard_normal((11, 500)), scale=3.0)
    want, wsrc = oracle.contrast(x8.astype(np.float32), 17, seed=5)
    got, gsrc = mdfs.contrast(cuda.from_numpy(x8).cuda(), 17, seed=5)
    assert got.dtype == cuda.int8
    assert np.array_equal(got.cpu().numpy().astype(np.float32), want)
    assert np.array_equal(gsrc.cpu().numpy(), wsrc)


@pytest.mark.parametrize("method", METHODS)
def test_p_adjust_matches_oracle(cuda, method):
    from paper_1811_00631_gb300 import mdfs
    rng = np.random.default_rng(METHODS.index(method))
    for m in (1, 2, 3, 31, 1024, 1025, 5000, 65536):
        p = rng.random(m) ** 4
        p[: m // 7] = p[0]  # ties
        want = oracle.p_adjust(p, method)
        got = mdfs.p_adjust(cuda.from_numpy(p).cuda(), method).cpu().numpy()
        assert np.allclose(got, want, rtol=1e-12, atol=0), (m, np.max(np.abs(got - want)))
    got_h = mdfs.p_adjust(p, method)
    assert np.allclose(got_h, want, rtol=1e-12, atol=0)


def test_p_adjust_nan_entries(cuda):
    """NaN p-values are not counted in m and stay NaN."""
    from paper_1811_00631_gb300 import mdfs
    p = np.array([0.01, np.nan, 0.04, 0.03, np.nan, 0.2])
    got = mdfs.p_adjust(p, "holm")
    finite = ~np.isnan(p)
    assert np.all(np.isnan(got[~finite]))
    assert np.allclose(got[finite], oracle.p_adjust(p[finite], "holm"), rtol=1e-12)


def _check_select(g, ref, M, k, divisions, level):
    atol, rtol = 1e-4, 1e-5
    ig = g["ig"].astype(np.float64)
    assert np.all(np.abs(ig - ref["ig"]) <= atol + rtol * np.abs(ref["ig"]))
    # p-values: the definition applied to the GPU's IG and fitted T
    c = divisions + 1
    df = (c - 1) * c ** (k - 1)
    want_p = np.array([1.0 - oracle.chi2_cdf(2.0 * v, df) ** g["n_eff"] if v > 0 else 1.0 for v in ig])
    assert np.allclose(g["p_value"], want_p, rtol=1e-9, atol=1e-12)
    assert g["n_eff"] == pytest.approx(ref["n_eff"], rel=1e-4)
    assert g["ig_lim"] == pytest.approx(ref["ig_lim"], rel=1e-4)
    assert np.array_equal(g["contrast_src"], ref["src"])
    want_adj = oracle.p_adjust(g["p_value"], "holm")
    assert np.allclose(g["adjusted_p_value"], want_adj, rtol=1e-12, atol=0)
    near = np.abs(want_adj - level) < 1e-6
    assert np.array_equal(g["relevant"][~near], (want_adj < level)[~near])
    assert np.array_equal(g["relevant"][~near], ref["relevant"][~near])


@pytest.mark.parametrize("k", [1, 2])
def test_select_matches_oracle(cuda, k):
    from paper_1811_00631_gb300 import mdfs
    rng = np.random.default_rng(30 + k)
    M, N, nc = 12, 400, 24
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[2] > 0) ^ (x[7] > 0)).astype(np.uint8) if k == 2 else (x[4] + 0.5 * rng.standard_normal(N) > 0).astype(np.uint8)
    flip = rng.random(N) < 0.05
    y[flip] ^= 1
    ref = oracle.select(x, y, nc, k, 1, 1, 0.0, 0.25, seed=7)
    g = mdfs.select(x, y, nc, k, 1, 1, 0.0, 0.25, seed=7)
    _check_select(g, ref, M, k, 1, 0.05)
    if k == 2:
        assert g["relevant"][2] and g["relevant"][7]
        # the argmax tuple of 2 is 7 (partners index the extended set)
        assert g["tuples"][2, 0] == 7 and g["tuples"][7, 0] == 2
    else:
        assert g["relevant"][4]


def test_select_device_outputs_and_discretisations(cuda):
    """Device tensors in and out, several discretisations and three classes."""
    from paper_1811_00631_gb300 import mdfs
    rng = np.random.default_rng(44)
    M, N, nc = 10, 600, 30
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = (x[1] + x[3] > 0.2).astype(np.uint8)
    ref = oracle.select(x, y, nc, 1, 2, 4, 0.5, 0.25, seed=123)
    g = mdfs.select(cuda.from_numpy(x).cuda(), cuda.from_numpy(y).cuda(), nc, 1, 2, 4, 0.5, 0.25, seed=123)
    gh = {key: (v.cpu().numpy() if hasattr(v, "cpu") else v) for key, v in g.items()}
    _check_select(gh, ref, M, 1, 2, 0.05)
    assert gh["relevant"][1] and gh["relevant"][3]


def test_select_errors(cuda):
    from paper_1811_00631_gb300 import mdfs
    x = np.random.default_rng(0).standard_normal((5, 50)).astype(np.float32)
    y = (np.arange(50) % 2).astype(np.uint8)
    with pytest.raises(mdfs.MdfsError):
        mdfs.select(x, y, 0, 1)  # n_contrast must be >= 1
    with pytest.raises(mdfs.MdfsError):
        mdfs.select(x, y, 65535, 1)  # M + n_contrast > 65535
    with pytest.raises(mdfs.MdfsError):
        mdfs.select(x, np.zeros(50, dtype=np.uint8), 10, 1)  # single class
    with pytest.raises(KeyError):
        mdfs.select(x, y, 10, 1, p_adjust_method="unknown")
