"""The lower bound of SH3 with which the k = 3 tensor-core epilogue skips
triples, checked on the CPU.

Each voxel's term of the regularised entropy (Eqs. H, p, beta) is
E(m0, m1) = f(m0 + m1) - f(m0) - f(m1), f(t) = t ln t, with the smoothed class
counts m_d = n_d + beta_d.  E = (m0 + m1) H(m0 / (m0 + m1)) and the binary
entropy bound H(p) >= 4 ln 2 p (1 - p) give SH3 >= 4 ln 2 sum_v m0 m1 / (m0 + m1).
The kernel evaluates that sum in float32 as one fraction num / den (two
lanes of packed FP32 pairs, then one cross-lane step) and skips
a triple when num > (hi + kBoundRel |hi| + kBoundAbs) den, where hi is the
largest SH3 (in units of 4 ln 2) for which some role could still reach its
key.  These tests repeat that float32 arithmetic and check, against the exact
FP64 entropies, that a skipped triple never has SH3 <= hi.
"""
import math

import numpy as np

LN2 = math.log(2.0)
REL, ABS = 1.0 / 4096.0, 0.05


def _f(t):
    return t * np.log(t)


def _sh_exact(n0, n1, b0, b1):
    """sum over voxels of E(n0 + b0, n1 + b1) in FP64 (nats)."""
    return np.sum(_f(n0 + n1 + b0 + b1) - _f(n0 + b0) - _f(n1 + b1), axis=-1)


def _fmaf(a, b, c):
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def _frac_add(a, b, c, d):
    return _fmaf(a, d, np.float32(c * b)), np.float32(b * d)


def _lb_fraction(m, w):
    """num, den of sum_v m_v w_v / (m_v + w_v) in the kernel's float32 order:
    two lanes of packed pairs, lane x accumulating voxels 0..3 and lane y
    voxels 4..7 as (0 + 1) + (2 + 3) fractions, then one cross-lane step."""
    m = m.astype(np.float32)
    w = w.astype(np.float32)
    p = (m * w).astype(np.float32)
    s = (m + w).astype(np.float32)
    out = []
    for lane in (0, 4):
        nab, dab = _frac_add(p[..., lane], s[..., lane], p[..., lane + 1], s[..., lane + 1])
        ncd, dcd = _frac_add(p[..., lane + 2], s[..., lane + 2], p[..., lane + 3], s[..., lane + 3])
        out.append(_frac_add(nab, dab, ncd, dcd))
    (nx, dx), (ny, dy) = out
    return _fmaf(nx, dy, np.float32(ny * dx)), np.float32(dx * dy)


def test_binary_entropy_bound():
    p = np.linspace(0.0, 1.0, 100001)
    with np.errstate(divide="ignore", invalid="ignore"):
        h = -np.where(p > 0, p * np.log(p), 0) - np.where(p < 1, (1 - p) * np.log(1 - p), 0)
    assert np.all(h >= 4 * LN2 * p * (1 - p) - 1e-15)
    assert abs(h[50000] - LN2) < 1e-15  # equality at p = 1/2


def test_bound_is_below_the_exact_entropy_and_the_skip_is_safe():
    rng = np.random.default_rng(0)
    for trial in range(40):
        b0, b1 = (float(v) for v in rng.choice([1e-3, 0.01, 0.25, 1.0, 7.0, 40.0], size=2))
        hi_scale = rng.choice([10, 200, 4095])
        n = rng.integers(0, hi_scale + 1, size=(20000, 2, 8)).astype(np.float64)
        n[::7, 0, :4] = 0  # empty classes in half the voxels
        n[::11, 1, 3] = 4095
        sh = _sh_exact(n[:, 0], n[:, 1], b0, b1) / (4 * LN2)  # SH3 in the bound's units
        num, den = _lb_fraction(n[:, 0] + np.float32(b0), n[:, 1] + np.float32(b1))
        lb = np.float64(num) / np.float64(den)
        assert np.all(lb <= sh * (1 + 1e-6) + 1e-9), trial
        # thresholds at, just below and just above the exact value
        for off in (0.0, -1e-3, 1e-3, -0.04, 0.04, -1.0, 1.0):
            hi = (sh + off).astype(np.float32)
            lim = _fmaf(np.abs(hi), np.float32(REL), np.float32(hi + np.float32(ABS)))
            skip = np.float32(num) > np.float32(lim * den)
            # skipping is allowed only when no role can be reached: SH3 > hi
            assert not np.any(skip & (sh <= hi.astype(np.float64))), (trial, off)


def test_bound_is_tight_for_balanced_voxels():
    """Voxels whose two classes are nearly equal (noise) leave a slack of a
    few hundredths of a nat each, so noise triples are skipped once the keys
    are a few nats above a typical triple's information."""
    rng = np.random.default_rng(1)
    tot = rng.integers(200, 300, size=(1000, 8))
    n0 = rng.binomial(tot, 0.5).astype(np.float64)
    n1 = tot - n0
    sh = _sh_exact(n0, n1, 0.25, 0.25)
    num, den = _lb_fraction(n0 + 0.25, n1 + 0.25)
    slack = sh - 4 * LN2 * np.float64(num) / np.float64(den)
    assert np.all(slack >= 0) and np.median(slack) < 2.0
