"""Pins of the FP64 CPU oracle against facts the paper and mathematics fix.

None of these tests compares the oracle with itself: every expected value is a
published known answer, a closed form, an independent library routine
(scipy, scikit-learn), an invariant, or a brute-force enumeration written
differently from the oracle.  Paper references are to arXiv 1811.00631.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_1811_00631_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Philox4x32-10 (generator of the discretisation shares)
# --------------------------------------------------------------------------
def test_philox_known_answers():
    """Published known-answer vectors of Philox4x32-10 (Salmon et al., SC'11)."""
    n = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            out = oracle.philox4x32_10(w[0:4], w[4:6])
            assert list(out) == w[6:10]
            n += 1
    assert n == 3


# --------------------------------------------------------------------------
# Discretisation (section "Algorithm and implementation")
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N,c", [(2000, 2), (2000, 3), (2000, 4), (7, 3), (5, 5)])
def test_range_zero_is_equipotent(N, c):
    """range = 0 gives an equipotent split: positions floor(N j / c)."""
    for v in range(3):
        for d in range(3):
            pos = oracle.cut_positions(N, c - 1, v, d, 0.0, seed=123)
            assert list(pos) == [max(j, (N * j) // c) for j in range(1, c)]


def test_range_zero_class_sizes_distinct_values():
    rng = np.random.default_rng(0)
    x = rng.permutation(2000).astype(np.float32).reshape(1, -1)
    codes = oracle.discretize(x, divisions=1, discretizations=2, range_=0.0, seed=9)
    assert np.bincount(codes[0, 0], minlength=2).tolist() == [1000, 1000]
    codes = oracle.discretize(x, divisions=2, discretizations=1, range_=0.0, seed=9)
    assert np.bincount(codes[0, 0], minlength=3).tolist() == [666, 667, 667]


@pytest.mark.parametrize("divisions", [1, 2, 3])
def test_codes_rank_consistent(divisions):
    """Codes are a monotone function of the value; class sizes equal the
    position differences (distinct values); every class is non-empty."""
    c = divisions + 1
    rng = np.random.default_rng(divisions)
    M, N, D = 4, 301, 5
    x = rng.standard_normal((M, N)).astype(np.float32)
    codes = oracle.discretize(x, divisions, D, 0.7, seed=77)
    for d in range(D):
        for v in range(M):
            order = np.argsort(x[v], kind="stable")
            cs = codes[d, v, order]
            assert np.all(np.diff(cs.astype(int)) >= 0)
            pos = oracle.cut_positions(N, divisions, v, d, 0.7, 77)
            bounds = [0] + list(pos) + [N]
            sizes = np.bincount(codes[d, v], minlength=c)
            assert sizes.tolist() == [bounds[j + 1] - bounds[j] for j in range(c)]
            assert np.all(sizes > 0)


def test_positions_strict_and_in_range():
    for N in [2, 3, 4, 10, 57]:
        for c in [2, 3, 4]:
            if N < c:
                continue
            for v in range(20):
                pos = oracle.cut_positions(N, c - 1, v, 3, 1.0, seed=5)
                assert pos[0] >= 1 and pos[-1] <= N - 1
                assert np.all(np.diff(pos) > 0)


def test_share_distribution():
    """Shares ~ U(1-r, 1+r): with c = 2 the first-class fraction is
    s0 / (s0 + s1); its mean is 1/2 by symmetry and its range is bounded by
    (1-r)/2 and (1+r)/2 (the ratio bounds of two shares in [1-r, 1+r])."""
    N, r = 100000, 0.5
    fr = np.array([oracle.cut_positions(N, 1, v, 0, r, seed=11)[0] / N for v in range(4000)])
    assert abs(fr.mean() - 0.5) < 3 * fr.std() / math.sqrt(len(fr)) + 1e-4
    lo = (1 - r) / ((1 - r) + (1 + r))
    hi = (1 + r) / ((1 - r) + (1 + r))
    assert fr.min() >= lo - 1e-4 and fr.max() <= hi + 1e-4
    # the spread is far from a point mass: shares really are random
    assert fr.std() > 0.05


def test_each_discretisation_draws_its_own_thresholds():
    """The discretisation is repeated with fresh random thresholds (section
    "Algorithm and implementation"): with range > 0 the cut positions of one
    variable differ between discretisations, and so do those of different
    variables within one discretisation."""
    N, div = 2000, 2
    per_disc = {tuple(oracle.cut_positions(N, div, 0, d, 0.5, seed=4)) for d in range(20)}
    per_var = {tuple(oracle.cut_positions(N, div, v, 0, 0.5, seed=4)) for v in range(20)}
    assert len(per_disc) >= 18 and len(per_var) >= 18


def test_ties_go_to_upper_class():
    x = np.array([[0, 1, 1, 1, 2, 3]], dtype=np.float32)
    codes = oracle.discretize(x, 1, 1, 0.0, seed=1)  # position 3 -> threshold 1.0
    assert codes[0, 0].tolist() == [0, 1, 1, 1, 1, 1]


# --------------------------------------------------------------------------
# Regularised entropy SH and IG (Eqs. 1, H, p, beta)
# --------------------------------------------------------------------------
def _sh_from_probabilities(cols, y, c, xi):
    """-sum_v sum_d (n^d_v + b^d) ln p^d_v with p from Eq. p and b from Eq. beta,
    enumerated voxel by voxel (the paper's form, not the oracle's x ln x form)."""
    n0 = int(np.sum(y == 0))
    n1 = int(np.sum(y == 1))
    b = [xi * n0 / min(n0, n1), xi * n1 / min(n0, n1)]
    total = 0.0
    for vox in itertools.product(range(c), repeat=len(cols)):
        sel = np.ones(len(y), dtype=bool)
        for col, a in zip(cols, vox):
            sel &= col == a
        cnt = [int(np.sum(sel & (y == 0))), int(np.sum(sel & (y == 1)))]
        den = cnt[0] + b[0] + cnt[1] + b[1]
        for d in (0, 1):
            p = (cnt[d] + b[d]) / den
            total -= (cnt[d] + b[d]) * math.log(p)
    return total


def test_sh_hand_enumerated_tables():
    """Tiny tables worked by hand.  y = 0,0,0,1 (N0 = 3, N1 = 1), xi = 0.5:
    beta0 = 1.5, beta1 = 0.5.  With x = 0,0,1,1:
      SH(empty) = 6 ln 6 - 4.5 ln 4.5 - 1.5 ln 1.5
      SH({x})   = [4 ln 4 - 3.5 ln 3.5 - 0.5 ln 0.5] + [4 ln 4 - 2.5 ln 2.5 - 1.5 ln 1.5]."""
    y = np.array([0, 0, 0, 1], dtype=np.uint8)
    x = np.array([0, 0, 1, 1], dtype=np.uint8)
    b0, b1 = oracle.pseudocounts(y, 0.5)
    assert (b0, b1) == (1.5, 0.5)
    L = math.log
    want0 = 6 * L(6) - 4.5 * L(4.5) - 1.5 * L(1.5)
    want1 = (4 * L(4) - 3.5 * L(3.5) - 0.5 * L(0.5)) + (4 * L(4) - 2.5 * L(2.5) - 1.5 * L(1.5))
    assert oracle.sh([], y, 2, b0, b1) == pytest.approx(want0, abs=1e-12)
    assert oracle.sh([x], y, 2, b0, b1) == pytest.approx(want1, abs=1e-12)
    # balanced case, xi = 0.5: independent x gives IG = -ln 2 (regularisation)
    y2 = np.array([0, 0, 1, 1], dtype=np.uint8)
    x2 = np.array([0, 1, 0, 1], dtype=np.uint8)
    codes = x2.reshape(1, 1, 4)
    assert oracle.ig_one(codes, y2, 2, 0.5, 0, 0, []) == pytest.approx(-math.log(2), abs=1e-12)


@pytest.mark.parametrize("c,nvars,xi", [(2, 1, 0.25), (3, 2, 0.1), (2, 3, 0.9), (4, 2, 0.5)])
def test_sh_matches_probability_form(c, nvars, xi):
    """The oracle's x ln x form equals the paper's -sum (n+b) ln p form (Eq. p)."""
    rng = np.random.default_rng(c * 10 + nvars)
    N = 37
    y = (rng.random(N) < 0.3).astype(np.uint8)
    y[0], y[1] = 0, 1
    cols = [rng.integers(0, c, N).astype(np.uint8) for _ in range(nvars)]
    b0, b1 = oracle.pseudocounts(y, xi)
    assert oracle.sh(cols, y, c, b0, b1) == pytest.approx(_sh_from_probabilities(cols, y, c, xi), rel=1e-12)


def test_sh_limit_is_plugin_conditional_entropy():
    """xi -> 0: SH(S) -> N * H_plugin(y | S) (scipy.stats.entropy per voxel, nats)."""
    from scipy.stats import entropy
    rng = np.random.default_rng(3)
    N, c = 500, 3
    y = (rng.random(N) < 0.4).astype(np.uint8)
    cols = [rng.integers(0, c, N).astype(np.uint8) for _ in range(2)]
    b0, b1 = oracle.pseudocounts(y, 1e-10)
    joint = cols[0].astype(int) * c + cols[1]
    h = 0.0
    for v in np.unique(joint):
        sel = joint == v
        h += sel.sum() / N * entropy(np.bincount(y[sel], minlength=2))
    assert oracle.sh(cols, y, c, b0, b1) == pytest.approx(N * h, abs=1e-6)


def test_k1_is_half_g_statistic():
    """Eq. 3: IG^1 = N (H(y) - H(y|x)) is the G-test statistic over 2 (nats):
    scipy's log-likelihood chi2_contingency without Yates correction gives G."""
    from scipy.stats import chi2_contingency
    rng = np.random.default_rng(4)
    N, c = 800, 3
    x = rng.standard_normal((3, N)).astype(np.float32)
    y = ((x[0] > 0.3) ^ (rng.random(N) < 0.35)).astype(np.uint8)
    codes = oracle.discretize(x, c - 1, 2, 0.3, seed=8)
    res = oracle.max_ig(codes, y, c, 1, 1e-10)
    for v in range(3):
        best = -np.inf
        for d in range(2):
            table = np.zeros((c, 2))
            np.add.at(table, (codes[d, v], y), 1)
            g, _, _, _ = chi2_contingency(table, correction=False, lambda_="log-likelihood")
            best = max(best, g / 2)
        assert res["ig"][v] == pytest.approx(best, abs=1e-5)


def _cmi_sklearn(y, cols_s, col_i, c):
    from sklearn.metrics import mutual_info_score
    def joint(cs):
        j = np.zeros(len(y), dtype=np.int64)
        for col in cs:
            j = j * c + col
        return j
    mi_si = mutual_info_score(y, joint(list(cols_s) + [col_i]))
    mi_s = mutual_info_score(y, joint(cols_s)) if cols_s else 0.0
    return mi_si - mi_s


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_ig_limit_is_n_times_conditional_mutual_information(k):
    """xi -> 0: IG(i | S) -> N * I(y; x_i | S) = N [I(y; S, x_i) - I(y; S)]
    (scikit-learn's plug-in mutual information, nats)."""
    pytest.importorskip("sklearn")
    rng = np.random.default_rng(k)
    N, M, c = 300, 5, 3
    codes = rng.integers(0, c, (1, M, N)).astype(np.uint8)
    y = ((codes[0, 0] + codes[0, 1]) % 2).astype(np.uint8) ^ (rng.random(N) < 0.2).astype(np.uint8)
    for S in itertools.combinations(range(1, M), k - 1):
        want = N * _cmi_sklearn(y, [codes[0, s] for s in S], codes[0, 0], c)
        got = oracle.ig_one(codes, y, c, 1e-10, 0, 0, list(S))
        assert got == pytest.approx(want, abs=1e-6)


@pytest.mark.parametrize("k,c,xi", [(2, 2, 0.25), (2, 3, 0.5), (3, 2, 0.25), (3, 4, 0.1), (4, 2, 0.25), (4, 3, 0.3),
                                    (5, 2, 0.25), (5, 3, 0.2)])
def test_duplicate_variable_closed_form(k, c, xi):
    """If x_i duplicates a member of S, the extra voxels are all empty:
    IG(i|S) = -c^(k-1) (c-1) [f(b0+b1) - f(b0) - f(b1)],  f(x) = x ln x."""
    rng = np.random.default_rng(7)
    N, M = 64, 6
    codes = rng.integers(0, c, (1, M, N)).astype(np.uint8)
    codes[0, 4] = codes[0, 1]
    y = (rng.random(N) < 0.4).astype(np.uint8)
    b0, b1 = oracle.pseudocounts(y, xi)
    f = lambda t: t * math.log(t)
    want = -(c ** (k - 1)) * (c - 1) * (f(b0 + b1) - f(b0) - f(b1))
    S = [1, 2, 3, 5][: k - 1]
    assert oracle.ig_one(codes, y, c, xi, 0, 4, S) == pytest.approx(want, abs=1e-9)


def test_null_scale_is_chi2():
    """A non-informative single tuple: 2 IG ~ chi^2 with (c-1) c^(k-1) degrees
    of freedom (section "Theory"); for k = 1, c = 2 the mean of IG is 1/2
    (it would be 0.72 in bits)."""
    rng = np.random.default_rng(12)
    N, c, reps = 5000, 2, 2000
    ys = (rng.random((reps, N)) < 0.5).astype(np.uint8)
    xs = rng.integers(0, c, (reps, N)).astype(np.uint8)
    vals = []
    for r in range(reps):
        vals.append(2 * oracle.ig_one(xs[r].reshape(1, 1, N), ys[r], c, 1e-9, 0, 0, []))
    vals = np.array(vals)
    df = 1
    assert abs(vals.mean() - df) < 3 * math.sqrt(2 * df / reps)


def test_null_scale_k4_c2():
    """k = 4, c = 2: 2 IG of a null single tuple has mean df = (c-1) c^3 = 8."""
    rng = np.random.default_rng(14)
    N, c, reps = 5000, 2, 600
    vals = []
    for r in range(reps):
        y = (rng.random(N) < 0.5).astype(np.uint8)
        codes = rng.integers(0, c, (1, 4, N)).astype(np.uint8)
        vals.append(2 * oracle.ig_one(codes, y, c, 1e-9, 0, 0, [1, 2, 3]))
    df = (c - 1) * c ** 3
    vals = np.array(vals)
    assert abs(vals.mean() - df) < 3 * math.sqrt(2 * df / reps)


def test_null_scale_k5_c2():
    """k = 5, c = 2: 2 IG of a null single tuple has mean df = (c-1) c^4 = 16."""
    rng = np.random.default_rng(15)
    N, c, reps = 5000, 2, 400
    vals = []
    for r in range(reps):
        y = (rng.random(N) < 0.5).astype(np.uint8)
        codes = rng.integers(0, c, (1, 5, N)).astype(np.uint8)
        vals.append(2 * oracle.ig_one(codes, y, c, 1e-9, 0, 0, [1, 2, 3, 4]))
    df = (c - 1) * c ** 4
    vals = np.array(vals)
    assert abs(vals.mean() - df) < 3 * math.sqrt(2 * df / reps)


def test_null_scale_k4_c3():
    """k = 4, c = 3: 2 IG of a null single tuple has mean df = (c-1) c^3 = 54
    (section "Theory").  The chi^2 law is asymptotic: with 162 cells the mean
    exceeds df by O(cells / N) (about 4 % at N = 8000), so N is large here."""
    rng = np.random.default_rng(16)
    N, c, reps = 40000, 3, 300
    vals = []
    for r in range(reps):
        y = (rng.random(N) < 0.5).astype(np.uint8)
        codes = rng.integers(0, c, (1, 4, N)).astype(np.uint8)
        vals.append(2 * oracle.ig_one(codes, y, c, 1e-9, 0, 0, [1, 2, 3]))
    df = (c - 1) * c ** 3
    vals = np.array(vals)
    assert abs(vals.mean() - df) < 3 * math.sqrt(2 * df / reps)


def test_null_scale_k2_c3():
    rng = np.random.default_rng(13)
    N, c, reps = 5000, 3, 600
    vals = []
    for r in range(reps):
        y = (rng.random(N) < 0.5).astype(np.uint8)
        codes = rng.integers(0, c, (1, 2, N)).astype(np.uint8)
        vals.append(2 * oracle.ig_one(codes, y, c, 1e-9, 0, 0, [1]))
    df = (c - 1) * c
    vals = np.array(vals)
    assert abs(vals.mean() - df) < 3 * math.sqrt(2 * df / reps)


# --------------------------------------------------------------------------
# max / argmax over tuples and discretisations
# --------------------------------------------------------------------------
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_max_ig_brute_force(k):
    """Exhaustive Python enumeration (sklearn CMI, xi -> 0) of the max over
    (discretisation, tuple) with the lowest-(d, S) tie-break."""
    pytest.importorskip("sklearn")
    rng = np.random.default_rng(20 + k)
    N, M, c, D = 120, 6, 2, 3
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[0] > 0) ^ (x[1] > 0) ^ (rng.random(N) < 0.15)).astype(np.uint8)
    codes = oracle.discretize(x, c - 1, D, 0.5, seed=3)
    res = oracle.max_ig(codes, y, c, k, 1e-10)
    for i in range(M):
        best, arg = -np.inf, None
        for d in range(D):
            others = [m for m in range(M) if m != i]
            for S in itertools.combinations(others, k - 1):
                g = N * _cmi_sklearn(y, [codes[d, s] for s in S], codes[d, i], c)
                if g > best + 1e-9:
                    best, arg = g, (d, S)
        assert res["ig"][i] == pytest.approx(best, abs=1e-6)
        assert res["disc"][i] == arg[0]
        assert tuple(res["tuples"][i]) == arg[1]
        assert res["second"][i] <= res["ig"][i]


def _brute_max(codes, y, c, k, xi, i):
    """IG(i | S) for every discretisation d and every set S of k - 1 distinct
    variables other than i (Eq. 1), in the order (d ascending, S
    lexicographic), with SH in the paper's -sum (n+b) ln p form.  Returns
    (max, runner-up over every other (d, S), {(d, S): IG} in that order)."""
    D, M, _ = codes.shape
    table = {}
    for d in range(D):
        for S in itertools.combinations([m for m in range(M) if m != i], k - 1):
            cols = [codes[d, s] for s in S]
            table[(d, S)] = (_sh_from_probabilities(cols, y, c, xi)
                             - _sh_from_probabilities(cols + [codes[d, i]], y, c, xi))
    vals = sorted(table.values(), reverse=True)
    return vals[0], (vals[1] if len(vals) > 1 else -np.inf), table


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_max_ig_brute_force_negative_gains(k):
    """Few samples, three classes and a large xi: the pseudocounts make most
    gains negative.  The maximum still ranges only over sets of k - 1 distinct
    variables other than i (Eq. 1), even where every such gain is below zero
    (a set holding i itself, or one variable twice, would score 0 or a
    lower-order gain instead).  Many (d, S) tie here in exact arithmetic, so
    the reported (d, S) must be a maximiser within rounding, and the runner-up
    must be the best of the other candidates."""
    rng = np.random.default_rng(40 + k)
    N, M, c, D, xi = 10, 6, 3, 2, 0.9
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = (rng.random(N) < 0.5).astype(np.uint8)
    y[0], y[1] = 0, 1
    codes = oracle.discretize(x, c - 1, D, 0.5, seed=5)
    res = oracle.max_ig(codes, y, c, k, xi)
    negative = 0
    for i in range(M):
        best, second, table = _brute_max(codes, y, c, k, xi, i)
        negative += best < 0
        d, S = int(res["disc"][i]), tuple(int(t) for t in res["tuples"][i])
        assert len(set(S)) == k - 1 and i not in S and list(S) == sorted(S)
        assert res["ig"][i] == pytest.approx(best, abs=1e-9)
        assert table[(d, S)] == pytest.approx(best, abs=1e-9)
        assert res["second"][i] == pytest.approx(second, abs=1e-9)
    assert negative >= 2, "the case must hold variables whose every gain is negative"


def test_max_ig_excludes_the_variable_itself():
    """Eq. 1 takes S within V minus {i}.  In this 4-sample, 2-variable case
    (xi = 0.3) the only admissible partner scores below what pairing x0 with
    itself would score (every off-diagonal voxel empty: -2 h(beta)), so a scan
    that let i into S would report the wrong maximum and partner."""
    codes = np.array([[[1, 1, 1, 0], [0, 1, 0, 0]]], dtype=np.uint8)
    y = np.array([1, 0, 1, 1], dtype=np.uint8)
    c, xi = 2, 0.3
    want = _sh_from_probabilities([codes[0, 1]], y, c, xi) - _sh_from_probabilities([codes[0, 1], codes[0, 0]], y, c, xi)
    self_pair = (_sh_from_probabilities([codes[0, 0]], y, c, xi)
                 - _sh_from_probabilities([codes[0, 0], codes[0, 0]], y, c, xi))
    assert want < self_pair
    res = oracle.max_ig(codes, y, c, 2, xi)
    assert res["ig"][0] == pytest.approx(want, abs=1e-12)
    assert int(res["tuples"][0][0]) == 1


def test_max_ig_ties_go_to_lowest_disc_and_tuple():
    """Reading of Eq. 1's argmax: ties go to the lowest (discretisation,
    lexicographic S).  With range = 0 every discretisation is the same
    equipotent split, and variables 1, 2 and 3 are copies of one column, so
    each maximum is reached by several (d, S) with bit-identical counts."""
    rng = np.random.default_rng(7)
    N, c, D, xi = 60, 2, 3, 0.25
    base = rng.standard_normal((3, N)).astype(np.float32)
    x = np.stack([base[0], base[1], base[1], base[1], base[2]])
    y = ((x[0] > 0) ^ (x[1] > 0) ^ (rng.random(N) < 0.1)).astype(np.uint8)
    codes = oracle.discretize(x, c - 1, D, 0.0, seed=1)
    assert all(np.array_equal(codes[0], codes[d]) for d in range(D))
    for k in (1, 2, 3):
        res = oracle.max_ig(codes, y, c, k, xi)
        for i in range(5):
            best, second, table = _brute_max(codes, y, c, k, xi, i)
            first = next(key for key, g in table.items() if g >= best - 1e-9)  # lowest (d, S) of the tie
            assert res["ig"][i] == pytest.approx(best, abs=1e-9)
            assert (int(res["disc"][i]), tuple(int(t) for t in res["tuples"][i])) == first
            assert res["second"][i] == pytest.approx(second, abs=1e-9)
        assert res["disc"][0] == 0
        if k > 1:
            assert tuple(res["tuples"][0])[0] == 1  # partner 1 of the three copies


def test_xor_pair_invisible_in_1d_found_in_2d():
    """Synergy (section "Introduction"/"Theory"): x0, x1 set y by XOR, so each
    is uninformative alone but the top pair at k = 2, each the other's partner."""
    ds = synth.xor_small()
    codes = oracle.discretize(ds.x, 1, 1, 0.25, seed=1)
    r1 = oracle.max_ig(codes, ds.y, 2, 1, 0.25)
    r2 = oracle.max_ig(codes, ds.y, 2, 2, 0.25)
    top2 = set(np.argsort(-r2["ig"])[:2].tolist())
    assert top2 == {0, 1}
    assert r2["tuples"][0, 0] == 1 and r2["tuples"][1, 0] == 0
    # in 1D both are inside the bulk of the noise variables
    rank1 = np.argsort(np.argsort(-r1["ig"]))
    assert rank1[0] > 5 and rank1[1] > 5
    assert r2["ig"][0] > 10 * np.median(r2["ig"])


def test_three_way_parity_needs_k3():
    """Synergy of three variables (section "Introduction"): y is the parity of
    x0, x3, x5, so no single member and no pair carries information about y;
    IG stays at the noise level for k = 1 and 2 and jumps at k = 3, where
    each member's argmax partners are the other two."""
    rng = np.random.default_rng(33)
    N, M = 400, 7
    codes = rng.integers(0, 2, (1, M, N)).astype(np.uint8)
    members = [0, 3, 5]
    y = (np.bitwise_xor.reduce(codes[0, members], axis=0) ^ (rng.random(N) < 0.05)).astype(np.uint8)
    r1 = oracle.max_ig(codes, y, 2, 1, 0.25)
    r2 = oracle.max_ig(codes, y, 2, 2, 0.25)
    r3 = oracle.max_ig(codes, y, 2, 3, 0.25)
    assert r1["ig"].max() < 10.0 and r2["ig"].max() < 15.0
    for v in members:
        assert r3["ig"][v] > 150.0
        assert sorted(r3["tuples"][v].tolist()) == [m for m in members if m != v]
    assert max(r3["ig"][v] for v in range(M) if v not in members) < 20.0


def test_five_way_parity_needs_k5():
    """y is the parity of five variables: every proper subset of them is
    independent of y, so IG stays at the noise level up to k = 4 and jumps
    at k = 5, where each member's argmax partners are the other four."""
    rng = np.random.default_rng(55)
    N, M = 400, 7
    codes = rng.integers(0, 2, (1, M, N)).astype(np.uint8)
    members = [0, 2, 3, 5, 6]
    y = (np.bitwise_xor.reduce(codes[0, members], axis=0) ^ (rng.random(N) < 0.05)).astype(np.uint8)
    r4 = oracle.max_ig(codes, y, 2, 4, 0.25)
    r5 = oracle.max_ig(codes, y, 2, 5, 0.25)
    assert r4["ig"].max() < 20.0
    for v in members:
        assert r5["ig"][v] > 150.0
        assert sorted(r5["tuples"][v].tolist()) == [m for m in members if m != v]
    assert r5["ig"][1] < 20.0 and r5["ig"][4] < 20.0


# --------------------------------------------------------------------------
# chi^2 CDF and the IG_lim fit
# --------------------------------------------------------------------------
def test_chi2_cdf_closed_forms_and_scipy():
    from scipy.stats import chi2
    for x in [1e-6, 0.01, 0.3, 1.0, 3.84, 10.0, 40.0, 120.0]:
        assert oracle.chi2_cdf(x, 1) == pytest.approx(math.erf(math.sqrt(x / 2)), rel=1e-12, abs=1e-300)
        assert oracle.chi2_cdf(x, 2) == pytest.approx(-math.expm1(-x / 2), rel=1e-12)
        for df in [3, 4, 6, 9, 12, 18, 27, 48]:
            assert oracle.chi2_cdf(x, df) == pytest.approx(chi2.cdf(x, df), rel=1e-10, abs=1e-300)
            assert oracle.chi2_sf(x, df) == pytest.approx(chi2.sf(x, df), rel=1e-9, abs=1e-300)


@pytest.mark.parametrize("df,T", [(1, 200), (2, 50), (4, 1000)])
def test_ig_lim_recovers_number_of_tests(df, T):
    """IG_max of a null variable is the max of T chi^2/2 draws: the fit's T_hat
    recovers T, p-values are uniform, and IG_lim is the (1-alpha) quantile of
    the max (checked with scipy.stats.chi2.ppf)."""
    from scipy.stats import chi2
    rng = np.random.default_rng(df * 1000 + T)
    M = 4000
    ig = 0.5 * rng.chisquare(df, size=(M, T)).max(axis=1)
    c = 2
    k = {1: 1, 2: 2, 4: 3}[df]  # (c-1) c^(k-1) = df for c = 2
    p, lim, t_hat = oracle.ig_lim(ig, k, c - 1, None, alpha=0.05)
    assert abs(t_hat / T - 1) < 4 / math.sqrt(M)
    assert abs(np.mean(p) - 0.5) < 4 * math.sqrt(1 / 12 / M)
    want = 0.5 * chi2.ppf(0.95 ** (1 / t_hat), df)
    assert lim == pytest.approx(want, rel=1e-9)


def test_ig_lim_mask_restricts_fit():
    rng = np.random.default_rng(99)
    M, T = 2000, 100
    ig = 0.5 * rng.chisquare(1, size=(M, T)).max(axis=1)
    ig[:10] += 50.0  # relevant variables, excluded by the mask
    mask = np.ones(M, dtype=np.uint8)
    mask[:10] = 0
    p_all, _, t_all = oracle.ig_lim(ig, 1, 1, None)
    p_m, _, t_m = oracle.ig_lim(ig, 1, 1, mask)
    assert abs(t_m / T - 1) < 0.15
    # unmasked, the 10 relevant variables add likelihood terms with ln u ~ 0,
    # which inflates T_hat; masked out, they do not enter the fit
    assert t_all > t_m
    assert np.all(p_m[:10] < 1e-6)
