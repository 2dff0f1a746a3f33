"""FP64 CPU oracle for the MDFS information-gain scan -- TEST INFRASTRUCTURE ONLY.

This package wraps ``mdfs_oracle.c`` (plain C, FP64, brute force) with ctypes.
Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
import it; the CUDA library and its Python binding never do, and the two share
no code.  Every function restates the paper (arXiv 1811.00631):

* ``discretize``   -- randomised rank-based discretisation, section
  "Algorithm and implementation";
* ``sh`` / ``ig_one`` / ``max_ig`` -- Eq. (1), Eq. (3), Eqs. H, p and beta;
* ``chi2_cdf`` / ``ig_lim`` -- the chi^2 / extreme-value significance fit of
  section "Theory";
* ``interesting_tuples`` -- every (variable, tuple) reaching an IG threshold
  (section "Examples");
* ``shuffle_index`` / ``contrast`` / ``p_adjust`` / ``select`` -- contrast
  variables and the canonical selection pipeline of section "Canonical
  package usage" (contrasts, IG, fit on the contrasts, adjusted p-values,
  relevant set).

The readings taken where the paper is silent are listed in the C file header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mdfs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) into oracle/_build/liboracle.so."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    """Loads the oracle library.  MDFS_ORACLE_LIB names another build of the
    oracle source to load instead; the mutation test uses it to run the pins
    against copies of the oracle with planted mistakes."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("MDFS_ORACLE_LIB") or build()
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.oracle_philox4x32_10.argtypes = [P, P, P]
    lib.oracle_philox4x32_10.restype = None
    lib.oracle_cut_positions.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_uint64, P]
    lib.oracle_cut_positions.restype = None
    lib.oracle_discretize.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_uint64, P]
    lib.oracle_discretize.restype = ctypes.c_int
    lib.oracle_pseudocounts.argtypes = [P, ctypes.c_int, ctypes.c_double, P, P]
    lib.oracle_pseudocounts.restype = None
    lib.oracle_sh.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                              ctypes.c_double]
    lib.oracle_sh.restype = ctypes.c_double
    lib.oracle_ig_one.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_int, ctypes.c_int, P, ctypes.c_int]
    lib.oracle_ig_one.restype = ctypes.c_double
    lib.oracle_max_ig.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_double, P, ctypes.c_int, P, P, P, P]
    lib.oracle_max_ig.restype = ctypes.c_int
    lib.oracle_chi2_cdf.argtypes = [ctypes.c_double, ctypes.c_int]
    lib.oracle_chi2_cdf.restype = ctypes.c_double
    lib.oracle_chi2_sf.argtypes = [ctypes.c_double, ctypes.c_int]
    lib.oracle_chi2_sf.restype = ctypes.c_double
    lib.oracle_ig_lim.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_double,
                                  P, P, P]
    lib.oracle_ig_lim.restype = ctypes.c_int
    lib.oracle_shuffle_index.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64]
    lib.oracle_shuffle_index.restype = ctypes.c_uint32
    lib.oracle_contrast.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, P, P]
    lib.oracle_contrast.restype = ctypes.c_int
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = ctypes.c_int
    lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
    lib.oracle_set_num_threads.restype = None
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(counter, key) -> np.ndarray:
    """One Philox4x32-10 block (Salmon et al., SC'11): 4 counter words, 2 key words."""
    lib = _load()
    ctr = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_ptr(ctr), _ptr(k), _ptr(out))
    return out


def cut_positions(N: int, divisions: int, v: int, d: int, range_: float, seed: int) -> np.ndarray:
    """0-based sorted positions of the c-1 thresholds of variable v, discretisation d."""
    lib = _load()
    c = divisions + 1
    pos = np.zeros(max(c - 1, 1), dtype=np.int64)
    lib.oracle_cut_positions(N, c, v, d, float(range_), int(seed) & (2**64 - 1), _ptr(pos))
    return pos[: c - 1]


def discretize(x: np.ndarray, divisions: int, discretizations: int, range_: float, seed: int) -> np.ndarray:
    """Codes u8[D][M][N] of x given variable-major as an (M, N) array."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    M, N = x.shape
    codes = np.zeros((discretizations, M, N), dtype=np.uint8)
    rc = lib.oracle_discretize(_ptr(x), N, M, divisions, discretizations, float(range_),
                               int(seed) & (2**64 - 1), _ptr(codes))
    if rc != 0:
        raise ValueError(f"oracle_discretize failed ({rc})")
    return codes


def pseudocounts(y: np.ndarray, xi: float):
    """(beta0, beta1) of Eq. beta."""
    lib = _load()
    y = np.ascontiguousarray(y, dtype=np.uint8)
    b0 = ctypes.c_double()
    b1 = ctypes.c_double()
    lib.oracle_pseudocounts(_ptr(y), len(y), float(xi), ctypes.byref(b0), ctypes.byref(b1))
    return b0.value, b1.value


def sh(cols, y: np.ndarray, c: int, beta0: float, beta1: float) -> float:
    """Regularised N-scaled conditional entropy SH(S) of y given the code columns ``cols``."""
    lib = _load()
    y = np.ascontiguousarray(y, dtype=np.uint8)
    cols = [np.ascontiguousarray(col, dtype=np.uint8) for col in cols]
    arr = (ctypes.c_void_p * max(len(cols), 1))(*[col.ctypes.data for col in cols])
    return lib.oracle_sh(arr, len(cols), _ptr(y), len(y), c, float(beta0), float(beta1))


def ig_one(codes: np.ndarray, y: np.ndarray, c: int, xi: float, d: int, i: int, S) -> float:
    """IG(i | S) at discretisation d, FP64."""
    lib = _load()
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    y = np.ascontiguousarray(y, dtype=np.uint8)
    D, M, N = codes.shape
    s = np.ascontiguousarray(list(S) if len(S) else [0], dtype=np.int32)
    return lib.oracle_ig_one(_ptr(codes), _ptr(y), N, M, c, float(xi), d, i, _ptr(s), len(S))


def max_ig(codes: np.ndarray, y: np.ndarray, c: int, k: int, xi: float, variables=None):
    """IG^k_max (Eq. 1, maximised over discretisations too) for ``variables`` (all if None).

    Returns dict(ig=f64[n], tuples=i32[n, k-1], disc=i32[n], second=f64[n]).
    """
    lib = _load()
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    y = np.ascontiguousarray(y, dtype=np.uint8)
    D, M, N = codes.shape
    if variables is None:
        n = M
        vptr = None
    else:
        vars_arr = np.ascontiguousarray(variables, dtype=np.int32)
        n = len(vars_arr)
        vptr = _ptr(vars_arr)
    ig = np.zeros(n, dtype=np.float64)
    tuples = np.full((n, max(k - 1, 1)), -1, dtype=np.int32)
    disc = np.zeros(n, dtype=np.int32)
    second = np.zeros(n, dtype=np.float64)
    rc = lib.oracle_max_ig(_ptr(codes), _ptr(y), N, M, D, c, k, float(xi), vptr, n, _ptr(ig),
                           _ptr(tuples), _ptr(disc), _ptr(second))
    if rc != 0:
        raise ValueError(f"oracle_max_ig failed ({rc})")
    return dict(ig=ig, tuples=tuples[:, : k - 1], disc=disc, second=second)


def chi2_cdf(x: float, df: int) -> float:
    return _load().oracle_chi2_cdf(float(x), int(df))


def chi2_sf(x: float, df: int) -> float:
    return _load().oracle_chi2_sf(float(x), int(df))


def ig_lim(ig: np.ndarray, k: int, divisions: int, irrelevant_mask=None, alpha: float = 0.05):
    """chi^2 / extreme-value fit: returns (p_values f64[M], IG_lim, T_hat)."""
    lib = _load()
    ig = np.ascontiguousarray(ig, dtype=np.float64)
    M = len(ig)
    mask_ptr = None
    if irrelevant_mask is not None:
        mask = np.ascontiguousarray(irrelevant_mask, dtype=np.uint8)
        mask_ptr = _ptr(mask)
    p = np.zeros(M, dtype=np.float64)
    lim = ctypes.c_double()
    neff = ctypes.c_double()
    rc = lib.oracle_ig_lim(_ptr(ig), M, k, divisions, mask_ptr, float(alpha), _ptr(p),
                           ctypes.byref(lim), ctypes.byref(neff))
    if rc != 0:
        raise ValueError(f"oracle_ig_lim failed ({rc})")
    return p, lim.value, neff.value


def interesting_tuples(codes: np.ndarray, y: np.ndarray, c: int, k: int, xi: float, threshold: float):
    """ComputeInterestingTuples (section "Examples"): every (variable v, partner
    set S, |S| = k-1, v not in S) whose IG(v | S), maximised over the
    discretisations, reaches ``threshold``; brute force in FP64 through
    ``ig_one``.  Returns a list of (v, S tuple ascending, ig, d) sorted by
    (v, S); d is the lowest discretisation reaching the maximum."""
    import itertools
    D, M, N = codes.shape
    out = []
    for v in range(M):
        others = [m for m in range(M) if m != v]
        for S in itertools.combinations(others, k - 1):
            best, bd = -np.inf, -1
            for d in range(D):
                g = ig_one(codes, y, c, xi, d, v, list(S))
                if g > best:
                    best, bd = g, d
            if best >= threshold:
                out.append((v, tuple(S), best, bd))
    return out


def shuffle_index(i: int, n: int, stream: int, seed: int) -> int:
    """Image of i under the counter-based pseudo-random permutation of [0, n)
    (10-round Feistel network with Philox round functions, cycle walking)."""
    return int(_load().oracle_shuffle_index(int(i), int(n), int(stream) & 0xFFFFFFFF, int(seed) & (2**64 - 1)))


def contrast(x: np.ndarray, n_contrast: int, seed: int):
    """Contrast variables (section "Canonical package usage"): returns
    (x_ext f32[M + n_contrast][N], src i32[n_contrast]); row M + j is
    variable src[j] with its samples shuffled."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    M, N = x.shape
    out = np.zeros((M + n_contrast, N), dtype=np.float32)
    src = np.zeros(max(n_contrast, 1), dtype=np.int32)
    rc = lib.oracle_contrast(_ptr(x), N, M, int(n_contrast), int(seed) & (2**64 - 1), _ptr(out), _ptr(src))
    if rc != 0:
        raise ValueError(f"oracle_contrast failed ({rc})")
    return out, src[:n_contrast]


P_ADJUST_METHODS = ("none", "bonferroni", "holm", "hochberg", "BH", "BY")


def p_adjust(p: np.ndarray, method: str = "holm") -> np.ndarray:
    """Multiple-testing adjustment of p-values, written from the definitions
    (p_(1) <= ... <= p_(m) the sorted values, results capped at 1):
    Bonferroni m p; Holm's step-down max_{k<=i} (m-k+1) p_(k); Hochberg's
    step-up min_{k>=i} (m-k+1) p_(k); Benjamini-Hochberg min_{k>=i} m/k p_(k);
    Benjamini-Yekutieli the same times sum_{k=1..m} 1/k."""
    p = np.asarray(p, dtype=np.float64)
    m = len(p)
    if m == 0 or method == "none":
        return p.copy()
    order = np.argsort(p, kind="stable")
    ps = p[order]
    adj = np.empty(m)
    if method == "bonferroni":
        adj = np.minimum(1.0, m * ps)
    elif method == "holm":
        run = 0.0
        for i in range(m):
            run = max(run, (m - i) * ps[i])
            adj[i] = min(1.0, run)
    elif method in ("hochberg", "BH", "BY"):
        q = sum(1.0 / k for k in range(1, m + 1)) if method == "BY" else 1.0
        run = np.inf
        for i in range(m - 1, -1, -1):
            f = (m - i) if method == "hochberg" else q * m / (i + 1)
            run = min(run, f * ps[i])
            adj[i] = min(1.0, run)
    else:
        raise ValueError(f"unknown method {method!r}")
    out = np.empty(m)
    out[order] = adj
    return out


def select(x: np.ndarray, y: np.ndarray, n_contrast: int, k: int, divisions: int, discretizations: int,
           range_: float, pc_xi: float, seed: int, method: str = "holm", level: float = 0.05, variables=None):
    """The canonical pipeline of section "Canonical package usage": contrast
    variables, IG^k_max over the extended set, the chi^2 / extreme-value fit on
    the contrast variables only, p-values of the original variables, their
    adjustment and the relevant set (adjusted p < level).  Returns a dict with
    ig / tuples / disc / p / adjusted / relevant for the M original variables
    and ig_lim, n_eff, src.  ``variables`` (optional) restricts the IG scan to
    those original rows plus all contrasts (the fit needs every contrast)."""
    M = x.shape[0]
    x_ext, src = contrast(x, n_contrast, seed)
    c = divisions + 1
    codes = discretize(x_ext, divisions, discretizations, range_, seed)
    Mx = M + n_contrast
    rows = np.arange(Mx, dtype=np.int32) if variables is None else \
        np.concatenate([np.asarray(variables, dtype=np.int32), np.arange(M, Mx, dtype=np.int32)])
    r = max_ig(codes, y, c, k, pc_xi, variables=rows)
    ig = np.full(Mx, np.nan)
    ig[rows] = r["ig"]
    mask = np.zeros(Mx, dtype=np.uint8)
    mask[M:] = 1
    p_ext, lim, neff = ig_lim(ig[M:], k, divisions)  # fitted on the contrasts only
    # p-values of the original variables under the fitted T
    df = (c - 1) * c ** (k - 1)
    p = np.array([1.0 - chi2_cdf(2.0 * g, df) ** neff if g > 0 else 1.0 for g in ig[:M]])
    adj = p_adjust(p, method)
    out = {"ig": ig[:M], "tuples": None, "disc": None, "p": p, "adjusted": adj, "relevant": adj < level,
           "ig_lim": lim, "n_eff": neff, "src": src, "rows": rows, "max_ig": r}
    return out


def num_threads() -> int:
    return _load().oracle_num_threads()


def set_num_threads(n: int) -> None:
    _load().oracle_set_num_threads(int(n))
