"""Planted mistakes in the oracle must fail its pins.

Each case copies ``oracle/mdfs_oracle.c``, changes one spot (a dropped term,
a wrong sign, an off-by-one, a swapped operand, a wrong constant), builds the
copy with the oracle's own compiler flags, and runs the CPU pins of
``tests/test_oracle_pins.py`` and ``tests/test_oracle_contrast_pins.py`` against it in a child process
(``MDFS_ORACLE_LIB`` points the wrapper at the copy).  Every mutant must make
at least one pin fail; the unchanged source must pass them all.  The mistakes
are planted in the oracle only, on the CPU.

Not listed: which Philox word feeds which share.  That layout is a choice of
this implementation (the paper names no generator), so no paper fact can pin
it; the bit-exact GPU parity of the discretised codes does.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mdfs_oracle.c")

# (what the mistake is, original text, planted text); each original occurs once
MUTANTS = [
    ("SH without the both-classes term f(n + b0 + b1)",
     "sh += f_xlogx(a + b) - f_xlogx(a) - f_xlogx(b);", "sh += -f_xlogx(a) - f_xlogx(b);"),
    ("SH with the class pseudocounts swapped",
     "double a = (double)n0[v] + beta0, b = (double)n1[v] + beta1;",
     "double a = (double)n0[v] + beta1, b = (double)n1[v] + beta0;"),
    ("pseudocounts over the larger class (Eq. beta uses the smaller)",
     "double mn = (double)(n0 < n1 ? n0 : n1);", "double mn = (double)(n0 > n1 ? n0 : n1);"),
    ("entropy in bits instead of nats",
     "return x > 0.0 ? x * log(x) : 0.0;", "return x > 0.0 ? x * log2(x) : 0.0;"),
    ("k = 2 information gain with the sign flipped",
     "double g = oracle_sh(cs, 1, y, N, c, b0, b1) - oracle_sh(csi, 2, y, N, c, b0, b1);",
     "double g = oracle_sh(csi, 2, y, N, c, b0, b1) - oracle_sh(cs, 1, y, N, c, b0, b1);"),
    ("k = 2 partner allowed to be the variable itself",
     "if (m == i) continue;", "if (m == i && 0) continue;"),
    ("k = 2 argmax keeps the last of equal maxima",
     "if (g > best) { runner = best; best = g; bd = d; bs[0] = m; }",
     "if (g >= best) { runner = best; best = g; bd = d; bs[0] = m; }"),
    ("k = 3 second partner index starts at the first",
     "for (int m2 = m1 + 1; m2 < M; ++m2) {\n                        if (m2 == i) continue;\n"
     "                        const uint8_t* c2 = codes + ((size_t)d * M + m2) * N;\n"
     "                        const uint8_t* cs[2]",
     "for (int m2 = m1; m2 < M; ++m2) {\n                        if (m2 == i) continue;\n"
     "                        const uint8_t* c2 = codes + ((size_t)d * M + m2) * N;\n"
     "                        const uint8_t* cs[2]"),
    ("a tie at a threshold goes to the lower class",
     "if (xs >= sorted[pos[j]]) code++;", "if (xs > sorted[pos[j]]) code++;"),
    ("cut position one above the floor",
     "p = (int64_t)(((uint64_t)N * (uint64_t)cum) / (uint64_t)total);",
     "p = (int64_t)(((uint64_t)N * (uint64_t)cum) / (uint64_t)total) + 1;"),
    ("Philox second key word bumped by the first Weyl constant",
     "k1 += 0xBB67AE85u;", "k1 += 0x9E3779B9u;"),
    ("chi^2 degrees of freedom c c^(k-1) instead of (c-1) c^(k-1)",
     "int df = c - 1;\n    for (int j = 1; j < k; ++j) df *= c;",
     "int df = c;\n    for (int j = 1; j < k; ++j) df *= c;"),
    ("fitted number of tests with the wrong sign",
     "double T = -(double)n / sum_log;", "double T = -(double)n / (2.0 * sum_log);"),
    ("odd-df chi^2 tail series with a shifted Gamma argument",
     "term *= z / ((double)j + 1.5);", "term *= z / ((double)j + 0.5);"),
    ("chi^2 lower-tail series with a shifted Gamma argument",
     "term *= z / (a + (double)n);", "term *= z / (a + (double)n + 1.0);"),
    ("p-values as F^T instead of 1 - F^T",
     "p_values[i] = (u <= 0.0) ? 1.0 : -expm1(T * log(u));", "p_values[i] = (u <= 0.0) ? 1.0 : exp(T * log(u));"),
    ("IG_lim from (1 - alpha)^T instead of (1 - alpha)^(1/T)",
     "double target = pow(1.0 - alpha, 1.0 / T);", "double target = pow(1.0 - alpha, T);"),
    ("IG_lim without halving the chi^2 quantile",
     "*ig_lim = 0.25 * (lo + hi);", "*ig_lim = 0.5 * (lo + hi);"),
    ("voxel index built from the first column only",
     "for (int j = n_cols - 1; j >= 0; --j) vox = vox * c + cols[j][s];",
     "for (int j = n_cols - 1; j >= 0; --j) vox = vox * c + cols[0][s];"),
    ("k = 1 information gain with the sign flipped",
     "double g = oracle_sh(NULL, 0, y, N, c, b0, b1) - oracle_sh(cols, 1, y, N, c, b0, b1);",
     "double g = oracle_sh(cols, 1, y, N, c, b0, b1) - oracle_sh(NULL, 0, y, N, c, b0, b1);"),
    ("k = 4 joint set with a partner twice instead of the variable",
     "const uint8_t* csi[4] = {c1, c2, c3, ci};", "const uint8_t* csi[4] = {c1, c2, c3, c3};"),
    ("k = 5 joint set with a partner repeated",
     "const uint8_t* csi[5] = {c1, c2, c3, c4, ci};", "const uint8_t* csi[5] = {c1, c2, c3, c3, ci};"),
    ("cut positions not forced strictly increasing",
     "if (j > 1 && p <= prev) p = prev + 1;", "if (j > 1 && p < prev) p = prev;"),
    ("contrast shuffle with 4 Feistel rounds",
     "for (uint32_t r = 0; r < 10; ++r) {", "for (uint32_t r = 0; r < 4; ++r) {"),
    ("contrast Feistel round that drops the left half",
     "uint32_t nl = R, nr = (L ^ out[0]) & mask;", "uint32_t nl = R, nr = out[0] & mask;"),
    ("cut positions without the lower clamp",
     "if (p < j) p = j;", "if (0) p = j;"),
    ("cut positions without the upper clamp",
     "if (p > N - c + j) p = N - c + j;", "if (0) p = N - c + j;"),
    ("threshold read one position low",
     "if (xs >= sorted[pos[j]]) code++;", "if (xs >= sorted[pos[j] - 1]) code++;"),
    ("shares that do not depend on the discretisation",
     "uint32_t ctr[4] = {(uint32_t)(j / 4), (uint32_t)v, (uint32_t)d, 0x4D444653u};",
     "uint32_t ctr[4] = {(uint32_t)(j / 4), (uint32_t)v, 0u, 0x4D444653u};"),
    ("shares that do not depend on the variable",
     "uint32_t ctr[4] = {(uint32_t)(j / 4), (uint32_t)v, (uint32_t)d, 0x4D444653u};",
     "uint32_t ctr[4] = {(uint32_t)(j / 4), 0u, (uint32_t)d, 0x4D444653u};"),
    ("class-1 pseudocount from the class-0 size",
     "*beta1 = xi * (double)n1 / mn;", "*beta1 = xi * (double)n0 / mn;"),
    ("k = 3 joint set with the first partner twice",
     "const uint8_t* csi[3] = {c1, c2, ci};", "const uint8_t* csi[3] = {c1, c1, ci};"),
    ("k = 2 runner-up not tracked",
     "if (g > best) { runner = best; best = g; bd = d; bs[0] = m; }\n                    else if (g > runner) runner = g;",
     "if (g > best) { runner = best; best = g; bd = d; bs[0] = m; }\n                    else if (0) runner = g;"),
    ("k = 1 argmax keeps the last of equal maxima",
     "if (g > best) { runner = best; best = g; bd = d; }", "if (g >= best) { runner = best; best = g; bd = d; }"),
    ("k = 3 runner-up not tracked",
     "bs[0] = m1; bs[1] = m2; }\n                        else if (g > runner) runner = g;",
     "bs[0] = m1; bs[1] = m2; }\n                        else if (0) runner = g;"),
    ("k = 4 runner-up not tracked",
     "bs[2] = m3; }\n                            else if (g > runner) runner = g;",
     "bs[2] = m3; }\n                            else if (0) runner = g;"),
    ("k = 5 runner-up not tracked",
     "} else if (g > runner) runner = g;\n                            }", "} else if (0) runner = g;\n                            }"),
    ("k = 4 third partner may repeat the second",
     "for (int m3 = m2 + 1; m3 < M; ++m3) {\n                            if (m3 == i) continue;\n"
     "                            const uint8_t* c3 = codes + ((size_t)d * M + m3) * N;\n"
     "                            const uint8_t* cs[3]",
     "for (int m3 = m2; m3 < M; ++m3) {\n                            if (m3 == i) continue;\n"
     "                            const uint8_t* c3 = codes + ((size_t)d * M + m3) * N;\n"
     "                            const uint8_t* cs[3]"),
    ("k = 5 fourth partner may repeat the third",
     "for (int m4 = m3 + 1; m4 < M; ++m4)", "for (int m4 = m3; m4 < M; ++m4)"),
    ("class sizes counted with the labels swapped",
     "for (int s = 0; s < N; ++s) n1 += y[s] ? 1 : 0;", "for (int s = 0; s < N; ++s) n1 += y[s] ? 0 : 1;"),
    ("voxel counts with the labels swapped",
     "if (y[s]) n1[vox]++; else n0[vox]++;", "if (y[s]) n0[vox]++; else n1[vox]++;"),
    ("single-set gain with the sign flipped", "return sh_s - sh_si;", "return sh_si - sh_s;"),
    ("even-df chi^2 tail series one term long",
     "for (int j = 0; j < df / 2; ++j) {", "for (int j = 0; j <= df / 2; ++j) {"),
    ("fit takes variables with F = 0 into the likelihood",
     "if (u <= 0.0) continue;", "if (u < 0.0) continue;"),
    ("IG_lim bisection moving the wrong end",
     "if (oracle_chi2_cdf(mid, df) < target) lo = mid; else hi = mid;",
     "if (oracle_chi2_cdf(mid, df) < target) hi = mid; else lo = mid;"),
    ("contrast samples left unshuffled",
     "row[i] = x[(size_t)s * N + oracle_shuffle_index((uint32_t)i, (uint32_t)N, (uint32_t)j, seed)];",
     "row[i] = x[(size_t)s * N + i];"),
    ("contrast sources with replacement",
     "oracle_shuffle_index((uint32_t)(j % M), (uint32_t)M, 0xFFFFFFFFu, seed);",
     "oracle_shuffle_index((uint32_t)(j % M), (uint32_t)M, (uint32_t)j, seed);"),
]


def _build(src_text: str, path: str):
    c_path = path[:-3] + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", c_path, "-o", path, "-lm"],
                   check=True, capture_output=True)


def _pins_pass(lib_path: str = None, first_path: str = ROOT) -> bool:
    """Runs the CPU pins in a child process against the oracle library at
    lib_path, or against the oracle package found first on the path."""
    env = dict(os.environ, OMP_NUM_THREADS="2",
               PYTHONPATH=first_path + os.pathsep + ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    env.pop("MDFS_ORACLE_LIB", None)
    if lib_path:
        env["MDFS_ORACLE_LIB"] = lib_path
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_contrast_pins.py"),
                        "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"],
                       cwd=first_path, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode == 0


def test_every_planted_mistake_fails_a_pin(tmp_path):
    with open(SRC) as f:
        src = f.read()
    jobs = [("unchanged", src)]
    for what, old, new in MUTANTS:
        assert src.count(old) == 1, f"mutation site not unique: {what}"
        jobs.append((what, src.replace(old, new)))

    def run(i_job):
        i, (what, text) = i_job
        lib = str(tmp_path / f"mutant{i}.so")
        _build(text, lib)
        return what, _pins_pass(lib)

    with concurrent.futures.ThreadPoolExecutor(max_workers=4) as ex:
        results = list(ex.map(run, enumerate(jobs)))
    assert results[0] == ("unchanged", True), "the unchanged oracle must pass its pins"
    survivors = [what for what, passed in results[1:] if passed]
    assert not survivors, f"planted mistakes that no pin catches: {survivors}"


# mistakes in the Python side of the oracle (p-value adjustment, interesting
# tuples, the selection pipeline)
PY_MUTANTS = [
    ("Holm multiplier one too small", "run = max(run, (m - i) * ps[i])", "run = max(run, (m - i - 1) * ps[i])"),
    ("Holm without the running maximum", "run = max(run, (m - i) * ps[i])", "run = (m - i) * ps[i]"),
    ("step-up adjustments taken from the smallest p-value",
     "for i in range(m - 1, -1, -1):", "for i in range(m):"),
    ("Benjamini-Hochberg rank off by one", "q * m / (i + 1)", "q * m / (i + 2)"),
    ("Benjamini-Yekutieli harmonic sum one term short",
     "sum(1.0 / k for k in range(1, m + 1))", "sum(1.0 / k for k in range(1, m))"),
    ("Bonferroni not capped at 1", "adj = np.minimum(1.0, m * ps)", "adj = m * ps"),
    ("adjusted values left in sorted order", "out[order] = adj", "out[:] = adj"),
    ("interesting only strictly above the threshold", "if best >= threshold:", "if best > threshold:"),
    ("interesting tuple keeps the last discretisation of a tie", "                if g > best:\n                    best, bd = g, d",
     "                if g >= best:\n                    best, bd = g, d"),
    ("selection p-values as F^T", "p = np.array([1.0 - chi2_cdf(2.0 * g, df) ** neff if g > 0 else 1.0 for g in ig[:M]])",
     "p = np.array([chi2_cdf(2.0 * g, df) ** neff if g > 0 else 1.0 for g in ig[:M]])"),
]


def test_every_planted_mistake_in_the_python_oracle_fails_a_pin(tmp_path):
    src_dir = os.path.join(ROOT, "oracle")
    with open(os.path.join(src_dir, "__init__.py")) as f:
        init = f.read()
    jobs = [("unchanged", init)]
    for what, old, new in PY_MUTANTS:
        assert init.count(old) == 1, f"mutation site not unique: {what}"
        jobs.append((what, init.replace(old, new)))

    def run(i_job):
        i, (what, text) = i_job
        root = tmp_path / f"m{i}"
        pkg = root / "oracle"
        pkg.mkdir(parents=True)
        shutil.copy(os.path.join(src_dir, "mdfs_oracle.c"), pkg / "mdfs_oracle.c")
        (pkg / "__init__.py").write_text(text)
        return what, _pins_pass(first_path=str(root))

    with concurrent.futures.ThreadPoolExecutor(max_workers=4) as ex:
        results = list(ex.map(run, enumerate(jobs)))
    assert results[0] == ("unchanged", True), "the unchanged oracle must pass its pins"
    survivors = [what for what, passed in results[1:] if passed]
    assert not survivors, f"planted mistakes that no pin catches: {survivors}"
