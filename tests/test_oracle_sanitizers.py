"""The C oracle under AddressSanitizer and UndefinedBehaviorSanitizer.

A small harness program (written here, test infrastructure) calls every oracle entry
point on tiny seeded inputs: all class counts, k = 1..5, ragged N, the
chi^2 fit with and without a mask, the contrast shuffle.  It is compiled with
-fsanitize=address,undefined and no recovery, so any out-of-bounds access,
leak or undefined operation in the oracle fails the test.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r"""
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

int oracle_discretize(const float*, int, int, int, int, double, uint64_t, uint8_t*);
int oracle_max_ig(const uint8_t*, const uint8_t*, int, int, int, int, int, double, const int32_t*, int, double*,
                  int32_t*, int32_t*, double*);
int oracle_ig_lim(const double*, int, int, int, const uint8_t*, double, double*, double*, double*);
int oracle_contrast(const float*, int, int, int, uint64_t, float*, int32_t*);

static uint64_t st = 88172645463325252ull;
static double unif(void) { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return (st >> 11) * (1.0 / 9007199254740992.0); }

int main(void) {
    const int Ns[3] = {7, 33, 65};
    for (int in = 0; in < 3; ++in) {
        const int N = Ns[in], M = 6, D = 2;
        float* x = malloc(sizeof(float) * N * M);
        uint8_t* y = malloc(N);
        for (int i = 0; i < N * M; ++i) x[i] = (float)(unif() * 4.0 - 2.0);
        for (int s = 0; s < N; ++s) y[s] = (uint8_t)(s % 3 == 0);
        for (int div = 1; div <= 3; ++div) {
            const int c = div + 1;
            if (N < c) continue;
            uint8_t* codes = malloc((size_t)D * M * N);
            if (oracle_discretize(x, N, M, div, D, 0.5, 12345u + div, codes)) return 10;
            for (int k = 1; k <= 5; ++k) {
                if (k >= 4 && c > 2) continue;
                double ig[6], second[6];
                int32_t tuples[6 * 4], disc[6];
                if (oracle_max_ig(codes, y, N, M, D, c, k, 0.25, NULL, 0, ig, tuples, disc, second)) return 11;
                const int32_t vars[2] = {0, 5};
                if (oracle_max_ig(codes, y, N, M, D, c, k, 0.25, vars, 2, ig, tuples, disc, second)) return 12;
                double p[6], lim, neff;
                const uint8_t mask[6] = {0, 1, 1, 1, 1, 1};
                const int rc = oracle_ig_lim(ig, 2, k, div, NULL, 0.05, p, &lim, &neff);
                if (rc != 0 && rc != -2) return 13;  /* -2: no positive IG to fit (tiny N) */
                for (int v = 0; v < 6; ++v) ig[v] = unif() * 10.0;
                if (oracle_ig_lim(ig, 6, k, div, mask, 0.05, p, &lim, &neff)) return 14;
            }
            free(codes);
        }
        float* xe = malloc(sizeof(float) * N * (M + 4));
        int32_t src[4];
        if (oracle_contrast(x, N, M, 4, 99u, xe, src)) return 15;
        free(xe);
        free(x);
        free(y);
    }
    printf("sanitized oracle ok\n");
    return 0;
}
"""


def test_oracle_under_address_and_undefined_behaviour_sanitizers(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    drv = tmp_path / "harness.c"
    drv.write_text(HARNESS)
    exe = tmp_path / "harness"
    cmd = [gcc, "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           os.path.join(ROOT, "oracle", "mdfs_oracle.c"), str(drv), "-lm", "-o", str(exe)]
    built = subprocess.run(cmd, capture_output=True, text=True)
    if built.returncode != 0 and "sanitize" in (built.stderr or ""):
        pytest.skip("sanitizer runtime not available: " + built.stderr.strip().splitlines()[-1])
    assert built.returncode == 0, built.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300,
                         env=dict(os.environ, ASAN_OPTIONS="detect_leaks=1"))
    assert run.returncode == 0, run.stdout + run.stderr
    assert "sanitized oracle ok" in run.stdout
