/*
 * MDFS FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, brute-force restatement of the MDFS information-gain scan
 * (Piliszek et al., "MDFS - MultiDimensional Feature Selection", arXiv
 * 1811.00631).  Only the tests, the smoke check and the benchmark's CPU
 * baseline leg may load this library; the product path never does.  It shares
 * no source with the CUDA library: every function here is written from the
 * paper's equations.
 *
 * Paper passages restated (sections/equations of arXiv 1811.00631):
 *   - Eq. (1), section "Theory": IG^k_max(y;x_i) = N max over (k-1)-subsets
 *     of [H(y|S) - H(y|S,x_i)].
 *   - Eq. (3), section "Theory": the k = 1 form N (H(y) - H(y|x_i)).
 *   - section "Algorithm and implementation": randomised rank-based
 *     discretisation (shares ~ U(1-range, 1+range), c-1 cut positions, values
 *     of the sorted variable at those positions are the thresholds), the max
 *     over discretisations, the entropy over voxels (Eq. H), the
 *     pseudocount-regularised class probability (Eq. p) and the pseudocount
 *     beta^d = xi N^d / min(N^0, N^1) (Eq. beta).
 *   - section "Theory", significance paragraph: chi^2 law of a single tuple's
 *     IG, extreme-value law of the max with one fitted parameter (number of
 *     independent tests).
 *
 * Readings adopted where the paper is silent or garbled:
 *   - Eq. H carries no voxel weights in print; the N-scaled regularised
 *     conditional entropy used here is
 *        SH(S) = sum_v [ f(n_v+b0+b1) - f(n0_v+b0) - f(n1_v+b1) ],
 *     f(x) = x ln x, which equals -sum_v sum_d (n^d_v+b^d) ln p^d_v with
 *     p^d_v from Eq. p (numerator pseudocount read as b^d).
 *   - natural logarithm (nats): 2 IG of a single null tuple is chi^2 with
 *     (c-1) c^(k-1) degrees of freedom (binary decision).
 *   - cut positions: 0-based, strictly increasing, within [1, N-1]; shares
 *     drawn with Philox4x32-10 in 20-bit fixed point (see discretize below).
 *   - a tie at a threshold goes to the upper class (x >= t).
 *   - argmax ties go to the lowest (discretisation, lexicographic tuple).
 *   - the chi^2 extreme-value fit: CDF F_df(2x)^T, T fitted by maximum
 *     likelihood on the irrelevant variables (closed form).
 *   - contrast variables (section "Canonical package usage"): copies of
 *     original variables with their samples shuffled.  The shuffle is our
 *     choice of a counter-based pseudo-random permutation (a 10-round Feistel
 *     network with Philox round functions, restricted to [0, n) by cycle
 *     walking); the sources are the same permutation of [0, M) at j mod M.
 *   - p-value adjustment: the step-down / step-up definitions of Holm,
 *     Hochberg, Bonferroni, Benjamini-Hochberg and Benjamini-Yekutieli.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition: Salmon, Moraes, Dror and   */
/* Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11.  Ten rounds  */
/* of the 4x32 S-box with round multipliers 0xD2511F53 / 0xCD9E8D57 and     */
/* Weyl key increments 0x9E3779B9 / 0xBB67AE85.                             */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ x1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ x3 ^ k1;
        uint32_t n3 = lo0;
        x0 = n0; x1 = n1; x2 = n2; x3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------ */
/* Discretisation (section "Algorithm and implementation").                 */
/*                                                                          */
/* For variable v and discretisation d, with c = divisions + 1 classes:     */
/*   Philox block b = 0, 1, ... with counter (b, v, d, 0x4D444653) and key  */
/*   (seed low word, seed high word) gives words u_j (j = 4b .. 4b+3).      */
/*   Share j (0 <= j < c): w_j = W - R + floor(u_j * 2R / 2^32), where      */
/*   W = 2^20 is "1" in fixed point and R = round(range * 2^20), i.e. a     */
/*   uniform draw on [W(1-range), W(1+range)).                              */
/*   Cumulative S_j = w_0 + ... + w_{j-1};  p_j = floor(N S_j / S_c) for    */
/*   j = 1..c-1 (all S_c = 0: p_j = floor(N j / c)).                        */
/*   Positions are clamped to [j, N-c+j] and forced strictly increasing.    */
/*   Threshold t_j = (sorted x_v)[p_j];  code(x) = #{ j : x >= t_j }.       */
/* ------------------------------------------------------------------------ */
static int cmp_float(const void* a, const void* b)
{
    float fa = *(const float*)a, fb = *(const float*)b;
    return (fa > fb) - (fa < fb);
}

void oracle_cut_positions(int N, int c, int v, int d, double range, uint64_t seed, int64_t* pos /*[c-1]*/)
{
    const int64_t W = (int64_t)1 << 20;
    const int64_t R = (int64_t)floor(range * (double)W + 0.5);
    int64_t share[64];
    for (int j = 0; j < c; ++j) {
        uint32_t ctr[4] = {(uint32_t)(j / 4), (uint32_t)v, (uint32_t)d, 0x4D444653u};
        uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
        uint32_t u[4];
        oracle_philox4x32_10(ctr, key, u);
        uint64_t draw = ((uint64_t)u[j % 4] * (uint64_t)(2 * R)) >> 32;
        share[j] = W - R + (int64_t)draw;
    }
    int64_t total = 0;
    for (int j = 0; j < c; ++j) total += share[j];
    int64_t cum = 0, prev = 0;
    for (int j = 1; j < c; ++j) {
        cum += share[j - 1];
        int64_t p;
        if (total > 0)
            p = (int64_t)(((uint64_t)N * (uint64_t)cum) / (uint64_t)total);
        else
            p = ((int64_t)N * j) / c;
        if (p < j) p = j;
        if (p > N - c + j) p = N - c + j;
        if (j > 1 && p <= prev) p = prev + 1;
        pos[j - 1] = p;
        prev = p;
    }
}

/* x: variable-major float32, x[v*N + s].  codes: [D][M][N].  Returns 0. */
int oracle_discretize(const float* x, int N, int M, int divisions, int D, double range, uint64_t seed,
                      uint8_t* codes)
{
    const int c = divisions + 1;
    if (c < 2 || c > 64 || N < c) return -1;
#pragma omp parallel for schedule(dynamic)
    for (int v = 0; v < M; ++v) {
        float* sorted = (float*)malloc(sizeof(float) * (size_t)N);
        memcpy(sorted, x + (size_t)v * N, sizeof(float) * (size_t)N);
        qsort(sorted, (size_t)N, sizeof(float), cmp_float);
        int64_t pos[63];
        for (int d = 0; d < D; ++d) {
            oracle_cut_positions(N, c, v, d, range, seed, pos);
            uint8_t* out = codes + ((size_t)d * M + v) * N;
            for (int s = 0; s < N; ++s) {
                float xs = x[(size_t)v * N + s];
                int code = 0;
                for (int j = 0; j < c - 1; ++j)
                    if (xs >= sorted[pos[j]]) code++;
                out[s] = (uint8_t)code;
            }
        }
        free(sorted);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Regularised entropy (Eqs. H, p, beta).                                    */
/* ------------------------------------------------------------------------ */
static double f_xlogx(double x) { return x > 0.0 ? x * log(x) : 0.0; }

/* beta^d = xi N^d / min(N^0, N^1)  (Eq. beta) */
void oracle_pseudocounts(const uint8_t* y, int N, double xi, double* beta0, double* beta1)
{
    long n1 = 0;
    for (int s = 0; s < N; ++s) n1 += y[s] ? 1 : 0;
    long n0 = N - n1;
    double mn = (double)(n0 < n1 ? n0 : n1);
    *beta0 = xi * (double)n0 / mn;
    *beta1 = xi * (double)n1 / mn;
}

/*
 * SH(S) for the variable set S given as n_cols code columns (each [N], values
 * in 0..c-1).  Counts every voxel (c^|S| of them, including empty ones) by
 * visiting every sample, then sums the regularised voxel entropies.
 */
double oracle_sh(const uint8_t* const* cols, int n_cols, const uint8_t* y, int N, int c, double beta0,
                 double beta1)
{
    int nvox = 1;
    for (int j = 0; j < n_cols; ++j) nvox *= c;
    long* n0 = (long*)calloc((size_t)nvox, sizeof(long));
    long* n1 = (long*)calloc((size_t)nvox, sizeof(long));
    for (int s = 0; s < N; ++s) {
        int vox = 0;
        for (int j = n_cols - 1; j >= 0; --j) vox = vox * c + cols[j][s];
        if (y[s]) n1[vox]++; else n0[vox]++;
    }
    double sh = 0.0;
    for (int v = 0; v < nvox; ++v) {
        double a = (double)n0[v] + beta0, b = (double)n1[v] + beta1;
        sh += f_xlogx(a + b) - f_xlogx(a) - f_xlogx(b);
    }
    free(n0);
    free(n1);
    return sh;
}

/* IG(i | S) = SH(S) - SH(S + {i}) for one variable, one partner set, one
 * discretisation (Eq. 1 before the max).  S has k-1 members (k-1 may be 0). */
double oracle_ig_one(const uint8_t* codes, const uint8_t* y, int N, int M, int c, double xi, int d, int i,
                     const int32_t* S, int n_s)
{
    double b0, b1;
    oracle_pseudocounts(y, N, xi, &b0, &b1);
    const uint8_t* cols[8];
    for (int j = 0; j < n_s; ++j) cols[j] = codes + ((size_t)d * M + S[j]) * N;
    double sh_s = oracle_sh(cols, n_s, y, N, c, b0, b1);
    cols[n_s] = codes + ((size_t)d * M + i) * N;
    double sh_si = oracle_sh(cols, n_s + 1, y, N, c, b0, b1);
    return sh_s - sh_si;
}

/*
 * IG^k_max (Eq. 1) maximised over discretisations as well, for the variables
 * listed in vars (all M if vars == NULL), k = 1..5.
 *   ig[n_vars]           FP64 maximum,
 *   tuples[n_vars][k-1]  partner set of the maximum (ascending), k >= 2,
 *   best_disc[n_vars]    discretisation of the maximum,
 *   second[n_vars]       largest IG over all other (discretisation, set) pairs
 *                        (-inf if there is none).
 * Scan order: d ascending, then S lexicographic ascending; strict '>' keeps
 * the first maximum, i.e. the lowest (d, S).
 */
int oracle_max_ig(const uint8_t* codes, const uint8_t* y, int N, int M, int D, int c, int k, double xi,
                  const int32_t* vars, int n_vars, double* ig, int32_t* tuples, int32_t* best_disc,
                  double* second)
{
    if (k < 1 || k > 5 || M < k) return -1;
    if (vars == NULL) n_vars = M;
    double b0, b1;
    oracle_pseudocounts(y, N, xi, &b0, &b1);
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < n_vars; ++t) {
        const int i = vars ? vars[t] : t;
        double best = -INFINITY, runner = -INFINITY;
        int32_t bs[4] = {-1, -1, -1, -1};
        int32_t bd = -1;
        for (int d = 0; d < D; ++d) {
            const uint8_t* ci = codes + ((size_t)d * M + i) * N;
            if (k == 1) {
                const uint8_t* cols[1] = {ci};
                double g = oracle_sh(NULL, 0, y, N, c, b0, b1) - oracle_sh(cols, 1, y, N, c, b0, b1);
                if (g > best) { runner = best; best = g; bd = d; }
                else if (g > runner) runner = g;
            } else if (k == 2) {
                for (int m = 0; m < M; ++m) {
                    if (m == i) continue;
                    const uint8_t* cm = codes + ((size_t)d * M + m) * N;
                    const uint8_t* cs[1] = {cm};
                    const uint8_t* csi[2] = {cm, ci};
                    double g = oracle_sh(cs, 1, y, N, c, b0, b1) - oracle_sh(csi, 2, y, N, c, b0, b1);
                    if (g > best) { runner = best; best = g; bd = d; bs[0] = m; }
                    else if (g > runner) runner = g;
                }
            } else if (k == 3) {
                for (int m1 = 0; m1 < M; ++m1) {
                    if (m1 == i) continue;
                    const uint8_t* c1 = codes + ((size_t)d * M + m1) * N;
                    for (int m2 = m1 + 1; m2 < M; ++m2) {
                        if (m2 == i) continue;
                        const uint8_t* c2 = codes + ((size_t)d * M + m2) * N;
                        const uint8_t* cs[2] = {c1, c2};
                        const uint8_t* csi[3] = {c1, c2, ci};
                        double g = oracle_sh(cs, 2, y, N, c, b0, b1) - oracle_sh(csi, 3, y, N, c, b0, b1);
                        if (g > best) { runner = best; best = g; bd = d; bs[0] = m1; bs[1] = m2; }
                        else if (g > runner) runner = g;
                    }
                }
            } else if (k == 4) {
                for (int m1 = 0; m1 < M; ++m1) {
                    if (m1 == i) continue;
                    const uint8_t* c1 = codes + ((size_t)d * M + m1) * N;
                    for (int m2 = m1 + 1; m2 < M; ++m2) {
                        if (m2 == i) continue;
                        const uint8_t* c2 = codes + ((size_t)d * M + m2) * N;
                        for (int m3 = m2 + 1; m3 < M; ++m3) {
                            if (m3 == i) continue;
                            const uint8_t* c3 = codes + ((size_t)d * M + m3) * N;
                            const uint8_t* cs[3] = {c1, c2, c3};
                            const uint8_t* csi[4] = {c1, c2, c3, ci};
                            double g = oracle_sh(cs, 3, y, N, c, b0, b1) - oracle_sh(csi, 4, y, N, c, b0, b1);
                            if (g > best) { runner = best; best = g; bd = d; bs[0] = m1; bs[1] = m2; bs[2] = m3; }
                            else if (g > runner) runner = g;
                        }
                    }
                }
            } else {
                for (int m1 = 0; m1 < M; ++m1) {
                    if (m1 == i) continue;
                    const uint8_t* c1 = codes + ((size_t)d * M + m1) * N;
                    for (int m2 = m1 + 1; m2 < M; ++m2) {
                        if (m2 == i) continue;
                        const uint8_t* c2 = codes + ((size_t)d * M + m2) * N;
                        for (int m3 = m2 + 1; m3 < M; ++m3) {
                            if (m3 == i) continue;
                            const uint8_t* c3 = codes + ((size_t)d * M + m3) * N;
                            for (int m4 = m3 + 1; m4 < M; ++m4) {
                                if (m4 == i) continue;
                                const uint8_t* c4 = codes + ((size_t)d * M + m4) * N;
                                const uint8_t* cs[4] = {c1, c2, c3, c4};
                                const uint8_t* csi[5] = {c1, c2, c3, c4, ci};
                                double g = oracle_sh(cs, 4, y, N, c, b0, b1) - oracle_sh(csi, 5, y, N, c, b0, b1);
                                if (g > best) {
                                    runner = best; best = g; bd = d;
                                    bs[0] = m1; bs[1] = m2; bs[2] = m3; bs[3] = m4;
                                } else if (g > runner) runner = g;
                            }
                        }
                    }
                }
            }
        }
        ig[t] = best;
        if (best_disc) best_disc[t] = bd;
        if (second) second[t] = runner;
        if (tuples && k >= 2)
            for (int j = 0; j < k - 1; ++j) tuples[(size_t)t * (k - 1) + j] = bs[j];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* chi^2 CDF for integer df, by the textbook finite forms of the regularised */
/* incomplete gamma function at half-integer order (Abramowitz & Stegun      */
/* 6.5.13 / 26.4.4-26.4.5, 26.2.11):                                         */
/*   upper tail Q(df, x) = e^{-x/2} sum_{j<df/2} (x/2)^j / j!   (df even)     */
/*   Q(df, x) = erfc(sqrt(x/2)) + e^{-x/2} sum_{j<(df-1)/2} (x/2)^{j+1/2} /   */
/*              Gamma(j + 3/2)                                  (df odd)      */
/* and, for small x, the lower-tail series                                    */
/*   P(a, z) = z^a e^{-z} sum_n z^n / Gamma(a + n + 1),   a = df/2, z = x/2.   */
/* All terms positive: no cancellation in either branch.                      */
/* ------------------------------------------------------------------------ */
static double chi2_upper(double x, int df)
{
    double z = 0.5 * x;
    double ez = exp(-z);
    double q, term;
    if (df % 2 == 0) {
        q = 0.0;
        term = ez; /* j = 0 */
        for (int j = 0; j < df / 2; ++j) {
            q += term;
            term *= z / (double)(j + 1);
        }
    } else {
        q = erfc(sqrt(z));
        term = ez * sqrt(z) / tgamma(1.5); /* j = 0 */
        for (int j = 0; j < (df - 1) / 2; ++j) {
            q += term;
            term *= z / ((double)j + 1.5);
        }
    }
    return q;
}

static double chi2_lower_series(double x, int df)
{
    double a = 0.5 * df, z = 0.5 * x;
    if (z <= 0.0) return 0.0;
    double lead = exp(a * log(z) - z - lgamma(a + 1.0)); /* z^a e^-z / Gamma(a+1) */
    double sum = 1.0, term = 1.0;
    for (int n = 1; n < 100000; ++n) {
        term *= z / (a + (double)n);
        sum += term;
        if (term < sum * 1e-17) break;
    }
    return lead * sum;
}

double oracle_chi2_cdf(double x, int df)
{
    if (x <= 0.0) return 0.0;
    if (0.5 * x < 0.5 * df + 1.0) return chi2_lower_series(x, df);
    return 1.0 - chi2_upper(x, df);
}

double oracle_chi2_sf(double x, int df)
{
    if (x <= 0.0) return 1.0;
    if (0.5 * x < 0.5 * df + 1.0) return 1.0 - chi2_lower_series(x, df);
    return chi2_upper(x, df);
}

/*
 * Extreme-value fit of the significance paragraph of section "Theory".
 * IG_max of an irrelevant variable is modelled as the largest of T
 * independent single-tuple statistics, 2 IG ~ chi^2_df, so
 *     P(IG_max <= g) = F_df(2 g)^T.
 * Maximum likelihood over the n irrelevant variables (u_i = F_df(2 IG_i),
 * density T u^(T-1)) gives T = -n / sum ln u_i.  Then
 *     p_i = 1 - F_df(2 IG_i)^T,
 *     IG_lim = F_df^{-1}((1 - alpha)^(1/T)) / 2   (bisection in FP64).
 * df = (c-1) c^(k-1).  Variables with u_i == 0 (IG <= 0) carry no finite
 * likelihood term and are left out of the fit (their p-value is 1).
 */
int oracle_ig_lim(const double* ig, int M, int k, int divisions, const uint8_t* irrelevant_mask,
                  double alpha, double* p_values, double* ig_lim, double* n_eff)
{
    const int c = divisions + 1;
    int df = c - 1;
    for (int j = 1; j < k; ++j) df *= c;
    double sum_log = 0.0;
    long n = 0;
    for (int i = 0; i < M; ++i) {
        if (irrelevant_mask && !irrelevant_mask[i]) continue;
        double u = oracle_chi2_cdf(2.0 * ig[i], df);
        if (u <= 0.0) continue;
        sum_log += log(u);
        n++;
    }
    if (n == 0 || !(sum_log < 0.0)) return -2;
    double T = -(double)n / sum_log;
    for (int i = 0; i < M; ++i) {
        double u = oracle_chi2_cdf(2.0 * ig[i], df);
        /* 1 - u^T = -expm1(T ln u) keeps small p-values accurate */
        p_values[i] = (u <= 0.0) ? 1.0 : -expm1(T * log(u));
    }
    double target = pow(1.0 - alpha, 1.0 / T);
    double lo = 0.0, hi = 1.0;
    while (oracle_chi2_cdf(hi, df) < target) hi *= 2.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (oracle_chi2_cdf(mid, df) < target) lo = mid; else hi = mid;
    }
    *ig_lim = 0.25 * (lo + hi);
    *n_eff = T;
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Contrast variables (section "Canonical package usage").                   */
/*                                                                            */
/* Pseudo-random permutation of [0, n): the Luby-Rackoff (Feistel) network    */
/* on 2h-bit words, h = ceil(ceil(log2 n) / 2), 10 rounds (fewer rounds leave */
/* measurable bias on small domains; 10 is the count of NIST's FF1)          */
/*     (L, R) -> (R, L xor F_r(R)),   F_r(R) = Philox4x32-10 word 0 of        */
/*     counter (R, r, stream, 0x43545253), key (seed_lo, seed_hi), masked to h */
/*     bits,                                                                  */
/* is a bijection of [0, 2^(2h)); cycle walking (Black and Rogaway, "Ciphers  */
/* with arbitrary finite domains", CT-RSA 2002) applies it until the value    */
/* falls below n, which restricts it to a bijection of [0, n).  The orbit of  */
/* i returns to i within 2^(2h) steps, so the walk ends.                      */
/* ------------------------------------------------------------------------ */
static const uint32_t kContrastTag = 0x43545253u;  /* "CTRS" */

static uint32_t feistel10(uint32_t v, int h, uint32_t stream, const uint32_t key[2])
{
    const uint32_t mask = (h >= 32) ? 0xFFFFFFFFu : ((1u << h) - 1u);
    uint32_t L = v >> h, R = v & mask;
    for (uint32_t r = 0; r < 10; ++r) {
        uint32_t ctr[4] = {R, r, stream, kContrastTag}, out[4];
        oracle_philox4x32_10(ctr, key, out);
        uint32_t nl = R, nr = (L ^ out[0]) & mask;
        L = nl;
        R = nr;
    }
    return (L << h) | R;
}

uint32_t oracle_shuffle_index(uint32_t i, uint32_t n, uint32_t stream, uint64_t seed)
{
    if (n <= 1) return 0;
    int b = 0;
    while ((1ull << b) < (unsigned long long)n) ++b;   /* 2^b >= n */
    int h = (b + 1) / 2;
    if (h < 1) h = 1;
    const uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t v = i;
    do {
        v = feistel10(v, h, stream, key);
    } while (v >= n);
    return v;
}

/* x_out [(M + n_contrast)][N]: rows 0..M-1 are x; row M + j is variable
 * src[j] = shuffle_M(j mod M) (stream 0xFFFFFFFF) with sample i taken from
 * sample shuffle_N(i) (stream j). */
int oracle_contrast(const float* x, int N, int M, int n_contrast, uint64_t seed, float* x_out, int32_t* src)
{
    if (N < 1 || M < 1 || n_contrast < 0) return -1;
    memcpy(x_out, x, sizeof(float) * (size_t)N * (size_t)M);
    for (int j = 0; j < n_contrast; ++j) {
        const uint32_t s = oracle_shuffle_index((uint32_t)(j % M), (uint32_t)M, 0xFFFFFFFFu, seed);
        if (src) src[j] = (int32_t)s;
        float* row = x_out + (size_t)(M + j) * N;
        for (int i = 0; i < N; ++i)
            row[i] = x[(size_t)s * N + oracle_shuffle_index((uint32_t)i, (uint32_t)N, (uint32_t)j, seed)];
    }
    return 0;
}

