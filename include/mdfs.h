/*
 * mdfs.h -- C ABI of the GB300-native MDFS information-gain scan.
 *
 * MDFS (Piliszek et al., arXiv 1811.00631) ranks variables by
 *     IG^k_max(y; x_i) = N max_S [ H(y | S) - H(y | S, x_i) ]            (Eq. 1)
 * where S runs over all (k-1)-subsets of the other variables and, in
 * addition, over several random discretisations of the data (section
 * "Algorithm and implementation").  This library computes that scan on one
 * GPU (sm_103a) for k = 1..5 and fits the chi^2 / extreme-value null that
 * turns the result into p-values (section "Theory").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Pointers: every array argument may be a host pointer or a device pointer of
 *   the current CUDA device; the library tells them apart with
 *   cudaPointerGetAttributes, and refuses device memory of another GPU with
 *   MDFS_EINVAL.  Host inputs are copied to the device inside the
 *   call; host outputs are written before the call returns.  All outputs are
 *   owned by the caller.  The library keeps only a cached device workspace per
 *   (device, stream), which mdfs_release() frees.
 * Layout: x is variable-major, x[v * N + s] is sample s of variable v
 *   (an N x M column-major matrix with leading dimension N).
 * Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).  A
 *   call with device outputs is stream-ordered on `stream` but waits once for
 *   the 16-byte validation result of its inputs; scans that run a tensor-core
 *   kernel (k = 2 with 2 or 3 classes, k = 3 with 2 classes) also wait for
 *   their kernels, to read the kernel's error flag.  A call with host
 *   outputs, or with stream == NULL, returns after its results are complete.
 *   Calls on different streams may run concurrently; calls sharing one stream
 *   from several host threads must be serialised by the caller.
 * Errors: 0 on success, a negative MDFS_E* code otherwise; mdfs_last_error()
 *   then describes the failure (thread-local string).  On error no output is
 *   guaranteed to have been written.
 * Limits: 1 <= divisions <= 3 (c = divisions + 1 classes per variable,
 *   section "Algorithm and implementation": the same c for all variables);
 *   2 <= c <= N <= 32768; 1 <= discretizations <= 1024; k <= M <= 65535;
 *   for k = 2, discretizations * M < 2^32; for k = 3,
 *   discretizations * M * M < 2^32; k = 4 needs divisions = 1 and
 *   discretizations * M^3 < 2^32; k = 5 needs divisions = 1 and
 *   C(M, 4) < 2^32 (M <= 568), and for mdfs_max_ig_shard also
 *   discretizations * C(M, 4) < 2^32.
 */
#ifndef MDFS_H
#define MDFS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define MDFS_OK 0
#define MDFS_EINVAL (-1)      /* argument out of range, or y not in {0, 1}           */
#define MDFS_EDEGENERATE (-2) /* one decision class is empty (Eq. beta undefined)    */
#define MDFS_ENONFINITE (-3)  /* x holds NaN or +-Inf                                 */
#define MDFS_ENOMEM (-4)      /* device workspace allocation failed                   */
#define MDFS_ECUDA (-5)       /* a CUDA runtime call or kernel launch failed          */
#define MDFS_ETIMEOUT (-6)    /* a bounded device-side wait gave up (tensor cores)    */
#define MDFS_ETRUNCATED (-7)  /* more output records than the caller's capacity        */

/* x element types */
#define MDFS_F32 0
#define MDFS_I8 1

typedef struct mdfs_data {
    int dtype;          /* MDFS_F32 or MDFS_I8                                       */
    const void* x;      /* [M][N] variable-major data, host or device               */
    const uint8_t* y;   /* [N] binary decision in {0, 1}, host or device (section
                           "Algorithm and implementation": binary decisions only);
                           may be NULL for mdfs_discretize                          */
    int N;              /* number of objects (samples)                              */
    int M;              /* number of variables                                      */
} mdfs_data;

/*
 * Randomised rank-based discretisation (section "Algorithm and
 * implementation").  For each variable v and discretisation d the c class
 * shares are drawn uniformly from [1-range, 1+range) (Philox4x32-10, key =
 * seed, counter = (j/4, v, d, 0x4D444653), 20-bit fixed point), turned into
 * c-1 strictly increasing 0-based positions in [1, N-1] of the sorted
 * variable, and the values at those positions become the thresholds t_j;
 * code(x) = #{ j : x >= t_j } (ties go to the upper class).
 *
 * codes: [discretizations][M][N] uint8, caller-owned, host or device.
 * range: 0 (equipotent split) .. 1 (completely random split).
 */
int mdfs_discretize(const mdfs_data* data, int divisions, int discretizations, double range,
                    uint64_t seed, uint8_t* codes, void* stream);

/*
 * IG^k_max (Eq. 1; Eq. 3 for k = 1), maximised over all (k-1)-subsets S of
 * the other variables and over all discretisations.  Entropies are the
 * pseudocount-regularised, N-scaled conditional entropies of Eqs. H, p and
 * beta, in nats:
 *     SH(S) = sum_v [ f(n_v + b0 + b1) - f(n0_v + b0) - f(n1_v + b1) ],
 *     f(t) = t ln t,  b^d = pc_xi * N^d / min(N^0, N^1),
 * summed over all c^|S| voxels v, and IG(i | S) = SH(S) - SH(S + {i}).
 *
 * k:          1 .. 5 (D M^3 < 2^32 at k = 4; C(M,4) < 2^32 at k = 5, and with
 *             divisions 2 or 3 also D C(M,4) < 2^32).
 * pc_xi:      the pseudocount parameter xi, 0 < pc_xi < 1.
 * ig:         [M] float, the maximum per variable (may be slightly negative
 *             when the pseudocounts dominate).
 * tuples:     [M][k-1] int32 or NULL: the partner set of the maximum in
 *             ascending order (ignored for k = 1).
 * best_disc:  [M] int32 or NULL: the discretisation of the maximum.
 * Ties are broken towards the lowest (discretisation, lexicographic S).
 * The discretisation is the one mdfs_discretize produces for the same seed.
 */
int mdfs_max_ig(const mdfs_data* data, int k, int divisions, int discretizations, double range,
                double pc_xi, uint64_t seed, float* ig, int32_t* tuples, int32_t* best_disc,
                void* stream);

/*
 * IG^k_max of several dimensions k of the same data and discretisations in
 * one call (the analyses "in all possible dimensionalities" of section
 * "Examples", Tables 1-2): entry j is exactly mdfs_max_ig with k = ks[j].
 *
 * ks:         n_k (1 .. 5) distinct values in 1 .. 5.
 * ig:         [n_k] pointers, ig[j] as mdfs_max_ig's ig for k = ks[j].
 * tuples:     NULL, or [n_k] pointers, each NULL or [M][ks[j]-1] int32.
 * best_disc:  NULL, or [n_k] pointers, each NULL or [M] int32.
 * The scans share the staged inputs and their validation (one host round
 * trip).  Where the tensor-core kernels serve both k = 2 and k = 3 (two
 * classes, class sizes below 4096), k = 1, 2 and 3 also share one
 * discretisation, its single counts and its one-hot rows.  Errors and
 * ownership as for mdfs_max_ig; on an error some outputs may be written.
 */
int mdfs_max_ig_multi(const mdfs_data* data, int n_k, const int* ks, int divisions, int discretizations,
                      double range, double pc_xi, uint64_t seed, float* const* ig, int32_t* const* tuples,
                      int32_t* const* best_disc, void* stream);

/*
 * Batched scan: n_jobs independent mdfs_max_ig jobs over resamples of one
 * dataset, e.g. bootstrap or cross-validation folds and y-permutation nulls
 * (the null distribution the significance test of section "Theory" is fitted
 * to).  Job j is exactly mdfs_max_ig on
 *     x_j[v][t] = x[v][idx_j[t]],   y_j[t] = y[perm_j[idx_j[t]]],   t = 0..N-1,
 * with idx_j = sample_idx + j N and perm_j = y_perm + j N (either may be NULL =
 * identity), the same k, divisions, discretizations, range, pc_xi and seed.
 *
 * sample_idx, y_perm:  [n_jobs][N] int32, host or device; entries in [0, N).
 * ig:                  [n_jobs][M] float; tuples [n_jobs][M][k-1] or NULL;
 *                      best_disc [n_jobs][M] or NULL (host or device).
 * Every job's class sizes are computed in one device pass and read back once;
 * a job whose decision has one class fails the call with MDFS_EDEGENERATE and
 * an index outside [0, N) with MDFS_EINVAL (the message names the job), before
 * any scan runs.  With k = 2 and 2 or 3 classes per variable the jobs run in
 * chunks, one tensor-core launch per chunk over (job, discretisation, tile)
 * work items; the environment variable MDFS_BATCH_BYTES (default 8 GB) bounds
 * the device memory of a chunk's one-hot operands.  The launch's pipeline
 * depth is chosen by timing on the first call per shape and cached in memory
 * and in the file named by MDFS_TUNE_FILE (lines "<kernel> M=.. N=.. c=.. D=..
 * -> <stages>"); MDFS_TUNE=0 takes the deepest pipeline that fits.  The
 * choice never changes a result.  Returns after all jobs are complete.
 */
int mdfs_max_ig_batch(const mdfs_data* data, int n_jobs, const int32_t* sample_idx, const int32_t* y_perm, int k,
                      int divisions, int discretizations, double range, double pc_xi, uint64_t seed, float* ig,
                      int32_t* tuples, int32_t* best_disc, void* stream);

/*
 * Sharded scan of one job over several processes or GPUs (the tuple space of
 * Eq. 1 is embarrassingly parallel).  Shard `shard` of `n_shards` scans its
 * contiguous share of the tuple tiles (the pair path without tensor cores and
 * k = 1 run whole on shard 0) and writes the packed max keys:
 *     key = (order-preserving bits of float IG) << 32 | ~(tie-break index),
 *     index = d M + m (k = 2), (d M + m1) M + m2 (k = 3), d (k = 1),
 * so that a larger key is a larger IG and, on a tie, the lower (d, S).  The
 * element-wise UNSIGNED maximum of all shards' keys equals the keys of the
 * unsharded scan exactly (for a signed all-reduce, flip bit 63 before and
 * after).  keys_out: [M] uint64, host or device.  Returns after completion.
 */
int mdfs_max_ig_shard(const mdfs_data* data, int k, int divisions, int discretizations, double range, double pc_xi,
                      uint64_t seed, int shard, int n_shards, uint64_t* keys_out, void* stream);

/*
 * Decodes merged keys into the outputs of mdfs_max_ig (same meaning):
 * ig [M] float, tuples [M][k-1] or NULL, best_disc [M] or NULL; keys of 0
 * (no candidate) give NaN and discretisation -1.  Host or device pointers.
 */
int mdfs_keys_decode(const uint64_t* keys, int M, int k, float* ig, int32_t* tuples, int32_t* best_disc, void* stream);

/*
 * Significance of IG^k_max (section "Theory"): a single tuple's 2 IG is
 * chi^2 with df = (c-1) c^(k-1) degrees of freedom; the maximum over T
 * effective tests has CDF F_df(2 g)^T.  T is fitted by maximum likelihood on
 * the irrelevant variables (T = -n / sum ln F_df(2 IG_i); variables with
 * IG <= 0 carry no likelihood term), then
 *     p_i    = 1 - F_df(2 IG_i)^T,
 *     IG_lim = F_df^{-1}((1 - alpha)^(1/T)) / 2.
 * Runs in FP64 on the device: the CDF of every variable in parallel, then T
 * and IG_lim (a parallel root search) in one CTA, then the p-values.
 *
 * ig:               [M] float, host or device (an mdfs_max_ig result).
 * discretizations:  recorded only; the fit absorbs it into T.
 * irrelevant_mask:  [M] uint8 or NULL (NULL = every variable is used).
 * p_values:         [M] double, host or device.  A device array also holds
 *                   the CDF values during the call; after MDFS_EDEGENERATE
 *                   its contents are unspecified.
 * ig_lim, n_eff:    one double each, host or device (n_eff = fitted T).
 * Returns MDFS_EDEGENERATE when no variable contributes to the fit.
 */
int mdfs_ig_lim(const float* ig, int M, int k, int divisions, int discretizations,
                const uint8_t* irrelevant_mask, double alpha, double* p_values, double* ig_lim,
                double* n_eff, void* stream);

/*
 * Contrast variables (section "Canonical package usage"): copies of original
 * variables with their samples shuffled, appended to the data so that the
 * significance fit sees variables known to be irrelevant.
 *
 * Row M + j of x_ext (j < n_contrast) is variable src[j] = P_M(j mod M) with
 * sample i taken from sample P_N^(j)(i), where P_n^(s) is a pseudo-random
 * permutation of [0, n): a 10-round Feistel network on 2h-bit words
 * (h = ceil(ceil(log2 n) / 2)) with round function word 0 of Philox4x32-10
 * (counter (R, round, s, 0x43545253), key = seed), restricted to [0, n) by
 * cycle walking; P_M uses stream s = 0xFFFFFFFF.  Sources are drawn without
 * replacement while j < M.  Rows 0 .. M-1 of x_ext are x.
 *
 * data:       x (dtype, [M][N] variable-major), y unused; host or device.
 * n_contrast: 0 .. 65535 - M.
 * x_ext:      [(M + n_contrast)][N] of x's dtype, caller-owned, host or device.
 * src:        [n_contrast] int32 or NULL, host or device.
 * Errors: MDFS_EINVAL (arguments), MDFS_ENOMEM, MDFS_ECUDA.
 */
int mdfs_contrast(const mdfs_data* data, int n_contrast, uint64_t seed, void* x_ext, int32_t* src, void* stream);

/* Multiple-testing adjustments of p-values (the selection step of section
 * "Canonical package usage"). */
#define MDFS_ADJUST_NONE 0
#define MDFS_ADJUST_BONFERRONI 1
#define MDFS_ADJUST_HOLM 2
#define MDFS_ADJUST_HOCHBERG 3
#define MDFS_ADJUST_BH 4
#define MDFS_ADJUST_BY 5

/*
 * Adjusts m p-values (p_(1) <= ... <= p_(m) sorted, ties by index, results
 * capped at 1): Bonferroni m p; Holm max_{s<=r} (m-s+1) p_(s); Hochberg
 * min_{s>=r} (m-s+1) p_(s); Benjamini-Hochberg min_{s>=r} m/s p_(s);
 * Benjamini-Yekutieli the same times sum_{s=1..m} 1/s.  NaN inputs are not
 * counted in m and stay NaN.  Runs as one CTA on the device.
 *
 * p, adjusted: [m] double, host or device; m in 1 .. 65536.
 * Errors: MDFS_EINVAL (arguments, unknown method), MDFS_ENOMEM, MDFS_ECUDA.
 */
int mdfs_p_adjust(const double* p, int m, int method, double* adjusted, void* stream);

/*
 * Interesting tuples (section "Examples": the package's third entry point
 * beside the max scan and the selection pipeline): every (variable v,
 * partner set S) with |S| = k - 1, v not in S, whose IG(v | S) maximised
 * over the discretisations reaches ig_threshold (nats).  Same data, k,
 * divisions, discretizations, range, pc_xi and seed as mdfs_max_ig (k = 1..5,
 * the same limits); every scan kernel emits the qualifying roles as it goes.
 *
 * Records are sorted by (v, S) ascending: var [n], tuples [n][k-1] (S
 * ascending; NULL allowed for k = 1), ig [n] float, best_disc [n] (the lowest
 * discretisation reaching the maximum; NULL allowed), all of at least
 * `capacity` entries, host or device.  *count (host) receives n.
 * capacity: 1 .. 2^22.
 * Errors: those of mdfs_max_ig; MDFS_ETRUNCATED when more than capacity
 * records reach the threshold (*count then holds their number, or a lower
 * bound when the message says "at least"; no record is written).
 */
int mdfs_interesting_tuples(const mdfs_data* data, int k, int divisions, int discretizations, double range,
                            double pc_xi, uint64_t seed, double ig_threshold, int capacity, int32_t* var,
                            int32_t* tuples, float* ig, int32_t* best_disc, int64_t* count, void* stream);

/*
 * The canonical selection pipeline (section "Canonical package usage"):
 *   1. n_contrast contrast variables (mdfs_contrast, same seed);
 *   2. IG^k_max over the M + n_contrast variables (mdfs_max_ig, same seed);
 *   3. the chi^2 / extreme-value fit (mdfs_ig_lim) on the contrast variables
 *      only, at alpha = level, and p-values for every variable;
 *   4. the adjustment (mdfs_p_adjust) of the p-values of the M original
 *      variables (contrast variables do not enter the adjustment);
 *   5. relevant[i] = adjusted[i] < level.
 *
 * Outputs are for the M original variables (host or device, caller-owned):
 * ig [M] float; tuples [M][k-1] int32 or NULL (partner indices in
 * [0, M + n_contrast): M + j is contrast j); best_disc [M] int32 or NULL;
 * p_values, adjusted [M] double; relevant [M] uint8; ig_lim, n_eff one
 * double each or NULL; contrast_src [n_contrast] int32 or NULL.
 * Limits: n_contrast >= 1 and M + n_contrast <= 65535, plus the limits of
 * mdfs_max_ig on the extended set.
 * Errors: those of mdfs_max_ig and mdfs_ig_lim (MDFS_EDEGENERATE when no
 * contrast variable has IG > 0).
 */
int mdfs_select(const mdfs_data* data, int n_contrast, int k, int divisions, int discretizations, double range,
                double pc_xi, uint64_t seed, int p_adjust_method, double level, float* ig, int32_t* tuples,
                int32_t* best_disc, double* p_values, double* adjusted, uint8_t* relevant, double* ig_lim,
                double* n_eff, int32_t* contrast_src, void* stream);

/*
 * mdfs_max_ig without any device allocation (the paper has no counterpart:
 * this is a deployment variant).
 *
 * Some callers cannot let a library allocate device memory: a serving process
 * whose allocator owns the device budget, a host application that only lets
 * plug-ins use memory it handed out, or a latency-bound loop that cannot pay
 * for cudaMalloc/cudaFree and the synchronisation they imply.  This entry point
 * computes the same result as mdfs_max_ig for k = 1 or 2, and calls no
 * cudaMalloc, cudaFree or other allocating routine.  Its scratch (bit planes,
 * tables, counts, keys) lives in one file-scope device array of
 * MDFS_NOALLOC_SCRATCH_BYTES, which every GPU that loads that part of the
 * library holds until the process exits.
 *
 * x, y, ig, tuples and best_disc must be device pointers of the current device
 * (MDFS_EINVAL otherwise).  Problems whose scratch does not fit the array are
 * rejected with MDFS_EINVAL and a message giving the bytes needed; roughly
 * discretizations * M * (divisions * (N/8 + 20) + 16) bytes must stay below
 * the array size.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current).  The address is kept until
 * mdfs_release(), which a caller must call after a cudaDeviceReset before the
 * next call.  All calls share the
 * array and it keeps the last call's contents: two calls whose work overlaps
 * on the GPU (different streams, or different host threads) race and must not
 * be issued; serialise them.  Every call copies a 16-byte validation result of
 * its inputs to a host buffer and synchronises its stream before the scan
 * kernels are enqueued, so a call cannot be captured into a CUDA graph; with a
 * non-NULL stream the rest is stream-ordered.
 */
#define MDFS_NOALLOC_SCRATCH_BYTES (32u << 20)
int mdfs_max_ig_noalloc(const mdfs_data* data, int k, int divisions, int discretizations, double range,
                        double pc_xi, uint64_t seed, float* ig, int32_t* tuples, int32_t* best_disc,
                        void* stream);

/* Thread-local description of the last failure of this thread ("" if none). */
const char* mdfs_last_error(void);

/* Frees every cached device workspace of this process.  No call may be in
 * flight.  Returns 0. */
int mdfs_release(void);

/* Frees the cached device workspace of one (current device, stream) pair,
 * e.g. when a long-lived stream that ran a large job goes on with small ones.
 * No call may be in flight on that stream.  Returns 0 (also when the stream
 * has no workspace). */
int mdfs_release_stream(void* stream);

/* ABI version, currently 1. */
int mdfs_abi_version(void);

/* Tracing: while enabled (enable != 0), every kernel launch of the library is
 * bracketed by CUDA events on its stream.  Process-wide switch; returns 0. */
int mdfs_profile(int enable);

/* Writes one line "name launches total_ms" per kernel recorded since the last
 * report into buf (len bytes, NUL-terminated), waiting for the events, and
 * clears the record.  Returns MDFS_EINVAL if the text was truncated. */
int mdfs_profile_report(char* buf, int len);

/* Diagnostic: number of kernels the calling thread's most recent mdfs_* call
 * launched (0 if it failed before its first launch). */
int mdfs_last_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* MDFS_H */
