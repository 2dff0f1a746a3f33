// Internal declarations shared by the CUDA translation units of the MDFS library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace mdfs {

// Fixed-point scale of the entropy tables: values are int64 multiples of 2^-32.
// Integer accumulation makes every SH sum exact and order-independent; the only
// rounding is one 2^-33 per table entry (tables are built in FP64).
constexpr double kFxScale = 4294967296.0;  // 2^32
constexpr int kMaxC = 4;                   // classes per variable (divisions <= 3)
constexpr int kMaxN = 32768;               // samples (bounded by the in-CTA sort)
constexpr int kMaxD = 1024;                // discretisations
constexpr uint32_t kPhiloxTag = 0x4D444653u;  // 'MDFS', fourth counter word

// Geometry of the class-sorted bit planes: class-0 samples occupy words
// [0, W0), class-1 samples words [W0, W0 + W1); rows are padded to Ws words
// (a multiple of 4) with zero words.
struct PlaneGeom {
    int N, N0, N1;
    int W0, W1, W, Ws;
};

inline PlaneGeom make_geom(int N, int N0) {
    PlaneGeom g;
    g.N = N;
    g.N0 = N0;
    g.N1 = N - N0;
    g.W0 = (g.N0 + 31) / 32;
    g.W1 = (g.N1 + 31) / 32;
    g.W = g.W0 + g.W1;
    g.Ws = (g.W + 3) & ~3;
    return g;
}

// K geometry of the one-hot tensor-core operands: class-0 samples in
// [0, N0), zero padding to K0p (a multiple of 128), class-1 samples in
// [K0p, K0p + N1), zero padding to Kp.
struct TcGeom {
    int N0, N1, K0p, Kp, nkb0, nkb;
};

// Pair record of the two-class (c = 2) k = 3 path, 8 bytes: class counts of
// the voxel (1, 1) of the pair times 4 (4 n0 | 4 n1 << 16; n < 16384) and its
// regularised entropy SH as an int32 multiple of 2^-fbits (wrap-around).
struct __align__(8) PairC {
    uint32_t cnt;
    int sh;
};

// Interesting-tuple emission (section "Examples"): every (variable, partner
// set) whose IG reaches a threshold is inserted into an open-addressing hash
// table keyed by v | p1 << 16 | p2 << 32 | p3 << 48 (unused partners 0xFFFF;
// an all-ones key marks an empty slot), with the maximum over discretisations
// kept as a packed key (IG, discretisation).  keys == NULL disables emission.
struct EmitTable {
    unsigned long long* keys = nullptr;  // [mask + 1]
    unsigned long long* vals = nullptr;  // [mask + 1], 0 = none
    unsigned int mask = 0;               // table size - 1, a power of two minus one
    long long thr_fx = 0;                // threshold in multiples of 2^-32 (the IG fixed point)
    int* n_keys = nullptr;               // distinct keys inserted
    int* full = nullptr;                 // set when an insert found no free slot
};

// The emission threshold as the int32 fixed point with fbits fraction bits of
// the tensor-core kernels (multiples of 2^-fbits, rounded up; clamped to the
// int range).
inline int emit_threshold_fx(const EmitTable& t, int fbits) {
    const long long v = (t.thr_fx + (1ll << (32 - fbits)) - 1) >> (32 - fbits);
    return (int)(v > 2147483647ll ? 2147483647ll : v < -2147483647ll ? -2147483647ll : v);
}

// ---- launchers (all asynchronous on `st`) -----------------------------------
// stats[0] = N1 (count of y == 1), stats[1] = number of y not in {0,1},
// stats[2] = number of non-finite x.  perm = class-stable sample order.
cudaError_t launch_stats(const uint8_t* y, int N, int* stats, int* perm, cudaStream_t st);
cudaError_t launch_check_finite(const float* x, long long count, int* flag, cudaStream_t st);

// Batch job j: x_j[v][t] = x[v][idx[t]], y_j[t] = y[yperm[idx[t]]] (NULL = identity);
// out-of-range indices increment *flag.
cudaError_t launch_gather_job(const void* x, int dtype, const uint8_t* y, int N, int M, const int* idx,
                              const int* yperm, void* xo, uint8_t* yo, int* flag, cudaStream_t st);

// Class sizes of every batch job: out[j] = (n1, bad) with n1 the number of
// y[yperm_j[idx_j[t]]] != 0 and bad != 0 when an index lies outside [0, N) or a
// label outside {0, 1} (idx, yperm [n_jobs][N] or NULL = identity).
cudaError_t launch_batch_counts(const uint8_t* y, int N, const int* idx, const int* yperm, int n_jobs, int2* out,
                                cudaStream_t st);

// int64 fixed-point tables T0[n] = f(n + b0), T1[n] = f(n + b1), TB[n] = f(n + b0 + b1),
// n = 0..N, f(t) = t ln t; laid out as [3][N + 1].
cudaError_t launch_ftable(int N, double b0, double b1, long long* tab, cudaStream_t st);
// f tables of the packed-count kernels (t3, k4, k5): f(n + b0) at [0, 2^16),
// f(n + b1) at [2^16, 2^17), f(n + b0 + b1) at [2^17, 2^18), so that any two
// 16-bit class counts index inside the table.
constexpr int kWideTab = 1 << 18;
cudaError_t launch_ftable_wide(double b0, double b1, long long* tab, cudaStream_t st);

// One CTA per variable: sort, thresholds, and codes and/or class-sorted bit planes.
// planes: [D][M][c-1][Ws] u32 (NULL = skip); codes: [D][M][N] u8 (NULL = skip);
// thr: [D][M][c-1] f32 (NULL = skip).
// onehot: [D][M (c-1)][Kp] bytes, E4M3 1.0 (0x38) where the sample falls in
// bin a >= 1 of the row (v, a), class-sorted with the TcGeom padding (NULL =
// skip); class-1 samples (K range [K0p, Kp)) get the byte class1_byte instead.
cudaError_t launch_discretize(const void* x, int dtype, int N, int M, int c, int D, double range,
                              uint64_t seed, const int* perm, PlaneGeom g, uint32_t* planes,
                              uint8_t* codes, float* thr, uint8_t* onehot, TcGeom tg, cudaStream_t st,
                              uint32_t class1_byte = 0x38, const float* thr_in = nullptr);
// With thr_in [D][M][c-1] (thresholds of launch_batch_thresholds) the column is
// not sorted: the given thresholds bin it.
//
// Batched resamples without a sort per job: launch_presort stores every
// variable's samples in ascending order as 64-bit keys (ordered float bits << 32
// | sample index) [M][N]; launch_multiplicity counts how often each original
// sample occurs in one job's index map (NULL = once each) into m [N];
// launch_batch_thresholds takes the cut positions of the resampled column from
// the sorted keys weighted by m: the thresholds of sort(x[v][idx]) exactly.
// N <= kPresortMaxN.
constexpr int kPresortMaxN = 8192;
cudaError_t launch_presort(const void* x, int dtype, int N, int M, unsigned long long* keys, cudaStream_t st);
cudaError_t launch_multiplicity(const int* idx, int N, int* m, cudaStream_t st);
cudaError_t launch_batch_thresholds(const unsigned long long* keys, const int* m, int N, int M, int c, int D,
                                    double range, uint64_t seed, float* thr, cudaStream_t st);

// Per (disc, variable): class counts of bins 1..c-1 -> cnt1 [D][M][c-1][2] i32,
// SH1 [D][M] i64.  If keys != NULL also folds IG^1 = SH0 - SH1 into keys.
cudaError_t launch_k1(const uint32_t* planes, PlaneGeom g, int M, int c, int D, const long long* tab,
                      int* cnt1, long long* sh1, unsigned long long* keys, cudaStream_t st,
                      EmitTable emit = EmitTable());

// Pair pass over discretisations [d0, d0 + nd).  keys != NULL: fold the two IG
// roles of every pair into keys (k = 2).  sh2/cnt2 != NULL: store the pair
// tables (k = 3): sh2 [nd][M][M] i64, cnt2 [nd][M][M][(c-1)^2][2] i32 (i < m only).
// pairs2 != NULL (c = 2 only): store PairC records [nd][M][M] instead, at
// both [ri][rm] and [rm][ri], with the entropy in fbits fraction bits; ri =
// rank[d][i] (rank [D][M], NULL = identity).
cudaError_t launch_k2(const uint32_t* planes, PlaneGeom g, int M, int c, int D, int d0, int nd,
                      const long long* tab, const int* cnt1, const long long* sh1,
                      unsigned long long* keys, long long* sh2, int* cnt2, PairC* pairs2, int fbits,
                      cudaStream_t st, const int* rank = nullptr, EmitTable emit = EmitTable());

// Triple pass over discretisations [d0, d0 + nd), using the pair tables of the
// same chunk.  Folds the three IG roles of every triple into keys.  items[j] =
// (a, tb << 16 | te): one variable a, a tile tb of b (k3_tile_b(c) variables
// starting at a + 1 + tb * tile) and a tile te of e (k3_tile_e(c) variables).
int k3_tile_b(int c);
int k3_tile_e(int c);
cudaError_t launch_k3_items(const uint32_t* planes, PlaneGeom g, int M, int c, int d0, int nd, const int2* items,
                            int n_items, const long long* tab, const int* cnt1, const long long* sh2,
                            const int* cnt2, unsigned long long* keys, cudaStream_t st,
                            EmitTable emit = EmitTable());

// Triple tables (c = 2) of discretisations [d0, d0 + nd): t3c [nd][C(M,3)]
// packed all-ones counts (class 0 | class 1 << 16) and t3s [nd][C(M,3)] int64
// fixed-point SH of every triple x < y < z at its lexicographic rank
// C(M,3) - 1 - [C(M-1-x,3) + C(M-1-y,2) + (M-1-z)].  items from build_t3_items.
void build_t3_items(int M, std::vector<int2>& items);
size_t t3_entries(int M);
cudaError_t launch_t3(const uint32_t* planes, PlaneGeom g, int M, int d0, int nd, const int2* items, int n_items,
                      const long long* tab, const int* cnt1, const int* cnt2, uint32_t* t3c, long long* t3s,
                      cudaStream_t st);

// Quadruple pass (k = 4, c = 2) over discretisations [d0, d0 + nd), using the
// pair counts cnt2 and the triple tables of the same chunk.  items from
// build_k4_items: (b, c-tile << 16 | e-tile); the kernel loops over a < b.
void build_k4_items(int M, std::vector<int2>& items);
cudaError_t launch_k4(const uint32_t* planes, PlaneGeom g, int M, int d0, int nd, const int2* items, int n_items,
                      const long long* tab, const int* cnt1, const int* cnt2, const uint32_t* t3c,
                      const long long* t3s, unsigned long long* keys, cudaStream_t st, EmitTable emit = EmitTable());
// Quadruple tables (c = 2, C(M,4) <= 2^32) of discretisations [d0, d0 + nd):
// t4c / t4s [nd][C(M,4)] packed all-ones count and SH of every quadruple at
// its lexicographic rank; same items and inputs as launch_k4.
size_t t4_entries(int M);
cudaError_t launch_t4(const uint32_t* planes, PlaneGeom g, int M, int d0, int nd, const int2* items, int n_items,
                      const long long* tab, const int* cnt1, const int* cnt2, const uint32_t* t3c,
                      const long long* t3s, uint32_t* t4c, long long* t4s, cudaStream_t st);
// Quintuple pass (k = 5, c = 2) over discretisations [d0, d0 + nd), using the
// pair counts cnt2, the triple counts t3c and the quadruple tables of the
// same chunk.  items from build_k5_items:
// (b | c << 16, e-tile << 16 | f-tile); keys index d C(M,4) + lexicographic
// rank of the partner set.
void build_k5_items(int M, std::vector<int2>& items);
// keys_stride = 0 and disc_in_index: keys [M], index d C(M,4) + rank;
// keys_stride = M and !disc_in_index: keys [nd][M] of this chunk, index = rank.
cudaError_t launch_k5(const uint32_t* planes, PlaneGeom g, int M, int d0, int nd, const int2* items, int n_items,
                      const long long* tab, const int* cnt1, const int* cnt2, const uint32_t* t3c,
                      const uint32_t* t4c, const long long* t4s, unsigned long long* keys, int keys_stride,
                      bool disc_in_index, cudaStream_t st, EmitTable emit = EmitTable());
// Folds per-discretisation keys [nd][M] of discretisations d0.. into (best [M],
// best_d [M]): a strictly larger IG replaces, so ties keep the lowest d.
cudaError_t launch_k5_merge(const unsigned long long* keys5, int nd, int M, int d0, unsigned long long* best,
                            int* best_d, cudaStream_t st);
// Interesting tuples: gather the occupied slots of the table into recs_key /
// recs_val (npad >= n entries, a power of two), sort them by (variable,
// partners) in one CTA and decode into var [n], tuples [n][k-1] (NULL ok),
// ig [n], disc [n].
cudaError_t launch_emit_collect(EmitTable t, int k, unsigned long long* recs_key, unsigned long long* recs_val,
                                int* counter, int npad, int* var, int* tuples, float* ig, int* disc, int n,
                                cudaStream_t st);

// Two-class k = 3 kernel on the tensor cores (tcgen05 kind::f8f6f4): one-hot
// operands through TMA, counts in TMEM, fused entropy epilogue.  pairs must be
// symmetric ([i][m] and [m][i] both written).  err: device flag set on a
// bounded-wait timeout.
// k = 4, 5 with three or four classes per variable (mdfs_kgen.cu): every voxel
// of every tuple counted from the bit planes, one warp per tuple.  items:
// pairs (a, b) of the two lowest variables (build_kgen_items), one CTA each, for
// discretisations [d0, d0 + nd); keys indexed as the two-class scans index
// them (k = 5: D C(M,4) < 2^32); emit.keys != NULL: also every qualifying role.
bool kgen_supported(int k, int c);
void build_kgen_items(int M, int k, std::vector<int2>& items);
cudaError_t launch_kgen(const uint32_t* planes, PlaneGeom g, int M, int c, int k, int d0, int nd, const int2* items,
                        int n_items, const long long* tab, unsigned long long* keys, EmitTable emit,
                        cudaStream_t st);

TcGeom make_tc_geom(int N0, int N1);
void build_k3tc_items(int M, std::vector<int2>& items);
size_t k3tc_smem_bytes(int N0, int N1);
int k3tc_fraction_bits(int N);
cudaError_t make_onehot_map(CUtensorMap* map, const uint8_t* oh, int rows, int D, int Kp);
// perm [D][M]: new label -> original variable; cnt1s [D][M][2], the one-hot
// rows of `map` and the pair records are in the new labels (see launch_k3tc_order).
// Test hooks of the triple kernel (defaults: off).  wait_ns: limit of every
// bounded mbarrier wait (0 = the library's 1 s); withhold_kb >= 0: the TMA
// producer of CTA 0 never fills the stage of that K block of its running
// count, so the consumers' wait runs out and the call reports MDFS_ETIMEOUT;
// exact: no triple is skipped by the SH3 lower bound.
struct TcTestHooks {
    unsigned long long wait_ns = 0;
    int withhold_kb = -1;
    bool exact = false;  // evaluate every triple exactly (no SH3 bound)
};
// dump != NULL (test hook): also writes the 8-voxel class counts of every
// triple, [D][C(M,3)][8] uint32 n0 | n1 << 16, lexicographic triple rank of the
// original variables, voxel 4 v_lo + 2 v_mid + v_hi.
// b0, b1: the pseudocounts of the two decision classes (they enter a lower
// bound of SH3 that lets the epilogue skip triples that cannot change a key).
cudaError_t launch_k3tc(const CUtensorMap& map, const uint8_t* oh, TcGeom tg, int M, int d0, int nd,
                        const int2* items, int n_items, const long long* tab, int fbits, const int* cnt1s,
                        const int* perm, const PairC* pairs, unsigned long long* keys, int* err, double b0, double b1,
                        cudaStream_t st, uint32_t* dump = nullptr, TcTestHooks hooks = TcTestHooks(),
                        EmitTable emit = EmitTable(), const int* order = nullptr, int* claim = nullptr);
// Claim order of a triple-kernel launch (launch_k3tc's order, a device copy):
// its n_items * nd tiles by descending cost of a model of the epilogue; with
// claim (one device int, zeroed by the launch) the CTAs take tiles from it
// dynamically, without it at a fixed stride.
void build_k3tc_order(int M, const int2* items, int n_items, int nd, std::vector<int>& out);
// Relabelling of the k = 3 tensor path, per discretisation: new labels in
// ascending order of the bin-1 count (ties by index) for M <= 8192, else the
// identity.  perm [D][M] new -> original, rank [D][M] original -> new,
// cnt1s [D][M][2] = cnt1 rows in the new order (c = 2 layout).
cudaError_t launch_k3tc_order(const int* cnt1, int M, int D, int* perm, int* rank, int* cnt1s, cudaStream_t st);
// The k = 3 tensor operand: dst [D][M][Kp] row r of disc d = src row
// perm[d][r] (one-hot rows of launch_discretize), class-1 samples (K range
// [K0p, Kp)) recoded from E4M3 1.0 to 64.0.
cudaError_t launch_k3tc_operand(const uint8_t* src, uint8_t* dst, const int* perm, int M, int D, TcGeom tg,
                                cudaStream_t st);

// k = 2 on the tensor cores for c = 2, 3: the one-hot rows [zdim][M (c-1)][Kp]
// bytes (zdim = jobs x discretisations per job) through TMA, the tiles of
// build_k2tc_items.  One launch scans up to kMaxK2Jobs jobs of the same N (the
// resamples of a batch): work items (job, discretisation, tile), every job's
// entropy tables in shared memory at once.
constexpr int kMaxK2Jobs = 16;
struct K2Job {
    TcGeom tg;                  // class sizes and K geometry of the job
    const long long* tab;       // int64 entropy tables [3][N + 1]
    const int* cnt1;            // [D][M][c-1][2] bin class counts
    const long long* sh1;       // [D][M] SH1
    unsigned long long* keys;   // [M] max keys of the job
    float b0, b1;               // pseudocounts of the two decision classes (the SH2 bound)
};
struct K2Jobs {
    int n;
    K2Job job[kMaxK2Jobs];
};
bool k2tc_supported(int c);
// the class sizes the kernel for c classes per variable can count exactly
bool k2tc_counts_fit(int c, int N0, int N1);
// the one-hot byte of a class-1 sample in that kernel's operand
uint32_t k2tc_class1_byte(int c);
void build_k2tc_items(int M, int c, std::vector<int2>& items);
// dynamic shared memory of a launch with n_jobs jobs of N samples and `stages` pipeline stages
size_t k2tc_smem_bytes(int c, int N, int n_jobs, int stages);
// the most jobs of N samples one launch can hold within smem_limit bytes (0: none)
int k2tc_max_jobs(int c, int N, int stages, size_t smem_limit);
// bound: with three classes, skip the pairs whose SH2 lower bound rules out
// both roles.  stages: 3 or 4.  dstride: discretisations per job in the operand.
// dump != NULL (test hook, one job, 4 stages): also writes the c x c class
// counts of every pair i < m, [D][C(M,2)][c c] uint32 n0 | n1 << 16 at the
// pair's rank in the upper triangle, voxel code_i c + code_m.  emit.keys !=
// NULL (one job, no dump): also inserts every (variable, partner) whose IG
// reaches emit.thr_fx into that interesting-tuple table.
cudaError_t launch_k2tc(const uint8_t* oh, int Kp, int zdim, const K2Jobs& jobs, int M, int c, int d0, int nd,
                        int dstride, const int2* items, int n_items, int fbits, int* err, bool bound, int stages,
                        cudaStream_t st, uint32_t* dump = nullptr, EmitTable emit = EmitTable());
// the c = 3 kernel (mdfs_k2tc3.cu) behind launch_k2tc; its one-hot operand
// carries class1_byte (k2tc_class1_byte) for class-1 samples, and it needs
// class sizes N0, N1 below 4096 (k2tc_counts_fit)
void build_k2tc3_items(int M, std::vector<int2>& items);
bool k2tc3_counts_fit(int N0, int N1);
uint32_t k2tc3_class1_byte();
size_t k2tc3_smem_bytes(int N, int n_jobs, int stages);
cudaError_t launch_k2tc3(const uint8_t* oh, int Kp, int zdim, const K2Jobs& jobs, int M, int d0, int nd, int dstride,
                         const int2* items, int n_items, int fbits, int* err, bool bound, int stages, cudaStream_t st,
                         uint32_t* dump, EmitTable emit);
// byte tensor map with the 128-byte swizzle (box[0] = 128 bytes), strides in bytes
cudaError_t make_tiled_map_u8(CUtensorMap* map, const void* base, int rank, const cuuint64_t* dims,
                              const cuuint64_t* strides, const cuuint32_t* box);

// Contrast rows M .. M + n_contrast - 1 of x_ext (dtype 0 f32, 1 i8); rows
// 0 .. M-1 are not written.  src [n_contrast] or NULL.
cudaError_t launch_contrast(const void* x, int dtype, int N, int M, int n_contrast, uint64_t seed, void* x_ext,
                            int* src, cudaStream_t st);
// p-value adjustment (MDFS_ADJUST_*), one CTA; scratch of p_adjust_scratch_bytes(m);
// relevant [m] (adjusted < level) or NULL.
size_t p_adjust_scratch_bytes(int m);
cudaError_t launch_p_adjust(const double* p, int m, int method, double level, void* scratch, double* adjusted,
                            uint8_t* relevant, cudaStream_t st);

// keys [M] -> ig [M] f32, tuples [M][k-1] i32 (NULL ok), disc [M] i32 (NULL ok).
// kdisc != NULL (k = 5 with per-discretisation keys): the keys index the
// partner rank only and kdisc [M] holds the discretisation.
cudaError_t launch_finalize(const unsigned long long* keys, int M, int k, float* ig, int* tuples,
                            int* disc, cudaStream_t st, const int* kdisc = nullptr);

// chi^2 / extreme-value fit in FP64, three launches on one stream:
//   cdf: p_values[i] = F_df(2 ig[i]) (one thread per variable);
//   fit: res[0] = IG_lim, res[1] = T, res[2] = number of variables in the fit
//        (one CTA; reads the CDF values left in p_values);
//   p:   p_values[i] = 1 - F^T in place (skipped when the fit failed).
cudaError_t launch_ig_lim_cdf(const float* ig, int M, int df, double* p_values, cudaStream_t st);
cudaError_t launch_ig_lim_fit(const double* p_values, int M, int df, const uint8_t* mask, double alpha, double* res,
                              cudaStream_t st);
cudaError_t launch_ig_lim_p(int M, const double* res, double* p_values, cudaStream_t st);

// Raises (never lowers) a kernel's dynamic shared-memory limit on the current
// device to at least `bytes`.  Thread-safe: concurrent calls on other streams
// can only see the limit grow, so a launch sized below it stays valid.
cudaError_t ensure_dynamic_smem(const void* kernel, size_t bytes);

// Sets the thread-local message that mdfs_last_error() returns.
void record_error(const char* msg);

// Drops the cached device addresses of the allocation-free entry point's
// scratch array (mdfs_release; they are looked up again on the next call).
void noalloc_forget_devices();

}  // namespace mdfs
