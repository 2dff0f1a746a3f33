// k = 2 scan on the 5th-generation tensor cores (tcgen05, kind::f8f6f4) for
// c = 2 or 3 classes per variable.  Voxel counters of section "Algorithm and
// implementation"; the two IG roles of Eq. 1 with |S| = 1.
//
// Every (variable, bin >= 1) is one E4M3 one-hot row over the class-sorted
// samples (rows v P + p, P = c - 1).  The pair counts of the voxels with both
// coordinates >= 1 are the symmetric GEMM C = OH OH^T; class-0 and class-1
// samples occupy separate K ranges and accumulate into two TMEM accumulators.
// Tiles of 128 x 128 rows/columns on and above the diagonal; no operand needs
// masking.  Counts are exact (0/1 products, FP32 sums below 2^24).
//
// Persistent kernel, one CTA per SM, 640 threads:
//   warp 0       TMA producer (A rows, B rows; 128B swizzle),
//   warp 1       TMEM owner and MMA issuer,
//   warps 4-19   epilogue: tcgen05.ld, c x c tables per class by
//                inclusion-exclusion, SH2 from int32 fixed-point tables in
//                shared memory, IG(i | m) = SH1(m) - SH2 and IG(m | i), keys.
// With c = 3 a variable spans two adjacent rows (TMEM lanes); the two lanes
// exchange their counts with shuffles and split the 27 table lookups.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "mdfs_device.cuh"
#include "mdfs_internal.cuh"
#include "mdfs_tc.cuh"

namespace mdfs {

namespace {

constexpr int kTile = 128;
constexpr int kBK = 128;
constexpr uint32_t kTileBytes = kTile * kBK;
constexpr uint32_t kAccCols = 2 * kTile;
constexpr uint32_t kTmemCols = 2 * kAccCols;
constexpr int kThreads = 640;
constexpr int kEpiWarp0 = 4, kEpiThreads = 512;
constexpr int kColsPerWarp = 32;
constexpr int kRegsLaunch = 96, kRegsProducer = 32, kRegsEpilogue = 112;
static_assert(128 * kRegsProducer + kEpiThreads * kRegsEpilogue == kThreads * kRegsLaunch,
              "register split must add up to the launch allocation");
// the entropy tables follow the S pipeline stages (A and B tiles)
constexpr size_t tab_offset(int S) { return 2 * (size_t)S * kTileBytes; }
// int32 entries per job in shared memory: T0 (N0 + 1), T1 (N1 + 1), TB (N + 1), rounded to 16 bytes
__host__ __device__ constexpr int tab_stride(int N) { return (2 * N + 3 + 3) & ~3; }

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) { return a > b ? a : b; }

__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
    const unsigned long long t0 = tc::global_ns();
    while (!tc::mbar_try_wait(bar, parity))
        if (tc::global_ns() - t0 > tc::kWaitLimitNs) return;
}

__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long k) {
    const uint32_t hi = (uint32_t)(k >> 32);
    const uint32_t hmax = __reduce_max_sync(0xffffffffu, hi);
    const uint32_t lo = (hi == hmax) ? (uint32_t)k : 0u;
    const uint32_t lmax = __reduce_max_sync(0xffffffffu, lo);
    return ((unsigned long long)hmax << 32) | lmax;
}

__device__ __forceinline__ int tab32(const int* t, int n, int nmax) { return t[min((unsigned)n, (unsigned)nmax)]; }

// Bound that lets the epilogue skip the table lookups of most pairs (three
// classes per variable).  Each voxel's term of SH is E(m0, m1) = f(m0 + m1) -
// f(m0) - f(m1) = (m0 + m1) H(m0 / (m0 + m1)) with the smoothed class counts
// m_d = n_d + beta_d, and H(p) >= 4 ln 2 p (1 - p) gives
//     SH2 >= 4 ln 2 sum_v m0_v m1_v / (m0_v + m1_v) = 4 ln 2 LB.
// IG(i | m) = SH1(m) - SH2 can raise i's key only if SH2 <= SH1(m) - IG_key(i),
// and likewise for m, so a pair with LB above both limits (in units of 4 ln 2
// nats, with the margins kBoundRel |hi| + kBoundAbs for float rounding) cannot
// change any result and skips its 27 lookups.
constexpr float kBoundRel = 1.0f / 4096.0f, kBoundAbs = 0.05f;
constexpr float kInv4Ln2 = 0.36067376022224085f;            // 1 / (4 ln 2)
constexpr float kFx32ToCount = 2.3283064365386963e-10f * kInv4Ln2;  // 2^-32 / (4 ln 2)

// The IG of a key in units of 4 ln 2 nats; -inf for a key not yet set.
__device__ __forceinline__ float key_ig_count(unsigned long long key) {
    return key ? order_bits_float((uint32_t)(key >> 32)) * kInv4Ln2 : -INFINITY;
}

// a / b + c / d as one fraction num / den (b, d > 0)
__device__ __forceinline__ void frac_add(float a, float b, float c, float d, float& num, float& den) {
    num = fmaf(a, d, c * b);
    den = b * d;
}

// Integers below 2^22 in magnitude between int and float, through the bits of
// 1.5 2^23 + v (exact; no conversion instruction).
__device__ __forceinline__ float i2f_exact(int v) { return __int_as_float(0x4B400000 + v) - 12582912.0f; }
__device__ __forceinline__ int f2i_exact(float f) { return __float_as_int(f + 12582912.0f) - 0x4B400000; }

// c x c voxel counts of one channel from the all->=1 block X (P x P) and the
// marginals of the row variable (ni[0..P-1]) and column variable (nm[..]);
// integer-valued floats (exact below 2^24).
template <int P, typename V>
__device__ __forceinline__ void complete2(const V (&X)[P][P], const V (&ni)[P], const V (&nm)[P], V ntot,
                                          V (&T)[P + 1][P + 1]) {
    V all = 0;
#pragma unroll
    for (int a = 0; a < P; ++a)
#pragma unroll
        for (int b = 0; b < P; ++b) T[a + 1][b + 1] = X[a][b];
#pragma unroll
    for (int a = 0; a < P; ++a) {
        V s = 0;
#pragma unroll
        for (int b = 0; b < P; ++b) s += X[a][b];
        T[a + 1][0] = ni[a] - s;
        all += ni[a];
    }
#pragma unroll
    for (int b = 0; b < P; ++b) {
        V s = 0;
#pragma unroll
        for (int a = 0; a < P; ++a) s += X[a][b];
        T[0][b + 1] = nm[b] - s;
        all += T[0][b + 1];
    }
    T[0][0] = ntot - all;
}

}  // namespace

// Work items of a launch: (job, discretisation, tile) for jobs.n jobs of the
// same N (a batch's resamples; one job for a plain scan), discretisations
// d0 .. d0 + nd - 1, and the n_items symmetric tiles; job j's operand rows are
// at z = j dstride + d of the tensor map.  Every job's entropy tables sit in
// shared memory at once.  S: pipeline stages.  kDump: also write the c x c
// class counts of every pair of job 0 to `dump` (test hook; the scan itself is
// unchanged).
template <int P, int S, bool kDump>
__global__ void __launch_bounds__(kThreads, 1)
    k2tc_kernel(const __grid_constant__ CUtensorMap map_oh, const __grid_constant__ K2Jobs jobs, int M, int d0,
                int nd, int dstride, const int2* __restrict__ items, int n_items, int fbits, int* __restrict__ err,
                int prune_on, uint32_t* __restrict__ dump) {
    constexpr int C = P + 1;
    // the bound pays for itself with three classes (27 lookups per pair)
    const bool use_bound = P == 2 && !kDump && prune_on;
    constexpr int VT = kTile / P;  // variables per tile
    extern __shared__ uint8_t dsmem_raw[];
    __shared__ uint64_t bar_full[S], bar_empty[S];
    __shared__ uint64_t bar_tfull[2], bar_tempty[2], bar_drain;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t* base = dsmem_raw + ((1024 - (tc::smem_u32(dsmem_raw) & 1023)) & 1023);
    uint8_t* sA = base;
    uint8_t* sB = base + S * kTileBytes;
    const int N = jobs.job[0].tg.N0 + jobs.job[0].tg.N1, np1 = N + 1;  // the same N for every job
    const int tstride = tab_stride(N);
    int* sTab = reinterpret_cast<int*>(base + tab_offset(S));
    volatile int* abort = &s_abort;

    uint32_t dyn_bytes;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_bytes));
    const bool fits = jobs.n >= 1 && jobs.n <= kMaxK2Jobs &&
                      (size_t)(base - dsmem_raw) + tab_offset(S) + (size_t)jobs.n * tstride * sizeof(int) <= dyn_bytes;

    if (tid == 0) {
        s_abort = (*(volatile int*)err ? 1 : 0) | (fits ? 0 : 2);
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&bar_full[s], 1);
            tc::mbar_init(&bar_empty[s], 1);
        }
        for (int j = 0; j < 2; ++j) {
            tc::mbar_init(&bar_tfull[j], 1);
            tc::mbar_init(&bar_tempty[j], kEpiThreads);
        }
        tc::mbar_init(&bar_drain, 1);
        tc::mbar_fence_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(&s_tmem, kTmemCols);
        tc::tmem_relinquish();
    }
    if (fits) {
        for (int j = 0; j < jobs.n; ++j) {
            const long long* tab = jobs.job[j].tab;
            const int N0j = jobs.job[j].tg.N0, N1j = jobs.job[j].tg.N1;
            int* t0 = sTab + j * tstride;
            for (int i = tid; i <= N0j; i += kThreads) t0[i] = fx_narrow(tab[i], fbits);
            for (int i = tid; i <= N1j; i += kThreads) t0[N0j + 1 + i] = fx_narrow(tab[np1 + i], fbits);
            for (int i = tid; i <= N; i += kThreads) t0[N0j + N1j + 2 + i] = fx_narrow(tab[2 * np1 + i], fbits);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = s_tmem;
    const int per_job = n_items * nd;
    const int n_tiles = per_job * jobs.n;

    if (warp < kEpiWarp0) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsProducer));
        if (warp == 0) {
            // ------------------------------ TMA producer --------------------------
            if (lane == 0 && !*abort) {
                uint32_t g = 0;
                int pend_mask = 0;
                uint32_t pend_use[S] = {};
                for (int t = blockIdx.x; t < n_tiles && !*abort; t += gridDim.x) {
                    const int job = t / per_job, r = t - job * per_job, dl = r / n_items;
                    const int2 item = items[r - dl * n_items];
                    const int z = job * dstride + d0 + dl;
                    const int nkb = jobs.job[job].tg.nkb;
                    const int r0 = item.x * kTile, c0 = item.y * kTile;
                    bool ok = true;
                    for (int kb = 0; kb < nkb; ++kb, ++g) {
                        const int s = (int)(g % S);
                        const uint32_t use = g / S;
                        if (use > 0 && !tc::mbar_wait(&bar_empty[s], (use - 1) & 1, abort)) {
                            ok = false;
                            break;
                        }
                        tc::mbar_arrive_expect_tx(&bar_full[s], 2 * kTileBytes);
                        tc::tma_load_3d(sA + s * kTileBytes, &map_oh, &bar_full[s], kb * kBK, r0, z);
                        tc::tma_load_3d(sB + s * kTileBytes, &map_oh, &bar_full[s], kb * kBK, c0, z);
                        pend_mask |= 1 << s;
                        pend_use[s] = use;
                    }
                    if (!ok) break;
                }
                for (int s = 0; s < S; ++s)
                    if (pend_mask & (1 << s)) mbar_drain(&bar_full[s], pend_use[s] & 1);
            }
        } else if (warp == 1) {
            // ------------------------------ MMA issuer ----------------------------
            if (lane == 0 && !*abort) {
                const uint32_t idesc = tc::idesc_e4m3_f32(kTile, kTile);
                uint32_t g = 0;
                int i = 0;
                bool issued = false;
                for (int t = blockIdx.x; t < n_tiles && !*abort; t += gridDim.x, ++i) {
                    const int buf = i & 1;
                    const uint32_t tuse = (uint32_t)(i >> 1);
                    const TcGeom& tg = jobs.job[t / per_job].tg;
                    const int nkb = tg.nkb;
                    if (tuse > 0 && !tc::mbar_wait(&bar_tempty[buf], (tuse - 1) & 1, abort)) break;
                    tc::tc_fence_after();
                    const uint32_t dbase = tmem + (uint32_t)buf * kAccCols;
                    bool ok = true;
                    for (int kb = 0; kb < nkb; ++kb, ++g) {
                        const int s = (int)(g % S);
                        const uint32_t use = g / S;
                        if (!tc::mbar_wait(&bar_full[s], use & 1, abort)) {
                            ok = false;
                            break;
                        }
                        tc::tc_fence_after();
                        const uint32_t d_tmem = dbase + (kb >= tg.nkb0 ? (uint32_t)kTile : 0u);
                        const uint32_t a_addr = tc::smem_u32(sA + s * kTileBytes);
                        const uint32_t b_addr = tc::smem_u32(sB + s * kTileBytes);
#pragma unroll
                        for (int kk = 0; kk < kBK / 32; ++kk) {
                            const uint32_t acc = (kb != 0 && kb != tg.nkb0) || kk > 0;
                            tc::mma_f8(d_tmem, tc::sw128_kmajor_desc(a_addr + 32 * kk),
                                       tc::sw128_kmajor_desc(b_addr + 32 * kk), idesc, acc);
                        }
                        tc::mma_commit(&bar_empty[s]);
                        issued = true;
                    }
                    if (!ok) break;
                    tc::mma_commit(&bar_tfull[buf]);
                }
                if (issued) {
                    tc::mma_commit(&bar_drain);
                    mbar_drain(&bar_drain, 0);
                }
            }
        }
        // warps 2-3 have no role in this kernel
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsEpilogue));
        // ------------------------------ epilogue ----------------------------------
        const int ew = warp - kEpiWarp0;
        const int q = warp & 3, h = ew >> 2;  // TMEM lane quarter, column quarter
        const int row = 32 * q + lane;
        const int alpha = row % P;            // bin index (0-based) of this row
        const float inv_scale = __int_as_float((127 - fbits) << 23);
        int i = 0;
        for (int t = blockIdx.x; t < n_tiles && !*abort; t += gridDim.x, ++i) {
            const int buf = i & 1;
            const uint32_t tuse = (uint32_t)(i >> 1);
            const int job = t / per_job, r = t - job * per_job, dl = r / n_items;
            const int2 item = items[r - dl * n_items];
            const int d = d0 + dl;
            const K2Job& J = jobs.job[job];
            const int N0 = J.tg.N0, N1 = J.tg.N1;
            const int* sT0 = sTab + job * tstride;
            const int* sT1 = sT0 + (N0 + 1);
            const int* sTB = sT1 + (N1 + 1);
            unsigned long long* keys = J.keys;
            const float beta0 = J.b0, beta1 = J.b1;
            const int vi = item.x * VT + row / P;       // row variable
            const int vm0 = item.y * VT + (kColsPerWarp / P) * h;  // first column variable of this warp
            const bool diag = item.x == item.y;
            const int* c1 = J.cnt1 + (size_t)d * M * P * 2;
            const long long* s1 = J.sh1 + (size_t)d * M;
            const bool irow = vi < M;
            // row-variable context (class counts of bins 1..P as exact floats)
            float ni0[P], ni1[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                ni0[p] = i2f_exact(irow ? c1[((size_t)vi * P + p) * 2] : 0);
                ni1[p] = i2f_exact(irow ? c1[((size_t)vi * P + p) * 2 + 1] : 0);
            }
            const int shi = irow ? fx_narrow(s1[vi], fbits) : 0;
            // SH1(i) and the key of i in units of 4 ln 2 nats (the bound's units)
            const float shi_c = irow ? (float)s1[vi] * kFx32ToCount : 0.0f;
            const float keyi_c = irow ? key_ig_count(__ldcg(keys + vi)) : 0.0f;
            const uint32_t dM = (uint32_t)d * (uint32_t)M;

            if (!__all_sync(0xffffffffu, tc::mbar_wait(&bar_tfull[buf], tuse & 1, abort))) break;  // warp-uniform
            tc::tc_fence_after();
            unsigned long long ki = 0ull;
            const bool warp_rows = (item.x * VT + (32 * q) / P) < M;
            if (warp_rows && vm0 < M) {
                const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)buf * kAccCols +
                                       (uint32_t)(kColsPerWarp * h);
                uint32_t r0[kColsPerWarp], r1[kColsPerWarp];
                tc::tmem_ld16(taddr, *reinterpret_cast<uint32_t(*)[16]>(&r0[0]));
                tc::tmem_ld16(taddr + 16, *reinterpret_cast<uint32_t(*)[16]>(&r0[16]));
                tc::tmem_ld16(taddr + kTile, *reinterpret_cast<uint32_t(*)[16]>(&r1[0]));
                tc::tmem_ld16(taddr + kTile + 16, *reinterpret_cast<uint32_t(*)[16]>(&r1[16]));
                tc::tmem_ld_wait();
                // column-variable context: lane j holds column vm0 + j (j < columns of
                // the warp), handed to every lane of the warp by shuffles per column
                constexpr int kCols = kColsPerWarp / P;
                const int vcol = vm0 + lane % kCols;
                const bool colok = vcol < M;
                float cn0[P], cn1[P];
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    cn0[p] = i2f_exact(colok ? c1[((size_t)vcol * P + p) * 2] : 0);
                    cn1[p] = i2f_exact(colok ? c1[((size_t)vcol * P + p) * 2 + 1] : 0);
                }
                const int csh = colok ? fx_narrow(s1[vcol], fbits) : 0;
                // SH1(m) and the key of m in units of 4 ln 2 nats (the bound's units)
                const float cshc = (use_bound && colok) ? (float)s1[vcol] * kFx32ToCount : 0.0f;
                const float ckey = (use_bound && colok) ? key_ig_count(__ldcg(keys + vcol)) : 0.0f;
                const float fN0 = i2f_exact(N0), fN1 = i2f_exact(N1);
#pragma unroll
                for (int jm = 0; jm < kCols; ++jm) {
                    const int vm = vm0 + jm;
                    const bool ok = irow && vm < M && (!diag || vi < vm);
                    // counts of the all->=1 block, both classes, exact in FP32: X?[alpha][beta]
                    // here, the other row(s) of the block from the neighbouring lane
                    float X0[P][P], X1[P][P];
#pragma unroll
                    for (int b = 0; b < P; ++b) {
                        const float v0 = __uint_as_float(r0[jm * P + b]);
                        const float v1 = __uint_as_float(r1[jm * P + b]);
                        if (P == 1) {
                            X0[0][b] = v0;
                            X1[0][b] = v1;
                        } else {
                            const float o0 = __shfl_xor_sync(0xffffffffu, v0, 1);
                            const float o1 = __shfl_xor_sync(0xffffffffu, v1, 1);
                            X0[0][b] = alpha ? o0 : v0;
                            X0[P - 1][b] = alpha ? v0 : o0;
                            X1[0][b] = alpha ? o1 : v1;
                            X1[P - 1][b] = alpha ? v1 : o1;
                        }
                    }
                    float nm0[P], nm1[P];
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        nm0[p] = __shfl_sync(0xffffffffu, cn0[p], jm);
                        nm1[p] = __shfl_sync(0xffffffffu, cn1[p], jm);
                    }
                    float T0v[C][C], T1v[C][C];
                    complete2<P>(X0, ni0, nm0, fN0, T0v);
                    complete2<P>(X1, ni1, nm1, fN1, T1v);
                    // pairs whose SH2 lower bound rules out both roles skip the lookups
                    bool need = ok;
                    if (use_bound) {
                        const float shm_c = __shfl_sync(0xffffffffu, cshc, jm);
                        const float keym_c = __shfl_sync(0xffffffffu, ckey, jm);
                        // this lane's voxels: alpha 0 takes 0..4, alpha 1 takes 5..8 (row-major)
                        float pn[5], ps[5];
#pragma unroll
                        for (int u = 0; u < 5; ++u) {
                            const int va = u, vb = u + 5;
                            const float n0 = alpha ? (vb < C * C ? T0v[vb / C][vb % C] : 0.0f) : T0v[va / C][va % C];
                            const float n1 = alpha ? (vb < C * C ? T1v[vb / C][vb % C] : 0.0f) : T1v[va / C][va % C];
                            const float m0 = n0 + beta0, m1 = n1 + beta1;
                            const bool used = !alpha || vb < C * C;
                            pn[u] = used ? m0 * m1 : 0.0f;  // an unused slot adds 0 / 1
                            ps[u] = used ? m0 + m1 : 1.0f;
                        }
                        float n01, d01, n23, d23, n03, d03, nl, dl;
                        frac_add(pn[0], ps[0], pn[1], ps[1], n01, d01);
                        frac_add(pn[2], ps[2], pn[3], ps[3], n23, d23);
                        frac_add(n01, d01, n23, d23, n03, d03);
                        frac_add(n03, d03, pn[4], ps[4], nl, dl);
                        // both lanes of the variable combine the two halves in the same order
                        const float on = __shfl_xor_sync(0xffffffffu, nl, 1), od = __shfl_xor_sync(0xffffffffu, dl, 1);
                        const float na = alpha ? on : nl, da = alpha ? od : dl, nb = alpha ? nl : on,
                                    db = alpha ? dl : od;
                        const float num = fmaf(na, db, nb * da), den = da * db;
                        // largest SH2 (units of 4 ln 2 nats) that lets one role reach its key
                        const float hi = fmaxf(shm_c - keyi_c, shi_c - keym_c);
                        const float lim = fmaf(fabsf(hi), kBoundRel, hi + kBoundAbs);
                        need = ok && num <= lim * den;
                    }
                    if (!__any_sync(0xffffffffu, need)) continue;
                    // exact path: integer counts and the table lookups
                    int T0i[C][C], T1i[C][C], TTi[C][C];
#pragma unroll
                    for (int a = 0; a < C; ++a)
#pragma unroll
                        for (int b = 0; b < C; ++b) {
                            T0i[a][b] = f2i_exact(T0v[a][b]);
                            T1i[a][b] = f2i_exact(T1v[a][b]);
                            TTi[a][b] = T0i[a][b] + T1i[a][b];
                        }
                    if constexpr (kDump) {
                        if (ok && (P == 1 || alpha == 0)) {
                            const unsigned long long np = (unsigned long long)M * (M - 1) / 2;
                            const unsigned long long rank =
                                (unsigned long long)vi * (2ull * M - vi - 1) / 2 + (unsigned long long)(vm - vi - 1);
                            uint32_t* o = dump + ((unsigned long long)d * np + rank) * (C * C);
#pragma unroll
                            for (int a = 0; a < C; ++a)
#pragma unroll
                                for (int b = 0; b < C; ++b)
                                    o[a * C + b] = (uint32_t)T0i[a][b] | ((uint32_t)T1i[a][b] << 16);
                        }
                    }
                    int part = 0;
                    if (P == 1) {
#pragma unroll
                        for (int a = 0; a < C; ++a)
#pragma unroll
                            for (int b = 0; b < C; ++b)
                                part += tab32(sTB, TTi[a][b], N) - tab32(sT0, T0i[a][b], N0) -
                                        tab32(sT1, T1i[a][b], N1);
                    } else {
                        // the two lanes of a variable split the lookups without diverging:
                        // lane alpha = 0 takes class 0 and total voxels 0..4, alpha = 1
                        // takes class 1 and total voxels 5..8
                        const int* tcls = alpha ? sT1 : sT0;
                        const int ncls = alpha ? N1 : N0;
#pragma unroll
                        for (int a = 0; a < C; ++a)
#pragma unroll
                            for (int b = 0; b < C; ++b) part -= tab32(tcls, alpha ? T1i[a][b] : T0i[a][b], ncls);
#pragma unroll
                        for (int u = 0; u < 5; ++u) {
                            const int lo = TTi[u / C][u % C];
                            const int hi = u + 5 < C * C ? TTi[(u + 5) / C][(u + 5) % C] : 0;
                            const int v = tab32(sTB, alpha ? hi : lo, N);
                            part += (alpha && u + 5 >= C * C) ? 0 : v;
                        }
                        part += __shfl_xor_sync(0xffffffffu, part, 1);
                    }
                    const int sh2 = part;
                    const int shm = __shfl_sync(0xffffffffu, csh, jm);
                    unsigned long long k_m = 0ull;
                    if (ok) {
                        if (P == 1 || alpha == 0) {
                            // IG(i | m) = SH1(m) - SH2
                            const float g = (float)(shm - sh2) * inv_scale;
                            ki = umax64(ki, pack_key(g, dM + (uint32_t)vm));
                        }
                        if (P == 1 || alpha == 1) {
                            // IG(m | i) = SH1(i) - SH2
                            const float g = (float)(shi - sh2) * inv_scale;
                            k_m = pack_key(g, dM + (uint32_t)vi);
                        }
                    }
                    const unsigned long long mk = warp_max_key(k_m);
                    if (lane == 0 && mk) atomicMax(keys + vm, mk);
                }
            }
            tc::tc_fence_before();
            tc::mbar_arrive(&bar_tempty[buf]);
            if (ki) atomicMax(keys + vi, ki);
        }
    }

    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, kTmemCols);
    if (tid == 0 && *abort) atomicOr(err, *abort);
}

void build_k2tc_items(int M, int c, std::vector<int2>& items) {
    const int P = c - 1;
    const int nt = (M * P + kTile - 1) / kTile;
    items.clear();
    for (int it = 0; it < nt; ++it)
        for (int mt = it; mt < nt; ++mt) items.push_back(make_int2(it, mt));
}

size_t k2tc_smem_bytes(int N, int n_jobs, int stages) {
    return tab_offset(stages) + (size_t)n_jobs * tab_stride(N) * sizeof(int) + 1024;
}

int k2tc_max_jobs(int N, int stages, size_t smem_limit) {
    const size_t base = tab_offset(stages) + 1024, per = (size_t)tab_stride(N) * sizeof(int);
    if (smem_limit < base + per) return 0;
    return (int)std::min<size_t>((smem_limit - base) / per, (size_t)kMaxK2Jobs);
}

bool k2tc_supported(int c) { return c == 2 || c == 3; }

cudaError_t launch_k2tc(const CUtensorMap& map, const K2Jobs& jobs, int M, int c, int d0, int nd, int dstride,
                        const int2* items, int n_items, int fbits, int* err, bool bound, int stages, cudaStream_t st,
                        uint32_t* dump) {
    if (n_items == 0 || jobs.n == 0) return cudaSuccess;
    if (c != 2 && c != 3) return cudaErrorInvalidValue;
    if (jobs.n < 1 || jobs.n > kMaxK2Jobs || (stages != 3 && stages != 4) || (dump && (jobs.n != 1 || stages != 4)))
        return cudaErrorInvalidValue;
    const int N = jobs.job[0].tg.N0 + jobs.job[0].tg.N1;
    for (int j = 0; j < jobs.n; ++j) {
        if (jobs.job[j].tg.N0 + jobs.job[j].tg.N1 != N) return cudaErrorInvalidValue;
        // the bound needs pseudocounts that keep its fraction away from 0 and infinity
        if (!(jobs.job[j].b0 >= 1e-3f && jobs.job[j].b1 >= 1e-3f)) bound = false;
    }
    const size_t smem = k2tc_smem_bytes(N, jobs.n, stages);
    const void* fn = nullptr;
    if (dump)
        fn = c == 2 ? (const void*)k2tc_kernel<1, 4, true> : (const void*)k2tc_kernel<2, 4, true>;
    else if (stages == 4)
        fn = c == 2 ? (const void*)k2tc_kernel<1, 4, false> : (const void*)k2tc_kernel<2, 4, false>;
    else
        fn = c == 2 ? (const void*)k2tc_kernel<1, 3, false> : (const void*)k2tc_kernel<2, 3, false>;
    cudaError_t e = ensure_dynamic_smem(fn, smem);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
    if (fa.numRegs != kRegsLaunch) return cudaErrorInvalidConfiguration;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const long long n_tiles = (long long)n_items * nd * jobs.n;
    if (n_tiles >= (1ll << 31)) return cudaErrorInvalidValue;
    const int grid = (int)std::min<long long>(n_tiles, (long long)sms);
    const int prune_on = bound ? 1 : 0;
    auto launch = [&](auto kern) {
        kern<<<grid, kThreads, smem, st>>>(map, jobs, M, d0, nd, dstride, items, n_items, fbits, err, prune_on, dump);
    };
    if (dump) {
        if (c == 2) launch(k2tc_kernel<1, 4, true>);
        else launch(k2tc_kernel<2, 4, true>);
    } else if (stages == 4) {
        if (c == 2) launch(k2tc_kernel<1, 4, false>);
        else launch(k2tc_kernel<2, 4, false>);
    } else {
        if (c == 2) launch(k2tc_kernel<1, 3, false>);
        else launch(k2tc_kernel<2, 3, false>);
    }
    return cudaGetLastError();
}

}  // namespace mdfs
