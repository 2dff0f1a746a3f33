// k = 2 scan on the tensor cores for c = 3 classes per variable (two one-hot
// bins per variable, P = 2).  Voxel counters of section "Algorithm and
// implementation"; the two IG roles of Eq. 1 with |S| = 1.
//
// One (variable, bin >= 1) is one one-hot row over the class-sorted samples,
// rows v P + p of the operand, with E4M3 1.0 for a class-0 sample and 64.0 for
// a class-1 sample in the bin.  A product of two rows is 1 for a class-0 sample
// in both bins and 4096 for a class-1 sample, so one FP32 accumulator holds
// n0 + 4096 n1; with n0, n1 < 4096 every partial sum is an integer below 2^24
// and both class counts are exact.
//
// A tile pairs 128 row variables with 64 column variables.  The A operand holds
// the 128 row variables twice, once per bin (a 4-D tensor map selects every
// second row), and B the 128 rows of the column variables, so two 128 x 128
// accumulators (one per row bin) give every thread, which owns one row
// variable (one TMEM lane), the whole 2 x 2 block of counts with both bins >= 1
// for each of its column variables.  A thread splits the classes, completes
// the 3 x 3 table of a pair by inclusion-exclusion and evaluates the SH2 lower
// bound with no exchange between lanes.  The few pairs that the bound cannot
// rule out go to a per-warp queue in shared memory; a full queue is evaluated
// with one pair per lane (27 table lookups each), so the lookups run on full
// warps whichever lanes produced the pairs.
//
// Persistent kernel, one CTA per SM, 640 threads, 3 pipeline stages:
//   warp 0       TMA producer (two A tiles and one B tile per K block),
//   warp 1       TMEM owner and MMA issuer (2 row bins x 128 columns x 2
//                buffers = all 512 columns),
//   warps 4-19   epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31 and
//                the columns of 16 of the 64 column variables.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "mdfs_device.cuh"
#include "mdfs_internal.cuh"
#include "mdfs_tc.cuh"

namespace mdfs {

namespace {

constexpr int kBK = 128;                                  // K bytes (samples) per block
constexpr int kRowVars = 128;                             // row variables per tile
constexpr int kColVars = 64;                              // column variables per tile
constexpr int kBRows = 2 * kColVars;                      // B rows: (column variable, bin)
constexpr uint32_t kABytes = kRowVars * kBK;              // one bin's A tile
constexpr uint32_t kBBytes = kBRows * kBK;
constexpr uint32_t kStageBytes = 2 * kABytes + kBBytes;   // 48 KB, a multiple of 1024
constexpr uint32_t kAccCols = kBRows;                     // 128 columns per accumulator
constexpr uint32_t kBufCols = 2 * kAccCols;               // one accumulator per row bin
constexpr uint32_t kTmemCols = 2 * kBufCols;              // double buffer: 512
constexpr int kThreads = 640;
constexpr int kEpiWarp0 = 4, kEpiWarps = 16, kEpiThreads = 32 * kEpiWarps;
constexpr int kColsPerWarp = kColVars / 4;                // column variables per epilogue warp
constexpr int kColsPerPass = 8;                           // column variables per TMEM read
constexpr int kRegsLaunch = 96, kRegsProducer = 32, kRegsEpilogue = 112;
static_assert(128 * kRegsProducer + kEpiThreads * kRegsEpilogue == kThreads * kRegsLaunch,
              "register split must add up to the launch allocation");
constexpr int kStages = 3;
// column-variable context per epilogue warp: 2 float4 per column variable
constexpr uint32_t kCtxBytes = kEpiWarps * kColsPerWarp * 32;
// pair queue per epilogue warp: kQueue records of the 9 voxels' smoothed
// class counts (two float arrays, structure of arrays) and (vi, vm, SH1(i), SH1(m))
constexpr int kQueue = 16;
constexpr uint32_t kQueueWarpBytes = kQueue * (9 * 8 + 16);
constexpr uint32_t kQueueBytes = kEpiWarps * kQueueWarpBytes;
__host__ __device__ constexpr size_t ctx_offset() { return (size_t)kStages * kStageBytes; }
__host__ __device__ constexpr size_t queue_offset() { return ctx_offset() + kCtxBytes; }
__host__ __device__ constexpr size_t tab_offset3() { return queue_offset() + kQueueBytes; }
// int32 entries per job: T0 (N0 + 1), T1 (N1 + 1), TB (N + 1), rounded to 16 bytes
__host__ __device__ constexpr int tab_stride3(int N) { return (2 * N + 3 + 3) & ~3; }

// SH2 lower bound (as in the two-class-per-variable kernel): each voxel's term
// of SH is (m0 + m1) H(m0 / (m0 + m1)) with the smoothed class counts m = n +
// beta, and H(p) >= 4 ln 2 p (1 - p), so SH2 >= 4 ln 2 sum_v m0 m1 / (m0 +
// m1).  A pair whose sum exceeds, with margins kBoundRel |hi| + kBoundAbs for
// float rounding, both roles' limits SH1(partner) - IG_key (units of 4 ln 2
// nats) cannot change a key and skips its lookups.
constexpr float kBoundRel = 1.0f / 4096.0f, kBoundAbs = 0.05f;
constexpr float kInv4Ln2 = 0.36067376022224085f;                    // 1 / (4 ln 2)
constexpr float kFx32ToCount = 2.3283064365386963e-10f * kInv4Ln2;  // 2^-32 / (4 ln 2)

__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
    const unsigned long long t0 = tc::global_ns();
    while (!tc::mbar_try_wait(bar, parity))
        if (tc::global_ns() - t0 > tc::kWaitLimitNs) return;
}

// IG of a key in units of 4 ln 2 nats; -inf for a key not yet set
__device__ __forceinline__ float key_ig_count(unsigned long long key) {
    return key ? order_bits_float((uint32_t)(key >> 32)) * kInv4Ln2 : -INFINITY;
}

// integer-valued float (exact, |v| < 2^22) -> int through the bits of 1.5 2^23 + v
__device__ __forceinline__ int f2i_exact(float f) { return __float_as_int(f + 12582912.0f) - 0x4B400000; }
__device__ __forceinline__ float i2f_exact(int v) { return __int_as_float(0x4B400000 + v) - 12582912.0f; }

__device__ __forceinline__ int tab32(const int* t, int n, int nmax) { return t[min((unsigned)n, (unsigned)nmax)]; }

// Two accumulator values v = n0 + 4096 n1 (exact integers below 2^24) split
// into n0 and n1: n1 = floor(v / 4096) is the sum 2^23 + v 2^-12 rounded
// toward zero (one fused multiply-add; the product is exact), then n0 = v -
// 4096 n1.  All three steps are exact.
__device__ __forceinline__ void split_classes(float2 v, float2& n0, float2& n1) {
    const float2 r = __ffma2_rz(v, make_float2(2.44140625e-4f, 2.44140625e-4f), make_float2(8388608.0f, 8388608.0f));
    n1 = add2(r, make_float2(-8388608.0f, -8388608.0f));
    n0 = fma2(n1, make_float2(-4096.0f, -4096.0f), v);
}

// regularised voxel term of SH in int32 fixed point, f(n0 + n1 + b0 + b1) -
// f(n0 + b0) - f(n1 + b1), from the smoothed counts m = n + beta
__device__ __forceinline__ int voxel32(const int* sT0, const int* sT1, const int* sTB, int N0, int N1, int N, float2 m,
                                       float beta0, float beta1) {
    const int n0 = f2i_exact(m.x - beta0), n1 = f2i_exact(m.y - beta1);
    return tab32(sTB, n0 + n1, N) - tab32(sT0, n0, N0) - tab32(sT1, n1, N1);
}

}  // namespace

// Work items: (job, discretisation, tile) for jobs.n jobs of the same N,
// discretisations d0 .. d0 + nd - 1 and the n_items tiles (row block of 128
// variables, column block of 64 variables at or after it); job j's operand rows
// are at z = j dstride + d of both tensor maps.  kMode 1 (kDump): also write
// the 3 x 3 class counts of every pair of job 0 to `dump` (test hook; the scan
// itself is unchanged).  kMode 2 (kEmit, one job): also insert every role whose
// IG reaches emit_thr (int32 fixed point) into the interesting-tuple table
// `emit`; the bound then also keeps every pair whose roles can reach
// emit_thr_c (the same threshold in units of 4 ln 2 nats).
template <int kMode>
__global__ void __launch_bounds__(kThreads, 1)
    k2tc3_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                 const __grid_constant__ K2Jobs jobs, int M, int d0, int nd, int dstride,
                 const int2* __restrict__ items, int n_items, int fbits, int* __restrict__ err, int prune_on,
                 uint32_t* __restrict__ dump, EmitTable emit, int emit_thr, float emit_thr_c) {
    constexpr bool kDump = kMode == 1, kEmit = kMode == 2;
    constexpr int S = kStages;
    const bool use_bound = !kDump && prune_on;
    extern __shared__ uint8_t dsmem_raw[];
    __shared__ uint64_t bar_full[S], bar_empty[S];
    __shared__ uint64_t bar_tfull[2], bar_tempty[2], bar_drain;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t* base = dsmem_raw + ((1024 - (tc::smem_u32(dsmem_raw) & 1023)) & 1023);
    float4* sCtx = reinterpret_cast<float4*>(base + ctx_offset());
    uint8_t* sQueue = base + queue_offset();
    const int N = jobs.job[0].tg.N0 + jobs.job[0].tg.N1, np1 = N + 1;  // the same N for every job
    const int tstride = tab_stride3(N);
    int* sTab = reinterpret_cast<int*>(base + tab_offset3());
    volatile int* abort = &s_abort;

    uint32_t dyn_bytes;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_bytes));
    const bool fits = jobs.n >= 1 && jobs.n <= kMaxK2Jobs &&
                      (size_t)(base - dsmem_raw) + tab_offset3() + (size_t)jobs.n * tstride * sizeof(int) <= dyn_bytes;

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
                    const int v0 = item.x * kRowVars, c0 = item.y * kBRows;
                    bool ok = true;
                    for (int kb = 0; kb < nkb; ++kb, ++g) {
                        const int s = (int)(g % S);
                        const uint32_t use = g / S;
                        if (use > 0 && !tc::mbar_wait(&bar_empty[s], (use - 1) & 1, abort)) {
                            ok = false;
                            break;
                        }
                        uint8_t* st = base + (size_t)s * kStageBytes;
                        tc::mbar_arrive_expect_tx(&bar_full[s], kStageBytes);
                        tc::tma_load_4d(st, &map_a, &bar_full[s], kb * kBK, 0, v0, z);
                        tc::tma_load_4d(st + kABytes, &map_a, &bar_full[s], kb * kBK, 1, v0, z);
                        tc::tma_load_3d(st + 2 * kABytes, &map_b, &bar_full[s], kb * kBK, c0, z);
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
                const uint32_t idesc = tc::idesc_e4m3_f32(kRowVars, kBRows);
                uint32_t g = 0;
                int i = 0;
                bool issued = false;
                for (int t = blockIdx.x; t < n_tiles && !*abort; t += gridDim.x, ++i) {
                    const int buf = i & 1;
                    const uint32_t tuse = (uint32_t)(i >> 1);
                    const int nkb = jobs.job[t / per_job].tg.nkb;
                    if (tuse > 0 && !tc::mbar_wait(&bar_tempty[buf], (tuse - 1) & 1, abort)) break;
                    tc::tc_fence_after();
                    const uint32_t dbase = tmem + (uint32_t)buf * kBufCols;
                    bool ok = true;
                    for (int kb = 0; kb < nkb; ++kb, ++g) {
                        const int s = (int)(g % S);
                        const uint32_t use = g / S;
                        if (!tc::mbar_wait(&bar_full[s], use & 1, abort)) {
                            ok = false;
                            break;
                        }
                        tc::tc_fence_after();
                        // both classes accumulate into one accumulator per row bin
                        const uint32_t st = tc::smem_u32(base + (size_t)s * kStageBytes);
                        const uint64_t dA0 = tc::sw128_kmajor_desc(st), dA1 = tc::sw128_kmajor_desc(st + kABytes);
                        const uint64_t dB = tc::sw128_kmajor_desc(st + 2 * kABytes);
                        const uint32_t first = kb == 0 ? 0u : 1u;
#pragma unroll
                        for (int kk = 0; kk < kBK / 32; ++kk) {
                            // a 32-byte step along K adds 2 to the descriptors' start address field
                            const uint32_t acc = kk > 0 ? 1u : first;
                            tc::mma_f8(dbase, dA0 + 2 * kk, dB + 2 * kk, idesc, acc);
                            tc::mma_f8(dbase + kAccCols, dA1 + 2 * kk, dB + 2 * kk, idesc, acc);
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
        const int q = warp & 3, h = ew >> 2;  // TMEM lane quarter, column-variable group
        const int row = 32 * q + lane;
        float4* ctx = sCtx + ew * (2 * kColsPerWarp);
        // pair queue of this warp: q0 / q1 [v * kQueue + r] hold the smoothed
        // class-0 / class-1 counts of voxel v (row-major (row bin, column bin))
        // of record r; qid[r] = (vi, vm, SH1(i), SH1(m))
        float* q0 = reinterpret_cast<float*>(sQueue + (size_t)ew * kQueueWarpBytes);
        float* q1 = q0 + 9 * kQueue;
        uint4* qid = reinterpret_cast<uint4*>(q1 + 9 * kQueue);
        const float inv_scale = __int_as_float((127 - fbits) << 23);
        const uint32_t lanes_below = (1u << lane) - 1u;
        int qn = 0, q_job = 0, q_d = 0;  // queued records, all of job q_job and discretisation q_d

        // Evaluates records 0 .. n-1 of the queue, one per lane: SH2 from the
        // tables, then both roles' keys, IG(i | m) = SH1(m) - SH2 and IG(m | i) =
        // SH1(i) - SH2.  A rolled voxel loop keeps this code, inlined at every
        // call, short.
        auto flush = [&](int n) {
            __syncwarp();
            if (lane < n) {
                const K2Job& J = jobs.job[q_job];
                const int N0 = J.tg.N0, N1 = J.tg.N1;
                const int* sT0 = sTab + q_job * tstride;
                const int* sT1 = sT0 + (N0 + 1);
                const int* sTB = sT1 + (N1 + 1);
                const float beta0 = J.b0, beta1 = J.b1;
                const uint4 id = qid[lane];  // vi, vm, SH1(i), SH1(m) (int32 fixed point)
                uint32_t* o = nullptr;
                if constexpr (kDump) {
                    const unsigned long long np = (unsigned long long)M * (M - 1) / 2;
                    const unsigned long long rank =
                        (unsigned long long)id.x * (2ull * M - id.x - 1) / 2 + (unsigned long long)(id.y - id.x - 1);
                    o = dump + ((unsigned long long)q_d * np + rank) * 9;
                }
                int sh2 = 0;
#pragma unroll 1
                for (int v = 0; v < 9; ++v) {
                    const int n0 = f2i_exact(q0[v * kQueue + lane] - beta0), n1 = f2i_exact(q1[v * kQueue + lane] - beta1);
                    sh2 += tab32(sTB, n0 + n1, N) - tab32(sT0, n0, N0) - tab32(sT1, n1, N1);
                    if constexpr (kDump) o[v] = (uint32_t)n0 | ((uint32_t)n1 << 16);
                }
                const uint32_t dM = (uint32_t)q_d * (uint32_t)M;
                atomicMax(J.keys + id.x, pack_key((float)((int)id.w - sh2) * inv_scale, dM + id.y));
                atomicMax(J.keys + id.y, pack_key((float)((int)id.z - sh2) * inv_scale, dM + id.x));
                if constexpr (kEmit) {
                    const int gi = (int)id.w - sh2, gm = (int)id.z - sh2;
                    if (gi >= emit_thr)
                        emit_insert(emit, emit_key((int)id.x, (int)id.y, -1, -1),
                                    pack_key((float)gi * inv_scale, (uint32_t)q_d));
                    if (gm >= emit_thr)
                        emit_insert(emit, emit_key((int)id.y, (int)id.x, -1, -1),
                                    pack_key((float)gm * inv_scale, (uint32_t)q_d));
                }
            }
            __syncwarp();
        };

        int i = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++i) {
            if (__any_sync(0xffffffffu, *abort != 0)) break;
            const int buf = i & 1;
            const uint32_t tuse = (uint32_t)(i >> 1);
            const int job = t / per_job, r = t - job * per_job, dl = r / n_items;
            const int2 item = items[r - dl * n_items];
            const int d = d0 + dl;
            if (qn > 0 && (job != q_job || d != q_d)) {  // warp-uniform
                flush(qn);
                qn = 0;
            }
            q_job = job;
            q_d = d;
            const K2Job& J = jobs.job[job];
            const int N0 = J.tg.N0, N1 = J.tg.N1;
            unsigned long long* keys = J.keys;
            const float beta0 = J.b0, beta1 = J.b1;
            const int vi = item.x * kRowVars + row;                  // row variable
            const int vm0 = item.y * kColVars + kColsPerWarp * h;    // first column variable of this warp
            // single counts [v][bin][class] of this discretisation: 4 ints per variable
            const int* c1 = J.cnt1 + (size_t)d * M * 4;
            const long long* s1 = J.sh1 + (size_t)d * M;
            const bool irow = vi < M;
            // column context, staged by lanes 0-15 of the warp: smoothed class-0
            // counts of bins 1, 2 and class-1 counts of bins 1, 2 (count + beta);
            // SH1 and key in units of 4 ln 2 nats; SH1 as int32 fixed point
            __syncwarp();
            if (lane < kColsPerWarp) {
                const int vc = vm0 + lane;
                const bool cok = vc < M;
                const int4 cc = cok ? *reinterpret_cast<const int4*>(c1 + (size_t)vc * 4) : make_int4(0, 0, 0, 0);
                const long long s = cok ? s1[vc] : 0ll;
                const unsigned long long kc = cok ? __ldcg(keys + vc) : 0ull;
                ctx[2 * lane] = make_float4(i2f_exact(cc.x) + beta0, i2f_exact(cc.z) + beta0,
                                            i2f_exact(cc.y) + beta1, i2f_exact(cc.w) + beta1);
                float kcc = cok ? key_ig_count(kc) : 0.0f;
                if constexpr (kEmit) kcc = fminf(kcc, emit_thr_c);
                ctx[2 * lane + 1] = make_float4((float)s * kFx32ToCount, kcc,
                                                __int_as_float(fx_narrow(s, fbits)), 0.0f);
            }
            __syncwarp();
            // row context, smoothed: class-c count of bin a + 1 plus beta_c
            // (ni_c_a), of bin 0 plus 3 beta_c (R_c)
            const int4 rc = irow ? *reinterpret_cast<const int4*>(c1 + (size_t)vi * 4) : make_int4(0, 0, 0, 0);
            const float ni_0_0 = i2f_exact(rc.x) + beta0, ni_1_0 = i2f_exact(rc.y) + beta1;
            const float ni_0_1 = i2f_exact(rc.z) + beta0, ni_1_1 = i2f_exact(rc.w) + beta1;
            const float R_0 = i2f_exact(N0 - rc.x - rc.z) + 3.0f * beta0;
            const float R_1 = i2f_exact(N1 - rc.y - rc.w) + 3.0f * beta1;
            const long long s1i = irow ? s1[vi] : 0ll;
            const int shi = fx_narrow(s1i, fbits);
            const float shi_c = (float)s1i * kFx32ToCount;
            float keyi_c = irow ? key_ig_count(__ldcg(keys + vi)) : 0.0f;
            if constexpr (kEmit) keyi_c = fminf(keyi_c, emit_thr_c);
            const float2 B0 = make_float2(beta0, beta0), B1 = make_float2(beta1, beta1);

            if (!__all_sync(0xffffffffu, tc::mbar_wait(&bar_tfull[buf], tuse & 1, abort))) break;  // warp-uniform
            tc::tc_fence_after();
            const bool live = (item.x * kRowVars + 32 * q) < M && vm0 < M;  // warp-uniform
            const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)buf * kBufCols +
                                   (uint32_t)(2 * kColsPerWarp * h);
#pragma unroll 1
            for (int pass = 0; pass < kColsPerWarp / kColsPerPass; ++pass) {
                // accumulator a (row bin a + 1), columns 2 j + b (column bin b + 1):
                // n0 + 4096 n1
                uint32_t v[2][2 * kColsPerPass];
                if (live) {
                    tc::tmem_ld16(taddr + 2u * kColsPerPass * pass, v[0]);
                    tc::tmem_ld16(taddr + kAccCols + 2u * kColsPerPass * pass, v[1]);
                    tc::tmem_ld_wait();
                }
                if (pass == kColsPerWarp / kColsPerPass - 1) {
                    // this thread's last TMEM read of the tile: the buffer may be refilled
                    tc::tc_fence_before();
                    tc::mbar_arrive(&bar_tempty[buf]);
                }
                if (!live) continue;
#pragma unroll
                for (int jj = 0; jj < kColsPerPass; ++jj) {
                    const int jv = kColsPerPass * pass + jj;
                    const int vm = vm0 + jv;
                    const bool ok = vi < vm && vm < M;
                    const float4 cA = ctx[2 * jv], cB = ctx[2 * jv + 1];
                    // counts with both bins >= 1: x_a_c = (row bin a + 1 with column
                    // bins 1, 2) of class c, and their smoothed values m_a_c
                    float2 x_0_0, x_0_1, x_1_0, x_1_1;
                    split_classes(make_float2(__uint_as_float(v[0][2 * jj]), __uint_as_float(v[0][2 * jj + 1])), x_0_0,
                                  x_0_1);
                    split_classes(make_float2(__uint_as_float(v[1][2 * jj]), __uint_as_float(v[1][2 * jj + 1])), x_1_0,
                                  x_1_1);
                    const float2 m_0_0 = add2(x_0_0, B0), m_0_1 = add2(x_0_1, B1);
                    const float2 m_1_0 = add2(x_1_0, B0), m_1_1 = add2(x_1_1, B1);
                    // the other voxels by inclusion-exclusion from the smoothed margins
                    // (each carries beta once): u_c row bin 0 with column bins 1, 2;
                    // w_c row bins 1, 2 with column bin 0; z_c bin 0 with bin 0
                    const float2 u_0 = sub2(sub2(make_float2(cA.x, cA.y), x_0_0), x_1_0);
                    const float2 u_1 = sub2(sub2(make_float2(cA.z, cA.w), x_0_1), x_1_1);
                    const float2 w_0 = make_float2(ni_0_0 - x_0_0.x - x_0_0.y, ni_0_1 - x_1_0.x - x_1_0.y);
                    const float2 w_1 = make_float2(ni_1_0 - x_0_1.x - x_0_1.y, ni_1_1 - x_1_1.x - x_1_1.y);
                    const float z_0 = R_0 - u_0.x - u_0.y, z_1 = R_1 - u_1.x - u_1.y;
                    bool need = ok;
                    if (use_bound) {
                        // sum over the 9 voxels of m0 m1 / (m0 + m1) as one fraction,
                        // two voxels per packed lane pair
                        const float2 pna = mul2(m_0_0, m_0_1), psa = add2(m_0_0, m_0_1);
                        const float2 pnb = mul2(m_1_0, m_1_1), psb = add2(m_1_0, m_1_1);
                        const float2 pnc = mul2(u_0, u_1), psc = add2(u_0, u_1);
                        const float2 pnd = mul2(w_0, w_1), psd = add2(w_0, w_1);
                        const float2 nab = fma2(pnb, psa, mul2(pna, psb)), dab = mul2(psa, psb);
                        const float2 ncd = fma2(pnd, psc, mul2(pnc, psd)), dcd = mul2(psc, psd);
                        const float2 n4 = fma2(ncd, dab, mul2(nab, dcd)), d4 = mul2(dab, dcd);
                        float num = fmaf(n4.x, d4.y, n4.y * d4.x), den = d4.x * d4.y;
                        num = fmaf(num, z_0 + z_1, z_0 * z_1 * den);
                        den *= z_0 + z_1;
                        // largest SH2 (units of 4 ln 2 nats) that lets one role reach its key
                        const float hi = fmaxf(cB.x - keyi_c, shi_c - cB.y);
                        const float lim = fmaf(fabsf(hi), kBoundRel, hi + kBoundAbs);
                        need = ok && num <= lim * den;
                    }
                    const uint32_t mask = __ballot_sync(0xffffffffu, need);
                    if (mask == 0u) continue;
                    // queue the pairs that need their lookups; a full queue is evaluated
                    const int cnt = __popc(mask), rank = __popc(mask & lanes_below), room = kQueue - qn;
                    auto put = [&](int slot) {
                        const float c0v[9] = {z_0,     u_0.x,   u_0.y, w_0.x, m_0_0.x,
                                              m_0_0.y, w_0.y,   m_1_0.x, m_1_0.y};
                        const float c1v[9] = {z_1,     u_1.x,   u_1.y, w_1.x, m_0_1.x,
                                              m_0_1.y, w_1.y,   m_1_1.x, m_1_1.y};
#pragma unroll
                        for (int v = 0; v < 9; ++v) {
                            q0[v * kQueue + slot] = c0v[v];
                            q1[v * kQueue + slot] = c1v[v];
                        }
                        qid[slot] = make_uint4((uint32_t)vi, (uint32_t)vm, (uint32_t)shi, __float_as_uint(cB.z));
                    };
                    // a full queue is evaluated as often as this column's pairs fill it
                    int room_left = room, placed = 0;
                    if (need && rank < room_left) put(qn + rank);
                    while (cnt - placed >= room_left) {  // warp-uniform
                        flush(kQueue);
                        placed += room_left;
                        room_left = kQueue;
                        qn = 0;
                        if (need && rank >= placed && rank < placed + room_left) put(rank - placed);
                    }
                    qn += cnt - placed;
                }
            }
        }
        if (qn > 0 && !__any_sync(0xffffffffu, *abort != 0)) flush(qn);
    }

    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, kTmemCols);
    if (tid == 0 && *abort) atomicOr(err, *abort);
}

// Tiles (row block it of 128 variables, column block mt of 64 variables) with
// column block start >= row block start: every unordered pair once, the pairs
// i < m of the diagonal tiles selected in the kernel.
void build_k2tc3_items(int M, std::vector<int2>& items) {
    const int nr = (M + kRowVars - 1) / kRowVars, nc = (M + kColVars - 1) / kColVars;
    constexpr int ratio = kRowVars / kColVars;
    items.clear();
    for (int it = 0; it < nr; ++it)
        for (int mt = it * ratio; mt < nc; ++mt) items.push_back(make_int2(it, mt));
}

// the kernel runs kStages pipeline stages: any other count does not fit
size_t k2tc3_smem_bytes(int N, int n_jobs, int stages) {
    if (stages != kStages) return ~(size_t)0;
    return tab_offset3() + (size_t)n_jobs * tab_stride3(N) * sizeof(int) + 1024;
}

bool k2tc3_counts_fit(int N0, int N1) { return N0 >= 1 && N1 >= 1 && N0 < 4096 && N1 < 4096; }

uint32_t k2tc3_class1_byte() { return 0x68; }  // E4M3 64.0

cudaError_t launch_k2tc3(const uint8_t* oh, int Kp, int zdim, const K2Jobs& jobs, int M, int d0, int nd, int dstride,
                         const int2* items, int n_items, int fbits, int* err, bool bound, int stages, cudaStream_t st,
                         uint32_t* dump, EmitTable emit) {
    if (n_items == 0 || jobs.n == 0) return cudaSuccess;
    if (jobs.n < 1 || jobs.n > kMaxK2Jobs || stages != kStages || (dump && jobs.n != 1) ||
        (emit.keys && (jobs.n != 1 || dump)))
        return cudaErrorInvalidValue;
    if (Kp <= 0 || Kp % kBK != 0 || M < 1 || zdim < 1) return cudaErrorInvalidValue;
    const int N = jobs.job[0].tg.N0 + jobs.job[0].tg.N1;
    for (int j = 0; j < jobs.n; ++j) {
        const TcGeom& tg = jobs.job[j].tg;
        if (tg.N0 + tg.N1 != N || !k2tc3_counts_fit(tg.N0, tg.N1) || tg.Kp > Kp || tg.nkb * kBK != tg.Kp ||
            tg.nkb0 < 1 || tg.nkb0 >= tg.nkb)
            return cudaErrorInvalidValue;
        // the bound needs pseudocounts that keep its fraction away from 0 and infinity
        if (!(jobs.job[j].b0 >= 1e-3f && jobs.job[j].b1 >= 1e-3f)) bound = false;
    }
    // A: the rows of one bin (every second row) of 128 variables; B: 128 consecutive rows
    CUtensorMap map_a, map_b;
    const cuuint64_t kp = (cuuint64_t)Kp, rows = 2 * (cuuint64_t)M;
    const cuuint64_t dims_a[4] = {kp, 2, (cuuint64_t)M, (cuuint64_t)zdim};
    const cuuint64_t str_a[3] = {kp, 2 * kp, rows * kp};
    const cuuint32_t box_a[4] = {(cuuint32_t)kBK, 1, (cuuint32_t)kRowVars, 1};
    const cuuint64_t dims_b[3] = {kp, rows, (cuuint64_t)zdim};
    const cuuint64_t str_b[2] = {kp, rows * kp};
    const cuuint32_t box_b[3] = {(cuuint32_t)kBK, (cuuint32_t)kBRows, 1};
    cudaError_t e = make_tiled_map_u8(&map_a, oh, 4, dims_a, str_a, box_a);
    if (e != cudaSuccess) return e;
    if ((e = make_tiled_map_u8(&map_b, oh, 3, dims_b, str_b, box_b)) != cudaSuccess) return e;
    const size_t smem = k2tc3_smem_bytes(N, jobs.n, stages);
    const void* fn = dump        ? (const void*)k2tc3_kernel<1>
                     : emit.keys ? (const void*)k2tc3_kernel<2>
                                 : (const void*)k2tc3_kernel<0>;
    if ((e = ensure_dynamic_smem(fn, smem)) != cudaSuccess) return e;
    // the register split inside the kernel needs exactly kRegsLaunch registers per thread
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
    // the emission threshold as int32 fixed point and in units of 4 ln 2 nats (the bound's)
    const int ethr = emit_threshold_fx(emit, fbits);
    const float ethr_c = (float)((double)emit.thr_fx * 2.3283064365386963e-10 / (4.0 * 0.6931471805599453));
    if (dump)
        k2tc3_kernel<1><<<grid, kThreads, smem, st>>>(map_a, map_b, jobs, M, d0, nd, dstride, items, n_items, fbits,
                                                      err, prune_on, dump, emit, ethr, ethr_c);
    else if (emit.keys)
        k2tc3_kernel<2><<<grid, kThreads, smem, st>>>(map_a, map_b, jobs, M, d0, nd, dstride, items, n_items, fbits,
                                                      err, prune_on, nullptr, emit, ethr, ethr_c);
    else
        k2tc3_kernel<0><<<grid, kThreads, smem, st>>>(map_a, map_b, jobs, M, d0, nd, dstride, items, n_items, fbits,
                                                      err, prune_on, nullptr, emit, ethr, ethr_c);
    return cudaGetLastError();
}

}  // namespace mdfs
