// k = 2 scan on the 5th-generation tensor cores (tcgen05, kind::f8f6f4).
// Voxel counters of section "Algorithm and implementation"; the two IG roles of
// Eq. 1 with |S| = 1.  This file holds the c = 2 kernel and the launcher for
// both class counts; c = 3 runs the kernel of mdfs_k2tc3.cu.
//
// c = 2: every variable is one E4M3 one-hot row (its bin 1) over the
// class-sorted samples.  The pair counts of the voxel (1, 1) are the symmetric
// GEMM C = OH OH^T; class-0 and class-1 samples occupy separate K ranges and
// accumulate into two TMEM accumulators.  Tiles of 128 x 128 variables on and
// above the diagonal; no operand needs masking.  Counts are exact (0/1
// products, FP32 sums below 2^24); the other three voxels follow from the bin
// counts of the two variables.
//
// Persistent kernel, one CTA per SM, 640 threads:
//   warp 0       TMA producer (A rows, B rows; 128B swizzle),
//   warp 1       TMEM owner and MMA issuer,
//   warps 4-19   epilogue: tcgen05.ld, 2 x 2 tables per class by
//                inclusion-exclusion, SH2 from int32 fixed-point tables in
//                shared memory, IG(i | m) = SH1(m) - SH2 and IG(m | i), keys.
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

// integer-valued float (exact, |v| < 2^22) -> int through the bits of 1.5 2^23 + v
__device__ __forceinline__ int f2i_exact(float f) { return __float_as_int(f + 12582912.0f) - 0x4B400000; }

}  // namespace

// Work items of a launch: (job, discretisation, tile) for jobs.n jobs of the
// same N (a batch's resamples; one job for a plain scan), discretisations
// d0 .. d0 + nd - 1, and the n_items symmetric tiles; job j's operand rows are
// at z = j dstride + d of the tensor map.  Every job's entropy tables sit in
// shared memory at once.  S: pipeline stages.  kMode 1 (kDump): also write
// the 2 x 2 class counts of every pair of job 0 to `dump` (test hook; the scan
// itself is unchanged).  kMode 2 (kEmit, one job): also insert every role whose
// IG reaches emit_thr (int32 fixed point, fbits fraction bits) into the
// interesting-tuple table `emit`.
template <int S, int kMode>
__global__ void __launch_bounds__(kThreads, 1)
    k2tc_kernel(const __grid_constant__ CUtensorMap map_oh, const __grid_constant__ K2Jobs jobs, int M, int d0,
                int nd, int dstride, const int2* __restrict__ items, int n_items, int fbits, int* __restrict__ err,
                uint32_t* __restrict__ dump, EmitTable emit, int emit_thr) {
    constexpr bool kDump = kMode == 1, kEmit = kMode == 2;
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
        const float inv_scale = __int_as_float((127 - fbits) << 23);
        int i = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++i) {
            if (__any_sync(0xffffffffu, *abort != 0)) break;
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
            const int vi = item.x * kTile + row;                  // row variable
            const int vm0 = item.y * kTile + kColsPerWarp * h;    // first column variable of this warp
            const bool diag = item.x == item.y;
            const int* c1 = J.cnt1 + (size_t)d * M * 2;
            const long long* s1 = J.sh1 + (size_t)d * M;
            const bool irow = vi < M;
            // bin-1 class counts of the row variable
            const int ni0 = irow ? c1[(size_t)vi * 2] : 0, ni1 = irow ? c1[(size_t)vi * 2 + 1] : 0;
            const int shi = irow ? fx_narrow(s1[vi], fbits) : 0;
            const uint32_t dM = (uint32_t)d * (uint32_t)M;

            if (!__all_sync(0xffffffffu, tc::mbar_wait(&bar_tfull[buf], tuse & 1, abort))) break;  // warp-uniform
            tc::tc_fence_after();
            unsigned long long ki = 0ull;
            const bool warp_rows = item.x * kTile + 32 * q < M;
            uint32_t r0[kColsPerWarp], r1[kColsPerWarp];
            if (warp_rows && vm0 < M) {
                const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)buf * kAccCols +
                                       (uint32_t)(kColsPerWarp * h);
                tc::tmem_ld16(taddr, *reinterpret_cast<uint32_t(*)[16]>(&r0[0]));
                tc::tmem_ld16(taddr + 16, *reinterpret_cast<uint32_t(*)[16]>(&r0[16]));
                tc::tmem_ld16(taddr + kTile, *reinterpret_cast<uint32_t(*)[16]>(&r1[0]));
                tc::tmem_ld16(taddr + kTile + 16, *reinterpret_cast<uint32_t(*)[16]>(&r1[16]));
                tc::tmem_ld_wait();
            }
            // every read of this tile's accumulators is done: the buffer may be refilled
            tc::tc_fence_before();
            tc::mbar_arrive(&bar_tempty[buf]);
            if (warp_rows && vm0 < M) {
                // column-variable context: lane j holds column vm0 + j, handed to
                // every lane of the warp by shuffles per column
                const int vcol = vm0 + lane;
                const bool colok = vcol < M;
                const int cn0 = colok ? c1[(size_t)vcol * 2] : 0, cn1 = colok ? c1[(size_t)vcol * 2 + 1] : 0;
                const int csh = colok ? fx_narrow(s1[vcol], fbits) : 0;
#pragma unroll
                for (int jm = 0; jm < kColsPerWarp; ++jm) {
                    const int vm = vm0 + jm;
                    const bool ok = irow && vm < M && (!diag || vi < vm);
                    const int nm0 = __shfl_sync(0xffffffffu, cn0, jm), nm1 = __shfl_sync(0xffffffffu, cn1, jm);
                    const int shm = __shfl_sync(0xffffffffu, csh, jm);
                    if (!__any_sync(0xffffffffu, ok)) continue;
                    // voxel (1, 1) per class from the accumulators (exact FP32 integers),
                    // the others from the bin-1 counts: T[a][b], a = code of i, b = code of m
                    const int x0 = f2i_exact(__uint_as_float(r0[jm])), x1 = f2i_exact(__uint_as_float(r1[jm]));
                    const int T0[2][2] = {{N0 - ni0 - nm0 + x0, nm0 - x0}, {ni0 - x0, x0}};
                    const int T1[2][2] = {{N1 - ni1 - nm1 + x1, nm1 - x1}, {ni1 - x1, x1}};
                    if constexpr (kDump) {
                        if (ok) {
                            const unsigned long long np = (unsigned long long)M * (M - 1) / 2;
                            const unsigned long long rank =
                                (unsigned long long)vi * (2ull * M - vi - 1) / 2 + (unsigned long long)(vm - vi - 1);
                            uint32_t* o = dump + ((unsigned long long)d * np + rank) * 4;
#pragma unroll
                            for (int a = 0; a < 2; ++a)
#pragma unroll
                                for (int b = 0; b < 2; ++b)
                                    o[a * 2 + b] = (uint32_t)T0[a][b] | ((uint32_t)T1[a][b] << 16);
                        }
                    }
                    int sh2 = 0;
#pragma unroll
                    for (int a = 0; a < 2; ++a)
#pragma unroll
                        for (int b = 0; b < 2; ++b)
                            sh2 += tab32(sTB, T0[a][b] + T1[a][b], N) - tab32(sT0, T0[a][b], N0) -
                                   tab32(sT1, T1[a][b], N1);
                    unsigned long long k_m = 0ull;
                    if (ok) {
                        // IG(i | m) = SH1(m) - SH2
                        ki = umax64(ki, pack_key((float)(shm - sh2) * inv_scale, dM + (uint32_t)vm));
                        // IG(m | i) = SH1(i) - SH2
                        k_m = pack_key((float)(shi - sh2) * inv_scale, dM + (uint32_t)vi);
                        if constexpr (kEmit) {
                            if (shm - sh2 >= emit_thr)
                                emit_insert(emit, emit_key(vi, vm, -1, -1),
                                            pack_key((float)(shm - sh2) * inv_scale, (uint32_t)d));
                            if (shi - sh2 >= emit_thr)
                                emit_insert(emit, emit_key(vm, vi, -1, -1),
                                            pack_key((float)(shi - sh2) * inv_scale, (uint32_t)d));
                        }
                    }
                    const unsigned long long mk = warp_max_key(k_m);
                    if (lane == 0 && mk) atomicMax(keys + vm, mk);
                }
            }
            if (ki) atomicMax(keys + vi, ki);
        }
    }

    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, kTmemCols);
    if (tid == 0 && *abort) atomicOr(err, *abort);
}

void build_k2tc_items(int M, int c, std::vector<int2>& items) {
    if (c == 3) {
        build_k2tc3_items(M, items);
        return;
    }
    const int nt = (M + kTile - 1) / kTile;
    items.clear();
    for (int it = 0; it < nt; ++it)
        for (int mt = it; mt < nt; ++mt) items.push_back(make_int2(it, mt));
}

size_t k2tc_smem_bytes(int c, int N, int n_jobs, int stages) {
    if (c == 3) return k2tc3_smem_bytes(N, n_jobs, stages);
    return tab_offset(stages) + (size_t)n_jobs * tab_stride(N) * sizeof(int) + 1024;
}

int k2tc_max_jobs(int c, int N, int stages, size_t smem_limit) {
    const size_t base = k2tc_smem_bytes(c, N, 0, stages), per = k2tc_smem_bytes(c, N, 1, stages) - base;
    if (smem_limit < base + per) return 0;
    return (int)std::min<size_t>((smem_limit - base) / per, (size_t)kMaxK2Jobs);
}

bool k2tc_supported(int c) { return c == 2 || c == 3; }

// c = 2 keeps the classes in separate accumulators: any class sizes below 2^24
bool k2tc_counts_fit(int c, int N0, int N1) { return c == 3 ? k2tc3_counts_fit(N0, N1) : N0 >= 1 && N1 >= 1; }

uint32_t k2tc_class1_byte(int c) { return c == 3 ? k2tc3_class1_byte() : 0x38u; }

cudaError_t launch_k2tc(const uint8_t* oh, int Kp, int zdim, const K2Jobs& jobs, int M, int c, int d0, int nd,
                        int dstride, const int2* items, int n_items, int fbits, int* err, bool bound, int stages,
                        cudaStream_t st, uint32_t* dump, EmitTable emit) {
    if (c == 3)
        return launch_k2tc3(oh, Kp, zdim, jobs, M, d0, nd, dstride, items, n_items, fbits, err, bound, stages, st,
                            dump, emit);
    if (c != 2) return cudaErrorInvalidValue;
    if (n_items == 0 || jobs.n == 0) return cudaSuccess;
    if (jobs.n < 1 || jobs.n > kMaxK2Jobs || (stages != 3 && stages != 4) || (dump && (jobs.n != 1 || stages != 4)) ||
        (emit.keys && (jobs.n != 1 || dump)))
        return cudaErrorInvalidValue;
    const int N = jobs.job[0].tg.N0 + jobs.job[0].tg.N1;
    for (int j = 0; j < jobs.n; ++j) {
        const TcGeom& tg = jobs.job[j].tg;
        if (tg.N0 + tg.N1 != N || tg.Kp > Kp || tg.nkb * kBK != tg.Kp || tg.nkb0 < 1 || tg.nkb0 >= tg.nkb)
            return cudaErrorInvalidValue;
    }
    CUtensorMap map;
    cudaError_t e = make_onehot_map(&map, oh, M, zdim, Kp);
    if (e != cudaSuccess) return e;
    const size_t smem = k2tc_smem_bytes(c, N, jobs.n, stages);
    const int mode = dump ? 1 : emit.keys ? 2 : 0;
    const void* fn = mode == 1   ? (const void*)k2tc_kernel<4, 1>
                     : mode == 2 ? (stages == 4 ? (const void*)k2tc_kernel<4, 2> : (const void*)k2tc_kernel<3, 2>)
                                 : (stages == 4 ? (const void*)k2tc_kernel<4, 0> : (const void*)k2tc_kernel<3, 0>);
    if ((e = ensure_dynamic_smem(fn, smem)) != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
    if (fa.numRegs != kRegsLaunch) return cudaErrorInvalidConfiguration;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const long long n_tiles = (long long)n_items * nd * jobs.n;
    if (n_tiles >= (1ll << 31)) return cudaErrorInvalidValue;
    const int grid = (int)std::min<long long>(n_tiles, (long long)sms);
    const int ethr = emit_threshold_fx(emit, fbits);
    if (mode == 1)
        k2tc_kernel<4, 1><<<grid, kThreads, smem, st>>>(map, jobs, M, d0, nd, dstride, items, n_items, fbits, err,
                                                        dump, emit, ethr);
    else if (mode == 2 && stages == 4)
        k2tc_kernel<4, 2><<<grid, kThreads, smem, st>>>(map, jobs, M, d0, nd, dstride, items, n_items, fbits, err,
                                                        nullptr, emit, ethr);
    else if (mode == 2)
        k2tc_kernel<3, 2><<<grid, kThreads, smem, st>>>(map, jobs, M, d0, nd, dstride, items, n_items, fbits, err,
                                                        nullptr, emit, ethr);
    else if (stages == 4)
        k2tc_kernel<4, 0><<<grid, kThreads, smem, st>>>(map, jobs, M, d0, nd, dstride, items, n_items, fbits, err,
                                                        nullptr, emit, ethr);
    else
        k2tc_kernel<3, 0><<<grid, kThreads, smem, st>>>(map, jobs, M, d0, nd, dstride, items, n_items, fbits, err,
                                                        nullptr, emit, ethr);
    return cudaGetLastError();
}

}  // namespace mdfs
