// k = 3 scan for two classes per variable (c = 2) on the 5th-generation tensor
// cores (tcgen05, kind::f8f6f4).  Voxel counters of section "Algorithm and
// implementation"; IG roles of Eq. 1 with |S| = 2.
//
// Each variable's bin-1 indicator over the class-sorted samples is stored as
// one-hot E4M3 bytes (1.0 or 0).  For a middle variable b, the count of the
// all-ones voxel of every triple (a, b, e) is
//     X[a][e] = sum_s OH[a][s] * OH[b][s] * OH[e][s],
// a GEMM with A = OH[a-tile] masked by OH[b] and B = OH[e-tile], both K-major.
// Products of 0/1 are exact and the FP32 accumulator is exact below 2^24, so
// the counts are exact integers.  Class-0 and class-1 samples occupy separate
// K ranges and accumulate into two TMEM accumulators.
//
// Variables are relabelled per discretisation in ascending order of their
// bin-1 count before the scan (k3tc_order_kernel).  The kernel enumerates the
// triples a < b < e of the new labels, which covers every unordered triple
// once; in that order the 32 rows a of a warp have similar marginal counts, so
// the voxel counts they look up fall in a narrow window of the entropy tables
// and the shared-memory loads see fewer bank conflicts.  The one-hot rows,
// pair records and single counts are stored in the new order; keys are
// written for the original variables with sorted original partner indices.
//
// Persistent, warp-specialised kernel (one CTA per SM, 640 threads):
//   warp 0       TMA producer: A (a rows), B (e rows), OH[b] row per K block,
//   warp 1       TMEM owner and MMA issuer (4 MMAs of K = 32 per K block),
//   warps 2-3    AND the A tile with OH[b] in shared memory (128B swizzle),
//   warps 4-19   epilogue: tcgen05.ld of both class accumulators, the 8-voxel
//                tables by inclusion-exclusion, SH3 from fixed-point tables
//                in shared memory, three IG roles, packed max keys.
// Registers: launched at kRegsLaunch per thread; the first warpgroup gives
// back to kRegsProducer, the four epilogue warpgroups take kRegsEpilogue
// (128 kRegsProducer + 512 kRegsEpilogue == 640 kRegsLaunch).
// Four shared-memory stages and two TMEM accumulator buffers (2 x 256
// columns) let the epilogue of one tile overlap the MMAs of the next.
//
// Entropy arithmetic: the FP64-built int64 tables (multiples of 2^-32) are
// rounded to int32 multiples of 2^-s and summed with wrap-around; the IG
// difference is exact modulo 2^32 and |IG| 2^s < 2^31 recovers it.  Error per
// IG <= 25 * 2^-(s+1) (24 table entries and the rounded pair entropy).
//
// Every mbarrier wait is bounded; on timeout the kernel records an error,
// drains its copies and MMAs, frees TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <climits>

#include "mdfs_device.cuh"
#include "mdfs_internal.cuh"
#include "mdfs_tc.cuh"

namespace mdfs {

namespace {

constexpr int kTile = 128;                    // a rows, e columns
constexpr int kBK = 128;                      // K bytes (samples) per stage
constexpr int kStages = 4;
constexpr uint32_t kTileBytes = kTile * kBK;  // 16 KB
constexpr uint32_t kAccCols = 2 * kTile;      // class 0 and class 1 accumulators
constexpr uint32_t kTmemCols = 2 * kAccCols;  // double buffer
constexpr int kThreads = 640;
constexpr int kMaskWarp0 = 2, kMaskThreads = 64;
constexpr int kEpiWarp0 = 4, kEpiThreads = 512;
constexpr int kColsPerWarp = 32;
constexpr int kRegsLaunch = 96, kRegsProducer = 32, kRegsEpilogue = 112;
static_assert(128 * kRegsProducer + kEpiThreads * kRegsEpilogue == kThreads * kRegsLaunch,
              "register split must add up to the launch allocation");
// Entropy tables sit first in dynamic shared memory at fixed byte offsets, so a
// lookup is one load with an immediate base: T0 [0, 4096), T1 [4096, 8192),
// TB [8192, 16384) int32 entries.  The stages follow, 1024-byte aligned.
constexpr int kT0Cap = 4096, kT1Cap = 4096, kTBCap = 8192;
constexpr size_t kTabBytes = (size_t)(kT0Cap + kT1Cap + kTBCap) * sizeof(int);
constexpr size_t kStageBytes = 2 * kStages * kTileBytes + kStages * kBK;  // A, B, OH[b] rows

// Waits for completion regardless of an abort (draining in-flight work); bounded.
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

// table entry at byte offset n4 = 4 n (counts are carried multiplied by 4), clamped to the table
__device__ __forceinline__ int tab4(const int* t, int n4, int nmax4) {
    return *reinterpret_cast<const int*>(reinterpret_cast<const char*>(t) + min((unsigned)n4, (unsigned)nmax4));
}

// exact integer value of an FP32 count, times 4
__device__ __forceinline__ int count4(uint32_t f) { return __float2int_rn(__uint_as_float(f)) << 2; }

struct ColCtx {
    int n0, n1;    // pair (b, e): class counts of voxel (1, 1), times 4
    int sh;        // pair (b, e): entropy, int32 fixed point
    int ne0, ne1;  // single e: class counts of bin 1, times 4
    int eo;        // original index of e
};

// partner index of a key: (d M + lo) M + hi with the two partners sorted
__device__ __forceinline__ uint32_t partner_index(uint32_t dM, int M, uint32_t p, uint32_t q) {
    return (dM + min(p, q)) * (uint32_t)M + max(p, q);
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 1)
    k3tc_kernel(const __grid_constant__ CUtensorMap map_oh, const uint8_t* __restrict__ oh, TcGeom tg, int M, int d0,
                int nd, const int2* __restrict__ items, int n_items, const long long* __restrict__ tab, int fbits,
                const int* __restrict__ cnt1s, const int* __restrict__ perm, const PairC* __restrict__ pairs,
                unsigned long long* __restrict__ keys,
                int* __restrict__ err) {
    extern __shared__ uint8_t dsmem_raw[];
    __shared__ uint64_t bar_full[kStages], bar_ready[kStages], bar_empty[kStages];
    __shared__ uint64_t bar_tfull[2], bar_tempty[2], bar_drain;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ ColCtx s_col[kEpiThreads / 32][kColsPerWarp];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int* sT0 = reinterpret_cast<int*>(dsmem_raw);
    int* sT1 = sT0 + kT0Cap;
    int* sTB = sT1 + kT1Cap;
    uint8_t* stage0 = dsmem_raw + kTabBytes;
    uint8_t* base = stage0 + ((1024 - (tc::smem_u32(stage0) & 1023)) & 1023);
    uint8_t* sA = base;
    uint8_t* sB = base + kStages * kTileBytes;
    uint8_t* sOHb = base + 2 * kStages * kTileBytes;
    const int N0 = tg.N0, N1 = tg.N1, N = N0 + N1, np1 = N + 1;
    volatile int* abort = &s_abort;

    // the layout above must fit the dynamic shared memory this launch received
    uint32_t dyn_bytes;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_bytes));
    const bool fits = N0 < kT0Cap && N1 < kT1Cap && N < kTBCap &&
                      (size_t)(base - dsmem_raw) + kStageBytes <= dyn_bytes;

    if (tid == 0) {
        // an earlier launch failed (skip the work), or the layout has no room (reason 2)
        s_abort = (*(volatile int*)err ? 1 : 0) | (fits ? 0 : 2);
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&bar_full[s], 1);
            tc::mbar_init(&bar_ready[s], kMaskThreads);
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
        for (int i = tid; i <= N0; i += kThreads) sT0[i] = fx_narrow(tab[i], fbits);
        for (int i = tid; i <= N1; i += kThreads) sT1[i] = fx_narrow(tab[np1 + i], fbits);
        for (int i = tid; i <= N; i += kThreads) sTB[i] = fx_narrow(tab[2 * np1 + i], fbits);
    }
    const int N0x4 = 4 * N0, N1x4 = 4 * N1, Nx4 = 4 * N;
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = s_tmem;
    const int n_tiles = n_items * nd;
    const int nkb = tg.nkb;
    if (warp < kEpiWarp0) {
      asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsProducer));
      if (warp == 0) {
        // ------------------------------ TMA producer ------------------------------
        if (lane == 0 && !*abort) {
            uint32_t g = 0;  // running K-block counter across this CTA's tiles
            int pend_mask = 0;
            uint32_t pend_use[kStages] = {0, 0, 0, 0};
            for (int t = blockIdx.x; t < n_tiles && !*abort; t += gridDim.x) {
                const int2 item = items[t % n_items];
                const int d = d0 + t / n_items;
                const int b = item.x, a0 = (item.y >> 16) * kTile, e0 = b + 1 + (item.y & 0xFFFF) * kTile;
                const uint8_t* ohb = oh + ((size_t)d * M + b) * tg.Kp;
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = (int)(g % kStages);
                    const uint32_t use = g / kStages;
                    if (use > 0 && !tc::mbar_wait(&bar_empty[s], (use - 1) & 1, abort)) {
                        ok = false;
                        break;
                    }
                    tc::mbar_arrive_expect_tx(&bar_full[s], 2 * kTileBytes + kBK);
                    tc::tma_load_3d(sA + s * kTileBytes, &map_oh, &bar_full[s], kb * kBK, a0, d);
                    tc::tma_load_3d(sB + s * kTileBytes, &map_oh, &bar_full[s], kb * kBK, e0, d);
                    tc::bulk_load(sOHb + s * kBK, ohb + (size_t)kb * kBK, kBK, &bar_full[s]);
                    pend_mask |= 1 << s;
                    pend_use[s] = use;
                }
                if (!ok) break;
            }
            // the newest copy of every stage completes its phase; waiting for
            // those (bounded) covers every copy this thread issued
            for (int s = 0; s < kStages; ++s)
                if (pend_mask & (1 << s)) mbar_drain(&bar_full[s], pend_use[s] & 1);
        }
      } else if (warp == 1) {
        // ------------------------------ MMA issuer --------------------------------
        if (lane == 0 && !*abort) {
            const uint32_t idesc = tc::idesc_e4m3_f32(kTile, kTile);
            uint32_t g = 0;
            int i = 0;
            bool issued = false;
            for (int t = blockIdx.x; t < n_tiles && !*abort; t += gridDim.x, ++i) {
                const int buf = i & 1;
                const uint32_t tuse = (uint32_t)(i >> 1);
                if (tuse > 0 && !tc::mbar_wait(&bar_tempty[buf], (tuse - 1) & 1, abort)) break;
                tc::tc_fence_after();
                const uint32_t dbase = tmem + (uint32_t)buf * kAccCols;
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = (int)(g % kStages);
                    const uint32_t use = g / kStages;
                    if (!tc::mbar_wait(&bar_ready[s], use & 1, abort)) {
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
            // every MMA this thread issued completes before TMEM and the stages are released
            if (issued) {
                tc::mma_commit(&bar_drain);
                mbar_drain(&bar_drain, 0);
            }
        }
      } else {
        // ------------------------------ A-tile maskers ----------------------------
        // Thread mt owns 16-byte slot (mt & 7) of rows (mt >> 3) + 8 i; since 8
        // divides the row step, its swizzled chunk j = slot ^ (row & 7) and hence
        // its mask chunk are the same for every row it touches.  Rows a >= b
        // are left as loaded: their counts are never used.
        const int mt = tid - kMaskWarp0 * 32;
        const int slot = mt & 7, r0 = mt >> 3;
        const int jchunk = slot ^ (r0 & 7);
        uint32_t g = 0;
        for (int t = blockIdx.x; t < n_tiles && !*abort; t += gridDim.x) {
            const int2 item = items[t % n_items];
            const int a0 = (item.y >> 16) * kTile;
            const int rows = min(kTile, item.x - a0);  // valid rows: a < b
            bool ok = true;
            for (int kb = 0; kb < nkb; ++kb, ++g) {
                const int s = (int)(g % kStages);
                const uint32_t use = g / kStages;
                if (!tc::mbar_wait(&bar_full[s], use & 1, abort)) {
                    ok = false;
                    break;
                }
                uint8_t* A = sA + s * kTileBytes + slot * 16;
                const uint4 m = *reinterpret_cast<const uint4*>(sOHb + s * kBK + jchunk * 16);
#pragma unroll 4
                for (int r = r0; r < rows; r += kMaskThreads / 8) {
                    uint4* p = reinterpret_cast<uint4*>(A + r * kBK);
                    uint4 v = *p;
                    v.x &= m.x;
                    v.y &= m.y;
                    v.z &= m.z;
                    v.w &= m.w;
                    *p = v;
                }
                tc::fence_proxy_async_smem();
                tc::mbar_arrive(&bar_ready[s]);
            }
            if (!ok) break;
        }
      }
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsEpilogue));
        // ------------------------------ epilogue ----------------------------------
        const int ew = warp - kEpiWarp0;      // 0..15
        const int q = warp & 3, h = ew >> 2;  // TMEM lane quarter (warp % 4), column quarter
        const int row = 32 * q + lane;
        const float inv_scale = __int_as_float((127 - fbits) << 23);  // 2^-fbits
        ColCtx* cc = s_col[ew];
        int i = 0;
        for (int t = blockIdx.x; t < n_tiles && !*abort; t += gridDim.x, ++i) {
            const int buf = i & 1;
            const uint32_t tuse = (uint32_t)(i >> 1);
            const int2 item = items[t % n_items];
            const int dl = t / n_items, d = d0 + dl;
            const int b = item.x, a0 = (item.y >> 16) * kTile, e0 = b + 1 + (item.y & 0xFFFF) * kTile;
            const PairC* pd = pairs + (size_t)dl * M * M;  // symmetric: [i][m] == [m][i]
            const int* c1 = cnt1s + (size_t)d * M * 2;
            const int* pm = perm + (size_t)d * M;        // new label -> original variable
            const int ecol0 = e0 + kColsPerWarp * h;
            const int ncols = min(kColsPerWarp, M - ecol0);
            // column context of this warp's columns: pair (b, e) and single e
            __syncwarp();
            for (int cidx = lane; cidx < kColsPerWarp; cidx += 32) {
                const int e = ecol0 + cidx;
                ColCtx x{0, 0, 0, 0, 0, 0};
                if (cidx < ncols) {
                    const PairC p = pd[(size_t)b * M + e];
                    x.n0 = (int)(p.cnt & 0xFFFFu);
                    x.n1 = (int)(p.cnt >> 16);
                    x.sh = p.sh;
                    x.ne0 = 4 * c1[2 * e];
                    x.ne1 = 4 * c1[2 * e + 1];
                    x.eo = pm[e];
                }
                cc[cidx] = x;
            }
            __syncwarp();
            // row context: pair (a, b), single a, and per-row constants (counts times 4)
            const int a = a0 + row;
            const bool arow = a < b;
            const bool warp_rows = (a0 + 32 * q) < b;  // some row of this warp is valid
            int pab0 = 0, pab1 = 0, shab = 0, na0 = 0, na1 = 0, ao = 0;
            if (arow) {
                const PairC p = pd[(size_t)b * M + a];
                pab0 = (int)(p.cnt & 0xFFFFu);
                pab1 = (int)(p.cnt >> 16);
                shab = p.sh;
                na0 = 4 * c1[2 * a];
                na1 = 4 * c1[2 * a + 1];
                ao = pm[a];
            }
            const uint32_t bo = (uint32_t)pm[b];
            const int nb0 = 4 * c1[2 * b], nb1 = 4 * c1[2 * b + 1];
            const int kab0 = N0x4 - na0 - nb0 + pab0, kab1 = N1x4 - na1 - nb1 + pab1;
            const uint32_t dM = (uint32_t)d * (uint32_t)M;
            // pair (a, e) records of the first 8 columns, fetched before the accumulators are ready
            const PairC* prow = pd + (size_t)min(ecol0, M - 1) * M + (arow ? a : 0);  // prow[(e - ecol0) * M]
            PairC pnext[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) pnext[j] = (arow && j < ncols) ? prow[(size_t)j * M] : PairC{0u, 0};

            if (!tc::mbar_wait(&bar_tfull[buf], tuse & 1, abort)) break;
            tc::tc_fence_after();
            // running maxima of the roles a (over e) and b (over this thread's (a, e));
            // the column loop visits e in ascending order, so ">" keeps the lowest e on ties
            int best_a = INT_MIN, best_a_col = -1, best_b = INT_MIN, best_b_col = -1;
            if (warp_rows && ncols > 0) {
                const uint32_t taddr =
                    tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)buf * kAccCols + (uint32_t)(kColsPerWarp * h);
#pragma unroll 1
                for (int c0 = 0; c0 < ncols; c0 += 8) {
                    uint32_t r0[8], r1[8];
                    tc::tmem_ld8(taddr + (uint32_t)c0, r0);
                    tc::tmem_ld8(taddr + (uint32_t)(kTile + c0), r1);
                    PairC pcur[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        pcur[j] = pnext[j];
                        const int cn = c0 + 8 + j;
                        pnext[j] = (arow && cn < ncols) ? prow[(size_t)cn * M] : PairC{0u, 0};
                    }
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int col = c0 + j;
                        const bool ok = arow && col < ncols;
                        int ig_e = INT_MIN;
                        if (ok) {
                            const ColCtx cx = cc[col];
                            const int pae0 = (int)(pcur[j].cnt & 0xFFFFu), pae1 = (int)(pcur[j].cnt >> 16);
                            int sh3, t0, t1, t2, t3, t4, t5, t6, t7;
                            {
                                const int x = count4(r0[j]);
                                const int c011 = cx.n0 - x, c101 = pae0 - x, c110 = pab0 - x;
                                const int c001 = cx.ne0 - pae0 - c011;
                                const int c010 = nb0 - pab0 - c011;
                                const int c100 = na0 - pab0 - c101;
                                const int c000 = kab0 - cx.ne0 + pae0 + c011;
                                sh3 = -(tab4(sT0, x, N0x4) + tab4(sT0, c011, N0x4) + tab4(sT0, c101, N0x4) +
                                        tab4(sT0, c110, N0x4) + tab4(sT0, c001, N0x4) + tab4(sT0, c010, N0x4) +
                                        tab4(sT0, c100, N0x4) + tab4(sT0, c000, N0x4));
                                t7 = x;
                                t3 = c011;
                                t5 = c101;
                                t6 = c110;
                                t1 = c001;
                                t2 = c010;
                                t4 = c100;
                                t0 = c000;
                            }
                            {
                                const int x = count4(r1[j]);
                                const int c011 = cx.n1 - x, c101 = pae1 - x, c110 = pab1 - x;
                                const int c001 = cx.ne1 - pae1 - c011;
                                const int c010 = nb1 - pab1 - c011;
                                const int c100 = na1 - pab1 - c101;
                                const int c000 = kab1 - cx.ne1 + pae1 + c011;
                                sh3 -= tab4(sT1, x, N1x4) + tab4(sT1, c011, N1x4) + tab4(sT1, c101, N1x4) +
                                       tab4(sT1, c110, N1x4) + tab4(sT1, c001, N1x4) + tab4(sT1, c010, N1x4) +
                                       tab4(sT1, c100, N1x4) + tab4(sT1, c000, N1x4);
                                t7 += x;
                                t3 += c011;
                                t5 += c101;
                                t6 += c110;
                                t1 += c001;
                                t2 += c010;
                                t4 += c100;
                                t0 += c000;
                            }
                            sh3 += tab4(sTB, t0, Nx4) + tab4(sTB, t1, Nx4) + tab4(sTB, t2, Nx4) + tab4(sTB, t3, Nx4) +
                                   tab4(sTB, t4, Nx4) + tab4(sTB, t5, Nx4) + tab4(sTB, t6, Nx4) + tab4(sTB, t7, Nx4);
                            // IG(a | b,e), IG(b | a,e), IG(e | a,b): wrap-around int32 differences
                            const int ig_a = cx.sh - sh3;
                            const int ig_b = pcur[j].sh - sh3;
                            ig_e = shab - sh3;
                            if (ig_a > best_a) {
                                best_a = ig_a;
                                best_a_col = col;
                            }
                            if (ig_b > best_b) {
                                best_b = ig_b;
                                best_b_col = col;
                            }
                        }
                        // role e: the column's maximum over the rows (lowest new label a on ties)
                        const int emax = __reduce_max_sync(0xffffffffu, ig_e);
                        if (emax != INT_MIN) {
                            const unsigned src = __reduce_min_sync(0xffffffffu, ig_e == emax ? (unsigned)lane : 32u);
                            const int am = __shfl_sync(0xffffffffu, ao, (int)src);
                            if (lane == 0)
                                atomicMax(keys + cc[col].eo,
                                          pack_key((float)emax * inv_scale, partner_index(dM, M, (uint32_t)am, bo)));
                        }
                    }
                }
            }
            tc::tc_fence_before();
            tc::mbar_arrive(&bar_tempty[buf]);
            if (best_a_col >= 0)  // IG(a | b, e): partners (b, e)
                atomicMax(keys + ao, pack_key((float)best_a * inv_scale,
                                              partner_index(dM, M, bo, (uint32_t)cc[best_a_col].eo)));
            const unsigned long long kb_key =
                best_b_col >= 0 ? pack_key((float)best_b * inv_scale,
                                           partner_index(dM, M, (uint32_t)ao, (uint32_t)cc[best_b_col].eo))
                                : 0ull;
            const unsigned long long mb = warp_max_key(kb_key);  // IG(b | a, e): partners (a, e)
            if (lane == 0 && mb) atomicMax(keys + bo, mb);
        }
    }

    // ---------------- teardown ------------------------------------------------
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, kTmemCols);
    if (tid == 0 && *abort) atomicOr(err, *abort);  // 1: bounded wait gave up, 2: shared layout too small
}

namespace {

// One CTA per discretisation: new labels in ascending order of the bin-1 count
// n0 + n1 (ties by original index), sorted as 32-bit keys (count << 16 | m) by
// a bitonic network in shared memory.  M above kOrderMax keeps the identity.
constexpr int kOrderMax = 8192;

__global__ void __launch_bounds__(1024) k3tc_order_kernel(const int* __restrict__ cnt1, int M, int* __restrict__ perm,
                                                          int* __restrict__ rank, int* __restrict__ cnt1s) {
    extern __shared__ uint32_t skey[];
    const int d = blockIdx.x, tid = threadIdx.x;
    const int* c1 = cnt1 + (size_t)d * M * 2;
    if (M <= kOrderMax) {
        int P2 = 1;
        while (P2 < M) P2 <<= 1;
        for (int i = tid; i < P2; i += blockDim.x)
            skey[i] = i < M ? ((uint32_t)(c1[2 * i] + c1[2 * i + 1]) << 16) | (uint32_t)i : 0xFFFFFFFFu;
        __syncthreads();
        for (int k = 2; k <= P2; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = tid; i < P2; i += blockDim.x) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const uint32_t x = skey[i], y = skey[ixj];
                        if ((x > y) == ((i & k) == 0)) {
                            skey[i] = y;
                            skey[ixj] = x;
                        }
                    }
                }
                __syncthreads();
            }
    }
    for (int r = tid; r < M; r += blockDim.x) {
        const int m = M <= kOrderMax ? (int)(skey[r] & 0xFFFFu) : r;
        perm[(size_t)d * M + r] = m;
        rank[(size_t)d * M + m] = r;
        cnt1s[((size_t)d * M + r) * 2] = c1[2 * m];
        cnt1s[((size_t)d * M + r) * 2 + 1] = c1[2 * m + 1];
    }
}

// dst row (d, r) = src row (d, perm[d][r]); rows of Kp bytes, Kp a multiple of 16
__global__ void __launch_bounds__(128) permute_rows_kernel(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst,
                                                           const int* __restrict__ perm, int M, int Kp) {
    const int r = blockIdx.x, d = blockIdx.y;
    const int m = perm[(size_t)d * M + r];
    const uint4* s4 = reinterpret_cast<const uint4*>(src + ((size_t)d * M + m) * Kp);
    uint4* d4 = reinterpret_cast<uint4*>(dst + ((size_t)d * M + r) * Kp);
    for (int i = threadIdx.x; i < Kp / 16; i += blockDim.x) d4[i] = s4[i];
}

}  // namespace

cudaError_t launch_k3tc_order(const int* cnt1, int M, int D, int* perm, int* rank, int* cnt1s, cudaStream_t st) {
    if (M > 65535) return cudaErrorInvalidValue;
    int P2 = 1;
    while (P2 < M) P2 <<= 1;
    const size_t smem = M <= kOrderMax ? (size_t)P2 * sizeof(uint32_t) : 0;
    k3tc_order_kernel<<<D, 1024, smem, st>>>(cnt1, M, perm, rank, cnt1s);
    return cudaGetLastError();
}

cudaError_t launch_permute_rows(const uint8_t* src, uint8_t* dst, const int* perm, int M, int D, int Kp,
                                cudaStream_t st) {
    if (Kp % 16 != 0 || ((uintptr_t)src & 15) || ((uintptr_t)dst & 15)) return cudaErrorInvalidValue;
    permute_rows_kernel<<<dim3(M, D), 128, 0, st>>>(src, dst, perm, M, Kp);
    return cudaGetLastError();
}

void build_k3tc_items(int M, std::vector<int2>& items) {
    items.clear();
    for (int b = 1; b + 1 < M; ++b) {
        const int nta = (b + kTile - 1) / kTile;
        const int nte = (M - 1 - b + kTile - 1) / kTile;
        for (int ta = 0; ta < nta; ++ta)
            for (int te = 0; te < nte; ++te) items.push_back(make_int2(b, (ta << 16) | te));
    }
}

// fixed-capacity tables + stages + alignment slack; 0 if the tables exceed their capacity
size_t k3tc_smem_bytes(int N0, int N1) {
    if (N0 >= kT0Cap || N1 >= kT1Cap || N0 + N1 >= kTBCap) return (size_t)-1;
    return kTabBytes + 1024 + kStageBytes;
}

// Largest fraction bits s <= 20 with |IG| 2^s < 2^31 for N samples
// (|IG| <= N ln 2 plus pseudocount terms, bounded here by N ln 2 + 64).
int k3tc_fraction_bits(int N) {
    const double bound = (double)N * 0.6931471805599453 + 64.0;
    int s = 20;
    while (s > 1 && bound * (double)(1 << s) >= 2147483647.0) --s;
    return s;
}

TcGeom make_tc_geom(int N0, int N1) {
    TcGeom t;
    t.N0 = N0;
    t.N1 = N1;
    t.K0p = (N0 + kBK - 1) / kBK * kBK;
    t.Kp = t.K0p + (N1 + kBK - 1) / kBK * kBK;
    t.nkb0 = t.K0p / kBK;
    t.nkb = t.Kp / kBK;
    return t;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    // resolved once (thread-safe static initialisation)
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
        return nullptr;
    }();
    return fn;
}

// One-hot operand [D][rows][Kp] bytes as a 3-D tensor map with 128 x 128 boxes
// and the 128-byte swizzle that the UMMA descriptors expect.
cudaError_t make_onehot_map(CUtensorMap* map, const uint8_t* oh, int rows, int D, int Kp) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    if (((uintptr_t)oh & 15) != 0 || (Kp % 128) != 0) return cudaErrorInvalidValue;
    cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)D};
    cuuint64_t strides[2] = {(cuuint64_t)Kp, (cuuint64_t)Kp * (cuuint64_t)rows};
    cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)kTile, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, (void*)oh, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_k3tc(const CUtensorMap& map, const uint8_t* oh, TcGeom tg, int M, int d0, int nd,
                        const int2* items, int n_items, const long long* tab, int fbits, const int* cnt1s,
                        const int* perm, const PairC* pairs, unsigned long long* keys, int* err, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    const size_t smem = k3tc_smem_bytes(tg.N0, tg.N1);
    cudaError_t e = ensure_dynamic_smem((const void*)k3tc_kernel, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const long long n_tiles = (long long)n_items * nd;
    if (n_tiles >= (1ll << 31)) return cudaErrorInvalidValue;
    // the register split inside the kernel needs exactly kRegsLaunch registers per thread
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, k3tc_kernel)) != cudaSuccess) return e;
    if (fa.numRegs != kRegsLaunch) return cudaErrorInvalidConfiguration;
    const int grid = (int)std::min<long long>(n_tiles, (long long)sms);
    k3tc_kernel<<<grid, kThreads, smem, st>>>(map, oh, tg, M, d0, nd, items, n_items, tab, fbits, cnt1s, perm, pairs,
                                              keys, err);
    return cudaGetLastError();
}

}  // namespace mdfs
