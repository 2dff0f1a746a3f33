// k = 3 scan for two classes per variable (c = 2) on the 5th-generation tensor
// cores (tcgen05, kind::f8f6f4).  Voxel counters of section "Algorithm and
// implementation"; IG roles of Eq. 1 with |S| = 2.
//
// Each variable's bin-1 indicator over the class-sorted samples is stored as
// one-hot E4M3 bytes: 1.0 for a class-0 sample, 64.0 for a class-1 sample, 0
// outside bin 1.  For a middle variable b, the all-ones voxel of every triple
// (a, b, e) is counted by
//     X[a][e] = sum_s OH[a][s] * OH[b][s] * OH[e][s] = n0 + 4096 n1,
// a GEMM with A = OH[a-tile] masked by OH[b] and B = OH[e-tile], both K-major.
// Products are 0, 1 or 4096, and with n0, n1 < 4096 every partial sum is an
// integer below 2^24, so the FP32 accumulator holds both class counts exactly.
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
// Work item: (b, a tile of 128 rows, e group of up to 256 columns); one MMA
// per 32 samples, N = the group's columns rounded up to 16 (256 for a full
// group), reuses the masked A tile across the whole group.
//
// Persistent, warp-specialised kernel (one CTA per SM, 640 threads):
//   warp 0       TMA producer: A (a rows), B (e rows), OH[b] row per K block,
//   warp 1       TMEM owner and MMA issuer (4 MMAs of K = 32 per K block),
//   warps 2-3    AND the A tile with OH[b] in shared memory (128B swizzle),
//   warps 4-19   epilogue: tcgen05.ld of the accumulator, the 8-voxel tables
//                by inclusion-exclusion, SH3 from fixed-point tables in shared
//                memory, three IG roles, packed max keys.
// Registers: launched at kRegsLaunch per thread; the first warpgroup gives
// back to kRegsProducer, the four epilogue warpgroups take kRegsEpilogue
// (128 kRegsProducer + 512 kRegsEpilogue == 640 kRegsLaunch).
// Three shared-memory stages and two TMEM accumulator buffers (2 x 256
// columns) let the epilogue of one item overlap the MMAs of the next.
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
#include <algorithm>
#include <climits>
#include <cmath>
#include <queue>
#include <utility>
#include <vector>

#include "mdfs_device.cuh"
#include "mdfs_internal.cuh"
#include "mdfs_tc.cuh"

namespace mdfs {

namespace {

constexpr int kTile = 128;                     // a rows
constexpr int kTileE = 256;                    // e columns of a wide group
constexpr int kBK = 128;                       // K bytes (samples) per stage
constexpr int kStages = 3;
constexpr uint32_t kTileBytes = kTile * kBK;   // 16 KB: A, or one 128-row half of B
constexpr uint32_t kBBytes = 2 * kTileBytes;   // B stage: up to 256 rows
constexpr uint32_t kAccCols = kTileE;          // one FP32 accumulator column per e
constexpr uint32_t kTmemCols = 2 * kAccCols;   // double buffer
constexpr int kThreads = 640;
constexpr int kMaskWarp0 = 2, kMaskThreads = 64;
constexpr int kEpiWarp0 = 4, kEpiThreads = 512;
// Tiles are claimed by the producer and handed to the other roles, in order,
// through a ring of tile ids in shared memory; every slot is released by the
// MMA thread, each masker thread and each epilogue warp.
constexpr int kRing = 8;
constexpr int kRingReaders = 1 + kMaskThreads + kEpiThreads / 32;
constexpr int kChunk = 32;                     // e columns per epilogue pass of a warp
constexpr int kGroup = 4;                      // columns per TMEM load; pair records prefetched one group ahead
constexpr int kRegsLaunch = 96, kRegsProducer = 32, kRegsEpilogue = 112;
constexpr uint8_t kClass1Byte = 0x68;          // E4M3 64.0
static_assert(128 * kRegsProducer + kEpiThreads * kRegsEpilogue == kThreads * kRegsLaunch,
              "register split must add up to the launch allocation");
// Dynamic shared memory layout (byte offsets from its start):
//   [align1024(0), +48 KB)        A stages
//   [kT0Off, +16 KB)              T0: int32 entries 0..4095 (class 0)
//   [kT1Off, +16 KB)              T1: class 1
//   [kTBOff, +32 KB)              TB: entries 0..8191 (both classes)
//   [align1024(kTabEnd), +96 KB)  B stages, then the OH[b] rows
// The tables sit at fixed offsets, so a lookup is one load with an immediate
// base.  Every table offset the epilogue forms from counts in [0, 4096) lies in
// [-32 KB, +32 KB) of T0/T1 and in [-64 KB, +64 KB) of TB; those windows lie
// inside the layout, so lookups need no clamp: inconsistent counts can only
// read wrong values, never leave shared memory.
constexpr int kT0Cap = 4096, kT1Cap = 4096, kTBCap = 8192;
constexpr uint32_t kAStageBytes = kStages * kTileBytes;                // 48 KB
constexpr uint32_t kT0Off = kAStageBytes + 1024;                       // after A and its alignment slack
constexpr uint32_t kT1Off = kT0Off + kT0Cap * 4;
constexpr uint32_t kTBOff = kT1Off + kT1Cap * 4;
constexpr uint32_t kTabEnd = kTBOff + kTBCap * 4;
static_assert(kT0Off >= 32768 && kTBOff >= 65536, "guard windows below the tables");
static_assert(kTBOff + 65536 <= kTabEnd + kStages * 2 * kTileBytes, "guard window above TB");
constexpr size_t kDynBytes = kTabEnd + 1024 + kStages * (kBBytes + kBK);  // + B stages, OH[b] rows
// dynamic + static (column contexts, barriers) within the 227 KB a block may opt in to on sm_103a
static_assert(kDynBytes + (size_t)(kEpiThreads / 32) * kChunk * (16 + 8) + 256 <= 232448, "shared memory layout");

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

// table entry at shared-window byte address `addr`.  Not volatile: the tables
// are read-only once built, so the compiler may reorder and overlap the loads
// of several voxels and columns.
__device__ __forceinline__ int lds(uint32_t addr) {
    int v;
    asm("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// every count (times 4) in [0, 16380] and a multiple of 4: the range the
// guard windows of the table layout are sized for
__device__ __forceinline__ bool counts_ok(int any_or) { return (any_or & (int)0xFFFFC003u) == 0; }

// Per-column constants of an item, in two shared arrays per epilogue warp (n_x:
// class count of bin 1 of x, n_xy: class count of the voxel (1, 1) of the pair
// (x, y)): nu = per class (n_be, n_e - n_be) + beta of the class (smoothed
// counts), class 0 then class 1; sht = (SH(b, e), role-e key threshold) in LB
// units (K3Prune, key_threshold).  The exact path, taken for few columns,
// reads SH(b, e) and the original index of e from global memory.

// Bound that lets the epilogue skip the exact SH3 of most triples.  Each
// voxel's term of SH is E(m0, m1) = f(m0 + m1) - f(m0) - f(m1) with the
// smoothed class counts m_d = n_d + beta_d; E = (m0 + m1) H(m0 / (m0 + m1)) with
// H the binary entropy in nats, and H(p) >= 4 ln 2 p (1 - p) gives
//     SH3 >= 4 ln 2 sum_v m0_v m1_v / (m0_v + m1_v) = 4 ln 2 LB.
// IG(x | S) = SH(S) - SH3 can raise x's key only if SH3 <= SH(S) - thr_x, so a
// triple with LB above (SH(S) - thr_x) / (4 ln 2 2^s) for all three roles
// cannot change any result and its 24 table lookups are skipped.  SH values
// are compared as their int32 fixed-point values, which equal the true values
// when (N + 8 (beta0 + beta1)) ln 2 2^s < 2^31 (on = 0 otherwise).  Float
// rounding of LB (relative < 1e-5) and of the thresholds (absolute < 1e-3)
// lies far inside the margins kBoundRel |hi| + kBoundAbs.
struct K3Prune {
    int on;
    float beta0, beta1;  // pseudocounts of the two decision classes
    float fx_to_count;   // 1 / (4 ln 2 2^s): int32 fixed point -> LB units
    float count_to_fx;   // 4 ln 2 2^s
};
constexpr float kBoundRel = 1.0f / 4096.0f, kBoundAbs = 0.05f;

// Two fractions per lane pair: (pa / sa) + (pb / sb) as num / den in each lane (sa, sb > 0).
__device__ __forceinline__ void frac_add2(float2 pa, float2 sa, float2 pb, float2 sb, float2& num, float2& den) {
    num = fma2(pa, sb, mul2(pb, sa));
    den = mul2(sa, sb);
}

// Lower bound, in int32 fixed point with fbits fraction bits, of the IG values
// that can still raise a key whose current value is `key` (0: no value yet).
// Converting an int to float moves it by at most 128 for |v| < 2^31, so any v
// whose float value reaches the key's IG is >= the bound.
__device__ __forceinline__ int key_threshold(unsigned long long key, int fbits) {
    if (key == 0ull) return INT_MIN;
    const float t = order_bits_float((uint32_t)(key >> 32)) * __int_as_float((127 + fbits) << 23);
    if (!(t < 2.0e9f)) return INT_MAX;
    if (t < -2.0e9f) return INT_MIN;
    return __float2int_rd(t) - 256;
}

// First a row of a-tile ta of middle variable b.  The a range [0, b) is tiled
// from 0 upward for even b and from b downward for odd b (a0 may then be
// negative: TMA fills those rows with zeros and the epilogue skips them).
// TMEM lane quarter q, the rows 32 q .. 32 q + 31 of the accumulator, is read
// by the warps of one SM sub-partition; alternating the alignment spreads the
// partial tiles' valid rows evenly over the four quarters.
__host__ __device__ __forceinline__ int tile_a0(int b, int ta) { return (b & 1) ? b - kTile * (ta + 1) : kTile * ta; }


// partner index of a key: (d M + lo) M + hi with the two partners sorted
__device__ __forceinline__ uint32_t partner_index(uint32_t dM, int M, uint32_t p, uint32_t q) {
    return (dM + min(p, q)) * (uint32_t)M + max(p, q);
}

// lexicographic rank of x < y < z among the C(M, 3) triples of [0, M)
__device__ __forceinline__ unsigned long long triple_rank(int M, int x, int y, int z) {
    auto c2 = [](long long n) { return n < 2 ? 0ll : n * (n - 1) / 2; };
    auto c3 = [](long long n) { return n < 3 ? 0ll : n * (n - 1) * (n - 2) / 6; };
    return (unsigned long long)(c3(M) - c3(M - x) + c2(M - x - 1) - c2(M - y) + (z - y - 1));
}

// Test hook: the 8 voxel counts (times 4) of the triple (a, b, e) of original
// variables, kernel voxel order (v_a v_b v_e) = 111, 011, 101, 110, 001, 010,
// 100, 000, written as n0 | n1 << 16 at dump[(d C(M,3) + rank) 8 + v] with v =
// 4 v_lo + 2 v_mid + v_hi in the sorted order lo < mid < hi.
struct Vox8 {
    int v[8];
};
__device__ __noinline__ void dump_triple(uint32_t* dump, int M, int d, int a, int b, int e, Vox8 n0, Vox8 n1) {
    const int lo = min(a, min(b, e)), hi = max(a, max(b, e)), mid = a + b + e - lo - hi;
    const int wa = 4 >> ((a > b) + (a > e)), wb = 4 >> ((b > a) + (b > e)), we = 4 >> ((e > a) + (e > b));
    const unsigned long long c3 = (unsigned long long)M * (M - 1) * (M - 2) / 6;
    uint32_t* o = dump + ((unsigned long long)d * c3 + triple_rank(M, lo, mid, hi)) * 8;
    const int va[8] = {1, 0, 1, 1, 0, 0, 1, 0}, vb[8] = {1, 1, 0, 1, 0, 1, 0, 0}, ve[8] = {1, 1, 1, 0, 1, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < 8; ++j)
        o[va[j] * wa + vb[j] * wb + ve[j] * we] = (uint32_t)(n0.v[j] >> 2) | ((uint32_t)(n1.v[j] >> 2) << 16);
}

}  // namespace

// kMode 1 (kDump): also write the 8-voxel class counts of every triple to
// `dump` (test hook; the scan itself is unchanged).  kMode 2 (kEmit): also
// insert every role whose IG reaches emit_thr (int32 fixed point, fbits
// fraction bits) into the interesting-tuple table `emit`, keyed by the
// original variable and its two partners ascending, valued by the packed (IG,
// discretisation); the SH3 bound then also keeps every triple whose roles can
// reach emit_thr.  wait_ns bounds every mbarrier wait;
// withhold_kb >= 0 makes the producer of CTA 0 skip the copies of that K block
// of its running count (test hook: the consumers' bounded wait then runs out).
template <int kMode>
__global__ void __launch_bounds__(kThreads, 1)
    k3tc_kernel(const __grid_constant__ CUtensorMap map_oh, const uint8_t* __restrict__ oh, TcGeom tg, int M, int d0,
                int nd, const int2* __restrict__ items, int n_items, const long long* __restrict__ tab, int fbits,
                const int* __restrict__ cnt1s, const int* __restrict__ perm, const PairC* __restrict__ pairs,
                unsigned long long* __restrict__ keys, int* __restrict__ err, K3Prune prune,
                uint32_t* __restrict__ dump, unsigned long long wait_ns, int withhold_kb, EmitTable emit,
                int emit_thr, const int* __restrict__ order, int* __restrict__ claim) {
    constexpr bool kDump = kMode == 1, kEmit = kMode == 2;
    extern __shared__ uint8_t dsmem_raw[];
    __shared__ uint64_t bar_full[kStages], bar_ready[kStages], bar_empty[kStages];
    __shared__ uint64_t bar_tfull[2], bar_tempty[2], bar_drain;
    __shared__ uint64_t bar_rfull[kRing], bar_rempty[kRing];
    __shared__ int s_ring[kRing];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ float4 s_nu[kEpiThreads / 32][kChunk];
    __shared__ float2 s_sht[kEpiThreads / 32][kChunk];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int* sT0 = reinterpret_cast<int*>(dsmem_raw + kT0Off);
    int* sT1 = reinterpret_cast<int*>(dsmem_raw + kT1Off);
    int* sTB = reinterpret_cast<int*>(dsmem_raw + kTBOff);
    const uint32_t uT0 = tc::smem_u32(sT0), uT1 = tc::smem_u32(sT1), uTB = tc::smem_u32(sTB);
    const uint32_t tb_off = uTB - uT0 - uT1;  // TB address of a voxel = T0 address + T1 address + tb_off
    uint8_t* sA = dsmem_raw + ((1024 - (tc::smem_u32(dsmem_raw) & 1023)) & 1023);
    uint8_t* sB = dsmem_raw + kTabEnd + ((1024 - (tc::smem_u32(dsmem_raw + kTabEnd) & 1023)) & 1023);
    uint8_t* sOHb = sB + kStages * kBBytes;
    const int N0 = tg.N0, N1 = tg.N1, N = N0 + N1, np1 = N + 1;
    volatile int* abort = &s_abort;

    // the layout above must fit the dynamic shared memory this launch received
    uint32_t dyn_bytes;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_bytes));
    const bool fits = N0 < kT0Cap && N1 < kT1Cap && N < kTBCap &&
                      (size_t)(sOHb - dsmem_raw) + kStages * kBK <= dyn_bytes &&
                      (size_t)(sA - dsmem_raw) + kAStageBytes <= kT0Off;

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
        for (int j = 0; j < kRing; ++j) {
            tc::mbar_init(&bar_rfull[j], 1);
            tc::mbar_init(&bar_rempty[j], kRingReaders);
        }
        tc::mbar_fence_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(&s_tmem, kTmemCols);
        tc::tmem_relinquish();
    }
    if (fits) {  // whole regions: entries past N_c are zero
        for (int i = tid; i < kT0Cap; i += kThreads) sT0[i] = i <= N0 ? fx_narrow(tab[i], fbits) : 0;
        for (int i = tid; i < kT1Cap; i += kThreads) sT1[i] = i <= N1 ? fx_narrow(tab[np1 + i], fbits) : 0;
        for (int i = tid; i < kTBCap; i += kThreads) sTB[i] = i <= N ? fx_narrow(tab[2 * np1 + i], fbits) : 0;
    }
    const int N0x4 = 4 * N0, N1x4 = 4 * N1;  // class sizes, times 4
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = s_tmem;
    const int n_tiles = n_items * nd;
    const int nkb = tg.nkb;
    volatile int* ring = s_ring;
    // The j-th tile of this CTA from the ring: waits (bounded) for the producer
    // to publish it, reads it, releases the slot; -1 when none is left or a
    // wait gave up.  Every reader takes every tile.
    auto ring_take = [&](int j) -> int {
        const int slot = j % kRing;
        if (!tc::mbar_wait(&bar_rfull[slot], (uint32_t)(j / kRing) & 1, abort, wait_ns)) return -1;
        const int t = ring[slot];
        tc::mbar_arrive(&bar_rempty[slot]);
        return t;
    };
    if (warp < kEpiWarp0) {
      asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsProducer));
      if (warp == 0) {
        // ------------------------------ TMA producer ------------------------------
        if (lane == 0 && !*abort) {
            const int withhold = blockIdx.x == 0 ? withhold_kb : -1;
            uint32_t g = 0;  // running K-block counter across this CTA's tiles
            int pend_mask = 0;
            uint32_t pend_use[kStages] = {};
            // claims: the first tile by block index, then from the shared counter
            // (dynamic; a fixed stride without one), in the order of `order`
            // (descending cost; the identity without one)
            int idx = blockIdx.x;
            for (int j = 0;; ++j) {
                const int slot = j % kRing;
                if (j >= kRing && !tc::mbar_wait(&bar_rempty[slot], (uint32_t)(j / kRing - 1) & 1, abort, wait_ns))
                    break;
                const int t = (idx < n_tiles && !*abort) ? (order ? __ldg(order + idx) : idx) : -1;
                ring[slot] = t;
                tc::mbar_arrive(&bar_rfull[slot]);
                if (t < 0) break;
                idx = claim ? (int)gridDim.x + atomicAdd(claim, 1) : idx + (int)gridDim.x;
                const int2 item = items[t % n_items];
                const int d = d0 + t / n_items;
                const int b = item.x, a0 = tile_a0(b, item.y >> 16), e0 = b + 1 + (item.y & 0xFFFF) * kTileE;
                const bool wide = M - e0 > kTile;  // second 128-row half of B needed
                const uint8_t* ohb = oh + ((size_t)d * M + b) * tg.Kp;
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = (int)(g % kStages);
                    const uint32_t use = g / kStages;
                    if (use > 0 && !tc::mbar_wait(&bar_empty[s], (use - 1) & 1, abort, wait_ns)) {
                        ok = false;
                        break;
                    }
                    if ((int)g == withhold) continue;  // test hook: this stage is never filled
                    tc::mbar_arrive_expect_tx(&bar_full[s], (wide ? 3 : 2) * kTileBytes + kBK);
                    tc::tma_load_3d(sA + s * kTileBytes, &map_oh, &bar_full[s], kb * kBK, a0, d);
                    tc::tma_load_3d(sB + s * kBBytes, &map_oh, &bar_full[s], kb * kBK, e0, d);
                    if (wide) tc::tma_load_3d(sB + s * kBBytes + kTileBytes, &map_oh, &bar_full[s], kb * kBK, e0 + kTile, d);
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

            uint32_t g = 0;
            bool issued = false;
            for (int i = 0;; ++i) {
                const int t = ring_take(i);
                if (t < 0 || *abort) break;
                const int buf = i & 1;
                const uint32_t tuse = (uint32_t)(i >> 1);
                const int2 item = items[t % n_items];
                const int e0 = item.x + 1 + (item.y & 0xFFFF) * kTileE;
                // the group's columns rounded up to the MMA's N granularity of 16 (the
                // accumulator columns past them are never read)
                const int ncol = min(kTileE, (M - e0 + 15) & ~15);
                const uint32_t idesc = tc::idesc_e4m3_f32(kTile, max(16, ncol));
                if (tuse > 0 && !tc::mbar_wait(&bar_tempty[buf], (tuse - 1) & 1, abort, wait_ns)) break;
                tc::tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)buf * kAccCols;
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = (int)(g % kStages);
                    const uint32_t use = g / kStages;
                    if (!tc::mbar_wait(&bar_ready[s], use & 1, abort, wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t a_addr = tc::smem_u32(sA + s * kTileBytes);
                    const uint32_t b_addr = tc::smem_u32(sB + s * kBBytes);
#pragma unroll
                    for (int kk = 0; kk < kBK / 32; ++kk) {
                        const uint32_t acc = kb > 0 || kk > 0;
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
        for (int j = 0;; ++j) {
            const int t = ring_take(j);
            if (t < 0 || *abort) break;
            const int2 item = items[t % n_items];
            const int a0 = tile_a0(item.x, item.y >> 16);
            const int rows = min(kTile, item.x - a0);  // rows with a < b (rows with a < 0 hold zeros)
            bool ok = true;
            for (int kb = 0; kb < nkb; ++kb, ++g) {
                const int s = (int)(g % kStages);
                const uint32_t use = g / kStages;
                if (!tc::mbar_wait(&bar_full[s], use & 1, abort, wait_ns)) {
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
        // Warp (q, h): TMEM lane quarter q = warp % 4 (rows 32 q ..), column
        // chunks h and h + 4 of 32 columns each.
        const int ew = warp - kEpiWarp0;      // 0..15
        const int q = warp & 3, h = ew >> 2;
        const int row = 32 * q + lane;
        const float inv_scale = __int_as_float((127 - fbits) << 23);  // 2^-fbits
        float4* cnu = s_nu[ew];
        float2* csht = s_sht[ew];
        bool bad = false;       // inconsistent row or column constants
        uint32_t badbits = 0;   // OR of the pair records' count fields (checked at the end)
        for (int i = 0;; ++i) {
            // the tile, warp-uniform: every lane waits, lane 0 releases the slot
            const int slot = i % kRing;
            if (!__all_sync(0xffffffffu, tc::mbar_wait(&bar_rfull[slot], (uint32_t)(i / kRing) & 1, abort, wait_ns)))
                break;
            const int t = __shfl_sync(0xffffffffu, ring[slot], 0);
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&bar_rempty[slot]);
            if (t < 0 || __any_sync(0xffffffffu, *abort != 0)) break;
            const int buf = i & 1;
            const uint32_t tuse = (uint32_t)(i >> 1);
            const int2 item = items[t % n_items];
            const int dl = t / n_items, d = d0 + dl;
            const int b = item.x, a0 = tile_a0(b, item.y >> 16), e0 = b + 1 + (item.y & 0xFFFF) * kTileE;
            const PairC* pd = pairs + (size_t)dl * M * M;  // symmetric: [i][m] == [m][i]
            const int* c1 = cnt1s + (size_t)d * M * 2;
            const int* pm = perm + (size_t)d * M;        // new label -> original variable
            // row constants (counts times 4): n_ab, n_b - n_ab, n_a - n_ab, N - n_a - n_b + n_ab
            const int a = a0 + row;
            const bool arow = a >= 0 && a < b;
            const bool warp_rows = (a0 + 32 * q) < b && (a0 + 32 * q + 31) >= 0;  // some row of this warp is valid
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
            int r2_0 = nb0 - pab0, r2_1 = nb1 - pab1;
            int r3_0 = na0 - pab0, r3_1 = na1 - pab1;
            int kab0 = N0x4 - na0 - nb0 + pab0, kab1 = N1x4 - na1 - nb1 + pab1;
            if (!counts_ok(pab0 | pab1 | na0 | na1 | r2_0 | r2_1 | r3_0 | r3_1 | kab0 | kab1)) {
                // inconsistent inputs: reported through the error flag; the
                // zeroed constants keep every table offset inside its window
                bad = true;
                pab0 = pab1 = r2_0 = r2_1 = r3_0 = r3_1 = kab0 = kab1 = 0;
            }
            // The constants carry the table base addresses (once, or twice where a
            // voxel count subtracts another biased constant), so each voxel's byte
            // address in T0 / T1 is one add or subtract away, and its address in TB
            // is the sum of the two plus tb_off.
            const uint32_t A110 = uT0 + pab0, A010 = 2 * uT0 + r2_0, A100 = 2 * uT0 + r3_0, A000 = 2 * uT0 + kab0;
            const uint32_t B110 = uT1 + pab1, B010 = 2 * uT1 + r2_1, B100 = 2 * uT1 + r3_1, B000 = 2 * uT1 + kab1;
            // The same row constants as smoothed class counts for the SH3 bound,
            // paired per class as the voxel pairs below need them: (n_ab + beta,
            // n_a - n_ab + beta) and (n_b - n_ab + 2 beta, N - n_a - n_b + n_ab + 2 beta).
            const float fb0 = prune.beta0, fb1 = prune.beta1;
            const float2 beta0 = make_float2(fb0, fb0), beta1 = make_float2(fb1, fb1);
            const float2 rpr3_0 = make_float2(fmaf((float)pab0, 0.25f, fb0), fmaf((float)r3_0, 0.25f, fb0));
            const float2 rpr3_1 = make_float2(fmaf((float)pab1, 0.25f, fb1), fmaf((float)r3_1, 0.25f, fb1));
            const float2 r2k_0 = make_float2(fmaf((float)r2_0, 0.25f, 2.0f * fb0), fmaf((float)kab0, 0.25f, 2.0f * fb0));
            const float2 r2k_1 = make_float2(fmaf((float)r2_1, 0.25f, 2.0f * fb1), fmaf((float)kab1, 0.25f, 2.0f * fb1));
            // role thresholds in LB units: IG(e | a,b) can raise e's key only if
            // SH3 <= SH(a,b) - thr_e, IG(a | b,e) only if SH3 <= SH(b,e) - thr_a,
            // IG(b | a,e) only if SH3 <= SH(a,e) - thr_b
            const float shab_c = (float)shab * prune.fx_to_count;
            // (with emission: the lower of the key's and the emission threshold)
            int thra = arow ? key_threshold(__ldcg(keys + ao), fbits) : 0;
            int thrb = key_threshold(__ldcg(keys + bo), fbits);
            if constexpr (kEmit) {
                thra = min(thra, emit_thr);
                thrb = min(thrb, emit_thr);
            }
            const float thra_c = (float)thra * prune.fx_to_count;
            const float thrb_c = (float)thrb * prune.fx_to_count;
            const uint32_t dM = (uint32_t)d * (uint32_t)M;
            // running maxima of the roles a (over e) and b (over this thread's (a, e));
            // columns are visited in ascending e, so ">" keeps the first maximum
            int best_a = INT_MIN, best_b = INT_MIN;
            int best_a_eo = 0, best_b_eo = 0;
            bool waited = false;
#pragma unroll 1
            for (int ch = h;; ch += 4) {
                const int ecol0 = e0 + kChunk * ch;
                const int ncols = ch < kTileE / kChunk ? min(kChunk, M - ecol0) : 0;
                const PairC* prow = pd + (size_t)min(ecol0, M - 1) * M + (arow ? a : 0);  // prow[(e - ecol0) * M]
                PairC pnext[kGroup];
                if (ncols > 0) {
                    // column constants of this chunk
                    __syncwarp();
                    const int e = ecol0 + lane;
                    int n0 = 0, n1 = 0, u0 = 0, u1 = 0, thr = INT_MAX, esh = 0;
                    if (lane < ncols) {
                        const PairC p = pd[(size_t)b * M + e];
                        n0 = (int)(p.cnt & 0xFFFFu);
                        n1 = (int)(p.cnt >> 16);
                        u0 = 4 * c1[2 * e] - n0;
                        u1 = 4 * c1[2 * e + 1] - n1;
                        esh = p.sh;
                        // keys only grow during the scan: a stale value is a valid lower bound
                        thr = key_threshold(__ldcg(keys + pm[e]), fbits);
                        if constexpr (kEmit) thr = min(thr, emit_thr);
                        if (!counts_ok(n0 | n1 | u0 | u1)) {
                            bad = true;
                            n0 = n1 = u0 = u1 = 0;
                        }
                    }
                    cnu[lane] = make_float4(fmaf((float)n0, 0.25f, fb0), fmaf((float)u0, 0.25f, fb0),
                                            fmaf((float)n1, 0.25f, fb1), fmaf((float)u1, 0.25f, fb1));
                    csht[lane] = make_float2((float)esh * prune.fx_to_count, (float)thr * prune.fx_to_count);
                    __syncwarp();
                    // pair (a, e) records of the first group, fetched before the accumulator is read
#pragma unroll
                    for (int j = 0; j < kGroup; ++j)
                        pnext[j] = (arow && j < ncols) ? prow[(size_t)j * M] : PairC{0u, 0};
                }
                // every epilogue warp waits for the accumulator of every item, with
                // or without columns, before it releases the buffer
                if (!waited) {
                    // warp-uniform outcome: the warp-wide reductions below need every lane
                    if (!__all_sync(0xffffffffu, tc::mbar_wait(&bar_tfull[buf], tuse & 1, abort, wait_ns))) break;
                    tc::tc_fence_after();
                    waited = true;
                }
                if (ncols <= 0) break;
                if (!warp_rows) continue;
                int ca = -1, cb = -1;  // columns of this chunk that raised best_a, best_b
                const uint32_t taddr =
                    tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)buf * kAccCols + (uint32_t)(kChunk * ch);
#pragma unroll 1
                for (int c0 = 0; c0 < ncols; c0 += kGroup) {
                    uint32_t r[kGroup];
                    tc::tmem_ld(taddr + (uint32_t)c0, r);
                    PairC pcur[kGroup];
#pragma unroll
                    for (int j = 0; j < kGroup; ++j) {
                        pcur[j] = pnext[j];
                        const int cn = c0 + kGroup + j;
                        pnext[j] = (arow && cn < ncols) ? prow[(size_t)cn * M] : PairC{0u, 0};
                    }
                    tc::tmem_ld_wait();
                    // Which (a, e) of the group need the exact SH3: those where the
                    // lower bound of SH3 does not already rule out all three roles.
                    unsigned need = 0;
#pragma unroll
                    for (int j = 0; j < kGroup; ++j) {
                        badbits |= pcur[j].cnt;
                        const bool valid = arow && c0 + j < ncols;
                        if (kDump || !prune.on) {
                            need |= valid ? 1u << j : 0u;
                            continue;
                        }
                        const float4 nu = cnu[c0 + j];
                        const float2 sht = csht[c0 + j];
                        const float2 nu0 = make_float2(nu.x, nu.y), nu1 = make_float2(nu.z, nu.w);
                        // class counts of the voxel (1,1,1): X = n0 + 4096 n1, exact in FP32
                        const float X = __uint_as_float(r[j]);
                        // floor(X / 4096): 2^23 + X 2^-12 rounded toward zero (exact product, one rounding)
                        const float x1 = __fmaf_rz(X, 1.0f / 4096.0f, 8388608.0f) - 8388608.0f;
                        const float x0 = fmaf(x1, -4096.0f, X);
                        // pair (a, e) class counts: 4 n in 16-bit fields, read as floats
                        const float q0 = fmaf(__uint_as_float((pcur[j].cnt & 0xFFFFu) | 0x4B000000u), 0.25f,
                                              -2097152.0f);
                        const float q1 = fmaf(__uint_as_float((pcur[j].cnt >> 16) | 0x4B000000u), 0.25f,
                                              -2097152.0f);
                        // per class, (x, t) with t = n_ae - x, and the smoothed class counts
                        // of four voxel pairs (v_a v_b v_e):
                        //   va = (011, 001) = (n_be, n_e - n_be) - (x, t)
                        //   vb = (110, 100) = (n_ab, n_a - n_ab) - (x, t)
                        //   vc = (111, 101) = (x, t) + beta
                        //   vd = (010, 000) = (n_b - n_ab, N - n_a - n_b + n_ab) - (n_be, n_e - n_be) + (x, t)
                        // (each constant carries its beta, twice where one is subtracted)
                        const float2 xt0 = make_float2(x0, q0 - x0), xt1 = make_float2(x1, q1 - x1);
                        const float2 va0 = sub2(nu0, xt0), va1 = sub2(nu1, xt1);
                        const float2 vb0 = sub2(rpr3_0, xt0), vb1 = sub2(rpr3_1, xt1);
                        const float2 vc0 = add2(xt0, beta0), vc1 = add2(xt1, beta1);
                        const float2 vd0 = add2(sub2(r2k_0, nu0), xt0), vd1 = add2(sub2(r2k_1, nu1), xt1);
                        // sum over the voxels of m w / (m + w) (m, w the two classes' smoothed
                        // counts), accumulated as one fraction per lane of the pairs
                        float2 nab, dab, ncd, dcd, num2, den2;
                        frac_add2(mul2(va0, va1), add2(va0, va1), mul2(vb0, vb1), add2(vb0, vb1), nab, dab);
                        frac_add2(mul2(vc0, vc1), add2(vc0, vc1), mul2(vd0, vd1), add2(vd0, vd1), ncd, dcd);
                        frac_add2(nab, dab, ncd, dcd, num2, den2);
                        const float num = fmaf(num2.x, den2.y, num2.y * den2.x), den = den2.x * den2.y;
                        // largest SH3 (LB units) that still lets one role reach its bound
                        const float sh_ae = (float)pcur[j].sh * prune.fx_to_count;
                        const float hi = fmaxf(fmaxf(sht.x - thra_c, sh_ae - thrb_c), shab_c - sht.y);
                        const float lim = fmaf(fabsf(hi), kBoundRel, hi + kBoundAbs);
                        need |= (valid && num <= lim * den) ? 1u << j : 0u;
                    }
                    if (!__any_sync(0xffffffffu, need != 0)) continue;
#pragma unroll
                    for (int j = 0; j < kGroup; ++j) {
                        if (!__any_sync(0xffffffffu, (need >> j) & 1u)) continue;
                        const int col = c0 + j;
                        const bool valid = arow && col < ncols;
                        const float4 cxn = cnu[col];
                        const float cx_thr_c = csht[col].y;
                        // SH(b, e) and the original index of e (rows and columns outside the
                        // item read the last column's and are masked out below)
                        const int ecol = min(ecol0 + col, M - 1);
                        const int cx_sh = pd[(size_t)b * M + ecol].sh;
                        const int cx_eo = pm[ecol];
                        // exact column counts (times 4), recovered from the smoothed floats
                        const uint32_t cn0 = 4u * (uint32_t)__float2int_rn(cxn.x - fb0);
                        const uint32_t cu0 = 4u * (uint32_t)__float2int_rn(cxn.y - fb0);
                        const uint32_t cn1 = 4u * (uint32_t)__float2int_rn(cxn.z - fb1);
                        const uint32_t cu1 = 4u * (uint32_t)__float2int_rn(cxn.w - fb1);
                        const uint32_t n0b = uT0 + cn0, n1b = uT1 + cn1, u0b = 2 * uT0 + cu0, u1b = 2 * uT1 + cu1;
                        const uint32_t pae0 = pcur[j].cnt & 0x3FFCu, pae1 = (pcur[j].cnt >> 16) & 0x3FFCu;
                        // X = n0 + 4096 n1, exact in FP32
                        const uint32_t xv = (uint32_t)__float2int_rn(__uint_as_float(r[j]));
                        const uint32_t x0 = (xv << 2) & 0x3FFCu, x1 = (xv >> 10) & 0x3FFCu;
                        // byte addresses of the voxels (v_a v_b v_e) by inclusion-exclusion
                        const uint32_t a111 = uT0 + x0, a011 = n0b - x0, a110 = A110 - x0, a101 = uT0 + pae0 - x0;
                        const uint32_t a001 = u0b - a101, a010 = A010 - n0b + x0, a100 = A100 - a101;
                        const uint32_t a000 = A000 - u0b + a101;
                        const uint32_t b111 = uT1 + x1, b011 = n1b - x1, b110 = B110 - x1, b101 = uT1 + pae1 - x1;
                        const uint32_t b001 = u1b - b101, b010 = B010 - n1b + x1, b100 = B100 - b101;
                        const uint32_t b000 = B000 - u1b + b101;
                        // straight-line for every lane: rows and columns outside the item
                        // compute in-window garbage that is masked out below
                        const int sh3 = (lds(a111 + b111 + tb_off) + lds(a011 + b011 + tb_off) +
                                         lds(a101 + b101 + tb_off) + lds(a110 + b110 + tb_off) +
                                         lds(a001 + b001 + tb_off) + lds(a010 + b010 + tb_off) +
                                         lds(a100 + b100 + tb_off) + lds(a000 + b000 + tb_off)) -
                                        (lds(a111) + lds(a011) + lds(a101) + lds(a110) + lds(a001) + lds(a010) +
                                         lds(a100) + lds(a000)) -
                                        (lds(b111) + lds(b011) + lds(b101) + lds(b110) + lds(b001) + lds(b010) +
                                         lds(b100) + lds(b000));
                        if constexpr (kDump) {
                            if (valid)
                                dump_triple(dump, M, d, ao, (int)bo, cx_eo,
                                            {(int)(a111 - uT0), (int)(a011 - uT0), (int)(a101 - uT0),
                                             (int)(a110 - uT0), (int)(a001 - uT0), (int)(a010 - uT0),
                                             (int)(a100 - uT0), (int)(a000 - uT0)},
                                            {(int)(b111 - uT1), (int)(b011 - uT1), (int)(b101 - uT1),
                                             (int)(b110 - uT1), (int)(b001 - uT1), (int)(b010 - uT1),
                                             (int)(b100 - uT1), (int)(b000 - uT1)});
                        }
                        // IG(a | b,e), IG(b | a,e), IG(e | a,b): wrap-around int32 differences
                        const int ig_a = cx_sh - sh3;
                        const int ig_b = pcur[j].sh - sh3;
                        const int ig_e = valid ? shab - sh3 : INT_MIN;
                        if constexpr (kEmit) {
                            if (valid) {
                                const int lo_be = min((int)bo, cx_eo), hi_be = max((int)bo, cx_eo);
                                const int lo_ae = min(ao, cx_eo), hi_ae = max(ao, cx_eo);
                                const int lo_ab = min(ao, (int)bo), hi_ab = max(ao, (int)bo);
                                if (ig_a >= emit_thr)
                                    emit_insert(emit, emit_key(ao, lo_be, hi_be, -1),
                                                pack_key((float)ig_a * inv_scale, (uint32_t)d));
                                if (ig_b >= emit_thr)
                                    emit_insert(emit, emit_key((int)bo, lo_ae, hi_ae, -1),
                                                pack_key((float)ig_b * inv_scale, (uint32_t)d));
                                if (ig_e >= emit_thr)
                                    emit_insert(emit, emit_key(cx_eo, lo_ab, hi_ab, -1),
                                                pack_key((float)ig_e * inv_scale, (uint32_t)d));
                            }
                        }
                        if (valid && ig_a > best_a) {
                            best_a = ig_a;
                            ca = col;
                        }
                        if (valid && ig_b > best_b) {
                            best_b = ig_b;
                            cb = col;
                        }
                        // role e: the column's maximum over the warp's rows, written by the
                        // lowest lane (lowest new label a) holding it; skipped when no lane
                        // reaches the column's key threshold (taken 1024 units low: the
                        // float form of the threshold is not exact)
                        const float thr_fx = fmaf(cx_thr_c, prune.count_to_fx, -1024.0f);
                        if (__any_sync(0xffffffffu, valid && (float)ig_e >= thr_fx)) {
                            const int emax = __reduce_max_sync(0xffffffffu, ig_e);
                            const unsigned hit = __ballot_sync(0xffffffffu, ig_e == emax);
                            if (lane == __ffs(hit) - 1)
                                atomicMax(keys + cx_eo,
                                          pack_key((float)emax * inv_scale, partner_index(dM, M, (uint32_t)ao, bo)));
                        }
                    }
                }
                if (ca >= 0) best_a_eo = pm[ecol0 + ca];
                if (cb >= 0) best_b_eo = pm[ecol0 + cb];
            }
            if (!waited) break;  // the accumulator wait gave up
            tc::tc_fence_before();
            tc::mbar_arrive(&bar_tempty[buf]);
            if (best_a != INT_MIN)  // IG(a | b, e): partners (b, e)
                atomicMax(keys + ao, pack_key((float)best_a * inv_scale, partner_index(dM, M, bo, (uint32_t)best_a_eo)));
            const unsigned long long kb_key =
                best_b != INT_MIN
                    ? pack_key((float)best_b * inv_scale, partner_index(dM, M, (uint32_t)ao, (uint32_t)best_b_eo))
                    : 0ull;
            const unsigned long long mb = warp_max_key(kb_key);  // IG(b | a, e): partners (a, e)
            if (lane == 0 && mb) atomicMax(keys + bo, mb);
        }
        // a pair count outside [0, 4096) was masked into range above: report it
        if ((badbits & 0xC003C003u) != 0) bad = true;
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(err, 4);
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

// nonzero bytes of w -> kClass1Byte, zero bytes stay zero
__device__ __forceinline__ uint32_t recode_class1(uint32_t w) {
    uint32_t nz = w | (w >> 4);
    nz |= nz >> 2;
    nz |= nz >> 1;
    return (nz & 0x01010101u) * kClass1Byte;
}

// dst row (d, r) = src row (d, perm[d][r]); rows of Kp bytes, Kp a multiple of
// 16.  Bytes from K0p on (class-1 samples, K0p a multiple of 16) become 64.0.
__global__ void __launch_bounds__(128) permute_rows_kernel(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst,
                                                           const int* __restrict__ perm, int M, int Kp, int K0p) {
    const int r = blockIdx.x, d = blockIdx.y;
    const int m = perm[(size_t)d * M + r];
    const uint4* s4 = reinterpret_cast<const uint4*>(src + ((size_t)d * M + m) * Kp);
    uint4* d4 = reinterpret_cast<uint4*>(dst + ((size_t)d * M + r) * Kp);
    for (int i = threadIdx.x; i < Kp / 16; i += blockDim.x) {
        uint4 v = s4[i];
        if (i >= K0p / 16) {
            v.x = recode_class1(v.x);
            v.y = recode_class1(v.y);
            v.z = recode_class1(v.z);
            v.w = recode_class1(v.w);
        }
        d4[i] = v;
    }
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

cudaError_t launch_k3tc_operand(const uint8_t* src, uint8_t* dst, const int* perm, int M, int D, TcGeom tg,
                                cudaStream_t st) {
    if (tg.Kp % 16 != 0 || tg.K0p % 16 != 0 || ((uintptr_t)src & 15) || ((uintptr_t)dst & 15))
        return cudaErrorInvalidValue;
    permute_rows_kernel<<<dim3(M, D), 128, 0, st>>>(src, dst, perm, M, tg.Kp, tg.K0p);
    return cudaGetLastError();
}

void build_k3tc_items(int M, std::vector<int2>& items) {
    items.clear();
    for (int b = 1; b + 1 < M; ++b) {
        const int nta = (b + kTile - 1) / kTile;
        const int nte = (M - 1 - b + kTileE - 1) / kTileE;
        for (int ta = 0; ta < nta; ++ta)
            for (int te = 0; te < nte; ++te) items.push_back(make_int2(b, (ta << 16) | te));
    }
}

// Relative cost of a tile: its epilogue work, the warps (32-row quarters of the
// a tile) with a valid row times the valid e columns, as a fraction of a full
// item, but at least the main loop's (the same K blocks for every item,
// overlapped with the epilogue of the previous one).  The floor was measured:
// launch times are flat for floors of 0.6 to 0.9 of a full item, 2-4 % longer
// at 0.25-0.4, and at 1.0 (every tile alike) as long as the fixed stride.
static double tile_cost(int M, int2 item) {
    const int b = item.x, a0 = tile_a0(b, item.y >> 16), e0 = b + 1 + (item.y & 0xFFFF) * kTileE;
    int warps = 0;
    for (int q = 0; q < 4; ++q) warps += (a0 + 32 * q < b && a0 + 32 * q + 31 >= 0) ? 1 : 0;
    const int cols = std::min(kTileE, M - e0);
    return std::max(0.75, (double)warps * 32.0 * cols / ((double)kTile * kTileE));
}

// Claim order of the n_items * nd tiles (tile t: item t % n_items of
// discretisation t / n_items): descending cost, ties by index.  CTAs claim the
// next tile of this list when their producer is ready for one, so the heavy
// tiles go first and the light ones fill the end (a dynamic
// longest-processing-time schedule).
void build_k3tc_order(int M, const int2* items, int n_items, int nd, std::vector<int>& out) {
    const int n_tiles = n_items * nd;
    std::vector<double> cost(n_items);
    for (int i = 0; i < n_items; ++i) cost[i] = tile_cost(M, items[i]);
    out.resize(n_tiles);
    for (int t = 0; t < n_tiles; ++t) out[t] = t;
    std::stable_sort(out.begin(), out.end(), [&](int x, int y) { return cost[x % n_items] > cost[y % n_items]; });
}

// the fixed layout above; (size_t)-1 if the tables exceed their capacity
size_t k3tc_smem_bytes(int N0, int N1) {
    if (N0 >= kT0Cap || N1 >= kT1Cap || N0 + N1 >= kTBCap) return (size_t)-1;
    return kDynBytes;
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

// Byte tensor (dims[0] contiguous, strides in bytes of dims 1 .. rank-1) as a
// tiled tensor map with the 128-byte swizzle; box[0] must be 128 bytes.
cudaError_t make_tiled_map_u8(CUtensorMap* map, const void* base, int rank, const cuuint64_t* dims,
                              const cuuint64_t* strides, const cuuint32_t* box) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    if (rank < 2 || rank > 5 || ((uintptr_t)base & 15) != 0 || box[0] != 128) return cudaErrorInvalidValue;
    for (int i = 0; i < rank - 1; ++i)
        if (strides[i] % 16 != 0) return cudaErrorInvalidValue;
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
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
                        const int* perm, const PairC* pairs, unsigned long long* keys, int* err, double b0, double b1,
                        cudaStream_t st, uint32_t* dump, TcTestHooks hooks, EmitTable emit, const int* order,
                        int* claim) {
    if (n_items == 0) return cudaSuccess;
    if (dump && emit.keys) return cudaErrorInvalidValue;
    const size_t smem = k3tc_smem_bytes(tg.N0, tg.N1);
    const void* fn = dump        ? (const void*)k3tc_kernel<1>
                     : emit.keys ? (const void*)k3tc_kernel<2>
                                 : (const void*)k3tc_kernel<0>;
    cudaError_t e = ensure_dynamic_smem(fn, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const long long n_tiles = (long long)n_items * nd;
    if (n_tiles >= (1ll << 31)) return cudaErrorInvalidValue;
    // the register split inside the kernel needs exactly kRegsLaunch registers per thread
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
    if (fa.numRegs != kRegsLaunch) return cudaErrorInvalidConfiguration;
    const int grid = (int)std::min<long long>(n_tiles, (long long)sms);
    if (claim && (e = cudaMemsetAsync(claim, 0, sizeof(int), st)) != cudaSuccess) return e;
    const unsigned long long wait_ns = hooks.wait_ns ? hooks.wait_ns : tc::kWaitLimitNs;
    K3Prune prune;
    const double scale = 4.0 * 0.6931471805599453 * std::ldexp(1.0, fbits);
    prune.on = !hooks.exact && !dump && b0 >= 1e-3 && b1 >= 1e-3 &&
               ((double)(tg.N0 + tg.N1) + 8.0 * (b0 + b1)) * 0.6931471805599453 * std::ldexp(1.0, fbits) <
                   2147483647.0;
    prune.beta0 = (float)b0;
    prune.beta1 = (float)b1;
    prune.fx_to_count = (float)(1.0 / scale);
    prune.count_to_fx = (float)scale;
    const int emit_thr = emit_threshold_fx(emit, fbits);
    if (dump)
        k3tc_kernel<1><<<grid, kThreads, smem, st>>>(map, oh, tg, M, d0, nd, items, n_items, tab, fbits, cnt1s, perm,
                                                     pairs, keys, err, prune, dump, wait_ns, hooks.withhold_kb, emit,
                                                     emit_thr, order, claim);
    else if (emit.keys)
        k3tc_kernel<2><<<grid, kThreads, smem, st>>>(map, oh, tg, M, d0, nd, items, n_items, tab, fbits, cnt1s, perm,
                                                     pairs, keys, err, prune, nullptr, wait_ns, hooks.withhold_kb,
                                                     emit, emit_thr, order, claim);
    else
        k3tc_kernel<0><<<grid, kThreads, smem, st>>>(map, oh, tg, M, d0, nd, items, n_items, tab, fbits, cnt1s, perm,
                                                     pairs, keys, err, prune, nullptr, wait_ns, hooks.withhold_kb,
                                                     emit, emit_thr, order, claim);
    return cudaGetLastError();
}

}  // namespace mdfs
