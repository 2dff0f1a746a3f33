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
// Block = one (b, 128 a, 128 e) tile, 256 threads:
//   thread 0   issues the TMA loads of A, B (128B-swizzled) and OH[b] per K block,
//   all        AND the A tile with OH[b] in shared memory,
//   thread 32  issues 4 MMAs (K = 32 each) per K block and commits,
//   all        read the accumulators back (tcgen05.ld) and run the entropy
//              epilogue: 8-voxel tables by inclusion-exclusion, SH3 from the
//              fixed-point tables in shared memory, three IG roles, packed max.
// Every mbarrier wait is bounded; on timeout the block records an error,
// drains its copies and MMAs, frees TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "mdfs_device.cuh"
#include "mdfs_internal.cuh"
#include "mdfs_tc.cuh"

namespace mdfs {

namespace {

constexpr int kTile = 128;               // a rows, e columns
constexpr int kBK = 128;                 // K bytes (samples) per stage
constexpr int kStages = 2;
constexpr uint32_t kTileBytes = kTile * kBK;  // 16 KB
constexpr uint32_t kTmemCols = 256;      // two classes x 128 columns
constexpr int kThreads = 256;
constexpr size_t kTabOffset = 2 * kStages * kTileBytes + kStages * kBK;  // after A, B, OH[b] rows

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) { return a > b ? a : b; }

// Waits for completion regardless of an abort (draining in-flight copies/MMAs);
// still bounded in time.
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

}  // namespace

__global__ void __launch_bounds__(kThreads, 2)
    k3tc_kernel(const __grid_constant__ CUtensorMap map_oh, const uint8_t* __restrict__ oh, TcGeom tg, int M, int d0,
                const int2* __restrict__ items, const long long* __restrict__ tab, const int* __restrict__ cnt1,
                const Pair2* __restrict__ pairs, unsigned long long* __restrict__ keys, int* __restrict__ err) {
    extern __shared__ uint8_t dsmem_raw[];
    __shared__ uint64_t bar_full[kStages], bar_ready[kStages], bar_empty[kStages], bar_done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort, s_committed;
    __shared__ Pair2 s_pbe[kTile];
    __shared__ int2 s_ne[kTile];
    __shared__ unsigned long long s_ka[kTile], s_ke[kTile], s_kb;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t* base = dsmem_raw + ((1024 - (tc::smem_u32(dsmem_raw) & 1023)) & 1023);
    uint8_t* sA = base;
    uint8_t* sB = base + kStages * kTileBytes;
    uint8_t* sOHb = base + 2 * kStages * kTileBytes;
    const int N0 = tg.N0, N1 = tg.N1, N = N0 + N1, np1 = N + 1;
    long long* sT0 = reinterpret_cast<long long*>(base + kTabOffset);
    long long* sT1 = sT0 + (N0 + 1);
    long long* sTB = sT1 + (N1 + 1);

    const int2 item = items[blockIdx.x];
    const int b = item.x;
    const int a0 = (item.y >> 16) * kTile;
    const int e0 = b + 1 + (item.y & 0xFFFF) * kTile;
    const int dl = blockIdx.y, d = d0 + dl;
    const Pair2* pd = pairs + (size_t)dl * M * M;  // symmetric: [i][m] == [m][i]
    const int* c1 = cnt1 + (size_t)d * M * 2;
    volatile int* abort = &s_abort;

    // the layout above must fit the dynamic shared memory this launch received
    uint32_t dyn_bytes;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_bytes));
    const bool fits = (size_t)(base - dsmem_raw) + kTabOffset + (size_t)(2 * N + 3) * sizeof(long long) <= dyn_bytes;
    if (!fits) {
        sT0 = sT1 = sTB = nullptr;  // never dereferenced: the block aborts below
    }

    if (tid == 0) {
        // an earlier block failed (skip the work), or the layout has no room (reason 2)
        s_abort = (*(volatile int*)err ? 1 : 0) | (fits ? 0 : 2);
        s_committed = 0;
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&bar_full[s], 1);
            tc::mbar_init(&bar_ready[s], kThreads);
            tc::mbar_init(&bar_empty[s], 1);
        }
        tc::mbar_init(&bar_done, 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, kTmemCols);
        tc::tmem_relinquish();
    }
    if (fits) {
        for (int i = tid; i <= N0; i += kThreads) sT0[i] = tab[i];
        for (int i = tid; i <= N1; i += kThreads) sT1[i] = tab[np1 + i];
        for (int i = tid; i <= N; i += kThreads) sTB[i] = tab[2 * np1 + i];
    }
    for (int r = tid; r < kTile; r += kThreads) {
        const int e = e0 + r;
        const bool ok = e < M;
        s_pbe[r] = ok ? pd[(size_t)b * M + e] : Pair2{0, 0, 0};
        s_ne[r] = ok ? make_int2(c1[2 * e], c1[2 * e + 1]) : make_int2(0, 0);
        s_ke[r] = 0ull;
        s_ka[r] = 0ull;
    }
    if (tid == 0) s_kb = 0ull;
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = s_tmem;

    // ---------------- main loop: TMA -> mask -> MMA -------------------------
    int pending = 0;                 // thread 0: stages with a TMA not yet observed complete
    uint32_t pending_use[kStages] = {0, 0};
    bool mma_issued = false;         // thread 32
    const uint32_t idesc = tc::idesc_e4m3_f32(kTile, kTile);
    if (!*abort) {
        for (int kb = 0; kb < tg.nkb; ++kb) {
            if (*abort) break;
            const int s = kb % kStages;
            const uint32_t use = (uint32_t)(kb / kStages);
            if (tid == 0) {
                bool ok = true;
                if (kb >= kStages) ok = tc::mbar_wait(&bar_empty[s], (use - 1) & 1, abort);
                if (ok) {
                    tc::mbar_arrive_expect_tx(&bar_full[s], 2 * kTileBytes + kBK);
                    tc::tma_load_3d(sA + s * kTileBytes, &map_oh, &bar_full[s], kb * kBK, a0, d);
                    tc::tma_load_3d(sB + s * kTileBytes, &map_oh, &bar_full[s], kb * kBK, e0, d);
                    tc::bulk_load(sOHb + s * kBK, oh + ((size_t)d * M + b) * tg.Kp + (size_t)kb * kBK, kBK,
                                  &bar_full[s]);
                    pending |= 1 << s;
                    pending_use[s] = use;
                }
            }
            if (!tc::mbar_wait(&bar_full[s], use & 1, abort)) break;
            if (tid == 0) pending &= ~(1 << s);
            {
                uint8_t* A = sA + s * kTileBytes;
                const uint8_t* mrow = sOHb + s * kBK;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int idx = tid + kThreads * i;
                    const int r = idx >> 3, slot = idx & 7;
                    const int j = slot ^ (r & 7);  // 128-byte swizzle: chunk slot = chunk ^ (row % 8)
                    uint4* p = reinterpret_cast<uint4*>(A + r * kBK + slot * 16);
                    const uint4 m = *reinterpret_cast<const uint4*>(mrow + j * 16);
                    uint4 v = *p;
                    v.x &= m.x;
                    v.y &= m.y;
                    v.z &= m.z;
                    v.w &= m.w;
                    *p = v;
                }
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&bar_ready[s]);
            if (tid == 32) {
                if (!tc::mbar_wait(&bar_ready[s], use & 1, abort)) break;
                tc::tc_fence_after();
                const uint32_t d_tmem = tmem + (kb >= tg.nkb0 ? (uint32_t)kTile : 0u);
                const uint32_t a_addr = tc::smem_u32(sA + s * kTileBytes);
                const uint32_t b_addr = tc::smem_u32(sB + s * kTileBytes);
#pragma unroll
                for (int kk = 0; kk < kBK / 32; ++kk) {
                    const uint32_t acc = (kb != 0 && kb != tg.nkb0) || kk > 0;
                    tc::mma_f8(d_tmem, tc::sw128_kmajor_desc(a_addr + 32 * kk), tc::sw128_kmajor_desc(b_addr + 32 * kk),
                               idesc, acc);
                }
                tc::mma_commit(&bar_empty[s]);
                mma_issued = true;
            }
        }
    }
    // ---------------- drain -------------------------------------------------
    if (tid == 32) {
        if (mma_issued) tc::mma_commit(&bar_done);
        s_committed = mma_issued ? 1 : 0;
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s)
            if (pending & (1 << s)) mbar_drain(&bar_full[s], pending_use[s] & 1);
    }
    __syncthreads();
    if (s_committed) mbar_drain(&bar_done, 0);
    tc::tc_fence_after();
    __syncthreads();

    // ---------------- epilogue ----------------------------------------------
    if (!*abort && s_committed) {
        const int q = warp & 3, h = warp >> 2;
        const int row = 32 * q + lane;
        const int a = a0 + row;
        const bool arow = a < b;
        const Pair2 pab = arow ? pd[(size_t)b * M + a] : Pair2{0, 0, 0};
        const int na0 = arow ? c1[2 * a] : 0, na1 = arow ? c1[2 * a + 1] : 0;
        const int nb0 = c1[2 * b], nb1 = c1[2 * b + 1];
        const uint32_t dM = (uint32_t)d * (uint32_t)M;
        unsigned long long ka = 0ull, kbest = 0ull;
#pragma unroll 1
        for (int chunk = 0; chunk < 2; ++chunk) {
            const int cbase = 64 * h + 32 * chunk;
            uint32_t r0[32], r1[32];
            tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)cbase, r0);
            tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(kTile + cbase), r1);
            tc::tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int col = cbase + j;
                const int e = e0 + col;
                unsigned long long k_e = 0ull;
                if (arow && e < M) {
                    const int x0 = (int)__uint_as_float(r0[j]);
                    const int x1 = (int)__uint_as_float(r1[j]);
                    const Pair2 pbe = s_pbe[col];
                    const int2 ne = s_ne[col];
                    const Pair2 pae = pd[(size_t)e * M + a];
                    long long sh3 = 0;
                    int t[8];
                    {
                        int v[8];
                        v[7] = x0;
                        v[3] = pbe.n0 - x0;
                        v[5] = pae.n0 - x0;
                        v[6] = pab.n0 - x0;
                        v[1] = ne.x - pae.n0 - pbe.n0 + x0;
                        v[2] = nb0 - pab.n0 - pbe.n0 + x0;
                        v[4] = na0 - pab.n0 - pae.n0 + x0;
                        v[0] = N0 - na0 - nb0 - ne.x + pab.n0 + pae.n0 + pbe.n0 - x0;
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            sh3 -= sT0[clamp_count(v[u], N0)];
                            t[u] = v[u];
                        }
                    }
                    {
                        int v[8];
                        v[7] = x1;
                        v[3] = pbe.n1 - x1;
                        v[5] = pae.n1 - x1;
                        v[6] = pab.n1 - x1;
                        v[1] = ne.y - pae.n1 - pbe.n1 + x1;
                        v[2] = nb1 - pab.n1 - pbe.n1 + x1;
                        v[4] = na1 - pab.n1 - pae.n1 + x1;
                        v[0] = N1 - na1 - nb1 - ne.y + pab.n1 + pae.n1 + pbe.n1 - x1;
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            sh3 -= sT1[clamp_count(v[u], N1)];
                            t[u] += v[u];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) sh3 += sTB[clamp_count(t[u], N)];
                    // IG(a | b,e), IG(b | a,e), IG(e | a,b)
                    const unsigned long long k_a =
                        pack_key(fx_to_float(pbe.sh - sh3), (dM + (uint32_t)b) * (uint32_t)M + (uint32_t)e);
                    const unsigned long long k_b =
                        pack_key(fx_to_float(pae.sh - sh3), (dM + (uint32_t)a) * (uint32_t)M + (uint32_t)e);
                    k_e = pack_key(fx_to_float(pab.sh - sh3), (dM + (uint32_t)a) * (uint32_t)M + (uint32_t)b);
                    ka = umax64(ka, k_a);
                    kbest = umax64(kbest, k_b);
                }
                const unsigned long long m = warp_max_key(k_e);
                if (lane == 0 && m) atomicMax(&s_ke[col], m);
            }
        }
        if (ka) atomicMax(&s_ka[row], ka);
        const unsigned long long mb = warp_max_key(kbest);
        if (lane == 0 && mb) atomicMax(&s_kb, mb);
    }
    __syncthreads();
    if (!*abort && s_committed) {
        if (tid == 0 && s_kb) atomicMax(keys + b, s_kb);
        for (int r = tid; r < kTile; r += kThreads) {
            if (s_ka[r]) atomicMax(keys + a0 + r, s_ka[r]);
            if (s_ke[r]) atomicMax(keys + e0 + r, s_ke[r]);
        }
    }
    // ---------------- teardown ----------------------------------------------
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
    if (tid == 0 && *abort) atomicOr(err, *abort);  // 1: bounded wait gave up, 2: shared layout too small
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

// stages + tables T0[0..N0], T1[0..N1], TB[0..N0+N1] + alignment slack
size_t k3tc_smem_bytes(int N0, int N1) {
    return kTabOffset + (size_t)(2 * (N0 + N1) + 3) * sizeof(long long) + 1024;
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
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    }
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
                        const int2* items, int n_items, const long long* tab, const int* cnt1, const Pair2* pairs,
                        unsigned long long* keys, int* err, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    const size_t smem = k3tc_smem_bytes(tg.N0, tg.N1);
    cudaError_t e = cudaFuncSetAttribute(k3tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(n_items, nd);
    k3tc_kernel<<<grid, kThreads, smem, st>>>(map, oh, tg, M, d0, items, tab, cnt1, pairs, keys, err);
    return cudaGetLastError();
}

}  // namespace mdfs
