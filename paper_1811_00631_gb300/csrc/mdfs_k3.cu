// k = 3 scan for two classes per variable (c = 2): the triple counting kernel
// of the MDFS scan (Eq. 1 with |S| = 2; voxel counters of section "Algorithm
// and implementation").
//
// A block takes the middle variable b of the triples a < b < e, a tile of 64
// variables a and a tile of 64 variables e.  For every 32-word chunk of the
// class-sorted bit planes it stages P_a & P_b (64 rows) and P_e (64 rows) in
// shared memory; each thread owns a 4 x 4 micro-tile of (a, e) and counts
// popc(P_a & P_b & P_e) with a Harley-Seal carry-save tree over groups of four
// words (one POPC per four words instead of four).  The class-0 and class-1
// word ranges give the two class counts of the voxel (1,1,1); the other seven
// voxels follow from the pair and single counts by inclusion-exclusion.  The
// regularised entropy SH({a,b,e}) is a sum of 24 fixed-point table entries
// (tables in shared memory), and the three roles
//     IG(a | b,e) = SH(b,e) - SH(a,b,e),  IG(b | a,e),  IG(e | a,b)
// are folded into the per-variable packed max keys.
#include "mdfs_device.cuh"
#include "mdfs_internal.cuh"

namespace mdfs {

namespace {

constexpr int TA = 64, TE = 64, WC = 32, LDW = WC + 4;

// carry-save adder: (hi, lo) = a + b + c bitwise
__device__ __forceinline__ void csa(uint32_t& hi, uint32_t& lo, uint32_t a, uint32_t b, uint32_t c) {
    const uint32_t u = a ^ b;
    hi = (a & b) | (u & c);
    lo = u ^ c;
}

struct HS {
    uint32_t ones, twos;
    int fours;
};

__device__ __forceinline__ void hs_add4(HS& s, uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3) {
    uint32_t twos_a, twos_b, fours;
    csa(twos_a, s.ones, s.ones, x0, x1);
    csa(twos_b, s.ones, s.ones, x2, x3);
    csa(fours, s.twos, s.twos, twos_a, twos_b);
    s.fours += __popc(fours);
}

__device__ __forceinline__ int hs_total(const HS& s) { return 4 * s.fours + 2 * __popc(s.twos) + __popc(s.ones); }

__device__ __forceinline__ long long tab_get(const long long* t, int n, int nmax) { return t[clamp_count(n, nmax)]; }

}  // namespace

// items[j] = (b, ta << 16 | te): a in [ta*64, ta*64 + 64) with a < b, e in
// [b + 1 + te*64, b + 1 + te*64 + 64) with e < M.
__global__ void __launch_bounds__(256, 2) k3c2_kernel(const uint32_t* __restrict__ planes, PlaneGeom g, int M, int d0,
                                                      const int2* __restrict__ items, const long long* __restrict__ tab,
                                                      const int* __restrict__ cnt1, const Pair2* __restrict__ pairs,
                                                      unsigned long long* __restrict__ keys) {
    extern __shared__ __align__(16) long long s_tab[];  // [3][N+1]: T0, T1, TB
    __shared__ __align__(16) uint32_t sab[TA][LDW];
    __shared__ __align__(16) uint32_t se[TE][LDW];
    __shared__ uint32_t sb[WC];
    __shared__ Pair2 s_pab[TA], s_pbe[TE];
    __shared__ int2 s_na[TA], s_ne[TE];
    __shared__ unsigned long long s_ka[TA], s_ke[TE], s_kb;

    const int2 item = items[blockIdx.x];
    const int b = item.x;
    const int a0 = (item.y >> 16) * TA;
    const int e0 = b + 1 + (item.y & 0xFFFF) * TE;
    const int dl = blockIdx.y, d = d0 + dl;
    const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
    const int np1 = g.N + 1;
    const uint32_t* pbase = planes + (size_t)d * M * g.Ws;
    const Pair2* pd = pairs + (size_t)dl * M * M;
    const int* c1 = cnt1 + (size_t)d * M * 2;

    // block context: tables, pair records, single counts, key slots
    for (int i = tid; i < 3 * np1; i += 256) s_tab[i] = tab[i];
    for (int r = tid; r < TA; r += 256) {
        const int a = a0 + r;
        const bool ok = a < b;
        s_pab[r] = ok ? pairs[((size_t)dl * M + a) * M + b] : Pair2{0, 0, 0};
        s_na[r] = ok ? make_int2(c1[2 * a], c1[2 * a + 1]) : make_int2(0, 0);
        s_ka[r] = 0ull;
    }
    for (int r = tid; r < TE; r += 256) {
        const int e = e0 + r;
        const bool ok = e < M;
        s_pbe[r] = ok ? pd[(size_t)b * M + e] : Pair2{0, 0, 0};
        s_ne[r] = ok ? make_int2(c1[2 * e], c1[2 * e + 1]) : make_int2(0, 0);
        s_ke[r] = 0ull;
    }
    if (tid == 0) s_kb = 0ull;

    int X[2][4][4];
#pragma unroll
    for (int cls = 0; cls < 2; ++cls) {
        HS st[4][4];
#pragma unroll
        for (int ra = 0; ra < 4; ++ra)
#pragma unroll
            for (int re = 0; re < 4; ++re) st[ra][re] = HS{0u, 0u, 0};
        const int wb = cls == 0 ? 0 : g.W0, we = cls == 0 ? g.W0 : g.W;
        for (int w0 = wb; w0 < we; w0 += WC) {
            const int nw = min(WC, we - w0);
            __syncthreads();
            if (tid < WC) sb[tid] = tid < nw ? pbase[(size_t)b * g.Ws + w0 + tid] : 0u;
            __syncthreads();
            for (int idx = tid; idx < TA * WC; idx += 256) {
                const int w = idx & (WC - 1), r = idx >> 5;
                const int a = a0 + r;
                sab[r][w] = (w < nw && a < b) ? (pbase[(size_t)a * g.Ws + w0 + w] & sb[w]) : 0u;
            }
            for (int idx = tid; idx < TE * WC; idx += 256) {
                const int w = idx & (WC - 1), r = idx >> 5;
                const int e = e0 + r;
                se[r][w] = (w < nw && e < M) ? pbase[(size_t)e * g.Ws + w0 + w] : 0u;
            }
            __syncthreads();
            const int nw4 = (nw + 3) & ~3;
            for (int w = 0; w < nw4; w += 4) {
                uint4 A[4], E[4];
#pragma unroll
                for (int ra = 0; ra < 4; ++ra) A[ra] = *reinterpret_cast<const uint4*>(&sab[ti + 16 * ra][w]);
#pragma unroll
                for (int re = 0; re < 4; ++re) E[re] = *reinterpret_cast<const uint4*>(&se[tj + 16 * re][w]);
#pragma unroll
                for (int ra = 0; ra < 4; ++ra)
#pragma unroll
                    for (int re = 0; re < 4; ++re)
                        hs_add4(st[ra][re], A[ra].x & E[re].x, A[ra].y & E[re].y, A[ra].z & E[re].z,
                                A[ra].w & E[re].w);
            }
        }
#pragma unroll
        for (int ra = 0; ra < 4; ++ra)
#pragma unroll
            for (int re = 0; re < 4; ++re) X[cls][ra][re] = hs_total(st[ra][re]);
    }

    // ---- epilogue: 8-voxel tables, SH3, three roles --------------------------
    const long long* T0 = s_tab;
    const long long* T1 = s_tab + np1;
    const long long* TB = s_tab + 2 * np1;
    const int n0max = g.N0, n1max = g.N1, nmax = g.N;
    const int nb0 = c1[2 * b], nb1 = c1[2 * b + 1];
    const uint32_t dM = (uint32_t)d * (uint32_t)M;
    unsigned long long kb_best = 0ull;
#pragma unroll
    for (int ra = 0; ra < 4; ++ra) {
        const int ar = ti + 16 * ra;
        const int a = a0 + ar;
        if (a >= b) continue;
        const Pair2 pab = s_pab[ar];
        const int2 na = s_na[ar];
        unsigned long long ka_best = 0ull;
#pragma unroll
        for (int re = 0; re < 4; ++re) {
            const int er = tj + 16 * re;
            const int e = e0 + er;
            if (e >= M) continue;
            const Pair2 pbe = s_pbe[er];
            const int2 ne = s_ne[er];
            const Pair2 pae = pd[(size_t)a * M + e];
            long long sh3 = 0;
            int tot[8];
            {  // class 0
                const int x = X[0][ra][re];
                int v[8];
                v[7] = x;                                              // (1,1,1)
                v[3] = pbe.n0 - x;                                     // (0,1,1)
                v[5] = pae.n0 - x;                                     // (1,0,1)
                v[6] = pab.n0 - x;                                     // (1,1,0)
                v[1] = ne.x - pae.n0 - pbe.n0 + x;                     // (0,0,1)
                v[2] = nb0 - pab.n0 - pbe.n0 + x;                      // (0,1,0)
                v[4] = na.x - pab.n0 - pae.n0 + x;                     // (1,0,0)
                v[0] = g.N0 - na.x - nb0 - ne.x + pab.n0 + pae.n0 + pbe.n0 - x;  // (0,0,0)
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    sh3 -= tab_get(T0, v[q], n0max);
                    tot[q] = v[q];
                }
            }
            {  // class 1
                const int x = X[1][ra][re];
                int v[8];
                v[7] = x;
                v[3] = pbe.n1 - x;
                v[5] = pae.n1 - x;
                v[6] = pab.n1 - x;
                v[1] = ne.y - pae.n1 - pbe.n1 + x;
                v[2] = nb1 - pab.n1 - pbe.n1 + x;
                v[4] = na.y - pab.n1 - pae.n1 + x;
                v[0] = g.N1 - na.y - nb1 - ne.y + pab.n1 + pae.n1 + pbe.n1 - x;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    sh3 -= tab_get(T1, v[q], n1max);
                    tot[q] += v[q];
                }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) sh3 += tab_get(TB, tot[q], nmax);
            const unsigned long long k_a =
                pack_key(fx_to_float(pbe.sh - sh3), (dM + (uint32_t)b) * (uint32_t)M + (uint32_t)e);
            const unsigned long long k_b =
                pack_key(fx_to_float(pae.sh - sh3), (dM + (uint32_t)a) * (uint32_t)M + (uint32_t)e);
            const unsigned long long k_e =
                pack_key(fx_to_float(pab.sh - sh3), (dM + (uint32_t)a) * (uint32_t)M + (uint32_t)b);
            ka_best = k_a > ka_best ? k_a : ka_best;
            kb_best = k_b > kb_best ? k_b : kb_best;
            atomicMax(&s_ke[er], k_e);
        }
        if (ka_best) atomicMax(&s_ka[ar], ka_best);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, kb_best, o);
        kb_best = other > kb_best ? other : kb_best;
    }
    if ((tid & 31) == 0 && kb_best) atomicMax(&s_kb, kb_best);
    __syncthreads();
    if (tid == 0 && s_kb) atomicMax(keys + b, s_kb);
    for (int r = tid; r < TA; r += 256)
        if (s_ka[r]) atomicMax(keys + a0 + r, s_ka[r]);
    for (int r = tid; r < TE; r += 256)
        if (s_ke[r]) atomicMax(keys + e0 + r, s_ke[r]);
}

void build_k3c2_items(int M, std::vector<int2>& items) {
    items.clear();
    for (int b = 1; b + 1 < M; ++b) {
        const int nta = (b + TA - 1) / TA;
        const int nte = (M - 1 - b + TE - 1) / TE;
        for (int ta = 0; ta < nta; ++ta)
            for (int te = 0; te < nte; ++te) items.push_back(make_int2(b, (ta << 16) | te));
    }
}

size_t k3c2_smem_bytes(int N) { return (size_t)3 * (N + 1) * sizeof(long long); }

cudaError_t launch_k3c2(const uint32_t* planes, PlaneGeom g, int M, int d0, int nd, const int2* items, int n_items,
                        const long long* tab, const int* cnt1, const Pair2* pairs, unsigned long long* keys,
                        cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    const size_t smem = k3c2_smem_bytes(g.N);
    cudaError_t e = cudaFuncSetAttribute(k3c2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(n_items, nd);
    k3c2_kernel<<<grid, 256, smem, st>>>(planes, g, M, d0, items, tab, cnt1, pairs, keys);
    return cudaGetLastError();
}

}  // namespace mdfs
