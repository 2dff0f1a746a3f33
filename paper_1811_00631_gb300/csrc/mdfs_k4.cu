// k = 4 scan for two classes per variable (c = 2) from class-sorted bit planes
// (Eq. 1 with |S| = 3; voxel counters of section "Algorithm and
// implementation").
//
// For a quadruple a < b < c < e and one class, the 16 voxel counts follow
// from the all-ones counts n_T of every subset T of {a, b, c, e} by Moebius
// inversion over supersets: count(ones exactly O) = sum_{T >= O}
// (-1)^{|T \ O|} n_T.  Singles and pairs come from the k = 1 and pair passes,
// the four triples' counts and entropies from the triple tables (t3_kernel);
// the kernel counts only n_abce = popc(A&B&C&E) per 32 samples, both classes
// packed in one word.  SH over the 16 voxels gives IG(a|bce), IG(b|ace),
// IG(c|abe), IG(e|abc) against the tabled triple entropies.  Entropies are
// exact int64 fixed-point sums of the f(n + beta) tables.
//
// Work item: a pair (a, b) with a tile of 32 c (c > b) and a tile of 32 e
// (e > c); 16 x 16 threads, 2 x 2 (c, e) per thread.  Keys index the partner
// triple as ((d M + p1) M + p2) M + p3.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "mdfs_device.cuh"
#include "mdfs_internal.cuh"
#include "mdfs_packed.cuh"

namespace mdfs {

namespace {

constexpr int kRC = 2, kRE = 2, kTC = 16 * kRC, kTE = 16 * kRE;
constexpr int kWC = 128;      // staged words per chunk (even)
constexpr int kLD = kWC + 2;  // row stride: uint2 loads, e rows two banks apart

__device__ __forceinline__ unsigned long long kmax(unsigned long long a, unsigned long long b) { return a > b ? a : b; }

// kTable: instead of folding the four roles into keys, store n_abce and
// SH(a,b,c,e) of every quadruple at its lexicographic rank (the quadruple
// tables of the k = 5 scan; C(M,4) < 2^32).
template <bool kTable>
__global__ void __launch_bounds__(256, 2) k4_kernel(const uint32_t* __restrict__ planes, PlaneGeom g, int M, int d0,
                                                 const int2* __restrict__ items, const long long* __restrict__ tab,
                                                 const int* __restrict__ cnt1, const int* __restrict__ cnt2,
                                                 const uint32_t* __restrict__ t3c, const long long* __restrict__ t3s,
                                                 unsigned long long* __restrict__ keys, EmitTable emit,
                                                 uint32_t* __restrict__ t4c, long long* __restrict__ t4s) {
    __shared__ __align__(16) uint32_t sABC[kTC * kLD], sE[kTE * kLD], sAB[kWC];
    __shared__ unsigned long long kc[kTC], ke[kTE], ka, kb;

    const int2 it = items[blockIdx.x];
    const int a = it.x & 0xFFFF, b = it.x >> 16;
    const int c0 = b + 1 + (it.y >> 16) * kTC;
    const int e0 = c0 + 1 + (it.y & 0xFFFF) * kTE;
    const int dl = blockIdx.y, d = d0 + dl;
    const int tid = threadIdx.x, tc = tid >> 4, te = tid & 15;
    const uint32_t* pbase = planes + (size_t)d * M * g.Ws;  // one plane per variable (c = 2)
    const Staging z = make_staging(g.W0, g.W1);

    // all-ones counts n_abce per (c, e), both classes packed
    uint32_t x4[kRC][kRE] = {{0u, 0u}, {0u, 0u}};
    for (int s0 = 0; s0 < z.Wst; s0 += kWC) {
        const int len = min(kWC, z.Wst - s0);
        __syncthreads();
        for (int j = tid; j < kWC; j += 256) {
            uint32_t w = 0u;
            if (j < len)
                w = staged_word(pbase + (size_t)a * g.Ws, s0 + j, z) & staged_word(pbase + (size_t)b * g.Ws, s0 + j, z);
            sAB[j] = w;
        }
        __syncthreads();
        for (int idx = tid; idx < (kTC + kTE) * kWC; idx += 256) {
            const int r = idx / kWC, j = idx % kWC;
            const int v = r < kTC ? c0 + r : e0 + (r - kTC);
            const uint32_t w = (j < len && v < M) ? staged_word(pbase + (size_t)v * g.Ws, s0 + j, z) : 0u;
            if (r < kTC) sABC[r * kLD + j] = w & sAB[j];
            else sE[(r - kTC) * kLD + j] = w;
        }
        __syncthreads();
        int lo[2], hi[2];
        class_segments(z, s0, kWC, lo, hi);
#pragma unroll
        for (int cls = 0; cls < 2; ++cls) {
            const uint32_t mul = cls ? 65536u : 1u;
            for (int j = lo[cls]; j < hi[cls]; j += 2) {
                uint2 u[kRC], w[kRE];
#pragma unroll
                for (int r = 0; r < kRC; ++r) u[r] = *reinterpret_cast<const uint2*>(sABC + (tc + 16 * r) * kLD + j);
#pragma unroll
                for (int r = 0; r < kRE; ++r) w[r] = *reinterpret_cast<const uint2*>(sE + (te + 16 * r) * kLD + j);
#pragma unroll
                for (int rc = 0; rc < kRC; ++rc)
#pragma unroll
                    for (int re = 0; re < kRE; ++re)
                        x4[rc][re] += (uint32_t)(__popc(u[rc].x & w[re].x) + __popc(u[rc].y & w[re].y)) * mul;
            }
        }
    }

    for (int i = tid; i < kTC; i += 256) kc[i] = 0ull;
    for (int i = tid; i < kTE; i += 256) ke[i] = 0ull;
    if (tid == 0) ka = kb = 0ull;
    __syncthreads();

    Tabs tb;
    tb.tab = tab;
    tb.np1 = g.N + 1;
    tb.N0 = g.N0;
    tb.N1 = g.N1;
    const uint32_t NC = pack2(g.N0, g.N1);
    auto single = [&](int v) -> uint32_t {
        const int* p = cnt1 + ((size_t)d * M + v) * 2;
        return pack2(__ldg(p), __ldg(p + 1));
    };
    auto pair = [&](int i, int m) -> uint32_t {  // i < m
        const int* p = cnt2 + (((size_t)dl * M + i) * M + m) * 2;
        return pack2(__ldg(p), __ldg(p + 1));
    };
    const Rank3 rk = make_rank3(M);
    const uint32_t* T3c = t3c + (size_t)dl * ((size_t)rk.top + 1);
    const long long* T3s = t3s + (size_t)dl * ((size_t)rk.top + 1);
    const uint32_t na = single(a), nb = single(b), nab = pair(a, b);
    const uint32_t ra = rk.part_x(a), rb = rk.part_x(b), rab = ra + rk.part_y(b);
    const uint32_t dM = (uint32_t)d * (uint32_t)M;
    unsigned long long my_ka = 0ull, my_kb = 0ull, my_ke[kRE] = {0ull, 0ull};
#pragma unroll
    for (int rc = 0; rc < kRC; ++rc) {
        const int c = c0 + tc + 16 * rc;
        if (c >= M) continue;
        const uint32_t nc = single(c), nac = pair(a, c), nbc = pair(b, c);
        const uint32_t i_abc = rk.top - (rab + (uint32_t)(rk.Mm1 - c));
        const uint32_t n_abc = __ldg(T3c + i_abc);
        const long long sh_abc = __ldg(T3s + i_abc);
        const uint32_t rac = ra + rk.part_y(c), rbc = rb + rk.part_y(c);
        unsigned long long my_kc = 0ull;
#pragma unroll
        for (int re = 0; re < kRE; ++re) {
            const int e = e0 + te + 16 * re;
            if (e >= M || e <= c) continue;
            const uint32_t ne = single(e), nae = pair(a, e), nbe = pair(b, e), nce = pair(c, e);
            const uint32_t t_e = (uint32_t)(rk.Mm1 - e);
            const uint32_t i_abe = rk.top - (rab + t_e), i_ace = rk.top - (rac + t_e), i_bce = rk.top - (rbc + t_e);
            // the four-variable table: bits a = 1, b = 2, c = 4, e = 8
            uint32_t q[16] = {NC, na,  nb,  nab,           nc,  nac,           nbc,           n_abc,
                              ne, nae, nbe, __ldg(T3c + i_abe), nce, __ldg(T3c + i_ace), __ldg(T3c + i_bce), x4[rc][re]};
            moebius_packed<4>(q);
            const long long sh4 = sh_packed<4>(q, tb);
            if (kTable) {
                const Rank4 r4 = make_rank4(M);
                const size_t at = (size_t)dl * ((size_t)r4.top + 1) +
                                  (r4.top - (r4.part_w(a) + r4.part_x(b) + r4.part_y(c) + (uint32_t)(r4.Mm1 - e)));
                t4c[at] = x4[rc][re];
                t4s[at] = sh4;
                continue;
            }
            const long long sh_abe = __ldg(T3s + i_abe), sh_ace = __ldg(T3s + i_ace), sh_bce = __ldg(T3s + i_bce);
            // IG(a | b,c,e), IG(b | a,c,e), IG(c | a,b,e), IG(e | a,b,c)
            const unsigned long long k_a =
                pack_key(fx_to_float(sh_bce - sh4), ((dM + (uint32_t)b) * M + (uint32_t)c) * M + (uint32_t)e);
            const unsigned long long k_b =
                pack_key(fx_to_float(sh_ace - sh4), ((dM + (uint32_t)a) * M + (uint32_t)c) * M + (uint32_t)e);
            const unsigned long long k_c =
                pack_key(fx_to_float(sh_abe - sh4), ((dM + (uint32_t)a) * M + (uint32_t)b) * M + (uint32_t)e);
            const unsigned long long k_e =
                pack_key(fx_to_float(sh_abc - sh4), ((dM + (uint32_t)a) * M + (uint32_t)b) * M + (uint32_t)c);
            my_ka = kmax(my_ka, k_a);
            my_kb = kmax(my_kb, k_b);
            my_kc = kmax(my_kc, k_c);
            my_ke[re] = kmax(my_ke[re], k_e);
            if (emit.keys) {  // the four roles, partners ascending
                const long long g4[4] = {sh_bce - sh4, sh_ace - sh4, sh_abe - sh4, sh_abc - sh4};
                const unsigned long long ek[4] = {emit_key(a, b, c, e), emit_key(b, a, c, e), emit_key(c, a, b, e),
                                                  emit_key(e, a, b, c)};
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (g4[r] >= emit.thr_fx) emit_insert(emit, ek[r], pack_key(fx_to_float(g4[r]), (uint32_t)d));
            }
        }
        if (my_kc) atomicMax(&kc[tc + 16 * rc], my_kc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_ka = kmax(my_ka, __shfl_xor_sync(0xffffffffu, my_ka, o));
        my_kb = kmax(my_kb, __shfl_xor_sync(0xffffffffu, my_kb, o));
    }
    // role e: the two c rows of a warp (lanes t and t + 16) share each e
#pragma unroll
    for (int re = 0; re < kRE; ++re) my_ke[re] = kmax(my_ke[re], __shfl_xor_sync(0xffffffffu, my_ke[re], 16));
    if ((tid & 31) < 16) {
#pragma unroll
        for (int re = 0; re < kRE; ++re)
            if (my_ke[re]) atomicMax(&ke[te + 16 * re], my_ke[re]);
    }
    if ((tid & 31) == 0) {
        if (my_ka) atomicMax(&ka, my_ka);
        if (my_kb) atomicMax(&kb, my_kb);
    }
    __syncthreads();
    for (int i = tid; i < kTC; i += 256)
        if (kc[i]) atomicMax(keys + c0 + i, kc[i]);
    for (int i = tid; i < kTE; i += 256)
        if (ke[i]) atomicMax(keys + e0 + i, ke[i]);
    if (tid == 0) {
        if (ka) atomicMax(keys + a, ka);
        if (kb) atomicMax(keys + b, kb);
    }
}

}  // namespace

// (a | b << 16, tc << 16 | te) for a < b < c-tile < e-tile, skipping tiles with no c < e
void build_k4_items(int M, std::vector<int2>& items) {
    items.clear();
    for (int b = 1; b + 2 < M; ++b) {
        for (int tc = 0;; ++tc) {
            const int cmin = b + 1 + tc * kTC;
            if (cmin > M - 2) break;
            for (int te = 0;; ++te) {
                const int emin = cmin + 1 + te * kTE;
                if (emin > M - 1) break;
                for (int a = 0; a < b; ++a) items.push_back(make_int2(a | (b << 16), (tc << 16) | te));
            }
        }
    }
}

cudaError_t launch_k4(const uint32_t* planes, PlaneGeom g, int M, int d0, int nd, const int2* items, int n_items,
                      const long long* tab, const int* cnt1, const int* cnt2, const uint32_t* t3c,
                      const long long* t3s, unsigned long long* keys, cudaStream_t st, EmitTable emit) {
    if (n_items == 0 || nd == 0) return cudaSuccess;
    if (nd > 65535) return cudaErrorInvalidValue;
    k4_kernel<false><<<dim3(n_items, nd), 256, 0, st>>>(planes, g, M, d0, items, tab, cnt1, cnt2, t3c, t3s, keys, emit,
                                                       nullptr, nullptr);
    return cudaGetLastError();
}

size_t t4_entries(int M) {
    const size_t m = (size_t)M;
    return M < 4 ? 0 : m * (m - 1) / 2 * (m - 2) / 3 * (m - 3) / 4;
}

cudaError_t launch_t4(const uint32_t* planes, PlaneGeom g, int M, int d0, int nd, const int2* items, int n_items,
                      const long long* tab, const int* cnt1, const int* cnt2, const uint32_t* t3c,
                      const long long* t3s, uint32_t* t4c, long long* t4s, cudaStream_t st) {
    if (n_items == 0 || nd == 0) return cudaSuccess;
    if (nd > 65535 || t4_entries(M) > (1ull << 32)) return cudaErrorInvalidValue;
    k4_kernel<true><<<dim3(n_items, nd), 256, 0, st>>>(planes, g, M, d0, items, tab, cnt1, cnt2, t3c, t3s, nullptr,
                                                      EmitTable(), t4c, t4s);
    return cudaGetLastError();
}

}  // namespace mdfs
