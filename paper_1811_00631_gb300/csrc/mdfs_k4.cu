// k = 4 scan for two classes per variable (c = 2) from class-sorted bit planes
// (Eq. 1 with |S| = 3; voxel counters of section "Algorithm and
// implementation").
//
// For a quadruple a < b < c < e and one class, the 16 voxel counts follow
// from the all-ones counts n_T of every subset T of {a, b, c, e} (n_{} = class
// size) by Moebius inversion over supersets: count(ones exactly O) =
// sum_{T >= O} (-1)^{|T \ O|} n_T.  Singles and pairs come from the k = 1 and
// pair passes; the kernel counts, per 32 samples and class,
//     n_abce = popc(A&B&C&E),  n_ace = popc(A&C&E),  n_bce = popc(B&C&E),
//     n_abe = popc(A&B&E) (per e),  n_abc = popc(A&B&C) (per c).
// SH over the 16 voxels gives IG(a|bce), IG(b|ace), IG(c|abe), IG(e|abc) from
// the four triple entropies, which the kernel builds the same way from 8
// voxels.  Entropies are exact int64 fixed-point sums of the f(n + beta)
// tables.
//
// Work item: a pair (a, b) with a tile of 32 c (c > b) and a tile of 32 e
// (e > c); 16 x 16 threads, 2 x 2 (c, e) per thread.  Keys index the partner
// triple as ((d M + p1) M + p2) M + p3.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "mdfs_device.cuh"
#include "mdfs_internal.cuh"

namespace mdfs {

namespace {

constexpr int kRC = 2, kRE = 2, kTC = 16 * kRC, kTE = 16 * kRE, kWC = 32;
constexpr int kLD = kWC + 2;  // even row stride: 8-byte word-pair loads, rows 2 banks apart

// In-place Moebius inversion over supersets of L bits: on entry n[T] is the
// all-ones count of subset T, on exit n[O] the count of the voxel whose ones
// are exactly O.
template <int L>
__device__ __forceinline__ void superset_moebius(int (&n)[1 << L]) {
#pragma unroll
    for (int j = 0; j < L; ++j)
#pragma unroll
        for (int m = 0; m < (1 << L); ++m)
            if (!(m & (1 << j))) n[m] -= n[m | (1 << j)];
}

// SH = sum over voxels of f(n0+n1+b0+b1) - f(n0+b0) - f(n1+b1) (int64 tables)
template <int L>
__device__ __forceinline__ long long sh_voxels(const int (&n0)[1 << L], const int (&n1)[1 << L],
                                               const long long* __restrict__ tab, int np1) {
    long long s = 0;
#pragma unroll
    for (int m = 0; m < (1 << L); ++m)
        s += __ldg(tab + 2 * np1 + n0[m] + n1[m]) - __ldg(tab + n0[m]) - __ldg(tab + np1 + n1[m]);
    return s;
}

__device__ __forceinline__ unsigned long long kmax(unsigned long long a, unsigned long long b) { return a > b ? a : b; }

__global__ void __launch_bounds__(256, 2) k4_kernel(const uint32_t* __restrict__ planes, PlaneGeom g, int M, int d0,
                                                 const int2* __restrict__ items, const long long* __restrict__ tab,
                                                 const int* __restrict__ cnt1, const int* __restrict__ cnt2,
                                                 unsigned long long* __restrict__ keys, EmitTable emit) {
    __shared__ __align__(8) uint32_t sa[kWC], sb[kWC], sab[kWC];
    __shared__ __align__(8) uint32_t sabc[kTC][kLD], sac[kTC][kLD], sbc[kTC][kLD], se[kTE][kLD];
    __shared__ unsigned long long kc[kTC], ke[kTE], ka, kb;

    const int2 it = items[blockIdx.x];
    const int a = it.x & 0xFFFF, b = it.x >> 16;
    const int c0 = b + 1 + (it.y >> 16) * kTC;
    const int e0 = c0 + 1 + (it.y & 0xFFFF) * kTE;
    const int dl = blockIdx.y, d = d0 + dl;
    const int tid = threadIdx.x, tc = tid >> 4, te = tid & 15;
    const uint32_t* pbase = planes + (size_t)d * M * g.Ws;  // one plane per variable (c = 2)

    // all-ones counts per class: [cls][rc][re] for abce, ace, bce; [cls][rc] abc; [cls][re] abe
    int x4[2][kRC][kRE], xace[2][kRC][kRE], xbce[2][kRC][kRE], xabc[2][kRC], xabe[2][kRE];
#pragma unroll
    for (int cl = 0; cl < 2; ++cl) {
#pragma unroll
        for (int rc = 0; rc < kRC; ++rc) {
            xabc[cl][rc] = 0;
#pragma unroll
            for (int re = 0; re < kRE; ++re) x4[cl][rc][re] = xace[cl][rc][re] = xbce[cl][rc][re] = 0;
        }
#pragma unroll
        for (int re = 0; re < kRE; ++re) xabe[cl][re] = 0;
    }

#pragma unroll
    for (int cls = 0; cls < 2; ++cls) {
        const int wb = cls == 0 ? 0 : g.W0, we = cls == 0 ? g.W0 : g.W;
        for (int w0 = wb; w0 < we; w0 += kWC) {
            const int nw = min(kWC, we - w0);
            __syncthreads();
            if (tid < kWC) {
                const uint32_t pa = tid < nw ? pbase[(size_t)a * g.Ws + w0 + tid] : 0u;
                const uint32_t pb = tid < nw ? pbase[(size_t)b * g.Ws + w0 + tid] : 0u;
                sa[tid] = pa;
                sb[tid] = pb;
                sab[tid] = pa & pb;
            }
            __syncthreads();
            for (int idx = tid; idx < kTC * kWC; idx += 256) {
                const int w = idx % kWC, r = idx / kWC;
                const int vc = c0 + r;
                const uint32_t pc = (w < nw && vc < M) ? pbase[(size_t)vc * g.Ws + w0 + w] : 0u;
                sabc[r][w] = sab[w] & pc;
                sac[r][w] = sa[w] & pc;
                sbc[r][w] = sb[w] & pc;
            }
            for (int idx = tid; idx < kTE * kWC; idx += 256) {
                const int w = idx % kWC, r = idx / kWC;
                const int ve = e0 + r;
                se[r][w] = (w < nw && ve < M) ? pbase[(size_t)ve * g.Ws + w0 + w] : 0u;
            }
            __syncthreads();
            // two words per step (entries past nw are zero)
            for (int w = 0; w < nw; w += 2) {
                const uint2 ab = *reinterpret_cast<const uint2*>(&sab[w]);
                uint2 ev[kRE];
#pragma unroll
                for (int re = 0; re < kRE; ++re) {
                    ev[re] = *reinterpret_cast<const uint2*>(&se[te + 16 * re][w]);
                    xabe[cls][re] += __popc(ab.x & ev[re].x) + __popc(ab.y & ev[re].y);
                }
#pragma unroll
                for (int rc = 0; rc < kRC; ++rc) {
                    const uint2 v3 = *reinterpret_cast<const uint2*>(&sabc[tc + 16 * rc][w]);
                    const uint2 vac = *reinterpret_cast<const uint2*>(&sac[tc + 16 * rc][w]);
                    const uint2 vbc = *reinterpret_cast<const uint2*>(&sbc[tc + 16 * rc][w]);
                    xabc[cls][rc] += __popc(v3.x) + __popc(v3.y);
#pragma unroll
                    for (int re = 0; re < kRE; ++re) {
                        x4[cls][rc][re] += __popc(v3.x & ev[re].x) + __popc(v3.y & ev[re].y);
                        xace[cls][rc][re] += __popc(vac.x & ev[re].x) + __popc(vac.y & ev[re].y);
                        xbce[cls][rc][re] += __popc(vbc.x & ev[re].x) + __popc(vbc.y & ev[re].y);
                    }
                }
            }
        }
    }

    for (int i = tid; i < kTC; i += 256) kc[i] = 0ull;
    for (int i = tid; i < kTE; i += 256) ke[i] = 0ull;
    if (tid == 0) ka = kb = 0ull;
    __syncthreads();

    const int np1 = g.N + 1;
    const int NC[2] = {g.N0, g.N1};
    auto single = [&](int v, int cl) { return __ldg(cnt1 + ((size_t)d * M + v) * 2 + cl); };
    auto pair = [&](int i, int m, int cl) {  // i < m
        return __ldg(cnt2 + ((((size_t)dl * M + i) * M + m)) * 2 + cl);
    };
    int na[2], nb[2], nab[2];
#pragma unroll
    for (int cl = 0; cl < 2; ++cl) {
        na[cl] = single(a, cl);
        nb[cl] = single(b, cl);
        nab[cl] = pair(a, b, cl);
    }
    const uint32_t dM = (uint32_t)d * (uint32_t)M;
    unsigned long long my_ka = 0ull, my_kb = 0ull;
#pragma unroll
    for (int rc = 0; rc < kRC; ++rc) {
        const int c = c0 + tc + 16 * rc;
        if (c >= M) continue;
        int nc[2], nac[2], nbc[2];
#pragma unroll
        for (int cl = 0; cl < 2; ++cl) {
            nc[cl] = single(c, cl);
            nac[cl] = pair(a, c, cl);
            nbc[cl] = pair(b, c, cl);
        }
        // SH(a, b, c): subsets of {a, b, c} as bits 0, 1, 2
        long long sh_abc;
        {
            int t0[8], t1[8];
#pragma unroll
            for (int cl = 0; cl < 2; ++cl) {
                int* t = cl ? t1 : t0;
                t[0] = NC[cl]; t[1] = na[cl]; t[2] = nb[cl]; t[3] = nab[cl];
                t[4] = nc[cl]; t[5] = nac[cl]; t[6] = nbc[cl]; t[7] = xabc[cl][rc];
            }
            superset_moebius<3>(t0);
            superset_moebius<3>(t1);
            sh_abc = sh_voxels<3>(t0, t1, tab, np1);
        }
        unsigned long long my_kc = 0ull;
#pragma unroll
        for (int re = 0; re < kRE; ++re) {
            const int e = e0 + te + 16 * re;
            if (e >= M || e <= c) continue;
            int ne[2], nae[2], nbe[2], nce[2];
#pragma unroll
            for (int cl = 0; cl < 2; ++cl) {
                ne[cl] = single(e, cl);
                nae[cl] = pair(a, e, cl);
                nbe[cl] = pair(b, e, cl);
                nce[cl] = pair(c, e, cl);
            }
            // the four-variable table: bits a = 1, b = 2, c = 4, e = 8
            int q0[16], q1[16];
#pragma unroll
            for (int cl = 0; cl < 2; ++cl) {
                int* q = cl ? q1 : q0;
                q[0] = NC[cl]; q[1] = na[cl]; q[2] = nb[cl]; q[3] = nab[cl];
                q[4] = nc[cl]; q[5] = nac[cl]; q[6] = nbc[cl]; q[7] = xabc[cl][rc];
                q[8] = ne[cl]; q[9] = nae[cl]; q[10] = nbe[cl]; q[11] = xabe[cl][re];
                q[12] = nce[cl]; q[13] = xace[cl][rc][re]; q[14] = xbce[cl][rc][re]; q[15] = x4[cl][rc][re];
            }
            // triples: (a, c, e), (b, c, e), (a, b, e) as 3-bit tables
            int u0[8], u1[8], v0[8], v1[8], w0t[8], w1t[8];
#pragma unroll
            for (int cl = 0; cl < 2; ++cl) {
                const int* q = cl ? q1 : q0;
                int* u = cl ? u1 : u0;  // a c e -> bits 0 1 2 from q bits 1 4 8
                int* v = cl ? v1 : v0;  // b c e from q bits 2 4 8
                int* w = cl ? w1t : w0t;  // a b e from q bits 1 2 8
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    u[m] = q[((m & 1) ? 1 : 0) | ((m & 2) ? 4 : 0) | ((m & 4) ? 8 : 0)];
                    v[m] = q[((m & 1) ? 2 : 0) | ((m & 2) ? 4 : 0) | ((m & 4) ? 8 : 0)];
                    w[m] = q[((m & 1) ? 1 : 0) | ((m & 2) ? 2 : 0) | ((m & 4) ? 8 : 0)];
                }
            }
            superset_moebius<4>(q0);
            superset_moebius<4>(q1);
            superset_moebius<3>(u0);
            superset_moebius<3>(u1);
            superset_moebius<3>(v0);
            superset_moebius<3>(v1);
            superset_moebius<3>(w0t);
            superset_moebius<3>(w1t);
            const long long sh4 = sh_voxels<4>(q0, q1, tab, np1);
            const long long sh_ace = sh_voxels<3>(u0, u1, tab, np1);
            const long long sh_bce = sh_voxels<3>(v0, v1, tab, np1);
            const long long sh_abe = sh_voxels<3>(w0t, w1t, tab, np1);
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
            atomicMax(&ke[te + 16 * re], k_e);
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
                      const long long* tab, const int* cnt1, const int* cnt2, unsigned long long* keys,
                      cudaStream_t st, EmitTable emit) {
    if (n_items == 0 || nd == 0) return cudaSuccess;
    if (nd > 65535) return cudaErrorInvalidValue;
    k4_kernel<<<dim3(n_items, nd), 256, 0, st>>>(planes, g, M, d0, items, tab, cnt1, cnt2, keys, emit);
    return cudaGetLastError();
}

}  // namespace mdfs
