// Counting and entropy kernels of the MDFS scan (Eq. 1, Eq. 3; Eqs. H, p, beta).
//
// Voxel counts are exact integers: every variable and discretisation carries
// one bit plane per bin 1..c-1 over the class-sorted samples, so the count of
// a voxel whose coordinates are all >= 1 is a popcount of the AND of planes
// over the class-0 (resp. class-1) word range.  Voxels with a zero coordinate
// follow by inclusion-exclusion from lower-order counts.  Entropies are sums
// of int64 fixed-point table entries (exact, order-independent); the only FP
// step per tuple is the final IG -> float rounding.  Max/argmax over tuples
// and discretisations is a packed 64-bit atomicMax (ordered IG | ~index).
#include "mdfs_device.cuh"
#include "mdfs_internal.cuh"

namespace mdfs {

// ---------------------------------------------------------------------------
// k = 1 (Eq. 3): per (discretisation, variable) one warp.
// ---------------------------------------------------------------------------
template <int C>
__global__ void __launch_bounds__(256) k1_kernel(const uint32_t* __restrict__ planes, PlaneGeom g, int M, int D,
                                                 const long long* __restrict__ tab, int* __restrict__ cnt1,
                                                 long long* __restrict__ sh1, unsigned long long* __restrict__ keys,
                                                 EmitTable emit) {
    constexpr int P = C - 1;
    const int lane = threadIdx.x & 31;
    const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (item >= D * M) return;
    const uint32_t* base = planes + (size_t)item * P * g.Ws;
    int n0[C], n1[C];
    int s0tot = 0, s1tot = 0;
#pragma unroll
    for (int a = 1; a < C; ++a) {
        const uint32_t* pl = base + (size_t)(a - 1) * g.Ws;
        int s0 = 0, s1 = 0;
        for (int w = lane; w < g.W0; w += 32) s0 += __popc(pl[w]);
        for (int w = g.W0 + lane; w < g.W; w += 32) s1 += __popc(pl[w]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        n0[a] = s0;
        n1[a] = s1;
        s0tot += s0;
        s1tot += s1;
    }
    n0[0] = g.N0 - s0tot;
    n1[0] = g.N1 - s1tot;
    if (lane != 0) return;
    const int np1 = g.N + 1;
    long long sh = 0;
#pragma unroll
    for (int a = 0; a < C; ++a) sh += voxel_h(tab, np1, n0[a], n1[a]);
    sh1[item] = sh;
#pragma unroll
    for (int a = 1; a < C; ++a) {
        cnt1[((size_t)item * P + (a - 1)) * 2 + 0] = n0[a];
        cnt1[((size_t)item * P + (a - 1)) * 2 + 1] = n1[a];
    }
    if (keys || emit.keys) {
        const int d = item / M, v = item - d * M;
        const long long ig = voxel_h(tab, np1, g.N0, g.N1) - sh;
        if (keys) atomicMax(keys + v, pack_key(fx_to_float(ig), (uint32_t)d));
        if (emit.keys && ig >= emit.thr_fx)
            emit_insert(emit, emit_key(v, -1, -1, -1), pack_key(fx_to_float(ig), (uint32_t)d));
    }
}

// ---------------------------------------------------------------------------
// Completion of a c x c (k = 2) or c x c x c (k = 3) count table of one
// channel (class 0, class 1 or both) from the counts of the all-nonzero
// voxels and the lower-order marginals, followed by sum_v tab[n_v].
// ---------------------------------------------------------------------------
template <int C>
__device__ __forceinline__ long long channel2(const int (&X)[C - 1][C - 1], const int* ni, const int* nm, int ntot,
                                              const long long* __restrict__ tabx) {
    int T[C][C];
#pragma unroll
    for (int a = 1; a < C; ++a)
#pragma unroll
        for (int b = 1; b < C; ++b) T[a][b] = X[a - 1][b - 1];
    int all = 0;
#pragma unroll
    for (int a = 1; a < C; ++a) {
        int s = 0;
#pragma unroll
        for (int b = 1; b < C; ++b) s += T[a][b];
        T[a][0] = ni[a - 1] - s;
        all += ni[a - 1];
    }
#pragma unroll
    for (int b = 1; b < C; ++b) {
        int s = 0;
#pragma unroll
        for (int a = 1; a < C; ++a) s += T[a][b];
        T[0][b] = nm[b - 1] - s;
        all += T[0][b];
    }
    T[0][0] = ntot - all;
    long long sum = 0;
#pragma unroll
    for (int a = 0; a < C; ++a)
#pragma unroll
        for (int b = 0; b < C; ++b) sum += __ldg(tabx + clamp_count(T[a][b], ntot));
    return sum;
}

template <int C>
__device__ __forceinline__ long long channel3(const int (&X)[C - 1][C - 1][C - 1], const int (&nab)[C - 1][C - 1],
                                              const int (&nae)[C - 1][C - 1], const int (&nbe)[C - 1][C - 1],
                                              const int (&na)[C - 1], const int (&nb)[C - 1], const int (&ne)[C - 1],
                                              int ntot, const long long* __restrict__ tabx) {
    int T[C][C][C];
#pragma unroll
    for (int a = 1; a < C; ++a)
#pragma unroll
        for (int b = 1; b < C; ++b)
#pragma unroll
            for (int e = 1; e < C; ++e) T[a][b][e] = X[a - 1][b - 1][e - 1];
    // one zero coordinate: pair marginals
#pragma unroll
    for (int b = 1; b < C; ++b)
#pragma unroll
        for (int e = 1; e < C; ++e) {
            int s = 0;
#pragma unroll
            for (int a = 1; a < C; ++a) s += T[a][b][e];
            T[0][b][e] = nbe[b - 1][e - 1] - s;
        }
#pragma unroll
    for (int a = 1; a < C; ++a)
#pragma unroll
        for (int e = 1; e < C; ++e) {
            int s = 0;
#pragma unroll
            for (int b = 1; b < C; ++b) s += T[a][b][e];
            T[a][0][e] = nae[a - 1][e - 1] - s;
        }
#pragma unroll
    for (int a = 1; a < C; ++a)
#pragma unroll
        for (int b = 1; b < C; ++b) {
            int s = 0;
#pragma unroll
            for (int e = 1; e < C; ++e) s += T[a][b][e];
            T[a][b][0] = nab[a - 1][b - 1] - s;
        }
    // two zero coordinates: single marginals
#pragma unroll
    for (int e = 1; e < C; ++e) {
        int s = 0;
#pragma unroll
        for (int a = 0; a < C; ++a)
#pragma unroll
            for (int b = 0; b < C; ++b)
                if (a != 0 || b != 0) s += T[a][b][e];
        T[0][0][e] = ne[e - 1] - s;
    }
#pragma unroll
    for (int b = 1; b < C; ++b) {
        int s = 0;
#pragma unroll
        for (int a = 0; a < C; ++a)
#pragma unroll
            for (int e = 0; e < C; ++e)
                if (a != 0 || e != 0) s += T[a][b][e];
        T[0][b][0] = nb[b - 1] - s;
    }
#pragma unroll
    for (int a = 1; a < C; ++a) {
        int s = 0;
#pragma unroll
        for (int b = 0; b < C; ++b)
#pragma unroll
            for (int e = 0; e < C; ++e)
                if (b != 0 || e != 0) s += T[a][b][e];
        T[a][0][0] = na[a - 1] - s;
    }
    {
        int s = 0;
#pragma unroll
        for (int a = 0; a < C; ++a)
#pragma unroll
            for (int b = 0; b < C; ++b)
#pragma unroll
                for (int e = 0; e < C; ++e)
                    if (a != 0 || b != 0 || e != 0) s += T[a][b][e];
        T[0][0][0] = ntot - s;
    }
    long long sum = 0;
#pragma unroll
    for (int a = 0; a < C; ++a)
#pragma unroll
        for (int b = 0; b < C; ++b)
#pragma unroll
            for (int e = 0; e < C; ++e) sum += __ldg(tabx + clamp_count(T[a][b][e], ntot));
    return sum;
}

// ---------------------------------------------------------------------------
// k = 2: pairs (i < m), 32 x 32 variable tiles on and above the diagonal,
// 256 threads, 4 pairs per thread.  Word chunks of 32 staged in shared memory
// (row stride 33 words: conflict-free column reads).
// ---------------------------------------------------------------------------
template <int C>
__global__ void __launch_bounds__(256) k2_kernel(const uint32_t* __restrict__ planes, PlaneGeom g, int M, int d0,
                                                 int ntile, const long long* __restrict__ tab,
                                                 const int* __restrict__ cnt1, const long long* __restrict__ sh1,
                                                 unsigned long long* __restrict__ keys, long long* __restrict__ sh2,
                                                 int* __restrict__ cnt2, PairC* __restrict__ pairs2, int fbits,
                                                 const int* __restrict__ rank, EmitTable emit) {
    constexpr int P = C - 1, TI = 32, WC = 32, LD = WC + 1;
    __shared__ uint32_t si[P][TI][LD];
    __shared__ uint32_t sm[P][TI][LD];
    __shared__ unsigned long long kmax[2 * TI];

    int t = blockIdx.x, it = 0;
    while (t >= ntile - it) {
        t -= ntile - it;
        ++it;
    }
    const int mt = it + t;
    const int dl = blockIdx.y, d = d0 + dl;
    const int i0 = it * TI, m0 = mt * TI;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const uint32_t* pbase = planes + (size_t)d * M * P * g.Ws;

    int acc[2][4][P][P];
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int p = 0; p < P; ++p)
#pragma unroll
                for (int q = 0; q < P; ++q) acc[c2][r][p][q] = 0;

#pragma unroll
    for (int cls = 0; cls < 2; ++cls) {
        const int wb = cls == 0 ? 0 : g.W0, we = cls == 0 ? g.W0 : g.W;
        for (int w0 = wb; w0 < we; w0 += WC) {
            const int nw = min(WC, we - w0);
            __syncthreads();
            for (int idx = tid; idx < P * TI * WC; idx += 256) {
                const int w = idx % WC, rest = idx / WC, r = rest % TI, p = rest / TI;
                const bool okw = w < nw;
                const int vi = i0 + r, vm = m0 + r;
                si[p][r][w] = (okw && vi < M) ? pbase[((size_t)vi * P + p) * g.Ws + w0 + w] : 0u;
                sm[p][r][w] = (okw && vm < M) ? pbase[((size_t)vm * P + p) * g.Ws + w0 + w] : 0u;
            }
            __syncthreads();
            for (int w = 0; w < nw; ++w) {
                uint32_t bm[P];
#pragma unroll
                for (int q = 0; q < P; ++q) bm[q] = sm[q][tx][w];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        const uint32_t ai = si[p][ty * 4 + r][w];
#pragma unroll
                        for (int q = 0; q < P; ++q) acc[cls][r][p][q] += __popc(ai & bm[q]);
                    }
            }
        }
    }

    if (tid < 2 * TI) kmax[tid] = 0ull;
    __syncthreads();
    const int np1 = g.N + 1;
    const int m = m0 + tx;
    if (m < M) {
        const int* cm = cnt1 + ((size_t)d * M + m) * P * 2;
        int nm0[P], nm1[P], nmt[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            nm0[q] = __ldg(cm + 2 * q);
            nm1[q] = __ldg(cm + 2 * q + 1);
            nmt[q] = nm0[q] + nm1[q];
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = i0 + ty * 4 + r;
            if (i >= m) continue;
            const int* ci = cnt1 + ((size_t)d * M + i) * P * 2;
            int ni0[P], ni1[P], nit[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                ni0[p] = __ldg(ci + 2 * p);
                ni1[p] = __ldg(ci + 2 * p + 1);
                nit[p] = ni0[p] + ni1[p];
            }
            int X0[P][P], X1[P][P], XT[P][P];
#pragma unroll
            for (int p = 0; p < P; ++p)
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    X0[p][q] = acc[0][r][p][q];
                    X1[p][q] = acc[1][r][p][q];
                    XT[p][q] = X0[p][q] + X1[p][q];
                }
            const long long sh = channel2<C>(XT, nit, nmt, g.N, tab + 2 * np1) -
                                 channel2<C>(X0, ni0, nm0, g.N0, tab) - channel2<C>(X1, ni1, nm1, g.N1, tab + np1);
            if (keys) {
                const float ig_i = fx_to_float(__ldg(sh1 + (size_t)d * M + m) - sh);  // IG(i | m)
                const float ig_m = fx_to_float(__ldg(sh1 + (size_t)d * M + i) - sh);  // IG(m | i)
                atomicMax(&kmax[ty * 4 + r], pack_key(ig_i, (uint32_t)(d * M + m)));
                atomicMax(&kmax[TI + tx], pack_key(ig_m, (uint32_t)(d * M + i)));
            }
            if (emit.keys) {  // IG(i | m), IG(m | i)
                const long long gi = __ldg(sh1 + (size_t)d * M + m) - sh, gm = __ldg(sh1 + (size_t)d * M + i) - sh;
                if (gi >= emit.thr_fx) emit_insert(emit, emit_key(i, m, -1, -1), pack_key(fx_to_float(gi), (uint32_t)d));
                if (gm >= emit.thr_fx) emit_insert(emit, emit_key(m, i, -1, -1), pack_key(fx_to_float(gm), (uint32_t)d));
            }
            if (pairs2) {
                // counts times 4 (byte offsets of the consuming table lookups)
                const PairC rec{(uint32_t)(4 * X0[0][0]) | ((uint32_t)(4 * X1[0][0]) << 16), fx_narrow(sh, fbits)};
                const int ri = rank ? __ldg(rank + (size_t)d * M + i) : i;
                const int rm = rank ? __ldg(rank + (size_t)d * M + m) : m;
                pairs2[((size_t)dl * M + ri) * M + rm] = rec;
                pairs2[((size_t)dl * M + rm) * M + ri] = rec;
            }
            if (sh2) {
                const size_t pidx = ((size_t)dl * M + i) * M + m;
                sh2[pidx] = sh;
#pragma unroll
                for (int p = 0; p < P; ++p)
#pragma unroll
                    for (int q = 0; q < P; ++q) {
                        cnt2[(pidx * P * P + p * P + q) * 2 + 0] = X0[p][q];
                        cnt2[(pidx * P * P + p * P + q) * 2 + 1] = X1[p][q];
                    }
            }
        }
    }
    if (keys) {
        __syncthreads();
        if (tid < 2 * TI) {
            const int var = tid < TI ? i0 + tid : m0 + tid - TI;
            const unsigned long long kv = kmax[tid];
            if (var < M && kv) atomicMax(keys + var, kv);
        }
    }
}

// ---------------------------------------------------------------------------
// k = 3: triples (a < b < e).  A block takes one a, a tile of b (TB = 16 RB)
// and a tile of e (TE = 16 RE); 16 x 16 threads, RB x RE triples each.
// Shared memory holds, per 32-word chunk, the AND planes of (a, b) for every
// bin pair and the planes of e.
// ---------------------------------------------------------------------------
template <int C>
struct K3Shape;
template <>
struct K3Shape<2> { static constexpr int RB = 4, RE = 4; };
template <>
struct K3Shape<3> { static constexpr int RB = 2, RE = 2; };
template <>
struct K3Shape<4> { static constexpr int RB = 1, RE = 2; };

template <int C>
__global__ void __launch_bounds__(256) k3_kernel(const uint32_t* __restrict__ planes, PlaneGeom g, int M, int d0,
                                                 const int2* __restrict__ items, const long long* __restrict__ tab,
                                                 const int* __restrict__ cnt1, const long long* __restrict__ sh2,
                                                 const int* __restrict__ cnt2, unsigned long long* __restrict__ keys,
                                                 EmitTable emit) {
    constexpr int P = C - 1, RB = K3Shape<C>::RB, RE = K3Shape<C>::RE;
    constexpr int TB = 16 * RB, TE = 16 * RE, WC = 32, LD = WC + 1;
    __shared__ uint32_t sa[P][WC];
    __shared__ uint32_t sab[P * P][TB][LD];
    __shared__ uint32_t se[P][TE][LD];
    __shared__ unsigned long long kb[TB], ke[TE], ka;

    const int2 it = items[blockIdx.x];
    const int a = it.x;
    const int b0 = a + 1 + (it.y >> 16) * TB;
    const int e0 = a + 1 + (it.y & 0xFFFF) * TE;
    const int dl = blockIdx.y, d = d0 + dl;
    const int tid = threadIdx.x, tb = tid >> 4, te = tid & 15;
    const uint32_t* pbase = planes + (size_t)d * M * P * g.Ws;

    int acc[2][RB][RE][P][P][P];
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
        for (int rb = 0; rb < RB; ++rb)
#pragma unroll
            for (int re = 0; re < RE; ++re)
#pragma unroll
                for (int p = 0; p < P; ++p)
#pragma unroll
                    for (int q = 0; q < P; ++q)
#pragma unroll
                        for (int s = 0; s < P; ++s) acc[c2][rb][re][p][q][s] = 0;

#pragma unroll
    for (int cls = 0; cls < 2; ++cls) {
        const int wb = cls == 0 ? 0 : g.W0, we = cls == 0 ? g.W0 : g.W;
        for (int w0 = wb; w0 < we; w0 += WC) {
            const int nw = min(WC, we - w0);
            __syncthreads();
            for (int idx = tid; idx < P * WC; idx += 256) {
                const int w = idx % WC, p = idx / WC;
                sa[p][w] = (w < nw) ? pbase[((size_t)a * P + p) * g.Ws + w0 + w] : 0u;
            }
            __syncthreads();
            for (int idx = tid; idx < P * TB * WC; idx += 256) {
                const int w = idx % WC, rest = idx / WC, r = rest % TB, q = rest / TB;
                const int vb = b0 + r;
                const uint32_t pb = (w < nw && vb < M) ? pbase[((size_t)vb * P + q) * g.Ws + w0 + w] : 0u;
#pragma unroll
                for (int p = 0; p < P; ++p) sab[p * P + q][r][w] = sa[p][w] & pb;
            }
            for (int idx = tid; idx < P * TE * WC; idx += 256) {
                const int w = idx % WC, rest = idx / WC, r = rest % TE, s = rest / TE;
                const int ve = e0 + r;
                se[s][r][w] = (w < nw && ve < M) ? pbase[((size_t)ve * P + s) * g.Ws + w0 + w] : 0u;
            }
            __syncthreads();
            for (int w = 0; w < nw; ++w) {
                uint32_t ee[RE][P];
#pragma unroll
                for (int re = 0; re < RE; ++re)
#pragma unroll
                    for (int s = 0; s < P; ++s) ee[re][s] = se[s][te + 16 * re][w];
#pragma unroll
                for (int rb = 0; rb < RB; ++rb)
#pragma unroll
                    for (int pq = 0; pq < P * P; ++pq) {
                        const uint32_t ab = sab[pq][tb + 16 * rb][w];
#pragma unroll
                        for (int re = 0; re < RE; ++re)
#pragma unroll
                            for (int s = 0; s < P; ++s) acc[cls][rb][re][pq / P][pq % P][s] += __popc(ab & ee[re][s]);
                    }
            }
        }
    }

    for (int i = tid; i < TB; i += 256) kb[i] = 0ull;
    for (int i = tid; i < TE; i += 256) ke[i] = 0ull;
    if (tid == 0) ka = 0ull;
    __syncthreads();

    const int np1 = g.N + 1;
    const long long* tab0 = tab;
    const long long* tab1 = tab + np1;
    const long long* tabT = tab + 2 * np1;
    const size_t dM = (size_t)dl * M;
    int na0[P], na1[P], naT[P];
    {
        const int* c = cnt1 + ((size_t)d * M + a) * P * 2;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            na0[p] = __ldg(c + 2 * p);
            na1[p] = __ldg(c + 2 * p + 1);
            naT[p] = na0[p] + na1[p];
        }
    }
    unsigned long long my_ka = 0ull;
#pragma unroll
    for (int rb = 0; rb < RB; ++rb) {
        const int b = b0 + tb + 16 * rb;
        if (b >= M) continue;
        int nb0[P], nb1[P], nbT[P];
        {
            const int* c = cnt1 + ((size_t)d * M + b) * P * 2;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                nb0[p] = __ldg(c + 2 * p);
                nb1[p] = __ldg(c + 2 * p + 1);
                nbT[p] = nb0[p] + nb1[p];
            }
        }
        const size_t pab = (dM + a) * M + b;
        int nab0[P][P], nab1[P][P], nabT[P][P];
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int q = 0; q < P; ++q) {
                nab0[p][q] = __ldg(cnt2 + (pab * P * P + p * P + q) * 2);
                nab1[p][q] = __ldg(cnt2 + (pab * P * P + p * P + q) * 2 + 1);
                nabT[p][q] = nab0[p][q] + nab1[p][q];
            }
        const long long sh_ab = __ldg(sh2 + pab);
        unsigned long long my_kb = 0ull;
#pragma unroll
        for (int re = 0; re < RE; ++re) {
            const int e = e0 + te + 16 * re;
            if (e >= M || e <= b) continue;
            int ne0[P], ne1[P], neT[P];
            {
                const int* c = cnt1 + ((size_t)d * M + e) * P * 2;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    ne0[p] = __ldg(c + 2 * p);
                    ne1[p] = __ldg(c + 2 * p + 1);
                    neT[p] = ne0[p] + ne1[p];
                }
            }
            const size_t pae = (dM + a) * M + e, pbe = (dM + b) * M + e;
            int nae0[P][P], nae1[P][P], naeT[P][P], nbe0[P][P], nbe1[P][P], nbeT[P][P];
#pragma unroll
            for (int p = 0; p < P; ++p)
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    nae0[p][q] = __ldg(cnt2 + (pae * P * P + p * P + q) * 2);
                    nae1[p][q] = __ldg(cnt2 + (pae * P * P + p * P + q) * 2 + 1);
                    naeT[p][q] = nae0[p][q] + nae1[p][q];
                    nbe0[p][q] = __ldg(cnt2 + (pbe * P * P + p * P + q) * 2);
                    nbe1[p][q] = __ldg(cnt2 + (pbe * P * P + p * P + q) * 2 + 1);
                    nbeT[p][q] = nbe0[p][q] + nbe1[p][q];
                }
            int X0[P][P][P], X1[P][P][P], XT[P][P][P];
#pragma unroll
            for (int p = 0; p < P; ++p)
#pragma unroll
                for (int q = 0; q < P; ++q)
#pragma unroll
                    for (int s = 0; s < P; ++s) {
                        X0[p][q][s] = acc[0][rb][re][p][q][s];
                        X1[p][q][s] = acc[1][rb][re][p][q][s];
                        XT[p][q][s] = X0[p][q][s] + X1[p][q][s];
                    }
            const long long sh3 = channel3<C>(XT, nabT, naeT, nbeT, naT, nbT, neT, g.N, tabT) -
                                  channel3<C>(X0, nab0, nae0, nbe0, na0, nb0, ne0, g.N0, tab0) -
                                  channel3<C>(X1, nab1, nae1, nbe1, na1, nb1, ne1, g.N1, tab1);
            const uint32_t base = (uint32_t)d * (uint32_t)M;
            // IG(a | b, e), IG(b | a, e), IG(e | a, b)
            const unsigned long long k_a =
                pack_key(fx_to_float(__ldg(sh2 + pbe) - sh3), (base + (uint32_t)b) * (uint32_t)M + (uint32_t)e);
            const unsigned long long k_b =
                pack_key(fx_to_float(__ldg(sh2 + pae) - sh3), (base + (uint32_t)a) * (uint32_t)M + (uint32_t)e);
            const unsigned long long k_e =
                pack_key(fx_to_float(sh_ab - sh3), (base + (uint32_t)a) * (uint32_t)M + (uint32_t)b);
            my_ka = k_a > my_ka ? k_a : my_ka;
            my_kb = k_b > my_kb ? k_b : my_kb;
            atomicMax(&ke[te + 16 * re], k_e);
            if (emit.keys) {  // IG(a | b,e), IG(b | a,e), IG(e | a,b)
                const long long ga = __ldg(sh2 + pbe) - sh3, gb = __ldg(sh2 + pae) - sh3, ge = sh_ab - sh3;
                if (ga >= emit.thr_fx) emit_insert(emit, emit_key(a, b, e, -1), pack_key(fx_to_float(ga), (uint32_t)d));
                if (gb >= emit.thr_fx) emit_insert(emit, emit_key(b, a, e, -1), pack_key(fx_to_float(gb), (uint32_t)d));
                if (ge >= emit.thr_fx) emit_insert(emit, emit_key(e, a, b, -1), pack_key(fx_to_float(ge), (uint32_t)d));
            }
        }
        if (my_kb) atomicMax(&kb[tb + 16 * rb], my_kb);
    }
    // warp max of the a-role keys
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, my_ka, o);
        my_ka = other > my_ka ? other : my_ka;
    }
    if ((tid & 31) == 0 && my_ka) atomicMax(&ka, my_ka);
    __syncthreads();
    if (tid == 0 && ka) atomicMax(keys + a, ka);
    for (int i = tid; i < TB; i += 256)
        if (kb[i] && b0 + i < M) atomicMax(keys + b0 + i, kb[i]);
    for (int i = tid; i < TE; i += 256)
        if (ke[i] && e0 + i < M) atomicMax(keys + e0 + i, ke[i]);
}

// ---------------------------------------------------------------------------
__global__ void finalize_kernel(const unsigned long long* __restrict__ keys, int M, int k, float* __restrict__ ig,
                                int* __restrict__ tuples, int* __restrict__ disc, const int* __restrict__ kdisc) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= M) return;
    const unsigned long long key = keys[v];
    const uint32_t index = ~(uint32_t)(key & 0xFFFFFFFFull);
    ig[v] = key ? order_bits_float((uint32_t)(key >> 32)) : __int_as_float(0x7fc00000);
    int d = 0;
    if (k == 1) {
        d = (int)index;
    } else if (k == 2) {
        d = (int)(index / (uint32_t)M);
        if (tuples) tuples[v] = (int)(index % (uint32_t)M);
    } else if (k == 3) {
        const uint32_t mm = (uint32_t)M * (uint32_t)M;
        d = (int)(index / mm);
        const uint32_t rem = index % mm;
        if (tuples) {
            tuples[2 * v] = (int)(rem / (uint32_t)M);
            tuples[2 * v + 1] = (int)(rem % (uint32_t)M);
        }
    } else if (k == 5) {
        // index = d C(M,4) + rho, rho = C(M,4) - 1 - R and
        // R = C(t1,4) + C(t2,3) + C(t3,2) + C(t4,1), t_j = M - 1 - p_j
        const unsigned long long m = (unsigned long long)M;
        const unsigned long long k4 = m * (m - 1) / 2 * (m - 2) / 3 * (m - 3) / 4;
        d = kdisc ? kdisc[v] : (int)(index / k4);
        unsigned long long R = k4 - 1ull - (kdisc ? (unsigned long long)index : index % k4);
        int p[4];
        unsigned long long t = m;  // t_j strictly decreasing
        for (int j = 0; j < 4; ++j) {
            const int r = 4 - j;  // C(t, r)
            auto binom = [r](unsigned long long x) {
                unsigned long long v = 1;
                for (int i = 0; i < r; ++i) v = v * (x - i) / (i + 1);
                return x < (unsigned long long)r ? 0ull : v;
            };
            unsigned long long x = t - 1;
            while (binom(x) > R) --x;
            R -= binom(x);
            p[j] = (int)(m - 1 - x);
            t = x;
        }
        if (tuples)
            for (int j = 0; j < 4; ++j) tuples[4 * v + j] = p[j];
    } else {  // k = 4: ((d M + p1) M + p2) M + p3
        const uint32_t p3 = index % (uint32_t)M, r2 = index / (uint32_t)M;
        const uint32_t p2 = r2 % (uint32_t)M, r1 = r2 / (uint32_t)M;
        const uint32_t p1 = r1 % (uint32_t)M;
        d = (int)(r1 / (uint32_t)M);
        if (tuples) {
            tuples[3 * v] = (int)p1;
            tuples[3 * v + 1] = (int)p2;
            tuples[3 * v + 2] = (int)p3;
        }
    }
    if (disc) disc[v] = key ? d : -1;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_k1(const uint32_t* planes, PlaneGeom g, int M, int c, int D, const long long* tab, int* cnt1,
                      long long* sh1, unsigned long long* keys, cudaStream_t st, EmitTable emit) {
    const int items = D * M;
    const int blocks = (items + 7) / 8;
    switch (c) {
        case 2: k1_kernel<2><<<blocks, 256, 0, st>>>(planes, g, M, D, tab, cnt1, sh1, keys, emit); break;
        case 3: k1_kernel<3><<<blocks, 256, 0, st>>>(planes, g, M, D, tab, cnt1, sh1, keys, emit); break;
        case 4: k1_kernel<4><<<blocks, 256, 0, st>>>(planes, g, M, D, tab, cnt1, sh1, keys, emit); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_k2(const uint32_t* planes, PlaneGeom g, int M, int c, int D, int d0, int nd, const long long* tab,
                      const int* cnt1, const long long* sh1, unsigned long long* keys, long long* sh2, int* cnt2,
                      PairC* pairs2, int fbits, cudaStream_t st, const int* rank, EmitTable emit) {
    if (pairs2 && c != 2) return cudaErrorInvalidValue;
    (void)D;
    const int ntile = (M + 31) / 32;
    dim3 grid(ntile * (ntile + 1) / 2, nd);
    switch (c) {
        case 2: k2_kernel<2><<<grid, 256, 0, st>>>(planes, g, M, d0, ntile, tab, cnt1, sh1, keys, sh2, cnt2, pairs2, fbits,
                                                    rank, emit); break;
        case 3: k2_kernel<3><<<grid, 256, 0, st>>>(planes, g, M, d0, ntile, tab, cnt1, sh1, keys, sh2, cnt2, pairs2, fbits,
                                                    rank, emit); break;
        case 4: k2_kernel<4><<<grid, 256, 0, st>>>(planes, g, M, d0, ntile, tab, cnt1, sh1, keys, sh2, cnt2, pairs2, fbits,
                                                    rank, emit); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int k3_tile_b(int c) { return c == 2 ? 64 : (c == 3 ? 32 : 16); }
int k3_tile_e(int c) { return c == 2 ? 64 : 32; }

cudaError_t launch_k3_items(const uint32_t* planes, PlaneGeom g, int M, int c, int d0, int nd, const int2* items,
                            int n_items, const long long* tab, const int* cnt1, const long long* sh2, const int* cnt2,
                            unsigned long long* keys, cudaStream_t st, EmitTable emit) {
    if (n_items == 0) return cudaSuccess;
    dim3 grid(n_items, nd);
    switch (c) {
        case 2: k3_kernel<2><<<grid, 256, 0, st>>>(planes, g, M, d0, items, tab, cnt1, sh2, cnt2, keys, emit); break;
        case 3: k3_kernel<3><<<grid, 256, 0, st>>>(planes, g, M, d0, items, tab, cnt1, sh2, cnt2, keys, emit); break;
        case 4: k3_kernel<4><<<grid, 256, 0, st>>>(planes, g, M, d0, items, tab, cnt1, sh2, cnt2, keys, emit); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize(const unsigned long long* keys, int M, int k, float* ig, int* tuples, int* disc,
                            cudaStream_t st, const int* kdisc) {
    finalize_kernel<<<(M + 255) / 256, 256, 0, st>>>(keys, M, k, ig, tuples, disc, k == 5 ? kdisc : nullptr);
    return cudaGetLastError();
}

}  // namespace mdfs
