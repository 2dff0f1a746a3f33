// k = 5 scan for two classes per variable (c = 2) from class-sorted bit planes
// (Eq. 1 with |S| = 4; voxel counters of section "Algorithm and
// implementation").
//
// For a quintuple a < b < c < e < f and one class, the 32 voxel counts follow
// from the all-ones counts n_T of the 32 subsets T of {a, b, c, e, f} by
// Moebius inversion over supersets (both classes packed in one word).  Every
// proper subset's count comes from the single, pair, triple and quadruple
// passes (the quadruple tables also hold SH of every quadruple), so the
// kernel counts only n_abcef = popc(A&B&C&E&F) per 32 samples.
//
// Work item: (b, c, a tile of 32 e > c, a tile of 32 f > e); the CTA loops
// over every a < b with B&C and the e and f rows staged once.  The five roles:
// IG(a | b,c,e,f) = SH(bcef) - SH(abcef), IG(b | ...) from SH(acef),
// IG(c | ...) from SH(abef), IG(e | ...) from SH(abcf), IG(f | ...) from
// SH(abce), the quadruple entropies read from the tables.  Entropies are
// exact int64 fixed-point sums of the f(n + beta) tables.
//
// Argmax key: index = d C(M,4) + rho(S), rho the lexicographic rank of the
// partner set S among the 4-subsets of [0, M) (the same rank indexes the
// quadruple tables).  The caller guarantees D C(M,4) < 2^32.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "mdfs_device.cuh"
#include "mdfs_internal.cuh"
#include "mdfs_packed.cuh"

namespace mdfs {

namespace {

constexpr int kThreads = 256;
constexpr int kTE = 32, kTF = 32;  // e and f tile; thread (ty, tx) owns e = 2 ty + {0,1}, f = tx + {0,16}
constexpr int kWC = 128;           // staged words per chunk (even)
constexpr int kLD = kWC + 2;       // row stride: uint2 loads, f rows two banks apart

__device__ __forceinline__ unsigned long long kmax(unsigned long long a, unsigned long long b) { return a > b ? a : b; }

// Interesting-tuple records of the five roles of (a, b, c, e, f), partners
// ascending; kept out of line (taken only when emitting).
__device__ __noinline__ void emit_roles5(EmitTable t, int a, int b, int c, int e, int f, long long ga, long long gb,
                                         long long gc, long long ge, long long gf, int d) {
    if (ga >= t.thr_fx) emit_insert(t, emit_key5(a, b, c, e, f), pack_key(fx_to_float(ga), (uint32_t)d));
    if (gb >= t.thr_fx) emit_insert(t, emit_key5(b, a, c, e, f), pack_key(fx_to_float(gb), (uint32_t)d));
    if (gc >= t.thr_fx) emit_insert(t, emit_key5(c, a, b, e, f), pack_key(fx_to_float(gc), (uint32_t)d));
    if (ge >= t.thr_fx) emit_insert(t, emit_key5(e, a, b, c, f), pack_key(fx_to_float(ge), (uint32_t)d));
    if (gf >= t.thr_fx) emit_insert(t, emit_key5(f, a, b, c, e), pack_key(fx_to_float(gf), (uint32_t)d));
}

__global__ void __launch_bounds__(kThreads, 2) k5_kernel(const uint32_t* __restrict__ planes, PlaneGeom g, int M,
                                                        int d0, const int2* __restrict__ items,
                                                        const long long* __restrict__ tab,
                                                        const int* __restrict__ cnt1, const int* __restrict__ cnt2,
                                                        const uint32_t* __restrict__ t3c,
                                                        const uint32_t* __restrict__ t4c,
                                                        const long long* __restrict__ t4s,
                                                        unsigned long long* __restrict__ keys, EmitTable emit) {
    __shared__ __align__(16) uint32_t sE[kTE * kLD], sF[kTF * kLD], sBC[kWC], sABC[kWC];
    // per e / f row: item part (n_x, n_bx, n_cx, n_bcx), a part (n_ax, n_abx, n_acx, n_abcx)
    __shared__ uint32_t eI[kTE][4], fI[kTF][4], eA[kTE][4], fA[kTF][4];
    __shared__ long long shE[kTE], shF[kTF];  // SH(a,b,c,e), SH(a,b,c,f)
    __shared__ uint32_t sa4[4];               // n_a, n_ab, n_ac, n_abc
    __shared__ unsigned long long ka, kbc[2], kf[kTF];

    const int2 it = items[blockIdx.x];
    const int b = it.x & 0xFFFF, c = it.x >> 16;
    const int e0 = c + 1 + (it.y >> 16) * kTE;
    const int f0 = e0 + 1 + (it.y & 0xFFFF) * kTF;
    const int dl = blockIdx.y, d = d0 + dl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ty = tid >> 4, tx = tid & 15;
    const uint32_t* pbase = planes + (size_t)d * M * g.Ws;
    const Staging z = make_staging(g.W0, g.W1);
    const int nchunk = (z.Wst + kWC - 1) / kWC;
    Tabs tb;
    tb.tab = tab;
    tb.np1 = g.N + 1;
    tb.N0 = g.N0;
    tb.N1 = g.N1;
    const uint32_t NC = pack2(g.N0, g.N1);
    const Rank3 r3 = make_rank3(M);
    const Rank4 r4 = make_rank4(M);
    const uint32_t* T3c = t3c + (size_t)dl * ((size_t)r3.top + 1);
    const uint32_t* T4c = t4c + (size_t)dl * ((size_t)r4.top + 1);
    const long long* T4s = t4s + (size_t)dl * ((size_t)r4.top + 1);

    auto single = [&](int v) -> uint32_t {
        const int* p = cnt1 + ((size_t)d * M + v) * 2;
        return pack2(__ldg(p), __ldg(p + 1));
    };
    auto pair = [&](int i, int m) -> uint32_t {  // i < m
        const int* p = cnt2 + (((size_t)dl * M + i) * M + m) * 2;
        return pack2(__ldg(p), __ldg(p + 1));
    };

    // this thread's e and f, and validity of its four pairs
    int ev[2], fv[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        ev[r] = e0 + 2 * ty + r;
        fv[r] = f0 + tx + 16 * r;
    }
    // a warp owns e rows 4w .. 4w+3: it has work iff its first e has an f above it
    const bool warp_live = e0 + 4 * warp < M - 1;

    auto stage_rows = [&](int ch) {
        const int s0 = ch * kWC, len = min(kWC, z.Wst - s0);
        for (int idx = tid; idx < (kTE + kTF) * kWC; idx += kThreads) {
            const int r = idx / kWC, j = idx % kWC;
            uint32_t w = 0u;
            if (j < len) {
                const int v = r < kTE ? e0 + r : f0 + (r - kTE);
                if (v < M) w = staged_word(pbase + (size_t)v * g.Ws, s0 + j, z);
            }
            if (r < kTE) sE[r * kLD + j] = w;
            else sF[(r - kTE) * kLD + j] = w;
        }
        for (int j = tid; j < kWC; j += kThreads)
            sBC[j] = j < len ? staged_word(pbase + (size_t)b * g.Ws, s0 + j, z) &
                                   staged_word(pbase + (size_t)c * g.Ws, s0 + j, z)
                             : 0u;
    };

    // rank parts: R(w,x,y,z) = C(M-1-w,4) + C(M-1-x,3) + C(M-1-y,2) + (M-1-z);
    // table rank = C(M,4) - 1 - R, key index = d C(M,4) + table rank
    const uint32_t b4 = r4.part_w(b), b3 = r4.part_x(b), c3 = r4.part_x(c), c2 = r4.part_y(c);
    const uint32_t base = (uint32_t)((unsigned long long)d * ((unsigned long long)r4.top + 1ull)) + r4.top;

    // ---------------- item part ----------------
    const uint32_t nb = single(b), nc = single(c), nbc = pair(b, c);
    if (tid < kTE + kTF) {
        const int r = tid < kTE ? tid : tid - kTE;
        const int v = tid < kTE ? e0 + r : f0 + r;
        uint32_t* o = tid < kTE ? eI[r] : fI[r];
        if (v < M) {
            o[0] = single(v);
            o[1] = pair(b, v);
            o[2] = pair(c, v);
            o[3] = __ldg(T3c + r3.of(b, c, v));
        } else {
            o[0] = o[1] = o[2] = o[3] = 0u;
        }
        if (tid < kTF) kf[tid] = 0ull;
    }
    if (tid == 0) {
        ka = 0ull;
        kbc[0] = kbc[1] = 0ull;
    }
    if (nchunk == 1) stage_rows(0);
    // per-pair item values in rotation slots p = 2 re + rf: the pair epilogue
    // below is a rolled loop that always works on slot 0 and rotates the slots
    uint32_t nefs[4], pIs[4][3];  // n_ef; n_bef, n_cef, n_bcef
    long long shIs[4];            // SH(b, c, e, f)
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int e = ev[p >> 1], f = fv[p & 1];
        nefs[p] = pIs[p][0] = pIs[p][1] = pIs[p][2] = 0u;
        shIs[p] = 0;
        if (e < M && f < M && f > e) {
            const uint32_t ef = r4.part_y(e) + (uint32_t)(r4.Mm1 - f);
            nefs[p] = pair(e, f);
            pIs[p][0] = __ldg(T3c + r3.of(b, e, f));
            pIs[p][1] = __ldg(T3c + r3.of(c, e, f));
            const uint32_t i_bcef = r4.top - (b4 + c3 + ef);
            pIs[p][2] = __ldg(T4c + i_bcef);
            shIs[p] = __ldg(T4s + i_bcef);
        }
    }

    unsigned long long kB = 0ull, kC = 0ull, kE0 = 0ull, kE1 = 0ull, kF0 = 0ull, kF1 = 0ull;

    // ---------------- loop over a < b ----------------
    for (int a = 0; a < b; ++a) {
        __syncthreads();  // previous iteration's readers of the a-part tables and sABC are done
        const uint32_t a4 = r4.part_w(a);
        if (tid == 0) {
            if (ka) atomicMax(keys + (a - 1), ka);
            ka = 0ull;
            sa4[0] = single(a);
            sa4[1] = pair(a, b);
            sa4[2] = pair(a, c);
            sa4[3] = __ldg(T3c + r3.of(a, b, c));
        }
        if (tid < kTE + kTF) {  // the a part of every e and f row, and SH(a,b,c,x)
            const int r = tid < kTE ? tid : tid - kTE;
            const int v = tid < kTE ? e0 + r : f0 + r;
            uint32_t* o = tid < kTE ? eA[r] : fA[r];
            long long sh = 0;
            if (v < M) {
                const uint32_t i4 = r4.top - (a4 + b3 + c2 + (uint32_t)(r4.Mm1 - v));
                o[0] = pair(a, v);
                o[1] = __ldg(T3c + r3.of(a, b, v));
                o[2] = __ldg(T3c + r3.of(a, c, v));
                o[3] = __ldg(T4c + i4);
                sh = __ldg(T4s + i4);
            }
            if (tid < kTE) shE[r] = sh;
            else shF[r] = sh;
        }
        // counts of the triple and quadruples with a and the pair (e, f)
        uint32_t gA[4][3];  // n_aef, n_abef, n_acef per slot
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int e = ev[p >> 1], f = fv[p & 1];
            gA[p][0] = gA[p][1] = gA[p][2] = 0u;
            if (warp_live && e < M && f < M && f > e) {
                const uint32_t ef = r4.part_y(e) + (uint32_t)(r4.Mm1 - f);
                gA[p][0] = __ldg(T3c + r3.of(a, e, f));
                gA[p][1] = __ldg(T4c + (r4.top - (a4 + b3 + ef)));
                gA[p][2] = __ldg(T4c + (r4.top - (a4 + c3 + ef)));
            }
        }
        // n_abcef per pair
        uint32_t acc[2][2] = {{0u, 0u}, {0u, 0u}};
        for (int ch = 0; ch < nchunk; ++ch) {
            const int s0 = ch * kWC, len = min(kWC, z.Wst - s0);
            if (nchunk > 1) {
                if (ch > 0) __syncthreads();  // the previous chunk's readers are done
                stage_rows(ch);
                __syncthreads();  // sBC of this chunk staged
            }
            for (int j = tid; j < kWC; j += kThreads)
                sABC[j] = j < len ? staged_word(pbase + (size_t)a * g.Ws, s0 + j, z) & sBC[j] : 0u;
            __syncthreads();
            if (warp_live) {
                int lo[2], hi[2];
                class_segments(z, s0, kWC, lo, hi);
#pragma unroll
                for (int cls = 0; cls < 2; ++cls) {
                    const uint32_t mul = cls ? 65536u : 1u;
                    for (int j = lo[cls]; j < hi[cls]; j += 2) {
                        const uint2 s = *reinterpret_cast<const uint2*>(sABC + j);
                        uint2 e[2], f[2];
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            e[r] = *reinterpret_cast<const uint2*>(sE + (2 * ty + r) * kLD + j);
                            f[r] = *reinterpret_cast<const uint2*>(sF + (tx + 16 * r) * kLD + j);
                        }
#pragma unroll
                        for (int re = 0; re < 2; ++re) {
                            const uint32_t x0 = s.x & e[re].x, x1 = s.y & e[re].y;
#pragma unroll
                            for (int rf = 0; rf < 2; ++rf)
                                acc[re][rf] += (uint32_t)(__popc(x0 & f[rf].x) + __popc(x1 & f[rf].y)) * mul;
                        }
                    }
                }
            }
        }
        if (!warp_live) continue;
        const uint32_t na = sa4[0], nab = sa4[1], nac = sa4[2], nabc = sa4[3];
        uint32_t accs[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) accs[p] = acc[p >> 1][p & 1];
        unsigned long long kA = 0ull;
#pragma unroll 1
        for (int p = 0; p < 4; ++p) {
            const int re = p >> 1, rf = p & 1;
            const int e = e0 + 2 * ty + re, f = f0 + tx + 16 * rf;
            if (e < M && f < M && f > e) {
                const uint32_t e1 = (uint32_t)(r4.Mm1 - e), f1 = (uint32_t)(r4.Mm1 - f);
                const uint32_t ef = r4.part_y(e) + f1;
                const uint32_t R_acef = a4 + c3 + ef, R_abef = a4 + b3 + ef;
                const long long sh_acef = __ldg(T4s + (r4.top - R_acef)), sh_abef = __ldg(T4s + (r4.top - R_abef));
                const uint32_t* EI = eI[2 * ty + re];
                const uint32_t* EA = eA[2 * ty + re];
                const uint32_t* FI = fI[tx + 16 * rf];
                const uint32_t* FA = fA[tx + 16 * rf];
                // bits a = 1, b = 2, c = 4, e = 8, f = 16
                uint32_t q[32] = {NC,       na,       nb,       nab,       nc,       nac,       nbc,       nabc,
                                  EI[0],    EA[0],    EI[1],    EA[1],     EI[2],    EA[2],     EI[3],     EA[3],
                                  FI[0],    FA[0],    FI[1],    FA[1],     FI[2],    FA[2],     FI[3],     FA[3],
                                  nefs[0],  gA[0][0], pIs[0][0], gA[0][1], pIs[0][1], gA[0][2], pIs[0][2], accs[0]};
                moebius_packed<5>(q);
                const long long sh5 = sh_packed<5>(q, tb);
                const long long she = shE[2 * ty + re], shf = shF[tx + 16 * rf];
                const unsigned long long k_a = pack_key(fx_to_float(shIs[0] - sh5), base - (b4 + c3 + ef));
                const unsigned long long k_b = pack_key(fx_to_float(sh_acef - sh5), base - R_acef);
                const unsigned long long k_c = pack_key(fx_to_float(sh_abef - sh5), base - R_abef);
                const unsigned long long k_e = pack_key(fx_to_float(shf - sh5), base - (a4 + b3 + c2 + f1));
                const unsigned long long k_f = pack_key(fx_to_float(she - sh5), base - (a4 + b3 + c2 + e1));
                if (emit.keys)
                    emit_roles5(emit, a, b, c, e, f, shIs[0] - sh5, sh_acef - sh5, sh_abef - sh5, shf - sh5, she - sh5,
                                d);
                kA = kmax(kA, k_a);
                kB = kmax(kB, k_b);
                kC = kmax(kC, k_c);
                if (re) kE1 = kmax(kE1, k_e);
                else kE0 = kmax(kE0, k_e);
                if (rf) kF1 = kmax(kF1, k_f);
                else kF0 = kmax(kF0, k_f);
            }
            // rotate the slots (four rotations restore the item values)
            {
                const uint32_t n0 = nefs[0], t1 = accs[0];
                const long long s0 = shIs[0];
                uint32_t t0[3], t2[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    t0[k] = pIs[0][k];
                    t2[k] = gA[0][k];
                }
#pragma unroll
                for (int q2 = 0; q2 < 3; ++q2) {
                    nefs[q2] = nefs[q2 + 1];
                    shIs[q2] = shIs[q2 + 1];
                    accs[q2] = accs[q2 + 1];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        pIs[q2][k] = pIs[q2 + 1][k];
                        gA[q2][k] = gA[q2 + 1][k];
                    }
                }
                nefs[3] = n0;
                shIs[3] = s0;
                accs[3] = t1;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    pIs[3][k] = t0[k];
                    gA[3][k] = t2[k];
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) kA = kmax(kA, __shfl_xor_sync(0xffffffffu, kA, o));
        if (lane == 0 && kA) atomicMax(&ka, kA);
    }
    __syncthreads();
    if (tid == 0 && ka) atomicMax(keys + (b - 1), ka);
    // roles b, c (one variable each), e (per e row), f (per f row)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kB = kmax(kB, __shfl_xor_sync(0xffffffffu, kB, o));
        kC = kmax(kC, __shfl_xor_sync(0xffffffffu, kC, o));
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
        kE0 = kmax(kE0, __shfl_xor_sync(0xffffffffu, kE0, o));
        kE1 = kmax(kE1, __shfl_xor_sync(0xffffffffu, kE1, o));
    }
    kF0 = kmax(kF0, __shfl_xor_sync(0xffffffffu, kF0, 16));
    kF1 = kmax(kF1, __shfl_xor_sync(0xffffffffu, kF1, 16));
    if (lane == 0) {
        if (kB) atomicMax(&kbc[0], kB);
        if (kC) atomicMax(&kbc[1], kC);
    }
    if (tx == 0) {
        if (kE0) atomicMax(keys + ev[0], kE0);
        if (kE1) atomicMax(keys + ev[1], kE1);
    }
    if (lane < 16) {
        if (kF0) atomicMax(&kf[tx], kF0);
        if (kF1) atomicMax(&kf[tx + 16], kF1);
    }
    __syncthreads();
    if (tid == 0) {
        if (kbc[0]) atomicMax(keys + b, kbc[0]);
        if (kbc[1]) atomicMax(keys + c, kbc[1]);
    }
    if (tid < kTF && kf[tid]) atomicMax(keys + f0 + tid, kf[tid]);
}

}  // namespace

// (b | c << 16, e-tile << 16 | f-tile) for 1 <= b < c with a valid (e, f)
// pair in the tiles; the heaviest items (largest b: b iterations of the
// a-loop) first.
void build_k5_items(int M, std::vector<int2>& items) {
    items.clear();
    for (int b = M - 4; b >= 1; --b)
        for (int c = b + 1; c + 2 < M; ++c)
            for (int te = 0;; ++te) {
                const int emin = c + 1 + te * kTE;
                if (emin > M - 2) break;
                for (int tf = 0;; ++tf) {
                    const int fmin = emin + 1 + tf * kTF;
                    if (fmin > M - 1) break;
                    items.push_back(make_int2(b | (c << 16), (te << 16) | tf));
                }
            }
}

cudaError_t launch_k5(const uint32_t* planes, PlaneGeom g, int M, int d0, int nd, const int2* items, int n_items,
                      const long long* tab, const int* cnt1, const int* cnt2, const uint32_t* t3c,
                      const uint32_t* t4c, const long long* t4s, unsigned long long* keys, cudaStream_t st,
                      EmitTable emit) {
    if (n_items == 0 || nd == 0) return cudaSuccess;
    if (nd > 65535) return cudaErrorInvalidValue;
    k5_kernel<<<dim3(n_items, nd), kThreads, 0, st>>>(planes, g, M, d0, items, tab, cnt1, cnt2, t3c, t4c, t4s, keys,
                                                      emit);
    return cudaGetLastError();
}

}  // namespace mdfs
