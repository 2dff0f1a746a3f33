// k = 5 scan for two classes per variable (c = 2) from class-sorted bit planes
// (Eq. 1 with |S| = 4; voxel counters of section "Algorithm and
// implementation").
//
// For a quintuple a < b < c < e < f and one class, the 32 voxel counts follow
// from the all-ones counts n_T of the 32 subsets T of {a, b, c, e, f} by
// Moebius inversion over supersets.  Counts of the two classes travel packed
// in one word (class 0 in bits 0..15, class 1 in bits 16..31): inversion and
// marginalisation only add and subtract counts that stay non-negative, so the
// halves never borrow from each other (class sizes below 2^16).
//
// Work item: (b, c, a tile of 32 e > c, a tile of 32 f > e); the CTA loops
// over every a < b.  Everything that does not involve a is counted once per
// item: per (e, f) the all-ones counts of {b,e,f}, {c,e,f}, {b,c,e,f} and
// SH(b, c, e, f); per e (f) the counts of {b,c,e} ({b,c,f}).  Per a, each
// (e, f) pair needs four popcounts per 32 samples,
//     n_aef, n_abef, n_acef, n_abcef,
// and each e (f) three, n_abe, n_ace, n_abce.  Pairs and singles come from
// the pair and single passes.
//
// The five roles: IG(a | b,c,e,f) = SH(bcef) - SH(abcef), IG(b | a,c,e,f) =
// SH(acef) - SH(abcef), IG(c | ...) from SH(abef), IG(e | ...) from SH(abcf)
// and IG(f | ...) from SH(abce); SH(acef) and SH(abef) are marginals of the
// 32-voxel table.  Entropies are exact int64 fixed-point sums of the
// f(n + beta) tables.
//
// Argmax key: index = d C(M,4) + rho(S), rho the rank of the partner set S
// (ascending) in lexicographic order among the 4-subsets of [0, M), computed
// from the combinatorial number system on M-1-s.  The caller guarantees
// D C(M,4) < 2^32.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "mdfs_device.cuh"
#include "mdfs_internal.cuh"

namespace mdfs {

namespace {

constexpr int kThreads = 256;
constexpr int kTE = 32, kTF = 32;  // e and f tile; thread (ty, tx) owns e = 2 ty + {0,1}, f = tx + {0,16}
constexpr int kWC = 128;           // staged words per chunk (even)
constexpr int kLD = kWC + 2;       // row stride: uint2 loads, f rows two banks apart
constexpr uint32_t kLo = 0xFFFFu;

// binomial coefficients C(x, 2..4) for 0 <= x < 2^16, as 64-bit
__device__ __forceinline__ unsigned long long bin2(unsigned long long x) { return x * (x - 1) / 2; }
__device__ __forceinline__ unsigned long long bin3(unsigned long long x) { return x * (x - 1) * (x - 2) / 6; }
__device__ __forceinline__ unsigned long long bin4(unsigned long long x) {
    return x * (x - 1) * (x - 2) * (x - 3) / 24;
}

template <int L>
__device__ __forceinline__ void moebius_packed(uint32_t (&n)[1 << L]) {
#pragma unroll
    for (int j = 0; j < L; ++j)
#pragma unroll
        for (int m = 0; m < (1 << L); ++m)
            if (!(m & (1 << j))) n[m] -= n[m | (1 << j)];
}

// Lookup geometry of the f(n + beta) tables: T0 at [0, N], T1 at [N+1, 2N+1],
// TB at [2N+2, 3N+2]; class sizes clamp the indices (a count never exceeds its
// class size, so the clamp only keeps every read inside the tables).
struct Tabs {
    const long long* tab;
    int np1, N0, N1;
};
// SH over packed voxel counts: sum of f(n0+n1+b0+b1) - f(n0+b0) - f(n1+b1)
__device__ __forceinline__ long long voxel_sh(uint32_t v, const Tabs& t) {
    const int n0 = min((int)(v & kLo), t.N0), n1 = min((int)(v >> 16), t.N1);
    return __ldg(t.tab + 2 * t.np1 + n0 + n1) - __ldg(t.tab + n0) - __ldg(t.tab + t.np1 + n1);
}
template <int L>
__device__ __forceinline__ long long sh_packed(const uint32_t (&n)[1 << L], const Tabs& t) {
    long long s = 0;
#pragma unroll
    for (int m = 0; m < (1 << L); ++m) s += voxel_sh(n[m], t);
    return s;
}

__device__ __forceinline__ unsigned long long kmax(unsigned long long a, unsigned long long b) { return a > b ? a : b; }

// Staged word space: class-0 words at [0, W0e), class-1 words at [W0e, Wst),
// each class zero-padded to an even length so word pairs never straddle it.
struct Staging {
    int W0, W1, W0e, Wst;
};
__device__ __forceinline__ uint32_t staged_word(const uint32_t* __restrict__ row, int s, const Staging& z) {
    if (s < z.W0e) return s < z.W0 ? __ldg(row + s) : 0u;
    const int w = s - z.W0e;
    return w < z.W1 ? __ldg(row + z.W0 + w) : 0u;
}

// Per-pair counts over staged words [lo, hi) of one class (multiplier mul = 1
// or 2^16): acc[re][rf][k] += popc(S_k & E & F).
template <int NS>
__device__ __forceinline__ void pair_counts(const uint32_t* __restrict__ sE, const uint32_t* __restrict__ sF,
                                            const uint32_t* const (&str)[NS], int lo, int hi, uint32_t mul, int ty,
                                            int tx, uint32_t (&acc)[2][2][NS]) {
    for (int j = lo; j < hi; j += 2) {
        uint2 e[2], f[2], s[NS];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            e[r] = *reinterpret_cast<const uint2*>(sE + (2 * ty + r) * kLD + j);
            f[r] = *reinterpret_cast<const uint2*>(sF + (tx + 16 * r) * kLD + j);
        }
#pragma unroll
        for (int k = 0; k < NS; ++k) s[k] = *reinterpret_cast<const uint2*>(str[k] + j);
#pragma unroll
        for (int re = 0; re < 2; ++re)
#pragma unroll
            for (int rf = 0; rf < 2; ++rf) {
                const uint32_t x0 = e[re].x & f[rf].x, x1 = e[re].y & f[rf].y;
#pragma unroll
                for (int k = 0; k < NS; ++k)
                    acc[re][rf][k] += (uint32_t)(__popc(s[k].x & x0) + __popc(s[k].y & x1)) * mul;
            }
    }
}

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
                                                        unsigned long long* __restrict__ keys, EmitTable emit) {
    __shared__ __align__(16) uint32_t sE[kTE * kLD], sF[kTF * kLD];
    __shared__ __align__(16) uint32_t sB[kWC], sC[kWC], sBC[kWC], sA[kWC], sAB[kWC], sAC[kWC], sABC[kWC];
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
    Staging z;
    z.W0 = g.W0;
    z.W1 = g.W1;
    z.W0e = (g.W0 + 1) & ~1;
    z.Wst = z.W0e + ((g.W1 + 1) & ~1);
    const int nchunk = (z.Wst + kWC - 1) / kWC;
    Tabs tb;
    tb.tab = tab;
    tb.np1 = g.N + 1;
    tb.N0 = g.N0;
    tb.N1 = g.N1;
    const uint32_t NC = (uint32_t)g.N0 | ((uint32_t)g.N1 << 16);

    auto single = [&](int v) -> uint32_t {
        const int* p = cnt1 + ((size_t)d * M + v) * 2;
        return (uint32_t)__ldg(p) | ((uint32_t)__ldg(p + 1) << 16);
    };
    auto pair = [&](int i, int m) -> uint32_t {  // i < m
        const int* p = cnt2 + (((size_t)dl * M + i) * M + m) * 2;
        return (uint32_t)__ldg(p) | ((uint32_t)__ldg(p + 1) << 16);
    };

    // this thread's e and f, and validity of its four pairs
    int ev[2], fv[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        ev[r] = e0 + 2 * ty + r;
        fv[r] = f0 + tx + 16 * r;
    }
    bool ok[2][2];
#pragma unroll
    for (int re = 0; re < 2; ++re)
#pragma unroll
        for (int rf = 0; rf < 2; ++rf) ok[re][rf] = ev[re] < M && fv[rf] < M && fv[rf] > ev[re];
    // a warp owns e rows 4w .. 4w+3: it has work iff its first e has an f above it
    const bool warp_live = e0 + 4 * warp < M - 1;

    // class segments of chunk ch in local staged indices
    auto segments = [&](int ch, int (&lo)[2], int (&hi)[2]) {
        const int s0 = ch * kWC, s1 = min(s0 + kWC, z.Wst);
        lo[0] = 0;
        hi[0] = max(0, min(s1, z.W0e) - s0);
        lo[1] = max(s0, z.W0e) - s0;
        hi[1] = s1 - s0;
    };
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
        for (int j = tid; j < kWC; j += kThreads) {
            uint32_t wb = 0u, wc = 0u;
            if (j < len) {
                wb = staged_word(pbase + (size_t)b * g.Ws, s0 + j, z);
                wc = staged_word(pbase + (size_t)c * g.Ws, s0 + j, z);
            }
            sB[j] = wb;
            sC[j] = wc;
            sBC[j] = wb & wc;
        }
    };
    // warp-cooperative row counts: rows 0..31 = e, 32..63 = f; row 64 = the
    // a-part scalar.  Streams and output chosen by `apart`.
    auto row_counts = [&](int ch, bool apart) {
        int lo[2], hi[2];
        segments(ch, lo, hi);
        for (int r = warp; r < kTE + kTF + (apart ? 1 : 0); r += kThreads / 32) {
            const uint32_t* row = r < kTE ? sE + r * kLD : (r < kTE + kTF ? sF + (r - kTE) * kLD : nullptr);
            uint32_t t0 = 0u, t1 = 0u, t2 = 0u;
#pragma unroll
            for (int cls = 0; cls < 2; ++cls) {
                const uint32_t mul = cls ? 65536u : 1u;
                for (int j = lo[cls] + lane; j < hi[cls]; j += 32) {
                    if (!row) {
                        t2 += (uint32_t)__popc(sABC[j]) * mul;
                    } else if (apart) {
                        const uint32_t x = row[j];
                        t0 += (uint32_t)__popc(sAB[j] & x) * mul;
                        t1 += (uint32_t)__popc(sAC[j] & x) * mul;
                        t2 += (uint32_t)__popc(sABC[j] & x) * mul;
                    } else {
                        t2 += (uint32_t)__popc(sBC[j] & row[j]) * mul;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                t0 += __shfl_xor_sync(0xffffffffu, t0, o);
                t1 += __shfl_xor_sync(0xffffffffu, t1, o);
                t2 += __shfl_xor_sync(0xffffffffu, t2, o);
            }
            if (lane == 0) {
                if (!row) {
                    sa4[3] += t2;
                } else if (apart) {
                    uint32_t* o = r < kTE ? eA[r] : fA[r - kTE];
                    o[1] += t0;
                    o[2] += t1;
                    o[3] += t2;
                } else {
                    uint32_t* o = r < kTE ? eI[r] : fI[r - kTE];
                    o[3] += t2;
                }
            }
        }
    };

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
        } else {
            o[0] = o[1] = o[2] = 0u;
        }
        o[3] = 0u;
        if (tid < kTF) kf[tid] = 0ull;
    }
    if (tid == 0) {
        ka = 0ull;
        kbc[0] = kbc[1] = 0ull;
    }
    uint32_t pI[2][2][3];  // n_bef, n_cef, n_bcef
#pragma unroll
    for (int re = 0; re < 2; ++re)
#pragma unroll
        for (int rf = 0; rf < 2; ++rf)
#pragma unroll
            for (int k = 0; k < 3; ++k) pI[re][rf][k] = 0u;
    for (int ch = 0; ch < nchunk; ++ch) {
        __syncthreads();
        stage_rows(ch);
        __syncthreads();
        row_counts(ch, false);
        if (warp_live) {
            int lo[2], hi[2];
            segments(ch, lo, hi);
            const uint32_t* const str[3] = {sB, sC, sBC};
#pragma unroll
            for (int cls = 0; cls < 2; ++cls) pair_counts<3>(sE, sF, str, lo[cls], hi[cls], cls ? 65536u : 1u, ty, tx, pI);
        }
    }
    __syncthreads();
    // per-pair values in rotation slots p = 2 re + rf: the pair epilogue below
    // is a rolled loop that always works on slot 0 and rotates the slots
    uint32_t pIs[4][3], nefs[4];
    long long shIs[4];
    // SH(b, c, e, f) per pair: bits b = 1, c = 2, e = 4, f = 8
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int re = p >> 1, rf = p & 1;
#pragma unroll
        for (int k = 0; k < 3; ++k) pIs[p][k] = pI[re][rf][k];
        shIs[p] = 0;
        nefs[p] = 0u;
        if (!ok[re][rf]) continue;
        const uint32_t* E = eI[2 * ty + re];
        const uint32_t* F = fI[tx + 16 * rf];
        nefs[p] = pair(ev[re], fv[rf]);
        uint32_t q[16] = {NC,   nb,   nc,   nbc,  E[0],     E[1],       E[2],       E[3],
                          F[0], F[1], F[2], F[3], nefs[p], pIs[p][0], pIs[p][1], pIs[p][2]};
        moebius_packed<4>(q);
        shIs[p] = sh_packed<4>(q, tb);
    }

    // rank parts: rho(S) = C(M,4) - 1 - [C(M-1-s1,4) + C(M-1-s2,3) + C(M-1-s3,2) + (M-1-s4)]
    const unsigned long long K4 = bin4((unsigned long long)M);
    const uint32_t base = (uint32_t)((unsigned long long)(d + 1) * K4 - 1ull);
    const unsigned long long Mm1 = (unsigned long long)(M - 1);
    const uint32_t b4 = (uint32_t)bin4(Mm1 - b), b3 = (uint32_t)bin3(Mm1 - b);
    const uint32_t c3 = (uint32_t)bin3(Mm1 - c), c2 = (uint32_t)bin2(Mm1 - c);

    unsigned long long kB = 0ull, kC = 0ull, kE0 = 0ull, kE1 = 0ull, kF0 = 0ull, kF1 = 0ull;

    // ---------------- loop over a < b ----------------
    for (int a = 0; a < b; ++a) {
        __syncthreads();  // previous iteration's readers of the a-part tables are done
        if (tid == 0) {
            if (ka) atomicMax(keys + (a - 1), ka);
            ka = 0ull;
            sa4[0] = single(a);
            sa4[1] = pair(a, b);
            sa4[2] = pair(a, c);
            sa4[3] = 0u;
        }
        if (tid < kTE + kTF) {
            uint32_t* o = tid < kTE ? eA[tid] : fA[tid - kTE];
            o[1] = o[2] = o[3] = 0u;
        }
        uint32_t acc[2][2][4];
#pragma unroll
        for (int re = 0; re < 2; ++re)
#pragma unroll
            for (int rf = 0; rf < 2; ++rf)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[re][rf][k] = 0u;
        const uint32_t* const str[4] = {sA, sAB, sAC, sABC};
        for (int ch = 0; ch < nchunk; ++ch) {
            const int s0 = ch * kWC, len = min(kWC, z.Wst - s0);
            if (nchunk > 1) {
                if (ch > 0) __syncthreads();  // the previous chunk's readers are done
                stage_rows(ch);
            }
            for (int j = tid; j < kWC; j += kThreads) {
                const uint32_t wa = j < len ? staged_word(pbase + (size_t)a * g.Ws, s0 + j, z) : 0u;
                sA[j] = wa;
                sAB[j] = wa & sB[j];
                sAC[j] = wa & sC[j];
                sABC[j] = wa & sBC[j];
            }
            __syncthreads();
            row_counts(ch, true);
            if (nchunk > 1 && warp_live) {
                int lo[2], hi[2];
                segments(ch, lo, hi);
#pragma unroll
                for (int cls = 0; cls < 2; ++cls)
                    pair_counts<4>(sE, sF, str, lo[cls], hi[cls], cls ? 65536u : 1u, ty, tx, acc);
            }
        }
        __syncthreads();  // row counts complete
        const uint32_t na = sa4[0], nab = sa4[1], nac = sa4[2], nabc = sa4[3];
        // SH(a, b, c, x) per e row and f row (bits a = 1, b = 2, c = 4, x = 8),
        // four threads per row, one quarter of the voxels each
        {
            const int r = tid >> 2, qq = tid & 3;
            const bool isE = r < kTE;
            const int rr = isE ? r : r - kTE;
            const int v = isE ? e0 + rr : f0 + rr;
            uint32_t* A = isE ? eA[rr] : fA[rr];
            const uint32_t* I = isE ? eI[rr] : fI[rr];
            long long sh = 0;
            if (v < M) {
                const uint32_t nax = pair(a, v);
                uint32_t q[16] = {NC, na, nb, nab, nc, nac, nbc, nabc, I[0], nax, I[1], A[1], I[2], A[2], I[3], A[3]};
                moebius_packed<4>(q);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t w = qq == 0 ? q[4 * j] : (qq == 1 ? q[4 * j + 1] : (qq == 2 ? q[4 * j + 2] : q[4 * j + 3]));
                    sh += voxel_sh(w, tb);
                }
                if (qq == 0) A[0] = nax;
            }
            sh += __shfl_xor_sync(0xffffffffu, sh, 1);
            sh += __shfl_xor_sync(0xffffffffu, sh, 2);
            if (qq == 0) {
                if (isE) shE[rr] = sh;
                else shF[rr] = sh;
            }
        }
        if (nchunk == 1 && warp_live) {
            int lo[2], hi[2];
            segments(0, lo, hi);
#pragma unroll
            for (int cls = 0; cls < 2; ++cls)
                pair_counts<4>(sE, sF, str, lo[cls], hi[cls], cls ? 65536u : 1u, ty, tx, acc);
        }
        __syncthreads();  // SH(a,b,c,x), n_ax and the pair counts complete
        if (!warp_live) continue;
        const uint32_t a4 = (uint32_t)bin4(Mm1 - a), a3 = (uint32_t)bin3(Mm1 - a);
        uint32_t accs[4][4];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int k = 0; k < 4; ++k) accs[p][k] = acc[p >> 1][p & 1][k];
        unsigned long long kA = 0ull;
#pragma unroll 1
        for (int p = 0; p < 4; ++p) {
            const int re = p >> 1, rf = p & 1;
            const int e = e0 + 2 * ty + re, f = f0 + tx + 16 * rf;
            if (e < M && f < M && f > e) {
                const uint32_t* EI = eI[2 * ty + re];
                const uint32_t* EA = eA[2 * ty + re];
                const uint32_t* FI = fI[tx + 16 * rf];
                const uint32_t* FA = fA[tx + 16 * rf];
                // bits a = 1, b = 2, c = 4, e = 8, f = 16
                uint32_t q[32] = {NC,       na,          nb,          nab,         nc,          nac,
                                  nbc,      nabc,        EI[0],       EA[0],       EI[1],       EA[1],
                                  EI[2],    EA[2],       EI[3],       EA[3],       FI[0],       FA[0],
                                  FI[1],    FA[1],       FI[2],       FA[2],       FI[3],       FA[3],
                                  nefs[0],  accs[0][0],  pIs[0][0],   accs[0][1],  pIs[0][1],   accs[0][2],
                                  pIs[0][2], accs[0][3]};
                moebius_packed<5>(q);
                const long long sh5 = sh_packed<5>(q, tb);
                long long sh_acef = 0, sh_abef = 0;
#pragma unroll
                for (int m = 0; m < 16; ++m) {
                    const int mb = (m & 1) | ((m >> 1) << 2);  // a c e f -> drop b (bit 1)
                    const int mc = (m & 3) | ((m >> 2) << 3);  // a b e f -> drop c (bit 2)
                    sh_acef += voxel_sh(q[mb] + q[mb | 2], tb);
                    sh_abef += voxel_sh(q[mc] + q[mc | 4], tb);
                }
                const long long she = shE[2 * ty + re], shf = shF[tx + 16 * rf];
                const uint32_t e1 = (uint32_t)(M - 1 - e), f1 = (uint32_t)(M - 1 - f);
                const uint32_t tef = (uint32_t)bin2((unsigned long long)e1) + f1;
                const unsigned long long k_a = pack_key(fx_to_float(shIs[0] - sh5), base - (b4 + c3 + tef));
                const unsigned long long k_b = pack_key(fx_to_float(sh_acef - sh5), base - (a4 + c3 + tef));
                const unsigned long long k_c = pack_key(fx_to_float(sh_abef - sh5), base - (a4 + b3 + tef));
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
            // rotate the slots (four rotations restore the item constants)
            {
                const uint32_t n0 = nefs[0];
                const long long s0 = shIs[0];
                uint32_t t0[3], t1[4];
#pragma unroll
                for (int k = 0; k < 3; ++k) t0[k] = pIs[0][k];
#pragma unroll
                for (int k = 0; k < 4; ++k) t1[k] = accs[0][k];
#pragma unroll
                for (int q2 = 0; q2 < 3; ++q2) {
                    nefs[q2] = nefs[q2 + 1];
                    shIs[q2] = shIs[q2 + 1];
#pragma unroll
                    for (int k = 0; k < 3; ++k) pIs[q2][k] = pIs[q2 + 1][k];
#pragma unroll
                    for (int k = 0; k < 4; ++k) accs[q2][k] = accs[q2 + 1][k];
                }
                nefs[3] = n0;
                shIs[3] = s0;
#pragma unroll
                for (int k = 0; k < 3; ++k) pIs[3][k] = t0[k];
#pragma unroll
                for (int k = 0; k < 4; ++k) accs[3][k] = t1[k];
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
                      const long long* tab, const int* cnt1, const int* cnt2, unsigned long long* keys,
                      cudaStream_t st, EmitTable emit) {
    if (n_items == 0 || nd == 0) return cudaSuccess;
    if (nd > 65535) return cudaErrorInvalidValue;
    k5_kernel<<<dim3(n_items, nd), kThreads, 0, st>>>(planes, g, M, d0, items, tab, cnt1, cnt2, keys, emit);
    return cudaGetLastError();
}

}  // namespace mdfs
