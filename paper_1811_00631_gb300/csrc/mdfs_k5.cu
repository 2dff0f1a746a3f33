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
// quadruple tables; C(M,4) < 2^32).  When D C(M,4) does not fit 32 bits the
// caller passes per-discretisation keys [nd][M] and the index is rho alone;
// a separate fold keeps the lowest discretisation on ties.
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


// the a part of one e or f row: n_ax (two class counts), n_abx, n_acx, n_abcx, SH(a,b,c,x)
struct RowA {
    int2 ax;
    uint32_t abx, acx, abcx, pad;
    long long sh;
};
// the a part of the item: n_a, n_ab, n_ac (class counts), n_abc
struct ScalA {
    int2 a, ab, ac;
    uint32_t abc, pad;
};
struct K5Smem {
    uint32_t sE[kTE * kLD], sF[kTF * kLD];  // e and f rows (staged words)
    uint32_t sBC[kWC], sABC[kWC];
    uint32_t eI[kTE][4], fI[kTF][4];        // per row: n_x, n_bx, n_cx, n_bcx
    RowA rows[2][kTE + kTF];                // a part, double-buffered by the parity of a
    ScalA sa[2];
    uint32_t pI[4][4][kThreads];            // per thread and pair slot: n_ef, n_bef, n_cef, n_bcef
    long long shI[4][kThreads];             // SH(b, c, e, f)
    uint32_t gA[2][3][4][kThreads];         // n_aef, n_abef, n_acef, double-buffered
    unsigned long long ka, kbc[2], kf[kTF];
};

__global__ void __launch_bounds__(kThreads, 2) k5_kernel(const uint32_t* __restrict__ planes, PlaneGeom g, int M,
                                                        int d0, const int2* __restrict__ items,
                                                        const long long* __restrict__ tab,
                                                        const int* __restrict__ cnt1, const int* __restrict__ cnt2,
                                                        const uint32_t* __restrict__ t3c,
                                                        const uint32_t* __restrict__ t4c,
                                                        const long long* __restrict__ t4s,
                                                        unsigned long long* __restrict__ keys, int keys_stride,
                                                        uint32_t disc_mul, EmitTable emit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K5Smem& sm = *reinterpret_cast<K5Smem*>(smem_raw);

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
    keys += (size_t)dl * keys_stride;
    Tabs tb;
    tb.tab = tab;  // wide layout
    const uint32_t NC = pack2(g.N0, g.N1);
    const Rank3 r3 = make_rank3(M);
    const Rank4 r4 = make_rank4(M);
    const uint32_t* T3c = t3c + (size_t)dl * ((size_t)r3.top + 1);
    const uint32_t* T4c = t4c + (size_t)dl * ((size_t)r4.top + 1);
    const long long* T4s = t4s + (size_t)dl * ((size_t)r4.top + 1);
    const int* C1 = cnt1 + (size_t)d * M * 2;
    const int* C2 = cnt2 + (size_t)dl * M * M * 2;

    auto single = [&](int v) -> uint32_t { return pack2(__ldg(C1 + 2 * v), __ldg(C1 + 2 * v + 1)); };
    auto pair = [&](int i, int m) -> uint32_t {  // i < m
        const int* p = C2 + ((size_t)i * M + m) * 2;
        return pack2(__ldg(p), __ldg(p + 1));
    };

    // this thread's e and f
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
            if (r < kTE) sm.sE[r * kLD + j] = w;
            else sm.sF[(r - kTE) * kLD + j] = w;
        }
        for (int j = tid; j < kWC; j += kThreads)
            sm.sBC[j] = j < len ? staged_word(pbase + (size_t)b * g.Ws, s0 + j, z) &
                                      staged_word(pbase + (size_t)c * g.Ws, s0 + j, z)
                                : 0u;
    };

    // rank parts: R(w,x,y,z) = C(M-1-w,4) + C(M-1-x,3) + C(M-1-y,2) + (M-1-z);
    // table rank = C(M,4) - 1 - R, key index = d C(M,4) + table rank
    const uint32_t b4 = r4.part_w(b), b3 = r4.part_x(b), c3 = r4.part_x(c), c2 = r4.part_y(c);
    const uint32_t base = (uint32_t)d * disc_mul + r4.top;

    // asynchronous fetch of the a part into buffer `buf`
    auto fetch_a = [&](int a, int buf) {
        const uint32_t a4 = r4.part_w(a);
        if (tid == 0) {
            ScalA& S = sm.sa[buf];
            cp_async8(&S.a, C1 + 2 * a, true);
            cp_async8(&S.ab, C2 + ((size_t)a * M + b) * 2, true);
            cp_async8(&S.ac, C2 + ((size_t)a * M + c) * 2, true);
            cp_async4(&S.abc, T3c + r3.of(a, b, c), true);
        }
        if (tid < kTE + kTF) {
            const int v = tid < kTE ? e0 + tid : f0 + (tid - kTE);
            const bool ok = v < M;
            const int vv = ok ? v : c + 1;  // any valid row for the address of a zero-filled copy
            const uint32_t i4 = r4.top - (a4 + b3 + c2 + (uint32_t)(r4.Mm1 - vv));
            RowA& R = sm.rows[buf][tid];
            cp_async8(&R.ax, C2 + ((size_t)a * M + vv) * 2, ok);
            cp_async4(&R.abx, T3c + r3.of(a, b, vv), ok);
            cp_async4(&R.acx, T3c + r3.of(a, c, vv), ok);
            cp_async4(&R.abcx, T4c + i4, ok);
            cp_async8(&R.sh, T4s + i4, ok);
        }
        if (warp_live) {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int e = ev[p >> 1], f = fv[p & 1];
                const bool ok = e < M && f < M && f > e;
                const int ee = ok ? e : c + 1, ff = ok ? f : c + 2;  // c + 2 < M: some (e, f) exists
                const uint32_t ef = r4.part_y(ee) + (uint32_t)(r4.Mm1 - ff);
                cp_async4(&sm.gA[buf][0][p][tid], T3c + r3.of(a, ee, ff), ok);
                cp_async4(&sm.gA[buf][1][p][tid], T4c + (r4.top - (a4 + b3 + ef)), ok);
                cp_async4(&sm.gA[buf][2][p][tid], T4c + (r4.top - (a4 + c3 + ef)), ok);
            }
        }
        cp_async_commit();
    };

    // ---------------- item part ----------------
    const uint32_t nb = single(b), nc = single(c), nbc = pair(b, c);
    if (tid < kTE + kTF) {
        const int r = tid < kTE ? tid : tid - kTE;
        const int v = tid < kTE ? e0 + r : f0 + r;
        uint32_t* o = tid < kTE ? sm.eI[r] : sm.fI[r];
        if (v < M) {
            o[0] = single(v);
            o[1] = pair(b, v);
            o[2] = pair(c, v);
            o[3] = __ldg(T3c + r3.of(b, c, v));
        } else {
            o[0] = o[1] = o[2] = o[3] = 0u;
        }
        if (tid < kTF) sm.kf[tid] = 0ull;
    }
    if (tid == 0) {
        sm.ka = 0ull;
        sm.kbc[0] = sm.kbc[1] = 0ull;
    }
    if (b > 0) fetch_a(0, 0);
    if (nchunk == 1) stage_rows(0);
    // per-pair item values, slot p = 2 re + rf
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int e = ev[p >> 1], f = fv[p & 1];
        uint32_t v0 = 0u, v1 = 0u, v2 = 0u, v3 = 0u;
        long long sh = 0;
        if (e < M && f < M && f > e) {
            const uint32_t ef = r4.part_y(e) + (uint32_t)(r4.Mm1 - f);
            const uint32_t i_bcef = r4.top - (b4 + c3 + ef);
            v0 = pair(e, f);
            v1 = __ldg(T3c + r3.of(b, e, f));
            v2 = __ldg(T3c + r3.of(c, e, f));
            v3 = __ldg(T4c + i_bcef);
            sh = __ldg(T4s + i_bcef);
        }
        sm.pI[0][p][tid] = v0;
        sm.pI[1][p][tid] = v1;
        sm.pI[2][p][tid] = v2;
        sm.pI[3][p][tid] = v3;
        sm.shI[p][tid] = sh;
    }

    unsigned long long kB = 0ull, kC = 0ull, kE0 = 0ull, kE1 = 0ull, kF0 = 0ull, kF1 = 0ull;

    // ---------------- loop over a < b ----------------
    // The table values of the a part arrive by asynchronous copies issued one
    // iteration ahead, into the buffer of the parity of a.
    for (int a = 0; a < b; ++a) {
        const int buf = a & 1;
        cp_async_wait_all();
        __syncthreads();  // the a part has landed; the previous iteration's readers are done
        const uint32_t a4 = r4.part_w(a);
        if (tid == 0) {
            if (sm.ka) atomicMax(keys + (a - 1), sm.ka);
            sm.ka = 0ull;
        }
        if (a + 1 < b) fetch_a(a + 1, buf ^ 1);
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
                sm.sABC[j] = j < len ? staged_word(pbase + (size_t)a * g.Ws, s0 + j, z) & sm.sBC[j] : 0u;
            __syncthreads();
            if (warp_live) {
                int lo[2], hi[2];
                class_segments(z, s0, kWC, lo, hi);
#pragma unroll
                for (int cls = 0; cls < 2; ++cls) {
                    const uint32_t mul = cls ? 65536u : 1u;
                    for (int j = lo[cls]; j < hi[cls]; j += 2) {
                        const uint2 s = *reinterpret_cast<const uint2*>(sm.sABC + j);
                        uint2 e[2], f[2];
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            e[r] = *reinterpret_cast<const uint2*>(sm.sE + (2 * ty + r) * kLD + j);
                            f[r] = *reinterpret_cast<const uint2*>(sm.sF + (tx + 16 * r) * kLD + j);
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
        const ScalA& S = sm.sa[buf];
        const uint32_t na = pack2(S.a.x, S.a.y), nab = pack2(S.ab.x, S.ab.y), nac = pack2(S.ac.x, S.ac.y), nabc = S.abc;
        uint32_t accs[4] = {acc[0][0], acc[0][1], acc[1][0], acc[1][1]};
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
                const uint32_t* EI = sm.eI[2 * ty + re];
                const uint32_t* FI = sm.fI[tx + 16 * rf];
                const RowA& EA = sm.rows[buf][2 * ty + re];
                const RowA& FA = sm.rows[buf][kTE + tx + 16 * rf];
                // bits a = 1, b = 2, c = 4, e = 8, f = 16
                uint32_t q[32] = {NC,
                                  na,
                                  nb,
                                  nab,
                                  nc,
                                  nac,
                                  nbc,
                                  nabc,
                                  EI[0],
                                  pack2(EA.ax.x, EA.ax.y),
                                  EI[1],
                                  EA.abx,
                                  EI[2],
                                  EA.acx,
                                  EI[3],
                                  EA.abcx,
                                  FI[0],
                                  pack2(FA.ax.x, FA.ax.y),
                                  FI[1],
                                  FA.abx,
                                  FI[2],
                                  FA.acx,
                                  FI[3],
                                  FA.abcx,
                                  sm.pI[0][p][tid],
                                  sm.gA[buf][0][p][tid],
                                  sm.pI[1][p][tid],
                                  sm.gA[buf][1][p][tid],
                                  sm.pI[2][p][tid],
                                  sm.gA[buf][2][p][tid],
                                  sm.pI[3][p][tid],
                                  accs[0]};
                moebius_packed<5>(q);
                const long long sh5 = sh_packed<5>(q, tb);
                const long long shI = sm.shI[p][tid];
                const long long she = EA.sh, shf = FA.sh;
                const unsigned long long k_a = pack_key(fx_to_float(shI - sh5), base - (b4 + c3 + ef));
                const unsigned long long k_b = pack_key(fx_to_float(sh_acef - sh5), base - R_acef);
                const unsigned long long k_c = pack_key(fx_to_float(sh_abef - sh5), base - R_abef);
                const unsigned long long k_e = pack_key(fx_to_float(shf - sh5), base - (a4 + b3 + c2 + f1));
                const unsigned long long k_f = pack_key(fx_to_float(she - sh5), base - (a4 + b3 + c2 + e1));
                if (emit.keys)
                    emit_roles5(emit, a, b, c, e, f, shI - sh5, sh_acef - sh5, sh_abef - sh5, shf - sh5, she - sh5, d);
                kA = kmax(kA, k_a);
                kB = kmax(kB, k_b);
                kC = kmax(kC, k_c);
                if (re) kE1 = kmax(kE1, k_e);
                else kE0 = kmax(kE0, k_e);
                if (rf) kF1 = kmax(kF1, k_f);
                else kF0 = kmax(kF0, k_f);
            }
            const uint32_t t = accs[0];  // rotate the counts: slot p + 1 comes next
            accs[0] = accs[1];
            accs[1] = accs[2];
            accs[2] = accs[3];
            accs[3] = t;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) kA = kmax(kA, __shfl_xor_sync(0xffffffffu, kA, o));
        if (lane == 0 && kA) atomicMax(&sm.ka, kA);
    }
    cp_async_wait_all();
    __syncthreads();
    if (tid == 0 && sm.ka) atomicMax(keys + (b - 1), sm.ka);
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
        if (kB) atomicMax(&sm.kbc[0], kB);
        if (kC) atomicMax(&sm.kbc[1], kC);
    }
    if (tx == 0) {
        if (kE0) atomicMax(keys + ev[0], kE0);
        if (kE1) atomicMax(keys + ev[1], kE1);
    }
    if (lane < 16) {
        if (kF0) atomicMax(&sm.kf[tx], kF0);
        if (kF1) atomicMax(&sm.kf[tx + 16], kF1);
    }
    __syncthreads();
    if (tid == 0) {
        if (sm.kbc[0]) atomicMax(keys + b, sm.kbc[0]);
        if (sm.kbc[1]) atomicMax(keys + c, sm.kbc[1]);
    }
    if (tid < kTF && sm.kf[tid]) atomicMax(keys + f0 + tid, sm.kf[tid]);
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
                      const uint32_t* t4c, const long long* t4s, unsigned long long* keys, int keys_stride,
                      bool disc_in_index, cudaStream_t st, EmitTable emit) {
    if (n_items == 0 || nd == 0) return cudaSuccess;
    if (nd > 65535) return cudaErrorInvalidValue;
    const size_t smem = sizeof(K5Smem);
    cudaError_t e = ensure_dynamic_smem((const void*)k5_kernel, smem);
    if (e != cudaSuccess) return e;
    const unsigned long long m = (unsigned long long)M;
    const uint32_t disc_mul = disc_in_index ? (uint32_t)(m * (m - 1) / 2 * (m - 2) / 3 * (m - 3) / 4) : 0u;
    k5_kernel<<<dim3(n_items, nd), kThreads, smem, st>>>(planes, g, M, d0, items, tab, cnt1, cnt2, t3c, t4c, t4s,
                                                         keys, keys_stride, disc_mul, emit);
    return cudaGetLastError();
}

namespace {
__global__ void k5_merge_kernel(const unsigned long long* __restrict__ keys5, int nd, int M, int d0,
                                unsigned long long* __restrict__ best, int* __restrict__ best_d) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= M) return;
    unsigned long long b = best[v];
    int bd = best_d[v];
    for (int dl = 0; dl < nd; ++dl) {
        const unsigned long long k = keys5[(size_t)dl * M + v];
        if (k && (!b || (k >> 32) > (b >> 32))) {
            b = k;
            bd = d0 + dl;
        }
    }
    best[v] = b;
    best_d[v] = bd;
}
}  // namespace

cudaError_t launch_k5_merge(const unsigned long long* keys5, int nd, int M, int d0, unsigned long long* best,
                            int* best_d, cudaStream_t st) {
    k5_merge_kernel<<<(M + 255) / 256, 256, 0, st>>>(keys5, nd, M, d0, best, best_d);
    return cudaGetLastError();
}

}  // namespace mdfs
