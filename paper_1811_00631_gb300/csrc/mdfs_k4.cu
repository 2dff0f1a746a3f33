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
// Work item: (b, a tile of 32 c > b, a tile of 32 e > c); the CTA loops over
// every a < b with the c and e rows staged once, and fetches the table values
// of the next a (per c, per e, per pair) with cp.async while it counts the
// current one.  16 x 16 threads, 2 x 2 (c, e) per thread.  Keys index the
// partner triple as ((d M + p1) M + p2) M + p3.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "mdfs_device.cuh"
#include "mdfs_internal.cuh"
#include "mdfs_packed.cuh"

namespace mdfs {

namespace {

constexpr int kThreads = 256;
constexpr int kTC = 32, kTE = 32;  // thread (tc, te) owns c = 2 tc + {0,1}, e = te + {0,16}
constexpr int kWC = 128;           // staged words per chunk (even)
constexpr int kLD = kWC + 2;       // row stride: uint2 loads, e rows two banks apart

__device__ __forceinline__ unsigned long long kmax(unsigned long long a, unsigned long long b) { return a > b ? a : b; }


// the a part of one c or e row: n_ax (two class counts), n_abx, SH(a, b, x)
struct RowA4 {
    int2 ax;
    uint32_t abx, pad;
    long long sh;
};
struct K4Smem {
    uint32_t sC[kTC * kLD], sE[kTE * kLD];  // c and e rows (staged words)
    uint32_t sAB[kWC];
    uint32_t cI[kTC][2], eI[kTE][2];        // per row: n_x, n_bx
    RowA4 rows[2][kTC + kTE];               // a part, double-buffered by the parity of a
    int2 sa[2][2];                          // n_a, n_ab (class counts)
    uint32_t pI[2][4][kThreads];            // per thread and pair slot: n_ce, n_bce
    long long shI[4][kThreads];             // SH(b, c, e)
    uint32_t gA[2][4][kThreads];            // n_ace, double-buffered
    long long gS[2][4][kThreads];           // SH(a, c, e), double-buffered
    unsigned long long ka, kb, ke[kTE];
};

// kTable: instead of folding the four roles into keys, store n_abce and
// SH(a,b,c,e) of every quadruple at its lexicographic rank (the quadruple
// tables of the k = 5 scan; C(M,4) < 2^32).
template <bool kTable>
__global__ void __launch_bounds__(kThreads, 2) k4_kernel(const uint32_t* __restrict__ planes, PlaneGeom g, int M,
                                                        int d0, const int2* __restrict__ items,
                                                        const long long* __restrict__ tab,
                                                        const int* __restrict__ cnt1, const int* __restrict__ cnt2,
                                                        const uint32_t* __restrict__ t3c,
                                                        const long long* __restrict__ t3s,
                                                        unsigned long long* __restrict__ keys, EmitTable emit,
                                                        uint32_t* __restrict__ t4c, long long* __restrict__ t4s) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K4Smem& sm = *reinterpret_cast<K4Smem*>(smem_raw);

    const int2 it = items[blockIdx.x];
    const int b = it.x;
    const int c0 = b + 1 + (it.y >> 16) * kTC;
    const int e0 = c0 + 1 + (it.y & 0xFFFF) * kTE;
    const int dl = blockIdx.y, d = d0 + dl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tc = tid >> 4, te = tid & 15;
    const uint32_t* pbase = planes + (size_t)d * M * g.Ws;  // one plane per variable (c = 2)
    const Staging z = make_staging(g.W0, g.W1);
    const int nchunk = (z.Wst + kWC - 1) / kWC;
    Tabs tb;
    tb.tab = tab;  // wide layout
    const uint32_t NC = pack2(g.N0, g.N1);
    const Rank3 r3 = make_rank3(M);
    const uint32_t* T3c = t3c + (size_t)dl * ((size_t)r3.top + 1);
    const long long* T3s = t3s + (size_t)dl * ((size_t)r3.top + 1);
    const int* C1 = cnt1 + (size_t)d * M * 2;
    const int* C2 = cnt2 + (size_t)dl * M * M * 2;
    auto single = [&](int v) -> uint32_t { return pack2(__ldg(C1 + 2 * v), __ldg(C1 + 2 * v + 1)); };
    auto pair = [&](int i, int m) -> uint32_t {  // i < m
        const int* p = C2 + ((size_t)i * M + m) * 2;
        return pack2(__ldg(p), __ldg(p + 1));
    };

    int cv[2], ev[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        cv[r] = c0 + 2 * tc + r;
        ev[r] = e0 + te + 16 * r;
    }
    // a warp owns c rows 4w .. 4w+3: it has work iff its first c has an e above it
    const bool warp_live = c0 + 4 * warp < M - 1;

    auto stage_rows = [&](int ch) {
        const int s0 = ch * kWC, len = min(kWC, z.Wst - s0);
        for (int idx = tid; idx < (kTC + kTE) * kWC; idx += kThreads) {
            const int r = idx / kWC, j = idx % kWC;
            uint32_t w = 0u;
            if (j < len) {
                const int v = r < kTC ? c0 + r : e0 + (r - kTC);
                if (v < M) w = staged_word(pbase + (size_t)v * g.Ws, s0 + j, z);
            }
            if (r < kTC) sm.sC[r * kLD + j] = w;
            else sm.sE[(r - kTC) * kLD + j] = w;
        }
    };

    // asynchronous fetch of the a part into buffer `buf`
    auto fetch_a = [&](int a, int buf) {
        const uint32_t ra = r3.part_x(a), rab = ra + r3.part_y(b);
        if (tid == 0) {
            cp_async8(&sm.sa[buf][0], C1 + 2 * a, true);
            cp_async8(&sm.sa[buf][1], C2 + ((size_t)a * M + b) * 2, true);
        }
        if (tid < kTC + kTE) {
            const int v = tid < kTC ? c0 + tid : e0 + (tid - kTC);
            const bool ok = v < M;
            const int vv = ok ? v : b + 1;  // any valid row for the address of a zero-filled copy
            const uint32_t i3 = r3.top - (rab + (uint32_t)(r3.Mm1 - vv));
            RowA4& R = sm.rows[buf][tid];
            cp_async8(&R.ax, C2 + ((size_t)a * M + vv) * 2, ok);
            cp_async4(&R.abx, T3c + i3, ok);
            cp_async8(&R.sh, T3s + i3, ok);
        }
        if (!kTable && warp_live) {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int cc = cv[p >> 1], e = ev[p & 1];
                const bool ok = cc < M && e < M && e > cc;
                const int c1 = ok ? cc : b + 1, e1 = ok ? e : b + 2;  // b + 2 < M: some (c, e) exists
                const uint32_t i3 = r3.top - (ra + r3.part_y(c1) + (uint32_t)(r3.Mm1 - e1));
                cp_async4(&sm.gA[buf][p][tid], T3c + i3, ok);
                cp_async8(&sm.gS[buf][p][tid], T3s + i3, ok);
            }
        } else if (kTable && warp_live) {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int cc = cv[p >> 1], e = ev[p & 1];
                const bool ok = cc < M && e < M && e > cc;
                const int c1 = ok ? cc : b + 1, e1 = ok ? e : b + 2;
                const uint32_t i3 = r3.top - (ra + r3.part_y(c1) + (uint32_t)(r3.Mm1 - e1));
                cp_async4(&sm.gA[buf][p][tid], T3c + i3, ok);
            }
        }
        cp_async_commit();
    };

    // ---------------- item part ----------------
    const uint32_t nb = single(b), rb = r3.part_x(b);
    if (tid < kTC + kTE) {
        const int r = tid < kTC ? tid : tid - kTC;
        const int v = tid < kTC ? c0 + r : e0 + r;
        uint32_t* o = tid < kTC ? sm.cI[r] : sm.eI[r];
        o[0] = v < M ? single(v) : 0u;
        o[1] = v < M ? pair(b, v) : 0u;
        if (tid < kTE) sm.ke[tid] = 0ull;
    }
    if (tid == 0) sm.ka = sm.kb = 0ull;
    fetch_a(0, 0);
    if (nchunk == 1) stage_rows(0);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int cc = cv[p >> 1], e = ev[p & 1];
        uint32_t n_ce = 0u, n_bce = 0u;
        long long sh = 0;
        if (cc < M && e < M && e > cc) {
            const uint32_t i3 = r3.top - (rb + r3.part_y(cc) + (uint32_t)(r3.Mm1 - e));
            n_ce = pair(cc, e);
            n_bce = __ldg(T3c + i3);
            sh = __ldg(T3s + i3);
        }
        sm.pI[0][p][tid] = n_ce;
        sm.pI[1][p][tid] = n_bce;
        sm.shI[p][tid] = sh;
    }

    const uint32_t dM = (uint32_t)d * (uint32_t)M;
    unsigned long long kB = 0ull, kC0 = 0ull, kC1 = 0ull, kE0 = 0ull, kE1 = 0ull;
    const Rank4 r4 = make_rank4(kTable ? M : 4);
    const size_t t4base = kTable ? (size_t)dl * ((size_t)r4.top + 1) : 0;

    // ---------------- loop over a < b ----------------
    for (int a = 0; a < b; ++a) {
        const int buf = a & 1;
        cp_async_wait_all();
        __syncthreads();  // the a part has landed; the previous iteration's readers are done
        if (!kTable && tid == 0) {
            if (sm.ka) atomicMax(keys + (a - 1), sm.ka);
            sm.ka = 0ull;
        }
        if (a + 1 < b) fetch_a(a + 1, buf ^ 1);
        uint32_t x4[2][2] = {{0u, 0u}, {0u, 0u}};
        for (int ch = 0; ch < nchunk; ++ch) {
            const int s0 = ch * kWC, len = min(kWC, z.Wst - s0);
            if (nchunk > 1) {
                if (ch > 0) __syncthreads();  // the previous chunk's readers are done
                stage_rows(ch);
            }
            for (int j = tid; j < kWC; j += kThreads)
                sm.sAB[j] = j < len ? staged_word(pbase + (size_t)a * g.Ws, s0 + j, z) &
                                          staged_word(pbase + (size_t)b * g.Ws, s0 + j, z)
                                    : 0u;
            __syncthreads();
            if (warp_live) {
                int lo[2], hi[2];
                class_segments(z, s0, kWC, lo, hi);
#pragma unroll
                for (int cls = 0; cls < 2; ++cls) {
                    const uint32_t mul = cls ? 65536u : 1u;
                    for (int j = lo[cls]; j < hi[cls]; j += 2) {
                        const uint2 s = *reinterpret_cast<const uint2*>(sm.sAB + j);
                        uint2 cw[2], ew[2];
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            cw[r] = *reinterpret_cast<const uint2*>(sm.sC + (2 * tc + r) * kLD + j);
                            ew[r] = *reinterpret_cast<const uint2*>(sm.sE + (te + 16 * r) * kLD + j);
                        }
#pragma unroll
                        for (int rc = 0; rc < 2; ++rc) {
                            const uint32_t x0 = s.x & cw[rc].x, x1 = s.y & cw[rc].y;
#pragma unroll
                            for (int re = 0; re < 2; ++re)
                                x4[rc][re] += (uint32_t)(__popc(x0 & ew[re].x) + __popc(x1 & ew[re].y)) * mul;
                        }
                    }
                }
            }
        }
        if (!warp_live) continue;
        const uint32_t na = pack2(sm.sa[buf][0].x, sm.sa[buf][0].y), nab = pack2(sm.sa[buf][1].x, sm.sa[buf][1].y);
        uint32_t xs[4] = {x4[0][0], x4[0][1], x4[1][0], x4[1][1]};
        unsigned long long kA = 0ull;
#pragma unroll 1
        for (int p = 0; p < 4; ++p) {
            const int rc = p >> 1, re = p & 1;
            const int cc = c0 + 2 * tc + rc, e = e0 + te + 16 * re;
            if (cc < M && e < M && e > cc) {
                const RowA4& CA = sm.rows[buf][2 * tc + rc];
                const RowA4& EA = sm.rows[buf][kTC + te + 16 * re];
                const uint32_t* CI = sm.cI[2 * tc + rc];
                const uint32_t* EI = sm.eI[te + 16 * re];
                // bits a = 1, b = 2, c = 4, e = 8
                uint32_t q[16] = {NC,    na,    nb,    nab,   CI[0], pack2(CA.ax.x, CA.ax.y), CI[1], CA.abx,
                                  EI[0], pack2(EA.ax.x, EA.ax.y), EI[1], EA.abx, sm.pI[0][p][tid],
                                  sm.gA[buf][p][tid], sm.pI[1][p][tid], xs[0]};
                moebius_packed<4>(q);
                const long long sh4 = sh_packed<4>(q, tb);
                if (kTable) {
                    const size_t at = t4base + (r4.top - (r4.part_w(a) + r4.part_x(b) + r4.part_y(cc) +
                                                          (uint32_t)(r4.Mm1 - e)));
                    t4c[at] = xs[0];
                    t4s[at] = sh4;
                } else {
                    const long long sh_bce = sm.shI[p][tid], sh_ace = sm.gS[buf][p][tid];
                    const long long sh_abe = EA.sh, sh_abc = CA.sh;
                    // IG(a | b,c,e), IG(b | a,c,e), IG(c | a,b,e), IG(e | a,b,c)
                    const unsigned long long k_a = pack_key(fx_to_float(sh_bce - sh4),
                                                            ((dM + (uint32_t)b) * M + (uint32_t)cc) * M + (uint32_t)e);
                    const unsigned long long k_b = pack_key(fx_to_float(sh_ace - sh4),
                                                            ((dM + (uint32_t)a) * M + (uint32_t)cc) * M + (uint32_t)e);
                    const unsigned long long k_c = pack_key(fx_to_float(sh_abe - sh4),
                                                            ((dM + (uint32_t)a) * M + (uint32_t)b) * M + (uint32_t)e);
                    const unsigned long long k_e = pack_key(fx_to_float(sh_abc - sh4),
                                                            ((dM + (uint32_t)a) * M + (uint32_t)b) * M + (uint32_t)cc);
                    kA = kmax(kA, k_a);
                    kB = kmax(kB, k_b);
                    if (rc) kC1 = kmax(kC1, k_c);
                    else kC0 = kmax(kC0, k_c);
                    if (re) kE1 = kmax(kE1, k_e);
                    else kE0 = kmax(kE0, k_e);
                    if (emit.keys) {  // the four roles, partners ascending
                        const long long g4[4] = {sh_bce - sh4, sh_ace - sh4, sh_abe - sh4, sh_abc - sh4};
                        const unsigned long long ek[4] = {emit_key(a, b, cc, e), emit_key(b, a, cc, e),
                                                          emit_key(cc, a, b, e), emit_key(e, a, b, cc)};
#pragma unroll
                        for (int r = 0; r < 4; ++r)
                            if (g4[r] >= emit.thr_fx)
                                emit_insert(emit, ek[r], pack_key(fx_to_float(g4[r]), (uint32_t)d));
                    }
                }
            }
            const uint32_t t = xs[0];  // rotate the counts: slot p + 1 comes next
            xs[0] = xs[1];
            xs[1] = xs[2];
            xs[2] = xs[3];
            xs[3] = t;
        }
        if (!kTable) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) kA = kmax(kA, __shfl_xor_sync(0xffffffffu, kA, o));
            if (lane == 0 && kA) atomicMax(&sm.ka, kA);
        }
    }
    cp_async_wait_all();
    if (kTable) return;
    __syncthreads();
    if (tid == 0 && sm.ka) atomicMax(keys + (b - 1), sm.ka);
    // roles b (one variable), c (per c row), e (per e row)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kB = kmax(kB, __shfl_xor_sync(0xffffffffu, kB, o));
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
        kC0 = kmax(kC0, __shfl_xor_sync(0xffffffffu, kC0, o));
        kC1 = kmax(kC1, __shfl_xor_sync(0xffffffffu, kC1, o));
    }
    kE0 = kmax(kE0, __shfl_xor_sync(0xffffffffu, kE0, 16));
    kE1 = kmax(kE1, __shfl_xor_sync(0xffffffffu, kE1, 16));
    if (lane == 0 && kB) atomicMax(&sm.kb, kB);
    if (te == 0) {
        if (kC0) atomicMax(keys + cv[0], kC0);
        if (kC1) atomicMax(keys + cv[1], kC1);
    }
    if (lane < 16) {
        if (kE0) atomicMax(&sm.ke[te], kE0);
        if (kE1) atomicMax(&sm.ke[te + 16], kE1);
    }
    __syncthreads();
    if (tid == 0 && sm.kb) atomicMax(keys + b, sm.kb);
    if (tid < kTE && sm.ke[tid]) atomicMax(keys + e0 + tid, sm.ke[tid]);
}

}  // namespace

// (b, c-tile << 16 | e-tile) for b >= 1 with a valid (c, e) pair in the
// tiles; the heaviest items (largest b: b iterations of the a-loop) first.
void build_k4_items(int M, std::vector<int2>& items) {
    items.clear();
    for (int b = M - 3; b >= 1; --b)
        for (int tc = 0;; ++tc) {
            const int cmin = b + 1 + tc * kTC;
            if (cmin > M - 2) break;
            for (int te = 0;; ++te) {
                const int emin = cmin + 1 + te * kTE;
                if (emin > M - 1) break;
                items.push_back(make_int2(b, (tc << 16) | te));
            }
        }
}

cudaError_t launch_k4(const uint32_t* planes, PlaneGeom g, int M, int d0, int nd, const int2* items, int n_items,
                      const long long* tab, const int* cnt1, const int* cnt2, const uint32_t* t3c,
                      const long long* t3s, unsigned long long* keys, cudaStream_t st, EmitTable emit) {
    if (n_items == 0 || nd == 0) return cudaSuccess;
    if (nd > 65535) return cudaErrorInvalidValue;
    const size_t smem = sizeof(K4Smem);
    cudaError_t e = ensure_dynamic_smem((const void*)k4_kernel<false>, smem);
    if (e != cudaSuccess) return e;
    k4_kernel<false><<<dim3(n_items, nd), kThreads, smem, st>>>(planes, g, M, d0, items, tab, cnt1, cnt2, t3c, t3s,
                                                                keys, emit, nullptr, nullptr);
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
    const size_t smem = sizeof(K4Smem);
    cudaError_t e = ensure_dynamic_smem((const void*)k4_kernel<true>, smem);
    if (e != cudaSuccess) return e;
    k4_kernel<true><<<dim3(n_items, nd), kThreads, smem, st>>>(planes, g, M, d0, items, tab, cnt1, cnt2, t3c, t3s,
                                                               nullptr, EmitTable(), t4c, t4s);
    return cudaGetLastError();
}

}  // namespace mdfs
