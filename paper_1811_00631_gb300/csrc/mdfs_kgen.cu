// k = 4 and k = 5 scans for three or four classes per variable (Eq. 1 with
// |S| = 3, 4; voxel counters of section "Algorithm and implementation" over
// all c^k voxels).  The two-class scans have their own kernels (mdfs_k4.cu,
// mdfs_k5.cu) that read lower-order tables; here every voxel of a tuple is
// counted directly from the class-sorted bit planes.
//
// One warp per tuple (k = 4: two tuples that differ in the last variable at
// a time, for independent warp reductions).  The samples are visited in chunks of 32 words (one word
// of 32 samples per lane), class 0 first, then class 1, so a chunk holds one
// class.  A lane ANDs its word of the variables' bin planes (bin 0 is the
// complement of bins 1 .. c-1 among the valid samples) along an unrolled tree
// over the bins, so every voxel's word is formed with compile-time indices;
// popc gives the lane's count and one warp reduction (redux.sync.add) the
// chunk's, which the voxel's owner lane (voxel index mod 32) accumulates.
//
// Entropies are exact int64 fixed-point sums of the f(n + beta) tables
// (Eqs. H, p, beta): SH of the tuple over its c^k voxels, and for each role
// the SH of the other k-1 variables from the marginal counts (the c voxels
// that differ only in that variable's bin, summed).  IG(v | S) = SH(S) -
// SH(S + {v}) for every variable v of the tuple; keys as the two-class scans
// write them (k = 4: ((d M + p1) M + p2) M + p3; k = 5: d C(M,4) + the
// lexicographic rank of the partners).
//
// Work item: one pair (a, b) of the two lowest variables per CTA of 8 warps
// and one discretisation per grid row; the warps take the remaining prefix
// variables round robin and loop over the last variable.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <vector>

#include "mdfs_device.cuh"
#include "mdfs_internal.cuh"

namespace mdfs {

namespace {

constexpr int kWarps = 8;

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

__device__ __forceinline__ unsigned long long binom_dev(unsigned long long n, int r) {
    if (n < (unsigned long long)r) return 0ull;
    unsigned long long v = 1;
    for (int i = 0; i < r; ++i) v = v * (n - i) / (i + 1);
    return v;
}

// lexicographic rank of p1 < p2 < p3 < p4 among the C(M, 4) quadruples of [0, M)
__device__ __forceinline__ unsigned long long rank4(int M, const int* p) {
    const unsigned long long m = (unsigned long long)M;
    unsigned long long R = 0;
    for (int j = 0; j < 4; ++j) R += binom_dev(m - 1 - (unsigned long long)p[j], 4 - j);
    return binom_dev(m, 4) - 1ull - R;
}

__device__ __forceinline__ long long warp_sum64(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// valid-sample mask of word w (class 0 in words [0, W0), class 1 from W0)
__device__ __forceinline__ uint32_t valid_bits(const PlaneGeom& g, int w) {
    int nb;
    if (w < g.W0) nb = g.N0 - 32 * w;
    else if (w < g.W) nb = g.N1 - 32 * (w - g.W0);
    else nb = 0;
    return nb >= 32 ? 0xffffffffu : (nb <= 0 ? 0u : (1u << nb) - 1u);
}

// The K variables' bin words of word w into pl[i][b] (b = 0 .. C-1).
template <int K, int C>
__device__ __forceinline__ void load_bins(const uint32_t* __restrict__ pbase, const PlaneGeom& g, const int* v, int w,
                                          uint32_t (&pl)[K][C]) {
    const uint32_t valid = valid_bits(g, w);
#pragma unroll
    for (int i = 0; i < K; ++i) {
        uint32_t any = 0u;
#pragma unroll
        for (int b = 1; b < C; ++b) {
            const uint32_t x = valid ? __ldg(pbase + ((size_t)v[i] * (C - 1) + (b - 1)) * g.Ws + w) : 0u;
            pl[i][b] = x;
            any |= x;
        }
        pl[i][0] = valid & ~any;
    }
}

// Counts of every voxel over the samples (class 0 | class 1 << 16), left at
// the owner lane: voxel vx = sum_i b_i C^(K-1-i) (variable 0 most
// significant) in n0[vx >> 5], n1[vx >> 5] of lane vx & 31.
template <int K, int C>
__device__ __forceinline__ void count_voxels(const uint32_t* __restrict__ pbase, const PlaneGeom& g, const int* v,
                                             int lane, int (&n0)[(ipow(C, K) + 31) / 32],
                                             int (&n1)[(ipow(C, K) + 31) / 32]) {
    constexpr int V = ipow(C, K), NP = ipow(C, K - 2);
#pragma unroll
    for (int t = 0; t < (V + 31) / 32; ++t) n0[t] = n1[t] = 0;
    for (int cls = 0; cls < 2; ++cls) {
        const int wbeg = cls ? g.W0 : 0, wend = cls ? g.W : g.W0;
        for (int w0 = wbeg; w0 < wend; w0 += 32) {
            const int w = w0 + lane;
            uint32_t pl[K][C];
            load_bins<K, C>(pbase, g, v, w < wend ? w : g.Ws, pl);  // past the class: no valid samples
            // prefix words of variables 0 .. K-3, then the bins of the last two variables
            uint32_t pre[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                uint32_t x = 0xffffffffu;
                int r = p;
#pragma unroll
                for (int i = K - 3; i >= 0; --i) {
                    x &= pl[i][r % C];
                    r /= C;
                }
                pre[p] = x;
            }
#pragma unroll
            for (int p = 0; p < NP; ++p) {
#pragma unroll
                for (int b1 = 0; b1 < C; ++b1) {
                    const uint32_t x = pre[p] & pl[K - 2][b1];
#pragma unroll
                    for (int b = 0; b < C; ++b) {
                        const int vx = (p * C + b1) * C + b;
                        const int s = (int)__reduce_add_sync(0xffffffffu, (unsigned)__popc(x & pl[K - 1][b]));
                        if (lane == (vx & 31)) {
                            if (cls) n1[vx >> 5] += s;
                            else n0[vx >> 5] += s;
                        }
                    }
                }
            }
        }
    }
}

// The voxel counts of two tuples that differ only in the last variable (v[K-1]
// and e2), interleaved for independent warp reductions.
template <int K, int C>
__device__ __forceinline__ void count_voxels2(const uint32_t* __restrict__ pbase, const PlaneGeom& g, const int* v,
                                              int e2, int lane, int (&n0)[(ipow(C, K) + 31) / 32],
                                              int (&n1)[(ipow(C, K) + 31) / 32], int (&m0)[(ipow(C, K) + 31) / 32],
                                              int (&m1)[(ipow(C, K) + 31) / 32]) {
    constexpr int V = ipow(C, K), NP = ipow(C, K - 2);
#pragma unroll
    for (int t = 0; t < (V + 31) / 32; ++t) n0[t] = n1[t] = m0[t] = m1[t] = 0;
    for (int cls = 0; cls < 2; ++cls) {
        const int wbeg = cls ? g.W0 : 0, wend = cls ? g.W : g.W0;
        for (int w0 = wbeg; w0 < wend; w0 += 32) {
            const int w = w0 + lane;
            const int ww = w < wend ? w : g.Ws;
            uint32_t pl[K][C];
            load_bins<K, C>(pbase, g, v, ww, pl);
            uint32_t q[1][C];
            load_bins<1, C>(pbase, g, &e2, ww, q);
            uint32_t pre[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                uint32_t x = 0xffffffffu;
                int r = p;
#pragma unroll
                for (int i = K - 3; i >= 0; --i) {
                    x &= pl[i][r % C];
                    r /= C;
                }
                pre[p] = x;
            }
#pragma unroll
            for (int p = 0; p < NP; ++p) {
#pragma unroll
                for (int b1 = 0; b1 < C; ++b1) {
                    const uint32_t x = pre[p] & pl[K - 2][b1];
#pragma unroll
                    for (int b = 0; b < C; ++b) {
                        const int vx = (p * C + b1) * C + b;
                        const int sa = (int)__reduce_add_sync(0xffffffffu, (unsigned)__popc(x & pl[K - 1][b]));
                        const int sb = (int)__reduce_add_sync(0xffffffffu, (unsigned)__popc(x & q[0][b]));
                        if (lane == (vx & 31)) {
                            if (cls) {
                                n1[vx >> 5] += sa;
                                m1[vx >> 5] += sb;
                            } else {
                                n0[vx >> 5] += sa;
                                m0[vx >> 5] += sb;
                            }
                        }
                    }
                }
            }
        }
    }
}

// IG of every role of the tuple v[0] < .. < v[K-1] (int64 fixed point), from
// its voxel counts at the owner lanes; scnt: this warp's c^K shared words.
template <int K, int C>
__device__ __forceinline__ void tuple_ig(const long long* __restrict__ tab, int np1, int lane,
                                         const int (&n0)[(ipow(C, K) + 31) / 32],
                                         const int (&n1)[(ipow(C, K) + 31) / 32], uint32_t* scnt,
                                         long long (&ig)[K]) {
    constexpr int V = ipow(C, K), NP = ipow(C, K - 1);  // voxels; marginal voxels of one role
    long long sh = 0;
    __syncwarp();
#pragma unroll
    for (int t = 0; t < (V + 31) / 32; ++t) {
        const int vx = 32 * t + lane;
        if (vx < V) {
            scnt[vx] = (uint32_t)n0[t] | ((uint32_t)n1[t] << 16);
            sh += voxel_h(tab, np1, n0[t], n1[t]);
        }
    }
    __syncwarp();
    const long long sh_all = warp_sum64(sh);
#pragma unroll
    for (int i = 0; i < K; ++i) {
        // marginal voxel u over the other variables: the c voxels with digit i = 0 .. C-1
        const int lo = ipow(C, K - 1 - i);  // place value of digit i
        long long part = 0;
        for (int u = lane; u < NP; u += 32) {
            const int hi = u / lo, rest = u - hi * lo;
            const int base = hi * lo * C + rest;
            int m0 = 0, m1 = 0;
#pragma unroll
            for (int b = 0; b < C; ++b) {
                const uint32_t x = scnt[base + b * lo];
                m0 += (int)(x & 0xFFFFu);
                m1 += (int)(x >> 16);
            }
            part += voxel_h(tab, np1, m0, m1);
        }
        ig[i] = warp_sum64(part) - sh_all;
    }
}

// Three CTAs per SM where the registers allow it without spills (three classes:
// 69 and 79 registers; measured 1.3x and 1.4x the rate at one CTA per SM).
template <int K, int C>
__global__ void __launch_bounds__(32 * kWarps, (K == 4 && C == 3) ? 3 : (K == 5 && C == 3) ? 3 : 1) kgen_kernel(const uint32_t* __restrict__ planes, PlaneGeom g, int M,
                                                           int d0, const int2* __restrict__ items,
                                                           const long long* __restrict__ tab,
                                                           unsigned long long* __restrict__ keys, EmitTable emit) {
    constexpr int V = ipow(C, K);
    __shared__ uint32_t s_cnt[kWarps][V];
    const int2 it = items[blockIdx.x];
    const int a = it.x, b = it.y;
    const int dl = blockIdx.y, d = d0 + dl;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t* pbase = planes + (size_t)d * M * (C - 1) * g.Ws;
    const int np1 = g.N + 1;
    const unsigned long long m = (unsigned long long)M;
    const unsigned long long c4 = binom_dev(m, 4);
    uint32_t* scnt = s_cnt[warp];

    // role maxima of the variables fixed during the innermost loop (lane 0)
    unsigned long long kfix[K - 1];
    auto flush = [&](const int* v) {
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < K - 1; ++i)
                if (kfix[i]) atomicMax(keys + v[i], kfix[i]);
        }
    };
    // keys and emission of the roles of tuple v (lane 0)
    auto keys_of = [&](const int* v, const long long (&ig)[K]) {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            int p[K - 1];
            int j = 0;
#pragma unroll
            for (int q = 0; q < K; ++q)
                if (q != i) p[j++] = v[q];
            uint32_t index;
            if constexpr (K == 4)
                index = (((uint32_t)d * (uint32_t)M + (uint32_t)p[0]) * (uint32_t)M + (uint32_t)p[1]) * (uint32_t)M +
                        (uint32_t)p[2];
            else
                index = (uint32_t)((unsigned long long)d * c4 + rank4(M, p));
            const unsigned long long key = pack_key(fx_to_float(ig[i]), index);
            if (i < K - 1) kfix[i] = key > kfix[i] ? key : kfix[i];
            else atomicMax(keys + v[i], key);
            if (emit.keys && ig[i] >= emit.thr_fx) {
                unsigned long long ek;
                if constexpr (K == 4) ek = emit_key(v[i], p[0], p[1], p[2]);
                else ek = emit_key5(v[i], p[0], p[1], p[2], p[3]);
                emit_insert(emit, ek, pack_key(fx_to_float(ig[i]), (uint32_t)d));
            }
        }
    };
    // one tuple
    auto visit = [&](const int* v) {
        int n0[(V + 31) / 32], n1[(V + 31) / 32];
        count_voxels<K, C>(pbase, g, v, lane, n0, n1);
        long long ig[K];
        tuple_ig<K, C>(tab, np1, lane, n0, n1, scnt, ig);
        if (lane == 0) keys_of(v, ig);
    };
    // the tuples v and v with its last variable replaced by v[K-1] + 1, counted together (k = 4)
    auto visit2 = [&](int* v) {
        int n0[(V + 31) / 32], n1[(V + 31) / 32], m0[(V + 31) / 32], m1[(V + 31) / 32];
        count_voxels2<K, C>(pbase, g, v, v[K - 1] + 1, lane, n0, n1, m0, m1);
        long long ig[K];
        tuple_ig<K, C>(tab, np1, lane, n0, n1, scnt, ig);
        if (lane == 0) keys_of(v, ig);
        tuple_ig<K, C>(tab, np1, lane, m0, m1, scnt, ig);
        ++v[K - 1];
        if (lane == 0) keys_of(v, ig);
        --v[K - 1];
    };

    int v[K];
    v[0] = a;
    v[1] = b;
    if constexpr (K == 4) {
        for (int c = b + 1 + warp; c < M - 1; c += kWarps) {
            v[2] = c;
#pragma unroll
            for (int i = 0; i < K - 1; ++i) kfix[i] = 0ull;
            int e = c + 1;
            for (; e + 1 < M; e += 2) {
                v[3] = e;
                visit2(v);
            }
            if (e < M) {
                v[3] = e;
                visit(v);
            }
            flush(v);
        }
    } else {
        int q = 0;
        for (int c = b + 1; c < M - 2; ++c)
            for (int e = c + 1; e < M - 1; ++e, ++q) {
                if (q % kWarps != warp) continue;
                v[2] = c;
                v[3] = e;
#pragma unroll
                for (int i = 0; i < K - 1; ++i) kfix[i] = 0ull;
                // one tuple at a time: two would need more registers than a
                // useful occupancy allows (measured slower)
                for (int f = e + 1; f < M; ++f) {
                    v[4] = f;
                    visit(v);
                }
                flush(v);
            }
    }
}

}  // namespace

bool kgen_supported(int k, int c) { return (k == 4 || k == 5) && (c == 3 || c == 4); }

// pairs (a, b), a < b, with at least k - 2 variables above b
void build_kgen_items(int M, int k, std::vector<int2>& items) {
    items.clear();
    for (int a = 0; a < M; ++a)
        for (int b = a + 1; b + (k - 2) < M; ++b) items.push_back(make_int2(a, b));
}

cudaError_t launch_kgen(const uint32_t* planes, PlaneGeom g, int M, int c, int k, int d0, int nd, const int2* items,
                        int n_items, const long long* tab, unsigned long long* keys, EmitTable emit,
                        cudaStream_t st) {
    if (n_items == 0 || nd == 0) return cudaSuccess;
    if (!kgen_supported(k, c) || nd > 65535 || g.N > 65535) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)n_items, (unsigned)nd), block(32 * kWarps);
    if (k == 4 && c == 3) kgen_kernel<4, 3><<<grid, block, 0, st>>>(planes, g, M, d0, items, tab, keys, emit);
    else if (k == 4) kgen_kernel<4, 4><<<grid, block, 0, st>>>(planes, g, M, d0, items, tab, keys, emit);
    else if (c == 3) kgen_kernel<5, 3><<<grid, block, 0, st>>>(planes, g, M, d0, items, tab, keys, emit);
    else kgen_kernel<5, 4><<<grid, block, 0, st>>>(planes, g, M, d0, items, tab, keys, emit);
    return cudaGetLastError();
}

}  // namespace mdfs
