// Input staging kernels of the MDFS scan: decision statistics and class-sorted
// sample order, the fixed-point entropy tables (Eqs. H, p, beta) and the
// randomised rank-based discretiser (section "Algorithm and implementation").
#include <math.h>

#include <algorithm>

#include "mdfs_device.cuh"
#include "mdfs_internal.cuh"

namespace mdfs {

// ---------------------------------------------------------------------------
// Decision statistics and the class-stable sample permutation (one CTA).
// perm[0 .. N0) = indices with y == 0 in ascending order, perm[N0 .. N) = the
// indices with y == 1 in ascending order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) stats_kernel(const uint8_t* __restrict__ y, int N,
                                                     int* __restrict__ stats, int* __restrict__ perm) {
    __shared__ int warp_sum[32];
    __shared__ int warp_bad[32];
    __shared__ int s_n1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

    // pass 1: count ones and invalid labels
    int ones = 0, bad = 0;
    for (int s = tid; s < N; s += blockDim.x) {
        const int v = y[s];
        ones += (v == 1);
        bad += (v > 1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        ones += __shfl_xor_sync(0xffffffffu, ones, o);
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if (lane == 0) {
        warp_sum[warp] = ones;
        warp_bad[warp] = bad;
    }
    __syncthreads();
    if (tid == 0) {
        int t1 = 0, tb = 0;
        for (int w = 0; w < nwarps; ++w) {
            t1 += warp_sum[w];
            tb += warp_bad[w];
        }
        s_n1 = t1;
        stats[0] = t1;
        stats[1] = tb;
    }
    __syncthreads();
    const int n0 = N - s_n1;

    // pass 2: stable scatter, one block-wide exclusive scan per chunk
    int base0 = 0, base1 = n0;
    for (int chunk = 0; chunk < N; chunk += blockDim.x) {
        const int s = chunk + tid;
        const int is1 = (s < N) ? (y[s] == 1) : 0;
        const int is0 = (s < N) ? (1 - is1) : 0;
        const unsigned b1 = __ballot_sync(0xffffffffu, is1);
        const unsigned b0 = __ballot_sync(0xffffffffu, is0);
        const unsigned lt = (1u << lane) - 1u;
        const int pre1 = __popc(b1 & lt), pre0 = __popc(b0 & lt);
        __syncthreads();
        if (lane == 0) {
            warp_sum[warp] = __popc(b0);
            warp_bad[warp] = __popc(b1);
        }
        __syncthreads();
        int off0 = 0, off1 = 0, tot0 = 0, tot1 = 0;
        for (int w = 0; w < nwarps; ++w) {
            const int c0 = warp_sum[w], c1 = warp_bad[w];
            if (w < warp) {
                off0 += c0;
                off1 += c1;
            }
            tot0 += c0;
            tot1 += c1;
        }
        if (is0) perm[base0 + off0 + pre0] = s;
        if (is1) perm[base1 + off1 + pre1] = s;
        base0 += tot0;
        base1 += tot1;
    }
}

cudaError_t launch_stats(const uint8_t* y, int N, int* stats, int* perm, cudaStream_t st) {
    stats_kernel<<<1, 1024, 0, st>>>(y, N, stats, perm);
    return cudaGetLastError();
}

__global__ void check_finite_kernel(const float* __restrict__ x, long long count, int* __restrict__ flag) {
    int bad = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        bad |= !isfinite(x[i]);
    bad = __any_sync(0xffffffffu, bad);
    if (bad && (threadIdx.x & 31) == 0) atomicAdd(flag, 1);
}

cudaError_t launch_check_finite(const float* x, long long count, int* flag, cudaStream_t st) {
    long long blocks = (count + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    check_finite_kernel<<<(int)blocks, 256, 0, st>>>(x, count, flag);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// One job of a batch: x_j[v][t] = x[v][idx[t]], y_j[t] = y[yperm[idx[t]]]
// (idx / yperm NULL = identity).  Indices outside [0, N) count in *flag and
// read sample 0 instead.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void gather_job_kernel(const T* __restrict__ x, const uint8_t* __restrict__ y, int N, int M,
                                  const int* __restrict__ idx, const int* __restrict__ yperm, T* __restrict__ xo,
                                  uint8_t* __restrict__ yo, int* __restrict__ flag) {
    const long long total = (long long)M * N;
    const long long stride = (long long)gridDim.x * blockDim.x;
    int bad = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int v = (int)(i / N), t = (int)(i - (long long)v * N);
        int s = idx ? idx[t] : t;
        if (s < 0 || s >= N) {
            bad = 1;
            s = 0;
        }
        xo[i] = x[(size_t)v * N + s];
    }
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < N; t += stride) {
        int s = idx ? idx[t] : (int)t;
        if (s < 0 || s >= N) {
            bad = 1;
            s = 0;
        }
        int s2 = yperm ? yperm[s] : s;
        if (s2 < 0 || s2 >= N) {
            bad = 1;
            s2 = 0;
        }
        yo[t] = y[s2];
    }
    if (bad) atomicAdd(flag, 1);
}

cudaError_t launch_gather_job(const void* x, int dtype, const uint8_t* y, int N, int M, const int* idx,
                              const int* yperm, void* xo, uint8_t* yo, int* flag, cudaStream_t st) {
    long long blocks = ((long long)M * N + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    if (dtype == 0)
        gather_job_kernel<float><<<(int)blocks, 256, 0, st>>>((const float*)x, y, N, M, idx, yperm, (float*)xo, yo,
                                                              flag);
    else
        gather_job_kernel<int8_t><<<(int)blocks, 256, 0, st>>>((const int8_t*)x, y, N, M, idx, yperm, (int8_t*)xo,
                                                               yo, flag);
    return cudaGetLastError();
}

// Class sizes of every job of a batch in one pass: one CTA per job sums
// y_j[t] = y[yperm_j[idx_j[t]]] over t (NULL maps = identity) and counts the
// indices outside [0, N): out[j] = (n1, bad).
__global__ void __launch_bounds__(256) batch_counts_kernel(const uint8_t* __restrict__ y, int N,
                                                           const int* __restrict__ idx, const int* __restrict__ yperm,
                                                           int2* __restrict__ out) {
    const int j = blockIdx.x;
    const int* ij = idx ? idx + (size_t)j * N : nullptr;
    const int* pj = yperm ? yperm + (size_t)j * N : nullptr;
    int n1 = 0, bad = 0;
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        int s = ij ? ij[t] : t;
        if (s < 0 || s >= N) {
            bad = 1;
            s = 0;
        }
        int s2 = pj ? pj[s] : s;
        if (s2 < 0 || s2 >= N) {
            bad = 1;
            s2 = 0;
        }
        n1 += y[s2] != 0;
        bad |= y[s2] > 1;
    }
    __shared__ int red[2][8];
    for (int o = 16; o > 0; o >>= 1) {
        n1 += __shfl_xor_sync(0xffffffffu, n1, o);
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = n1;
        red[1][threadIdx.x >> 5] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0, b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += red[0][w];
            b |= red[1][w];
        }
        out[j] = make_int2(a, b);
    }
}

cudaError_t launch_batch_counts(const uint8_t* y, int N, const int* idx, const int* yperm, int n_jobs, int2* out,
                                cudaStream_t st) {
    if (n_jobs < 1) return cudaSuccess;
    batch_counts_kernel<<<n_jobs, 256, 0, st>>>(y, N, idx, yperm, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Entropy tables (Eqs. H, p, beta).  f(t) = t ln t in FP64, stored as int64
// multiples of 2^-32 (round to nearest).
// ---------------------------------------------------------------------------
__global__ void ftable_kernel(int N, double b0, double b1, long long* __restrict__ tab) {
    const int np1 = N + 1;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * np1) return;
    const int which = i / np1, n = i - which * np1;
    const double beta = which == 0 ? b0 : (which == 1 ? b1 : b0 + b1);
    const double t = (double)n + beta;
    const double f = t > 0.0 ? t * log(t) : 0.0;
    tab[i] = __double2ll_rn(f * kFxScale);
}

cudaError_t launch_ftable(int N, double b0, double b1, long long* tab, cudaStream_t st) {
    const int total = 3 * (N + 1);
    ftable_kernel<<<(total + 255) / 256, 256, 0, st>>>(N, b0, b1, tab);
    return cudaGetLastError();
}

// The same f(n + beta) values in the fixed layout of the packed-count kernels:
// n + b0 at [0, 2^16), n + b1 at [2^16, 2^17), n + b0 + b1 at [2^17, 2^18).
__global__ void ftable_wide_kernel(double b0, double b1, long long* __restrict__ tab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (1 << 18)) return;
    const int which = i < (1 << 16) ? 0 : (i < (1 << 17) ? 1 : 2);
    const int n = which == 2 ? i - (1 << 17) : (which == 1 ? i - (1 << 16) : i);
    const double beta = which == 0 ? b0 : (which == 1 ? b1 : b0 + b1);
    const double t = (double)n + beta;
    const double f = t > 0.0 ? t * log(t) : 0.0;
    tab[i] = __double2ll_rn(f * kFxScale);
}

cudaError_t launch_ftable_wide(double b0, double b1, long long* tab, cudaStream_t st) {
    ftable_wide_kernel<<<(1 << 18) / 256, 256, 0, st>>>(b0, b1, tab);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Discretiser: one CTA per variable.
//   1. bitonic sort of the column in shared memory (padded with +inf),
//   2. per discretisation: c Philox shares -> c-1 cut positions -> thresholds,
//   3. codes (original sample order), and bit planes of bins 1..c-1 in the
//      class-sorted sample order: with the E4M3 one-hot rows, one pass per 32
//      class-sorted samples writes both (the plane word from the same
//      compares); alone, one ballot per 32 samples.
// Share j of (v, d): w_j = W - R + floor(u_j * 2R / 2^32), W = 2^20,
// R = round(range * 2^20), u_j = word j%4 of Philox(counter (j/4, v, d, tag),
// key = seed).  Positions p_j = floor(N S_j / S_c) with S_j = w_0 + .. + w_{j-1},
// clamped to [j, N-c+j] and made strictly increasing.
// ---------------------------------------------------------------------------
// Cut positions pos[1 .. c-1] of (variable v, discretisation d) among N sorted
// samples, from the shares above.
__device__ __forceinline__ void cut_positions(int v, int d, int N, int c, uint32_t R, uint32_t key0, uint32_t key1,
                                              int* pos) {
    const long long W = 1LL << 20;
    long long share[kMaxC];
    uint32_t u[4];
    for (int j = 0; j < c; ++j) {
        if ((j & 3) == 0) philox4x32_10((uint32_t)(j >> 2), (uint32_t)v, (uint32_t)d, kPhiloxTag, key0, key1, u);
        const unsigned long long draw = ((unsigned long long)u[j & 3] * (unsigned long long)(2u * R)) >> 32;
        share[j] = W - (long long)R + (long long)draw;
    }
    long long total = 0;
    for (int j = 0; j < c; ++j) total += share[j];
    long long cum = 0, prev = 0;
    for (int j = 1; j < c; ++j) {
        cum += share[j - 1];
        long long p = total > 0 ? (long long)(((unsigned long long)N * (unsigned long long)cum) / (unsigned long long)total)
                                : ((long long)N * j) / c;
        if (p < j) p = j;
        if (p > N - c + j) p = N - c + j;
        if (j > 1 && p <= prev) p = prev + 1;
        prev = p;
        pos[j] = (int)p;
    }
}

// Ascending bitonic sort of s[0 .. npad) (npad a power of two) by the whole block,
// every stage through shared memory.
__device__ void bitonic_sort_smem(float* s, int npad, int tid, int nthreads) {
    for (int k = 2; k <= npad; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < npad; i += nthreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const float a = s[i], b = s[ixj];
                    const bool ascending = (i & k) == 0;
                    if ((a > b) == ascending) {
                        s[i] = b;
                        s[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// The same network with 512 threads holding E = npad / 512 consecutive elements
// each (indices E t + r): compare-exchange distances j < E stay in registers,
// E <= j < 32 E pair lanes of one warp (shuffles), and only j >= 32 E goes
// through shared memory with block barriers.  Leaves the sorted values in s.
template <int E>
__device__ void bitonic_sort_regs(float* s, int npad, int tid) {
    float v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) v[r] = s[E * tid + r];
    for (int k = 2; k <= npad; k <<= 1) {
        int j = k >> 1;
        if (j >= 32 * E) {  // long distances: shared memory
            __syncthreads();
#pragma unroll
            for (int r = 0; r < E; ++r) s[E * tid + r] = v[r];
            __syncthreads();
            for (; j >= 32 * E; j >>= 1) {
                for (int i = tid; i < npad; i += 512) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const float a = s[i], b = s[ixj];
                        if ((a > b) == ((i & k) == 0)) {
                            s[i] = b;
                            s[ixj] = a;
                        }
                    }
                }
                __syncthreads();
            }
#pragma unroll
            for (int r = 0; r < E; ++r) v[r] = s[E * tid + r];
        }
        for (; j >= E; j >>= 1) {  // partner in lane tid ^ (j / E), same r
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int i = E * tid + r;
                const float p = __shfl_xor_sync(0xffffffffu, v[r], j / E);
                const bool lower = (i & j) == 0, asc = (i & k) == 0;
                v[r] = (lower == asc) ? fminf(v[r], p) : fmaxf(v[r], p);
            }
        }
        // partner r ^ jj in this thread; jj runs over the compile-time distances
        // below E that this k uses (jj <= j), so v stays in registers
#pragma unroll
        for (int jj = E / 2; jj > 0; jj >>= 1) {
            if (jj > j) continue;
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int rp = r ^ jj;
                if (rp > r) {
                    const bool asc = ((E * tid + r) & k) == 0;
                    const float a = v[r], b = v[rp];
                    v[r] = asc ? fminf(a, b) : fmaxf(a, b);
                    v[rp] = asc ? fmaxf(a, b) : fminf(a, b);
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < E; ++r) s[E * tid + r] = v[r];
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(512) discretize_kernel(const T* __restrict__ x, int N, int M, int c, int D,
                                                         uint32_t R, uint32_t key0, uint32_t key1, int npad,
                                                         const int* __restrict__ perm, PlaneGeom g,
                                                         uint32_t* __restrict__ planes, uint8_t* __restrict__ codes,
                                                         float* __restrict__ thr_out, uint8_t* __restrict__ onehot,
                                                         TcGeom tg, int scol, uint32_t class1_byte,
                                                         const float* __restrict__ thr_in) {
    extern __shared__ __align__(16) float smem[];
    float* s = smem;           // [scol]: sorted column, then the class-sorted one-hot staging
    float* thr = smem + scol;  // [D][c-1] thresholds
    const int v = blockIdx.x;
    const int tid = threadIdx.x;
    const T* xv = x + (size_t)v * N;
    const int cm1 = c - 1;

    if (thr_in) {  // thresholds given: no sort
        for (int i = tid; i < D * cm1; i += blockDim.x) {
            const float t = thr_in[((size_t)(i / cm1) * M + v) * cm1 + i % cm1];
            thr[i] = t;
            if (thr_out) thr_out[((size_t)(i / cm1) * M + v) * cm1 + i % cm1] = t;
        }
        __syncthreads();
    } else {
        for (int i = tid; i < npad; i += blockDim.x) s[i] = (i < N) ? (float)xv[i] : INFINITY;
        __syncthreads();
        switch (blockDim.x == 512 ? npad : 0) {
            case 1024: bitonic_sort_regs<2>(s, npad, tid); break;
            case 2048: bitonic_sort_regs<4>(s, npad, tid); break;
            case 4096: bitonic_sort_regs<8>(s, npad, tid); break;
            case 8192: bitonic_sort_regs<16>(s, npad, tid); break;
            default: bitonic_sort_smem(s, npad, tid, blockDim.x); break;
        }
        for (int d = tid; d < D; d += blockDim.x) {
            int pos[kMaxC];
            cut_positions(v, d, N, c, R, key0, key1, pos);
            for (int j = 1; j < c; ++j) {
                const float t = s[pos[j]];
                thr[d * cm1 + (j - 1)] = t;
                if (thr_out) thr_out[((size_t)d * M + v) * cm1 + (j - 1)] = t;
            }
        }
        __syncthreads();
    }

    if (codes) {
        for (int i = tid; i < N; i += blockDim.x) {
            const float xs = (float)xv[i];
            for (int d = 0; d < D; ++d) {
                int code = 0;
                for (int j = 0; j < cm1; ++j) code += (xs >= thr[d * cm1 + j]);
                codes[((size_t)d * M + v) * N + i] = (uint8_t)code;
            }
        }
    }

    if (onehot) {
        // the sorted column is no longer needed: stage x in the class-sorted
        // one-hot order (NaN in the padding, which compares false)
        __syncthreads();
        for (int pos = tid; pos < tg.Kp; pos += blockDim.x) {
            int sidx = -1;
            if (pos < tg.K0p) {
                if (pos < g.N0) sidx = perm[pos];
            } else if (pos - tg.K0p < g.N1) {
                sidx = perm[g.N0 + pos - tg.K0p];
            }
            s[pos] = sidx >= 0 ? (float)xv[sidx] : __int_as_float(0x7fc00000);
        }
        __syncthreads();
        {
            // one pass for both outputs: per (32 positions, discretisation, bin)
            // two 16-byte one-hot stores and the bit-plane word of the same 32
            // class-sorted samples (class 0 at word g, class 1 from word W0)
            const int ngroup = tg.Kp >> 5;
            for (int w = tid; w < ngroup * D; w += blockDim.x) {
                const int gi = w % ngroup, d = w / ngroup;
                const int pos0 = gi * 32;
                const uint32_t one = pos0 < tg.K0p ? 0x38u : class1_byte;  // a group lies in one class range
                int pw = -1;  // plane word of this group, if any
                if (pos0 < tg.K0p) {
                    if (gi < g.W0) pw = gi;
                } else if (((pos0 - tg.K0p) >> 5) < g.W1) {
                    pw = g.W0 + ((pos0 - tg.K0p) >> 5);
                }
                float xs[32];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 f = reinterpret_cast<const float4*>(s)[gi * 8 + q];
                    xs[4 * q] = f.x;
                    xs[4 * q + 1] = f.y;
                    xs[4 * q + 2] = f.z;
                    xs[4 * q + 3] = f.w;
                }
                for (int a = 1; a <= cm1; ++a) {
                    const float lo = thr[d * cm1 + a - 1];
                    const float hi = a < cm1 ? thr[d * cm1 + a] : INFINITY;
                    uint32_t wd[8], bits = 0u;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        uint32_t b = 0;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const float xv_ = xs[4 * q + k];
                            // code == a  <=>  x >= thr[a-1] and not x >= thr[a] (thresholds ascending)
                            const bool in = xv_ >= lo && !(xv_ >= hi);
                            b |= in ? one << (8 * k) : 0u;
                            bits |= in ? 1u << (4 * q + k) : 0u;
                        }
                        wd[q] = b;
                    }
                    uint4* row = reinterpret_cast<uint4*>(onehot + (((size_t)d * M + v) * cm1 + (a - 1)) * tg.Kp);
                    row[2 * gi] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
                    row[2 * gi + 1] = make_uint4(wd[4], wd[5], wd[6], wd[7]);
                    if (planes && pw >= 0) planes[(((size_t)d * M + v) * cm1 + (a - 1)) * g.Ws + pw] = bits;
                }
            }
            // the padding words [W, Ws) of every plane
            const int npad = planes ? g.Ws - g.W : 0;
            for (int w = tid; w < npad * D * cm1; w += blockDim.x) {
                const int pwd = w % npad, row = w / npad;  // row = d * cm1 + (a - 1)
                const int d = row / cm1, a1 = row % cm1;
                planes[(((size_t)d * M + v) * cm1 + a1) * g.Ws + g.W + pwd] = 0u;
            }
        }
    }

    if (planes && !onehot) {  // planes alone: one ballot per (32 samples, discretisation, bin)
        const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
        for (int w = warp; w < g.Ws; w += nwarps) {
            int sidx = -1;
            if (w < g.W0) {
                const int q = w * 32 + lane;
                if (q < g.N0) sidx = perm[q];
            } else if (w < g.W) {
                const int q = (w - g.W0) * 32 + lane;
                if (q < g.N1) sidx = perm[g.N0 + q];
            }
            const float xs = sidx >= 0 ? (float)xv[sidx] : 0.0f;
            for (int d = 0; d < D; ++d) {
                int code = 0;
                for (int j = 0; j < cm1; ++j) code += (xs >= thr[d * cm1 + j]);
                for (int a = 1; a <= cm1; ++a) {
                    const unsigned m = __ballot_sync(0xffffffffu, sidx >= 0 && code == a);
                    if (lane == 0) planes[(((size_t)d * M + v) * cm1 + (a - 1)) * g.Ws + w] = m;
                }
            }
        }
    }
}

cudaError_t launch_discretize(const void* x, int dtype, int N, int M, int c, int D, double range,
                              uint64_t seed, const int* perm, PlaneGeom g, uint32_t* planes,
                              uint8_t* codes, float* thr, uint8_t* onehot, TcGeom tg, cudaStream_t st,
                              uint32_t class1_byte, const float* thr_in) {
    int npad = 1;
    while (npad < N) npad <<= 1;
    // sorted column, reused for the class-sorted one-hot staging (Kp may exceed npad)
    const size_t scol = (size_t)std::max(npad, tg.Kp);
    const size_t smem = sizeof(float) * (scol + (size_t)D * (c - 1));
    const uint32_t R = (uint32_t)floor(range * 1048576.0 + 0.5);
    const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFull), k1 = (uint32_t)(seed >> 32);
    cudaError_t e;
    if (dtype == 0) {
        e = ensure_dynamic_smem((const void*)discretize_kernel<float>, smem);
        if (e != cudaSuccess) return e;
        discretize_kernel<float><<<M, 512, smem, st>>>((const float*)x, N, M, c, D, R, k0, k1, npad, perm, g,
                                                       planes, codes, thr, onehot, tg, (int)scol, class1_byte,
                                                       thr_in);
    } else {
        e = ensure_dynamic_smem((const void*)discretize_kernel<int8_t>, smem);
        if (e != cudaSuccess) return e;
        discretize_kernel<int8_t><<<M, 512, smem, st>>>((const int8_t*)x, N, M, c, D, R, k0, k1, npad, perm, g,
                                                        planes, codes, thr, onehot, tg, (int)scol, class1_byte,
                                                       thr_in);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched resamples: one sort per variable for all jobs.  Job j's column is
// x[v][idx_j[t]], t = 0..N-1, whose sorted order is the original sorted order
// with sample s repeated m_j[s] times (m_j = how often s occurs in idx_j), so
// its cut thresholds (the values at the cut positions of the sorted column)
// follow from the original sorted keys (float_order_bits of the value << 32 |
// the sample index) and a prefix sum of m_j.
// ---------------------------------------------------------------------------
// ascending bitonic sort of 64-bit keys s[0 .. npad) by the whole block
__device__ void bitonic_sort_u64(unsigned long long* s, int npad, int tid, int nthreads) {
    for (int k = 2; k <= npad; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < npad; i += nthreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long a = s[i], b = s[ixj];
                    if ((a > b) == ((i & k) == 0)) {
                        s[i] = b;
                        s[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(512) presort_kernel(const T* __restrict__ x, int N, int npad,
                                                      unsigned long long* __restrict__ keys) {
    extern __shared__ unsigned long long sk[];
    const int v = blockIdx.x, tid = threadIdx.x;
    const T* xv = x + (size_t)v * N;
    for (int i = tid; i < npad; i += blockDim.x)
        sk[i] = i < N ? ((unsigned long long)float_order_bits((float)xv[i]) << 32) | (uint32_t)i : ~0ull;
    __syncthreads();
    bitonic_sort_u64(sk, npad, tid, blockDim.x);
    for (int i = tid; i < N; i += blockDim.x) keys[(size_t)v * N + i] = sk[i];
}

cudaError_t launch_presort(const void* x, int dtype, int N, int M, unsigned long long* keys, cudaStream_t st) {
    if (N < 1 || N > kPresortMaxN) return cudaErrorInvalidValue;
    int npad = 2;
    while (npad < N) npad <<= 1;
    const size_t smem = (size_t)npad * sizeof(unsigned long long);
    cudaError_t e;
    if (dtype == 0) {
        if ((e = ensure_dynamic_smem((const void*)presort_kernel<float>, smem)) != cudaSuccess) return e;
        presort_kernel<float><<<M, 512, smem, st>>>((const float*)x, N, npad, keys);
    } else {
        if ((e = ensure_dynamic_smem((const void*)presort_kernel<int8_t>, smem)) != cudaSuccess) return e;
        presort_kernel<int8_t><<<M, 512, smem, st>>>((const int8_t*)x, N, npad, keys);
    }
    return cudaGetLastError();
}

__global__ void multiplicity_kernel(const int* __restrict__ idx, int N, int* __restrict__ m) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N; t += gridDim.x * blockDim.x) atomicAdd(m + idx[t], 1);
}

cudaError_t launch_multiplicity(const int* idx, int N, int* m, cudaStream_t st) {
    if (!idx) return cudaSuccess;  // identity: every sample once (the thresholds kernel takes m = NULL)
    cudaError_t e = cudaMemsetAsync(m, 0, (size_t)N * sizeof(int), st);
    if (e != cudaSuccess) return e;
    multiplicity_kernel<<<(N + 255) / 256, 256, 0, st>>>(idx, N, m);
    return cudaGetLastError();
}

// One CTA per variable: inclusive prefix C[r] of the multiplicities along the
// sorted order; the sample at cut position p of the resampled column is the
// first r with C[r] > p.
__global__ void __launch_bounds__(512) batch_thresholds_kernel(const unsigned long long* __restrict__ keys,
                                                               const int* __restrict__ m, int N, int M, int c, int D,
                                                               uint32_t R, uint32_t key0, uint32_t key1,
                                                               float* __restrict__ thr) {
    extern __shared__ int C[];  // [N]
    __shared__ int warp_sum[16];
    const int v = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long* kv = keys + (size_t)v * N;
    const int per = (N + blockDim.x - 1) / blockDim.x;
    const int lo = min(N, tid * per), hi = min(N, lo + per);
    int run = 0;
    for (int r = lo; r < hi; ++r) {
        run += m ? m[(uint32_t)kv[r]] : 1;
        C[r] = run;
    }
    // exclusive block scan of the threads' totals
    int incl = run;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += warp_sum[w];
    const int offset = before + incl - run;
    for (int r = lo; r < hi; ++r) C[r] += offset;
    __syncthreads();
    const int cm1 = c - 1;
    for (int d = tid; d < D; d += blockDim.x) {
        int pos[kMaxC];
        cut_positions(v, d, N, c, R, key0, key1, pos);
        for (int j = 1; j < c; ++j) {
            const int p = pos[j];
            int a = 0, b = N - 1;  // C[N - 1] = N > p
            while (a < b) {
                const int mid = (a + b) >> 1;
                if (C[mid] > p) b = mid;
                else a = mid + 1;
            }
            thr[((size_t)d * M + v) * cm1 + (j - 1)] = order_bits_float((uint32_t)(kv[a] >> 32));
        }
    }
}

cudaError_t launch_batch_thresholds(const unsigned long long* keys, const int* m, int N, int M, int c, int D,
                                    double range, uint64_t seed, float* thr, cudaStream_t st) {
    if (N < 1 || N > kPresortMaxN) return cudaErrorInvalidValue;
    const uint32_t R = (uint32_t)floor(range * 1048576.0 + 0.5);
    const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFull), k1 = (uint32_t)(seed >> 32);
    const size_t smem = (size_t)N * sizeof(int);
    cudaError_t e = ensure_dynamic_smem((const void*)batch_thresholds_kernel, smem);
    if (e != cudaSuccess) return e;
    batch_thresholds_kernel<<<M, 512, smem, st>>>(keys, m, N, M, c, D, R, k0, k1, thr);
    return cudaGetLastError();
}

}  // namespace mdfs
