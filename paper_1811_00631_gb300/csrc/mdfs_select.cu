// Contrast variables and multiple-testing adjustment for the canonical
// selection pipeline (section "Canonical package usage" of arXiv 1811.00631):
// contrast variables are copies of original variables with their samples
// shuffled; IG^k_max runs on the extended set, the chi^2 / extreme-value fit
// uses the contrast variables only, and the p-values of the original
// variables are adjusted for multiple testing.
//
// The shuffle is a counter-based pseudo-random permutation, so every element
// of a contrast row is produced independently by one thread: a 10-round
// Luby-Rackoff (Feistel) network on 2h-bit words whose round function is word
// 0 of Philox4x32-10 (counter (R, round, stream, 'CTRS'), key = seed), made a
// permutation of [0, n) by cycle walking (Black and Rogaway, CT-RSA 2002).
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/mdfs.h"
#include "mdfs_device.cuh"
#include "mdfs_internal.cuh"

namespace mdfs {

namespace {

constexpr uint32_t kContrastTag = 0x43545253u;  // 'CTRS', fourth counter word
constexpr uint32_t kSourceStream = 0xFFFFFFFFu; // stream of the source-variable permutation

// One pass of the 10-round Feistel network on a 2h-bit word.
__device__ __forceinline__ uint32_t feistel_pass(uint32_t v, int h, uint32_t stream, uint32_t k0, uint32_t k1) {
    const uint32_t mask = (1u << h) - 1u;
    uint32_t L = v >> h, R = v & mask;
#pragma unroll 1
    for (uint32_t r = 0; r < 10; ++r) {
        uint32_t u[4];
        philox4x32_10(R, r, stream, kContrastTag, k0, k1, u);
        const uint32_t t = (L ^ u[0]) & mask;
        L = R;
        R = t;
    }
    return (L << h) | R;
}

// Image of i < n under the permutation (h: half-width with 2^(2h) >= n).  The
// orbit of i under the network returns to i within 2^(2h) passes, which bounds
// the walk.
__device__ __forceinline__ uint32_t shuffle_index(uint32_t i, uint32_t n, int h, uint32_t stream, uint32_t k0,
                                                  uint32_t k1) {
    if (n <= 1) return 0;
    const uint32_t limit = 1u << (2 * h);
    uint32_t v = i;
    for (uint32_t it = 0; it < limit; ++it) {
        v = feistel_pass(v, h, stream, k0, k1);
        if (v < n) return v;
    }
    return i;  // not reached
}

// Row M + j of x_ext = variable src[j] with sample i taken from sample
// shuffle_N(i) (stream j); src[j] = shuffle_M(j mod M) (source stream).
template <typename T>
__global__ void __launch_bounds__(256) contrast_kernel(const T* __restrict__ x, int N, int M, int hN, int hM,
                                                       uint32_t k0, uint32_t k1, T* __restrict__ x_ext,
                                                       int* __restrict__ src) {
    __shared__ uint32_t s_src;
    const int j = blockIdx.y;
    if (threadIdx.x == 0) {
        s_src = shuffle_index((uint32_t)(j % M), (uint32_t)M, hM, kSourceStream, k0, k1);
        if (blockIdx.x == 0 && src) src[j] = (int)s_src;
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        const uint32_t from = shuffle_index((uint32_t)i, (uint32_t)N, hN, (uint32_t)j, k0, k1);
        x_ext[((size_t)M + j) * N + i] = x[(size_t)s_src * N + from];
    }
}

// h = ceil(ceil(log2 n) / 2), at least 1
int half_width(int n) {
    int b = 0;
    while ((1ll << b) < (long long)n) ++b;
    const int h = (b + 1) / 2;
    return h < 1 ? 1 : h;
}

// ---------------------------------------------------------------------------
// p-value adjustment, one CTA.  (p, index) pairs are sorted ascending (ties by
// index) with a bitonic network in global scratch; then, in sorted order
// (0-based rank r, m non-NaN values):
//   Bonferroni  min(1, m p)
//   Holm        min(1, max_{s <= r} (m - s) p_(s))         (step-down)
//   Hochberg    min(1, min_{s >= r} (m - s) p_(s))         (step-up)
//   BH          min(1, min_{s >= r} m / (s + 1) p_(s))
//   BY          BH times sum_{s=1..m} 1/s
// NaN p-values sort last, are not counted in m and stay NaN.
// ---------------------------------------------------------------------------
constexpr int kAdjThreads = 1024;

__device__ __forceinline__ bool pair_greater(double a, int ia, double b, int ib) {
    return a > b || (a == b && ia > ib);
}

__global__ void __launch_bounds__(kAdjThreads) p_adjust_kernel(const double* __restrict__ p, int m_in, int mpad,
                                                               int method, double level, double* __restrict__ key,
                                                               int* __restrict__ idx, double* __restrict__ scan,
                                                               double* __restrict__ adjusted,
                                                               uint8_t* __restrict__ relevant) {
    __shared__ double s_agg[kAdjThreads];
    __shared__ int s_cnt[kAdjThreads];
    const int tid = threadIdx.x;
    int cnt = 0;
    for (int i = tid; i < mpad; i += kAdjThreads) {
        const double v = i < m_in ? p[i] : NAN;
        const bool nan = !(v == v);
        key[i] = nan ? INFINITY : v;
        idx[i] = i;
        cnt += (i < m_in && !nan);
    }
    s_cnt[tid] = cnt;
    __syncthreads();
    for (int k = 2; k <= mpad; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < mpad; i += kAdjThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const double a = key[i], b = key[ixj];
                    const int ia = idx[i], ib = idx[ixj];
                    if (pair_greater(a, ia, b, ib) == ((i & k) == 0)) {
                        key[i] = b;
                        key[ixj] = a;
                        idx[i] = ib;
                        idx[ixj] = ia;
                    }
                }
            }
            __syncthreads();
        }
    // m = number of non-NaN values (they occupy ranks 0..m-1 after the sort)
    for (int s = kAdjThreads / 2; s > 0; s >>= 1) {
        if (tid < s) s_cnt[tid] += s_cnt[tid + s];
        __syncthreads();
    }
    const int m = s_cnt[0];
    const double md = (double)m;
    double q = 1.0;
    if (method == MDFS_ADJUST_BY) {  // harmonic number, summed in a fixed order
        double h = 0.0;
        for (int s = tid + 1; s <= m; s += kAdjThreads) h += 1.0 / (double)s;
        s_agg[tid] = h;
        __syncthreads();
        for (int s = kAdjThreads / 2; s > 0; s >>= 1) {
            if (tid < s) s_agg[tid] += s_agg[tid + s];
            __syncthreads();
        }
        q = s_agg[0];
        __syncthreads();
    }
    // value before the running max / min, at rank r
    auto term = [&](int r) -> double {
        const double v = key[r];
        switch (method) {
            case MDFS_ADJUST_BONFERRONI: return md * v;
            case MDFS_ADJUST_HOLM:
            case MDFS_ADJUST_HOCHBERG: return (md - (double)r) * v;
            case MDFS_ADJUST_BH: return md / (double)(r + 1) * v;
            case MDFS_ADJUST_BY: return q * md / (double)(r + 1) * v;
            default: return v;
        }
    };
    const bool step_down = method == MDFS_ADJUST_HOLM;                       // running max from rank 0
    const bool step_up = method == MDFS_ADJUST_HOCHBERG || method == MDFS_ADJUST_BH || method == MDFS_ADJUST_BY;
    const int cs = (m + kAdjThreads - 1) / kAdjThreads;
    const int lo = min(m, tid * cs), hi = min(m, lo + cs);
    if (step_down) {
        double run = -INFINITY;
        for (int r = lo; r < hi; ++r) scan[r] = run = fmax(run, term(r));
        s_agg[tid] = run;
    } else if (step_up) {
        double run = INFINITY;
        for (int r = hi - 1; r >= lo; --r) scan[r] = run = fmin(run, term(r));
        s_agg[tid] = run;
    } else {
        for (int r = lo; r < hi; ++r) scan[r] = term(r);
    }
    __syncthreads();
    if (step_down || step_up) {
        // exclusive running max over lower chunks / min over higher chunks (Hillis-Steele)
        for (int off = 1; off < kAdjThreads; off <<= 1) {
            double other = step_down ? -INFINITY : INFINITY;
            if (step_down && tid >= off) other = s_agg[tid - off];
            if (step_up && tid + off < kAdjThreads) other = s_agg[tid + off];
            __syncthreads();
            s_agg[tid] = step_down ? fmax(s_agg[tid], other) : fmin(s_agg[tid], other);
            __syncthreads();
        }
        double carry = step_down ? -INFINITY : INFINITY;
        if (step_down && tid > 0) carry = s_agg[tid - 1];
        if (step_up && tid + 1 < kAdjThreads) carry = s_agg[tid + 1];
        for (int r = lo; r < hi; ++r) scan[r] = step_down ? fmax(scan[r], carry) : fmin(scan[r], carry);
    }
    __syncthreads();
    for (int r = tid; r < mpad; r += kAdjThreads) {
        const int i = idx[r];
        if (i >= m_in) continue;
        const double a = r < m ? fmin(1.0, scan[r]) : NAN;
        adjusted[i] = a;
        if (relevant) relevant[i] = (uint8_t)(a < level);
    }
}

}  // namespace

cudaError_t launch_contrast(const void* x, int dtype, int N, int M, int n_contrast, uint64_t seed, void* x_ext,
                            int* src, cudaStream_t st) {
    if (n_contrast <= 0) return cudaSuccess;
    const int hN = half_width(N), hM = half_width(M);
    if (2 * hN > 31 || 2 * hM > 31) return cudaErrorInvalidValue;
    const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFull), k1 = (uint32_t)(seed >> 32);
    const dim3 grid((N + 255) / 256, n_contrast);
    if (dtype == 0)
        contrast_kernel<float><<<grid, 256, 0, st>>>((const float*)x, N, M, hN, hM, k0, k1, (float*)x_ext, src);
    else
        contrast_kernel<int8_t><<<grid, 256, 0, st>>>((const int8_t*)x, N, M, hN, hM, k0, k1, (int8_t*)x_ext, src);
    return cudaGetLastError();
}

size_t p_adjust_scratch_bytes(int m) {
    int mpad = 1;
    while (mpad < m) mpad <<= 1;
    return (size_t)mpad * (2 * sizeof(double) + sizeof(int));
}

cudaError_t launch_p_adjust(const double* p, int m, int method, double level, void* scratch, double* adjusted,
                            uint8_t* relevant, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    int mpad = 1;
    while (mpad < m) mpad <<= 1;
    double* key = (double*)scratch;
    double* scan = key + mpad;
    int* idx = (int*)(scan + mpad);
    p_adjust_kernel<<<1, kAdjThreads, 0, st>>>(p, m, mpad, method, level, key, idx, scan, adjusted, relevant);
    return cudaGetLastError();
}

}  // namespace mdfs
