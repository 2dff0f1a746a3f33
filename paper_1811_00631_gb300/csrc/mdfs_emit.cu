// Interesting tuples (section "Examples": every variable-tuple pair whose IG
// reaches a threshold): collection of the emission hash table that the scan
// kernels fill (EmitTable).  The occupied slots are gathered, sorted by
// (variable, partners) and decoded into caller arrays.
#include <cuda_runtime.h>

#include <algorithm>

#include "mdfs_device.cuh"
#include "mdfs_internal.cuh"

namespace mdfs {

namespace {

constexpr int kSortThreads = 1024;

// (v, p1, p2, p3) lexicographic order: the 16-bit fields with v most
// significant; k = 5: the five 12-bit fields (v, p1, .., p4) in that order.
__device__ __forceinline__ unsigned long long sort_key(unsigned long long key, int k) {
    if (k == 5)
        return ((key & 0xFFFull) << 48) | (((key >> 12) & 0xFFFull) << 36) | (((key >> 24) & 0xFFFull) << 24) |
               (((key >> 36) & 0xFFFull) << 12) | (key >> 48);
    return ((key & 0xFFFFull) << 48) | (((key >> 16) & 0xFFFFull) << 32) | (((key >> 32) & 0xFFFFull) << 16) |
           (key >> 48);
}

__global__ void emit_gather_kernel(EmitTable t, int k, unsigned long long* __restrict__ rk,
                                   unsigned long long* __restrict__ rv, int* __restrict__ counter, int n_max) {
    const unsigned int size = t.mask + 1u;
    for (unsigned int s = blockIdx.x * blockDim.x + threadIdx.x; s < size; s += gridDim.x * blockDim.x) {
        const unsigned long long key = t.keys[s];
        if (key == kEmptyEmitKey) continue;
        const int pos = atomicAdd(counter, 1);
        if (pos < n_max) {
            rk[pos] = sort_key(key, k);
            rv[pos] = t.vals[s];
        }
    }
}

// One CTA: bitonic sort of n (sort key, value) pairs padded to npad, then decode.
// Keys are distinct, so the order is fully determined.
__global__ void __launch_bounds__(kSortThreads) emit_sort_decode_kernel(unsigned long long* __restrict__ rk,
                                                                        unsigned long long* __restrict__ rv, int n,
                                                                        int npad, int k, int* __restrict__ var,
                                                                        int* __restrict__ tuples, float* __restrict__ ig,
                                                                        int* __restrict__ disc) {
    const int tid = threadIdx.x;
    for (int i = n + tid; i < npad; i += kSortThreads) {
        rk[i] = ~0ull;
        rv[i] = 0ull;
    }
    __syncthreads();
    for (int kk = 2; kk <= npad; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < npad; i += kSortThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long a = rk[i], b = rk[ixj];
                    if ((a > b) == ((i & kk) == 0)) {
                        rk[i] = b;
                        rk[ixj] = a;
                        const unsigned long long va = rv[i];
                        rv[i] = rv[ixj];
                        rv[ixj] = va;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = tid; i < n; i += kSortThreads) {
        const unsigned long long s = rk[i], v = rv[i];
        int p[4];
        if (k == 5) {
            var[i] = (int)(s >> 48);
            for (int j = 0; j < 4; ++j) p[j] = (int)((s >> (36 - 12 * j)) & 0xFFF);
        } else {
            var[i] = (int)(s >> 48);
            for (int j = 0; j < 3; ++j) p[j] = (int)((s >> (32 - 16 * j)) & 0xFFFF);
        }
        if (tuples)
            for (int j = 0; j < k - 1; ++j) tuples[(size_t)i * (k - 1) + j] = p[j];
        ig[i] = order_bits_float((uint32_t)(v >> 32));
        disc[i] = (int)(~(uint32_t)v);
    }
}

}  // namespace

cudaError_t launch_emit_collect(EmitTable t, int k, unsigned long long* recs_key, unsigned long long* recs_val,
                                int* counter, int npad, int* var, int* tuples, float* ig, int* disc, int n,
                                cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const unsigned int size = t.mask + 1u;
    const int blocks = (int)std::min<unsigned int>((size + 255u) / 256u, 4096u);
    emit_gather_kernel<<<blocks, 256, 0, st>>>(t, k, recs_key, recs_val, counter, npad);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    emit_sort_decode_kernel<<<1, kSortThreads, 0, st>>>(recs_key, recs_val, n, npad, k, var, tuples, ig, disc);
    return cudaGetLastError();
}

}  // namespace mdfs
