// Microbenchmarks of the two hardware rates that bound the scan kernels, for
// the roofline figures of the benchmark (not part of the method):
//   - dense E4M3 x E4M3 -> F32 tensor-core throughput: tcgen05.mma kind::f8f6f4
//     with M = 128, N = 256, K = 32 per instruction and both operands in shared
//     memory, the instruction shape of the k = 3 counting kernel;
//   - 4-byte shared-memory table loads at random indices, over the whole table
//     or within a window of consecutive entries around a warp-wide centre (the
//     access pattern of the entropy lookups).
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/mdfs_bench.h"
#include "mdfs_internal.cuh"
#include "mdfs_tc.cuh"

namespace {

constexpr int kMmaM = 128, kMmaN = 256, kMmaK = 32;
constexpr uint32_t kABytes = kMmaM * 128, kBBytes = kMmaN * 128;  // 128 K bytes per row (4 MMAs)
constexpr size_t kMmaSmem = kABytes + kBBytes + 1024;
constexpr int kLookupEntries = 16384;  // 64 KB table

// One CTA per SM: thread 0 issues iters x 4 MMAs of 128 x 256 x 32 into one
// TMEM accumulator (a plain GEMM main loop on operands that stay in shared
// memory), then waits, bounded, for their completion.
__global__ void __launch_bounds__(128, 1) mma_peak_kernel(int iters, int* err) {
    extern __shared__ uint8_t dsmem_raw[];
    __shared__ uint64_t bar_done;
    __shared__ uint32_t s_tmem;
    uint8_t* base = dsmem_raw + ((1024 - (mdfs::tc::smem_u32(dsmem_raw) & 1023)) & 1023);
    uint8_t* sA = base;
    uint8_t* sB = base + kABytes;
    for (uint32_t i = threadIdx.x; i < (kABytes + kBBytes) / 4; i += blockDim.x)
        reinterpret_cast<uint32_t*>(base)[i] = 0x38383838u;  // E4M3 1.0
    if (threadIdx.x == 0) {
        mdfs::tc::mbar_init(&bar_done, 1);
        mdfs::tc::mbar_fence_init();
    }
    if (threadIdx.x < 32) {
        mdfs::tc::tmem_alloc(&s_tmem, kMmaN);
        mdfs::tc::tmem_relinquish();
    }
    mdfs::tc::fence_proxy_async_smem();
    mdfs::tc::tc_fence_before();
    __syncthreads();
    mdfs::tc::tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (threadIdx.x == 0) {
        const uint32_t idesc = mdfs::tc::idesc_e4m3_f32(kMmaM, kMmaN);
        const uint32_t a_addr = mdfs::tc::smem_u32(sA), b_addr = mdfs::tc::smem_u32(sB);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                mdfs::tc::mma_f8(tmem, mdfs::tc::sw128_kmajor_desc(a_addr + 32 * kk),
                                 mdfs::tc::sw128_kmajor_desc(b_addr + 32 * kk), idesc, (it > 0 || kk > 0) ? 1u : 0u);
        }
        mdfs::tc::mma_commit(&bar_done);
        const unsigned long long t0 = mdfs::tc::global_ns();
        while (!mdfs::tc::mbar_try_wait(&bar_done, 0))
            if (mdfs::tc::global_ns() - t0 > mdfs::tc::kWaitLimitNs) {
                atomicOr(err, 1);
                break;
            }
    }
    mdfs::tc::tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) mdfs::tc::tmem_dealloc(tmem, kMmaN);
}

// Every thread runs 8 independent lookup streams; xorshift32 indices, masked to
// the whole table (window == 0) or to `window` consecutive entries starting at
// a warp-wide offset that moves with every lookup.
__global__ void __launch_bounds__(512) lookup_peak_kernel(int iters, int window, unsigned int* sink) {
    extern __shared__ int table[];  // kLookupEntries
    for (int i = threadIdx.x; i < kLookupEntries; i += blockDim.x) table[i] = i * 2654435761u;
    __syncthreads();
    uint32_t x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = 0x9E3779B9u * (uint32_t)(blockIdx.x * blockDim.x + threadIdx.x + 1) + 977u * j;
    const uint32_t mask = window > 0 ? (uint32_t)window - 1 : (uint32_t)kLookupEntries - 1;
    uint32_t centre = 0, acc = 0;
    for (int it = 0; it < iters; ++it) {
        centre = (centre + 4099u) & (kLookupEntries - 1 - mask);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            x[j] ^= x[j] << 13;
            x[j] ^= x[j] >> 17;
            x[j] ^= x[j] << 5;
            acc += (uint32_t)table[centre + (x[j] & mask)];
        }
    }
    if (acc == 0x12345678u) sink[0] = acc;  // keeps the loads
}

}  // namespace

extern "C" int mdfs_bench_mma_f8(int iters, double* tflops, double* seconds) {
    if (iters < 1 || iters > (1 << 24) || !tflops || !seconds) {
        mdfs::record_error("mdfs_bench_mma_f8: iters outside [1, 2^24] or NULL output");
        return MDFS_EINVAL;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) {
        cudaGetLastError();
        mdfs::record_error("mdfs_bench_mma_f8: no CUDA device");
        return MDFS_ECUDA;
    }
    int* err = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MDFS_OK;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess || cudaMemset(err, 0, sizeof(int)) != cudaSuccess ||
        mdfs::ensure_dynamic_smem((const void*)mma_peak_kernel, kMmaSmem) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = MDFS_ECUDA;
    } else {
        mma_peak_kernel<<<sms, 128, kMmaSmem>>>(1, err);  // warm-up
        cudaEventRecord(e0);
        mma_peak_kernel<<<sms, 128, kMmaSmem>>>(iters, err);
        cudaEventRecord(e1);
        float ms = 0.0f;
        int flag = 0;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaMemcpy(&flag, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = MDFS_ECUDA;
        } else if (flag) {
            rc = MDFS_ETIMEOUT;
        } else {
            *seconds = ms / 1e3;
            *tflops = 2.0 * kMmaM * kMmaN * kMmaK * 4.0 * iters * sms / (*seconds) / 1e12;
        }
    }
    if (rc == MDFS_ECUDA) mdfs::record_error(cudaGetErrorString(cudaGetLastError()));
    if (rc == MDFS_ETIMEOUT) mdfs::record_error("mdfs_bench_mma_f8: the MMA wait timed out");
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (err) cudaFree(err);
    return rc;
}

extern "C" int mdfs_bench_smem_lookup(int iters, int window, double* lookups_per_s, double* seconds) {
    if (iters < 1 || iters > (1 << 24) || !lookups_per_s || !seconds ||
        (window != 0 && (window < 32 || window > kLookupEntries / 2 || (window & (window - 1))))) {
        mdfs::record_error("mdfs_bench_smem_lookup: iters outside [1, 2^24], window not 0 or a power of two "
                           "in [32, 8192], or NULL output");
        return MDFS_EINVAL;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) {
        cudaGetLastError();
        mdfs::record_error("mdfs_bench_smem_lookup: no CUDA device");
        return MDFS_ECUDA;
    }
    unsigned int* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MDFS_OK;
    const int blocks = 2 * sms, threads = 512;  // 2 x 64 KB tables per SM
    const size_t smem = kLookupEntries * sizeof(int);
    if (cudaMalloc(&sink, sizeof(unsigned int)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess ||
        mdfs::ensure_dynamic_smem((const void*)lookup_peak_kernel, smem) != cudaSuccess) {
        rc = MDFS_ECUDA;
    } else {
        lookup_peak_kernel<<<blocks, threads, smem>>>(1, window, sink);
        cudaEventRecord(e0);
        lookup_peak_kernel<<<blocks, threads, smem>>>(iters, window, sink);
        cudaEventRecord(e1);
        float ms = 0.0f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = MDFS_ECUDA;
        } else {
            *seconds = ms / 1e3;
            *lookups_per_s = 8.0 * iters * (double)blocks * threads / (*seconds);
        }
    }
    if (rc == MDFS_ECUDA) mdfs::record_error(cudaGetErrorString(cudaGetLastError()));
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    return rc;
}
