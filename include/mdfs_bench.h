/*
 * mdfs_bench.h -- hardware microbenchmarks of the MDFS library.
 *
 * They measure, on the current device, the two rates that bound the scan
 * kernels, so that the benchmark can state roofline fractions against
 * measured peaks.  Not part of the method; the paper has no counterpart.
 * Return codes and mdfs_last_error() follow mdfs.h.
 */
#ifndef MDFS_BENCH_H
#define MDFS_BENCH_H

#include "mdfs.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Dense E4M3 x E4M3 -> F32 tensor-core throughput: one CTA per SM issues
 * iters x 4 tcgen05.mma (kind::f8f6f4, M = 128, N = 256, K = 32, both operands
 * in shared memory) into one tensor-memory accumulator; timed with CUDA events
 * after a warm-up launch.  *tflops = 2 M N K x instructions / seconds / 1e12.
 * iters: 1 .. 2^24.  Synchronous.  MDFS_ETIMEOUT if the final wait (bounded,
 * 1 s) gave up.
 */
int mdfs_bench_mma_f8(int iters, double* tflops, double* seconds);

/*
 * Random 4-byte shared-memory loads: 2 CTAs per SM of 512 threads, each
 * thread 8 independent xorshift32 index streams over a 64 KB table
 * (window = 0) or within `window` consecutive entries (a power of two in
 * [32, 8192]) at a warp-wide offset; *lookups_per_s counts thread loads.
 * iters: 1 .. 2^24.  Synchronous.
 */
int mdfs_bench_smem_lookup(int iters, int window, double* lookups_per_s, double* seconds);

#ifdef __cplusplus
}
#endif

#endif /* MDFS_BENCH_H */
