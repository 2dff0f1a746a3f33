/*
 * mdfs_testing.h -- test-only entry points of the MDFS library.
 *
 * These calls exist so that the test suite can check internals of the scan
 * kernels that the method's interface (mdfs.h) does not expose.  They are not
 * part of that interface and have no counterpart in the paper; return codes
 * and mdfs_last_error() follow mdfs.h.
 */
#ifndef MDFS_TESTING_H
#define MDFS_TESTING_H

#include <stdint.h>

#include "mdfs.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Voxel counters of the tensor-core scans (section "Algorithm and
 * implementation": the counts of objects of each decision class in every
 * voxel of a tuple's discretised subspace).  Runs mdfs_max_ig's scan for k = 2
 * (divisions 1 or 2) or k = 3 (divisions 1) with pc_xi = 0.25 and the given
 * seed, and has the tensor-core counting kernel also write its class counts:
 *   k = 2: counts[d][r][u c + v]    for every pair i < m, r its rank in the
 *          upper triangle (r = i (2M - i - 1) / 2 + m - i - 1), u and v the
 *          codes of i and m (c = divisions + 1);
 *   k = 3: counts[d][r][4 u + 2 v + w]  for every triple i < m < e, r its
 *          lexicographic rank among the C(M, 3) triples, u, v, w the codes of
 *          i, m, e;
 * each entry n0 | n1 << 16 (class-0 and class-1 objects).  counts is device
 * memory of the current device, caller-owned, with discretizations * C(M, k) *
 * c^k entries.  MDFS_EINVAL when no tensor-core kernel serves the case (k = 2
 * with divisions 3, k = 3 with divisions > 1, class sizes beyond the kernels'
 * shared-memory tables).  Returns after completion.
 */
int mdfs_testing_counts(const mdfs_data* data, int k, int divisions, int discretizations, double range, uint64_t seed,
                        uint32_t* counts, void* stream);

/*
 * Bounded-wait test of the tensor-core triple kernel (k = 3, two classes).
 * Arms a one-shot hook that the next such scan of any thread takes and
 * clears: every mbarrier wait of that launch gives up after wait_ns
 * nanoseconds (0 = the library's 1 s), and with withhold_kb >= 0 the TMA
 * producer of CTA 0 never fills the stage of that K block of its running
 * count, so its consumers' wait runs out and the scan returns MDFS_ETIMEOUT
 * after draining its copies and MMAs and freeing its tensor memory.
 * withhold_kb = -1 with wait_ns = 0 disarms the hook.
 * Errors: MDFS_EINVAL for withhold_kb < -1 or wait_ns outside [0, 10 s].
 */
int mdfs_testing_k3_wait_fault(int withhold_kb, long long wait_ns);

/*
 * Arms a one-shot hook that the next tensor-core scan (k = 2 or k = 3) of any
 * thread takes and clears: that scan evaluates the regularised entropy of
 * every tuple exactly, without skipping the tuples that a lower bound of the
 * entropy rules out.  Its results must equal those of the normal scan bit for
 * bit.  Returns 0.
 */
int mdfs_testing_exact(void);

/*
 * Host only (no CUDA call): the order in which the k = 3 tensor-core scan of
 * M variables over nd discretisations hands out its tiles (tile t = item
 * t % n_items of discretisation t / n_items, items (b, a-tile, e-group) in
 * the scan's order), by descending modelled epilogue cost.  Writes up to cap
 * tile indices to order (host memory) and returns the number of tiles, or a
 * negative MDFS error for M outside [3, 65535], nd outside [1, 1024] or a NULL
 * order with cap > 0.
 */
int mdfs_testing_k3_claim_order(int M, int nd, int32_t* order, int cap);

#ifdef __cplusplus
}
#endif

#endif /* MDFS_TESTING_H */
