// Device helpers of the two-class (c = 2) higher-order scans (k = 3 tables,
// k = 4, k = 5): class-sorted bit planes staged word by word, voxel counts of
// both classes packed in one 32-bit word, Moebius inversion over supersets,
// entropy sums from the f(n + beta) tables, and lexicographic ranks of
// variable subsets.
#pragma once

#include <cstdint>

namespace mdfs {

// Packed counts: class 0 in bits 0..15, class 1 in bits 16..31.  Inversion
// and marginalisation only add and subtract counts that stay non-negative, so
// the halves never borrow from each other (class sizes below 2^16).
constexpr uint32_t kPackLo = 0xFFFFu;

__device__ __forceinline__ uint32_t pack2(int n0, int n1) { return (uint32_t)n0 | ((uint32_t)n1 << 16); }

// In-place Moebius inversion over supersets of L bits: on entry n[T] is the
// all-ones count of subset T, on exit n[O] the count of the voxel whose ones
// are exactly O.
template <int L>
__device__ __forceinline__ void moebius_packed(uint32_t (&n)[1 << L]) {
#pragma unroll
    for (int j = 0; j < L; ++j)
#pragma unroll
        for (int m = 0; m < (1 << L); ++m)
            if (!(m & (1 << j))) n[m] -= n[m | (1 << j)];
}

// The f(n + beta) tables in the wide layout (launch_ftable_wide): f(n + b0) at
// [0, 2^16), f(n + b1) at [2^16, 2^17), f(n + b0 + b1) at [2^17, 2^18), so
// that every packed word indexes inside the tables.
struct Tabs {
    const long long* tab;
};
// one voxel's f(n0+n1+b0+b1) - f(n0+b0) - f(n1+b1)
__device__ __forceinline__ long long voxel_sh(uint32_t v, const Tabs& t) {
    const uint32_t n0 = v & kPackLo, n1 = v >> 16;
    return __ldg(t.tab + (1u << 17) + n0 + n1) - __ldg(t.tab + n0) - __ldg(t.tab + (1u << 16) + n1);
}
template <int L>
__device__ __forceinline__ long long sh_packed(const uint32_t (&n)[1 << L], const Tabs& t) {
    long long s = 0;
#pragma unroll
    for (int m = 0; m < (1 << L); ++m) s += voxel_sh(n[m], t);
    return s;
}

// binomial coefficients C(x, 2..4) for 0 <= x < 2^16, as 64-bit (0 for x < r)
__device__ __forceinline__ unsigned long long bin2(unsigned long long x) { return x * (x - 1) / 2; }
__device__ __forceinline__ unsigned long long bin3(unsigned long long x) { return x * (x - 1) * (x - 2) / 6; }
__device__ __forceinline__ unsigned long long bin4(unsigned long long x) {
    return x * (x - 1) * (x - 2) * (x - 3) / 24;
}

// Lexicographic rank of the triple x < y < z among the 3-subsets of [0, M):
// C(M,3) - 1 - [C(M-1-x,3) + C(M-1-y,2) + (M-1-z)] (combinatorial number
// system on M-1-s); consecutive z give consecutive ranks.
struct Rank3 {
    uint32_t top;  // C(M,3) - 1
    int Mm1;
    __device__ __forceinline__ uint32_t part_x(int x) const { return (uint32_t)bin3((unsigned long long)(Mm1 - x)); }
    __device__ __forceinline__ uint32_t part_y(int y) const { return (uint32_t)bin2((unsigned long long)(Mm1 - y)); }
    __device__ __forceinline__ uint32_t of(int x, int y, int z) const {
        return top - (part_x(x) + part_y(y) + (uint32_t)(Mm1 - z));
    }
};
__device__ __forceinline__ Rank3 make_rank3(int M) {
    Rank3 r;
    r.top = (uint32_t)(bin3((unsigned long long)M) - 1ull);
    r.Mm1 = M - 1;
    return r;
}

// Lexicographic rank of the quadruple w < x < y < z among the 4-subsets of
// [0, M): C(M,4) - 1 - [C(M-1-w,4) + C(M-1-x,3) + C(M-1-y,2) + (M-1-z)]
// (requires C(M,4) < 2^32); consecutive z give consecutive ranks.
struct Rank4 {
    uint32_t top;  // C(M,4) - 1
    int Mm1;
    __device__ __forceinline__ uint32_t part_w(int w) const { return (uint32_t)bin4((unsigned long long)(Mm1 - w)); }
    __device__ __forceinline__ uint32_t part_x(int x) const { return (uint32_t)bin3((unsigned long long)(Mm1 - x)); }
    __device__ __forceinline__ uint32_t part_y(int y) const { return (uint32_t)bin2((unsigned long long)(Mm1 - y)); }
};
__device__ __forceinline__ Rank4 make_rank4(int M) {
    Rank4 r;
    r.top = (uint32_t)(bin4((unsigned long long)M) - 1ull);
    r.Mm1 = M - 1;
    return r;
}

// Staged word space: class-0 words at [0, W0e), class-1 words at [W0e, Wst),
// each class zero-padded to an even length so word pairs never straddle it.
struct Staging {
    int W0, W1, W0e, Wst;
};
__device__ __forceinline__ Staging make_staging(int W0, int W1) {
    Staging z;
    z.W0 = W0;
    z.W1 = W1;
    z.W0e = (W0 + 1) & ~1;
    z.Wst = z.W0e + ((W1 + 1) & ~1);
    return z;
}
__device__ __forceinline__ uint32_t staged_word(const uint32_t* __restrict__ row, int s, const Staging& z) {
    if (s < z.W0e) return s < z.W0 ? __ldg(row + s) : 0u;
    const int w = s - z.W0e;
    return w < z.W1 ? __ldg(row + z.W0 + w) : 0u;
}
// class segments [lo, hi) of the chunk [s0, s0 + kw) in chunk-local indices
__device__ __forceinline__ void class_segments(const Staging& z, int s0, int kw, int (&lo)[2], int (&hi)[2]) {
    const int s1 = min(s0 + kw, z.Wst);
    lo[0] = 0;
    hi[0] = max(0, min(s1, z.W0e) - s0);
    lo[1] = max(s0, z.W0e) - s0;
    hi[1] = s1 - s0;
}

// Asynchronous global -> shared copies of 4 or 8 bytes (cp.async); a copy
// with valid == false writes zeros and reads nothing.
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace mdfs
