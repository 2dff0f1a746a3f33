// Device helpers of the MDFS kernels: Philox4x32-10, max/argmax keys, entropy tables.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mdfs {

// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11):
// ten rounds of two 32x32->64 multiplications with the published multipliers
// and Weyl key schedule.
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t out[4]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// Order-preserving map of an IEEE float to uint32 (larger float -> larger key).
__device__ __forceinline__ uint32_t float_order_bits(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float order_bits_float(uint32_t o) {
    const uint32_t b = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
    return __uint_as_float(b);
}

// Packed max/argmax key: high word = ordered IG, low word = ~index, so that a
// larger key is a larger IG and, on an exact tie, a smaller index.
__device__ __forceinline__ unsigned long long pack_key(float ig, uint32_t index) {
    return ((unsigned long long)float_order_bits(ig) << 32) | (unsigned long long)(~index);
}

// Hash-table key of an interesting (variable, partners) record; unused partners 0xFFFF.
__device__ __forceinline__ unsigned long long emit_key(int v, int p1, int p2, int p3) {
    return (unsigned long long)(uint16_t)v | ((unsigned long long)(uint16_t)p1 << 16) |
           ((unsigned long long)(uint16_t)p2 << 32) | ((unsigned long long)(uint16_t)p3 << 48);
}

// SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014): a bijective
// 64-bit mixer, used to spread record keys over the hash table.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// k = 5 record key: five 12-bit fields (variable, then partners ascending),
// v in bits 0..11 and p4 in bits 48..59 (the k = 5 limit D C(M,4) < 2^32
// keeps M below 569); never equal to the empty key.
__device__ __forceinline__ unsigned long long emit_key5(int v, int p1, int p2, int p3, int p4) {
    return (unsigned long long)v | ((unsigned long long)p1 << 12) | ((unsigned long long)p2 << 24) |
           ((unsigned long long)p3 << 36) | ((unsigned long long)p4 << 48);
}

// Inserts (key, packed value) into an emission table (EmitTable of
// mdfs_internal.cuh): linear probing from mix64(key), the slot claimed by
// compare-and-swap, the value max-reduced.  The probe count is bounded by the
// table size; a table with no free slot raises t.full.
constexpr unsigned long long kEmptyEmitKey = ~0ull;
template <class Table>
__device__ __forceinline__ void emit_insert(const Table& t, unsigned long long key, unsigned long long val) {
    unsigned int slot = (unsigned int)mix64(key) & t.mask;
    for (unsigned int probe = 0; probe <= t.mask; ++probe) {
        const unsigned long long prev = atomicCAS(t.keys + slot, kEmptyEmitKey, key);
        if (prev == kEmptyEmitKey || prev == key) {
            if (prev == kEmptyEmitKey) atomicAdd(t.n_keys, 1);
            atomicMax(t.vals + slot, val);
            return;
        }
        slot = (slot + 1) & t.mask;
    }
    atomicOr(t.full, 1);
}

// Fixed-point IG (multiples of 2^-32) to float with a single rounding.
__device__ __forceinline__ float fx_to_float(long long v) {
    return __ll2float_rn(v) * 2.3283064365386963e-10f;  // exact scaling by 2^-32
}

// int64 multiple of 2^-32  ->  int32 multiple of 2^-s (round to nearest, mod 2^32)
__device__ __forceinline__ int fx_narrow(long long v, int s) {
    const int shift = 32 - s;
    return (int)((v + (1ll << (shift - 1))) >> shift);
}

// Packed FP32 pairs: two independent lanes per instruction (sm_100 and later),
// each rounded as the scalar operation would be.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Counts index the [0, n] tables; a count outside that range cannot arise from
// consistent inputs, and clamping keeps every table read inside its buffer.
__device__ __forceinline__ int clamp_count(int v, int n) { return min(max(v, 0), n); }

// Regularised voxel entropy h(n0, n1) = f(n0+n1+b0+b1) - f(n0+b0) - f(n1+b1)
// from the [3][N+1] fixed-point tables.
__device__ __forceinline__ long long voxel_h(const long long* __restrict__ tab, int np1, int n0, int n1) {
    const int n = np1 - 1;
    n0 = clamp_count(n0, n);
    n1 = clamp_count(n1, n);
    return __ldg(tab + 2 * np1 + clamp_count(n0 + n1, n)) - __ldg(tab + n0) - __ldg(tab + np1 + n1);
}

}  // namespace mdfs
