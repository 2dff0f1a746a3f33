// Triple tables for the k = 4 and k = 5 scans (two classes per variable):
// for every triple x < y < z of one discretisation, the packed all-ones count
// n_xyz (both classes) and the entropy SH(x, y, z) of Eq. 1's voxel counters
// (section "Algorithm and implementation"), stored at the triple's
// lexicographic rank.  The higher-order kernels then count only the subsets
// that contain all of their variables and read every lower-order count and
// entropy from these tables instead of recounting it per tuple.
//
// Work item: (x, a tile of 32 y > x, a tile of 32 z > y); 16 x 16 threads,
// 2 x 2 (y, z) per thread; X & Y and Z rows staged in shared memory in
// chunks of 128 words.
#include <cuda_runtime.h>

#include <vector>

#include "mdfs_device.cuh"
#include "mdfs_internal.cuh"
#include "mdfs_packed.cuh"

namespace mdfs {

namespace {

constexpr int kThreads = 256;
constexpr int kTY = 32, kTZ = 32;
constexpr int kWC = 128;      // staged words per chunk (even)
constexpr int kLD = kWC + 2;  // row stride: uint2 loads, z rows two banks apart

__global__ void __launch_bounds__(kThreads) t3_kernel(const uint32_t* __restrict__ planes, PlaneGeom g, int M, int d0,
                                                      const int2* __restrict__ items,
                                                      const long long* __restrict__ tab,
                                                      const int* __restrict__ cnt1, const int* __restrict__ cnt2,
                                                      uint32_t* __restrict__ t3c, long long* __restrict__ t3s) {
    __shared__ __align__(16) uint32_t sXY[kTY * kLD], sZ[kTZ * kLD], sX[kWC];
    const int2 it = items[blockIdx.x];
    const int x = it.x & 0xFFFF;
    const int y0 = x + 1 + (it.x >> 16) * kTY;
    const int z0 = y0 + 1 + it.y * kTZ;
    const int dl = blockIdx.y, d = d0 + dl;
    const int tid = threadIdx.x, ty = tid >> 4, tz = tid & 15;
    const uint32_t* pbase = planes + (size_t)d * M * g.Ws;
    const Staging z = make_staging(g.W0, g.W1);

    uint32_t acc[2][2] = {{0u, 0u}, {0u, 0u}};
    for (int s0 = 0; s0 < z.Wst; s0 += kWC) {
        const int len = min(kWC, z.Wst - s0);
        __syncthreads();
        for (int j = tid; j < kWC; j += kThreads) sX[j] = j < len ? staged_word(pbase + (size_t)x * g.Ws, s0 + j, z) : 0u;
        __syncthreads();
        for (int idx = tid; idx < (kTY + kTZ) * kWC; idx += kThreads) {
            const int r = idx / kWC, j = idx % kWC;
            const int v = r < kTY ? y0 + r : z0 + (r - kTY);
            const uint32_t w = (j < len && v < M) ? staged_word(pbase + (size_t)v * g.Ws, s0 + j, z) : 0u;
            if (r < kTY) sXY[r * kLD + j] = w & sX[j];
            else sZ[(r - kTY) * kLD + j] = w;
        }
        __syncthreads();
        int lo[2], hi[2];
        class_segments(z, s0, kWC, lo, hi);
#pragma unroll
        for (int cls = 0; cls < 2; ++cls) {
            const uint32_t mul = cls ? 65536u : 1u;
            for (int j = lo[cls]; j < hi[cls]; j += 2) {
                uint2 u[2], w[2];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    u[r] = *reinterpret_cast<const uint2*>(sXY + (ty + 16 * r) * kLD + j);
                    w[r] = *reinterpret_cast<const uint2*>(sZ + (tz + 16 * r) * kLD + j);
                }
#pragma unroll
                for (int ry = 0; ry < 2; ++ry)
#pragma unroll
                    for (int rz = 0; rz < 2; ++rz)
                        acc[ry][rz] += (uint32_t)(__popc(u[ry].x & w[rz].x) + __popc(u[ry].y & w[rz].y)) * mul;
            }
        }
    }

    Tabs tb;
    tb.tab = tab;  // wide layout
    const uint32_t NC = pack2(g.N0, g.N1);
    auto single = [&](int v) -> uint32_t {
        const int* p = cnt1 + ((size_t)d * M + v) * 2;
        return pack2(__ldg(p), __ldg(p + 1));
    };
    auto pair = [&](int i, int m) -> uint32_t {  // i < m
        const int* p = cnt2 + (((size_t)dl * M + i) * M + m) * 2;
        return pack2(__ldg(p), __ldg(p + 1));
    };
    const Rank3 rk = make_rank3(M);
    const size_t K3 = (size_t)rk.top + 1;
    const uint32_t nx = single(x), rx = rk.part_x(x);
#pragma unroll
    for (int ry = 0; ry < 2; ++ry) {
        const int y = y0 + ty + 16 * ry;
        if (y >= M) continue;
        const uint32_t ny = single(y), nxy = pair(x, y), rxy = rx + rk.part_y(y);
#pragma unroll
        for (int rz = 0; rz < 2; ++rz) {
            const int zz = z0 + tz + 16 * rz;
            if (zz >= M || zz <= y) continue;
            // bits x = 1, y = 2, z = 4
            uint32_t q[8] = {NC, nx, ny, nxy, single(zz), pair(x, zz), pair(y, zz), acc[ry][rz]};
            moebius_packed<3>(q);
            const size_t at = (size_t)dl * K3 + (rk.top - (rxy + (uint32_t)(rk.Mm1 - zz)));
            t3c[at] = acc[ry][rz];
            t3s[at] = sh_packed<3>(q, tb);
        }
    }
}

}  // namespace

// (x | y-tile << 16, z-tile) for x < y-tile < z-tile with a valid (y, z) pair
void build_t3_items(int M, std::vector<int2>& items) {
    items.clear();
    for (int x = 0; x + 2 < M; ++x)
        for (int ty = 0;; ++ty) {
            const int ymin = x + 1 + ty * kTY;
            if (ymin > M - 2) break;
            for (int tz = 0;; ++tz) {
                const int zmin = ymin + 1 + tz * kTZ;
                if (zmin > M - 1) break;
                items.push_back(make_int2(x | (ty << 16), tz));
            }
        }
}

size_t t3_entries(int M) {
    const size_t m = (size_t)M;
    return M < 3 ? 0 : m * (m - 1) / 2 * (m - 2) / 3;
}

cudaError_t launch_t3(const uint32_t* planes, PlaneGeom g, int M, int d0, int nd, const int2* items, int n_items,
                      const long long* tab, const int* cnt1, const int* cnt2, uint32_t* t3c, long long* t3s,
                      cudaStream_t st) {
    if (n_items == 0 || nd == 0) return cudaSuccess;
    if (nd > 65535) return cudaErrorInvalidValue;
    t3_kernel<<<dim3(n_items, nd), kThreads, 0, st>>>(planes, g, M, d0, items, tab, cnt1, cnt2, t3c, t3s);
    return cudaGetLastError();
}

}  // namespace mdfs
