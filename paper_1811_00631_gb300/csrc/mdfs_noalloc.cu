// mdfs_max_ig_noalloc: the k = 1 / k = 2 scan without any device allocation.
//
// Some callers cannot let a library allocate device memory: a serving process
// whose allocator owns the whole device budget, a host application that only
// lets plug-ins use memory it handed out, or a latency-bound loop that cannot
// pay for cudaMalloc/cudaFree and the synchronisation they imply.  This entry
// point runs the same kernels as mdfs_max_ig (k = 1, 2) with every scratch
// buffer carved from one file-scope device array of fixed size.  The caller
// passes device pointers for all inputs and outputs.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/mdfs.h"
#include "mdfs_internal.cuh"

using namespace mdfs;

// Scratch shared by every call of mdfs_max_ig_noalloc on a device.  Every
// GPU that loads this library holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MDFS_NOALLOC_SCRATCH_BYTES];

namespace {

int fail(int code, const char* msg) {
    record_error(msg);  // shown by mdfs_last_error()
    return code;
}

// Device address of g_noalloc_scratch, looked up once per device with that
// device current (host code only sees a host-side stand-in under that name).
// The address belongs to the device's current context: mdfs_release() drops
// the cache, which a caller must do after a cudaDeviceReset.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

int scratch_for_current_device(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(MDFS_ECUDA, "mdfs_max_ig_noalloc: no current CUDA device");
    }
    if (dev < 0 || dev >= kMaxDevices) return fail(MDFS_EINVAL, "mdfs_max_ig_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(MDFS_ECUDA, "mdfs_max_ig_noalloc: cudaGetSymbolAddress of the scratch array failed");
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return MDFS_OK;
}

// Device memory of the current device, or managed memory.
bool on_device(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Carves 256-byte-aligned pieces off the scratch array; `used` is the running total.
struct Carver {
    unsigned char* base;
    size_t used = 0;
    void* take(size_t bytes) {
        used = (used + 255) & ~(size_t)255;
        void* p = base ? base + used : nullptr;
        used += bytes;
        return p;
    }
};

}  // namespace

namespace mdfs {
void noalloc_forget_devices() {
    std::lock_guard<std::mutex> lock(g_mu);
    for (void*& p : g_scratch_ptr) p = nullptr;
}
}  // namespace mdfs

extern "C" int mdfs_max_ig_noalloc(const mdfs_data* data, int k, int divisions, int discretizations, double range,
                                   double pc_xi, uint64_t seed, float* ig, int32_t* tuples, int32_t* best_disc,
                                   void* stream) {
    record_error("");
    if (!data || !data->x || !data->y || !ig) return fail(MDFS_EINVAL, "mdfs_max_ig_noalloc: NULL argument");
    const int N = data->N, M = data->M, D = discretizations, c = divisions + 1;
    if (data->dtype != MDFS_F32 && data->dtype != MDFS_I8) return fail(MDFS_EINVAL, "mdfs_max_ig_noalloc: bad dtype");
    if (k < 1 || k > 2) return fail(MDFS_EINVAL, "mdfs_max_ig_noalloc: k must be 1 or 2");
    if (divisions < 1 || c > kMaxC) return fail(MDFS_EINVAL, "mdfs_max_ig_noalloc: divisions outside [1, 3]");
    if (N < c || N > kMaxN || M < k || M > 65535 || D < 1 || D > kMaxD)
        return fail(MDFS_EINVAL, "mdfs_max_ig_noalloc: N, M or discretizations out of range");
    if ((unsigned long long)D * M >= (1ull << 32)) return fail(MDFS_EINVAL, "mdfs_max_ig_noalloc: discretizations * M too large");
    if (!(range >= 0.0 && range <= 1.0) || !(pc_xi > 0.0 && pc_xi < 1.0))
        return fail(MDFS_EINVAL, "mdfs_max_ig_noalloc: range must lie in [0, 1] and pc_xi in (0, 1)");
    if (!on_device(data->x) || !on_device(data->y) || !on_device(ig) || (tuples && !on_device(tuples)) ||
        (best_disc && !on_device(best_disc)))
        return fail(MDFS_EINVAL,
                    "mdfs_max_ig_noalloc: x, y and every output must be device pointers of the current device");

    // scratch layout; planes sized for the worst class split (Ws <= round_up(ceil(N/32) + 1, 4))
    const int P = c - 1;
    const int ws_max = ((N + 31) / 32 + 2 + 3) & ~3;
    Carver sizer{nullptr};
    sizer.take(16 * sizeof(int));                               // stats
    sizer.take((size_t)N * sizeof(int));                        // perm
    sizer.take((size_t)3 * (N + 1) * sizeof(long long));        // entropy tables
    sizer.take((size_t)D * M * P * ws_max * sizeof(uint32_t));  // bit planes
    sizer.take((size_t)D * M * P * 2 * sizeof(int));            // single counts
    sizer.take((size_t)D * M * sizeof(long long));              // SH1
    sizer.take((size_t)M * sizeof(unsigned long long));         // keys
    if (sizer.used > (size_t)MDFS_NOALLOC_SCRATCH_BYTES) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "mdfs_max_ig_noalloc: this problem needs %zu bytes of scratch; the fixed scratch array holds %zu",
                 sizer.used, (size_t)MDFS_NOALLOC_SCRATCH_BYTES);
        return fail(MDFS_EINVAL, msg);
    }
    void* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    Carver cv{(unsigned char*)scratch};
    int* stats = (int*)cv.take(16 * sizeof(int));
    int* perm = (int*)cv.take((size_t)N * sizeof(int));
    long long* tab = (long long*)cv.take((size_t)3 * (N + 1) * sizeof(long long));
    uint32_t* planes = (uint32_t*)cv.take((size_t)D * M * P * ws_max * sizeof(uint32_t));
    int* cnt1 = (int*)cv.take((size_t)D * M * P * 2 * sizeof(int));
    long long* sh1 = (long long*)cv.take((size_t)D * M * sizeof(long long));
    unsigned long long* keys = (unsigned long long*)cv.take((size_t)M * sizeof(unsigned long long));

    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
#define NOALLOC_TRY(expr)                                                                             \
    do {                                                                                              \
        if ((e = (expr)) != cudaSuccess) {                                                            \
            char msg[256];                                                                            \
            snprintf(msg, sizeof msg, "mdfs_max_ig_noalloc: %s: %s", #expr, cudaGetErrorString(e));    \
            return fail(MDFS_ECUDA, msg);                                                             \
        }                                                                                             \
    } while (0)
    // validation: class counts, labels, finiteness (16 bytes read back into a host stack buffer)
    NOALLOC_TRY(cudaMemsetAsync(stats, 0, 16 * sizeof(int), st));
    NOALLOC_TRY(launch_stats(data->y, N, stats, perm, st));
    if (data->dtype == MDFS_F32) NOALLOC_TRY(launch_check_finite((const float*)data->x, (long long)M * N, stats + 2, st));
    int hs[4] = {0, 0, 0, 0};
    NOALLOC_TRY(cudaMemcpyAsync(hs, stats, sizeof hs, cudaMemcpyDeviceToHost, st));
    NOALLOC_TRY(cudaStreamSynchronize(st));
    if (hs[2] != 0) return fail(MDFS_ENONFINITE, "mdfs_max_ig_noalloc: x holds NaN or Inf values");
    if (hs[1] != 0) return fail(MDFS_EINVAL, "mdfs_max_ig_noalloc: y holds values outside {0, 1}");
    const int n1 = hs[0], n0 = N - n1;
    if (n0 == 0 || n1 == 0) return fail(MDFS_EDEGENERATE, "mdfs_max_ig_noalloc: decision has a single class");
    const double mn = (double)(n0 < n1 ? n0 : n1);
    const PlaneGeom g = make_geom(N, n0);

    NOALLOC_TRY(launch_ftable(N, pc_xi * n0 / mn, pc_xi * n1 / mn, tab, st));
    NOALLOC_TRY(launch_discretize(data->x, data->dtype, N, M, c, D, range, seed, perm, g, planes, nullptr, nullptr,
                                  nullptr, TcGeom{}, st));
    // the array keeps the previous call's contents: the keys must start at zero
    NOALLOC_TRY(cudaMemsetAsync(keys, 0, (size_t)M * sizeof(unsigned long long), st));
    NOALLOC_TRY(launch_k1(planes, g, M, c, D, tab, cnt1, sh1, k == 1 ? keys : nullptr, st));
    if (k == 2)
        NOALLOC_TRY(launch_k2(planes, g, M, c, D, 0, D, tab, cnt1, sh1, keys, nullptr, nullptr, nullptr, 0, st));
    NOALLOC_TRY(launch_finalize(keys, M, k, ig, k == 2 ? tuples : nullptr, best_disc, st));
    if (st == nullptr) NOALLOC_TRY(cudaStreamSynchronize(st));
#undef NOALLOC_TRY
    return MDFS_OK;
}
