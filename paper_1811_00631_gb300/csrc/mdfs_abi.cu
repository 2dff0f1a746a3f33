// Host side of the MDFS C ABI (include/mdfs.h): argument checks, input staging,
// per-(device, stream) workspaces and the launch sequence of the scan.
#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>

#include <cmath>

#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <initializer_list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mdfs.h"
#include "../../include/mdfs_testing.h"
#include "mdfs_internal.cuh"

using namespace mdfs;

// dynamic shared memory the tensor-core k = 3 kernel may take (stages + tables)
static const size_t kK3tcMaxSmem = 212 * 1024;

namespace {

thread_local std::string g_err;
thread_local int g_launches = 0;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

struct Buffer {
    void* p = nullptr;
    size_t cap = 0;
};

struct Workspace {
    int device = 0;
    cudaStream_t stream = nullptr;
    Buffer x, y, stats, perm, tab, planes, cnt1, sh1, keys, sh2, cnt2, items, ig, tuples, disc, codes, mask, pv, res;
    Buffer pairs2, items2, onehot, err;
    Buffer bx, by, bidx, bperm;  // batch: gathered job data and the job index maps
    Buffer items3;               // k = 2 tensor-core tile list
    Buffer bcounts, bonehot, btab, bcnt1, bsh1, bkeys;  // batch: class sizes; a chunk's operands and tables
    Buffer bsorted, bmult, bthr;  // batch: sorted keys of every variable; one job's multiplicities and thresholds
    Buffer lperm, lrank, cnt1s, onehot2;  // k = 3 tensor path: relabelling and relabelled operands
    Buffer k3sched[2], k3claim;           // k = 3 tensor path: tile orders of recent launch shapes, claim counter
    Buffer mkeys;                         // several-k calls: the k = 1 and k = 2 keys of a fused scan
    Buffer itemsg;                        // k = 4, 5 with three or four classes: pair items
    int itemsg_M = -1, itemsg_k = -1, n_itemsg = 0;
    long long k3sched_key[2][4] = {{-1}, {-1}};
    int k3sched_next = 0;
    std::vector<int2> items2_host;        // the k = 3 tensor path's tile list (host copy)
    Buffer xe, srcb, igx, tux, dix, pext, padj, adjb, relb;  // contrast variables and the selection pipeline
    Buffer items4;                                           // k = 4 work items
    Buffer items5;                                           // k = 5 work items
    Buffer items3t, t3c, t3s;                                // triple tables (k = 4, 5)
    Buffer t4c, t4s;                                         // quadruple tables (k = 5)
    Buffer tabw;                                             // wide-layout f tables (k = 4, 5)
    Buffer keys5, kdisc;                                     // k = 5 per-discretisation keys, best discretisation
    bool k5_wide = false;                                    // keys hold (IG, rank) and kdisc the discretisation
    Buffer ekeys, evals, ecnt, erk, erv;                     // interesting-tuple table and its records
    int items4_M = -1, n_items4 = 0;
    int items5_M = -1, n_items5 = 0;
    int items3t_M = -1, n_items3t = 0;
    int items3_M = -1, items3_c = -1, n_items3 = 0;
    int items2_M = -1, n_items2 = 0;
    int* host_stats = nullptr;  // pinned, 16 ints
    double* host_res = nullptr; // pinned, 4 doubles
    int items_M = -1, items_c = -1, n_items = 0;

    ~Workspace() {
        Buffer* all[] = {&x,  &y,  &stats, &perm,   &tab, &planes, &cnt1, &sh1,   &keys, &sh2,  &cnt2,
                         &items, &ig, &tuples, &disc, &codes, &mask,  &pv,   &res, &pairs2, &items2,
                         &onehot, &err, &bx,   &by,  &bidx, &bperm, &items3, &lperm, &lrank, &cnt1s,
                         &onehot2, &k3sched[0], &k3sched[1], &k3claim, &mkeys, &itemsg, &xe, &srcb, &igx, &tux, &dix, &pext, &padj, &adjb, &relb, &items4, &items5, &items3t, &t3c, &t3s, &t4c, &t4s, &tabw, &keys5, &kdisc, &ekeys, &evals, &ecnt, &erk, &erv,
                         &bcounts, &bonehot, &btab, &bcnt1, &bsh1, &bkeys, &bsorted, &bmult, &bthr};
        for (Buffer* b : all)
            if (b->p) cudaFree(b->p);
        if (host_stats) cudaFreeHost(host_stats);
        if (host_res) cudaFreeHost(host_res);
    }

    // Grows a buffer to at least `bytes`; waits for the stream before freeing.
    bool ensure(Buffer& b, size_t bytes) {
        if (bytes == 0) bytes = 16;
        if (b.cap >= bytes) return true;
        if (b.p) {
            cudaStreamSynchronize(stream);
            cudaFree(b.p);
            b.p = nullptr;
            b.cap = 0;
        }
        size_t want = bytes + bytes / 8;
        if (cudaMalloc(&b.p, want) != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            return false;
        }
        b.cap = want;
        return true;
    }
};

std::mutex g_mu;
std::map<std::pair<int, cudaStream_t>, std::unique_ptr<Workspace>> g_ws;

// Error flag of the tensor-core kernels: 1 a bounded wait gave up, 2 dynamic
// shared memory smaller than the table layout, 4 voxel counts outside the
// entropy tables (inconsistent pair records).  job >= 0 names a batch job.
int kernel_flag_error(int flag, int job = -1) {
    char where[32] = "";
    if (job >= 0) snprintf(where, sizeof where, "job %d: ", job);
    if (flag & 2) return fail(MDFS_ECUDA, "%stensor-core kernel: dynamic shared memory smaller than its table layout", where);
    if (flag & 4) return fail(MDFS_ECUDA, "%stensor-core kernel: voxel counts outside the entropy tables", where);
    return fail(MDFS_ETIMEOUT, "%sa device-side wait timed out in a tensor-core kernel", where);
}

// Test hooks of the tensor-core kernels: the wait fault (mdfs_testing_k3_wait_fault)
// is taken by the next k = 3 tensor-core scan, the exact evaluation
// (mdfs_testing_exact) by the next k = 2 or k = 3 one, each then cleared.
std::mutex g_hooks_mu;
TcTestHooks g_hooks;
TcTestHooks take_test_hooks(bool k3) {
    std::lock_guard<std::mutex> lock(g_hooks_mu);
    TcTestHooks h = g_hooks;
    if (k3) {
        g_hooks = TcTestHooks();
    } else {
        h.wait_ns = 0;
        h.withhold_kb = -1;
        g_hooks.exact = false;
    }
    return h;
}

Workspace* get_ws(cudaStream_t st, int* err) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        *err = fail(MDFS_ECUDA, "no CUDA device is available");
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    auto key = std::make_pair(dev, st);
    auto it = g_ws.find(key);
    if (it != g_ws.end()) return it->second.get();
    std::unique_ptr<Workspace> ws(new Workspace());
    ws->device = dev;
    ws->stream = st;
    if (cudaMallocHost(&ws->host_stats, 16 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&ws->host_res, 4 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        *err = fail(MDFS_ENOMEM, "pinned host staging allocation failed");
        return nullptr;
    }
    Workspace* raw = ws.get();
    g_ws[key] = std::move(ws);
    return raw;
}

// Device index of p when it is device memory of a GPU other than the current
// one (the library would hand it to the current device's kernels); -1 for
// host memory, managed memory, device memory of the current GPU or NULL.
int foreign_device(const void* p) {
    if (!p) return -1;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (a.type != cudaMemoryTypeDevice) return -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return a.device == dev ? -1 : a.device;
}

// MDFS_EINVAL naming the first argument that lives on another GPU.
int check_devices(std::initializer_list<std::pair<const void*, const char*>> ptrs) {
    for (const auto& pr : ptrs) {
        const int d = foreign_device(pr.first);
        if (d >= 0) return fail(MDFS_EINVAL, "%s is device memory of GPU %d, not of the current device", pr.second, d);
    }
    return MDFS_OK;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

#define MDFS_CUDA_TRY(expr)                                                                         \
    do {                                                                                            \
        cudaError_t _e = (expr);                                                                    \
        if (_e != cudaSuccess) return fail(MDFS_ECUDA, "%s: %s", #expr, cudaGetErrorString(_e));     \
    } while (0)

// ---- optional per-kernel CUDA-event timing (mdfs_profile) -------------------
struct ProfRec {
    const char* name;
    cudaEvent_t ev0, ev1;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_recs;
std::vector<cudaEvent_t> g_prof_pool;

cudaEvent_t prof_event() {
    if (!g_prof_pool.empty()) {
        cudaEvent_t e = g_prof_pool.back();
        g_prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

#define MDFS_LAUNCH(name, stream, expr)                                                             \
    do {                                                                                            \
        ++g_launches;                                                                               \
        cudaEvent_t _e0 = nullptr, _e1 = nullptr;                                                   \
        bool _prof;                                                                                 \
        {                                                                                           \
            std::lock_guard<std::mutex> _l(g_prof_mu);                                              \
            _prof = g_prof_on;                                                                      \
            if (_prof) {                                                                            \
                _e0 = prof_event();                                                                 \
                _e1 = prof_event();                                                                 \
            }                                                                                       \
        }                                                                                           \
        if (_prof) cudaEventRecord(_e0, (stream));                                                  \
        nvtxRangePushA(name); /* host-side range per stage, seen by NVTX-aware profilers */       \
        cudaError_t _e = (expr);                                                                    \
        nvtxRangePop();                                                                             \
        if (_prof) {                                                                                \
            cudaEventRecord(_e1, (stream));                                                         \
            std::lock_guard<std::mutex> _l(g_prof_mu);                                              \
            g_prof_recs.push_back(ProfRec{(name), _e0, _e1});                                       \
        }                                                                                           \
        if (_e != cudaSuccess) return fail(MDFS_ECUDA, "%s: %s", #expr, cudaGetErrorString(_e));     \
    } while (0)

#define MDFS_ENSURE(ws, buf, bytes)                                                                 \
    do {                                                                                            \
        if (!(ws)->ensure((ws)->buf, (bytes)))                                                      \
            return fail(MDFS_ENOMEM, "device allocation of %zu bytes failed", (size_t)(bytes));      \
    } while (0)

// k = 5 limits: two classes per variable, class sizes that fit the packed
// 16-bit counters, partner ranks below 2^32 (C(M,4) < 2^32), and for the
// single-word keys of the sharded scan d C(M,4) + rank below 2^32.
unsigned long long binom4(int M) {
    const unsigned long long m = (unsigned long long)M;
    return M < 4 ? 0ull : m * (m - 1) / 2 * (m - 2) / 3 * (m - 3) / 4;
}
int check_k5(int M, int c, int D, int N, bool single_key = false) {
    if (c != 2 && !kgen_supported(5, c))
        return fail(MDFS_EINVAL, "k = 5 supports two to four classes per variable (divisions 1 .. 3)");
    // the scan of three or more classes keeps one key word: d C(M,4) + rank
    if (c != 2) single_key = true;
    if (N > 65535) return fail(MDFS_EINVAL, "k = 5 supports N up to 65535 samples");
    if (binom4(M) >= (1ull << 32)) return fail(MDFS_EINVAL, "C(M, 4) must stay below 2^32 for k = 5");
    if (single_key && (unsigned long long)D * binom4(M) >= (1ull << 32))
        return fail(MDFS_EINVAL, "discretizations * C(M, 4) must stay below 2^32 for the keys of a k = 5 shard");
    return MDFS_OK;
}

// Arguments shared by every scan entry point (k, M variables, divisions, N,
// discretizations, range, pc_xi) and the index limits of each k's argmax key;
// shard_keys: the single-word keys of mdfs_max_ig_shard (k = 5 limit).
int check_scan_args(int k, int M, int divisions, int N, int D, double range, double pc_xi, bool shard_keys = false) {
    const int c = divisions + 1;
    int rc = 0;
    if (k < 1 || k > 5) return fail(MDFS_EINVAL, "k = %d outside [1, 5]", k);
    if (M < k) return fail(MDFS_EINVAL, "M = %d smaller than k = %d", M, k);
    if (divisions < 1 || c > kMaxC) return fail(MDFS_EINVAL, "divisions = %d outside [1, %d]", divisions, kMaxC - 1);
    if (N < c) return fail(MDFS_EINVAL, "N = %d smaller than the number of classes %d", N, c);
    if (D < 1 || D > kMaxD) return fail(MDFS_EINVAL, "discretizations = %d outside [1, %d]", D, kMaxD);
    if (!(range >= 0.0 && range <= 1.0)) return fail(MDFS_EINVAL, "range must lie in [0, 1]");
    if (!(pc_xi > 0.0 && pc_xi < 1.0)) return fail(MDFS_EINVAL, "pc_xi must lie in (0, 1)");
    const unsigned long long m = (unsigned long long)M, d = (unsigned long long)D;
    if (k == 2 && d * m >= (1ull << 32)) return fail(MDFS_EINVAL, "discretizations * M too large");
    if (k == 3 && d * m * m >= (1ull << 32))
        return fail(MDFS_EINVAL, "discretizations * M^2 must stay below 2^32 for k = 3");
    if (k == 4 && c != 2 && !kgen_supported(4, c))
        return fail(MDFS_EINVAL, "k = 4 supports two to four classes per variable (divisions 1 .. 3)");
    if (k == 4 && d * m * m * m >= (1ull << 32))
        return fail(MDFS_EINVAL, "discretizations * M^3 must stay below 2^32 for k = 4");
    if (k == 5 && (rc = check_k5(M, c, D, N, shard_keys))) return rc;
    return MDFS_OK;
}

// discretisation of each key when the k = 5 scan kept per-discretisation keys
const int* wide_disc(const Workspace* ws) { return ws->k5_wide ? (const int*)ws->kdisc.p : nullptr; }

int check_data(const mdfs_data* data, bool need_y) {
    if (!data) return fail(MDFS_EINVAL, "data is NULL");
    if (data->dtype != MDFS_F32 && data->dtype != MDFS_I8) return fail(MDFS_EINVAL, "dtype must be MDFS_F32 or MDFS_I8");
    if (!data->x) return fail(MDFS_EINVAL, "x is NULL");
    if (need_y && !data->y) return fail(MDFS_EINVAL, "y is NULL");
    if (data->N < 2 || data->N > kMaxN) return fail(MDFS_EINVAL, "N = %d outside [2, %d]", data->N, kMaxN);
    if (data->M < 1 || data->M > 65535) return fail(MDFS_EINVAL, "M = %d outside [1, 65535]", data->M);
    return MDFS_OK;
}

// Stages x (and y) on the device and runs the validation kernels.  On success
// *n1 is the number of class-1 objects and ws->perm holds the class-sorted order.
int stage_inputs(Workspace* ws, const mdfs_data* data, bool need_y, const void** xd, const uint8_t** yd, int* n1) {
    cudaStream_t st = ws->stream;
    const size_t xbytes = (size_t)data->M * data->N * (data->dtype == MDFS_F32 ? 4 : 1);
    *xd = data->x;
    if (!is_device_ptr(data->x)) {
        MDFS_ENSURE(ws, x, xbytes);
        MDFS_CUDA_TRY(cudaMemcpyAsync(ws->x.p, data->x, xbytes, cudaMemcpyHostToDevice, st));
        *xd = ws->x.p;
    }
    MDFS_ENSURE(ws, stats, 16 * sizeof(int));
    MDFS_CUDA_TRY(cudaMemsetAsync(ws->stats.p, 0, 16 * sizeof(int), st));
    int* stats = (int*)ws->stats.p;
    if (need_y) {
        *yd = data->y;
        if (!is_device_ptr(data->y)) {
            MDFS_ENSURE(ws, y, (size_t)data->N);
            MDFS_CUDA_TRY(cudaMemcpyAsync(ws->y.p, data->y, (size_t)data->N, cudaMemcpyHostToDevice, st));
            *yd = (const uint8_t*)ws->y.p;
        }
        MDFS_ENSURE(ws, perm, (size_t)data->N * sizeof(int));
        MDFS_LAUNCH("stats", st, launch_stats(*yd, data->N, stats, (int*)ws->perm.p, st));
    }
    if (data->dtype == MDFS_F32)
        MDFS_LAUNCH("check_finite", st, launch_check_finite((const float*)*xd, (long long)data->M * data->N, stats + 2, st));
    MDFS_CUDA_TRY(cudaMemcpyAsync(ws->host_stats, stats, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    MDFS_CUDA_TRY(cudaStreamSynchronize(st));
    const int* hs = ws->host_stats;
    if (hs[2] != 0) return fail(MDFS_ENONFINITE, "x holds NaN or Inf values");
    if (need_y) {
        if (hs[1] != 0) return fail(MDFS_EINVAL, "y holds %d values outside {0, 1}", hs[1]);
        *n1 = hs[0];
        if (*n1 == 0 || *n1 == data->N)
            return fail(MDFS_EDEGENERATE, "decision has a single class (N0 = %d, N1 = %d)", data->N - *n1, *n1);
    }
    return MDFS_OK;
}

// Output target: the caller's device pointer, or a staging buffer copied back later.
template <typename T>
struct Out {
    T* user = nullptr;
    T* dev = nullptr;
    size_t bytes = 0;
    bool staged = false;
};

template <typename T>
int bind_out(Workspace* ws, Buffer& buf, T* user, size_t count, Out<T>* o) {
    o->user = user;
    o->bytes = count * sizeof(T);
    if (!user) return MDFS_OK;
    if (is_device_ptr(user)) {
        o->dev = user;
        return MDFS_OK;
    }
    if (!ws->ensure(buf, o->bytes)) return fail(MDFS_ENOMEM, "device allocation of %zu bytes failed", o->bytes);
    o->dev = (T*)buf.p;
    o->staged = true;
    return MDFS_OK;
}

template <typename T>
int copy_back(Workspace* ws, const Out<T>& o) {
    if (o.staged) MDFS_CUDA_TRY(cudaMemcpyAsync(o.user, o.dev, o.bytes, cudaMemcpyDeviceToHost, ws->stream));
    return MDFS_OK;
}

// Copies `count` elements of a device array to a caller pointer (host or device).
template <typename T>
int emit(Workspace* ws, const T* dev, T* user, size_t count) {
    if (!user || count == 0) return MDFS_OK;
    MDFS_CUDA_TRY(cudaMemcpyAsync(user, dev, count * sizeof(T),
                                  is_device_ptr(user) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ws->stream));
    return MDFS_OK;
}

void build_k3_items(int M, int c, std::vector<int2>& items) {
    const int TB = k3_tile_b(c), TE = k3_tile_e(c);
    items.clear();
    for (int a = 0; a + 2 < M; ++a) {
        const int L = M - 1 - a;
        const int nbt = (L + TB - 1) / TB, net = (L + TE - 1) / TE;
        for (int tb = 0; tb < nbt; ++tb) {
            const int bmin = a + 1 + tb * TB;
            if (bmin > M - 2) break;
            for (int te = 0; te < net; ++te) {
                const int emin = a + 1 + te * TE;
                if (emin > M - 1) break;
                const int emax = std::min(emin + TE - 1, M - 1);
                if (emax <= bmin) continue;
                items.push_back(make_int2(a, (tb << 16) | te));
            }
        }
    }
}

// The scan of one job whose x and y are on the device and validated (ws->perm
// holds the class-stable order, n1 the class-1 count): entropy tables,
// discretisation and the counting kernels.  Leaves the packed max keys in ws->keys.
// shard / n_shards: this call folds only its share of the tuple tiles into the
// keys (tensor-core and generic triple paths); the popcount pair path and k = 1
// run whole on shard 0.  Merging the keys of all shards by maximum gives the
// keys of the unsharded scan.
// emit != NULL: interesting-tuple emission into that table (the tensor-core kernels
// emit as the popcount kernels do).
// ---- launch-parameter tuner -------------------------------------------------
// The tunable launch parameter of the k = 2 tensor-core kernel (its pipeline
// stages, which also set how many batch jobs one launch can hold) is chosen per
// shape by timing the candidates on the first call that needs it.  Each
// candidate runs the real scan: the max keys are idempotent, so running it
// more than once leaves the same result.  The choice is kept in memory and,
// when the environment variable MDFS_TUNE_FILE names a file, appended there as
// "<kernel> M=.. N=.. c=.. D=.. -> <choice>" lines that later processes read
// back.  MDFS_TUNE=0 skips the measurement (the deepest pipeline that fits).
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

std::string tune_key(const char* kernel, int M, int N, int c, int D) {
    char b[128];
    snprintf(b, sizeof b, "%s M=%d N=%d c=%d D=%d", kernel, M, N, c, D);
    return b;
}

int tune_get(const std::string& key) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (!g_tune_loaded) {
        g_tune_loaded = true;
        if (const char* f = getenv("MDFS_TUNE_FILE")) {
            if (FILE* fp = fopen(f, "r")) {
                char line[256];
                while (fgets(line, sizeof line, fp)) {
                    char* arrow = strstr(line, " -> ");
                    if (!arrow) continue;
                    *arrow = 0;
                    const int v = atoi(arrow + 4);
                    if (v > 0) g_tune[line] = v;
                }
                fclose(fp);
            }
        }
    }
    auto it = g_tune.find(key);
    return it == g_tune.end() ? 0 : it->second;
}

void tune_put(const std::string& key, int v) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = v;
    if (const char* f = getenv("MDFS_TUNE_FILE")) {
        if (FILE* fp = fopen(f, "a")) {
            fprintf(fp, "%s -> %d\n", key.c_str(), v);
            fclose(fp);
        }
    }
}

// The tuned stage count of the k = 2 tensor-core launch of `jobs` (0 on a CUDA
// error); `kernel` names the cache entry (single scans and batches apart).
int tuned_k2_stages(Workspace* ws, const char* kernel, const K2Jobs& jobs, int M, int c, int D, const int2* items,
                    int n_items, const uint8_t* oh, int Kp, int zdim, int fbits, bool bound) {
    const int N = jobs.job[0].tg.N0 + jobs.job[0].tg.N1;
    const std::string key = tune_key(kernel, M, N, c, D);
    // a cached choice that does not fit this launch is measured again
    if (const int v = tune_get(key))
        if ((v == 3 || v == 4) && k2tc_smem_bytes(c, N, jobs.n, v) <= kK3tcMaxSmem) return v;
    int n_fit = 0, deepest = 0;
    for (const int stages : {4, 3})
        if (k2tc_smem_bytes(c, N, jobs.n, stages) <= kK3tcMaxSmem) {
            ++n_fit;
            if (!deepest) deepest = stages;
        }
    if (n_fit == 0) return 0;
    if (n_fit == 1) {  // nothing to choose between
        tune_put(key, deepest);
        return deepest;
    }
    const char* en = getenv("MDFS_TUNE");
    if (en && en[0] == '0') return deepest;
    cudaStream_t st = ws->stream;
    // a stream being captured into a graph cannot be timed: untuned default
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (cap != cudaStreamCaptureStatusNone) return deepest;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return 0;
    }
    // each candidate twice, alternating, best time of each (the first launch
    // also warms the caches); the keys are maxima, so the repeats leave them as
    // one launch would
    float best_ms[5] = {0, 0, 0, 0, 0};
    bool ok = true;
    for (int rep = 0; rep < 2 && ok; ++rep) {
        for (const int stages : {4, 3}) {
            if (k2tc_smem_bytes(c, N, jobs.n, stages) > kK3tcMaxSmem) continue;
            float ms = 0.0f;
            if (cudaEventRecord(e0, st) != cudaSuccess ||
                launch_k2tc(oh, Kp, zdim, jobs, M, c, 0, D, D, items, n_items, fbits, (int*)ws->err.p, bound, stages,
                            st) !=
                    cudaSuccess ||
                cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                cudaGetLastError();
                ok = false;
                break;
            }
            if (best_ms[stages] == 0.0f || ms < best_ms[stages]) best_ms[stages] = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) return 0;
    int best = 0;
    for (const int stages : {4, 3})
        if (best_ms[stages] > 0.0f && (!best || best_ms[stages] < best_ms[best])) best = stages;
    if (best) tune_put(key, best);
    return best;
}

// Whether the tensor-core kernels serve k = 2 (two or three classes) and k = 3
// (two classes): their fixed-point tables must fit shared memory, and the class
// sizes their counters hold.
bool tc2_applies(int c, int N, int n0, int n1) {
    return k2tc_supported(c) && k2tc_counts_fit(c, n0, n1) && k2tc_smem_bytes(c, N, 1, 3) <= kK3tcMaxSmem;
}
bool tc3_applies(int c, int n0, int n1) { return c == 2 && k3tc_smem_bytes(n0, n1) != (size_t)-1; }
// a k = 2 and a k = 3 scan of the same data can share one discretisation and its one-hot rows
bool fused_k23_applies(int c, int N, int n0, int n1) { return tc3_applies(c, n0, n1) && tc2_applies(c, N, n0, n1); }

// dump != NULL (test hook, mdfs_testing_counts): the tensor-core kernel also
// writes its class counts there; the call fails if that kernel does not apply.
// keep_err: leave the tensor-core error flag as it is (a batch clears it once
// and reads it after its last job).  keys1x != NULL: also the k = 1 keys of the
// same discretisation there.  keys2x != NULL (k = 3 on the tensor-core path
// with a k = 2 tensor-core scan that applies, fused_k23_applies): also the k = 2
// keys, from the same one-hot rows.
int scan_core(Workspace* ws, const void* xd, int dtype, int N, int M, int n1, int k, int divisions, int D, double range,
              double pc_xi, uint64_t seed, bool* check_err, int shard = 0, int n_shards = 1,
              const EmitTable* emit = nullptr, uint32_t* dump = nullptr, bool keep_err = false,
              unsigned long long* keys1x = nullptr, unsigned long long* keys2x = nullptr) {
    cudaStream_t st = ws->stream;
    auto share = [&](int n, int* lo) {
        *lo = (int)((long long)n * shard / n_shards);
        return (int)((long long)n * (shard + 1) / n_shards) - *lo;
    };
    const int c = divisions + 1;
    *check_err = false;
    const int n0 = N - n1;
    const double mn = (double)(n0 < n1 ? n0 : n1);
    const double b0 = pc_xi * n0 / mn, b1 = pc_xi * n1 / mn;
    const PlaneGeom g = make_geom(N, n0);
    const int P = c - 1;

    MDFS_ENSURE(ws, tab, (size_t)3 * (N + 1) * sizeof(long long));
    MDFS_ENSURE(ws, planes, (size_t)D * M * P * g.Ws * sizeof(uint32_t));
    MDFS_ENSURE(ws, cnt1, (size_t)D * M * P * 2 * sizeof(int));
    MDFS_ENSURE(ws, sh1, (size_t)D * M * sizeof(long long));
    MDFS_ENSURE(ws, keys, (size_t)M * sizeof(unsigned long long));
    long long* tab = (long long*)ws->tab.p;
    uint32_t* planes = (uint32_t*)ws->planes.p;
    int* cnt1 = (int*)ws->cnt1.p;
    long long* sh1 = (long long*)ws->sh1.p;
    unsigned long long* keys = (unsigned long long*)ws->keys.p;

    ws->k5_wide = false;
    MDFS_LAUNCH("ftable", st, launch_ftable(N, b0, b1, tab, st));
    const long long* tabw = nullptr;  // wide-layout tables of the packed-count kernels (k = 4, 5)
    if (k >= 4) {
        MDFS_ENSURE(ws, tabw, (size_t)kWideTab * sizeof(long long));
        MDFS_LAUNCH("ftable_wide", st, launch_ftable_wide(b0, b1, (long long*)ws->tabw.p, st));
        tabw = (const long long*)ws->tabw.p;
    }
    // tensor-core paths: k = 2 for two or three classes, k = 3 for two classes,
    // when their fixed-point tables fit in shared memory
    const EmitTable em = emit ? *emit : EmitTable();
    const bool use_tc2 = k == 2 && tc2_applies(c, N, n0, n1);
    const bool use_tc3 = k == 3 && tc3_applies(c, n0, n1);
    if (keys2x && !(use_tc3 && tc2_applies(c, N, n0, n1) && shard == 0 && n_shards == 1 && !emit && !dump))
        return fail(MDFS_EINVAL, "internal: the fused k = 2, 3 scan does not apply");
    TcGeom tg = make_tc_geom(n0, n1);
    if (dump && !use_tc2 && !use_tc3)
        return fail(MDFS_EINVAL, "no tensor-core kernel serves k = %d, %d classes, N0 = %d, N1 = %d", k, c, n0, n1);
    uint8_t* onehot = nullptr;
    if (use_tc2 || use_tc3) {
        MDFS_ENSURE(ws, onehot, (size_t)D * M * P * tg.Kp);
        onehot = (uint8_t*)ws->onehot.p;
    }
    MDFS_LAUNCH("discretize", st, launch_discretize(xd, dtype, N, M, c, D, range, seed, (const int*)ws->perm.p, g,
                                                    planes, nullptr, nullptr, onehot, tg, st,
                                                    use_tc2 ? k2tc_class1_byte(c) : 0x38u));
    MDFS_CUDA_TRY(cudaMemsetAsync(keys, 0, (size_t)M * sizeof(unsigned long long), st));
    if (keys1x) MDFS_CUDA_TRY(cudaMemsetAsync(keys1x, 0, (size_t)M * sizeof(unsigned long long), st));
    if (keys2x) MDFS_CUDA_TRY(cudaMemsetAsync(keys2x, 0, (size_t)M * sizeof(unsigned long long), st));
    MDFS_LAUNCH("k1", st, launch_k1(planes, g, M, c, D, tab, cnt1, sh1, (k == 1 && shard == 0) ? keys : keys1x, st,
                                    k == 1 ? em : EmitTable()));
    // the k = 2 tensor-core scan of the one-hot rows into kout (a k = 2 call, or
    // the k = 2 part of a fused k = 2, 3 call, which clears the error flag once)
    auto run_tc2 = [&](unsigned long long* kout, bool clear_err) -> int {
        MDFS_ENSURE(ws, err, sizeof(int));
        if (clear_err) MDFS_CUDA_TRY(cudaMemsetAsync(ws->err.p, 0, sizeof(int), st));
        if (ws->items3_M != M || ws->items3_c != c) {
            std::vector<int2> items;
            build_k2tc_items(M, c, items);
            MDFS_ENSURE(ws, items3, items.size() * sizeof(int2));
            MDFS_CUDA_TRY(cudaMemcpyAsync(ws->items3.p, items.data(), items.size() * sizeof(int2),
                                          cudaMemcpyHostToDevice, st));
            MDFS_CUDA_TRY(cudaStreamSynchronize(st));  // `items` is a pageable host vector
            ws->items3_M = M;
            ws->items3_c = c;
            ws->n_items3 = (int)items.size();
        }
        int lo = 0;
        const int cnt = share(ws->n_items3, &lo);
        const bool exact = take_test_hooks(false).exact;
        K2Jobs jobs{};
        jobs.n = 1;
        jobs.job[0] = K2Job{tg, tab, cnt1, sh1, kout, (float)b0, (float)b1};
        // the count test hook and emission run the deepest pipeline that fits (no tuning runs)
        const int stages = (dump || emit) ? (k2tc_smem_bytes(c, N, 1, 4) <= kK3tcMaxSmem ? 4 : 3)
                                          : tuned_k2_stages(ws, "k2tc_stages", jobs, M, c, D,
                                                            (const int2*)ws->items3.p + lo, cnt, onehot, tg.Kp, D,
                                                            k3tc_fraction_bits(N), !exact);
        if (stages <= 0) return fail(MDFS_ECUDA, "k = 2 stage tuning failed (CUDA error)");
        MDFS_LAUNCH("k2", st, launch_k2tc(onehot, tg.Kp, D, jobs, M, c, 0, D, D, (const int2*)ws->items3.p + lo, cnt,
                                          k3tc_fraction_bits(N), (int*)ws->err.p, !exact, stages, st, dump, em));
        *check_err = true;
        return MDFS_OK;
    };
    if (use_tc2) {
        const int rc2 = run_tc2(keys, !keep_err);
        if (rc2) return rc2;
    } else if (k == 2) {
        if (shard == 0)
            MDFS_LAUNCH("k2", st, launch_k2(planes, g, M, c, D, 0, D, tab, cnt1, sh1, keys, nullptr, nullptr, nullptr, 0, st,
                                            nullptr, em));
    } else if (use_tc3) {
        // two classes: symmetric 8-byte pair records and the tcgen05 triple kernel
        const size_t per_disc = (size_t)M * M * sizeof(PairC);
        const int fbits = k3tc_fraction_bits(N);
        size_t budget = (size_t)4 << 30;
        if (const char* env = getenv("MDFS_PAIR_TABLE_BYTES")) budget = (size_t)strtoull(env, nullptr, 10);
        int nd = (int)(budget / per_disc);
        if (nd < 1) nd = 1;
        if (nd > D) nd = D;
        MDFS_ENSURE(ws, pairs2, (size_t)nd * per_disc);
        MDFS_ENSURE(ws, err, sizeof(int));
        if (!keep_err) MDFS_CUDA_TRY(cudaMemsetAsync(ws->err.p, 0, sizeof(int), st));
        if (ws->items2_M != M) {
            std::vector<int2>& items = ws->items2_host;
            build_k3tc_items(M, items);
            MDFS_ENSURE(ws, items2, items.size() * sizeof(int2));
            MDFS_CUDA_TRY(cudaMemcpyAsync(ws->items2.p, items.data(), items.size() * sizeof(int2),
                                          cudaMemcpyHostToDevice, st));
            MDFS_CUDA_TRY(cudaStreamSynchronize(st));  // `items` is a pageable host vector
            ws->items2_M = M;
            ws->n_items2 = (int)items.size();
        }
        // relabel the variables of every discretisation by bin-1 count and
        // store the one-hot rows in that order (class-1 samples weighted 64)
        MDFS_ENSURE(ws, lperm, (size_t)D * M * sizeof(int));
        MDFS_ENSURE(ws, lrank, (size_t)D * M * sizeof(int));
        MDFS_ENSURE(ws, cnt1s, (size_t)D * M * 2 * sizeof(int));
        MDFS_ENSURE(ws, onehot2, (size_t)D * M * tg.Kp);
        const int* lperm = (const int*)ws->lperm.p;
        MDFS_LAUNCH("k3_order", st, launch_k3tc_order(cnt1, M, D, (int*)ws->lperm.p, (int*)ws->lrank.p,
                                                      (int*)ws->cnt1s.p, st));
        MDFS_LAUNCH("k3_operand", st, launch_k3tc_operand(onehot, (uint8_t*)ws->onehot2.p, lperm, M, D, tg, st));
        CUtensorMap map;
        MDFS_CUDA_TRY(make_onehot_map(&map, (const uint8_t*)ws->onehot2.p, M, D, tg.Kp));
        const TcTestHooks hooks = take_test_hooks(true);
        for (int d0 = 0; d0 < D; d0 += nd) {
            const int nn = std::min(nd, D - d0);
            MDFS_LAUNCH("k2_tables", st, launch_k2(planes, g, M, c, D, d0, nn, tab, cnt1, sh1, nullptr, nullptr,
                                                   nullptr, (PairC*)ws->pairs2.p, fbits, st, (const int*)ws->lrank.p));
            int lo = 0;
            const int cnt = share(ws->n_items2, &lo);
            // the tiles' claim order for this launch shape, built once and kept (two shapes)
            const int* order = nullptr;
            if (cnt > 0) {
                const long long key[4] = {M, lo, cnt, nn};
                int slot = -1;
                for (int e = 0; e < 2; ++e)
                    if (std::equal(key, key + 4, ws->k3sched_key[e])) slot = e;
                if (slot < 0) {
                    slot = ws->k3sched_next;
                    ws->k3sched_next ^= 1;
                    ws->k3sched_key[slot][0] = -1;
                    std::vector<int> sv;
                    build_k3tc_order(M, ws->items2_host.data() + lo, cnt, nn, sv);
                    MDFS_ENSURE(ws, k3sched[slot], sv.size() * sizeof(int));
                    MDFS_CUDA_TRY(cudaMemcpyAsync(ws->k3sched[slot].p, sv.data(), sv.size() * sizeof(int),
                                                  cudaMemcpyHostToDevice, st));
                    MDFS_CUDA_TRY(cudaStreamSynchronize(st));  // `sv` is a pageable host vector
                    std::copy(key, key + 4, ws->k3sched_key[slot]);
                }
                order = (const int*)ws->k3sched[slot].p;
            }
            MDFS_ENSURE(ws, k3claim, sizeof(int));
            if (keys2x && d0 == 0) {  // the k = 2 keys of the fused call, once
                const int rc2 = run_tc2(keys2x, false);
                if (rc2) return rc2;
            }
            MDFS_LAUNCH("k3", st, launch_k3tc(map, (const uint8_t*)ws->onehot2.p, tg, M, d0, nn,
                                              (const int2*)ws->items2.p + lo, cnt, tab, fbits, (const int*)ws->cnt1s.p,
                                              lperm, (const PairC*)ws->pairs2.p, keys, (int*)ws->err.p, b0, b1, st,
                                              dump, hooks, em, order, (int*)ws->k3claim.p));
        }
        *check_err = true;
    } else if (k == 3) {
        const size_t per_disc = (size_t)M * M * (sizeof(long long) + (size_t)P * P * 2 * sizeof(int));
        size_t budget = (size_t)4 << 30;
        if (const char* env = getenv("MDFS_PAIR_TABLE_BYTES")) budget = (size_t)strtoull(env, nullptr, 10);
        int nd = (int)(budget / per_disc);
        if (nd < 1) nd = 1;
        if (nd > D) nd = D;
        MDFS_ENSURE(ws, sh2, (size_t)nd * M * M * sizeof(long long));
        MDFS_ENSURE(ws, cnt2, (size_t)nd * M * M * P * P * 2 * sizeof(int));
        if (ws->items_M != M || ws->items_c != c) {
            std::vector<int2> items;
            build_k3_items(M, c, items);
            MDFS_ENSURE(ws, items, items.size() * sizeof(int2));
            MDFS_CUDA_TRY(cudaMemcpyAsync(ws->items.p, items.data(), items.size() * sizeof(int2),
                                          cudaMemcpyHostToDevice, st));
            MDFS_CUDA_TRY(cudaStreamSynchronize(st));  // `items` is a pageable host vector
            ws->items_M = M;
            ws->items_c = c;
            ws->n_items = (int)items.size();
        }
        for (int d0 = 0; d0 < D; d0 += nd) {
            const int nn = std::min(nd, D - d0);
            MDFS_LAUNCH("k2_tables", st, launch_k2(planes, g, M, c, D, d0, nn, tab, cnt1, sh1, nullptr,
                                                   (long long*)ws->sh2.p, (int*)ws->cnt2.p, nullptr, 0, st));
            int lo = 0;
            const int cnt = share(ws->n_items, &lo);
            MDFS_LAUNCH("k3", st, launch_k3_items(planes, g, M, c, d0, nn, (const int2*)ws->items.p + lo, cnt, tab,
                                                  cnt1, (const long long*)ws->sh2.p, (const int*)ws->cnt2.p, keys, st,
                                                  em));
        }
    } else if ((k == 4 || k == 5) && c != 2) {
        // three or four classes: every voxel of every tuple from the bit planes
        if (ws->itemsg_M != M || ws->itemsg_k != k) {
            std::vector<int2> items;
            build_kgen_items(M, k, items);
            MDFS_ENSURE(ws, itemsg, std::max<size_t>(items.size(), 1) * sizeof(int2));
            if (!items.empty())
                MDFS_CUDA_TRY(cudaMemcpyAsync(ws->itemsg.p, items.data(), items.size() * sizeof(int2),
                                              cudaMemcpyHostToDevice, st));
            MDFS_CUDA_TRY(cudaStreamSynchronize(st));  // `items` is a pageable host vector
            ws->itemsg_M = M;
            ws->itemsg_k = k;
            ws->n_itemsg = (int)items.size();
        }
        int lo = 0;
        const int cnt = share(ws->n_itemsg, &lo);
        for (int d0 = 0; d0 < D; d0 += 65535) {
            const int nn = std::min(65535, D - d0);
            MDFS_LAUNCH(k == 4 ? "k4" : "k5", st, launch_kgen(planes, g, M, c, k, d0, nn,
                                                              (const int2*)ws->itemsg.p + lo, cnt, tab, keys, em, st));
        }
    } else if (k == 4) {
        // two classes: pair counts from the pair pass, triple tables, then the quadruple kernel
        const size_t n3 = t3_entries(M);
        const size_t per_disc = (size_t)M * M * (sizeof(long long) + 2 * sizeof(int)) +
                                n3 * (sizeof(uint32_t) + sizeof(long long));
        size_t budget = (size_t)4 << 30;
        if (const char* env = getenv("MDFS_PAIR_TABLE_BYTES")) budget = (size_t)strtoull(env, nullptr, 10);
        int nd = (int)(budget / per_disc);
        if (nd < 1) nd = 1;
        if (nd > D) nd = D;
        if (nd > 65535) nd = 65535;
        MDFS_ENSURE(ws, sh2, (size_t)nd * M * M * sizeof(long long));
        MDFS_ENSURE(ws, cnt2, (size_t)nd * M * M * 2 * sizeof(int));
        MDFS_ENSURE(ws, t3c, std::max<size_t>((size_t)nd * n3, 1) * sizeof(uint32_t));
        MDFS_ENSURE(ws, t3s, std::max<size_t>((size_t)nd * n3, 1) * sizeof(long long));
        if (ws->items3t_M != M) {
            std::vector<int2> items;
            build_t3_items(M, items);
            MDFS_ENSURE(ws, items3t, std::max<size_t>(items.size(), 1) * sizeof(int2));
            MDFS_CUDA_TRY(cudaMemcpyAsync(ws->items3t.p, items.data(), items.size() * sizeof(int2),
                                          cudaMemcpyHostToDevice, st));
            MDFS_CUDA_TRY(cudaStreamSynchronize(st));  // `items` is a pageable host vector
            ws->items3t_M = M;
            ws->n_items3t = (int)items.size();
        }
        if (ws->items4_M != M) {
            std::vector<int2> items;
            build_k4_items(M, items);
            MDFS_ENSURE(ws, items4, std::max<size_t>(items.size(), 1) * sizeof(int2));
            MDFS_CUDA_TRY(cudaMemcpyAsync(ws->items4.p, items.data(), items.size() * sizeof(int2),
                                          cudaMemcpyHostToDevice, st));
            MDFS_CUDA_TRY(cudaStreamSynchronize(st));  // `items` is a pageable host vector
            ws->items4_M = M;
            ws->n_items4 = (int)items.size();
        }
        for (int d0 = 0; d0 < D; d0 += nd) {
            const int nn = std::min(nd, D - d0);
            MDFS_LAUNCH("k2_tables", st, launch_k2(planes, g, M, c, D, d0, nn, tab, cnt1, sh1, nullptr,
                                                   (long long*)ws->sh2.p, (int*)ws->cnt2.p, nullptr, 0, st));
            MDFS_LAUNCH("t3", st, launch_t3(planes, g, M, d0, nn, (const int2*)ws->items3t.p, ws->n_items3t, tabw, cnt1,
                                            (const int*)ws->cnt2.p, (uint32_t*)ws->t3c.p, (long long*)ws->t3s.p,
                                            st));
            int lo = 0;
            const int cnt = share(ws->n_items4, &lo);
            MDFS_LAUNCH("k4", st, launch_k4(planes, g, M, d0, nn, (const int2*)ws->items4.p + lo, cnt, tabw, cnt1,
                                            (const int*)ws->cnt2.p, (const uint32_t*)ws->t3c.p,
                                            (const long long*)ws->t3s.p, keys, st, em));
        }
    } else if (k == 5) {
        // two classes: pair counts, triple tables, quadruple tables (counts and
        // entropies of all C(M,4) quadruples), then the quintuple kernel
        const size_t n3 = t3_entries(M), n4 = t4_entries(M);
        const size_t per_disc = (size_t)M * M * (sizeof(long long) + 2 * sizeof(int)) +
                                (n3 + n4) * (sizeof(uint32_t) + sizeof(long long));
        size_t budget = (size_t)4 << 30;
        if (const char* env = getenv("MDFS_PAIR_TABLE_BYTES")) budget = (size_t)strtoull(env, nullptr, 10);
        int nd = (int)(budget / per_disc);
        if (nd < 1) nd = 1;
        if (nd > D) nd = D;
        if (nd > 65535) nd = 65535;
        MDFS_ENSURE(ws, sh2, (size_t)nd * M * M * sizeof(long long));
        MDFS_ENSURE(ws, cnt2, (size_t)nd * M * M * 2 * sizeof(int));
        MDFS_ENSURE(ws, t3c, std::max<size_t>((size_t)nd * n3, 1) * sizeof(uint32_t));
        MDFS_ENSURE(ws, t3s, std::max<size_t>((size_t)nd * n3, 1) * sizeof(long long));
        MDFS_ENSURE(ws, t4c, std::max<size_t>((size_t)nd * n4, 1) * sizeof(uint32_t));
        MDFS_ENSURE(ws, t4s, std::max<size_t>((size_t)nd * n4, 1) * sizeof(long long));
        // one 64-bit key cannot hold d C(M,4) + rank: per-discretisation keys
        const bool wide = (unsigned long long)D * n4 >= (1ull << 32) || getenv("MDFS_K5_DISC_KEYS") != nullptr;
        ws->k5_wide = wide;
        if (wide) {
            MDFS_ENSURE(ws, keys5, (size_t)nd * M * sizeof(unsigned long long));
            MDFS_ENSURE(ws, kdisc, (size_t)M * sizeof(int));
            MDFS_CUDA_TRY(cudaMemsetAsync(ws->kdisc.p, 0, (size_t)M * sizeof(int), st));
        }
        const struct {
            Buffer* buf;
            int* m;
            int* n;
            void (*build)(int, std::vector<int2>&);
        } lists[3] = {{&ws->items3t, &ws->items3t_M, &ws->n_items3t, build_t3_items},
                      {&ws->items4, &ws->items4_M, &ws->n_items4, build_k4_items},
                      {&ws->items5, &ws->items5_M, &ws->n_items5, build_k5_items}};
        for (const auto& l : lists) {
            if (*l.m == M) continue;
            std::vector<int2> items;
            l.build(M, items);
            if (!ws->ensure(*l.buf, std::max<size_t>(items.size(), 1) * sizeof(int2)))
                return fail(MDFS_ENOMEM, "device allocation of %zu bytes failed", items.size() * sizeof(int2));
            MDFS_CUDA_TRY(cudaMemcpyAsync(l.buf->p, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
            MDFS_CUDA_TRY(cudaStreamSynchronize(st));  // `items` is a pageable host vector
            *l.m = M;
            *l.n = (int)items.size();
        }
        for (int d0 = 0; d0 < D; d0 += nd) {
            const int nn = std::min(nd, D - d0);
            MDFS_LAUNCH("k2_tables", st, launch_k2(planes, g, M, c, D, d0, nn, tab, cnt1, sh1, nullptr,
                                                   (long long*)ws->sh2.p, (int*)ws->cnt2.p, nullptr, 0, st));
            MDFS_LAUNCH("t3", st, launch_t3(planes, g, M, d0, nn, (const int2*)ws->items3t.p, ws->n_items3t, tabw, cnt1,
                                            (const int*)ws->cnt2.p, (uint32_t*)ws->t3c.p, (long long*)ws->t3s.p,
                                            st));
            MDFS_LAUNCH("t4", st, launch_t4(planes, g, M, d0, nn, (const int2*)ws->items4.p, ws->n_items4, tabw, cnt1,
                                            (const int*)ws->cnt2.p, (const uint32_t*)ws->t3c.p,
                                            (const long long*)ws->t3s.p, (uint32_t*)ws->t4c.p, (long long*)ws->t4s.p,
                                            st));
            int lo = 0;
            const int cnt = share(ws->n_items5, &lo);
            if (!wide) {
                MDFS_LAUNCH("k5", st, launch_k5(planes, g, M, d0, nn, (const int2*)ws->items5.p + lo, cnt, tabw, cnt1,
                                                (const int*)ws->cnt2.p, (const uint32_t*)ws->t3c.p,
                                                (const uint32_t*)ws->t4c.p, (const long long*)ws->t4s.p, keys, 0,
                                                true, st, em));
            } else {
                // keys of this chunk per discretisation (IG, partner rank), folded
                // into (keys, kdisc) in discretisation order
                unsigned long long* k5 = (unsigned long long*)ws->keys5.p;
                MDFS_CUDA_TRY(cudaMemsetAsync(k5, 0, (size_t)nn * M * sizeof(unsigned long long), st));
                MDFS_LAUNCH("k5", st, launch_k5(planes, g, M, d0, nn, (const int2*)ws->items5.p + lo, cnt, tabw, cnt1,
                                                (const int*)ws->cnt2.p, (const uint32_t*)ws->t3c.p,
                                                (const uint32_t*)ws->t4c.p, (const long long*)ws->t4s.p, k5, M,
                                                false, st, em));
                MDFS_LAUNCH("k5_merge", st, launch_k5_merge(k5, nn, M, d0, keys, (int*)ws->kdisc.p, st));
            }
        }
    }

    return MDFS_OK;
}

}  // namespace

namespace mdfs {
void record_error(const char* msg) { g_err = msg; }

cudaError_t ensure_dynamic_smem(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = limit[std::make_pair(kernel, dev)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}
}  // namespace mdfs

extern "C" {

int mdfs_abi_version(void) { return 1; }

const char* mdfs_last_error(void) { return g_err.c_str(); }

int mdfs_last_launch_count(void) { return g_launches; }

int mdfs_profile(int enable) {
    std::lock_guard<std::mutex> lock(g_prof_mu);
    g_prof_on = enable != 0;
    return MDFS_OK;
}

int mdfs_profile_report(char* buf, int len) {
    std::vector<ProfRec> recs;
    {
        std::lock_guard<std::mutex> lock(g_prof_mu);
        recs.swap(g_prof_recs);
    }
    std::vector<std::string> names;
    std::vector<double> ms;
    std::vector<int> cnt;
    int rc = MDFS_OK;
    for (const ProfRec& r : recs) {
        float t = 0.0f;
        if (cudaEventSynchronize(r.ev1) != cudaSuccess || cudaEventElapsedTime(&t, r.ev0, r.ev1) != cudaSuccess) {
            cudaGetLastError();
            rc = fail(MDFS_ECUDA, "profile event query failed");
            continue;
        }
        size_t j = 0;
        while (j < names.size() && names[j] != r.name) ++j;
        if (j == names.size()) {
            names.push_back(r.name);
            ms.push_back(0.0);
            cnt.push_back(0);
        }
        ms[j] += t;
        cnt[j] += 1;
    }
    {
        std::lock_guard<std::mutex> lock(g_prof_mu);
        for (const ProfRec& r : recs) {
            g_prof_pool.push_back(r.ev0);
            g_prof_pool.push_back(r.ev1);
        }
    }
    std::string out;
    char line[160];
    for (size_t j = 0; j < names.size(); ++j) {
        snprintf(line, sizeof line, "%s %d %.6f\n", names[j].c_str(), cnt[j], ms[j]);
        out += line;
    }
    if (buf && len > 0) {
        strncpy(buf, out.c_str(), (size_t)len - 1);
        buf[len - 1] = 0;
    }
    if (rc == MDFS_OK && (int)out.size() >= len) rc = fail(MDFS_EINVAL, "report truncated (%zu bytes)", out.size());
    return rc;
}

int mdfs_release_stream(void* stream) {
    g_err.clear();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(MDFS_ECUDA, "no CUDA device is available");
    }
    std::unique_ptr<Workspace> ws;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_ws.find(std::make_pair(dev, (cudaStream_t)stream));
        if (it == g_ws.end()) return MDFS_OK;
        ws = std::move(it->second);
        g_ws.erase(it);
    }
    // the workspace's buffers are freed here, outside the lock
    return MDFS_OK;
}

int mdfs_release(void) {
    {
        std::lock_guard<std::mutex> lock(g_mu);
        g_ws.clear();
    }
    noalloc_forget_devices();
    return MDFS_OK;
}

int mdfs_discretize(const mdfs_data* data, int divisions, int discretizations, double range, uint64_t seed,
                    uint8_t* codes, void* stream) {
    g_err.clear();
    g_launches = 0;
    int rc = check_data(data, false);
    if (rc) return rc;
    const int c = divisions + 1;
    if (divisions < 1 || c > kMaxC) return fail(MDFS_EINVAL, "divisions = %d outside [1, %d]", divisions, kMaxC - 1);
    if (data->N < c) return fail(MDFS_EINVAL, "N = %d smaller than the number of classes %d", data->N, c);
    if (discretizations < 1 || discretizations > kMaxD)
        return fail(MDFS_EINVAL, "discretizations = %d outside [1, %d]", discretizations, kMaxD);
    if (!(range >= 0.0 && range <= 1.0)) return fail(MDFS_EINVAL, "range must lie in [0, 1]");
    if (!codes) return fail(MDFS_EINVAL, "codes is NULL");
    if ((rc = check_devices({{data->x, "x"}, {codes, "codes"}}))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace* ws = get_ws(st, &rc);
    if (!ws) return rc;
    const void* xd = nullptr;
    const uint8_t* yd = nullptr;
    int n1 = 0;
    rc = stage_inputs(ws, data, false, &xd, &yd, &n1);
    if (rc) return rc;
    Out<uint8_t> oc;
    rc = bind_out(ws, ws->codes, codes, (size_t)discretizations * data->M * data->N, &oc);
    if (rc) return rc;
    PlaneGeom g = make_geom(data->N, data->N);
    MDFS_LAUNCH("discretize", st, launch_discretize(xd, data->dtype, data->N, data->M, c, discretizations, range, seed,
                                                    nullptr, g, nullptr, oc.dev, nullptr, nullptr, TcGeom{}, st));
    rc = copy_back(ws, oc);
    if (rc) return rc;
    if (oc.staged || st == nullptr) MDFS_CUDA_TRY(cudaStreamSynchronize(st));
    return MDFS_OK;
}

int mdfs_max_ig(const mdfs_data* data, int k, int divisions, int discretizations, double range, double pc_xi,
                uint64_t seed, float* ig, int32_t* tuples, int32_t* best_disc, void* stream) {
    g_err.clear();
    g_launches = 0;
    int rc = check_data(data, true);
    if (rc) return rc;
    const int N = data->N, M = data->M, D = discretizations;
    if ((rc = check_scan_args(k, M, divisions, N, D, range, pc_xi))) return rc;
    if (!ig) return fail(MDFS_EINVAL, "ig is NULL");

    if ((rc = check_devices({{data->x, "x"}, {data->y, "y"}, {ig, "ig"}, {tuples, "tuples"}, {best_disc, "best_disc"}}))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace* ws = get_ws(st, &rc);
    if (!ws) return rc;
    const void* xd = nullptr;
    const uint8_t* yd = nullptr;
    int n1 = 0;
    rc = stage_inputs(ws, data, true, &xd, &yd, &n1);
    if (rc) return rc;
    bool check_err = false;
    rc = scan_core(ws, xd, data->dtype, N, M, n1, k, divisions, D, range, pc_xi, seed, &check_err);
    if (rc) return rc;
    unsigned long long* keys = (unsigned long long*)ws->keys.p;

    Out<float> oig;
    Out<int32_t> otu, odi;
    rc = bind_out(ws, ws->ig, ig, (size_t)M, &oig);
    if (rc) return rc;
    rc = bind_out(ws, ws->tuples, k > 1 ? tuples : (int32_t*)nullptr, (size_t)M * (k > 1 ? k - 1 : 1), &otu);
    if (rc) return rc;
    rc = bind_out(ws, ws->disc, best_disc, (size_t)M, &odi);
    if (rc) return rc;
    MDFS_LAUNCH("finalize", st, launch_finalize(keys, M, k, oig.dev, otu.dev, odi.dev, st, wide_disc(ws)));
    if ((rc = copy_back(ws, oig)) || (rc = copy_back(ws, otu)) || (rc = copy_back(ws, odi))) return rc;
    if (check_err) {
        // the tensor-core kernel reports bounded-wait timeouts through this flag
        MDFS_CUDA_TRY(cudaMemcpyAsync(ws->host_stats + 8, ws->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        MDFS_CUDA_TRY(cudaStreamSynchronize(st));
        const int flag = ws->host_stats[8];
        if (flag) return kernel_flag_error(flag);
    } else if (oig.staged || otu.staged || odi.staged || st == nullptr) {
        MDFS_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return MDFS_OK;
}

int mdfs_max_ig_multi(const mdfs_data* data, int n_k, const int* ks, int divisions, int discretizations, double range,
                      double pc_xi, uint64_t seed, float* const* ig, int32_t* const* tuples, int32_t* const* best_disc,
                      void* stream) {
    g_err.clear();
    g_launches = 0;
    int rc = check_data(data, true);
    if (rc) return rc;
    const int N = data->N, M = data->M, D = discretizations, c = divisions + 1;
    if (n_k < 1 || n_k > 5 || !ks || !ig) return fail(MDFS_EINVAL, "n_k = %d outside [1, 5], or ks / ig NULL", n_k);
    int slot_of[6] = {-1, -1, -1, -1, -1, -1};  // output slot of each k
    for (int j = 0; j < n_k; ++j) {
        const int k = ks[j];
        if (k < 1 || k > 5) return fail(MDFS_EINVAL, "ks[%d] = %d outside [1, 5]", j, k);
        if (slot_of[k] >= 0) return fail(MDFS_EINVAL, "k = %d appears twice in ks", k);
        slot_of[k] = j;
        if ((rc = check_scan_args(k, M, divisions, N, D, range, pc_xi))) return rc;
        if (!ig[j]) return fail(MDFS_EINVAL, "ig[%d] is NULL", j);
    }
    for (int j = 0; j < n_k; ++j)
        if ((rc = check_devices({{data->x, "x"}, {data->y, "y"}, {ig[j], "ig"}, {tuples ? tuples[j] : nullptr, "tuples"},
                                 {best_disc ? best_disc[j] : nullptr, "best_disc"}})))
            return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace* ws = get_ws(st, &rc);
    if (!ws) return rc;
    const void* xd = nullptr;
    const uint8_t* yd = nullptr;
    int n1 = 0;
    rc = stage_inputs(ws, data, true, &xd, &yd, &n1);
    if (rc) return rc;
    // decodes keys of dimension k into output slot j (staged outputs copied back at once)
    bool any_staged = false;
    auto finish = [&](const unsigned long long* keys, int k) -> int {
        const int j = slot_of[k];
        Out<float> oig;
        Out<int32_t> otu, odi;
        int r = bind_out(ws, ws->ig, ig[j], (size_t)M, &oig);
        if (!r) r = bind_out(ws, ws->tuples, (k > 1 && tuples) ? tuples[j] : (int32_t*)nullptr,
                             (size_t)M * (k > 1 ? k - 1 : 1), &otu);
        if (!r) r = bind_out(ws, ws->disc, best_disc ? best_disc[j] : (int32_t*)nullptr, (size_t)M, &odi);
        if (r) return r;
        MDFS_LAUNCH("finalize", st, launch_finalize(keys, M, k, oig.dev, otu.dev, odi.dev, st, wide_disc(ws)));
        if ((r = copy_back(ws, oig)) || (r = copy_back(ws, otu)) || (r = copy_back(ws, odi))) return r;
        any_staged = any_staged || oig.staged || otu.staged || odi.staged;
        return MDFS_OK;
    };
    bool check_err = false, done[6] = {};
    // k = 1, 2 and 3 from one discretisation where the tensor-core kernels serve k = 2 and k = 3
    if (slot_of[3] >= 0 && (slot_of[1] >= 0 || slot_of[2] >= 0) && fused_k23_applies(c, N, N - n1, n1)) {
        MDFS_ENSURE(ws, mkeys, (size_t)2 * M * sizeof(unsigned long long));
        unsigned long long* k1x = slot_of[1] >= 0 ? (unsigned long long*)ws->mkeys.p : nullptr;
        unsigned long long* k2x = slot_of[2] >= 0 ? (unsigned long long*)ws->mkeys.p + M : nullptr;
        bool ce = false;
        rc = scan_core(ws, xd, data->dtype, N, M, n1, 3, divisions, D, range, pc_xi, seed, &ce, 0, 1, nullptr,
                       nullptr, false, k1x, k2x);
        if (rc) return rc;
        check_err = check_err || ce;
        if ((rc = finish((const unsigned long long*)ws->keys.p, 3))) return rc;
        if (k1x && (rc = finish(k1x, 1))) return rc;
        if (k2x && (rc = finish(k2x, 2))) return rc;
        done[1] = done[2] = done[3] = true;
    }
    for (int k = 1; k <= 5; ++k) {
        if (slot_of[k] < 0 || done[k]) continue;
        bool ce = false;
        // a later scan keeps the tensor-core error flag of an earlier one
        rc = scan_core(ws, xd, data->dtype, N, M, n1, k, divisions, D, range, pc_xi, seed, &ce, 0, 1, nullptr,
                       nullptr, check_err);
        if (rc) return rc;
        check_err = check_err || ce;
        if ((rc = finish((const unsigned long long*)ws->keys.p, k))) return rc;
    }
    if (check_err) {
        MDFS_CUDA_TRY(cudaMemcpyAsync(ws->host_stats + 8, ws->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        MDFS_CUDA_TRY(cudaStreamSynchronize(st));
        const int flag = ws->host_stats[8];
        if (flag) return kernel_flag_error(flag);
    } else if (any_staged || st == nullptr) {
        MDFS_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return MDFS_OK;
}

int mdfs_max_ig_batch(const mdfs_data* data, int n_jobs, const int32_t* sample_idx, const int32_t* y_perm, int k,
                      int divisions, int discretizations, double range, double pc_xi, uint64_t seed, float* ig,
                      int32_t* tuples, int32_t* best_disc, void* stream) {
    g_err.clear();
    g_launches = 0;
    int rc = check_data(data, true);
    if (rc) return rc;
    const int N = data->N, M = data->M, D = discretizations, c = divisions + 1, P = c - 1;
    if (n_jobs < 1) return fail(MDFS_EINVAL, "n_jobs = %d < 1", n_jobs);
    if ((rc = check_scan_args(k, M, divisions, N, D, range, pc_xi))) return rc;
    if (!ig) return fail(MDFS_EINVAL, "ig is NULL");
    if ((rc = check_devices({{data->x, "x"}, {data->y, "y"}, {sample_idx, "sample_idx"}, {y_perm, "y_perm"}, {ig, "ig"}, {tuples, "tuples"}, {best_disc, "best_disc"}}))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace* ws = get_ws(st, &rc);
    if (!ws) return rc;
    const void* xd = nullptr;
    const uint8_t* yd = nullptr;
    int n1_all = 0;
    // validates x (finite) and the labels of y; a y with one class stays one class in every job
    rc = stage_inputs(ws, data, true, &xd, &yd, &n1_all);
    if (rc) return rc;
    const size_t nidx = (size_t)n_jobs * N * sizeof(int32_t);
    const int32_t* idxd = sample_idx;
    if (sample_idx && !is_device_ptr(sample_idx)) {
        MDFS_ENSURE(ws, bidx, nidx);
        MDFS_CUDA_TRY(cudaMemcpyAsync(ws->bidx.p, sample_idx, nidx, cudaMemcpyHostToDevice, st));
        idxd = (const int32_t*)ws->bidx.p;
    }
    const int32_t* permd = y_perm;
    if (y_perm && !is_device_ptr(y_perm)) {
        MDFS_ENSURE(ws, bperm, nidx);
        MDFS_CUDA_TRY(cudaMemcpyAsync(ws->bperm.p, y_perm, nidx, cudaMemcpyHostToDevice, st));
        permd = (const int32_t*)ws->bperm.p;
    }
    // the class sizes of every job in one device pass and one read back: no
    // job waits for the host after this
    MDFS_ENSURE(ws, bcounts, (size_t)n_jobs * sizeof(int2));
    MDFS_LAUNCH("batch_counts", st, launch_batch_counts(yd, N, idxd, permd, n_jobs, (int2*)ws->bcounts.p, st));
    std::vector<int2> counts((size_t)n_jobs);
    MDFS_CUDA_TRY(cudaMemcpyAsync(counts.data(), ws->bcounts.p, (size_t)n_jobs * sizeof(int2), cudaMemcpyDeviceToHost,
                                  st));
    MDFS_CUDA_TRY(cudaStreamSynchronize(st));
    for (int j = 0; j < n_jobs; ++j) {
        if (counts[j].y) return fail(MDFS_EINVAL, "job %d: sample or permutation index outside [0, N)", j);
        if (counts[j].x == 0 || counts[j].x == N) return fail(MDFS_EDEGENERATE, "job %d: decision has a single class", j);
    }
    const size_t xbytes = (size_t)M * N * (data->dtype == MDFS_F32 ? 4 : 1);
    MDFS_ENSURE(ws, bx, xbytes);
    MDFS_ENSURE(ws, by, (size_t)N);
    Out<float> oig;
    Out<int32_t> otu, odi;
    const int kk = k > 1 ? k - 1 : 1;
    rc = bind_out(ws, ws->ig, ig, (size_t)n_jobs * M, &oig);
    if (rc) return rc;
    rc = bind_out(ws, ws->tuples, k > 1 ? tuples : (int32_t*)nullptr, (size_t)n_jobs * M * kk, &otu);
    if (rc) return rc;
    rc = bind_out(ws, ws->disc, best_disc, (size_t)n_jobs * M, &odi);
    if (rc) return rc;
    MDFS_ENSURE(ws, err, sizeof(int));
    MDFS_CUDA_TRY(cudaMemsetAsync(ws->err.p, 0, sizeof(int), st));
    int* stats = (int*)ws->stats.p;
    bool check_err = false;
    // k = 2 on the tensor cores: chunks of jobs share one launch over (job,
    // discretisation, tile) work items
    bool tc_fit = k == 2 && k2tc_supported(c) && k2tc_smem_bytes(c, N, 1, 3) <= kK3tcMaxSmem;
    for (int j = 0; j < n_jobs && tc_fit; ++j) tc_fit = k2tc_counts_fit(c, N - counts[j].x, counts[j].x);
    if (tc_fit) {
        int Kp_max = 0, Ws_max = 0;
        for (int j = 0; j < n_jobs; ++j) {
            Kp_max = std::max(Kp_max, make_tc_geom(N - counts[j].x, counts[j].x).Kp);
            Ws_max = std::max(Ws_max, make_geom(N, N - counts[j].x).Ws);
        }
        // jobs per launch: what the entropy tables in shared memory allow, and a
        // device-memory budget for the chunk's one-hot operands
        size_t budget = (size_t)8 << 30;
        if (const char* env = getenv("MDFS_BATCH_BYTES")) budget = (size_t)strtoull(env, nullptr, 10);
        const size_t op_bytes = (size_t)D * M * P * Kp_max;
        const int by_mem = (int)std::max<size_t>(1, budget / std::max<size_t>(op_bytes, 1));
        int stages = tune_get(tune_key("k2tc_batch_stages", M, N, c, D));
        if (stages != 3 && stages != 4) stages = 0;
        if (stages && k2tc_max_jobs(c, N, stages, kK3tcMaxSmem) < 1) stages = 0;  // a cached choice that cannot run
        // untuned: size the chunk for the deepest pipeline that holds a job
        const int cap_stages = stages ? stages : (k2tc_max_jobs(c, N, 4, kK3tcMaxSmem) > 0 ? 4 : 3);
        const int chunk_cap =
            std::min({n_jobs, by_mem, std::max(1, k2tc_max_jobs(c, N, cap_stages, kK3tcMaxSmem))});
        const size_t np1 = (size_t)N + 1;
        MDFS_ENSURE(ws, bonehot, (size_t)chunk_cap * op_bytes);
        MDFS_ENSURE(ws, btab, (size_t)chunk_cap * 3 * np1 * sizeof(long long));
        MDFS_ENSURE(ws, bcnt1, (size_t)chunk_cap * D * M * P * 2 * sizeof(int));
        MDFS_ENSURE(ws, bsh1, (size_t)chunk_cap * D * M * sizeof(long long));
        MDFS_ENSURE(ws, bkeys, (size_t)chunk_cap * M * sizeof(unsigned long long));
        MDFS_ENSURE(ws, planes, (size_t)D * M * P * Ws_max * sizeof(uint32_t));
        MDFS_ENSURE(ws, perm, (size_t)N * sizeof(int));
        if (ws->items3_M != M || ws->items3_c != c) {
            std::vector<int2> items;
            build_k2tc_items(M, c, items);
            MDFS_ENSURE(ws, items3, items.size() * sizeof(int2));
            MDFS_CUDA_TRY(cudaMemcpyAsync(ws->items3.p, items.data(), items.size() * sizeof(int2),
                                          cudaMemcpyHostToDevice, st));
            MDFS_CUDA_TRY(cudaStreamSynchronize(st));  // `items` is a pageable host vector
            ws->items3_M = M;
            ws->items3_c = c;
            ws->n_items3 = (int)items.size();
        }
        const int fbits = k3tc_fraction_bits(N);
        // every variable sorted once for all jobs; a job's thresholds then come from
        // the sorted keys and the job's sample multiplicities, without a sort
        const bool presorted = N <= kPresortMaxN;
        if (presorted) {
            MDFS_ENSURE(ws, bsorted, (size_t)M * N * sizeof(unsigned long long));
            MDFS_ENSURE(ws, bmult, (size_t)N * sizeof(int));
            MDFS_ENSURE(ws, bthr, (size_t)D * M * P * sizeof(float));
            MDFS_LAUNCH("presort", st, launch_presort(xd, data->dtype, N, M, (unsigned long long*)ws->bsorted.p, st));
        }
        for (int j0 = 0; j0 < n_jobs; j0 += chunk_cap) {
            const int nj = std::min(chunk_cap, n_jobs - j0);
            K2Jobs jobs{};
            jobs.n = nj;
            for (int jj = 0; jj < nj; ++jj) {
                const int j = j0 + jj, n1 = counts[j].x, n0 = N - n1;
                const double mn = (double)(n0 < n1 ? n0 : n1);
                const double b0 = pc_xi * n0 / mn, b1 = pc_xi * n1 / mn;
                MDFS_LAUNCH("gather", st, launch_gather_job(xd, data->dtype, yd, N, M, idxd ? idxd + (size_t)j * N : nullptr,
                                                            permd ? permd + (size_t)j * N : nullptr, ws->bx.p,
                                                            (uint8_t*)ws->by.p, stats + 3, st));
                MDFS_LAUNCH("stats", st, launch_stats((const uint8_t*)ws->by.p, N, stats, (int*)ws->perm.p, st));
                long long* tab = (long long*)ws->btab.p + (size_t)jj * 3 * np1;
                int* cnt1 = (int*)ws->bcnt1.p + (size_t)jj * D * M * P * 2;
                long long* sh1 = (long long*)ws->bsh1.p + (size_t)jj * D * M;
                unsigned long long* keys = (unsigned long long*)ws->bkeys.p + (size_t)jj * M;
                uint8_t* onehot = (uint8_t*)ws->bonehot.p + (size_t)jj * op_bytes;
                const TcGeom tg = make_tc_geom(n0, n1);
                TcGeom tgd = tg;  // the discretiser writes rows of the chunk's common length
                tgd.Kp = Kp_max;
                const PlaneGeom g = make_geom(N, n0);
                MDFS_LAUNCH("ftable", st, launch_ftable(N, b0, b1, tab, st));
                const float* thr_in = nullptr;
                if (presorted) {
                    const int* idx_j = idxd ? idxd + (size_t)j * N : nullptr;
                    MDFS_LAUNCH("multiplicity", st, launch_multiplicity(idx_j, N, (int*)ws->bmult.p, st));
                    MDFS_LAUNCH("thresholds", st,
                                launch_batch_thresholds((const unsigned long long*)ws->bsorted.p,
                                                        idx_j ? (const int*)ws->bmult.p : nullptr, N, M, c, D, range,
                                                        seed, (float*)ws->bthr.p, st));
                    thr_in = (const float*)ws->bthr.p;
                }
                MDFS_LAUNCH("discretize", st, launch_discretize(ws->bx.p, data->dtype, N, M, c, D, range, seed,
                                                                (const int*)ws->perm.p, g, (uint32_t*)ws->planes.p,
                                                                nullptr, nullptr, onehot, tgd, st, k2tc_class1_byte(c),
                                                                thr_in));
                MDFS_LAUNCH("k1", st, launch_k1((const uint32_t*)ws->planes.p, g, M, c, D, tab, cnt1, sh1, nullptr, st));
                MDFS_CUDA_TRY(cudaMemsetAsync(keys, 0, (size_t)M * sizeof(unsigned long long), st));
                jobs.job[jj] = K2Job{tg, tab, cnt1, sh1, keys, (float)b0, (float)b1};
            }
            const uint8_t* oh = (const uint8_t*)ws->bonehot.p;
            if (!stages) {
                // 3 stages need less shared memory than the 4 the chunk was sized for
                stages = tuned_k2_stages(ws, "k2tc_batch_stages", jobs, M, c, D, (const int2*)ws->items3.p,
                                         ws->n_items3, oh, Kp_max, nj * D, fbits, true);
                if (stages <= 0) return fail(MDFS_ECUDA, "k = 2 stage tuning failed (CUDA error)");
            }
            MDFS_LAUNCH("k2", st, launch_k2tc(oh, Kp_max, nj * D, jobs, M, c, 0, D, D, (const int2*)ws->items3.p,
                                              ws->n_items3, fbits, (int*)ws->err.p, true, stages, st));
            for (int jj = 0; jj < nj; ++jj) {
                const int j = j0 + jj;
                MDFS_LAUNCH("finalize", st,
                            launch_finalize((const unsigned long long*)ws->bkeys.p + (size_t)jj * M, M, k,
                                            oig.dev + (size_t)j * M, otu.dev ? otu.dev + (size_t)j * M * kk : nullptr,
                                            odi.dev ? odi.dev + (size_t)j * M : nullptr, st));
            }
        }
        check_err = true;
    } else {
        for (int j = 0; j < n_jobs; ++j) {
            MDFS_LAUNCH("gather", st, launch_gather_job(xd, data->dtype, yd, N, M, idxd ? idxd + (size_t)j * N : nullptr,
                                                        permd ? permd + (size_t)j * N : nullptr, ws->bx.p,
                                                        (uint8_t*)ws->by.p, stats + 3, st));
            MDFS_LAUNCH("stats", st, launch_stats((const uint8_t*)ws->by.p, N, stats, (int*)ws->perm.p, st));
            bool job_err = false;
            rc = scan_core(ws, ws->bx.p, data->dtype, N, M, counts[j].x, k, divisions, D, range, pc_xi, seed, &job_err,
                           0, 1, nullptr, nullptr, true);
            if (rc) return rc;
            check_err |= job_err;
            MDFS_LAUNCH("finalize", st,
                        launch_finalize((const unsigned long long*)ws->keys.p, M, k, oig.dev + (size_t)j * M,
                                        otu.dev ? otu.dev + (size_t)j * M * kk : nullptr,
                                        odi.dev ? odi.dev + (size_t)j * M : nullptr, st, wide_disc(ws)));
        }
    }
    if ((rc = copy_back(ws, oig)) || (rc = copy_back(ws, otu)) || (rc = copy_back(ws, odi))) return rc;
    if (check_err)
        MDFS_CUDA_TRY(cudaMemcpyAsync(ws->host_stats + 8, ws->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    MDFS_CUDA_TRY(cudaStreamSynchronize(st));
    if (check_err && ws->host_stats[8]) return kernel_flag_error(ws->host_stats[8]);
    return MDFS_OK;
}

int mdfs_max_ig_shard(const mdfs_data* data, int k, int divisions, int discretizations, double range, double pc_xi,
                      uint64_t seed, int shard, int n_shards, uint64_t* keys_out, void* stream) {
    g_err.clear();
    g_launches = 0;
    int rc = check_data(data, true);
    if (rc) return rc;
    const int N = data->N, M = data->M, D = discretizations;
    if (n_shards < 1 || shard < 0 || shard >= n_shards) return fail(MDFS_EINVAL, "shard %d of %d", shard, n_shards);
    if ((rc = check_scan_args(k, M, divisions, N, D, range, pc_xi, true))) return rc;
    if (!keys_out) return fail(MDFS_EINVAL, "keys is NULL");
    if ((rc = check_devices({{data->x, "x"}, {data->y, "y"}, {keys_out, "keys"}}))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace* ws = get_ws(st, &rc);
    if (!ws) return rc;
    const void* xd = nullptr;
    const uint8_t* yd = nullptr;
    int n1 = 0;
    rc = stage_inputs(ws, data, true, &xd, &yd, &n1);
    if (rc) return rc;
    bool check_err = false;
    rc = scan_core(ws, xd, data->dtype, N, M, n1, k, divisions, D, range, pc_xi, seed, &check_err, shard, n_shards);
    if (rc) return rc;
    MDFS_CUDA_TRY(cudaMemcpyAsync(keys_out, ws->keys.p, (size_t)M * sizeof(uint64_t), cudaMemcpyDefault, st));
    if (check_err) {
        MDFS_CUDA_TRY(cudaMemcpyAsync(ws->host_stats + 8, ws->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        MDFS_CUDA_TRY(cudaStreamSynchronize(st));
        const int flag = ws->host_stats[8];
        if (flag) return kernel_flag_error(flag);
    }
    MDFS_CUDA_TRY(cudaStreamSynchronize(st));
    return MDFS_OK;
}

int mdfs_keys_decode(const uint64_t* keys, int M, int k, float* ig, int32_t* tuples, int32_t* best_disc, void* stream) {
    g_err.clear();
    g_launches = 0;
    if (!keys || !ig) return fail(MDFS_EINVAL, "keys and ig must not be NULL");
    if (M < 1 || M > 65535 || k < 1 || k > 5) return fail(MDFS_EINVAL, "M or k out of range");
    int rc = 0;
    if ((rc = check_devices({{keys, "keys"}, {ig, "ig"}, {tuples, "tuples"}, {best_disc, "best_disc"}}))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace* ws = get_ws(st, &rc);
    if (!ws) return rc;
    const unsigned long long* kd = (const unsigned long long*)keys;
    if (!is_device_ptr(keys)) {
        MDFS_ENSURE(ws, keys, (size_t)M * sizeof(uint64_t));
        MDFS_CUDA_TRY(cudaMemcpyAsync(ws->keys.p, keys, (size_t)M * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
        kd = (const unsigned long long*)ws->keys.p;
    }
    Out<float> oig;
    Out<int32_t> otu, odi;
    rc = bind_out(ws, ws->ig, ig, (size_t)M, &oig);
    if (rc) return rc;
    rc = bind_out(ws, ws->tuples, k > 1 ? tuples : (int32_t*)nullptr, (size_t)M * (k > 1 ? k - 1 : 1), &otu);
    if (rc) return rc;
    rc = bind_out(ws, ws->disc, best_disc, (size_t)M, &odi);
    if (rc) return rc;
    MDFS_LAUNCH("finalize", st, launch_finalize(kd, M, k, oig.dev, otu.dev, odi.dev, st));
    if ((rc = copy_back(ws, oig)) || (rc = copy_back(ws, otu)) || (rc = copy_back(ws, odi))) return rc;
    MDFS_CUDA_TRY(cudaStreamSynchronize(st));
    return MDFS_OK;
}

int mdfs_ig_lim(const float* ig, int M, int k, int divisions, int discretizations, const uint8_t* irrelevant_mask,
                double alpha, double* p_values, double* ig_lim, double* n_eff, void* stream) {
    g_err.clear();
    g_launches = 0;
    (void)discretizations;
    if (!ig || !p_values) return fail(MDFS_EINVAL, "ig and p_values must not be NULL");
    if (M < 1) return fail(MDFS_EINVAL, "M = %d < 1", M);
    if (k < 1 || k > 5) return fail(MDFS_EINVAL, "k = %d outside [1, 5]", k);
    const int c = divisions + 1;
    if (divisions < 1 || c > kMaxC) return fail(MDFS_EINVAL, "divisions = %d outside [1, %d]", divisions, kMaxC - 1);
    if (!(alpha > 0.0 && alpha < 1.0)) return fail(MDFS_EINVAL, "alpha must lie in (0, 1)");
    int df = c - 1;
    for (int j = 1; j < k; ++j) df *= c;
    int rc = 0;
    if ((rc = check_devices({{ig, "ig"}, {irrelevant_mask, "irrelevant_mask"}, {p_values, "p_values"}, {ig_lim, "ig_lim"}, {n_eff, "n_eff"}}))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace* ws = get_ws(st, &rc);
    if (!ws) return rc;
    const float* igd = ig;
    if (!is_device_ptr(ig)) {
        MDFS_ENSURE(ws, ig, (size_t)M * sizeof(float));
        MDFS_CUDA_TRY(cudaMemcpyAsync(ws->ig.p, ig, (size_t)M * sizeof(float), cudaMemcpyHostToDevice, st));
        igd = (const float*)ws->ig.p;
    }
    const uint8_t* maskd = irrelevant_mask;
    if (irrelevant_mask && !is_device_ptr(irrelevant_mask)) {
        MDFS_ENSURE(ws, mask, (size_t)M);
        MDFS_CUDA_TRY(cudaMemcpyAsync(ws->mask.p, irrelevant_mask, (size_t)M, cudaMemcpyHostToDevice, st));
        maskd = (const uint8_t*)ws->mask.p;
    }
    Out<double> op;
    rc = bind_out(ws, ws->pv, p_values, (size_t)M, &op);
    if (rc) return rc;
    MDFS_ENSURE(ws, res, 4 * sizeof(double));
    double* res = (double*)ws->res.p;
    MDFS_CUDA_TRY(cudaMemsetAsync(res, 0, 4 * sizeof(double), st));
    MDFS_LAUNCH("ig_lim_cdf", st, launch_ig_lim_cdf(igd, M, df, op.dev, st));
    MDFS_LAUNCH("ig_lim_fit", st, launch_ig_lim_fit(op.dev, M, df, maskd, alpha, res, st));
    MDFS_LAUNCH("ig_lim_p", st, launch_ig_lim_p(M, res, op.dev, st));
    MDFS_CUDA_TRY(cudaMemcpyAsync(ws->host_res, res, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    MDFS_CUDA_TRY(cudaStreamSynchronize(st));
    if (!(ws->host_res[2] > 0.0) || !(ws->host_res[1] > 0.0))
        return fail(MDFS_EDEGENERATE, "no variable with IG > 0 in the fitted set");
    rc = copy_back(ws, op);
    if (rc) return rc;
    if (ig_lim) {
        if (is_device_ptr(ig_lim)) MDFS_CUDA_TRY(cudaMemcpyAsync(ig_lim, res, sizeof(double), cudaMemcpyDeviceToDevice, st));
        else *ig_lim = ws->host_res[0];
    }
    if (n_eff) {
        if (is_device_ptr(n_eff)) MDFS_CUDA_TRY(cudaMemcpyAsync(n_eff, res + 1, sizeof(double), cudaMemcpyDeviceToDevice, st));
        else *n_eff = ws->host_res[1];
    }
    MDFS_CUDA_TRY(cudaStreamSynchronize(st));
    return MDFS_OK;
}

int mdfs_contrast(const mdfs_data* data, int n_contrast, uint64_t seed, void* x_ext, int32_t* src, void* stream) {
    g_err.clear();
    g_launches = 0;
    int rc = check_data(data, false);
    if (rc) return rc;
    const int N = data->N, M = data->M;
    if (n_contrast < 0 || M + n_contrast > 65535)
        return fail(MDFS_EINVAL, "n_contrast = %d: M + n_contrast must lie in [M, 65535]", n_contrast);
    if (!x_ext) return fail(MDFS_EINVAL, "x_ext is NULL");
    if ((rc = check_devices({{data->x, "x"}, {x_ext, "x_ext"}, {src, "src"}}))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace* ws = get_ws(st, &rc);
    if (!ws) return rc;
    const void* xd = nullptr;
    const uint8_t* yd = nullptr;
    int n1 = 0;
    rc = stage_inputs(ws, data, false, &xd, &yd, &n1);
    if (rc) return rc;
    const size_t elem = data->dtype == MDFS_F32 ? 4 : 1;
    Out<uint8_t> ox;
    Out<int32_t> os;
    rc = bind_out(ws, ws->xe, (uint8_t*)x_ext, (size_t)(M + n_contrast) * N * elem, &ox);
    if (rc) return rc;
    rc = bind_out(ws, ws->srcb, src, (size_t)n_contrast, &os);
    if (rc) return rc;
    MDFS_CUDA_TRY(cudaMemcpyAsync(ox.dev, xd, (size_t)M * N * elem, cudaMemcpyDeviceToDevice, st));
    MDFS_LAUNCH("contrast", st, launch_contrast(xd, data->dtype, N, M, n_contrast, seed, ox.dev, os.dev, st));
    if ((rc = copy_back(ws, ox)) || (rc = copy_back(ws, os))) return rc;
    if (ox.staged || os.staged || st == nullptr) MDFS_CUDA_TRY(cudaStreamSynchronize(st));
    return MDFS_OK;
}

int mdfs_p_adjust(const double* p, int m, int method, double* adjusted, void* stream) {
    g_err.clear();
    g_launches = 0;
    if (!p || !adjusted) return fail(MDFS_EINVAL, "p and adjusted must not be NULL");
    if (m < 1 || m > 65536) return fail(MDFS_EINVAL, "m = %d outside [1, 65536]", m);
    if (method < MDFS_ADJUST_NONE || method > MDFS_ADJUST_BY) return fail(MDFS_EINVAL, "unknown method %d", method);
    int rc = 0;
    if ((rc = check_devices({{p, "p"}, {adjusted, "adjusted"}}))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace* ws = get_ws(st, &rc);
    if (!ws) return rc;
    const double* pd = p;
    if (!is_device_ptr(p)) {
        MDFS_ENSURE(ws, pext, (size_t)m * sizeof(double));
        MDFS_CUDA_TRY(cudaMemcpyAsync(ws->pext.p, p, (size_t)m * sizeof(double), cudaMemcpyHostToDevice, st));
        pd = (const double*)ws->pext.p;
    }
    Out<double> oa;
    rc = bind_out(ws, ws->adjb, adjusted, (size_t)m, &oa);
    if (rc) return rc;
    MDFS_ENSURE(ws, padj, p_adjust_scratch_bytes(m));
    MDFS_LAUNCH("p_adjust", st, launch_p_adjust(pd, m, method, 1.0, ws->padj.p, oa.dev, nullptr, st));
    rc = copy_back(ws, oa);
    if (rc) return rc;
    if (oa.staged || st == nullptr) MDFS_CUDA_TRY(cudaStreamSynchronize(st));
    return MDFS_OK;
}

int mdfs_select(const mdfs_data* data, int n_contrast, int k, int divisions, int discretizations, double range,
                double pc_xi, uint64_t seed, int p_adjust_method, double level, float* ig, int32_t* tuples,
                int32_t* best_disc, double* p_values, double* adjusted, uint8_t* relevant, double* ig_lim,
                double* n_eff, int32_t* contrast_src, void* stream) {
    g_err.clear();
    g_launches = 0;
    int rc = check_data(data, true);
    if (rc) return rc;
    const int N = data->N, M = data->M, D = discretizations, c = divisions + 1;
    const int Mx = M + n_contrast;
    if (n_contrast < 1 || Mx > 65535)
        return fail(MDFS_EINVAL, "n_contrast = %d: need n_contrast >= 1 and M + n_contrast <= 65535", n_contrast);
    if ((rc = check_scan_args(k, Mx, divisions, N, D, range, pc_xi))) return rc;
    if (!(level > 0.0 && level < 1.0)) return fail(MDFS_EINVAL, "level must lie in (0, 1)");
    if (p_adjust_method < MDFS_ADJUST_NONE || p_adjust_method > MDFS_ADJUST_BY)
        return fail(MDFS_EINVAL, "unknown p_adjust_method %d", p_adjust_method);
    if (!ig || !p_values || !adjusted || !relevant)
        return fail(MDFS_EINVAL, "ig, p_values, adjusted and relevant must not be NULL");
    int df = c - 1;
    for (int j = 1; j < k; ++j) df *= c;

    if ((rc = check_devices({{data->x, "x"}, {data->y, "y"}, {ig, "ig"}, {tuples, "tuples"}, {best_disc, "best_disc"}, {p_values, "p_values"}, {adjusted, "adjusted"}, {relevant, "relevant"}, {ig_lim, "ig_lim"}, {n_eff, "n_eff"}, {contrast_src, "contrast_src"}}))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace* ws = get_ws(st, &rc);
    if (!ws) return rc;
    const void* xd = nullptr;
    const uint8_t* yd = nullptr;
    int n1 = 0;
    rc = stage_inputs(ws, data, true, &xd, &yd, &n1);
    if (rc) return rc;
    // 1. the extended variable set
    const size_t elem = data->dtype == MDFS_F32 ? 4 : 1;
    MDFS_ENSURE(ws, xe, (size_t)Mx * N * elem);
    MDFS_ENSURE(ws, srcb, (size_t)n_contrast * sizeof(int));
    MDFS_CUDA_TRY(cudaMemcpyAsync(ws->xe.p, xd, (size_t)M * N * elem, cudaMemcpyDeviceToDevice, st));
    MDFS_LAUNCH("contrast", st,
                launch_contrast(xd, data->dtype, N, M, n_contrast, seed, ws->xe.p, (int*)ws->srcb.p, st));
    // 2. IG^k_max over it
    bool check_err = false;
    rc = scan_core(ws, ws->xe.p, data->dtype, N, Mx, n1, k, divisions, D, range, pc_xi, seed, &check_err);
    if (rc) return rc;
    const int kk = k > 1 ? k - 1 : 1;
    MDFS_ENSURE(ws, igx, (size_t)Mx * sizeof(float));
    MDFS_ENSURE(ws, tux, (size_t)Mx * kk * sizeof(int));
    MDFS_ENSURE(ws, dix, (size_t)Mx * sizeof(int));
    float* igx = (float*)ws->igx.p;
    MDFS_LAUNCH("finalize", st, launch_finalize((const unsigned long long*)ws->keys.p, Mx, k, igx,
                                                k > 1 ? (int*)ws->tux.p : nullptr, (int*)ws->dix.p, st,
                                                wide_disc(ws)));
    if (check_err) {
        MDFS_CUDA_TRY(cudaMemcpyAsync(ws->host_stats + 8, ws->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        MDFS_CUDA_TRY(cudaStreamSynchronize(st));
        if (ws->host_stats[8]) return kernel_flag_error(ws->host_stats[8]);
    }
    // 3. the fit on the contrast variables, p-values of every variable
    MDFS_ENSURE(ws, mask, (size_t)Mx);
    MDFS_CUDA_TRY(cudaMemsetAsync(ws->mask.p, 0, (size_t)M, st));
    MDFS_CUDA_TRY(cudaMemsetAsync((uint8_t*)ws->mask.p + M, 1, (size_t)n_contrast, st));
    MDFS_ENSURE(ws, pext, (size_t)Mx * sizeof(double));
    MDFS_ENSURE(ws, res, 4 * sizeof(double));
    double* pext = (double*)ws->pext.p;
    double* res = (double*)ws->res.p;
    MDFS_CUDA_TRY(cudaMemsetAsync(res, 0, 4 * sizeof(double), st));
    MDFS_LAUNCH("ig_lim_cdf", st, launch_ig_lim_cdf(igx, Mx, df, pext, st));
    MDFS_LAUNCH("ig_lim_fit", st, launch_ig_lim_fit(pext, Mx, df, (const uint8_t*)ws->mask.p, level, res, st));
    MDFS_LAUNCH("ig_lim_p", st, launch_ig_lim_p(Mx, res, pext, st));
    // 4-5. adjustment over the original variables and the relevant set
    MDFS_ENSURE(ws, adjb, (size_t)M * sizeof(double));
    MDFS_ENSURE(ws, relb, (size_t)M);
    MDFS_ENSURE(ws, padj, p_adjust_scratch_bytes(M));
    MDFS_LAUNCH("p_adjust", st, launch_p_adjust(pext, M, p_adjust_method, level, ws->padj.p, (double*)ws->adjb.p,
                                                (uint8_t*)ws->relb.p, st));
    MDFS_CUDA_TRY(cudaMemcpyAsync(ws->host_res, res, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    MDFS_CUDA_TRY(cudaStreamSynchronize(st));
    if (!(ws->host_res[2] > 0.0) || !(ws->host_res[1] > 0.0))
        return fail(MDFS_EDEGENERATE, "no contrast variable with IG > 0");
    if ((rc = emit(ws, igx, ig, (size_t)M)) || (rc = emit(ws, (const int*)ws->tux.p, tuples, (size_t)M * (k - 1))) ||
        (rc = emit(ws, (const int*)ws->dix.p, best_disc, (size_t)M)) || (rc = emit(ws, (const double*)pext, p_values, (size_t)M)) ||
        (rc = emit(ws, (const double*)ws->adjb.p, adjusted, (size_t)M)) ||
        (rc = emit(ws, (const uint8_t*)ws->relb.p, relevant, (size_t)M)) ||
        (rc = emit(ws, (const int*)ws->srcb.p, contrast_src, (size_t)n_contrast)) ||
        (rc = emit(ws, (const double*)res, ig_lim, 1)) || (rc = emit(ws, (const double*)res + 1, n_eff, 1)))
        return rc;
    MDFS_CUDA_TRY(cudaStreamSynchronize(st));
    return MDFS_OK;
}

int mdfs_interesting_tuples(const mdfs_data* data, int k, int divisions, int discretizations, double range,
                            double pc_xi, uint64_t seed, double ig_threshold, int capacity, int32_t* var,
                            int32_t* tuples, float* ig, int32_t* best_disc, int64_t* count, void* stream) {
    g_err.clear();
    g_launches = 0;
    int rc = check_data(data, true);
    if (rc) return rc;
    const int N = data->N, M = data->M, D = discretizations;
    if ((rc = check_scan_args(k, M, divisions, N, D, range, pc_xi))) return rc;
    if (!(ig_threshold > -1e9 && ig_threshold < 1e9)) return fail(MDFS_EINVAL, "ig_threshold must be finite");
    if (capacity < 1 || capacity > (1 << 22)) return fail(MDFS_EINVAL, "capacity = %d outside [1, 2^22]", capacity);
    if (!var || !ig || !count || (k > 1 && !tuples))
        return fail(MDFS_EINVAL, "var, ig, tuples (k > 1) and count must not be NULL");
    if ((rc = check_devices({{data->x, "x"}, {data->y, "y"}, {var, "var"}, {tuples, "tuples"}, {ig, "ig"}, {best_disc, "best_disc"}}))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace* ws = get_ws(st, &rc);
    if (!ws) return rc;
    const void* xd = nullptr;
    const uint8_t* yd = nullptr;
    int n1 = 0;
    rc = stage_inputs(ws, data, true, &xd, &yd, &n1);
    if (rc) return rc;
    // room for twice the capacity: more records than capacity are detected, not lost silently
    size_t tsize = 1024;
    while (tsize < 2 * (size_t)capacity + 1) tsize <<= 1;
    MDFS_ENSURE(ws, ekeys, tsize * sizeof(unsigned long long));
    MDFS_ENSURE(ws, evals, tsize * sizeof(unsigned long long));
    MDFS_ENSURE(ws, ecnt, 4 * sizeof(int));
    MDFS_CUDA_TRY(cudaMemsetAsync(ws->ekeys.p, 0xFF, tsize * sizeof(unsigned long long), st));
    MDFS_CUDA_TRY(cudaMemsetAsync(ws->evals.p, 0, tsize * sizeof(unsigned long long), st));
    MDFS_CUDA_TRY(cudaMemsetAsync(ws->ecnt.p, 0, 4 * sizeof(int), st));
    EmitTable em;
    em.keys = (unsigned long long*)ws->ekeys.p;
    em.vals = (unsigned long long*)ws->evals.p;
    em.mask = (unsigned int)(tsize - 1);
    em.thr_fx = llround(ig_threshold * kFxScale);
    em.n_keys = (int*)ws->ecnt.p;
    em.full = (int*)ws->ecnt.p + 1;
    bool check_err = false;
    rc = scan_core(ws, xd, data->dtype, N, M, n1, k, divisions, D, range, pc_xi, seed, &check_err, 0, 1, &em);
    if (rc) return rc;
    MDFS_CUDA_TRY(cudaMemcpyAsync(ws->host_stats + 8, ws->ecnt.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    MDFS_CUDA_TRY(cudaStreamSynchronize(st));
    const int n = ws->host_stats[8], full = ws->host_stats[9];
    *count = n;
    if (full || n > capacity)
        return fail(MDFS_ETRUNCATED, "%s%d records reach the threshold; capacity is %d", full ? "at least " : "", n,
                    capacity);
    int npad = 1;
    while (npad < n) npad <<= 1;
    MDFS_ENSURE(ws, erk, (size_t)npad * sizeof(unsigned long long));
    MDFS_ENSURE(ws, erv, (size_t)npad * sizeof(unsigned long long));
    const size_t nn = (size_t)std::max(n, 1);
    Out<int32_t> ov, otu, odi;
    Out<float> oig;
    if ((rc = bind_out(ws, ws->tux, var, nn, &ov)) ||
        (rc = bind_out(ws, ws->dix, k > 1 ? tuples : (int32_t*)nullptr, nn * (k > 1 ? k - 1 : 1), &otu)) ||
        (rc = bind_out(ws, ws->relb, best_disc, nn, &odi)) || (rc = bind_out(ws, ws->igx, ig, nn, &oig)))
        return rc;
    int* disc_dev = odi.dev;  // the decoder always writes a discretisation
    if (!disc_dev) {
        MDFS_ENSURE(ws, adjb, nn * sizeof(int));
        disc_dev = (int*)ws->adjb.p;
    }
    MDFS_LAUNCH("emit_collect", st,
                launch_emit_collect(em, k, (unsigned long long*)ws->erk.p, (unsigned long long*)ws->erv.p,
                                    (int*)ws->ecnt.p + 2, npad, ov.dev, otu.dev, oig.dev, disc_dev, n, st));
    if (n > 0) {
        ov.bytes = (size_t)n * sizeof(int32_t);
        otu.bytes = (size_t)n * (k > 1 ? k - 1 : 1) * sizeof(int32_t);
        odi.bytes = (size_t)n * sizeof(int32_t);
        oig.bytes = (size_t)n * sizeof(float);
        if ((rc = copy_back(ws, ov)) || (rc = copy_back(ws, otu)) || (rc = copy_back(ws, odi)) ||
            (rc = copy_back(ws, oig)))
            return rc;
    }
    MDFS_CUDA_TRY(cudaStreamSynchronize(st));
    return MDFS_OK;
}

// ---- test-only entry points (include/mdfs_testing.h) -------------------------

int mdfs_testing_counts(const mdfs_data* data, int k, int divisions, int discretizations, double range, uint64_t seed,
                        uint32_t* counts, void* stream) {
    g_err.clear();
    g_launches = 0;
    int rc = check_data(data, true);
    if (rc) return rc;
    const int N = data->N, M = data->M, D = discretizations;
    if (k != 2 && k != 3) return fail(MDFS_EINVAL, "k = %d: the count hook serves k = 2 and k = 3", k);
    if ((rc = check_scan_args(k, M, divisions, N, D, range, 0.25))) return rc;
    if (!counts) return fail(MDFS_EINVAL, "counts is NULL");
    if (!is_device_ptr(counts) || foreign_device(counts) >= 0)
        return fail(MDFS_EINVAL, "counts must be device memory of the current device");
    cudaStream_t st = (cudaStream_t)stream;
    Workspace* ws = get_ws(st, &rc);
    if (!ws) return rc;
    const void* xd = nullptr;
    const uint8_t* yd = nullptr;
    int n1 = 0;
    if ((rc = stage_inputs(ws, data, true, &xd, &yd, &n1))) return rc;
    bool check_err = false;
    rc = scan_core(ws, xd, data->dtype, N, M, n1, k, divisions, D, range, 0.25, seed, &check_err, 0, 1, nullptr,
                   counts);
    if (rc) return rc;
    MDFS_CUDA_TRY(cudaMemcpyAsync(ws->host_stats + 8, ws->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    MDFS_CUDA_TRY(cudaStreamSynchronize(st));
    if (ws->host_stats[8]) return kernel_flag_error(ws->host_stats[8]);
    return MDFS_OK;
}

int mdfs_testing_exact(void) {
    g_err.clear();
    std::lock_guard<std::mutex> lock(g_hooks_mu);
    g_hooks.exact = true;
    return MDFS_OK;
}

int mdfs_testing_k3_claim_order(int M, int nd, int32_t* order, int cap) {
    g_err.clear();
    if (M < 3 || M > 65535) return fail(MDFS_EINVAL, "M = %d outside [3, 65535]", M);
    if (nd < 1 || nd > kMaxD) return fail(MDFS_EINVAL, "nd = %d outside [1, %d]", nd, kMaxD);
    if (cap > 0 && !order) return fail(MDFS_EINVAL, "order is NULL");
    std::vector<int2> items;
    build_k3tc_items(M, items);
    std::vector<int> out;
    build_k3tc_order(M, items.data(), (int)items.size(), nd, out);
    for (int i = 0; i < cap && i < (int)out.size(); ++i) order[i] = out[i];
    return (int)out.size();
}

int mdfs_testing_k3_wait_fault(int withhold_kb, long long wait_ns) {
    g_err.clear();
    if (withhold_kb < -1) return fail(MDFS_EINVAL, "withhold_kb = %d < -1", withhold_kb);
    if (wait_ns < 0 || wait_ns > 10000000000ll) return fail(MDFS_EINVAL, "wait_ns outside [0, 10 s]");
    std::lock_guard<std::mutex> lock(g_hooks_mu);
    g_hooks.withhold_kb = withhold_kb;
    g_hooks.wait_ns = (unsigned long long)wait_ns;
    return MDFS_OK;
}

}  // extern "C"
