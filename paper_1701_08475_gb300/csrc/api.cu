// api.cu -- the C ABI (include/knng.h): argument checks, pointer marshalling,
// workspace, the build schedule of Alg. 1 (Sec. 3.1) plus refinement rounds,
// and kernel statistics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace knng {

size_t join_smem_bytes(int D, int mcap);
int join_blocks_per_lane(int mcap);

// ---------------------------------------------------------------- errors
namespace {
thread_local std::string g_last_error;

struct Error {
    int code;
};

[[noreturn]] void fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    throw Error{code};
}

void cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    if (e == cudaErrorMemoryAllocation) fail(KNNG_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    fail(KNNG_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

// Sets the message knng_last_error returns (for entry points outside this file).
void record_error(const char* msg) { g_last_error = msg; }

// ---------------------------------------------------------------- fault injection
// KNNG_FAULT=alloc|launch makes the next calls fail on the host, for tests of
// the error paths (no device fault is ever made): "alloc" fails the workspace
// allocation as if the pool were out of memory (KNNG_ENOMEM); "launch" adds,
// before the call's first kernel, one launch the runtime refuses on the host
// (more threads per block than any GPU allows), which the call's launch check
// reports (KNNG_ECUDA).  The variable is read at the start of every call.
namespace {
thread_local int g_fault = 0;  // 0 none, 1 alloc, 2 launch
thread_local bool g_fault_fired = false;
// The first launch error of the current call, taken right after the launch:
// later runtime calls of the same call may clear the runtime's own record.
thread_local cudaError_t g_launch_error = cudaSuccess;

__global__ void k_refused() {}
}  // namespace

void fault_begin() {
    const char* e = getenv("KNNG_FAULT");
    g_fault = !e ? 0 : strcmp(e, "alloc") == 0 ? 1 : strcmp(e, "launch") == 0 ? 2 : 0;
    g_fault_fired = false;
    g_launch_error = cudaSuccess;
}

cudaError_t launch_error() {
    const cudaError_t last = cudaGetLastError();
    return g_launch_error != cudaSuccess ? g_launch_error : last;
}

bool fault_alloc() { return g_fault == 1; }

void fault_launch_point(cudaStream_t s) {
    if (g_fault != 2 || g_fault_fired) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    g_fault_fired = true;
    k_refused<<<1, 2048, 0, s>>>();
}

namespace {
template <class F>
int guarded(F&& f) {
    g_last_error.clear();
    fault_begin();
    try {
        f();
        return KNNG_OK;
    } catch (const Error& e) {
        return e.code;
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        return KNNG_ENOMEM;
    }
}
}  // namespace

// ---------------------------------------------------------------- stats
namespace {
struct StatRegistry {
    std::mutex mu;
    bool on = false, timing = false;
    std::map<std::string, knng_kernel_stat> stats;
    struct Pending {
        std::string name;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> free_events;

    cudaEvent_t event() {
        if (!free_events.empty()) {
            cudaEvent_t e = free_events.back();
            free_events.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    // called after the stream has been synchronised
    void flush() {
        std::lock_guard<std::mutex> lk(mu);
        for (auto& p : pending) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) stats[p.name].ms += ms;
            free_events.push_back(p.a);
            free_events.push_back(p.b);
        }
        pending.clear();
        cudaGetLastError();
    }
};
StatRegistry& reg() {
    static StatRegistry* r = new StatRegistry();
    return *r;
}
}  // namespace

// KNNG_LAUNCH_LOG=1: every launch scope (and every later byte count) is
// written to stderr as "launch <name> <bytes> <flops>", for matching
// profiler captures to their algorithmic work.
bool launch_log() {
    static const bool on = [] {
        const char* e = getenv("KNNG_LAUNCH_LOG");
        return e && e[0] == '1';
    }();
    return on;
}

LaunchScope::LaunchScope(const char* name, cudaStream_t s, double bytes, double flops, int kernels)
    : name_(name), s_(s), bytes_(bytes), flops_(flops), slot_(-1) {
    fault_launch_point(s);
    if (launch_log()) fprintf(stderr, "launch %s %.0f %.0f\n", name, bytes, flops);
    StatRegistry& r = reg();
    std::lock_guard<std::mutex> lk(r.mu);
    if (!r.on) return;
    knng_kernel_stat& st = r.stats[name];
    if (st.name[0] == 0) snprintf(st.name, sizeof st.name, "%s", name);
    st.launches += kernels;
    st.bytes += bytes;
    st.flops += flops;
    if (r.timing) {
        StatRegistry::Pending p{name, r.event(), r.event()};
        cudaEventRecord(p.a, s);
        r.pending.push_back(p);
        slot_ = (int)r.pending.size() - 1;
    }
}

void record_items(const char* name, double items) {
    StatRegistry& r = reg();
    std::lock_guard<std::mutex> lk(r.mu);
    if (!r.on) return;
    knng_kernel_stat& st = r.stats[name];
    if (st.name[0] == 0) snprintf(st.name, sizeof st.name, "%s", name);
    st.items += items;
}

void record_bytes(const char* name, double bytes) {
    if (launch_log()) fprintf(stderr, "bytes %s %.0f\n", name, bytes);
    StatRegistry& r = reg();
    std::lock_guard<std::mutex> lk(r.mu);
    if (!r.on) return;
    knng_kernel_stat& st = r.stats[name];
    if (st.name[0] == 0) snprintf(st.name, sizeof st.name, "%s", name);
    st.bytes += bytes;
}

void stats_set(bool on) {
    StatRegistry& r = reg();
    std::lock_guard<std::mutex> lk(r.mu);
    r.on = on;
}

bool stats_on() {
    StatRegistry& r = reg();
    std::lock_guard<std::mutex> lk(r.mu);
    return r.on;
}

void stats_flush() { reg().flush(); }

LaunchScope::~LaunchScope() {
    const cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess && g_launch_error == cudaSuccess) g_launch_error = e;
    StatRegistry& r = reg();
    std::lock_guard<std::mutex> lk(r.mu);
    if (slot_ >= 0 && slot_ < (int)r.pending.size()) cudaEventRecord(r.pending[slot_].b, s_);
}

// ---------------------------------------------------------------- memory
namespace {
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

cudaMemPool_t device_pool() {
    int dev = 0;
    cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) return it->second;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    cuda_check(cudaMemPoolCreate(&pool, &props), "cudaMemPoolCreate");
    uint64_t keep = ~0ull;  // keep freed memory for the next call
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
    return pool;
}

// One stream-ordered allocation carved into aligned pieces.
struct Workspace {
    cudaStream_t s = nullptr;
    char* base = nullptr;
    size_t size = 0, used = 0;

    template <class T>
    T* take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        size_t off = used;
        used += bytes;
        return base ? reinterpret_cast<T*>(base + off) : nullptr;
    }
    void allocate(cudaStream_t stream) {
        s = stream;
        size = used;
        used = 0;
        if (size == 0) return;
        if (fault_alloc()) fail(KNNG_ENOMEM, "workspace allocation: injected fault (KNNG_FAULT=alloc)");
        void* p = nullptr;
        cuda_check(cudaMallocFromPoolAsync(&p, size, device_pool(), s), "workspace allocation");
        base = static_cast<char*>(p);
    }
    ~Workspace() {
        if (base) cudaFreeAsync(base, s);
    }
};

bool is_device_ptr(const void* p) {
    if (p == nullptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Page-locked host memory (cudaHostAlloc, cudaMallocHost or cudaHostRegister):
// the only host memory a recorded copy may name.
bool is_pinned_host_ptr(const void* p) {
    if (p == nullptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// A caller buffer as the kernels see it: the caller's device pointer, or a
// workspace copy of a host buffer.
template <class T>
struct DevBuf {
    T* host = nullptr;  // non-null when the caller passed host memory
    T* dev = nullptr;
    size_t count = 0;
};

template <class T>
void bind(Workspace& ws, DevBuf<T>& b, const T* caller, size_t count, bool pass) {
    b.count = count;
    if (is_device_ptr(caller)) {
        b.dev = const_cast<T*>(caller);
        b.host = nullptr;
    } else {
        b.host = const_cast<T*>(caller);
        b.dev = ws.take<T>(count);
        (void)pass;
    }
}

template <class T>
void upload(DevBuf<T>& b, cudaStream_t s) {
    if (b.host && b.count)
        cuda_check(cudaMemcpyAsync(b.dev, b.host, b.count * sizeof(T), cudaMemcpyHostToDevice, s), "H2D copy");
}
template <class T>
void download(DevBuf<T>& b, cudaStream_t s) {
    if (b.host && b.count)
        cuda_check(cudaMemcpyAsync(b.host, b.dev, b.count * sizeof(T), cudaMemcpyDeviceToHost, s), "D2H copy");
}

__global__ void k_iota(int32_t* p, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        p[e] = (int32_t)e;
}

__global__ void k_fill_f32(float* p, int64_t n, float v) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        p[e] = v;
}

void launch_fill_value(float* p, int64_t n, float v, cudaStream_t s) {
    LaunchScope ls("k_fill_f32", s, n * 4.0, 0);
    k_fill_f32<<<(int)std::min<int64_t>((n + 255) / 256 + 1, 152 * 16), 256, 0, s>>>(p, n, v);
}
}  // namespace

// ---------------------------------------------------------------- tree plan
namespace {
int tree_depth(int64_t n, int leaf_max) {
    int L = 0;
    while ((n + ((int64_t)1 << L) - 1) / ((int64_t)1 << L) > leaf_max) ++L;
    return L;
}

int bits_for(int64_t v) {  // bits to hold values 0..v
    int b = 0;
    while (((int64_t)1 << b) <= v) ++b;
    return b;
}

// Offsets of every level, the tiles of every sweep, and where they live in
// one device array.
struct TreePlan {
    int L = 0;
    int64_t n = 0;
    std::vector<std::vector<int32_t>> off;  // per level (L + 1 levels; off[L] = leaves)
    std::vector<LevelPlan> levels;
    std::vector<int32_t> host;               // packed device image
    struct Idx {
        size_t seg_off, tiles, seg_tile0, sweep, seg_sweep0, seg_local;  // element offsets into the image
    };
    bool forest = false;
    std::vector<Idx> idx;
    size_t leaf_off_at = 0;
    int nseg_max = 0, ntiles_max = 0, nsweep_max = 0, nseg_large_max = 0, max_leaf = 0;

    // tiles of at most `size` positions inside one segment: {seg, begin, end,
    // first}; segments with split[sgi] == 0 get none
    static void tile_level(const std::vector<int32_t>& o, const std::vector<char>& split, int size,
                           std::vector<int32_t>& tiles, std::vector<int32_t>& first) {
        const int nseg = (int)o.size() - 1;
        for (int sgi = 0; sgi < nseg; ++sgi) {
            first.push_back((int32_t)(tiles.size() / 4));
            if (!split[sgi]) continue;
            const int a = o[sgi], b = o[sgi + 1];
            for (int t = a; t < b; t += size) {
                tiles.push_back(sgi);
                tiles.push_back(t);
                tiles.push_back(std::min(b, t + size));
                tiles.push_back(t == a ? 1 : 0);
            }
        }
        first.push_back((int32_t)(tiles.size() / 4));
    }

    void make(int64_t n_, int leaf_max) { make_forest({n_}, {leaf_max}); }

    // Independent trees side by side (instance i owns positions
    // [sum of n_j for j < i, + n_i)); tree i stops splitting at its own depth,
    // and its segments keep their own indices for the seeds.
    void make_forest(const std::vector<int64_t>& sizes, const std::vector<int>& leaf_maxes) {
        const int ni = (int)sizes.size();
        n = 0;
        for (int64_t v : sizes) n += v;
        std::vector<int> depth(ni);
        L = 0;
        for (int i = 0; i < ni; ++i) {
            depth[i] = tree_depth(sizes[i], leaf_maxes[i]);
            L = std::max(L, depth[i]);
        }
        forest = ni > 1;
        off.assign(L + 1, {});
        std::vector<std::vector<int32_t>> owner(L + 1), local(L + 1);
        off[0].push_back(0);
        for (int i = 0; i < ni; ++i) {
            off[0].push_back(off[0].back() + (int32_t)sizes[i]);
            owner[0].push_back(i);
            local[0].push_back(0);
        }
        std::vector<std::vector<char>> split(L);
        for (int l = 0; l < L; ++l) {
            const auto& o = off[l];
            auto& nx = off[l + 1];
            for (size_t sgi = 0; sgi + 1 < o.size(); ++sgi) {
                const int inst = owner[l][sgi];
                const bool sp = l < depth[inst];
                split[l].push_back(sp ? 1 : 0);
                nx.push_back(o[sgi]);
                owner[l + 1].push_back(inst);
                local[l + 1].push_back(sp ? 2 * local[l][sgi] : local[l][sgi]);
                if (sp) {
                    nx.push_back(o[sgi] + (o[sgi + 1] - o[sgi]) / 2);
                    owner[l + 1].push_back(inst);
                    local[l + 1].push_back(2 * local[l][sgi] + 1);
                }
            }
            nx.push_back((int32_t)n);
        }
        host.clear();
        levels.assign(L, {});
        idx.assign(L, {});
        nseg_max = ntiles_max = nsweep_max = nseg_large_max = 0;
        for (int l = 0; l < L; ++l) {
            const auto& o = off[l];
            const int nseg = (int)o.size() - 1;
            std::vector<int32_t> tiles, tile0, sweep, sweep0;
            tile_level(o, split[l], kTile, tiles, tile0);
            tile_level(o, split[l], kSweepTile, sweep, sweep0);
            int max_m = 0;
            bool frozen = false;
            for (int sgi = 0; sgi < nseg; ++sgi) {
                if (split[l][sgi]) max_m = std::max(max_m, o[sgi + 1] - o[sgi]);
                else frozen = true;
            }
            LevelPlan& lp = levels[l];
            lp.level = l;
            lp.n = (int)n;
            lp.nseg = nseg;
            lp.ntiles = (int)tiles.size() / 4;
            lp.nsweep = (int)sweep.size() / 4;
            lp.max_m = max_m;
            lp.pos_bits = bits_for(max_m - 1);
            lp.small = max_m <= kSmallMax;
            lp.frozen = frozen;
            nseg_max = std::max(nseg_max, nseg);
            ntiles_max = std::max(ntiles_max, lp.ntiles);
            nsweep_max = std::max(nsweep_max, lp.nsweep);
            if (!lp.small) nseg_large_max = std::max(nseg_large_max, nseg);
            // int4 tiles need 16-byte alignment in the packed image
            while (host.size() % 4) host.push_back(0);
            idx[l].tiles = host.size();
            host.insert(host.end(), tiles.begin(), tiles.end());
            idx[l].sweep = host.size();
            host.insert(host.end(), sweep.begin(), sweep.end());
            idx[l].seg_off = host.size();
            host.insert(host.end(), o.begin(), o.end());
            idx[l].seg_tile0 = host.size();
            host.insert(host.end(), tile0.begin(), tile0.end());
            idx[l].seg_sweep0 = host.size();
            host.insert(host.end(), sweep0.begin(), sweep0.end());
            idx[l].seg_local = host.size();
            if (forest) host.insert(host.end(), local[l].begin(), local[l].end());
        }
        leaf_off_at = host.size();
        host.insert(host.end(), off[L].begin(), off[L].end());
        max_leaf = 0;
        for (size_t i = 0; i + 1 < off[L].size(); ++i) max_leaf = std::max(max_leaf, off[L][i + 1] - off[L][i]);
    }
    // point the level plans into the uploaded image
    void rebase(const int32_t* dev) {
        for (int l = 0; l < L; ++l) {
            levels[l].tiles = reinterpret_cast<const int4*>(dev + idx[l].tiles);
            levels[l].sweep = reinterpret_cast<const int4*>(dev + idx[l].sweep);
            levels[l].seg_off = dev + idx[l].seg_off;
            levels[l].seg_tile0 = dev + idx[l].seg_tile0;
            levels[l].seg_sweep0 = dev + idx[l].seg_sweep0;
            levels[l].seg_local = forest ? dev + idx[l].seg_local : nullptr;
        }
    }
};
}  // namespace

// ---------------------------------------------------------------- the build
namespace {

struct Args {
    int64_t n;
    int D;
    knng_params p;
    size_t offer_budget = 0;  // bytes for one chunk's offers; 0: offer_budget_bytes()
};

void validate_common(const void* data, int64_t n, int D, int k) {
    if (!data) fail(KNNG_EINVAL, "data is NULL");
    if (D < 1 || D > 4096) fail(KNNG_EINVAL, "D = %d out of range [1, 4096]", D);
    if (k < 1 || k > 64) fail(KNNG_EINVAL, "k = %d out of range [1, 64]", k);
    if (n <= k) fail(KNNG_EINVAL, "n = %lld must exceed k = %d", (long long)n, k);
    if (n >= ((int64_t)1 << 31)) fail(KNNG_EINVAL, "n = %lld must be below 2^31", (long long)n);
    if (n * (int64_t)k >= ((int64_t)1 << 31)) fail(KNNG_EINVAL, "n * k must be below 2^31");
}

void validate_params(const knng_params* p, int64_t n) {
    if (!p) fail(KNNG_EINVAL, "params is NULL");
    if (p->tree_passes < 0) fail(KNNG_EINVAL, "tree_passes = %d < 0", p->tree_passes);
    if (p->refine_rounds < 0) fail(KNNG_EINVAL, "refine_rounds = %d < 0", p->refine_rounds);
    if (p->tree_passes == 0 && p->refine_rounds > 0)
        fail(KNNG_EINVAL, "refine_rounds > 0 needs tree_passes >= 1");
    if (p->tree_passes > 0 && (p->leaf_max < 2 * (p->k + 1) || p->leaf_max > 256))
        fail(KNNG_EINVAL, "leaf_max = %d out of range [2(k+1) = %d, 256]", p->leaf_max, 2 * (p->k + 1));
    if (p->join_mode != KNNG_JOIN_FWD && p->join_mode != KNNG_JOIN_FWD_REV && p->join_mode != KNNG_JOIN_SAMPLED)
        fail(KNNG_EINVAL, "join_mode = %d unknown", p->join_mode);
    if (p->join_mode == KNNG_JOIN_SAMPLED && (p->sample < 1 || 2 * p->sample > p->k))
        fail(KNNG_EINVAL, "sample = %d outside [1, k / 2] for the sampled join", p->sample);
    if (p->precision != KNNG_FP32 && p->precision != KNNG_BF16 && p->precision != KNNG_FP16 &&
        p->precision != KNNG_FP8)
        fail(KNNG_EINVAL, "precision = %d unknown", p->precision);
    if (p->twomeans_iters < 0 || p->twomeans_iters > 64)
        fail(KNNG_EINVAL, "twomeans_iters = %d out of range [0, 64]", p->twomeans_iters);
    const int m = p->join_mode != KNNG_JOIN_FWD ? 2 * p->k : p->k;
    if (p->refine_rounds > 0 && m > 64) fail(KNNG_EINVAL, "refinement supports k <= 32 with reverse lists");
    (void)n;
}

// Device bytes for one chunk's offers (target, key, grouped key: 20 B each).
// KNNG_OFFER_BUDGET_MB overrides it (smaller budgets mean more chunks).
size_t offer_budget_bytes() {
    const char* e = getenv("KNNG_OFFER_BUDGET_MB");
    if (e && atol(e) > 0) return (size_t)atol(e) << 20;
    return size_t(8) << 30;
}

struct BuildLayout {
    // sizes only; filled twice (layout, then real pointers)
    SplitBuffers sb{};
    JoinBuffers jb{};
    int32_t *perm_a = nullptr, *perm_b = nullptr, *plan_dev = nullptr;
    uint64_t *G = nullptr, *G2 = nullptr;
    int* status = nullptr;  // [0] status bits, [1] rows re-ranked exactly after a failed certificate
    int64_t nodes_per_chunk = 0;
    // low-precision leaf stage
    uint16_t* Xl = nullptr;
    float *lp_nrm = nullptr, *lp_err = nullptr, *lp_scale = nullptr;
    int* notexact = nullptr;
    // tensor-core join
    uint16_t* Xq = nullptr;
    float *q_nrm = nullptr, *q_err = nullptr, *q_scale = nullptr;
    // byte copy for the tree sweeps
    uint8_t* Xb = nullptr;
    int* bflag = nullptr;
    // leaves of the last tree passes, for the join ([npass][n])
    int32_t* lid = nullptr;
    // the tree passes' partitions are independent and run concurrently, each
    // on its own stream with its own permutations and split buffers (slot 0:
    // perm_a, perm_b and sb above; slots 1 ..: these); the leaf stages follow
    // in pass order on the caller's stream
    struct PartSlot {
        int32_t *perm_a = nullptr, *perm_b = nullptr;
        float *W = nullptr, *S = nullptr, *S2 = nullptr;
        uint64_t *thr = nullptr, *thr2 = nullptr;
        SelState* st = nullptr;
        uint32_t *ghist = nullptr, *ticket = nullptr;
        double *partial = nullptr, *segsum = nullptr, *segleft = nullptr;
        int32_t* tile_left = nullptr;
    };
    static constexpr int kPartSlots = 3;
    int nslots = 1;
    PartSlot slot[kPartSlots];
};

int byte_dim(int D) { return (D + 15) & ~15; }

// Byte copy of X for the tree sweeps, used when every value is an integer in
// [0, 255] (the kernels read the device flag; the host copy picks the sums
// kernel and sizes the statistics' algorithmic bytes).
void make_bytes(const float* X, const Args& a, BuildLayout& b, cudaStream_t s) {
    if (!b.Xb) return;
    cuda_check(cudaMemsetAsync(b.bflag, 0, sizeof(int), s), "flag clear");
    launch_bytes(X, a.n, a.D, byte_dim(a.D), b.Xb, b.bflag, s);
    if (b.jb.capture) return;  // a graph records no host reads
    int f = 1;
    cuda_check(cudaMemcpyAsync(&f, b.bflag, sizeof f, cudaMemcpyDeviceToHost, s), "flag read");
    cuda_check(cudaStreamSynchronize(s), "stream synchronize");
    b.sb.u8_host = f == 0;
}

// Quantisation type of the low-precision copy for a precision (0 FP16, 1
// BF16, 2 FP8 E4M3) and the name of its leaf kernel.
int qtype(int precision) { return precision == KNNG_BF16 ? 1 : precision == KNNG_FP16 ? 0 : 2; }
const char* leaf_kernel_name(int precision) {
    return precision == KNNG_BF16 ? "k2_leaf_bf16" : precision == KNNG_FP16 ? "k2_leaf_fp16" : "k2_leaf_fp8";
}

// Original-order 16-bit copy for the tensor-core stages (also sets the
// exactness flag); nothing in FP32.
void quantize_for_join(const float* X, const Args& a, BuildLayout& b, cudaStream_t s) {
    if (!b.Xq) return;
    launch_quantize(X, a.n, a.D, nullptr, qtype(a.p.precision), b.Xq, b.q_nrm, b.q_err, b.q_scale, b.notexact, s);
    if (b.jb.capture) return;  // a graph records no host reads
    // the kernels pick their path from the device flag; the host copy only
    // sizes the statistics' algorithmic bytes
    int f = 0;
    cuda_check(cudaMemcpyAsync(&f, b.notexact, sizeof f, cudaMemcpyDeviceToHost, s), "flag read");
    cuda_check(cudaStreamSynchronize(s), "stream synchronize");
    b.sb.q16_host = b.sb.Xq != nullptr && (f & 1) == 0 && !((f & 2) && (f & 4));
}

bool lp_leaf(const Args& a, const TreePlan& tp) {
    return a.p.precision != KNNG_FP32 && a.p.tree_passes > 0 && tp.max_leaf <= 256;
}

void carve(Workspace& ws, BuildLayout& b, const Args& a, const TreePlan& tp, bool tree, bool join) {
    const int64_t n = a.n;
    const int k = a.p.k, D = a.D;
    b.status = ws.take<int>(4);
    b.G = ws.take<uint64_t>((size_t)n * k);
    bool lp_any = a.p.precision != KNNG_FP32;
    if (lp_any) b.notexact = ws.take<int>(4);
    const int qt = qtype(a.p.precision);
    const size_t row_halves = (size_t)lp_row_bytes(D, qt) / 2;
    if (tree && lp_leaf(a, tp)) {
        b.Xl = ws.take<uint16_t>((size_t)n * row_halves);
        b.lp_nrm = ws.take<float>(n);
        b.lp_err = ws.take<float>(n);
        if (qt == 2) b.lp_scale = ws.take<float>(n);
    }
    if (lp_any && (join || tree)) {  // original-order low-precision copy
        b.Xq = ws.take<uint16_t>((size_t)n * row_halves);
        b.q_nrm = ws.take<float>(n);
        b.q_err = ws.take<float>(n);
        if (qt == 2) b.q_scale = ws.take<float>(n);
    }
    // the tensor-core join and the tree sweeps read a 16-bit copy when it is
    // exact; an FP8 copy never is
    lp_any = lp_any && qt != 2;
    if (join && lp_any) {  // the tensor-core join reads the original-order copy
        b.jb.lp = true;
        b.jb.bf16 = a.p.precision == KNNG_BF16;
        b.jb.Xq = b.Xq;
        b.jb.qnrm = b.q_nrm;
        b.jb.qerr = b.q_err;
        b.jb.notexact = b.notexact;
    }
    if (tree && lp_any) {  // the tree sweeps read the 16-bit copy when it is exact
        b.sb.Xq = b.Xq;
        b.sb.Dq = lp_dim(D);
        b.sb.qtype = a.p.precision == KNNG_BF16 ? 1 : 2;
        b.sb.qflag = b.notexact;
    }
    if (tree && join) {
        const int np = std::min(a.p.tree_passes, kMaxLeafPasses);
        b.lid = ws.take<int32_t>((size_t)n * kMaxLeafPasses);
        b.jb.leafid = b.lid;
        b.jb.npass = np;
    }
    if (tree) {
        b.Xb = ws.take<uint8_t>((size_t)n * byte_dim(D));
        b.bflag = ws.take<int>(4);
        b.sb.Xb = b.Xb;
        b.sb.Db = byte_dim(D);
        b.sb.bflag = b.bflag;
        b.plan_dev = ws.take<int32_t>(tp.host.size());
        const int ns = std::max(tp.nseg_max, 1), nt = std::max(tp.ntiles_max, 1);
        const int nl = std::max(tp.nseg_large_max, 1);
        b.nslots = std::max(1, std::min(a.p.tree_passes, (int)BuildLayout::kPartSlots));
        for (int q = 0; q < b.nslots; ++q) {
            BuildLayout::PartSlot& ps = b.slot[q];
            ps.perm_a = ws.take<int32_t>(n);
            ps.perm_b = ws.take<int32_t>(n);
            ps.W = ws.take<float>((size_t)ns * D);
            ps.S = ws.take<float>(n);
            ps.thr = ws.take<uint64_t>(ns);
            ps.S2 = ws.take<float>(n);
            ps.thr2 = ws.take<uint64_t>(ns);
            ps.st = ws.take<SelState>(ns);
            ps.ghist = ws.take<uint32_t>((size_t)nl << kRadixBits);
            ps.ticket = ws.take<uint32_t>(nl);
            ps.partial = ws.take<double>((size_t)std::max(tp.nsweep_max, 1) * 2 * D);
            ps.segsum = ws.take<double>((size_t)ns * D);
            ps.segleft = ws.take<double>((size_t)ns * D);
            ps.tile_left = ws.take<int32_t>(nt);
        }
        b.perm_a = b.slot[0].perm_a;
        b.perm_b = b.slot[0].perm_b;
        b.sb.W = b.slot[0].W;
        b.sb.S = b.slot[0].S;
        b.sb.thr = b.slot[0].thr;
        b.sb.S2 = b.slot[0].S2;
        b.sb.thr2 = b.slot[0].thr2;
        b.sb.st = b.slot[0].st;
        b.sb.ghist = b.slot[0].ghist;
        b.sb.ticket = b.slot[0].ticket;
        b.sb.nseg_large = nl;
        b.sb.partial = b.slot[0].partial;
        b.sb.segsum = b.slot[0].segsum;
        b.sb.segleft = b.slot[0].segleft;
        b.sb.tile_left = b.slot[0].tile_left;
        b.sb.status = b.status;
    }
    if (join) {
        const bool rev = a.p.join_mode != KNNG_JOIN_FWD;
        const int64_t m = rev ? 2 * k : k;
        const int64_t per_node = std::max<int64_t>(m * (m - 1), 1);
        int64_t cap = (int64_t)((a.offer_budget ? a.offer_budget : offer_budget_bytes()) / 20);
        cap = std::min<int64_t>(cap, per_node * n);
        cap = std::min<int64_t>(cap, ((int64_t)1 << 31) - 1);
        b.nodes_per_chunk = std::max<int64_t>(cap / per_node, 1);
        cap = b.nodes_per_chunk * per_node;
        b.G2 = ws.take<uint64_t>((size_t)n * k);
        if (rev) {
            b.jb.deg = ws.take<int32_t>(n + 1);
            b.jb.roff = ws.take<int32_t>(n + 1);
            b.jb.cur = ws.take<int32_t>(n);
            b.jb.rbuf = ws.take<uint64_t>((size_t)n * k);
            b.jb.R = ws.take<uint64_t>((size_t)n * k);
            b.jb.R2 = ws.take<uint64_t>((size_t)n * k);
            b.jb.rnew_buf = ws.take<uint64_t>(n);
        }
        b.jb.fnew_buf = ws.take<uint64_t>(n);
        b.jb.active = ws.take<int32_t>(n);
        b.jb.nactive = ws.take<int32_t>(4);
        if (rev) {
            b.jb.ovf_list = ws.take<int32_t>(n);
            b.jb.ovf_count = ws.take<int32_t>(4);
        }
        b.jb.pcnt = ws.take<int32_t>(n + 1);
        b.jb.poff = ws.take<int32_t>(n + 1);
        b.jb.pcur = ws.take<int32_t>(n);
        b.jb.ptgt = ws.take<uint32_t>(cap);
        b.jb.pkey = ws.take<uint64_t>(cap);
        b.jb.grouped = ws.take<uint64_t>(cap);
        b.jb.cap = cap;
        b.jb.counter = ws.take<uint32_t>(4);
        b.jb.scan_tmp = ws.take<int32_t>(scan_tmp_ints(n));
        b.jb.offers_total = ws.take<unsigned long long>(1);
        if (a.p.join_mode == KNNG_JOIN_SAMPLED) {
            b.jb.flags = ws.take<uint64_t>(n);
            b.jb.flags_post = ws.take<uint64_t>(n);
        }
    }
}

int grid_1d(int64_t count) {
    int64_t g = (count + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

void check_status(const int* dstatus, cudaStream_t s, const char* fallback_kernel = nullptr) {
    int hs[2] = {0, 0};
    cuda_check(cudaMemcpyAsync(hs, dstatus, sizeof hs, cudaMemcpyDeviceToHost, s), "status read");
    cuda_check(cudaStreamSynchronize(s), "stream synchronize");
    reg().flush();
    if (fallback_kernel) record_items(fallback_kernel, (double)hs[1]);
    const int st = hs[0];
    if (st & kStatusTimeout) fail(KNNG_ETIMEOUT, "a bounded device wait ran out");
    if (st & kStatusNonFinite) fail(KNNG_EINVAL, "data holds a non-finite value");
    if (st & kStatusBadInput) fail(KNNG_EINVAL, "an id or offset given by the caller is out of range");
    if (st & kStatusOverflow) fail(KNNG_ECUDA, "internal offer buffer overflow");
    if (st & kStatusInternal) fail(KNNG_ECUDA, "internal consistency check failed");
}

// Offer counting for the statistics: cleared before a call, read after it.
void offers_begin(BuildLayout& b, cudaStream_t s) {
    if (b.jb.offers_total) cuda_check(cudaMemsetAsync(b.jb.offers_total, 0, 8, s), "offer counter clear");
}
void offers_end(BuildLayout& b) {
    if (!b.jb.offers_total || !stats_on()) return;
    unsigned long long v = 0;
    cuda_check(cudaMemcpy(&v, b.jb.offers_total, 8, cudaMemcpyDeviceToHost), "offer counter read");
    record_items("k5_join", (double)v);
}

// Partition of one pass into perm_a (leaves contiguous).  Returns the buffer
// holding the result.
int32_t* run_partition(const float* X, const Args& a, const TreePlan& tp, BuildLayout& b, int pass, cudaStream_t s,
                       int q = 0) {
    const uint64_t ps = splitmix64(a.p.seed ^ (uint64_t)pass);
    const BuildLayout::PartSlot& sl = b.slot[q];
    // slot q's private buffers, the rest (copies of X, flags, status) shared
    SplitBuffers sb = b.sb;
    sb.W = sl.W;
    sb.S = sl.S;
    sb.thr = sl.thr;
    sb.S2 = sl.S2;
    sb.thr2 = sl.thr2;
    sb.st = sl.st;
    sb.ghist = sl.ghist;
    sb.ticket = sl.ticket;
    sb.partial = sl.partial;
    sb.segsum = sl.segsum;
    sb.segleft = sl.segleft;
    sb.tile_left = sl.tile_left;
    int32_t* pin = sl.perm_a;
    int32_t* pout = sl.perm_b;
    // the cross-CTA selection accumulates into these and leaves them zero
    cuda_check(cudaMemsetAsync(sb.ghist, 0, sizeof(uint32_t) * ((size_t)sb.nseg_large << kRadixBits), s),
               "histogram clear");
    cuda_check(cudaMemsetAsync(sb.ticket, 0, sizeof(uint32_t) * sb.nseg_large, s), "ticket clear");
    {
        LaunchScope ls("k_iota", s, a.n * 4.0, 0);
        k_iota<<<grid_1d(a.n), 256, 0, s>>>(pin, a.n);
    }
    for (int l = 0; l < tp.L; ++l) {
        run_split_level(X, a.D, tp.levels[l], a.p.twomeans_iters, ps, pin, pout, sb, s);
        std::swap(pin, pout);
    }
    return pin;
}

// Helper streams and events of one call (created and destroyed with it).
struct SideStreams {
    cudaStream_t h[BuildLayout::kPartSlots] = {};
    std::vector<cudaEvent_t> ev;
    int nh = 0;
    cudaEvent_t event() {
        cudaEvent_t e;
        cuda_check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event creation");
        ev.push_back(e);
        return e;
    }
    void make(int count) {
        for (; nh < count; ++nh) cuda_check(cudaStreamCreateWithFlags(&h[nh], cudaStreamNonBlocking), "stream creation");
    }
    ~SideStreams() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        for (int i = 0; i < nh; ++i) cudaStreamDestroy(h[i]);
    }
};

// The device work that reads X before the tree passes, over rows
// [r0, r0 + rows): the finiteness check, the original-order low-precision copy
// (norms, errors, exactness flag) and the byte copy (its flag).  The flags are
// cleared once, before the first piece.
void prepare_rows(const float* X, int64_t r0, int64_t rows, const Args& a, BuildLayout& b, cudaStream_t s) {
    const int D = a.D;
    launch_check_finite(X + r0 * D, rows * D, b.status, s);
    if (b.Xq) {
        const int qt = qtype(a.p.precision);
        launch_quantize(X + r0 * D, rows, D, nullptr, qt,
                        reinterpret_cast<uint8_t*>(b.Xq) + r0 * (int64_t)lp_row_bytes(D, qt), b.q_nrm + r0,
                        b.q_err + r0, b.q_scale ? b.q_scale + r0 : nullptr, b.notexact, s);
    }
    if (b.Xb) launch_bytes(X + r0 * D, rows, D, byte_dim(D), b.Xb + r0 * byte_dim(D), b.bflag, s);
}

// side: helper streams that outlive the call's stream capture (a recorded
// build); NULL: made here for this call.  up: the caller's rows when they are
// in host memory (up->dev is X): they are copied in pieces on a helper stream
// while the caller's stream prepares the pieces already in, so the work of
// prepare_rows hides under the copy, which the host link bounds.
void build_core(const float* X, const Args& a, BuildLayout& b, const TreePlan& tp, cudaStream_t s,
                SideStreams* side_in = nullptr, const DevBuf<float>* up = nullptr) {
    const int64_t n = a.n;
    const int k = a.p.k;
    launch_fill_empty(b.G, n * k, s);
    if (a.p.tree_passes > 0 && !b.jb.capture)  // a captured build has its plan uploaded beforehand
        cuda_check(cudaMemcpyAsync(b.plan_dev, tp.host.data(), tp.host.size() * 4, cudaMemcpyHostToDevice, s),
                   "plan upload");
    const bool lp = lp_leaf(a, tp);
    const int qt = qtype(a.p.precision);
    // re-ranked candidates per row: k plus a margin, at most 63
    const int kp = std::min(63, k + std::max(k / 2, 8));
    if (b.notexact) cuda_check(cudaMemsetAsync(b.notexact, 0, sizeof(int), s), "flag clear");
    if (b.Xb) cuda_check(cudaMemsetAsync(b.bflag, 0, sizeof(int), s), "flag clear");
    SideStreams side_local;
    SideStreams& side = side_in ? *side_in : side_local;
    if (up && up->host && up->count) {
        side.make(1);
        cudaStream_t cp = side.h[0];
        cudaEvent_t fork = side.event();
        cuda_check(cudaEventRecord(fork, s), "event record");
        cuda_check(cudaStreamWaitEvent(cp, fork, 0), "stream wait");
        // eight pieces of a multiple of 4 rows (16-byte aligned starts)
        const int64_t piece = std::max<int64_t>(4, ((n + 7) / 8 + 3) & ~(int64_t)3);
        for (int64_t r0 = 0; r0 < n; r0 += piece) {
            const int64_t rows = std::min(piece, n - r0);
            cuda_check(cudaMemcpyAsync(up->dev + r0 * a.D, up->host + r0 * a.D, (size_t)rows * a.D * sizeof(float),
                                       cudaMemcpyHostToDevice, cp),
                       "H2D copy");
            cudaEvent_t in = side.event();
            cuda_check(cudaEventRecord(in, cp), "event record");
            cuda_check(cudaStreamWaitEvent(s, in, 0), "stream wait");
            prepare_rows(X, r0, rows, a, b, s);
        }
    } else {
        if (up) upload(*const_cast<DevBuf<float>*>(up), s);
        prepare_rows(X, 0, n, a, b, s);
    }
    if (!b.jb.capture && (b.Xq || b.Xb)) {  // a graph records no host reads
        // the kernels pick their paths from the device flags; the host copies
        // pick the sums kernel and size the statistics' algorithmic bytes
        int f[2] = {0, 1};
        if (b.Xq) cuda_check(cudaMemcpyAsync(&f[0], b.notexact, sizeof(int), cudaMemcpyDeviceToHost, s), "flag read");
        if (b.Xb) cuda_check(cudaMemcpyAsync(&f[1], b.bflag, sizeof(int), cudaMemcpyDeviceToHost, s), "flag read");
        cuda_check(cudaStreamSynchronize(s), "stream synchronize");
        if (b.Xq) b.sb.q16_host = b.sb.Xq != nullptr && (f[0] & 1) == 0 && !((f[0] & 2) && (f[0] & 4));
        if (b.Xb) b.sb.u8_host = f[1] == 0;
    }
    // partitions: pass p on slot p % nslots (slot 0 on the caller's stream,
    // slot q > 0 on helper stream q - 1, forked from the caller's stream); a
    // slot's next partition waits for the leaf stage that read its last one
    const int P = a.p.tree_passes, Q = b.nslots;
    std::vector<int32_t*> perms((size_t)std::max(P, 0), nullptr);
    std::vector<cudaEvent_t> part_done((size_t)std::max(P, 0), nullptr), leaf_done((size_t)std::max(P, 0), nullptr);
    if (Q > 1 && P > 1) {
        side.make(Q - 1);
        cudaEvent_t fork = side.event();
        cuda_check(cudaEventRecord(fork, s), "event record");
        for (int q = 1; q < Q; ++q) cuda_check(cudaStreamWaitEvent(side.h[q - 1], fork, 0), "stream wait");
    }
    auto launch_partition = [&](int pass) {
        const int q = pass % Q;
        cudaStream_t ps = q == 0 ? s : side.h[q - 1];
        if (pass >= Q && q > 0) cuda_check(cudaStreamWaitEvent(ps, leaf_done[pass - Q], 0), "stream wait");
        perms[pass] = run_partition(X, a, tp, b, pass, ps, q);
        if (q > 0) {
            part_done[pass] = side.event();
            cuda_check(cudaEventRecord(part_done[pass], ps), "event record");
        }
    };
    for (int pass = 0; pass < std::min(P, Q); ++pass)
        if (pass % Q != 0) launch_partition(pass);
    for (int pass = 0; pass < P; ++pass) {
        if (pass % Q == 0) launch_partition(pass);  // slot 0: in order on the caller's stream
        else cuda_check(cudaStreamWaitEvent(s, part_done[pass], 0), "stream wait");
        int32_t* perm = perms[pass];
        const int32_t* leaf_off = b.plan_dev + tp.leaf_off_at;
        const int nleaf = (int)(tp.off[tp.L].size() - 1);
        bool done = false;
        if (lp) {
            launch_permute16(b.Xq, b.q_nrm, b.q_err, b.q_scale, n, lp_row_bytes(a.D, qt), perm, b.Xl, b.lp_nrm,
                             b.lp_err, b.lp_scale, s);
            done = launch_leaf_tc(b.Xl, n, X, a.D, perm, leaf_off, nleaf, tp.max_leaf, b.lp_nrm, b.lp_err,
                                  b.lp_scale, k, kp, qt, b.G, b.status, b.notexact, s);
        }
        if (!done) launch_leaf_fp32(X, a.D, perm, leaf_off, nleaf, tp.max_leaf, k, b.G, b.status, s);
        const int slot = pass - (a.p.tree_passes - b.jb.npass);
        if (b.lid && slot >= 0) launch_leaf_ids(perm, leaf_off, nleaf, n, slot, b.lid, s);
        // the next partition on this pass's slot may reuse its permutations
        if (pass + Q < P && (pass + Q) % Q != 0) {
            leaf_done[pass] = side.event();
            cuda_check(cudaEventRecord(leaf_done[pass], s), "event record");
            launch_partition(pass + Q);
        }
    }
    // the rounds take the nodes in the last tree pass's leaf order
    JoinBuffers jb = b.jb;
    jb.order = P > 0 ? perms[P - 1] : nullptr;
    if (a.p.join_mode == KNNG_JOIN_SAMPLED)
        run_refine_sampled(X, n, a.D, k, b.G, b.G2, jb, b.nodes_per_chunk, a.p.refine_rounds, a.p.sample,
                           a.p.seed, b.status, s);
    else
        run_refine(X, n, a.D, k, a.p.join_mode == KNNG_JOIN_FWD_REV, b.G, b.G2, jb, b.nodes_per_chunk,
                   a.p.refine_rounds, b.status, s);
}

}  // namespace
}  // namespace knng

using namespace knng;

extern "C" {

void knng_default_params(knng_params* p) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->k = 10;
    p->leaf_max = 64;
    p->tree_passes = 1;
    p->refine_rounds = 0;
    p->join_mode = KNNG_JOIN_FWD_REV;
    p->precision = KNNG_FP32;
    p->twomeans_iters = 4;
    p->seed = 0;
    p->sample = 0;
}

const char* knng_last_error(void) { return g_last_error.c_str(); }

int knng_tree_depth(int64_t n, int leaf_max) {
    if (n < 1 || leaf_max < 1) return -1;
    return tree_depth(n, leaf_max);
}

int knng_build_ex(const float* data, int64_t n, int D, const knng_params* p, int32_t* out_ids, float* out_dists,
                  void* stream) {
    return guarded([&] {
        if (!p) fail(KNNG_EINVAL, "params is NULL");
        validate_common(data, n, D, p->k);
        validate_params(p, n);
        if (!out_ids || !out_dists) fail(KNNG_EINVAL, "output pointer is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        Args a{n, D, *p};
        TreePlan tp;
        if (p->tree_passes > 0) tp.make(n, p->leaf_max);
        Workspace ws;
        BuildLayout b;
        DevBuf<float> X;
        DevBuf<int32_t> oi;
        DevBuf<float> od;
        const size_t nk = (size_t)n * p->k;
        for (int pass = 0; pass < 2; ++pass) {  // layout, then real pointers
            ws.used = 0;
            bind(ws, X, data, (size_t)n * D, pass);
            bind(ws, oi, out_ids, nk, pass);
            bind(ws, od, out_dists, nk, pass);
            carve(ws, b, a, tp, p->tree_passes > 0, p->refine_rounds > 0);
            if (pass == 0) ws.allocate(s);
        }
        if (p->tree_passes > 0) tp.rebase(b.plan_dev);
        cuda_check(cudaMemsetAsync(b.status, 0, 4 * sizeof(int), s), "status clear");
        offers_begin(b, s);
        build_core(X.dev, a, b, tp, s, nullptr, &X);
        launch_unpack(b.G, oi.dev, od.dev, (int64_t)nk, s);
        download(oi, s);
        download(od, s);
        cuda_check(launch_error(), "kernel launch");
        check_status(b.status, s,
                     lp_leaf(a, tp) ? leaf_kernel_name(p->precision) : nullptr);
        offers_end(b);
    });
}

}  // extern "C"

namespace {
// One group of batched instances (those of one D), concatenated into one
// forest: its parameters, tree plan, workspace, layout and where each
// instance's rows and lists lie.
struct Group {
    Args a;
    TreePlan tp;
    Workspace ws;
    BuildLayout b;
    float* X = nullptr;  // the instances' rows, concatenated
    int32_t* oi = nullptr;
    float* od = nullptr;
    std::vector<int> inst;
    std::vector<int64_t> first, sizes;
};

// Checks every instance before any device work; returns the instance
// indices grouped by D.
std::map<int, std::vector<int>> validate_batch(int n_inst, const knng_instance* inst, const knng_params* p) {
    if (!p) fail(KNNG_EINVAL, "params is NULL");
    if (n_inst < 1 || !inst) fail(KNNG_EINVAL, "n_inst = %d (need >= 1 and an instance array)", n_inst);
    std::map<int, std::vector<int>> by_dim;
    for (int i = 0; i < n_inst; ++i) {
        const knng_instance& in = inst[i];
        knng_params q = *p;
        if (in.leaf_max > 0) q.leaf_max = in.leaf_max;
        if (in.twomeans_iters > 0) q.twomeans_iters = in.twomeans_iters;
        try {
            if (in.twomeans_iters < 0) fail(KNNG_EINVAL, "twomeans_iters = %d < 0", in.twomeans_iters);
            validate_common(in.data, in.n, in.D, q.k);
            validate_params(&q, in.n);
            if (q.join_mode == KNNG_JOIN_SAMPLED && q.refine_rounds > 0)
                fail(KNNG_EINVAL, "batched builds do not take the sampled join");
            if (!in.out_ids || !in.out_dists) fail(KNNG_EINVAL, "output pointer is NULL");
        } catch (const Error& e) {
            const std::string msg = g_last_error;
            fail(e.code, "instance %d: %s", i, msg.c_str());
        }
        by_dim[in.D].push_back(i);
    }
    for (const auto& grp : by_dim) {  // one forest per D: one Lloyd schedule
        const int t0 = inst[grp.second[0]].twomeans_iters;
        for (int i : grp.second)
            if (inst[i].twomeans_iters != t0)
                fail(KNNG_EINVAL, "instances of D = %d differ in twomeans_iters (%d, %d)", grp.first, t0,
                     inst[i].twomeans_iters);
    }
    return by_dim;
}

// Sizes, tree plan and workspace of one group (offer budget: `budget`
// bytes, 0 = the default).
void setup_group(Group& g, int D, const std::vector<int>& ids, const knng_instance* inst, const knng_params* p,
                 size_t budget, cudaStream_t s) {
    const int k = p->k;
    std::vector<int> leafs;
    int64_t n = 0;
    g.inst = ids;
    for (int i : ids) {
        g.first.push_back(n);
        g.sizes.push_back(inst[i].n);
        leafs.push_back(inst[i].leaf_max > 0 ? inst[i].leaf_max : p->leaf_max);
        n += inst[i].n;
    }
    if (n >= ((int64_t)1 << 31) || n * (int64_t)k >= ((int64_t)1 << 31))
        fail(KNNG_EINVAL, "the instances of D = %d hold %lld points together (must stay below 2^31, "
             "and n * k too)", D, (long long)n);
    g.a = Args{n, D, *p};
    if (inst[ids[0]].twomeans_iters > 0) g.a.p.twomeans_iters = inst[ids[0]].twomeans_iters;
    g.a.offer_budget = budget;
    if (p->tree_passes > 0) g.tp.make_forest(g.sizes, leafs);
    const size_t nk = (size_t)n * k;
    for (int pass = 0; pass < 2; ++pass) {  // layout, then real pointers
        g.ws.used = 0;
        g.X = g.ws.take<float>((size_t)n * D);
        g.oi = g.ws.take<int32_t>(nk);
        g.od = g.ws.take<float>(nk);
        carve(g.ws, g.b, g.a, g.tp, p->tree_passes > 0, p->refine_rounds > 0);
        if (pass == 0) g.ws.allocate(s);
    }
    if (p->tree_passes > 0) g.tp.rebase(g.b.plan_dev);
}

// The group's device work: instance rows in, one forest build, every
// instance's lists (local ids) out.
void run_group(Group& g, const knng_instance* inst, cudaStream_t s, SideStreams* side = nullptr) {
    const int k = g.a.p.k, D = g.a.D;
    cuda_check(cudaMemsetAsync(g.b.status, 0, 4 * sizeof(int), s), "status clear");
    for (size_t t = 0; t < g.inst.size(); ++t)
        cuda_check(cudaMemcpyAsync(g.X + g.first[t] * D, inst[g.inst[t]].data, sizeof(float) * g.sizes[t] * D,
                                   cudaMemcpyDefault, s),
                   "instance copy");
    build_core(g.X, g.a, g.b, g.tp, s, side);
    for (size_t t = 0; t < g.inst.size(); ++t) {
        const knng_instance& in = inst[g.inst[t]];
        const size_t off = (size_t)g.first[t] * k, cnt = (size_t)g.sizes[t] * k;
        launch_unpack(g.b.G + off, g.oi + off, g.od + off, (int64_t)cnt, s, g.first[t]);
        cuda_check(cudaMemcpyAsync(in.out_ids, g.oi + off, cnt * 4, cudaMemcpyDefault, s), "ids copy");
        cuda_check(cudaMemcpyAsync(in.out_dists, g.od + off, cnt * 4, cudaMemcpyDefault, s), "dists copy");
    }
}
}  // namespace

extern "C" {

int knng_build_batched(int n_inst, const knng_instance* inst, const knng_params* p, void* stream) {
    return guarded([&] {
        const std::map<int, std::vector<int>> by_dim = validate_batch(n_inst, inst, p);
        cudaStream_t s = (cudaStream_t)stream;
        for (const auto& grp : by_dim) {
            Group g;
            setup_group(g, grp.first, grp.second, inst, p, 0, s);
            offers_begin(g.b, s);
            run_group(g, inst, s);
            cuda_check(launch_error(), "kernel launch");
            check_status(g.b.status, s, lp_leaf(g.a, g.tp) ? leaf_kernel_name(p->precision) : nullptr);
            offers_end(g.b);
        }
    });
}

}  // extern "C"

// A build recorded into a CUDA graph: its groups (one for a single build,
// one per D for a batch), each with its workspace and plan image, and the
// graph.
struct knng_plan {
    std::vector<std::unique_ptr<Group>> groups;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {
// Validation shared by the three residue-quantisation entries.
void validate_vocab(int W1, int W2, int D) {
    if (D < 1) fail(KNNG_EINVAL, "D = %d < 1", D);
    if (W1 < 1 || W1 > 256 || W2 < 1 || W2 > 256) fail(KNNG_EINVAL, "W1 = %d, W2 = %d outside [1, 256]", W1, W2);
}

// One stage of Lloyd's k-means on the device (Sec. 4.1): the vectors are the
// points, or their residues against W1 (codes c1) when W1 is given.
void rvq_lloyd(const float* X, int64_t N, int D, const float* W1, const int32_t* c1, int W, int iters,
               uint64_t seed, int stage, float* words, int32_t* codes, int32_t* order, int32_t* hist, int32_t* gofs,
               int32_t* scan_tmp, int64_t* dpos, std::vector<int64_t>& hpos, cudaStream_t s) {
    const uint64_t h0 = splitmix64(seed ^ ((uint64_t)stage << 32));
    hpos.assign(W, 0);
    for (int c = 0; c < W; ++c) {
        const int64_t lo = (int64_t)c * N / W, hi = (int64_t)(c + 1) * N / W;
        hpos[c] = lo + (int64_t)(splitmix64(h0 ^ (uint64_t)c) % (uint64_t)(hi - lo));
    }
    cuda_check(cudaMemcpyAsync(dpos, hpos.data(), sizeof(int64_t) * W, cudaMemcpyHostToDevice, s), "positions");
    launch_rvq_init(X, D, W1, c1, 1, dpos, W, words, s);
    const int nb = digit_sort_blocks(N);
    for (int it = 0; it < iters; ++it) {
        launch_rvq_assign(X, N, D, W1, c1, 1, words, W, codes, 1, s);
        launch_digit_sort(nullptr, N, codes, 1, order, hist, gofs, scan_tmp, s);
        launch_rvq_update(X, N, D, W1, c1, 1, order, gofs, nb, W, words, s);
    }
}
}  // namespace

namespace {
// Offer buffer of a recorded build: no host reads are possible in a graph,
// so the chunks are the worst case's size; one chunk per round when the
// worst case fits `cap` bytes.
size_t recorded_offer_budget(int64_t n, const knng_params* p, double cap) {
    const int64_t m = p->join_mode == KNNG_JOIN_FWD_REV ? 2 * p->k : p->k;
    const double worst = (double)n * std::max<int64_t>(m * (m - 1), 1) * 20.0;
    return (size_t)std::max<double>((double)offer_budget_bytes(), std::min(worst, cap));
}

// Records body(stream) into the plan's graph on a stream of its own, with
// the launch-time statistics off, and instantiates it.
template <class F>
void record_plan(knng_plan* pl, F&& body) {
    // helper streams for the concurrent partitions: made before and destroyed
    // after the capture they join
    SideStreams side;
    side.make(BuildLayout::kPartSlots - 1);
    cudaStream_t cs;
    cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "stream creation");
    const bool stats_were = stats_on();
    stats_set(false);
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        try {
            body(cs, &side);
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(cs, &g);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            stats_set(stats_were);
            throw;
        }
        e = cudaStreamEndCapture(cs, &pl->graph);
    }
    cudaStreamDestroy(cs);
    stats_set(stats_were);
    cuda_check(e, "stream capture");
    cuda_check(cudaGraphInstantiate(&pl->exec, pl->graph, 0), "graph instantiation");
}

// A group's workspace is allocated on the default stream (freed there at
// destroy); its tree plan is uploaded before recording; its kernels make
// every data-dependent choice on the device.
void prepare_recorded(Group& g) {
    cuda_check(cudaStreamSynchronize(nullptr), "workspace allocation");
    if (g.a.p.tree_passes > 0)
        cuda_check(cudaMemcpy(g.b.plan_dev, g.tp.host.data(), g.tp.host.size() * 4, cudaMemcpyHostToDevice),
                   "plan upload");
    g.b.jb.capture = true;
    g.b.sb.capture = true;
}
}  // namespace

extern "C" {

int knng_plan_create(const float* data, int64_t n, int D, const knng_params* p, int32_t* out_ids, float* out_dists,
                     void* stream, knng_plan** out_plan) {
    return guarded([&] {
        if (!out_plan) fail(KNNG_EINVAL, "out_plan is NULL");
        *out_plan = nullptr;
        if (!p) fail(KNNG_EINVAL, "params is NULL");
        validate_common(data, n, D, p->k);
        validate_params(p, n);
        if (!out_ids || !out_dists) fail(KNNG_EINVAL, "output pointer is NULL");
        const void* bufs[3] = {data, out_ids, out_dists};
        for (const void* q : bufs)
            if (!is_device_ptr(q) && !is_pinned_host_ptr(q))
                fail(KNNG_EINVAL, "a recorded build needs device or page-locked host buffers (data and outputs)");
        if (p->join_mode == KNNG_JOIN_SAMPLED && p->refine_rounds > 0)
            fail(KNNG_EINVAL, "a recorded build does not take the sampled join");
        // work the caller queued on `stream` (its inputs) completes first
        cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronize");
        std::unique_ptr<knng_plan> pl(new knng_plan());
        pl->groups.emplace_back(new Group());
        Group& g = *pl->groups[0];
        g.a = Args{n, D, *p};
        g.a.offer_budget = recorded_offer_budget(n, p, 48e9);
        if (p->tree_passes > 0) g.tp.make(n, p->leaf_max);
        // host buffers get workspace copies; the graph copies in and out
        DevBuf<float> X;
        DevBuf<int32_t> oi;
        DevBuf<float> od;
        const size_t nk = (size_t)n * p->k;
        for (int pass = 0; pass < 2; ++pass) {
            g.ws.used = 0;
            bind(g.ws, X, data, (size_t)n * D, pass);
            bind(g.ws, oi, out_ids, nk, pass);
            bind(g.ws, od, out_dists, nk, pass);
            carve(g.ws, g.b, g.a, g.tp, p->tree_passes > 0, p->refine_rounds > 0);
            if (pass == 0) g.ws.allocate(nullptr);
        }
        if (p->tree_passes > 0) g.tp.rebase(g.b.plan_dev);
        prepare_recorded(g);
        record_plan(pl.get(), [&](cudaStream_t cs, SideStreams* side) {
            cuda_check(cudaMemsetAsync(g.b.status, 0, 4 * sizeof(int), cs), "status clear");
            build_core(X.dev, g.a, g.b, g.tp, cs, side, &X);
            launch_unpack(g.b.G, oi.dev, od.dev, (int64_t)nk, cs);
            download(oi, cs);
            download(od, cs);
        });
        *out_plan = pl.release();
    });
}

int knng_plan_create_batched(int n_inst, const knng_instance* inst, const knng_params* p, void* stream,
                             knng_plan** out_plan) {
    return guarded([&] {
        if (!out_plan) fail(KNNG_EINVAL, "out_plan is NULL");
        *out_plan = nullptr;
        const std::map<int, std::vector<int>> by_dim = validate_batch(n_inst, inst, p);
        for (int i = 0; i < n_inst; ++i)
            if (!is_device_ptr(inst[i].data) || !is_device_ptr(inst[i].out_ids) || !is_device_ptr(inst[i].out_dists))
                fail(KNNG_EINVAL, "instance %d: a recorded build needs device buffers (data and outputs)", i);
        cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronize");
        std::unique_ptr<knng_plan> pl(new knng_plan());
        // the groups run one after another: each holds an equal share of the
        // 48 GB a recorded build may give its offers
        const double cap = 48e9 / (double)by_dim.size();
        for (const auto& grp : by_dim) {
            pl->groups.emplace_back(new Group());
            Group& g = *pl->groups.back();
            int64_t n = 0;
            for (int i : grp.second) n += inst[i].n;
            setup_group(g, grp.first, grp.second, inst, p, recorded_offer_budget(n, p, cap), nullptr);
            prepare_recorded(g);
        }
        // the instance array is read while recording only
        record_plan(pl.get(), [&](cudaStream_t cs, SideStreams* side) {
            for (auto& g : pl->groups) run_group(*g, inst, cs, side);
        });
        *out_plan = pl.release();
    });
}

int64_t knng_plan_kernels(knng_plan* plan) {
    if (!plan || !plan->graph) return -1;
    size_t nn = 0;
    if (cudaGraphGetNodes(plan->graph, nullptr, &nn) != cudaSuccess) return -1;
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn && cudaGraphGetNodes(plan->graph, nodes.data(), &nn) != cudaSuccess) return -1;
    int64_t kernels = 0;
    for (cudaGraphNode_t v : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(v, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
    }
    return kernels;
}

int knng_plan_launch(knng_plan* plan, void* stream) {
    return guarded([&] {
        if (!plan || !plan->exec) fail(KNNG_EINVAL, "no plan");
        cuda_check(cudaGraphLaunch(plan->exec, (cudaStream_t)stream), "graph launch");
    });
}

int knng_plan_check(knng_plan* plan, void* stream) {
    return guarded([&] {
        if (!plan) fail(KNNG_EINVAL, "no plan");
        for (auto& g : plan->groups) check_status(g->b.status, (cudaStream_t)stream);
    });
}

void knng_plan_destroy(knng_plan* plan) {
    if (!plan) return;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    delete plan;
}

int knng_build(const float* data, int64_t n, int D, int k, int leaf_max, int rounds, uint64_t seed,
               int32_t* out_ids, float* out_dists) {
    knng_params p;
    knng_default_params(&p);
    p.k = k;
    p.leaf_max = leaf_max;
    p.tree_passes = rounds;
    p.refine_rounds = 0;
    p.seed = seed;
    if (rounds < 1) {
        g_last_error = "rounds must be >= 1";
        return KNNG_EINVAL;
    }
    return knng_build_ex(data, n, D, &p, out_ids, out_dists, nullptr);
}

int knng_refine(const float* data, int64_t n, int D, const knng_params* p, int32_t* ids_inout,
                float* dists_inout, void* stream) {
    return guarded([&] {
        if (!p) fail(KNNG_EINVAL, "params is NULL");
        validate_common(data, n, D, p->k);
        knng_params q = *p;
        q.tree_passes = 1;  // validation of the join parameters only
        q.leaf_max = std::max(q.leaf_max, 2 * (q.k + 1));
        q.leaf_max = std::min(q.leaf_max, 256);
        validate_params(&q, n);
        if (!ids_inout || !dists_inout) fail(KNNG_EINVAL, "graph pointer is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        Args a{n, D, *p};
        a.p.tree_passes = 0;
        TreePlan tp;
        Workspace ws;
        BuildLayout b;
        DevBuf<float> X;
        DevBuf<int32_t> gi;
        DevBuf<float> gd;
        const size_t nk = (size_t)n * p->k;
        for (int pass = 0; pass < 2; ++pass) {
            ws.used = 0;
            bind(ws, X, data, (size_t)n * D, pass);
            bind(ws, gi, ids_inout, nk, pass);
            bind(ws, gd, dists_inout, nk, pass);
            carve(ws, b, a, tp, false, p->refine_rounds > 0);
            if (pass == 0) ws.allocate(s);
        }
        cuda_check(cudaMemsetAsync(b.status, 0, 4 * sizeof(int), s), "status clear");
        offers_begin(b, s);
        upload(X, s);
        upload(gi, s);
        upload(gd, s);
        launch_check_finite(X.dev, n * (int64_t)D, b.status, s);
        launch_pack(gi.dev, gd.dev, b.G, (int64_t)nk, n, b.status, s);
        if (b.notexact) cuda_check(cudaMemsetAsync(b.notexact, 0, sizeof(int), s), "flag clear");
        quantize_for_join(X.dev, a, b, s);
        if (p->join_mode == KNNG_JOIN_SAMPLED)
            run_refine_sampled(X.dev, n, D, p->k, b.G, b.G2, b.jb, b.nodes_per_chunk, p->refine_rounds, p->sample,
                               p->seed, b.status, s);
        else
            run_refine(X.dev, n, D, p->k, p->join_mode == KNNG_JOIN_FWD_REV, b.G, b.G2, b.jb, b.nodes_per_chunk,
                       p->refine_rounds, b.status, s);
        launch_unpack(b.G, gi.dev, gd.dev, (int64_t)nk, s);
        download(gi, s);
        download(gd, s);
        cuda_check(launch_error(), "kernel launch");
        check_status(b.status, s);
        offers_end(b);
    });
}

int knng_partition(const float* data, int64_t n, int D, int leaf_max, int twomeans_iters, uint64_t seed, int pass,
                   int32_t* out_perm, int64_t* out_leaf_offsets, void* stream) {
    return guarded([&] {
        if (!data || !out_perm || !out_leaf_offsets) fail(KNNG_EINVAL, "NULL pointer");
        if (D < 1 || D > 4096) fail(KNNG_EINVAL, "D = %d out of range [1, 4096]", D);
        if (n < 1 || n >= ((int64_t)1 << 31)) fail(KNNG_EINVAL, "n = %lld out of range", (long long)n);
        if (leaf_max < 2) fail(KNNG_EINVAL, "leaf_max = %d < 2", leaf_max);
        if (twomeans_iters < 0 || twomeans_iters > 64) fail(KNNG_EINVAL, "twomeans_iters out of range");
        if (pass < 0) fail(KNNG_EINVAL, "pass < 0");
        cudaStream_t s = (cudaStream_t)stream;
        Args a{n, D, {}};
        knng_default_params(&a.p);
        a.p.k = 1;
        a.p.leaf_max = leaf_max;
        a.p.twomeans_iters = twomeans_iters;
        a.p.seed = seed;
        TreePlan tp;
        tp.make(n, leaf_max);
        Workspace ws;
        BuildLayout b;
        DevBuf<float> X;
        DevBuf<int32_t> op;
        const size_t noff = tp.off[tp.L].size();
        for (int ps = 0; ps < 2; ++ps) {
            ws.used = 0;
            bind(ws, X, data, (size_t)n * D, ps);
            bind(ws, op, out_perm, (size_t)n, ps);
            carve(ws, b, a, tp, true, false);
            if (ps == 0) ws.allocate(s);
        }
        tp.rebase(b.plan_dev);
        cuda_check(cudaMemsetAsync(b.status, 0, 4 * sizeof(int), s), "status clear");
        upload(X, s);
        launch_check_finite(X.dev, n * (int64_t)D, b.status, s);
        cuda_check(cudaMemcpyAsync(b.plan_dev, tp.host.data(), tp.host.size() * 4, cudaMemcpyHostToDevice, s),
                   "plan upload");
        make_bytes(X.dev, a, b, s);
        int32_t* perm = run_partition(X.dev, a, tp, b, pass, s);
        cuda_check(cudaMemcpyAsync(op.dev, perm, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s), "perm copy");
        download(op, s);
        std::vector<int64_t> off(tp.off[tp.L].begin(), tp.off[tp.L].end());
        if (is_device_ptr(out_leaf_offsets))
            cuda_check(cudaMemcpyAsync(out_leaf_offsets, off.data(), noff * 8, cudaMemcpyHostToDevice, s),
                       "offsets copy");
        else
            memcpy(out_leaf_offsets, off.data(), noff * 8);
        cuda_check(launch_error(), "kernel launch");
        check_status(b.status, s);
    });
}

int knng_leaf_dhat(const float* data, int64_t m, int D, int precision, float* out_dhat, float* out_q,
                   float* out_scale, float* out_nrm, float* out_err, void* stream) {
    return guarded([&] {
        if (!data || !out_dhat || !out_q || !out_scale || !out_nrm || !out_err) fail(KNNG_EINVAL, "NULL pointer");
        if (m < 2 || m > 256) fail(KNNG_EINVAL, "m = %lld outside [2, 256]", (long long)m);
        if (D < 1 || D > 4096) fail(KNNG_EINVAL, "D = %d out of range [1, 4096]", D);
        if (precision != KNNG_BF16 && precision != KNNG_FP16 && precision != KNNG_FP8)
            fail(KNNG_EINVAL, "precision = %d is not a low-precision form", precision);
        const int qt = qtype(precision);
        cudaStream_t s = (cudaStream_t)stream;
        Workspace ws;
        DevBuf<float> X, dh, q, sc, nr, er;
        uint16_t* Xq = nullptr;
        int32_t *perm = nullptr, *off = nullptr;
        int *status = nullptr, *notexact = nullptr;
        uint64_t* G = nullptr;
        for (int ps = 0; ps < 2; ++ps) {
            ws.used = 0;
            bind(ws, X, data, (size_t)m * D, ps);
            bind(ws, dh, out_dhat, (size_t)m * m, ps);
            bind(ws, q, out_q, (size_t)m * D, ps);
            bind(ws, sc, out_scale, (size_t)m, ps);
            bind(ws, nr, out_nrm, (size_t)m, ps);
            bind(ws, er, out_err, (size_t)m, ps);
            Xq = ws.take<uint16_t>((size_t)m * lp_row_bytes(D, qt) / 2);
            perm = ws.take<int32_t>(m);
            off = ws.take<int32_t>(2);
            status = ws.take<int>(4);
            notexact = ws.take<int>(4);
            G = ws.take<uint64_t>(m);
            if (ps == 0) ws.allocate(s);
        }
        cuda_check(cudaMemsetAsync(status, 0, 4 * sizeof(int), s), "status clear");
        cuda_check(cudaMemsetAsync(notexact, 0, 4 * sizeof(int), s), "flag clear");
        const int32_t hoff[2] = {0, (int32_t)m};
        cuda_check(cudaMemcpyAsync(off, hoff, sizeof hoff, cudaMemcpyHostToDevice, s), "offsets");
        upload(X, s);
        launch_check_finite(X.dev, m * (int64_t)D, status, s);
        {
            LaunchScope ls("k_iota", s, m * 4.0, 0);
            k_iota<<<1, 256, 0, s>>>(perm, m);
        }
        // scales: FP8 writes them; 16-bit copies have none (1)
        if (qt != 2) launch_fill_value(sc.dev, m, 1.f, s);
        launch_quantize(X.dev, m, D, nullptr, qt, Xq, nr.dev, er.dev, qt == 2 ? sc.dev : nullptr, notexact, s);
        if (!launch_leaf_tc(Xq, m, X.dev, D, perm, off, 1, (int)m, nr.dev, er.dev, qt == 2 ? sc.dev : nullptr, 1, 1,
                            qt, G, status, notexact, s, dh.dev))
            fail(KNNG_ECUDA, "the tensor-core leaf kernel cannot run for D = %d", D);
        launch_lp_to_float(Xq, m, D, qt, q.dev, s);
        download(dh, s);
        download(q, s);
        download(sc, s);
        download(nr, s);
        download(er, s);
        cuda_check(launch_error(), "kernel launch");
        check_status(status, s);
    });
}

int knng_leaf_update(const float* data, int64_t n, int D, int k, const int32_t* perm, const int64_t* leaf_offsets,
                     int64_t n_leaves, int32_t* ids_inout, float* dists_inout, void* stream) {
    return guarded([&] {
        validate_common(data, n, D, k);
        if (!perm || !leaf_offsets || !ids_inout || !dists_inout) fail(KNNG_EINVAL, "NULL pointer");
        if (n_leaves < 0) fail(KNNG_EINVAL, "n_leaves < 0");
        cudaStream_t s = (cudaStream_t)stream;
        std::vector<int64_t> off((size_t)n_leaves + 1);
        if (is_device_ptr(leaf_offsets)) {
            cuda_check(cudaMemcpyAsync(off.data(), leaf_offsets, off.size() * 8, cudaMemcpyDeviceToHost, s),
                       "offsets read");
            cuda_check(cudaStreamSynchronize(s), "stream synchronize");
        } else {
            memcpy(off.data(), leaf_offsets, off.size() * 8);
        }
        int max_leaf = 0;
        for (int64_t l = 0; l < n_leaves; ++l) {
            const int64_t m = off[l + 1] - off[l];
            if (m < 0 || m > 256 || off[l] < 0 || off[l + 1] > n)
                fail(KNNG_EINVAL, "leaf %lld has bad offsets", (long long)l);
            max_leaf = std::max<int>(max_leaf, (int)m);
        }
        std::vector<int32_t> off32(off.begin(), off.end());
        Workspace ws;
        DevBuf<float> X;
        DevBuf<int32_t> pm, gi;
        DevBuf<float> gd;
        uint64_t* G = nullptr;
        int32_t* doff = nullptr;
        int* status = nullptr;
        const size_t nk = (size_t)n * k;
        for (int ps = 0; ps < 2; ++ps) {
            ws.used = 0;
            bind(ws, X, data, (size_t)n * D, ps);
            bind(ws, pm, perm, (size_t)n, ps);
            bind(ws, gi, ids_inout, nk, ps);
            bind(ws, gd, dists_inout, nk, ps);
            G = ws.take<uint64_t>(nk);
            doff = ws.take<int32_t>(off32.size());
            status = ws.take<int>(4);
            if (ps == 0) ws.allocate(s);
        }
        cuda_check(cudaMemsetAsync(status, 0, 4 * sizeof(int), s), "status clear");
        upload(X, s);
        upload(pm, s);
        upload(gi, s);
        upload(gd, s);
        cuda_check(cudaMemcpyAsync(doff, off32.data(), off32.size() * 4, cudaMemcpyHostToDevice, s), "offsets");
        launch_check_finite(X.dev, n * (int64_t)D, status, s);
        launch_pack(gi.dev, gd.dev, G, (int64_t)nk, n, status, s);
        launch_check_ids(pm.dev, n, 0, n, status, s);
        if (n_leaves > 0 && max_leaf >= 2)
            launch_leaf_fp32(X.dev, D, pm.dev, doff, (int)n_leaves, max_leaf, k, G, status, s);
        launch_unpack(G, gi.dev, gd.dev, (int64_t)nk, s);
        download(gi, s);
        download(gd, s);
        cuda_check(launch_error(), "kernel launch");
        check_status(status, s);
    });
}

int knng_search(const float* data, int64_t n, int D, const int32_t* graph_ids, int k, const float* queries,
                int64_t m, const int32_t* seeds, int s, int t0, int ks, int32_t* out_ids, float* out_dists,
                void* stream) {
    return guarded([&] {
        if (!data || n < 1 || D < 1) fail(KNNG_EINVAL, "data, n or D invalid");
        if (!graph_ids || k < 1) fail(KNNG_EINVAL, "graph_ids NULL or k < 1");
        if (m < 0 || s < 0 || t0 < 0) fail(KNNG_EINVAL, "m, s or t0 negative");
        if (ks < 1 || ks > 32) fail(KNNG_EINVAL, "ks = %d out of range [1, 32]", ks);
        if ((size_t)4 * D * sizeof(float) > 200 * 1024) fail(KNNG_EINVAL, "D = %d too large for the search", D);
        if (m == 0) return;
        if (!queries || !out_ids || !out_dists || (s > 0 && !seeds)) fail(KNNG_EINVAL, "a pointer is NULL");
        cudaStream_t st = (cudaStream_t)stream;
        const int cl = search_cap_log2(s, t0, ks, k);
        // queries per launch: their visited tables within 1 GiB
        const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(m, ((int64_t)1 << 28) >> cl));
        Workspace ws;
        DevBuf<float> X, Qb;
        DevBuf<int32_t> Gb, Sb, oi;
        DevBuf<float> od;
        int32_t* tab = nullptr;
        int* status = nullptr;
        for (int ps = 0; ps < 2; ++ps) {
            ws.used = 0;
            bind(ws, X, data, (size_t)n * D, ps);
            bind(ws, Gb, graph_ids, (size_t)n * k, ps);
            bind(ws, Qb, queries, (size_t)m * D, ps);
            if (s > 0) bind(ws, Sb, seeds, (size_t)m * s, ps);
            bind(ws, oi, out_ids, (size_t)m * ks, ps);
            bind(ws, od, out_dists, (size_t)m * ks, ps);
            tab = ws.take<int32_t>((size_t)chunk << cl);
            status = ws.take<int>(4);
            if (ps == 0) ws.allocate(st);
        }
        cuda_check(cudaMemsetAsync(status, 0, 4 * sizeof(int), st), "status clear");
        upload(X, st);
        upload(Gb, st);
        upload(Qb, st);
        if (s > 0) upload(Sb, st);
        launch_check_finite(X.dev, n * (int64_t)D, status, st);
        launch_check_finite(Qb.dev, m * (int64_t)D, status, st);
        for (int64_t q0 = 0; q0 < m; q0 += chunk)
            launch_search(X.dev, n, D, Gb.dev, k, Qb.dev, q0, std::min(m, q0 + chunk), s > 0 ? Sb.dev : nullptr, s,
                          t0, ks, tab, cl, oi.dev, od.dev, st);
        download(oi, st);
        download(od, st);
        cuda_check(launch_error(), "kernel launch");
        check_status(status, st);
    });
}

int knng_rvq_train(const float* data, int64_t n, int D, int W1, int W2, int iters, uint64_t seed, float* words1,
                   float* words2, void* stream) {
    return guarded([&] {
        validate_vocab(W1, W2, D);
        if (!data || n < 1 || n > INT32_MAX) fail(KNNG_EINVAL, "data NULL or n out of range");
        if (W1 > n || W2 > n) fail(KNNG_EINVAL, "more words than points");
        if (iters < 0) fail(KNNG_EINVAL, "iters < 0");
        if (!words1 || !words2) fail(KNNG_EINVAL, "an output pointer is NULL");
        cudaStream_t st = (cudaStream_t)stream;
        const size_t nh = digit_sort_hist_ints(n);
        Workspace ws;
        DevBuf<float> X, o1, o2;
        int32_t *codes = nullptr, *c1 = nullptr, *order = nullptr, *hist = nullptr, *gofs = nullptr, *tmp = nullptr;
        int64_t* pos = nullptr;
        float* R = nullptr;
        int* status = nullptr;
        for (int ps = 0; ps < 2; ++ps) {
            ws.used = 0;
            bind(ws, X, data, (size_t)n * D, ps);
            R = ws.take<float>((size_t)n * D);
            bind(ws, o1, (const float*)words1, (size_t)W1 * D, ps);
            bind(ws, o2, (const float*)words2, (size_t)W2 * D, ps);
            codes = ws.take<int32_t>(n);
            c1 = ws.take<int32_t>(n);
            order = ws.take<int32_t>(n);
            hist = ws.take<int32_t>(nh);
            gofs = ws.take<int32_t>(nh + 1);
            tmp = ws.take<int32_t>(scan_tmp_ints((int64_t)nh));
            pos = ws.take<int64_t>(256);
            status = ws.take<int>(4);
            if (ps == 0) ws.allocate(st);
        }
        cuda_check(cudaMemsetAsync(status, 0, 4 * sizeof(int), st), "status clear");
        upload(X, st);
        launch_check_finite(X.dev, n * (int64_t)D, status, st);
        std::vector<int64_t> hpos;
        rvq_lloyd(X.dev, n, D, nullptr, nullptr, W1, iters, seed, 1, o1.dev, codes, order, hist, gofs, tmp, pos, hpos,
                  st);
        launch_rvq_assign(X.dev, n, D, nullptr, nullptr, 1, o1.dev, W1, c1, 1, st);
        launch_rvq_residues(X.dev, n, D, o1.dev, c1, R, st);   // stage 2 trains on the residues
        rvq_lloyd(R, n, D, nullptr, nullptr, W2, iters, seed, 2, o2.dev, codes, order, hist, gofs, tmp, pos, hpos, st);
        download(o1, st);
        download(o2, st);
        cuda_check(launch_error(), "kernel launch");
        check_status(status, st);
    });
}

int knng_rvq_index(const float* data, int64_t n, int D, const float* words1, int W1, const float* words2, int W2,
                   int32_t* codes, int32_t* list_offsets, int32_t* list_ids, void* stream) {
    return guarded([&] {
        validate_vocab(W1, W2, D);
        if (!data || n < 1 || n > INT32_MAX) fail(KNNG_EINVAL, "data NULL or n out of range");
        if (!words1 || !words2 || !codes || !list_offsets || !list_ids) fail(KNNG_EINVAL, "a pointer is NULL");
        cudaStream_t st = (cudaStream_t)stream;
        const int64_t nk = (int64_t)W1 * W2;
        const size_t nh = digit_sort_hist_ints(n);
        Workspace ws;
        DevBuf<float> X, w1, w2;
        DevBuf<int32_t> cd, off, li;
        int32_t *order = nullptr, *hist = nullptr, *gofs = nullptr, *tmp = nullptr, *cnt = nullptr;
        int* status = nullptr;
        for (int ps = 0; ps < 2; ++ps) {
            ws.used = 0;
            bind(ws, X, data, (size_t)n * D, ps);
            bind(ws, w1, words1, (size_t)W1 * D, ps);
            bind(ws, w2, words2, (size_t)W2 * D, ps);
            bind(ws, cd, (const int32_t*)codes, (size_t)n * 2, ps);
            bind(ws, off, (const int32_t*)list_offsets, (size_t)nk + 1, ps);
            bind(ws, li, (const int32_t*)list_ids, (size_t)n, ps);
            order = ws.take<int32_t>(n);
            hist = ws.take<int32_t>(nh);
            gofs = ws.take<int32_t>(nh + 1);
            tmp = ws.take<int32_t>(std::max(scan_tmp_ints((int64_t)nh), scan_tmp_ints(nk)));
            cnt = ws.take<int32_t>(nk);
            status = ws.take<int>(4);
            if (ps == 0) ws.allocate(st);
        }
        cuda_check(cudaMemsetAsync(status, 0, 4 * sizeof(int), st), "status clear");
        upload(X, st);
        upload(w1, st);
        upload(w2, st);
        launch_check_finite(X.dev, n * (int64_t)D, status, st);
        launch_check_finite(w1.dev, (int64_t)W1 * D, status, st);
        launch_check_finite(w2.dev, (int64_t)W2 * D, status, st);
        launch_rvq_assign(X.dev, n, D, nullptr, nullptr, 2, w1.dev, W1, cd.dev, 2, st);
        launch_rvq_assign(X.dev, n, D, w1.dev, cd.dev, 2, w2.dev, W2, cd.dev + 1, 2, st);
        launch_digit_sort(nullptr, n, cd.dev + 1, 2, order, hist, gofs, tmp, st);   // by c2
        launch_digit_sort(order, n, cd.dev, 2, li.dev, hist, gofs, tmp, st);        // then by c1, stable
        cuda_check(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * nk, st), "count clear");
        launch_rvq_key_count(cd.dev, n, W2, cnt, st);
        launch_scan(cnt, off.dev, nk, tmp, st);
        download(cd, st);
        download(off, st);
        download(li, st);
        cuda_check(launch_error(), "kernel launch");
        check_status(status, st);
    });
}

int knng_rvq_seeds(const float* words1, int W1, const float* words2, int W2, int D, const int32_t* list_offsets,
                   const int32_t* list_ids, int64_t n, const float* queries, int64_t m, int probe1, int s,
                   int32_t* seeds, void* stream) {
    return guarded([&] {
        validate_vocab(W1, W2, D);
        if (n < 0 || n > INT32_MAX || m < 0 || m > INT32_MAX || s < 0) fail(KNNG_EINVAL, "n, m or s out of range");
        if (probe1 < 1 || probe1 > W1) fail(KNNG_EINVAL, "probe1 = %d outside [1, W1]", probe1);
        if (probe1 * W2 > 8192) fail(KNNG_EINVAL, "probe1 * W2 = %d above 8192", probe1 * W2);
        if (rvq_seeds_smem(probe1, W2, D) > 200 * 1024) fail(KNNG_EINVAL, "D = %d too large for the seeds", D);
        if (m == 0 || s == 0) return;
        if (!words1 || !words2 || !list_offsets || (n > 0 && !list_ids) || !queries || !seeds)
            fail(KNNG_EINVAL, "a pointer is NULL");
        cudaStream_t st = (cudaStream_t)stream;
        const int64_t nk = (int64_t)W1 * W2;
        Workspace ws;
        DevBuf<float> w1, w2, Qb;
        DevBuf<int32_t> off, li, Sb;
        float *n1 = nullptr, *n2 = nullptr, *x12 = nullptr, *w1T = nullptr, *w2T = nullptr;
        int* status = nullptr;
        for (int ps = 0; ps < 2; ++ps) {
            ws.used = 0;
            bind(ws, w1, words1, (size_t)W1 * D, ps);
            bind(ws, w2, words2, (size_t)W2 * D, ps);
            bind(ws, off, list_offsets, (size_t)nk + 1, ps);
            bind(ws, li, list_ids, (size_t)n, ps);
            bind(ws, Qb, queries, (size_t)m * D, ps);
            bind(ws, Sb, (const int32_t*)seeds, (size_t)m * s, ps);
            n1 = ws.take<float>(W1);
            n2 = ws.take<float>(W2);
            x12 = ws.take<float>((size_t)nk);
            w1T = ws.take<float>((size_t)W1 * D);
            w2T = ws.take<float>((size_t)W2 * D);
            status = ws.take<int>(4);
            if (ps == 0) ws.allocate(st);
        }
        cuda_check(cudaMemsetAsync(status, 0, 4 * sizeof(int), st), "status clear");
        upload(w1, st);
        upload(w2, st);
        upload(off, st);
        upload(li, st);
        upload(Qb, st);
        launch_check_finite(w1.dev, (int64_t)W1 * D, status, st);
        launch_check_finite(w2.dev, (int64_t)W2 * D, status, st);
        launch_check_finite(Qb.dev, m * (int64_t)D, status, st);
        launch_check_offsets(off.dev, nk, n, status, st);
        launch_rvq_tables(w1.dev, W1, w2.dev, W2, D, n1, n2, x12, w1T, w2T, st);
        launch_rvq_seeds(w1T, W1, w2T, W2, D, n1, n2, x12, off.dev, li.dev, Qb.dev, m, probe1, s, Sb.dev, status, st);
        download(Sb, st);
        cuda_check(launch_error(), "kernel launch");
        check_status(status, st);
    });
}

int knng_exact(const float* data, int64_t n, int D, int k, const int32_t* sample, int64_t s_rows, int32_t* out_ids,
               float* out_dists, void* stream) {
    return guarded([&] {
        validate_common(data, n, D, k);
        if (s_rows < 0) fail(KNNG_EINVAL, "s < 0");
        if (s_rows == 0) return;  // nothing to compute (empty buffers may be NULL)
        if (!out_ids || !out_dists) fail(KNNG_EINVAL, "output pointer is NULL");
        if (!sample && s_rows != n) fail(KNNG_EINVAL, "without a sample s must equal n");
        cudaStream_t s = (cudaStream_t)stream;
        Workspace ws;
        DevBuf<float> X;
        DevBuf<int32_t> smp, oi;
        DevBuf<float> od;
        uint64_t* keys = nullptr;
        int* status = nullptr;
        const size_t sk = (size_t)s_rows * k;
        for (int ps = 0; ps < 2; ++ps) {
            ws.used = 0;
            bind(ws, X, data, (size_t)n * D, ps);
            if (sample) bind(ws, smp, sample, (size_t)s_rows, ps);
            bind(ws, oi, out_ids, sk, ps);
            bind(ws, od, out_dists, sk, ps);
            keys = ws.take<uint64_t>(std::max<size_t>(sk, 1));
            status = ws.take<int>(4);
            if (ps == 0) ws.allocate(s);
        }
        cuda_check(cudaMemsetAsync(status, 0, 4 * sizeof(int), s), "status clear");
        upload(X, s);
        if (sample) upload(smp, s);
        launch_check_finite(X.dev, n * (int64_t)D, status, s);
        if (s_rows > 0) {
            if (sample) launch_check_ids(smp.dev, s_rows, 0, n, status, s);
            launch_exact(X.dev, n, D, k, sample ? smp.dev : nullptr, s_rows, keys, status, s);
            launch_unpack(keys, oi.dev, od.dev, (int64_t)sk, s);
        }
        download(oi, s);
        download(od, s);
        cuda_check(launch_error(), "kernel launch");
        check_status(status, s);
    });
}

int knng_recall(const int32_t* ids, const float* dists, const int32_t* gt_ids, const float* gt_dists,
                const int32_t* sample, int64_t s_rows, int k, double* out_recall_ids, double* out_recall_tie,
                void* stream) {
    return guarded([&] {
        if (!out_recall_ids || !out_recall_tie) fail(KNNG_EINVAL, "NULL output pointer");
        if (k < 1 || k > 64) fail(KNNG_EINVAL, "k out of range");
        if (s_rows < 0) fail(KNNG_EINVAL, "s < 0");
        if (s_rows == 0) {  // no rows: recall is defined as 0
            *out_recall_ids = *out_recall_tie = 0.0;
            return;
        }
        if (!ids || !dists || !gt_ids || !gt_dists || !sample) fail(KNNG_EINVAL, "NULL pointer");
        cudaStream_t s = (cudaStream_t)stream;
        const size_t sk = (size_t)s_rows * k;
        // host graphs: gather the sampled rows on the host (marshalling only)
        std::vector<int32_t> hids, hsmp;
        std::vector<float> hd;
        const bool dev = is_device_ptr(ids);
        if (!dev) {
            std::vector<int32_t> sm((size_t)s_rows);
            if (is_device_ptr(sample)) {
                cuda_check(cudaMemcpy(sm.data(), sample, s_rows * 4, cudaMemcpyDeviceToHost), "sample read");
            } else {
                memcpy(sm.data(), sample, s_rows * 4);
            }
            hids.resize(sk);
            hd.resize(sk);
            hsmp.resize((size_t)s_rows);
            for (int64_t r = 0; r < s_rows; ++r) {
                memcpy(&hids[r * k], ids + (size_t)sm[r] * k, 4 * k);
                memcpy(&hd[r * k], dists + (size_t)sm[r] * k, 4 * k);
                hsmp[r] = (int32_t)r;
            }
        }
        Workspace ws;
        DevBuf<int32_t> di, gi, smp;
        DevBuf<float> dd, gd;
        unsigned long long* counts = nullptr;
        for (int ps = 0; ps < 2; ++ps) {
            ws.used = 0;
            if (dev) {
                di.dev = const_cast<int32_t*>(ids);
                dd.dev = const_cast<float*>(dists);
                bind(ws, smp, sample, (size_t)s_rows, ps);
            } else {
                bind(ws, di, hids.data(), sk, ps);
                bind(ws, dd, hd.data(), sk, ps);
                bind(ws, smp, hsmp.data(), (size_t)s_rows, ps);
            }
            bind(ws, gi, gt_ids, sk, ps);
            bind(ws, gd, gt_dists, sk, ps);
            counts = ws.take<unsigned long long>(2);
            if (ps == 0) ws.allocate(s);
        }
        if (!dev) {
            upload(di, s);
            upload(dd, s);
        }
        upload(smp, s);
        upload(gi, s);
        upload(gd, s);
        launch_recall(di.dev, dd.dev, gi.dev, gd.dev, smp.dev, s_rows, k, counts, s);
        unsigned long long hc[2] = {0, 0};
        cuda_check(cudaMemcpyAsync(hc, counts, sizeof hc, cudaMemcpyDeviceToHost, s), "counts read");
        cuda_check(launch_error(), "kernel launch");
        cuda_check(cudaStreamSynchronize(s), "stream synchronize");
        reg().flush();
        const double denom = (double)s_rows * k;
        *out_recall_ids = s_rows ? hc[0] / denom : 0.0;
        *out_recall_tie = s_rows ? hc[1] / denom : 0.0;
    });
}

size_t knng_workspace_bytes(int64_t n, int D, const knng_params* p) {
    size_t out = 0;
    guarded([&] {
        validate_common((const void*)1, n, D, p ? p->k : 0);
        validate_params(p, n);
        Args a{n, D, *p};
        TreePlan tp;
        if (p->tree_passes > 0) tp.make(n, p->leaf_max);
        Workspace ws;
        BuildLayout b;
        carve(ws, b, a, tp, p->tree_passes > 0, p->refine_rounds > 0);
        out = ws.used;
    });
    return out;
}

int knng_stats_enable(int on, int timing) {
    StatRegistry& r = reg();
    std::lock_guard<std::mutex> lk(r.mu);
    r.on = on != 0;
    r.timing = on != 0 && timing != 0;
    return KNNG_OK;
}

void knng_stats_reset(void) {
    StatRegistry& r = reg();
    std::lock_guard<std::mutex> lk(r.mu);
    r.stats.clear();
}

int knng_stats_count(void) {
    StatRegistry& r = reg();
    std::lock_guard<std::mutex> lk(r.mu);
    return (int)r.stats.size();
}

int knng_stats_get(int index, knng_kernel_stat* out) {
    StatRegistry& r = reg();
    std::lock_guard<std::mutex> lk(r.mu);
    if (!out || index < 0 || index >= (int)r.stats.size()) return KNNG_EINVAL;
    auto it = r.stats.begin();
    std::advance(it, index);
    *out = it->second;
    return KNNG_OK;
}

}  // extern "C"
