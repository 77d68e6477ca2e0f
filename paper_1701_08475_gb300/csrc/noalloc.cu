// noalloc.cu -- knng_exact_noalloc: exact neighbour lists without any device
// allocation.
//
// Some callers cannot allocate device memory at the point where they need
// ground-truth lists: code that runs under a memory manager owning all of the
// device's memory (a cudaMalloc there fails or escapes its accounting), or a
// latency-bound loop in which the implicit synchronisation of an allocation
// is not allowed.  This entry point serves them: its only scratch (the
// packed lists and a status word) lives in the file-scope device arrays
// below, which every GPU that loads the library holds until the process
// exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace knng {

void record_error(const char* msg);

namespace {

// Largest s * k one call may request: 2^18 list entries (2 MiB of keys).
constexpr int64_t kNoAllocMaxEntries = int64_t(1) << 18;

static __device__ __align__(256) uint64_t g_noalloc_keys[kNoAllocMaxEntries];
static __device__ __align__(256) int g_noalloc_status;

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
bool g_ready[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};
uint64_t* g_keys_addr[kMaxDevices] = {};
int* g_status_addr[kMaxDevices] = {};

// The unique id of the current context (cuCtxGetId through the runtime's
// driver entry points, so the library needs no link to libcuda).  A device
// reset destroys the context and the next runtime call makes a new one with
// a new id, into which the module (and so the scratch) is loaded afresh.
bool current_context_id(unsigned long long* id) {
    typedef CUresult (*get_current_fn)(CUcontext*);
    typedef CUresult (*get_id_fn)(CUcontext, unsigned long long*);
    static get_current_fn get_current = nullptr;
    static get_id_fn get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<get_current_fn>(f1);
            get_id = reinterpret_cast<get_id_fn>(f2);
        }
        cudaGetLastError();
        looked = true;
    }
    if (!get_current || !get_id) return false;
    CUcontext c = nullptr;
    return get_current(&c) == CUDA_SUCCESS && c != nullptr && get_id(c, id) == CUDA_SUCCESS;
}

// Device addresses of the scratch arrays in the current device's context.
// The set-up (cudaGetSymbolAddress with the device current) runs on the
// first call on a device, and again on the first call after that device's
// context was replaced (cudaDeviceReset), whose module holds a new copy of
// the arrays; otherwise the cached addresses serve.
bool scratch_for_current_device(uint64_t** keys, int** status, const char** why) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        *why = "no usable current CUDA device";
        return false;
    }
    // makes the device's primary context current (creating it after a
    // reset), so that its id can be read
    if (cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        *why = "the device's context could not be made current";
        return false;
    }
    unsigned long long ctx = 0;
    if (!current_context_id(&ctx)) {
        *why = "the current context's id could not be read";
        return false;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_ready[dev] || g_ctx_id[dev] != ctx) {
        g_ready[dev] = false;
        void* k = nullptr;
        void* s = nullptr;
        if (cudaGetSymbolAddress(&k, g_noalloc_keys) != cudaSuccess ||
            cudaGetSymbolAddress(&s, g_noalloc_status) != cudaSuccess) {
            cudaGetLastError();
            *why = "cudaGetSymbolAddress failed for the scratch arrays";
            return false;
        }
        g_keys_addr[dev] = static_cast<uint64_t*>(k);
        g_status_addr[dev] = static_cast<int*>(s);
        g_ctx_id[dev] = ctx;
        g_ready[dev] = true;
    }
    *keys = g_keys_addr[dev];
    *status = g_status_addr[dev];
    return true;
}

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int fail(int code, const char* msg) {
    record_error(msg);
    return code;
}

}  // namespace
}  // namespace knng

using namespace knng;

extern "C" KNNG_API int knng_exact_noalloc(const float* data, int64_t n, int D, int k, const int32_t* sample,
                                           int64_t s, int32_t* out_ids, float* out_dists, void* stream) {
    record_error("");
    fault_begin();
    if (!data || !sample || !out_ids || !out_dists) return fail(KNNG_EINVAL, "NULL pointer");
    if (D < 1 || D > 4096) return fail(KNNG_EINVAL, "D out of range [1, 4096]");
    if (k < 1 || k > 64) return fail(KNNG_EINVAL, "k out of range [1, 64]");
    if (n <= k || n >= (int64_t(1) << 31)) return fail(KNNG_EINVAL, "n must exceed k and be below 2^31");
    if (s < 1) return fail(KNNG_EINVAL, "s must be >= 1");
    if (s * (int64_t)k > kNoAllocMaxEntries)
        return fail(KNNG_EINVAL, "s * k exceeds the 262144 entries of the static scratch (use knng_exact)");
    if (!on_device(data) || !on_device(sample) || !on_device(out_ids) || !on_device(out_dists))
        return fail(KNNG_EINVAL, "knng_exact_noalloc takes device pointers only");
    uint64_t* keys = nullptr;
    int* status = nullptr;
    const char* why = nullptr;
    if (!scratch_for_current_device(&keys, &status, &why)) return fail(KNNG_ECUDA, why);
    cudaStream_t st = (cudaStream_t)stream;
    // the status word must start at zero; the keys are overwritten in full
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return fail(KNNG_ECUDA, "status clear failed");
    launch_check_finite(data, n * (int64_t)D, status, st);
    launch_check_ids(sample, s, 0, n, status, st);
    launch_exact(data, n, D, k, sample, s, keys, status, st);
    launch_unpack(keys, out_ids, out_dists, s * (int64_t)k, st);
    // a launch the runtime refused (for example the dynamic shared memory of
    // the exact kernel) leaves the outputs unwritten: report it before the
    // status word, which would read zero
    const cudaError_t le = launch_error();
    if (le != cudaSuccess) return fail(KNNG_ECUDA, cudaGetErrorString(le));
    int hs = 0;
    if (cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        return fail(KNNG_ECUDA, cudaGetErrorString(e));
    }
    stats_flush();
    if (hs & kStatusNonFinite) return fail(KNNG_EINVAL, "data holds a non-finite value");
    if (hs & kStatusBadInput) return fail(KNNG_EINVAL, "a sampled row index is out of range");
    return KNNG_OK;
}
