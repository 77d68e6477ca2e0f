// search.cu -- the enhanced hill-climbing search over a kNN graph (Sec. 3.2,
// Alg. 2) for a batch of queries.
//
// One warp per query.  The rank list R matters only through its first ks
// entries by (d, id): they are what each iteration expands and what the
// search returns, and an entry outside them never re-enters them (R only
// grows).  So the warp keeps those ks keys (ks <= 32, entry e in lane e) and
// a visited set, an open-addressing table of ids in global memory (twice the
// most visits the query can make, so probes stay short and never fill it).
// An iteration takes the ks entries as they stand at its start, and every
// neighbour of theirs not visited yet is visited: its canonical FP32 distance
// is computed and its key merged into the list.  The entries' graph slots are
// taken 32 at a time across entries, one per lane.  A key enters the list at
// most once and the fresh ids of an iteration do not depend on the order the
// slots are taken in, so the order does not change the result.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace knng {

namespace {

constexpr int kSearchWarps = 4;

// Marks `id` visited in the query's table (2^cap_log2 slots, -1 = free);
// true on its first visit.  Fibonacci hashing, linear probing.
__device__ __forceinline__ bool visit(int32_t* tab, int cap_log2, int32_t id) {
    const uint32_t mask = (1u << cap_log2) - 1u;
    uint32_t h = ((uint32_t)id * 2654435761u) >> (32 - cap_log2);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const int32_t old = atomicCAS(tab + h, -1, id);
        if (old == -1) return true;
        if (old == id) return false;
        h = (h + 1u) & mask;
    }
    return false;  // not reached: the table holds twice the possible visits
}

// Canonical FP32 squared l2 of row x against the query q (dims ascending,
// t = x_j - q_j, acc = fmaf(t, t, acc)).  V4: x and q 16-byte aligned and D a
// multiple of 4, so both are read four dims at a time (the same chain).
template <bool V4>
__device__ __forceinline__ float dist_to_query(const float* __restrict__ x, const float* q, int D) {
    float acc = 0.f;
    if (V4) {
        const float4* x4 = reinterpret_cast<const float4*>(x);
        const float4* q4 = reinterpret_cast<const float4*>(q);
        for (int j = 0; j < D / 4; ++j) {
            const float4 a = __ldg(x4 + j), b = q4[j];
            float t = __fsub_rn(a.x, b.x);
            acc = __fmaf_rn(t, t, acc);
            t = __fsub_rn(a.y, b.y);
            acc = __fmaf_rn(t, t, acc);
            t = __fsub_rn(a.z, b.z);
            acc = __fmaf_rn(t, t, acc);
            t = __fsub_rn(a.w, b.w);
            acc = __fmaf_rn(t, t, acc);
        }
        return acc;
    }
    for (int j = 0; j < D; ++j) {
        const float t = __fsub_rn(__ldg(x + j), q[j]);
        acc = __fmaf_rn(t, t, acc);
    }
    return acc;
}

template <bool V4>
__global__ void __launch_bounds__(32 * kSearchWarps) k8_search(const float* __restrict__ X, int64_t n, int D,
                                                              const int32_t* __restrict__ G, int k,
                                                              const float* __restrict__ Q, int64_t q0, int64_t q1,
                                                              const int32_t* __restrict__ S, int s, int t0, int ks,
                                                              int32_t* __restrict__ tab, int cap_log2,
                                                              int32_t* __restrict__ out_ids,
                                                              float* __restrict__ out_d) {
    extern __shared__ float4 qs4[];  // [kSearchWarps][D]
    float* qs = reinterpret_cast<float*>(qs4);
    __shared__ uint64_t scratch[kSearchWarps][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t qi = q0 + (int64_t)blockIdx.x * kSearchWarps + w;
    if (qi >= q1) return;  // the whole warp; nothing below synchronises the CTA
    float* q = qs + (size_t)w * D;
    for (int j = lane; j < D; j += 32) q[j] = Q[qi * D + j];
    __syncwarp();
    int32_t* T = tab + ((qi - q0) << cap_log2);
    uint64_t* sc = scratch[w];
    uint64_t list = kEmptyKey;  // entry `lane` of R's first ks
    // every lane offers one id (or -1): the fresh ones are visited and merged
    auto offer = [&](int32_t id) {
        const bool fresh = id >= 0 && id < n && visit(T, cap_log2, id);
        const uint64_t key = fresh ? make_key(dist_to_query<V4>(X + (int64_t)id * D, q, D), (uint32_t)id) : kEmptyKey;
        uint64_t cand[1] = {key}, out;
        bool changed;
        if (!warp_merge_few<1>(cand, list, ks, sc, out, changed)) {
            // not reached (the keys are distinct and at most 64): the general merge
            uint64_t a[2] = {key, list}, res[1];
            sort_regs<2>(a);
            warp_select_unique<2, 1>(a, ks, res);
            out = res[0];
        }
        list = lane < ks ? out : kEmptyKey;
    };
    for (int a0 = 0; a0 < s; a0 += 32) offer(a0 + lane < s ? S[qi * s + a0 + lane] : -1);
    for (int t = 0; t < t0; ++t) {
        // R's first ks at the iteration's start: its real entries are a
        // prefix; their nt * k graph slots are offered 32 at a time (slot
        // u = entry u / k, neighbour u % k)
        const uint64_t snap = list;
        const int nt = __popc(__ballot_sync(0xffffffffu, snap != kEmptyKey));
        const int slots = nt * k;
        for (int u0 = 0; u0 < slots; u0 += 32) {
            const int u = u0 + lane;
            const int a = u < slots ? u / k : 0;
            const uint64_t e = shfl64(snap, a);
            offer(u < slots ? G[(int64_t)key_id(e) * k + (u - a * k)] : -1);
        }
    }
    if (lane < ks) {
        const bool real = list != kEmptyKey;
        out_ids[qi * ks + lane] = real ? (int32_t)key_id(list) : -1;
        out_d[qi * ks + lane] = real ? key_dist(list) : __int_as_float(0x7f800000);
    }
}

}  // namespace

int search_cap_log2(int s, int t0, int ks, int k) {
    const double visits = (double)s + (double)t0 * ks * k;
    int c = 6;
    while (c < 30 && (double)(1ll << c) < 2.0 * visits) ++c;
    return c;
}

void launch_search(const float* X, int64_t n, int D, const int32_t* G, int k, const float* Q, int64_t q0,
                   int64_t q1, const int32_t* S, int s, int t0, int ks, int32_t* tab, int cap_log2, int32_t* out_ids,
                   float* out_d, cudaStream_t st) {
    if (q1 <= q0) return;
    const int64_t m = q1 - q0;
    cudaMemsetAsync(tab, 0xFF, (size_t)(m << cap_log2) * sizeof(int32_t), st);
    // algorithmic bytes: every possible visit reads a row and every expansion a
    // list (an upper bound; the visits actually made are fewer)
    const double visits = (double)s + (double)t0 * ks * k;
    LaunchScope ls("k8_search", st, (double)m * (visits * (D * 4.0 + 8.0) + (double)t0 * ks * k * 4.0 + D * 4.0),
                   (double)m * visits * 3.0 * D);
    const size_t smem = (size_t)kSearchWarps * D * sizeof(float);
    const int64_t grid = (m + kSearchWarps - 1) / kSearchWarps;
    if (D % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0) {
        cudaFuncSetAttribute(k8_search<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k8_search<true><<<(unsigned)grid, 32 * kSearchWarps, smem, st>>>(X, n, D, G, k, Q, q0, q1, S, s, t0, ks, tab,
                                                                         cap_log2, out_ids, out_d);
    } else {
        cudaFuncSetAttribute(k8_search<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k8_search<false><<<(unsigned)grid, 32 * kSearchWarps, smem, st>>>(X, n, D, G, k, Q, q0, q1, S, s, t0, ks,
                                                                          tab, cap_log2, out_ids, out_d);
    }
}

}  // namespace knng
