// common.cuh -- device helpers shared by the kNN-graph kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/knng.h"

namespace knng {

// A graph entry is one 64-bit key: the order-preserving image of the FP32
// distance in the high word and the id in the low word, so that unsigned
// comparison of keys is the (dist, id) order used everywhere.  The empty slot
// (id -1, dist +inf) is the all-ones key and sorts after every real entry.
constexpr uint64_t kEmptyKey = ~0ull;

// Order-preserving map of an FP32 value to uint32 (valid for every non-NaN,
// with -0 mapped like +0 by the caller adding +0.0f first).
__host__ __device__ __forceinline__ uint32_t f2u(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
#endif
}
__host__ __device__ __forceinline__ float u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}
__host__ __device__ __forceinline__ uint32_t ord32(float f) {
    uint32_t b = f2u(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__host__ __device__ __forceinline__ float unord32(uint32_t o) {
    uint32_t b = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    return u2f(b);
}
__host__ __device__ __forceinline__ uint64_t make_key(float d, uint32_t id) {
    return ((uint64_t)ord32(d) << 32) | id;
}
__host__ __device__ __forceinline__ uint32_t key_id(uint64_t k) { return (uint32_t)k; }
__host__ __device__ __forceinline__ float key_dist(uint64_t k) { return unord32((uint32_t)(k >> 32)); }

// SplitMix64 output for state z (Steele, Lea & Flood 2014).
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t shfl_xor64(uint64_t v, int m) {
    uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
    uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), m);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
    const uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)v, src);
    const uint32_t hi = __shfl_sync(0xffffffffu, (uint32_t)(v >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}
// The candidate members of node i for one warp (all 32 lanes call it):
// lane e holds entry e of G_old[i] (key0, new0) and entry e of R[i] (with
// reverse lists, k <= 32) or entry 32 + e of G_old[i] (without, k <= 64) in
// key1, new1; fb / rb hold the entries' new flags.  A reverse entry that is a
// forward one too (a mutual neighbour: the same pair, so the same key) is
// one member: it is dropped from key1, and the forward copy is new if either
// copy is (its pairs then cover what the two copies gave).  G_old[i] is sorted,
// so a branch-free binary search over its lanes finds the copy.
__device__ __forceinline__ void member_keys(const uint64_t* __restrict__ Gold, const uint64_t* __restrict__ R,
                                            int64_t i, int k, bool rev, uint64_t fb, uint64_t rb, uint64_t& key0,
                                            uint64_t& key1, bool& new0, bool& new1) {
    const int lane = threadIdx.x & 31;
    const uint64_t* row1 = rev ? R + i * k : Gold + i * k + 32;
    const int lim1 = rev ? k : k - 32;
    key0 = lane < k ? Gold[i * k + lane] : kEmptyKey;
    key1 = lane < lim1 ? row1[lane] : kEmptyKey;
    new0 = ((fb >> lane) & 1ull) != 0;
    new1 = (((rev ? rb : fb >> 32) >> lane) & 1ull) != 0;
    if (!rev) return;
    int lo = 0;  // entries of G_old[i] below key1 (every lane shuffles: the probes differ)
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int probe = lo + step - 1;  // at most 30
        const uint64_t v = shfl64(key0, probe);
        if (probe < k && v < key1) lo += step;
    }
    const uint64_t at = shfl64(key0, lo);  // lo <= 31
    const bool dup = key1 != kEmptyKey && lo < k && at == key1;
    const unsigned promote = __reduce_or_sync(0xffffffffu, (dup && new1) ? (1u << lo) : 0u);
    new0 = new0 || ((promote >> lane) & 1u) != 0;
    if (dup) key1 = kEmptyKey;
}

__device__ __forceinline__ uint64_t warp_min64(uint64_t v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        uint64_t o = shfl_xor64(v, m);
        v = o < v ? o : v;
    }
    return v;
}

// Sort NS keys held in registers ascending (odd-even transposition; NS small).
template <int NS>
__device__ __forceinline__ void sort_regs(uint64_t (&a)[NS]) {
#pragma unroll
    for (int r = 0; r < NS; ++r) {
#pragma unroll
        for (int i = (r & 1); i + 1 < NS; i += 2) {
            uint64_t x = a[i], y = a[i + 1];
            a[i] = x < y ? x : y;
            a[i + 1] = x < y ? y : x;
        }
    }
}

// Warp-cooperative selection.  Every lane holds NS keys sorted ascending
// (kEmptyKey pads).  Produces, in order, the first `k` distinct keys of the
// multiset of all 32*NS keys (equal keys are one graph entry seen twice).
// Lane r % 32 keeps output r in out[r / 32].  All 32 lanes must call it.
template <int NS, int NO>
__device__ __forceinline__ void warp_select_unique(uint64_t (&a)[NS], int k, uint64_t (&out)[NO]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 0; o < NO; ++o) out[o] = kEmptyKey;
    for (int r = 0; r < k; ++r) {
        uint64_t m = warp_min64(a[0]);
        if ((r & 31) == lane) {
#pragma unroll
            for (int o = 0; o < NO; ++o)
                if (o == (r >> 5)) out[o] = m;
        }
        if (m == kEmptyKey) break;
        // drop every copy of m: only heads can equal the minimum (lanes are
        // sorted), and a lane can hold several copies in a row
        for (int t = 0; t < NS && a[0] == m; ++t) {
#pragma unroll
            for (int i = 0; i + 1 < NS; ++i) a[i] = a[i + 1];
            a[NS - 1] = kEmptyKey;
        }
    }
}

// Ascending bitonic sort of one key per lane across the warp.
__device__ __forceinline__ uint64_t warp_sort32(uint64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const uint64_t o = shfl_xor64(v, stride);
            // the lower lane of a pair keeps the smaller key in ascending runs
            const bool up = (lane & size) == 0, lower = (lane & stride) == 0;
            v = (lower == up) ? (o < v ? o : v) : (o < v ? v : o);
        }
    }
    return v;
}

// Fast path of "first k distinct keys of list U candidates" for k <= 32.
// `list`: the current sorted list, entry e in lane e (empty slots kEmptyKey);
// `cand`: NC keys per lane, distinct among themselves (any may equal a list
// entry).  A candidate not below the list's k-th key cannot enter.  The
// survivors (at most 32) are sorted, the 32 smallest keys of the union come
// from one bitonic merge step and a bitonic sort, and duplicates drop out.
// Returns false, with nothing decided, when more than 32 candidates survive
// or those 32 keys hold fewer than k distinct ones while more may follow; the
// caller then takes the general path.  `scratch`: 32 keys of shared memory
// owned by the warp.  On true, `out` is the new list (entry e in lane e) and
// `changed` says whether it differs from `list`.
template <int NC>
__device__ __forceinline__ bool warp_merge_few(const uint64_t (&cand)[NC], uint64_t list, int k, uint64_t* scratch,
                                               uint64_t& out, bool& changed) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t klo = __shfl_sync(0xffffffffu, (uint32_t)list, k - 1);
    const uint32_t khi = __shfl_sync(0xffffffffu, (uint32_t)(list >> 32), k - 1);
    const uint64_t kth = ((uint64_t)khi << 32) | klo;
    unsigned bal[NC];
    int total = 0;
#pragma unroll
    for (int s = 0; s < NC; ++s) {
        bal[s] = __ballot_sync(0xffffffffu, cand[s] < kth);
        total += __popc(bal[s]);
    }
    if (total == 0) {
        out = list;
        changed = false;
        return true;
    }
    if (total > 32) return false;
    int base = 0;
#pragma unroll
    for (int s = 0; s < NC; ++s) {
        if (cand[s] < kth) scratch[base + __popc(bal[s] & lt)] = cand[s];
        base += __popc(bal[s]);
    }
    __syncwarp();
    uint64_t b = lane < total ? scratch[lane] : kEmptyKey;
    __syncwarp();
    b = warp_sort32(b);
    // list ascending and the survivors descending form a bitonic sequence of
    // 64; its lower half-cleaner holds the 32 smallest, itself bitonic
    const uint64_t br = shfl64(b, 31 - lane);
    uint64_t c = list < br ? list : br;
#pragma unroll
    for (int stride = 16; stride > 0; stride >>= 1) {
        const uint64_t o = shfl_xor64(c, stride);
        c = (lane & stride) == 0 ? (o < c ? o : c) : (o < c ? c : o);
    }
    const uint64_t prev = shfl64(c, (lane + 31) & 31);
    const bool keep = c != kEmptyKey && (lane == 0 || c != prev);
    const unsigned ub = __ballot_sync(0xffffffffu, keep);
    const int nu = __popc(ub);
    const uint64_t last = shfl64(c, 31);
    if (nu < k && last != kEmptyKey) return false;  // a 33rd key may be needed
    if (keep) scratch[__popc(ub & lt)] = c;
    __syncwarp();
    out = lane < nu ? scratch[lane] : kEmptyKey;
    __syncwarp();
    changed = __any_sync(0xffffffffu, lane < k && out != list);
    return true;
}

// warp_merge_few for more candidates than survive at once (a first pass
// into an empty list): each lane sorts its NC candidates, the lanes' smallest
// ones (one per lane) merge first, and the rest then face the new k-th entry.
// Same contract and fallback as warp_merge_few.
template <int NC>
__device__ __forceinline__ bool warp_merge_many(uint64_t (&cand)[NC], uint64_t list, int k, uint64_t* scratch,
                                                uint64_t& out, bool& changed) {
    static_assert(NC >= 2, "one candidate per lane: use warp_merge_few");
    const int lane = threadIdx.x & 31;
    sort_regs<NC>(cand);
    uint64_t first[1] = {cand[0]}, mid;
    bool ch0;
    if (!warp_merge_few<1>(first, list, k, scratch, mid, ch0)) return false;
    mid = lane < k ? mid : kEmptyKey;
    uint64_t rest[NC - 1];
#pragma unroll
    for (int s = 0; s < NC - 1; ++s) rest[s] = cand[s + 1];
    bool ch1;
    if (!warp_merge_few<NC - 1>(rest, mid, k, scratch, out, ch1)) return false;
    changed = __any_sync(0xffffffffu, lane < k && out != list);
    return true;
}

// canonical FP32 squared distance between rows xa and xb (dims ascending,
// fmaf); vec: D % 4 == 0 and 16-byte aligned rows
__device__ __forceinline__ float canon_dist(const float* __restrict__ xa, const float* __restrict__ xb, int D,
                                            bool vec) {
    float acc = 0.f;
    if (vec) {
        for (int d = 0; d < D; d += 4) {
            const float4 u = __ldg(reinterpret_cast<const float4*>(xa + d));
            const float4 v = __ldg(reinterpret_cast<const float4*>(xb + d));
            float t = __fsub_rn(u.x, v.x);
            acc = __fmaf_rn(t, t, acc);
            t = __fsub_rn(u.y, v.y);
            acc = __fmaf_rn(t, t, acc);
            t = __fsub_rn(u.z, v.z);
            acc = __fmaf_rn(t, t, acc);
            t = __fsub_rn(u.w, v.w);
            acc = __fmaf_rn(t, t, acc);
        }
    } else {
        for (int d = 0; d < D; ++d) {
            const float t = __fsub_rn(__ldg(xa + d), __ldg(xb + d));
            acc = __fmaf_rn(t, t, acc);
        }
    }
    return acc;
}


// Status word written by kernels that detect a bad input or an internal
// limit; the host reads it once per call.
enum DevStatus : int {
    kStatusOk = 0,
    kStatusNonFinite = 1,   // input holds NaN or Inf
    kStatusOverflow = 2,    // an internal buffer would overflow: later stages skip
    kStatusBadInput = 4,    // an id or offset given by the caller is out of range
    kStatusInternal = 8,    // a consistency check failed: the write was skipped
    kStatusTimeout = 16,    // a bounded device wait ran out
};
constexpr int kStatusStop = kStatusOverflow | kStatusBadInput | kStatusInternal | kStatusTimeout;

}  // namespace knng
