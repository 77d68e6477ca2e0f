// sampled.cu -- the sampled refinement round: nearest-neighbour descent with
// sampling (Dong, Charikar and Li, WWW 2011), the prior art Sec. 1 cites.
//
// Every list entry carries a flag, new (not yet joined) or old.  A round
// draws, per node v, the ms new entries of least priority (new[v]; they turn
// old), and per node u the ms least-priority members of each of its reverse
// lists, one of the nodes whose new[v] holds u and one of the nodes whose old
// entries hold u.  The join then pairs new x new and new x old members, which
// is the rule the join kernels already apply to flagged members: they run on
// a member view of the lists (unsampled new entries emptied) with the sampled
// reverse rows in the R slots.  After the merge an id that was not in a
// node's list enters flagged new; the others keep their flags.
//
// Priority of member u of node v: the upper 32 bits of
// SplitMix64(SplitMix64(seed ^ round) ^ (v << 32 | u)) above the 32 bits of u,
// so one unsigned comparison orders by hash and then by id.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace knng {

namespace {

constexpr int kSampWarps = 8;  // nodes per CTA, one warp each

__device__ __forceinline__ uint64_t sample_key(uint64_t h0, int64_t v, uint32_t u) {
    const uint64_t h = splitmix64(h0 ^ (((uint64_t)v << 32) | u));
    return (h & 0xFFFFFFFF00000000ull) | u;
}

// The ms least of a sorted list (lane e holds entry e, kEmptyKey pads) and 32
// further keys, all distinct: one bitonic half-cleaner and merge.
__device__ __forceinline__ uint64_t keep_least(uint64_t list, uint64_t cand, int ms) {
    const int lane = threadIdx.x & 31;
    const uint64_t b = warp_sort32(cand);
    const uint64_t br = shfl64(b, 31 - lane);
    uint64_t c = list < br ? list : br;
#pragma unroll
    for (int stride = 16; stride > 0; stride >>= 1) {
        const uint64_t o = shfl_xor64(c, stride);
        c = (lane & stride) == 0 ? (o < c ? o : c) : (o < c ? c : o);
    }
    return lane < ms ? c : kEmptyKey;
}

// Per node v (k <= 32: entry e in lane e): new[v] = the ms entries flagged new
// in F[v] with the least priority.  Gm[v] keeps new[v] and the old entries at
// their slots (other slots empty); fm[v] marks new[v]; Fp[v] = F[v] without it.
__global__ void __launch_bounds__(32 * kSampWarps) k10_sample(const uint64_t* __restrict__ G,
                                                              const uint64_t* __restrict__ F, int64_t n, int k,
                                                              int ms, uint64_t h0, uint64_t* __restrict__ Gm,
                                                              uint64_t* __restrict__ fm, uint64_t* __restrict__ Fp) {
    const int lane = threadIdx.x & 31;
    const int64_t v = (int64_t)blockIdx.x * kSampWarps + (threadIdx.x >> 5);
    if (v >= n) return;  // the whole warp
    const uint64_t f = F[v];
    const uint64_t key = lane < k ? G[v * k + lane] : kEmptyKey;
    const bool fresh = key != kEmptyKey && ((f >> lane) & 1ull);
    const uint64_t sk = fresh ? sample_key(h0, v, key_id(key)) : kEmptyKey;
    int rank = 0;  // distinct keys: the number below sk
    for (int src = 0; src < 32; ++src) rank += shfl64(sk, src) < sk ? 1 : 0;
    const uint64_t sel = __ballot_sync(0xffffffffu, fresh && rank < ms);
    if (lane < k) {
        const bool keep = key != kEmptyKey && (((sel >> lane) & 1u) || !((f >> lane) & 1ull));
        Gm[v * k + lane] = keep ? key : kEmptyKey;
    }
    if (lane == 0) {
        fm[v] = sel;
        Fp[v] = f & ~sel;
    }
}

// Reverse entries from new[v] (fm) and from old entries (flag clear in F):
// counted per target, then written as (from new << 32 | v).
__global__ void k10_rcount(const uint64_t* __restrict__ G, const uint64_t* __restrict__ F,
                           const uint64_t* __restrict__ fm, int64_t n, int k, int32_t* __restrict__ deg) {
    const int64_t nk = n * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nk; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = G[e];
        if (key == kEmptyKey) continue;
        const int64_t v = e / k;
        const int t = (int)(e - v * k);
        if (((fm[v] >> t) & 1ull) || !((F[v] >> t) & 1ull)) atomicAdd(deg + key_id(key), 1);
    }
}

__global__ void k10_rfill(const uint64_t* __restrict__ G, const uint64_t* __restrict__ F,
                          const uint64_t* __restrict__ fm, int64_t n, int k, const int32_t* __restrict__ roff,
                          int32_t* __restrict__ cur, uint64_t* __restrict__ rbuf) {
    const int64_t nk = n * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nk; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = G[e];
        if (key == kEmptyKey) continue;
        const int64_t v = e / k;
        const int t = (int)(e - v * k);
        const bool isnew = (fm[v] >> t) & 1ull;
        if (isnew || !((F[v] >> t) & 1ull)) {
            const uint32_t u = key_id(key);
            rbuf[roff[u] + atomicAdd(cur + u, 1)] = ((uint64_t)(isnew ? 1u : 0u) << 32) | (uint32_t)v;
        }
    }
}

// Per node u (k <= 32): the ms least-priority members of each reverse list;
// R[u] = the new ones, then the old ones, then empty slots (2 ms <= k);
// rm[u] marks the new ones.
__global__ void __launch_bounds__(32 * kSampWarps) k10_rsample(const uint64_t* __restrict__ rbuf,
                                                               const int32_t* __restrict__ roff, int64_t n, int k,
                                                               int ms, uint64_t h0, uint64_t* __restrict__ R,
                                                               uint64_t* __restrict__ rm) {
    const int lane = threadIdx.x & 31;
    const int64_t u = (int64_t)blockIdx.x * kSampWarps + (threadIdx.x >> 5);
    if (u >= n) return;  // the whole warp
    uint64_t ln = kEmptyKey, lo = kEmptyKey;
    const int a = roff[u], b = roff[u + 1];
    for (int t0 = a; t0 < b; t0 += 32) {
        const int t = t0 + lane;
        uint64_t cn = kEmptyKey, co = kEmptyKey;
        if (t < b) {
            const uint64_t r = rbuf[t];
            const uint64_t sk = sample_key(h0, u, (uint32_t)r);
            if (r >> 32) cn = sk;
            else co = sk;
        }
        ln = keep_least(ln, cn, ms);
        lo = keep_least(lo, co, ms);
    }
    const int an = __popc(__ballot_sync(0xffffffffu, ln != kEmptyKey));
    const int ao = __popc(__ballot_sync(0xffffffffu, lo != kEmptyKey));
    const uint64_t from_old = shfl64(lo, (lane - an) & 31);
    if (lane < k) {
        uint64_t key = kEmptyKey;
        if (lane < an) key = make_key(0.f, (uint32_t)ln);
        else if (lane < an + ao) key = make_key(0.f, (uint32_t)from_old);
        R[u * k + lane] = key;
    }
    if (lane == 0) rm[u] = an >= 64 ? ~0ull : ((1ull << an) - 1ull);
}

// Per node u (k <= 32): entry e of Gnew[u] is new when its id was not in
// Gold[u], else it keeps Fp's flag of its slot there; empty slots are old.
__global__ void __launch_bounds__(32 * kSampWarps) k10_flags_after(const uint64_t* __restrict__ Gnew,
                                                                   const uint64_t* __restrict__ Gold,
                                                                   const uint64_t* __restrict__ Fp, int64_t n, int k,
                                                                   uint64_t* __restrict__ F,
                                                                   unsigned long long* __restrict__ entered) {
    const int lane = threadIdx.x & 31;
    const int64_t u = (int64_t)blockIdx.x * kSampWarps + (threadIdx.x >> 5);
    if (u >= n) return;  // the whole warp
    const uint64_t kn = lane < k ? Gnew[u * k + lane] : kEmptyKey;
    const uint64_t ko = lane < k ? Gold[u * k + lane] : kEmptyKey;
    int found = -1;
    for (int src = 0; src < 32; ++src) {
        const uint64_t o = shfl64(ko, src);
        if (kn != kEmptyKey && o != kEmptyKey && key_id(o) == key_id(kn)) found = src;
    }
    const uint64_t fp = Fp[u];
    const bool isnew = kn != kEmptyKey && (found < 0 || ((fp >> found) & 1ull));
    const unsigned bits = __ballot_sync(0xffffffffu, isnew);
    const unsigned came = __ballot_sync(0xffffffffu, kn != kEmptyKey && found < 0);
    if (lane == 0) {
        F[u] = bits;
        if (entered && came) atomicAdd(entered, (unsigned long long)__popc(came));
    }
}

int grid_nodes(int64_t n) { return (int)((n + kSampWarps - 1) / kSampWarps); }

}  // namespace

void launch_sampled_prepare(const uint64_t* G, uint64_t* F, int64_t n, int k, int ms, uint64_t h0, uint64_t* Gm,
                            uint64_t* fm, uint64_t* Fp, int32_t* deg, int32_t* roff, int32_t* cur, int32_t* scan_tmp,
                            uint64_t* rbuf, uint64_t* R, uint64_t* rm, cudaStream_t s) {
    const int64_t nk = n * k;
    {
        LaunchScope ls("k10_sample", s, nk * 16.0 + n * 24.0, 0);
        k10_sample<<<grid_nodes(n), 32 * kSampWarps, 0, s>>>(G, F, n, k, ms, h0, Gm, fm, Fp);
    }
    cudaMemsetAsync(deg, 0, sizeof(int32_t) * (n + 1), s);
    cudaMemsetAsync(cur, 0, sizeof(int32_t) * n, s);
    const int grid = (int)std::min<int64_t>((nk + 255) / 256, 152 * 16);
    {
        LaunchScope ls("k10_rcount", s, nk * 8.0 + n * 16.0, 0);
        k10_rcount<<<grid < 1 ? 1 : grid, 256, 0, s>>>(G, F, fm, n, k, deg);
    }
    launch_scan(deg, roff, n, scan_tmp, s);
    {
        LaunchScope ls("k10_rfill", s, nk * 16.0 + n * 16.0, 0);
        k10_rfill<<<grid < 1 ? 1 : grid, 256, 0, s>>>(G, F, fm, n, k, roff, cur, rbuf);
    }
    LaunchScope ls("k10_rsample", s, nk * 16.0 + n * 8.0, 0);
    k10_rsample<<<grid_nodes(n), 32 * kSampWarps, 0, s>>>(rbuf, roff, n, k, ms, h0, R, rm);
}

void launch_sampled_flags(const uint64_t* Gnew, const uint64_t* Gold, const uint64_t* Fp, int64_t n, int k,
                          uint64_t* F, unsigned long long* entered, cudaStream_t s) {
    LaunchScope ls("k10_flags_after", s, n * k * 16.0 + n * 16.0, 0);
    k10_flags_after<<<grid_nodes(n), 32 * kSampWarps, 0, s>>>(Gnew, Gold, Fp, n, k, F, entered);
}

}  // namespace knng
