// join.cu -- neighbour-of-neighbour refinement (the nearest-neighbour-descent
// prior art cited in Sec. 1), in Jacobi form: every offer of a round is made
// from the graph as it stood before the round, so the result does not depend
// on the order in which offers arrive.
//
//   K6 reverse lists  R[i] = the k closest j with i in G[j], by (d, j)
//   K5 local join     for every node i and every pair {u, v} of
//                     N_i = G[i] (+ R[i]), u != v: offer v to u and u to v
//                     with the canonical distance; an offer that cannot beat
//                     the target's k-th entry is dropped at the source (it
//                     could never enter the target's list)
//   scatter           group the offers by target (counts, prefix sum)
//   K4 merge          G_new[u] = first k unique of G_old[u] + offers to u
#include <algorithm>
#include <cstdlib>
#include <utility>

#include "common.cuh"
#include "kernels.h"

namespace knng {

namespace {

constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanBlock * kScanItems;

__device__ __forceinline__ int warp_incl_scan(int x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_partial(const int32_t* __restrict__ cnt, int64_t n,
                                                             int32_t* __restrict__ bsum) {
    __shared__ int wt[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int s = 0;
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        const int64_t e = base + (int64_t)threadIdx.x * kScanItems + t;
        if (e < n) s += cnt[e];
    }
    s = warp_incl_scan(s);
    if ((threadIdx.x & 31) == 31) wt[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int w = warp_incl_scan(wt[threadIdx.x]);
        if (threadIdx.x == 31) bsum[blockIdx.x] = w;
    }
}

__global__ void __launch_bounds__(kScanBlock) k_scan_blocks(int32_t* __restrict__ bsum, int nb) {
    __shared__ int wt[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += kScanBlock) {
        const int e = base + threadIdx.x;
        const int v = e < nb ? bsum[e] : 0;
        int x = warp_incl_scan(v);
        if ((threadIdx.x & 31) == 31) wt[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) wt[threadIdx.x] = warp_incl_scan(wt[threadIdx.x]);
        __syncthreads();
        const int before = (threadIdx.x >= 32 ? wt[(threadIdx.x >> 5) - 1] : 0) + carry;
        if (e < nb) bsum[e] = before + x - v;
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) carry = before + x;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanBlock) k_scan_final(const int32_t* __restrict__ cnt, int64_t n,
                                                           const int32_t* __restrict__ bsum,
                                                           int32_t* __restrict__ off) {
    __shared__ int wt[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        const int64_t e = base + (int64_t)threadIdx.x * kScanItems + t;
        v[t] = e < n ? cnt[e] : 0;
        s += v[t];
    }
    const int x = warp_incl_scan(s);
    if ((threadIdx.x & 31) == 31) wt[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) wt[threadIdx.x] = warp_incl_scan(wt[threadIdx.x]);
    __syncthreads();
    int run = bsum[blockIdx.x] + (threadIdx.x >= 32 ? wt[(threadIdx.x >> 5) - 1] : 0) + x - s;
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        const int64_t e = base + (int64_t)threadIdx.x * kScanItems + t;
        if (e < n) off[e] = run;
        run += v[t];
        if (e == n - 1) off[n] = run;
    }
}

__global__ void k_fill_empty(uint64_t* __restrict__ G, int64_t count) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        G[e] = kEmptyKey;
}

__global__ void k_pack(const int32_t* __restrict__ ids, const float* __restrict__ d, uint64_t* __restrict__ G,
                       int64_t count, int64_t n, int* __restrict__ status) {
    bool bad = false;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t id = ids[e];
        bad |= id < -1 || id >= n;
        G[e] = (id < 0 || id >= n) ? kEmptyKey : make_key(__fadd_rn(d[e], 0.f), (uint32_t)id);
    }
    if (bad) atomicOr(status, kStatusBadInput);
}

__global__ void k_check_ids(const int32_t* __restrict__ ids, int64_t count, int64_t lo, int64_t hi,
                            int* __restrict__ status) {
    bool bad = false;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        bad |= ids[e] < lo || ids[e] >= hi;
    if (bad) atomicOr(status, kStatusBadInput);
}

__global__ void k_unpack(const uint64_t* __restrict__ G, int32_t* __restrict__ ids, float* __restrict__ d,
                         int64_t count, int64_t id_offset) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = G[e];
        if (key == kEmptyKey) {
            ids[e] = -1;
            d[e] = __int_as_float(0x7f800000);
        } else {
            ids[e] = (int32_t)((int64_t)key_id(key) - id_offset);
            d[e] = key_dist(key);
        }
    }
}

// ---------------------------------------------------------------- K6
__global__ void k6_count(const uint64_t* __restrict__ G, int64_t nk, int32_t* __restrict__ deg) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nk; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = G[e];
        if (key != kEmptyKey) atomicAdd(&deg[key_id(key)], 1);
    }
}

__global__ void k6_fill(const uint64_t* __restrict__ G, int64_t nk, int k, const int32_t* __restrict__ roff,
                        int32_t* __restrict__ cur, uint64_t* __restrict__ rbuf) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nk; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = G[e];
        if (key == kEmptyKey) continue;
        const uint32_t i = key_id(key);
        const uint32_t j = (uint32_t)(e / k);
        const int pos = roff[i] + atomicAdd(&cur[i], 1);
        rbuf[pos] = (key & 0xFFFFFFFF00000000ull) | j;
    }
}

// k best keys of list[beg, end) merged with `run` (NO slots per lane, sorted
// list of k keys spread lane-major); duplicates merged.  Warp-wide.
template <int NO>
__device__ __forceinline__ void warp_merge_list(const uint64_t* __restrict__ list, int beg, int end, int k,
                                                uint64_t (&run)[NO]) {
    const int lane = threadIdx.x & 31;
    constexpr int NC = 4;
    for (int c = beg; c < end; c += 32 * NC) {
        uint64_t a[NC + NO];
#pragma unroll
        for (int s = 0; s < NC; ++s) {
            const int e = c + lane + 32 * s;
            a[s] = e < end ? list[e] : kEmptyKey;
        }
        // skip the merge when nothing can enter: compare with the k-th key
        uint64_t mine = run[0];
#pragma unroll
        for (int o = 1; o < NO; ++o)
            if (o == ((k - 1) >> 5)) mine = run[o];
        const uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)mine, (k - 1) & 31);
        const uint32_t hi = __shfl_sync(0xffffffffu, (uint32_t)(mine >> 32), (k - 1) & 31);
        const uint64_t last = ((uint64_t)hi << 32) | lo;
        bool any = false;
#pragma unroll
        for (int s = 0; s < NC; ++s) any |= a[s] < last;
        if (!__any_sync(0xffffffffu, any)) continue;
#pragma unroll
        for (int o = 0; o < NO; ++o) a[NC + o] = run[o];
        sort_regs<NC + NO>(a);
        warp_select_unique<NC + NO, NO>(a, k, run);
    }
}

template <int NO>
__global__ void __launch_bounds__(256) k6_select(const uint64_t* __restrict__ rbuf, const int32_t* __restrict__ roff,
                                                 int64_t n, int k, uint64_t* __restrict__ R) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const int lane = threadIdx.x & 31;
    const int beg = roff[i], deg = roff[i + 1] - beg;
    if (deg <= 32) {
        // the usual case: every candidate fits a lane; the keys are distinct
        // (one per source list), so the sorted run's first k are the list.
        // With k <= 32 the list's order is not used (the flags look ids up
        // in a hash set and the join takes members in any order): up to k
        // candidates are the list as they come.
        uint64_t v = lane < deg ? rbuf[beg + lane] : kEmptyKey;
        if (NO > 1 || deg > k) v = warp_sort32(v);
#pragma unroll
        for (int o = 0; o < NO; ++o) {
            const int e = lane + 32 * o;
            if (e < k) R[i * k + e] = o == 0 ? v : kEmptyKey;
        }
        return;
    }
    uint64_t run[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) run[o] = kEmptyKey;
    warp_merge_list<NO>(rbuf, roff[i], roff[i + 1], k, run);
#pragma unroll
    for (int o = 0; o < NO; ++o)
        if (lane + 32 * o < k) R[i * k + lane + 32 * o] = run[o];
}

// Whether `key` is one of the sorted keys list[0 .. k).
__device__ __forceinline__ bool sorted_has(const uint64_t* list, int k, uint64_t key) {
    int lo = 0, len = k;
    while (len > 0) {
        const int half = len >> 1;
        if (list[lo + half] < key) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo < k && list[lo] == key;
}

// Member flags of one round.  A member of node i (an entry of G_old[i] or of
// R[i]) is old when the same key was a member of i in the previous round
// (in G_prev[i] or R_prev[i]): both directions of a pair of old members were
// offered then, and such an offer is now either in its target's list already
// or beaten by the target's k-th entry (which never gets worse), so the join
// may skip the pair without changing the result.  One warp per node; bit e of
// fnew[i] (rnew[i]) marks entry e of G_old[i] (R[i]) new; nodes with a new
// member are appended to `active` (one atomic per block), unless `active` is
// NULL: then k6_active lists them afterwards in a given order.
constexpr int kFlagWarps = 16;
template <int NO>
__global__ void __launch_bounds__(32 * kFlagWarps) k6_flags(const uint64_t* __restrict__ Gcur,
                                                            const uint64_t* __restrict__ Rcur,
                                                            const uint64_t* __restrict__ Gprev,
                                                            const uint64_t* __restrict__ Rprev, int64_t n, int k,
                                                            uint64_t* __restrict__ fnew, uint64_t* __restrict__ rnew,
                                                            int32_t* __restrict__ active,
                                                            int32_t* __restrict__ nactive) {
    __shared__ uint64_t prev[kFlagWarps][2][32 * NO];
    __shared__ int act[kFlagWarps];
    __shared__ int base;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kFlagWarps + w;
    int on = 0;
    if (i < n) {
        uint64_t fb = 0, rb = 0;
        if (NO == 1) {
            // k <= 32: by id (a pair always has the same canonical distance,
            // the same both ways), in a hash set of the previous members'
            // ids (at most 64 in 128 slots, linear probing); no list needs
            // to be sorted
            uint32_t* tab = reinterpret_cast<uint32_t*>(prev[w]);
            constexpr uint32_t kFree = 0xFFFFFFFFu;
            const uint64_t gk = lane < k ? Gcur[i * k + lane] : kEmptyKey;
            const uint64_t rk = (Rcur && lane < k) ? Rcur[i * k + lane] : kEmptyKey;
            const uint64_t pgk = lane < k ? Gprev[i * k + lane] : kEmptyKey;
            const uint64_t prk = (Rprev && lane < k) ? Rprev[i * k + lane] : kEmptyKey;
            for (int t = lane; t < 128; t += 32) tab[t] = kFree;
            __syncwarp();
            auto home = [](uint32_t id) { return (id * 2654435761u) >> 25; };
            for (int src = 0; src < 2; ++src) {
                const uint64_t key = src == 0 ? pgk : prk;
                if (key == kEmptyKey) continue;
                const uint32_t id = key_id(key);
                for (uint32_t h = home(id), t = 0; t < 128; ++t, h = (h + 1) & 127) {
                    const uint32_t old = atomicCAS(&tab[h], kFree, id);
                    if (old == kFree || old == id) break;
                }
            }
            __syncwarp();
            auto seen = [&](uint64_t key) {
                const uint32_t id = key_id(key);
                for (uint32_t h = home(id), t = 0; t < 128; ++t, h = (h + 1) & 127) {
                    const uint32_t v = tab[h];
                    if (v == id) return true;
                    if (v == kFree) return false;
                }
                return false;
            };
            fb = __ballot_sync(0xffffffffu, gk != kEmptyKey && !seen(gk));
            if (Rcur) rb = __ballot_sync(0xffffffffu, rk != kEmptyKey && !seen(rk));
        } else {
            uint64_t* pg = prev[w][0];
            uint64_t* pr = prev[w][1];
#pragma unroll
            for (int o = 0; o < NO; ++o) {
                const int e = lane + 32 * o;
                pg[e] = e < k ? Gprev[i * k + e] : kEmptyKey;
                pr[e] = (Rprev && e < k) ? Rprev[i * k + e] : kEmptyKey;
            }
            __syncwarp();
#pragma unroll
            for (int o = 0; o < NO; ++o) {
                const int e = lane + 32 * o;
                uint64_t key = e < k ? Gcur[i * k + e] : kEmptyKey;
                bool nw = key != kEmptyKey && !sorted_has(pg, k, key) && !(Rprev && sorted_has(pr, k, key));
                fb |= (uint64_t)__ballot_sync(0xffffffffu, nw) << (32 * o);
                if (Rcur) {
                    key = e < k ? Rcur[i * k + e] : kEmptyKey;
                    nw = key != kEmptyKey && !sorted_has(pg, k, key) && !(Rprev && sorted_has(pr, k, key));
                    rb |= (uint64_t)__ballot_sync(0xffffffffu, nw) << (32 * o);
                }
            }
        }
        if (lane == 0) {
            fnew[i] = fb;
            if (Rcur) rnew[i] = rb;
        }
        on = (fb | rb) != 0;
    }
    if (active == nullptr) return;  // the nodes are listed by k6_active (uniform over the CTA)
    if (lane == 0) act[w] = on;
    __syncthreads();
    if (threadIdx.x == 0) {
        int c = 0;
        for (int q = 0; q < kFlagWarps; ++q) c += act[q];
        base = c > 0 ? atomicAdd(nactive, c) : 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int at = base;
        for (int q = 0; q < kFlagWarps; ++q)
            if (act[q]) active[at++] = (int32_t)((int64_t)blockIdx.x * kFlagWarps + q);
    }
}

// The nodes with a new member listed in the order of `order` (position p
// listed when node order[p] has a new member in fnew / rnew, as k6_flags
// wrote them): positions keep their order inside a CTA, one atomic per CTA.
__global__ void __launch_bounds__(256) k6_active(const int32_t* __restrict__ order,
                                                 const uint64_t* __restrict__ fnew,
                                                 const uint64_t* __restrict__ rnew, int64_t n,
                                                 int32_t* __restrict__ active, int32_t* __restrict__ nactive) {
    __shared__ int wbefore[8];
    __shared__ int base;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x;
    int32_t i = 0;
    bool on = false;
    if (p < n) {
        i = order[p];
        // a permutation of the nodes; a stray id (a failed partition, which
        // the status word reports) lists nothing
        on = i >= 0 && i < n && (fnew[i] | (rnew ? rnew[i] : 0ull)) != 0;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, on);
    if (lane == 0) wbefore[w] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        int c = 0;
        for (int q = 0; q < 8; ++q) {
            const int t = wbefore[q];
            wbefore[q] = c;
            c += t;
        }
        base = c > 0 ? atomicAdd(nactive, c) : 0;
    }
    __syncthreads();
    if (on) active[base + wbefore[w] + __popc(bal & ((1u << lane) - 1u))] = i;
}

// ---------------------------------------------------------------- K5
// One warp per node i.  Members N_i in shared memory; the upper triangle of
// member pairs is cut into 4 x 4 blocks, BPL blocks per lane; distances are
// canonical (dims ascending, fmaf); surviving offers are appended to the
// chunk's buffer.
constexpr int kJoinWarps = 4;

// Dims per shared-memory chunk (about 12 KB of member rows per warp, equal
// chunks) and the row stride (stride / 4 odd: consecutive rows in different
// banks for float4 reads).
__host__ __device__ inline void join_chunk(int D, int mcap, int* dch, int* stride) {
    const int d4 = (D + 3) & ~3;
    int cap = (12 * 1024 / (mcap * 4) - 4) & ~3;
    if (cap < 4) cap = 4;
    const int nch = (d4 + cap - 1) / cap;
    const int c = ((d4 + nch - 1) / nch + 3) & ~3;
    *dch = c;
    *stride = ((c / 4) & 1) ? c : c + 4;
}

// Whether entry (a, b) of block row ia, column ib is a pair to evaluate:
// in the rectangle ia is a new member and ib any later member or an old one;
// in the triangle `upper` says the entry is above the diagonal.  Pairs of
// two old members (indices >= nn) are skipped.
__device__ __forceinline__ bool pair_live(bool rect, int ia, int ib, int M, int nn, bool upper) {
    if (rect) return ia < nn && ib < M && (ib >= nn || ib > ia);
    return ia < M && ib < M && upper && (ia < nn || ib < nn);
}

// The local join of node i by one warp (members, distances, offers).
template <int BPL>
__device__ __forceinline__ void join_node(const float* __restrict__ X, int D, int k, int rev, int mcap,
                                          const uint64_t* __restrict__ Gold, const uint64_t* __restrict__ R,
                                          const uint64_t* __restrict__ fnew, const uint64_t* __restrict__ rnew,
                                          int64_t i, uint32_t* __restrict__ counter, int64_t cap,
                                          uint32_t* __restrict__ ptgt, uint64_t* __restrict__ pkey,
                                          int32_t* __restrict__ pcnt, int* __restrict__ status, float* xs,
                                          uint64_t* thr, int32_t* mem, int dch, int stride) {
    const int lane = threadIdx.x & 31;
    __syncwarp();  // the warp's previous node is done with xs, thr and mem
    // members: the new ones first (flags from the previous round; none =
    // all new), then the old ones; each takes ids of G_old[i], then of R[i]
    int M = 0, nn = 0;
    const uint64_t fbits = fnew ? fnew[i] : ~0ull, rbits = rnew ? rnew[i] : ~0ull;
    auto take_member = [&](uint64_t key, bool take) {
        const unsigned bal = __ballot_sync(0xffffffffu, take);
        if (take) {
            const int at = M + __popc(bal & ((1u << lane) - 1u));
            const uint32_t u = key_id(key);
            mem[at] = (int32_t)u;
            thr[at] = Gold[(int64_t)u * k + k - 1];
        }
        M += __popc(bal);
    };
    if (!(rev && k > 32)) {
        // at most 64 entries, a mutual neighbour once
        uint64_t key0, key1;
        bool new0, new1;
        member_keys(Gold, R, i, k, rev != 0, fbits, rbits, key0, key1, new0, new1);
        for (int want = 1; want >= 0; --want) {
            take_member(key0, key0 != kEmptyKey && new0 == (want == 1));
            take_member(key1, key1 != kEmptyKey && new1 == (want == 1));
            if (want == 1) nn = M;
        }
    } else {
        for (int want = 1; want >= 0; --want) {
            for (int src = 0; src < 2; ++src) {
                const uint64_t* row = (src == 0 ? Gold : R) + i * k;
                const uint64_t bits = src == 0 ? fbits : rbits;
                for (int e0 = 0; e0 < k; e0 += 32) {
                    const int e = e0 + lane;
                    const uint64_t key = e < k ? row[e] : kEmptyKey;
                    take_member(key, key != kEmptyKey && (int)((bits >> e) & 1ull) == want);
                }
            }
            if (want == 1) nn = M;
        }
    }
    __syncwarp();
    if (M < 2 || nn == 0) return;
    // Pairs with a new member: the upper triangle of all members cut into
    // 4 x 4 blocks, or, when fewer blocks do, the rectangle new x all (rows
    // 0 .. nn-1 against every member, each new x new pair kept once).
    const int RGN = (M + 3) >> 2;
    const int nb_tri = RGN * (RGN + 1) / 2;
    const int RBN = (nn + 3) >> 2;
    const bool rect = RBN * RGN < nb_tri;
    const int nb = rect ? RBN * RGN : nb_tri;
    const int RSTEP = rect ? RBN : RGN;  // member index step between a block's rows
    int brg[BPL], bcg[BPL];
#pragma unroll
    for (int q = 0; q < BPL; ++q) {
        int b = lane + 32 * q;
        brg[q] = -1;
        bcg[q] = 0;
        if (b < nb) {
            if (rect) {
                brg[q] = b / RGN;
                bcg[q] = b - brg[q] * RGN;
            } else {
                int rg = 0;
                while (b >= RGN - rg) {
                    b -= RGN - rg;
                    ++rg;
                }
                brg[q] = rg;
                bcg[q] = rg + b;
            }
        }
    }
    float acc[BPL][4][4];
#pragma unroll
    for (int q = 0; q < BPL; ++q)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[q][a][b] = 0.f;
    const bool vec = (D % 4 == 0);
    for (int d0 = 0; d0 < D; d0 += dch) {
        const int dl = min(dch, D - d0);
        // gather the members' dims [d0, d0 + dch)
        if (vec) {
            const int q4 = dch >> 2;
            for (int e = lane; e < M * q4; e += 32) {
                const int r = e / q4, c4 = e - r * q4;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (c4 * 4 < dl) v = __ldg(reinterpret_cast<const float4*>(X + (int64_t)mem[r] * D + d0) + c4);
                *reinterpret_cast<float4*>(xs + r * stride + c4 * 4) = v;
            }
        } else {
            for (int e = lane; e < M * dch; e += 32) {
                const int r = e / dch, c = e - r * dch;
                xs[r * stride + c] = c < dl ? __ldg(X + (int64_t)mem[r] * D + d0 + c) : 0.f;
            }
        }
        // rows M .. 4*RGN-1 read as zeros
        for (int e = lane; e < (RGN * 4 - M) * dch; e += 32) {
            const int r = M + e / dch, c = e % dch;
            xs[r * stride + c] = 0.f;
        }
        __syncwarp();
        // block (rg, cg) holds members {rg + a * RGN} x {cg + b * RGN}: lanes
        // then read consecutive rows, which the odd stride / 4 puts in
        // different banks
#pragma unroll
        for (int q = 0; q < BPL; ++q) {
            if (brg[q] < 0) continue;
            const float* rp = xs + brg[q] * stride;
            const float* cp = xs + bcg[q] * stride;
            const int rstep = RSTEP * stride, cstep = RGN * stride;
            for (int dq = 0; dq < dch; dq += 4) {
                float4 rv[4], cv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) rv[a] = *reinterpret_cast<const float4*>(rp + a * rstep + dq);
#pragma unroll
                for (int b = 0; b < 4; ++b) cv[b] = *reinterpret_cast<const float4*>(cp + b * cstep + dq);
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        float t = __fsub_rn(rv[a].x, cv[b].x);
                        acc[q][a][b] = __fmaf_rn(t, t, acc[q][a][b]);
                        t = __fsub_rn(rv[a].y, cv[b].y);
                        acc[q][a][b] = __fmaf_rn(t, t, acc[q][a][b]);
                        t = __fsub_rn(rv[a].z, cv[b].z);
                        acc[q][a][b] = __fmaf_rn(t, t, acc[q][a][b]);
                        t = __fsub_rn(rv[a].w, cv[b].w);
                        acc[q][a][b] = __fmaf_rn(t, t, acc[q][a][b]);
                    }
            }
        }
        __syncwarp();
    }
    // offers: count, reserve, write.  In the triangle every unordered member
    // pair lies in exactly one block once diagonal blocks keep only a < b;
    // pairs of two old members are dropped.
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < BPL; ++q) {
        if (brg[q] < 0) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int ia = brg[q] + a * RSTEP, ib = bcg[q] + b * RGN;
                if (pair_live(rect, ia, ib, M, nn, brg[q] < bcg[q] || a < b)) {
                    const uint32_t u = (uint32_t)mem[ia], v = (uint32_t)mem[ib];
                    if (u != v) {
                        cnt += make_key(acc[q][a][b], v) < thr[ia];
                        cnt += make_key(acc[q][a][b], u) < thr[ib];
                    }
                }
            }
    }
    const int incl = warp_incl_scan(cnt);
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    uint32_t at = 0;
    if (lane == 31) at = atomicAdd(counter, (uint32_t)total);
    at = __shfl_sync(0xffffffffu, at, 31);
    if ((int64_t)at + total > cap) {
        if (lane == 0) atomicOr(status, kStatusOverflow);
        return;
    }
    uint32_t w = at + incl - cnt;
#pragma unroll
    for (int q = 0; q < BPL; ++q) {
        if (brg[q] < 0) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int ia = brg[q] + a * RSTEP, ib = bcg[q] + b * RGN;
                if (pair_live(rect, ia, ib, M, nn, brg[q] < bcg[q] || a < b)) {
                    const uint32_t u = (uint32_t)mem[ia], v = (uint32_t)mem[ib];
                    if (u != v) {
                        const uint64_t ku = make_key(acc[q][a][b], v);
                        if (ku < thr[ia]) {
                            ptgt[w] = u;
                            pkey[w] = ku;
                            ++w;
                            atomicAdd(&pcnt[u], 1);
                        }
                        const uint64_t kv = make_key(acc[q][a][b], u);
                        if (kv < thr[ib]) {
                            ptgt[w] = v;
                            pkey[w] = kv;
                            ++w;
                            atomicAdd(&pcnt[v], 1);
                        }
                    }
                }
            }
    }
}

// Warps stride over the node positions [node0, node1) (of `list` when given).
template <int BPL>
__global__ void __launch_bounds__(32 * kJoinWarps) k5_join(const float* __restrict__ X, int D, int k, int rev,
                                                          int mcap, const uint64_t* __restrict__ Gold,
                                                          const uint64_t* __restrict__ R,
                                                          const int32_t* __restrict__ list,
                                                          const uint64_t* __restrict__ fnew,
                                                          const uint64_t* __restrict__ rnew, int64_t node0,
                                                          int64_t node1, uint32_t* __restrict__ counter,
                                                          int64_t cap, uint32_t* __restrict__ ptgt,
                                                          uint64_t* __restrict__ pkey,
                                                          int32_t* __restrict__ pcnt, int* __restrict__ status,
                                                          const int* __restrict__ skip_if_exact,
                                                          const int32_t* __restrict__ count_dev) {
    extern __shared__ float4 smem4[];
    if (*status & kStatusStop) return;
    if (count_dev && (int64_t)*count_dev < node1) node1 = *count_dev;
    // the tensor-core join does this round when the 16-bit copy is exact
    if (skip_if_exact) {
        const int f = *skip_if_exact;
        if ((f & 1) == 0 && !((f & 2) && (f & 4))) return;
    }
    int dch, stride;
    join_chunk(D, mcap, &dch, &stride);
    const int warp = threadIdx.x >> 5;
    char* base = reinterpret_cast<char*>(smem4) + (size_t)warp * ((size_t)mcap * (stride * 4 + 12) + 16);
    float* xs = reinterpret_cast<float*>(base);                                   // [mcap][stride]
    uint64_t* thr = reinterpret_cast<uint64_t*>(xs + (size_t)mcap * stride);      // [mcap]
    int32_t* mem = reinterpret_cast<int32_t*>(thr + mcap);                        // [mcap]
    for (int64_t pos = node0 + (int64_t)blockIdx.x * kJoinWarps + warp; pos < node1;
         pos += (int64_t)gridDim.x * kJoinWarps)
        join_node<BPL>(X, D, k, rev, mcap, Gold, R, fnew, rnew, list ? (int64_t)list[pos] : pos, counter, cap, ptgt,
                       pkey, pcnt, status, xs, thr, mem, dch, stride);
}

// ---------------------------------------------------------------- K5, CTA-wide
// The FP32 local join with the pairs of several nodes spread over one CTA.
// A node's member pairs are cut into the 4 x 4 blocks of the upper triangle
// of its (mcap / 4)-group member grid: NB = RGN (RGN + 1) / 2 blocks, RGN =
// mcap / 4; a CTA of 256 threads takes G = 256 / NB nodes at a time and
// thread t computes block t % NB of node t / NB, so a warp's lanes stay busy
// whatever NB is (one node per warp leaves lanes idle when NB is not a
// multiple of 32).  Block (rg, cg) holds members {4 rg + a} x {4 cg + b};
// member m of a node sits in shared-memory row (m % 4) RGN + m / 4, so lanes
// of consecutive cg read consecutive rows (an odd float4 stride puts them in
// different banks) and lanes of one rg read the same row.  Members are new
// first, so blocks whose two groups hold only old members are skipped whole.
// Offers as in k5_join; a pair of members that shared a leaf in one of the
// build's last tree passes makes none (the leaf stage offered it already).
constexpr int kJ2Threads = 256;

struct J2Layout {
    int RGN, NB, G, dch, stride;
    size_t thr, lid, rows, mem, cnt, total;
};

__host__ __device__ inline J2Layout j2_layout(int D, int mcap, bool leafids) {
    J2Layout L;
    L.RGN = mcap / 4;
    L.NB = L.RGN * (L.RGN + 1) / 2;
    L.G = L.NB > kJ2Threads ? 1 : kJ2Threads / L.NB;
    const int slots = L.G * mcap;
    const int d4 = (D + 3) & ~3;
    int cap = (44 * 1024 / (slots * 4) - 4) & ~3;
    if (cap < 4) cap = 4;
    const int nch = (d4 + cap - 1) / cap;
    L.dch = ((d4 + nch - 1) / nch + 3) & ~3;
    L.stride = ((L.dch / 4) & 1) ? L.dch : L.dch + 4;
    L.thr = 0;
    L.lid = L.thr + (size_t)slots * 8;
    L.rows = L.lid + (leafids ? (size_t)slots * 16 : 0);
    L.mem = L.rows + (size_t)slots * L.stride * 4;
    L.cnt = L.mem + (size_t)slots * 4;
    L.total = L.cnt + (size_t)L.G * 2 * 4;
    return L;
}

__device__ __forceinline__ int j2_slot(int m, int RGN) { return (m & 3) * RGN + (m >> 2); }

__global__ void __launch_bounds__(kJ2Threads, 4) k5_join_cta(const float* __restrict__ X, int D, int k, int rev,
                                                         int mcap, const uint64_t* __restrict__ Gold,
                                                         const uint64_t* __restrict__ R,
                                                         const int32_t* __restrict__ list,
                                                         const uint64_t* __restrict__ fnew,
                                                         const uint64_t* __restrict__ rnew, int64_t node0,
                                                         int64_t node1, uint32_t* __restrict__ counter, int64_t cap,
                                                         uint32_t* __restrict__ ptgt, uint64_t* __restrict__ pkey,
                                                         int32_t* __restrict__ pcnt, int* __restrict__ status,
                                                         const int* __restrict__ skip_if_exact,
                                                         const int32_t* __restrict__ count_dev,
                                                         const int32_t* __restrict__ leafid, int npass,
                                                         int32_t* __restrict__ ovf_list,
                                                         int32_t* __restrict__ ovf_count) {
    extern __shared__ float4 smem4[];
    if (*status & kStatusStop) return;
    if (count_dev && (int64_t)*count_dev < node1) node1 = *count_dev;
    if (skip_if_exact) {  // the tensor-core join does this round when the 16-bit copy is exact
        const int f = *skip_if_exact;
        if ((f & 1) == 0 && !((f & 2) && (f & 4))) return;
    }
    const bool lids = leafid != nullptr && npass > 0;
    const J2Layout L = j2_layout(D, mcap, lids);
    char* base = reinterpret_cast<char*>(smem4);
    uint64_t* thr = reinterpret_cast<uint64_t*>(base + L.thr);  // [G][mcap] by slot
    int4* slid = reinterpret_cast<int4*>(base + L.lid);         // [G][mcap] by slot
    float* rows = reinterpret_cast<float*>(base + L.rows);      // [G][mcap][stride] by slot
    int32_t* mem = reinterpret_cast<int32_t*>(base + L.mem);    // [G][mcap] by member index
    int* cnt = reinterpret_cast<int*>(base + L.cnt);            // [G] members, then [G] new members
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int RGN = L.RGN, NB = L.NB, G = L.G, dch = L.dch, stride = L.stride;
    // this thread's block, fixed for the launch
    const int jn = tid / NB, bk = tid - jn * NB;
    int rg = 0, cg = 0;
    {
        int b = bk;
        while (b >= RGN - rg) {
            b -= RGN - rg;
            ++rg;
        }
        cg = rg + b;
    }
    const bool vec = (D % 4 == 0);
    const int64_t ngroups = (node1 - node0 + G - 1) / G;
    for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int64_t first = node0 + grp * G;
        // members of the group's nodes (warp w collects nodes w, w + 8, ...):
        // the new ones first, then the old ones; each takes ids of G_old[i],
        // then of R[i]
        for (int j = warp; j < G; j += kJ2Threads / 32) {
            const int64_t pos = first + j;
            int M = 0, nn = 0;
            if (pos < node1) {
                const int64_t i = list ? (int64_t)list[pos] : pos;
                const uint64_t fbits = fnew ? fnew[i] : ~0ull, rbits = rnew ? rnew[i] : ~0ull;
                auto take_member = [&](uint64_t key, bool take) {
                    const unsigned bal = __ballot_sync(0xffffffffu, take);
                    if (take) {
                        const int m = M + __popc(bal & ((1u << lane) - 1u));
                        const uint32_t u = key_id(key);
                        const int sl = j * mcap + j2_slot(m, RGN);
                        mem[j * mcap + m] = (int32_t)u;
                        thr[sl] = Gold[(int64_t)u * k + k - 1];
                        if (lids) slid[sl] = __ldg(reinterpret_cast<const int4*>(leafid) + u);
                    }
                    M += __popc(bal);
                };
                if (!(rev && k > 32)) {
                    // at most 64 entries, a mutual neighbour once
                    uint64_t key0, key1;
                    bool new0, new1;
                    member_keys(Gold, R, i, k, rev != 0, fbits, rbits, key0, key1, new0, new1);
                    // more members than the slot holds (slots smaller than 2k):
                    // the node goes to the overflow list, for the full-slot launch
                    const int all = __popc(__ballot_sync(0xffffffffu, key0 != kEmptyKey)) +
                                    __popc(__ballot_sync(0xffffffffu, key1 != kEmptyKey));
                    if (all > mcap) {
                        if (lane == 0) ovf_list[atomicAdd(ovf_count, 1)] = (int32_t)i;
                        key0 = key1 = kEmptyKey;
                    }
                    for (int want = 1; want >= 0; --want) {
                        take_member(key0, key0 != kEmptyKey && new0 == (want == 1));
                        take_member(key1, key1 != kEmptyKey && new1 == (want == 1));
                        if (want == 1) nn = M;
                    }
                } else {
                    for (int want = 1; want >= 0; --want) {
                        for (int src = 0; src < 2; ++src) {
                            const uint64_t* row = (src == 0 ? Gold : R) + i * k;
                            const uint64_t bits = src == 0 ? fbits : rbits;
                            for (int e0 = 0; e0 < k; e0 += 32) {
                                const int e = e0 + lane;
                                const uint64_t key = e < k ? row[e] : kEmptyKey;
                                take_member(key, key != kEmptyKey && (int)((bits >> e) & 1ull) == want);
                            }
                        }
                        if (want == 1) nn = M;
                    }
                }
            }
            if (lane == 0) {
                cnt[j] = M;
                cnt[G + j] = nn;
            }
        }
        __syncthreads();
        const int Mj = jn < G ? cnt[jn] : 0, nnj = jn < G ? cnt[G + jn] : 0;
        // a block with a live pair: both groups hold members, one holds a new one
        const bool live = jn < G && 4 * rg < Mj && 4 * cg < Mj && (4 * rg < nnj || 4 * cg < nnj);
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
        const int q4 = dch >> 2;
        for (int d0 = 0; d0 < D; d0 += dch) {
            const int dl = min(dch, D - d0);
            // gather dims [d0, d0 + dch) of every member slot (zeros past
            // the members and past D)
            if (vec) {
                for (int e = tid; e < G * mcap * q4; e += kJ2Threads) {
                    const int sl = e / q4, c4 = e - sl * q4;
                    const int j = sl / mcap, s = sl - j * mcap;
                    const int m = (s % RGN) * 4 + s / RGN;  // the member stored in slot s
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (m < cnt[j] && c4 * 4 < dl)
                        v = __ldg(reinterpret_cast<const float4*>(X + (int64_t)mem[j * mcap + m] * D + d0) + c4);
                    *reinterpret_cast<float4*>(rows + (size_t)sl * stride + c4 * 4) = v;
                }
            } else {
                for (int e = tid; e < G * mcap * dch; e += kJ2Threads) {
                    const int sl = e / dch, c = e - sl * dch;
                    const int j = sl / mcap, s = sl - j * mcap;
                    const int m = (s % RGN) * 4 + s / RGN;
                    rows[(size_t)sl * stride + c] =
                        (m < cnt[j] && c < dl) ? __ldg(X + (int64_t)mem[j * mcap + m] * D + d0 + c) : 0.f;
                }
            }
            __syncthreads();
            if (live) {
                const float* rp = rows + (size_t)(jn * mcap + rg) * stride;
                const float* cp = rows + (size_t)(jn * mcap + cg) * stride;
                const int step = RGN * stride;  // member 4 g + a sits a RGN rows below member 4 g
                for (int dq = 0; dq < dch; dq += 4) {
                    float4 rv[4], cv[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) rv[a] = *reinterpret_cast<const float4*>(rp + a * step + dq);
#pragma unroll
                    for (int b = 0; b < 4; ++b) cv[b] = *reinterpret_cast<const float4*>(cp + b * step + dq);
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            float t = __fsub_rn(rv[a].x, cv[b].x);
                            acc[a][b] = __fmaf_rn(t, t, acc[a][b]);
                            t = __fsub_rn(rv[a].y, cv[b].y);
                            acc[a][b] = __fmaf_rn(t, t, acc[a][b]);
                            t = __fsub_rn(rv[a].z, cv[b].z);
                            acc[a][b] = __fmaf_rn(t, t, acc[a][b]);
                            t = __fsub_rn(rv[a].w, cv[b].w);
                            acc[a][b] = __fmaf_rn(t, t, acc[a][b]);
                        }
                }
            }
            __syncthreads();  // the next chunk overwrites the rows
        }
        // offers: count, reserve (one atomic per warp), write
        int c = 0;
        if (live) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int ia = 4 * rg + a, ib = 4 * cg + b;
                    if (ia < Mj && ib < Mj && (ia < nnj || ib < nnj) && (rg < cg || a < b)) {
                        const uint32_t u = (uint32_t)mem[jn * mcap + ia], v = (uint32_t)mem[jn * mcap + ib];
                        if (u != v) {
                            const int sa = jn * mcap + a * RGN + rg, sb = jn * mcap + b * RGN + cg;
                            const bool ou = make_key(acc[a][b], v) < thr[sa];
                            const bool ov = make_key(acc[a][b], u) < thr[sb];
                            if ((ou || ov) && !(lids && leaf_mates(slid[sa], slid[sb], npass))) c += ou + ov;
                        }
                    }
                }
        }
        const int incl = warp_incl_scan(c);
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (total > 0) {
            uint32_t at = 0;
            if (lane == 31) at = atomicAdd(counter, (uint32_t)total);
            at = __shfl_sync(0xffffffffu, at, 31);
            if ((int64_t)at + total > cap) {
                if (lane == 0) atomicOr(status, kStatusOverflow);
            } else if (c > 0) {
                uint32_t w = at + incl - c;
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int ia = 4 * rg + a, ib = 4 * cg + b;
                        if (ia < Mj && ib < Mj && (ia < nnj || ib < nnj) && (rg < cg || a < b)) {
                            const uint32_t u = (uint32_t)mem[jn * mcap + ia], v = (uint32_t)mem[jn * mcap + ib];
                            if (u != v) {
                                const int sa = jn * mcap + a * RGN + rg, sb = jn * mcap + b * RGN + cg;
                                const uint64_t ku = make_key(acc[a][b], v), kv = make_key(acc[a][b], u);
                                const bool ou = ku < thr[sa], ov = kv < thr[sb];
                                if ((ou || ov) && !(lids && leaf_mates(slid[sa], slid[sb], npass))) {
                                    if (ou) {
                                        ptgt[w] = u;
                                        pkey[w] = ku;
                                        ++w;
                                        atomicAdd(&pcnt[u], 1);
                                    }
                                    if (ov) {
                                        ptgt[w] = v;
                                        pkey[w] = kv;
                                        ++w;
                                        atomicAdd(&pcnt[v], 1);
                                    }
                                }
                            }
                        }
                    }
            }
        }
        __syncthreads();  // the next group overwrites members, thresholds and counts
    }
}

__global__ void k5_scatter(const uint32_t* __restrict__ ptgt, const uint64_t* __restrict__ pkey,
                           const uint32_t* __restrict__ counter, int64_t cap, const int32_t* __restrict__ poff,
                           int32_t* __restrict__ pcur, uint64_t* __restrict__ grouped,
                           const int* __restrict__ status, unsigned long long* __restrict__ offers_total) {
    // after an overflow some reserved slots were never written: group nothing
    if (*status & kStatusStop) return;
    const int64_t total = min((int64_t)*counter, cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(offers_total, (unsigned long long)total);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = ptgt[q];
        const int pos = poff[t] + atomicAdd(&pcur[t], 1);
        grouped[pos] = pkey[q];
    }
}

// An offer of `key` to a node whose sorted list is row[0..k) can change the
// list only if it beats the k-th entry and is not one of the entries already
// (an id always comes with the same canonical distance, hence the same key).
__device__ __forceinline__ bool offer_useful(uint64_t key, const uint64_t* row, int k) {
    if (!(key < row[k - 1])) return false;
    int lo = 0, len = k;
    while (len > 0) {
        const int half = len >> 1;
        if (row[lo + half] < key) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return row[lo] != key;
}

// Inserts id into a warp's open-addressing set of kSeenSlots ids (linear
// probing); true when it was not there.  The callers insert fewer ids than
// there are slots, so a probe always ends.
constexpr int kSeenSlots = 256;
constexpr int kSeenOffers = 160;  // offers per node taken through the set (with at most 32 list ids)
__device__ __forceinline__ bool seen_insert(uint32_t* tab, uint32_t id) {
    for (uint32_t h = (id * 2654435761u) >> 24, t = 0; t < kSeenSlots; ++t, h = (h + 1) & (kSeenSlots - 1)) {
        const uint32_t old = atomicCAS(&tab[h], 0xFFFFFFFFu, id);
        if (old == 0xFFFFFFFFu) return true;
        if (old == id) return false;
    }
    return false;
}

// Merges one node's offers into its list: the list sits in shared memory;
// every lane drops the offers that cannot change it, and only the rest go
// through the warp selection.  For k <= 32 and at most kSeenOffers offers the
// drop is by id in the warp's set `seen` (a pair always has the same canonical
// distance): the list's ids first, then each offer below the k-th key enters
// once, so the survivors are distinct and new and usually one bitonic merge
// takes them; a repeat of an offer that did not make the list cannot make it
// later either (the k-th key only falls).
template <int NO>
__device__ __forceinline__ void merge_node(uint64_t* __restrict__ Gnew, const uint64_t* __restrict__ grouped,
                                           int64_t u, int beg, int end, int k, uint64_t* srow, uint64_t* scratch,
                                           uint32_t* seen) {
    const int lane = threadIdx.x & 31;
    uint64_t* row = Gnew + u * k;
    uint64_t run[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) {
        run[o] = lane + 32 * o < k ? row[lane + 32 * o] : kEmptyKey;
        srow[lane + 32 * o] = run[o];
    }
    __syncwarp();
    constexpr int NC = 4;
    bool changed = false;
    const bool hashed = NO == 1 && end - beg <= kSeenOffers;
    if (hashed) {
        for (int t = lane; t < kSeenSlots; t += 32) seen[t] = 0xFFFFFFFFu;
        __syncwarp();
        if (run[0] != kEmptyKey) seen_insert(seen, key_id(run[0]));
        __syncwarp();
    }
    for (int c = beg; c < end; c += 32 * NC) {
        uint64_t a[NC + NO];
        bool any = false;
        const uint64_t kth = hashed ? shfl64(run[0], k - 1) : kEmptyKey;
#pragma unroll
        for (int s = 0; s < NC; ++s) {
            const int e = c + lane + 32 * s;
            a[s] = (e < end) ? grouped[e] : kEmptyKey;
            if (a[s] != kEmptyKey &&
                !(hashed ? (a[s] < kth && seen_insert(seen, key_id(a[s]))) : offer_useful(a[s], srow, k)))
                a[s] = kEmptyKey;
            any |= a[s] != kEmptyKey;
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        if (NO == 1) {  // usually few offers survive: one bitonic merge
            uint64_t few[NC], out;
            bool ch;
#pragma unroll
            for (int s = 0; s < NC; ++s) few[s] = a[s];
            if (warp_merge_few<NC>(few, run[0], k, scratch, out, ch)) {
                if (ch) {
                    run[0] = lane < k ? out : kEmptyKey;
                    __syncwarp();
                    srow[lane] = run[0];
                    __syncwarp();
                    changed = true;
                }
                continue;
            }
        }
#pragma unroll
        for (int o = 0; o < NO; ++o) a[NC + o] = run[o];
        sort_regs<NC + NO>(a);
        warp_select_unique<NC + NO, NO>(a, k, run);
        __syncwarp();
#pragma unroll
        for (int o = 0; o < NO; ++o) srow[lane + 32 * o] = run[o];
        __syncwarp();
        changed = true;
    }
    if (changed) {
#pragma unroll
        for (int o = 0; o < NO; ++o)
            if (lane + 32 * o < k) row[lane + 32 * o] = run[o];
    }
    __syncwarp();  // srow is reused by the warp's next node
}

// Warps stride over groups of 32 targets; the targets of a group that
// received offers are merged one after the other.
template <int NO>
__global__ void __launch_bounds__(256) k4_merge(uint64_t* __restrict__ Gnew, const uint64_t* __restrict__ grouped,
                                                const int32_t* __restrict__ poff, int64_t n, int k,
                                                const int* __restrict__ status) {
    __shared__ uint64_t rows[8][32 * NO];
    __shared__ uint64_t scratch[8][32];
    __shared__ uint32_t seen[8][NO == 1 ? kSeenSlots : 1];
    if (*status & kStatusStop) return;
    const int lane = threadIdx.x & 31;
    uint64_t* srow = rows[threadIdx.x >> 5];
    const int64_t warps = (int64_t)gridDim.x * 8;
    for (int64_t g0 = ((int64_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * 32; g0 < n; g0 += warps * 32) {
        const int64_t u = g0 + lane;
        const int beg = u < n ? poff[u] : 0, end = u < n ? poff[u + 1] : 0;
        unsigned todo = __ballot_sync(0xffffffffu, end > beg);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            merge_node<NO>(Gnew, grouped, g0 + src, __shfl_sync(0xffffffffu, beg, src),
                           __shfl_sync(0xffffffffu, end, src), k, srow, scratch[threadIdx.x >> 5],
                           seen[threadIdx.x >> 5]);
        }
    }
}

// One warp per leaf: slot `slot` of point perm[p]'s leaf ids = leaf, for the
// leaf's positions p.
__global__ void __launch_bounds__(256) k_leaf_ids(const int32_t* __restrict__ perm,
                                                  const int32_t* __restrict__ leaf_off, int nleaf, int slot,
                                                  int32_t* __restrict__ lid) {
    const int lane = threadIdx.x & 31;
    for (int l = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); l < nleaf;
         l += (int)((gridDim.x * (int64_t)blockDim.x) >> 5))
        for (int p = leaf_off[l] + lane; p < leaf_off[l + 1]; p += 32)
            lid[(int64_t)perm[p] * kMaxLeafPasses + slot] = l;
}

inline int grid_for(int64_t count, int block) {
    int64_t g = (count + block - 1) / block;
    if (g > 152 * 32) g = 152 * 32;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

size_t scan_tmp_ints(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 1; }

void launch_scan(const int32_t* cnt, int32_t* off, int64_t n, int32_t* tmp, cudaStream_t s) {
    const int nb = (int)((n + kScanTile - 1) / kScanTile);
    LaunchScope ls("k_scan", s, n * 8.0, 0, nb == 0 ? 0 : 3);
    if (nb == 0) {
        cudaMemsetAsync(off, 0, sizeof(int32_t), s);
        return;
    }
    k_scan_partial<<<nb, kScanBlock, 0, s>>>(cnt, n, tmp);
    k_scan_blocks<<<1, kScanBlock, 0, s>>>(tmp, nb);
    k_scan_final<<<nb, kScanBlock, 0, s>>>(cnt, n, tmp, off);
}

void launch_leaf_ids(const int32_t* perm, const int32_t* leaf_off, int nleaf, int64_t n, int slot, int32_t* lid,
                     cudaStream_t s) {
    if (nleaf <= 0) return;
    LaunchScope ls("k_leaf_ids", s, n * 8.0 + nleaf * 4.0, 0);
    k_leaf_ids<<<grid_for((int64_t)nleaf * 32, 256), 256, 0, s>>>(perm, leaf_off, nleaf, slot, lid);
}

void launch_fill_empty(uint64_t* G, int64_t count, cudaStream_t s) {
    LaunchScope ls("k_fill_empty", s, count * 8.0, 0);
    k_fill_empty<<<grid_for(count, 256), 256, 0, s>>>(G, count);
}

void launch_pack(const int32_t* ids, const float* d, uint64_t* G, int64_t count, int64_t n, int* status,
                 cudaStream_t s) {
    LaunchScope ls("k_pack", s, count * 16.0, 0);
    k_pack<<<grid_for(count, 256), 256, 0, s>>>(ids, d, G, count, n, status);
}

void launch_check_ids(const int32_t* ids, int64_t count, int64_t lo, int64_t hi, int* status, cudaStream_t s) {
    if (count <= 0) return;
    LaunchScope ls("k_check_ids", s, count * 4.0, 0);
    k_check_ids<<<grid_for(count, 256), 256, 0, s>>>(ids, count, lo, hi, status);
}

void launch_unpack(const uint64_t* G, int32_t* ids, float* d, int64_t count, cudaStream_t s, int64_t id_offset) {
    LaunchScope ls("k_unpack", s, count * 16.0, 0);
    k_unpack<<<grid_for(count, 256), 256, 0, s>>>(G, ids, d, count, id_offset);
}

void launch_reverse_lists(const uint64_t* G, int64_t n, int k, const JoinBuffers& b, cudaStream_t s) {
    const int64_t nk = n * k;
    cudaMemsetAsync(b.deg, 0, sizeof(int32_t) * (n + 1), s);
    cudaMemsetAsync(b.cur, 0, sizeof(int32_t) * n, s);
    {
        LaunchScope ls("k6_count", s, nk * 8.0 + nk * 4.0, 0);
        k6_count<<<grid_for(nk, 256), 256, 0, s>>>(G, nk, b.deg);
    }
    launch_scan(b.deg, b.roff, n, b.scan_tmp, s);
    {
        LaunchScope ls("k6_fill", s, nk * (8.0 + 8.0 + 8.0), 0);
        k6_fill<<<grid_for(nk, 256), 256, 0, s>>>(G, nk, k, b.roff, b.cur, b.rbuf);
    }
    LaunchScope ls("k6_select", s, nk * 16.0 + n * 8.0, 0);
    const int grid = (int)((n * 32 + 255) / 256);
    if (k > 32)
        k6_select<2><<<grid, 256, 0, s>>>(b.rbuf, b.roff, n, k, b.R);
    else
        k6_select<1><<<grid, 256, 0, s>>>(b.rbuf, b.roff, n, k, b.R);
}

int join_blocks_per_lane(int mcap) {
    const int rgn = (mcap + 3) / 4;
    const int nb = rgn * (rgn + 1) / 2;
    return (nb + 31) / 32;
}

// shared memory of one join CTA: per warp the member rows (mcap, a multiple
// of 4, rows of one dim chunk), their thresholds and their ids
size_t join_smem_bytes(int D, int mcap) {
    int dch, stride;
    join_chunk(D, mcap, &dch, &stride);
    return (size_t)kJoinWarps * ((size_t)mcap * (stride * 4 + 12) + 16);
}

namespace {

// One refinement round over the nodes at positions [0, count) of b.list
// (all nodes when b.list is NULL): reads Gold (and b.R), writes Gnew.
const char* launch_join_chunk(const float* X, int64_t n, int D, int k, bool rev, const uint64_t* Gold,
                              const JoinBuffers& b, bool tc, int64_t c0, int64_t c1, int mcap, int bpl, size_t smem,
                              int* status, cudaStream_t s);
void finish_chunk(int64_t n, int k, uint64_t* Gnew, const JoinBuffers& b, double offers, int* status,
                  cudaStream_t s);

// KNNG_JOIN_SCREEN=1: with a 16-bit copy that is not exact, the join screens
// pairs on the tensor cores and computes canonical distances only for those
// the screen cannot exclude (k5_join_tc_cert) instead of running the FP32 join.
// The screen runs on request (KNNG_JOIN_SCREEN=1): on every measured float
// workload the FP32 join was faster (unit-sphere D = 96: 934 against 730 ms;
// GIST-like D = 960: 434 against 285 ms), its canonical distances of the
// surviving pairs (a thread per pair over two FP32 rows) costing more than the
// pairs it saves.
bool join_screen(int D) {
    (void)D;
    const char* e = getenv("KNNG_JOIN_SCREEN");
    return e && e[0] == '1';
}

// Chunks are sized from `est` (offers per node, measured on the previous
// chunk), but never below nodes_per_chunk, which fits the offer buffer even
// when every member pair offers both ways.  After each join the offer
// counter is read back; on an overflow the flag is cleared and the join
// re-runs on a smaller chunk (no target list has been touched yet).  `tc`:
// the tensor-core join does the work.
// `Gbase`, when given, is the list Gnew starts from and Gold only the
// members' view (the sampled round); thresholds come from Gold either way.
void join_round(const float* X, int64_t n, int D, int k, bool rev, const uint64_t* Gold, uint64_t* Gnew,
                const JoinBuffers& b, bool tc, int64_t count, int64_t nodes_per_chunk, double& est, int* status,
                cudaStream_t s, const uint64_t* Gbase = nullptr) {
    cudaMemcpyAsync(Gnew, Gbase ? Gbase : Gold, sizeof(uint64_t) * n * k, cudaMemcpyDeviceToDevice, s);
    const int mcap = ((rev ? 2 * k : k) + 3) & ~3;
    const int bpl = join_blocks_per_lane(mcap);
    const size_t smem = join_smem_bytes(D, mcap);
    const double m_max = rev ? 2.0 * k : (double)k;
    // the 32-bit offer counter must not wrap, even in the worst case
    const int64_t wrap_nodes = (int64_t)(4294967295.0 / std::max(1.0, m_max * (m_max - 1)));
    if (b.capture) {  // no host reads: worst-case chunks over every position
        for (int64_t c0 = 0; c0 < count; c0 += nodes_per_chunk) {
            const int64_t c1 = std::min(count, c0 + nodes_per_chunk);
            launch_join_chunk(X, n, D, k, rev, Gold, b, tc, c0, c1, mcap, bpl, smem, status, s);
            finish_chunk(n, k, Gnew, b, 0.0, status, s);
        }
        return;
    }
    for (int64_t c0 = 0, c1 = 0; c0 < count; c0 = c1) {
        int64_t want = (int64_t)((double)b.cap / std::max(est, 1.0));
        want = std::max(nodes_per_chunk, std::min(want, wrap_nodes));
        c1 = std::min(count, c0 + want);
        uint32_t offers = 0;
        for (;;) {
            const char* who = launch_join_chunk(X, n, D, k, rev, Gold, b, tc, c0, c1, mcap, bpl, smem, status, s);
            int st = 0;
            cudaMemcpyAsync(&offers, b.counter, sizeof offers, cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(&st, status, sizeof st, cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            est = std::max((double)offers / (double)(c1 - c0), 1.0);
            // a chunk of nodes_per_chunk nodes cannot overflow; should it all
            // the same, the flag stays and the call reports it
            if ((int64_t)offers <= b.cap || c1 - c0 <= nodes_per_chunk) {
                record_bytes(who, std::min<double>(offers, (double)b.cap) * 12.0);  // offers written (id + key)
                break;
            }
            st &= ~kStatusOverflow;
            cudaMemcpyAsync(status, &st, sizeof st, cudaMemcpyHostToDevice, s);
            cudaStreamSynchronize(s);
            c1 = c0 + std::max(nodes_per_chunk, (int64_t)((double)(c1 - c0) * (double)b.cap / offers * 0.9));
            record_items("k5_join_retry", 1.0);
        }
        finish_chunk(n, k, Gnew, b, (double)offers, status, s);
    }
}

// The join of the chunk [c0, c1); returns the name of the kernel that ran.
const char* launch_join_chunk(const float* X, int64_t n, int D, int k, bool rev, const uint64_t* Gold,
                              const JoinBuffers& b, bool tc, int64_t c0, int64_t c1, int mcap, int bpl, size_t smem,
                              int* status, cudaStream_t s) {
    {
        cudaMemsetAsync(b.pcnt, 0, sizeof(int32_t) * (n + 1), s);
        cudaMemsetAsync(b.pcur, 0, sizeof(int32_t) * n, s);
        cudaMemsetAsync(b.counter, 0, sizeof(uint32_t), s);
        if (tc && launch_join_tc(b.Xq, D, b.qnrm, k, rev, Gold, b.R, c0, c1, b, status, b.notexact, b.bf16, s))
            return "k5_join_tc";
        // capture: the tensor-core join returns at once on the device unless
        // the copy is exact, and the FP32 join below returns at once if it is
        const bool tc_dev = b.capture && b.lp &&
                            launch_join_tc(b.Xq, D, b.qnrm, k, rev, Gold, b.R, c0, c1, b, status, b.notexact,
                                           b.bf16, s);
        // not exact: the tensor cores screen the pairs and canonical distances
        // decide (on request).  In a capture the screening join returns at
        // once on the device when the copy is exact (the exact join above has
        // run), so no FP32 join is needed
        if ((!tc || b.capture) && b.lp && join_screen(D) &&
            launch_join_tc(b.Xq, D, b.qnrm, k, rev, Gold, b.R, c0, c1, b, status, b.notexact, b.bf16, s, true, X))
            return "k5_join_tc_cert";
        {
            const double m = rev ? 2.0 * k : (double)k;
            const bool lids = b.leafid != nullptr && b.npass > 0;
            const J2Layout L2 = j2_layout(D, mcap, lids);
            // the CTA-wide kernel when it keeps clearly more lanes busy than
            // one node per warp (whose lanes idle when the block count is not
            // a multiple of 32)
            const double warp_eff = (double)L2.NB / (32.0 * ((L2.NB + 31) / 32));
            const double cta_eff = (double)(L2.G * L2.NB) / kJ2Threads;
            const bool cta = cta_eff >= warp_eff + 0.1;
            // With reverse lists a mutual neighbour is one member: slots of
            // three quarters of 2k when that packs more nodes into a CTA, the
            // nodes that overflow joined after them with full slots (their
            // count read on the device)
            const int small = (mcap * 3 / 4 + 3) & ~3;
            const bool packed = cta && rev && k <= 32 && b.ovf_list && b.ovf_count && small >= 4 &&
                                j2_layout(D, small, lids).G > L2.G;
            LaunchScope ls("k5_join", s, (double)(c1 - c0) * (m * D * 4.0 + 2 * k * 8.0 + m * 8.0),
                           (double)(c1 - c0) * m * (m - 1) / 2 * 3.0 * D, packed ? 2 : 1);
            if (cta) {
                auto cta_launch = [&](int mc, const int32_t* lst, const int32_t* cnt_dev, int64_t n0, int64_t n1,
                                      bool ovf) {
                    const J2Layout Lc = j2_layout(D, mc, lids);
                    cudaFuncSetAttribute(k5_join_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lc.total);
                    int per_sm = 0;
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k5_join_cta, kJ2Threads, Lc.total);
                    if (per_sm < 1) per_sm = 1;
                    const int64_t groups = (n1 - n0 + Lc.G - 1) / Lc.G;
                    const int grid2 = (int)std::max<int64_t>(1, std::min<int64_t>(groups, (int64_t)152 * per_sm));
                    k5_join_cta<<<grid2, kJ2Threads, Lc.total, s>>>(
                        X, D, k, rev ? 1 : 0, mc, Gold, b.R, lst, b.fnew, b.rnew, n0, n1, b.counter, b.cap, b.ptgt,
                        b.pkey, b.pcnt, status, tc_dev ? b.notexact : nullptr, cnt_dev, lids ? b.leafid : nullptr,
                        b.npass, ovf ? b.ovf_list : nullptr, ovf ? b.ovf_count : nullptr);
                };
                if (packed) {
                    cudaMemsetAsync(b.ovf_count, 0, sizeof(int32_t), s);
                    cta_launch(small, b.list, b.count_dev, c0, c1, true);
                    cta_launch(mcap, b.ovf_list, b.ovf_count, 0, c1 - c0, false);
                } else {
                    cta_launch(mcap, b.list, b.count_dev, c0, c1, false);
                }
                return "k5_join";
            }
            const int grid = (int)std::min<int64_t>((c1 - c0 + kJoinWarps - 1) / kJoinWarps, 152 * 32);
#define KNNG_JOIN(BPL)                                                                                     \
    do {                                                                                                   \
        cudaFuncSetAttribute(k5_join<BPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);        \
        k5_join<BPL><<<grid, 32 * kJoinWarps, smem, s>>>(X, D, k, rev ? 1 : 0, mcap, Gold, b.R, b.list,     \
                                                         b.fnew, b.rnew, c0, c1, b.counter, b.cap, b.ptgt,  \
                                                         b.pkey, b.pcnt, status,                            \
                                                         tc_dev ? b.notexact : nullptr,                     \
                                                         b.count_dev);                                      \
    } while (0)
            if (bpl <= 1) KNNG_JOIN(1);
            else if (bpl <= 2) KNNG_JOIN(2);
            else if (bpl <= 3) KNNG_JOIN(3);
            else if (bpl <= 4) KNNG_JOIN(4);
            else KNNG_JOIN(5);
#undef KNNG_JOIN
        }
    }
    return "k5_join";
}

// Groups the chunk's offers by target and merges them into Gnew.
void finish_chunk(int64_t n, int k, uint64_t* Gnew, const JoinBuffers& b, double offers, int* status,
                  cudaStream_t s) {
    {
        launch_scan(b.pcnt, b.poff, n, b.scan_tmp, s);
        {
            // per offer: target and key read, its target's offset, the key written
            LaunchScope ls("k5_scatter", s, offers * 24.0, 0);
            k5_scatter<<<152 * 16, 256, 0, s>>>(b.ptgt, b.pkey, b.counter, b.cap, b.poff, b.pcur, b.grouped,
                                                status, b.offers_total);
        }
        {
            // offsets, every grouped offer, and the list of each target reached
            // (at most min(n, offers) of them) read and written
            LaunchScope ls("k4_merge", s, n * 4.0 + offers * 8.0 + std::min((double)n, offers) * 16.0 * k, 0);
            const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
            if (k > 32)
                k4_merge<2><<<grid, 256, 0, s>>>(Gnew, b.grouped, b.poff, n, k, status);
            else
                k4_merge<1><<<grid, 256, 0, s>>>(Gnew, b.grouped, b.poff, n, k, status);
        }
    }
}

}  // namespace

void run_refine(const float* X, int64_t n, int D, int k, bool rev, uint64_t*& G, uint64_t*& G2,
                const JoinBuffers& jb, int64_t nodes_per_chunk, int rounds, int* status, cudaStream_t s) {
    JoinBuffers b = jb;
    // offers per node of the first round's chunks: a guess (a quarter of the
    // worst case); then what the previous chunk measured
    const double m_max = rev ? 2.0 * k : (double)k;
    double est = m_max * (m_max - 1) / 4;
    // the tensor-core join runs when the 16-bit copy is exact for this input
    bool tc = false;
    if (b.lp && !b.capture) {
        int f = 0;
        cudaMemcpyAsync(&f, b.notexact, sizeof f, cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        tc = (f & 1) == 0 && !((f & 2) && (f & 4));
    }
    for (int r = 0; r < rounds; ++r) {
        if (rev) launch_reverse_lists(G, n, k, b, s);  // into b.R; b.R2 keeps the previous round's
        b.list = b.order;  // every node (in the last tree pass's leaf order when it is known)
        b.fnew = b.rnew = nullptr;
        b.count_dev = nullptr;
        int64_t count = n;
        if (r > 0) {
            // G2 still holds the previous round's G_old
            cudaMemsetAsync(b.nactive, 0, sizeof(int32_t), s);
            {
                LaunchScope ls("k6_flags", s, n * k * 8.0 * (rev ? 4.0 : 2.0) + n * 20.0, 0);
                const int grid = (int)((n + kFlagWarps - 1) / kFlagWarps);
                // with an order, k6_active lists the nodes after the flags
                int32_t* act = b.order ? nullptr : b.active;
                if (k > 32)
                    k6_flags<2><<<grid, 32 * kFlagWarps, 0, s>>>(G, rev ? b.R : nullptr, G2, rev ? b.R2 : nullptr,
                                                                 n, k, b.fnew_buf, b.rnew_buf, act, b.nactive);
                else
                    k6_flags<1><<<grid, 32 * kFlagWarps, 0, s>>>(G, rev ? b.R : nullptr, G2, rev ? b.R2 : nullptr,
                                                                 n, k, b.fnew_buf, b.rnew_buf, act, b.nactive);
            }
            if (b.order) {
                // the order (4 B), the flags of each node (8 or 16 B), the list written (4 B)
                LaunchScope ls("k6_active", s, n * (rev ? 24.0 : 16.0), 0);
                k6_active<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(b.order, b.fnew_buf, rev ? b.rnew_buf : nullptr,
                                                                     n, b.active, b.nactive);
            }
            if (b.capture) {
                b.count_dev = b.nactive;  // the kernels read how many nodes are listed
            } else {
                int32_t h = 0;
                cudaMemcpyAsync(&h, b.nactive, sizeof h, cudaMemcpyDeviceToHost, s);
                cudaStreamSynchronize(s);
                count = h;
                record_items("k6_flags", (double)count);
            }
            b.list = b.active;
            b.fnew = b.fnew_buf;
            b.rnew = rev ? b.rnew_buf : nullptr;
        }
        join_round(X, n, D, k, rev, G, G2, b, tc, count, nodes_per_chunk, est, status, s);
        std::swap(G, G2);
        if (rev) std::swap(b.R, b.R2);
    }
}

void run_refine_sampled(const float* X, int64_t n, int D, int k, uint64_t*& G, uint64_t*& G2, const JoinBuffers& jb,
                        int64_t nodes_per_chunk, int rounds, int ms, uint64_t seed, int* status, cudaStream_t s) {
    JoinBuffers b = jb;
    double est = 2.0 * k * (2.0 * k - 1) / 4;
    bool tc = false;
    if (b.lp) {
        int f = 0;
        cudaMemcpyAsync(&f, b.notexact, sizeof f, cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        tc = (f & 1) == 0 && !((f & 2) && (f & 4));
    }
    cudaMemsetAsync(b.flags, 0xFF, sizeof(uint64_t) * n, s);  // every entry new before the first round
    for (int r = 0; r < rounds; ++r) {
        const uint64_t h0 = splitmix64(seed ^ (uint64_t)(uint32_t)r);
        // member view in R2, sampled-new mask in fnew_buf, reverse samples in R
        launch_sampled_prepare(G, b.flags, n, k, ms, h0, b.R2, b.fnew_buf, b.flags_post, b.deg, b.roff, b.cur,
                               b.scan_tmp, b.rbuf, b.R, b.rnew_buf, s);
        b.list = b.order;  // every node (in the last tree pass's leaf order when it is known)
        b.count_dev = nullptr;
        b.fnew = b.fnew_buf;
        b.rnew = b.rnew_buf;
        join_round(X, n, D, k, true, b.R2, G2, b, tc, n, nodes_per_chunk, est, status, s, G);
        launch_sampled_flags(G2, G, b.flags_post, n, k, b.flags, nullptr, s);
        std::swap(G, G2);
    }
}

}  // namespace knng
