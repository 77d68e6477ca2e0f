// rvq.cu -- residue vector quantisation (Sec. 4.1, Eqn. 1) and the inverted
// index whose lists seed the graph search (Sec. 4.2, Eqns. 2 and 3).
//
// Two stages of Lloyd's k-means: stage 1 on the points, stage 2 on the FP32
// residues x - w1[c1(x)].  An iteration assigns every vector to its nearest
// word (canonical FP32 distance, ties to the smaller word index), groups the
// vectors by word with a stable counting sort, and sets each word with members
// to the FP64 mean of its members summed in ascending vector order, rounded to
// FP32 (a word without members keeps its value).  So the words do not depend
// on the launch configuration: each sum has one fixed order.
//
// The index key of a point is c1 * W2 + c2; its lists hold ids ascending (two
// stable 8-bit counting-sort passes, c2 then c1).  A query ranks the stage-1
// words by term 1 of Eqn. 3, keeps the first probe1, ranks their keys by the
// full Eqn. 2 distance built from lookup tables (q.w1, q.w2, |w|^2, w1.w2) and
// takes the ids of the lists in that order as its seeds.  Every decision that
// a float makes (an argmin, a ranking) is taken in FP32 with a fixed operation
// order, the same on every launch.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace knng {

namespace {

// ---------------------------------------------------------------- assignment
constexpr int kAR = 64;    // vectors per CTA
constexpr int kAC = 128;   // words per column tile
constexpr int kAT = 256;   // threads: 16 row groups x 16 column groups, 4 x 8 each

// Dims per shared-memory chunk and the padded row stride (an odd number of
// float4 per row keeps the 16 row groups' float4 reads on distinct banks).
__host__ __device__ inline void assign_chunk(int D, int* dch, int* stride) {
    const int d4 = (D + 3) & ~3;
    const int c = d4 < 64 ? d4 : 64;
    *dch = c;
    *stride = ((c / 4) & 1) ? c : c + 4;
}

size_t assign_smem(int D) {
    int dch, stride;
    assign_chunk(D, &dch, &stride);
    return (size_t)(kAR + kAC) * stride * 4 + (size_t)(8 + 1) * kAR * 8 + kAR * 4;
}

// codes[i * out_stride] = argmin_c |v_i - words_c|^2 for the N vectors
// v_i = X_i (RES false) or X_i - W1[c1[i * c1_stride]] (RES true, FP32).
template <bool RES>
__global__ void __launch_bounds__(kAT) k9_assign(const float* __restrict__ X, int64_t N, int D,
                                                const float* __restrict__ W1, const int32_t* __restrict__ c1,
                                                int c1_stride, const float* __restrict__ words, int W,
                                                int32_t* __restrict__ out, int out_stride) {
    extern __shared__ float4 sm4[];
    int dch, stride;
    assign_chunk(D, &dch, &stride);
    float* rs = reinterpret_cast<float*>(sm4);                      // [kAR][stride]
    float* ws = rs + kAR * stride;                                  // [kAC][stride]
    uint64_t* red = reinterpret_cast<uint64_t*>(ws + kAC * stride);  // [8][kAR]
    uint64_t* best = red + 8 * kAR;                                 // [kAR]
    int32_t* rcode = reinterpret_cast<int32_t*>(best + kAR);        // [kAR]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rg = tid % 16, cg = tid / 16;
    const int64_t r0 = (int64_t)blockIdx.x * kAR;
    const int nr = (int)min((int64_t)kAR, N - r0);
    if (tid < kAR) {
        best[tid] = kEmptyKey;
        rcode[tid] = (RES && tid < nr) ? c1[(r0 + tid) * c1_stride] : 0;
    }
    for (int c0 = 0; c0 < W; c0 += kAC) {
        float acc[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
        for (int d0 = 0; d0 < D; d0 += dch) {
            const int dl = min(dch, D - d0);
            __syncthreads();
            for (int e = tid; e < kAR * dch; e += kAT) {
                const int r = e / dch, dd = e - r * dch;
                float v = 0.f;
                if (r < nr && dd < dl) {
                    v = __ldg(X + (r0 + r) * D + d0 + dd);
                    if (RES) v = __fsub_rn(v, __ldg(W1 + (int64_t)rcode[r] * D + d0 + dd));
                }
                rs[r * stride + dd] = v;
            }
            for (int e = tid; e < kAC * dch; e += kAT) {
                const int r = e / dch, dd = e - r * dch;
                float v = 0.f;
                if (c0 + r < W && dd < dl) v = __ldg(words + (int64_t)(c0 + r) * D + d0 + dd);
                ws[r * stride + dd] = v;
            }
            __syncthreads();
            const float* rp = rs + rg * stride;
            const float* cp = ws + cg * stride;
            for (int dq = 0; dq < dch; dq += 4) {
                float4 rv[4], cv[8];
#pragma unroll
                for (int i = 0; i < 4; ++i) rv[i] = *reinterpret_cast<const float4*>(rp + i * 16 * stride + dq);
#pragma unroll
                for (int j = 0; j < 8; ++j) cv[j] = *reinterpret_cast<const float4*>(cp + j * 16 * stride + dq);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        float t = __fsub_rn(rv[i].x, cv[j].x);
                        acc[i][j] = __fmaf_rn(t, t, acc[i][j]);
                        t = __fsub_rn(rv[i].y, cv[j].y);
                        acc[i][j] = __fmaf_rn(t, t, acc[i][j]);
                        t = __fsub_rn(rv[i].z, cv[j].z);
                        acc[i][j] = __fmaf_rn(t, t, acc[i][j]);
                        t = __fsub_rn(rv[i].w, cv[j].w);
                        acc[i][j] = __fmaf_rn(t, t, acc[i][j]);
                    }
            }
        }
        // the least (d, word) of each row in this tile: the thread's 8 words,
        // its partner of the other column group (lane ^ 16), then the 8 warps
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint64_t b = kEmptyKey;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = c0 + cg + 16 * j;
                if (c < W) b = min(b, make_key(acc[i][j], (uint32_t)c));
            }
            b = min(b, shfl_xor64(b, 16));
            if (lane < 16) red[warp * kAR + rg + 16 * i] = b;
        }
        __syncthreads();
        if (tid < kAR) {
            uint64_t b = best[tid];
#pragma unroll
            for (int w = 0; w < 8; ++w) b = min(b, red[w * kAR + tid]);
            best[tid] = b;
        }
    }
    __syncthreads();
    if (tid < nr) out[(r0 + tid) * out_stride] = (int32_t)key_id(best[tid]);
}

// ---------------------------------------------------------------- stable digit sort
constexpr int kDsThreads = 256;
constexpr int kDsItems = 8;
constexpr int kDsTile = kDsThreads * kDsItems;  // elements per CTA; a warp takes 256 consecutive ones

// Per-CTA histogram of the 8-bit digit key[id * kstride] of its elements
// (id = in[e], or e when in is null), stored digit-major: hist[d * nb + b].
__global__ void __launch_bounds__(kDsThreads) k9_digit_hist(const int32_t* __restrict__ in, int64_t n,
                                                           const int32_t* __restrict__ key, int kstride,
                                                           int32_t* __restrict__ hist, int nb) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kDsTile;
#pragma unroll
    for (int t = 0; t < kDsItems; ++t) {
        const int64_t e = base + t * kDsThreads + threadIdx.x;
        if (e < n) {
            const int64_t id = in ? (int64_t)__ldg(in + e) : e;
            atomicAdd(&h[__ldg(key + id * kstride) & 255], 1);
        }
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: element e goes to gofs[d * nb + b] + (elements of digit d
// before it in its CTA).  Warps take consecutive runs of 32 in element order;
// lanes with the same digit rank among themselves by lane (match_any).
__global__ void __launch_bounds__(kDsThreads) k9_digit_scatter(const int32_t* __restrict__ in, int64_t n,
                                                              const int32_t* __restrict__ key, int kstride,
                                                              const int32_t* __restrict__ gofs, int nb,
                                                              int32_t* __restrict__ out) {
    __shared__ int cnt[8][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < 8 * 256; d += kDsThreads) (&cnt[0][0])[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kDsTile + (int64_t)w * (32 * kDsItems);
    const unsigned lt = (1u << lane) - 1u;
    int32_t ids[kDsItems];
    int dig[kDsItems], rk[kDsItems];
#pragma unroll
    for (int t = 0; t < kDsItems; ++t) {
        const int64_t e = base + t * 32 + lane;
        const bool ok = e < n;
        const int32_t id = ok ? (in ? __ldg(in + e) : (int32_t)e) : 0;
        const int d = ok ? (__ldg(key + (int64_t)id * kstride) & 255) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        int r = __popc(peers & lt);
        if (ok) r += cnt[w][d];
        __syncwarp();
        if (ok && (peers & lt) == 0) cnt[w][d] += __popc(peers);
        __syncwarp();
        ids[t] = id;
        dig[t] = d;
        rk[t] = r;
    }
    __syncthreads();
    {   // exclusive prefix over the warps, one digit per thread
        int run = 0;
#pragma unroll
        for (int ww = 0; ww < 8; ++ww) {
            const int v = cnt[ww][threadIdx.x];
            cnt[ww][threadIdx.x] = run;
            run += v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kDsItems; ++t)
        if (dig[t] < 256) out[__ldg(gofs + (int64_t)dig[t] * nb + blockIdx.x) + cnt[w][dig[t]] + rk[t]] = ids[t];
}

// ---------------------------------------------------------------- word update
// One warp per (word, 32 dims): the FP64 sum of the members in ascending
// vector order (the sorted run order[gofs[c * nb] .. gofs[(c + 1) * nb])),
// divided by the count, rounded to FP32.  Loads run eight members ahead of
// the additions; the additions keep their order.
template <bool RES>
__global__ void __launch_bounds__(128) k9_update(const float* __restrict__ X, int D, const float* __restrict__ W1,
                                                const int32_t* __restrict__ c1, int c1_stride,
                                                const int32_t* __restrict__ order, const int32_t* __restrict__ gofs,
                                                int nb, int W, float* __restrict__ words) {
    const int nch = (D + 31) / 32;
    const int gw = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (gw >= W * nch) return;
    const int c = gw / nch, j = (gw - c * nch) * 32 + lane;
    const int a = __ldg(gofs + (int64_t)c * nb), b = __ldg(gofs + (int64_t)(c + 1) * nb);
    if (b == a || j >= D) return;  // no members: the word keeps its value
    auto value = [&](int t) {
        const int32_t id = __ldg(order + t);
        float v = __ldg(X + (int64_t)id * D + j);
        if (RES) v = __fsub_rn(v, __ldg(W1 + (int64_t)__ldg(c1 + (int64_t)id * c1_stride) * D + j));
        return v;
    };
    double acc = 0.0;
    int t = a;
    for (; t + 8 <= b; t += 8) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = value(t + u);
#pragma unroll
        for (int u = 0; u < 8; ++u) acc = __dadd_rn(acc, (double)v[u]);
    }
    for (; t < b; ++t) acc = __dadd_rn(acc, (double)value(t));
    words[(int64_t)c * D + j] = __double2float_rn(__ddiv_rn(acc, (double)(b - a)));
}

// words[c] = v_{pos[c]} (the initial words).
template <bool RES>
__global__ void k9_init_words(const float* __restrict__ X, int D, const float* __restrict__ W1,
                              const int32_t* __restrict__ c1, int c1_stride, const int64_t* __restrict__ pos, int W,
                              float* __restrict__ words) {
    const int64_t total = (int64_t)W * D;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / D), j = (int)(e - (int64_t)c * D);
        const int64_t id = pos[c];
        float v = X[id * D + j];
        if (RES) v = __fsub_rn(v, W1[(int64_t)c1[id * c1_stride] * D + j]);
        words[e] = v;
    }
}

// R_i = X_i - W1[c1[i]] (FP32), the stage-2 vectors, written once for all
// of stage 2's iterations.
__global__ void k9_residues(const float* __restrict__ X, int64_t N, int D, const float* __restrict__ W1,
                            const int32_t* __restrict__ c1, float* __restrict__ R) {
    const int64_t total = N * D;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / D;
        R[e] = __fsub_rn(X[e], W1[(int64_t)c1[i] * D + (e - i * D)]);
    }
}

// ---------------------------------------------------------------- index
__global__ void k9_key_count(const int32_t* __restrict__ codes, int64_t n, int W2, int32_t* __restrict__ cnt) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + (int64_t)codes[2 * e] * W2 + codes[2 * e + 1], 1);
}

// Offsets given by the caller: off[0] >= 0, non-decreasing, off[nk] <= n.
__global__ void k9_check_offsets(const int32_t* __restrict__ off, int64_t nk, int64_t n, int* status) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e <= nk; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = off[e];
        const bool bad = (e == 0 && v < 0) || (e > 0 && v < off[e - 1]) || (e == nk && (int64_t)v > n);
        if (bad) atomicOr(status, kStatusBadInput);
    }
}

// ---------------------------------------------------------------- query tables
__device__ __forceinline__ float dot_canon(const float* __restrict__ a, const float* __restrict__ b, int D) {
    float acc = 0.f;
    for (int j = 0; j < D; ++j) acc = __fmaf_rn(__ldg(a + j), __ldg(b + j), acc);
    return acc;
}

// n1[a] = |w1_a|^2, n2[b] = |w2_b|^2, x12[a][b] = w1_a . w2_b (canonical), and
// the transposed vocabularies w1T (D x W1), w2T (D x W2) for coalesced query
// products.
__global__ void k9_tables(const float* __restrict__ w1, int W1, const float* __restrict__ w2, int W2, int D,
                          float* __restrict__ n1, float* __restrict__ n2, float* __restrict__ x12,
                          float* __restrict__ w1T, float* __restrict__ w2T) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = g; e < (int64_t)W1 * W2; e += gs) {
        const int a = (int)(e / W2), b = (int)(e - (int64_t)a * W2);
        x12[e] = dot_canon(w1 + (int64_t)a * D, w2 + (int64_t)b * D, D);
    }
    for (int64_t e = g; e < W1; e += gs) n1[e] = dot_canon(w1 + e * D, w1 + e * D, D);
    for (int64_t e = g; e < W2; e += gs) n2[e] = dot_canon(w2 + e * D, w2 + e * D, D);
    for (int64_t e = g; e < (int64_t)W1 * D; e += gs) {
        const int a = (int)(e / D), j = (int)(e - (int64_t)a * D);
        w1T[(int64_t)j * W1 + a] = w1[e];
    }
    for (int64_t e = g; e < (int64_t)W2 * D; e += gs) {
        const int b = (int)(e / D), j = (int)(e - (int64_t)b * D);
        w2T[(int64_t)j * W2 + b] = w2[e];
    }
}

// ---------------------------------------------------------------- seeds
constexpr int kSdT = 256;

// Ascending bitonic sort of P keys (P a power of two >= 2) in shared memory by
// the whole CTA.  The caller synchronises before; this returns synchronised.
__device__ void block_bitonic(uint64_t* a, int P) {
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += kSdT) {
                const int l = i ^ j;
                if (l > i) {
                    const uint64_t x = a[i], y = a[l];
                    if ((x > y) == ((i & k) == 0)) {
                        a[i] = y;
                        a[l] = x;
                    }
                }
            }
            __syncthreads();
        }
}

// Exclusive scan of one int per thread over the CTA; *total gets the sum.
__device__ int block_excl_scan(int v, int* wsum, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int i = 0; i < kSdT / 32; ++i) {
            const int t = wsum[i];
            wsum[i] = run;
            run += t;
        }
        *total = run;
    }
    __syncthreads();
    return wsum[w] + x - v;
}

size_t seeds_smem(int P, int D) { return (size_t)P * 8 + 256 * 8 + (kSdT / 32 + 1) * 4 + 256 * 4 + (size_t)D * 4; }

// One CTA per query.  P: room for the candidate keys (probe1 * W2 rounded up
// to a power of two, at least kSdT); only those with a non-empty list are
// ranked.
__global__ void __launch_bounds__(kSdT) k9_seeds(const float* __restrict__ w1T, int W1,
                                                const float* __restrict__ w2T, int W2, int D,
                                                const float* __restrict__ n1, const float* __restrict__ n2,
                                                const float* __restrict__ x12, const int32_t* __restrict__ off,
                                                const int32_t* __restrict__ ids, const float* __restrict__ Q,
                                                int p1, int P, int s, int32_t* __restrict__ S,
                                                const int* __restrict__ status) {
    if (*status & kStatusStop) return;  // the caller's offsets failed their check
    extern __shared__ uint64_t smk[];
    uint64_t* cand = smk;                                   // [P]
    uint64_t* t1 = cand + P;                                // [256]
    int* wsum = reinterpret_cast<int*>(t1 + 256);           // [kSdT / 32 + 1]
    float* qw2 = reinterpret_cast<float*>(wsum + kSdT / 32 + 1);  // [256]
    float* q = qw2 + 256;                                   // [D]
    const int tid = threadIdx.x;
    const int64_t qi = blockIdx.x;
    for (int j = tid; j < D; j += kSdT) q[j] = __ldg(Q + qi * D + j);
    __syncthreads();
    float qq = 0.f;  // every thread, the same value
    for (int j = 0; j < D; ++j) qq = __fmaf_rn(q[j], q[j], qq);
    // Eqn. 3's term 1 for every stage-1 word, and q . w2
    uint64_t k1 = kEmptyKey;
    if (tid < W1) {
        float a = 0.f;
        for (int j = 0; j < D; ++j) a = __fmaf_rn(q[j], __ldg(w1T + (int64_t)j * W1 + tid), a);
        const float t = __fadd_rn(__fadd_rn(__fmaf_rn(-2.f, a, qq), __ldg(n1 + tid)), 0.f);
        k1 = make_key(t, (uint32_t)tid);
    }
    t1[tid] = k1;
    if (tid < W2) {
        float a = 0.f;
        for (int j = 0; j < D; ++j) a = __fmaf_rn(q[j], __ldg(w2T + (int64_t)j * W2 + tid), a);
        qw2[tid] = a;
    }
    __syncthreads();
    block_bitonic(t1, 256);
    // term 2 for the kept words' keys, d(q, I) = term 1 + term 2 (Eqn. 2).
    // Keys of empty lists add no seed: only the others are kept (in any
    // order, the sort below fixes it), with their list's start and length.
    __shared__ int nkeep;
    if (tid == 0) nkeep = 0;
    __syncthreads();
    const int nc = p1 * W2;
    for (int e0 = 0; e0 < nc; e0 += kSdT) {
        const int e = e0 + tid;
        uint64_t key = kEmptyKey;
        if (e < nc) {
            const int r = e / W2, b = e - r * W2;
            const uint64_t kk = t1[r];
            const int a = (int)key_id(kk), I = a * W2 + b;
            if (__ldg(off + I + 1) > __ldg(off + I)) {
                const float t2 =
                    __fmaf_rn(-2.f, qw2[b], __fmaf_rn(2.f, __ldg(x12 + (int64_t)a * W2 + b), __ldg(n2 + b)));
                const float d = __fadd_rn(__fadd_rn(key_dist(kk), t2), 0.f);
                key = make_key(d, (uint32_t)I);
            }
        }
        const unsigned ball = __ballot_sync(0xffffffffu, key != kEmptyKey);
        int base = 0;
        if ((tid & 31) == 0 && ball) base = atomicAdd(&nkeep, __popc(ball));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (key != kEmptyKey) cand[base + __popc(ball & ((1u << (tid & 31)) - 1u))] = key;
    }
    __syncthreads();
    const int nk = nkeep;
    int Pk = 2;
    while (Pk < nk) Pk <<= 1;
    for (int e = nk + tid; e < Pk; e += kSdT) cand[e] = kEmptyKey;
    __syncthreads();
    block_bitonic(cand, Pk);
    // the lists in that order: thread t walks keys [t * per, (t + 1) * per)
    const int per = (Pk + kSdT - 1) / kSdT;
    int mine = 0;
    for (int u = 0; u < per; ++u) {
        const int e = tid * per + u;
        if (e >= nk) break;
        const int I = (int)key_id(cand[e]);
        mine += __ldg(off + I + 1) - __ldg(off + I);
    }
    __shared__ int total;
    int pos = block_excl_scan(mine, wsum, &total);
    for (int u = 0; u < per && pos < s; ++u) {
        const int e = tid * per + u;
        if (e >= nk) break;
        const int I = (int)key_id(cand[e]);
        const int a0 = __ldg(off + I), a1 = __ldg(off + I + 1);
        for (int t = a0; t < a1 && pos < s; ++t) S[qi * s + pos++] = __ldg(ids + t);
    }
    for (int p = min(total, s) + tid; p < s; p += kSdT) S[qi * s + p] = -1;
}

int grid_for_count(int64_t count) {
    const int64_t g = (count + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

}  // namespace

// ---------------------------------------------------------------- launchers
void launch_rvq_assign(const float* X, int64_t N, int D, const float* W1, const int32_t* c1, int c1_stride,
                       const float* words, int W, int32_t* out, int out_stride, cudaStream_t s) {
    if (N <= 0) return;
    const size_t smem = assign_smem(D);
    const int64_t grid = (N + kAR - 1) / kAR;
    const bool res = W1 != nullptr;
    LaunchScope ls(res ? "k9_assign_res" : "k9_assign", s, (double)N * D * (res ? 8.0 : 4.0) + N * 4.0,
                   (double)N * W * D * 3.0);
    if (res) {
        cudaFuncSetAttribute(k9_assign<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k9_assign<true><<<(unsigned)grid, kAT, smem, s>>>(X, N, D, W1, c1, c1_stride, words, W, out, out_stride);
    } else {
        cudaFuncSetAttribute(k9_assign<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k9_assign<false><<<(unsigned)grid, kAT, smem, s>>>(X, N, D, nullptr, nullptr, 0, words, W, out, out_stride);
    }
}

int digit_sort_blocks(int64_t n) { return (int)std::max<int64_t>(1, (n + kDsTile - 1) / kDsTile); }

size_t digit_sort_hist_ints(int64_t n) { return (size_t)256 * digit_sort_blocks(n); }

void launch_digit_sort(const int32_t* in, int64_t n, const int32_t* key, int kstride, int32_t* out, int32_t* hist,
                       int32_t* gofs, int32_t* scan_tmp, cudaStream_t s) {
    const int nb = digit_sort_blocks(n);
    {
        LaunchScope ls("k9_digit_hist", s, n * (in ? 8.0 : 4.0) + 256.0 * nb * 4, 0);
        k9_digit_hist<<<nb, kDsThreads, 0, s>>>(in, n, key, kstride, hist, nb);
    }
    launch_scan(hist, gofs, (int64_t)256 * nb, scan_tmp, s);
    LaunchScope ls("k9_digit_scatter", s, n * (in ? 12.0 : 8.0) + 256.0 * nb * 4, 0);
    k9_digit_scatter<<<nb, kDsThreads, 0, s>>>(in, n, key, kstride, gofs, nb, out);
}

void launch_rvq_update(const float* X, int64_t N, int D, const float* W1, const int32_t* c1, int c1_stride,
                       const int32_t* order, const int32_t* gofs, int nb, int W, float* words, cudaStream_t s) {
    const int warps = W * ((D + 31) / 32);
    LaunchScope ls(W1 ? "k9_update_res" : "k9_update", s, (double)N * D * (W1 ? 8.0 : 4.0) + N * 4.0, (double)N * D);
    if (W1)
        k9_update<true><<<(warps + 3) / 4, 128, 0, s>>>(X, D, W1, c1, c1_stride, order, gofs, nb, W, words);
    else
        k9_update<false><<<(warps + 3) / 4, 128, 0, s>>>(X, D, nullptr, nullptr, 0, order, gofs, nb, W, words);
}

void launch_rvq_init(const float* X, int D, const float* W1, const int32_t* c1, int c1_stride, const int64_t* pos,
                     int W, float* words, cudaStream_t s) {
    LaunchScope ls("k9_init_words", s, (double)W * D * 8.0, 0);
    const int grid = grid_for_count((int64_t)W * D);
    if (W1)
        k9_init_words<true><<<grid, 256, 0, s>>>(X, D, W1, c1, c1_stride, pos, W, words);
    else
        k9_init_words<false><<<grid, 256, 0, s>>>(X, D, nullptr, nullptr, 0, pos, W, words);
}

void launch_rvq_residues(const float* X, int64_t N, int D, const float* W1, const int32_t* c1, float* R,
                         cudaStream_t s) {
    if (N <= 0) return;
    LaunchScope ls("k9_residues", s, (double)N * D * 12.0 + N * 4.0, (double)N * D);
    k9_residues<<<grid_for_count(N * D), 256, 0, s>>>(X, N, D, W1, c1, R);
}

void launch_rvq_key_count(const int32_t* codes, int64_t n, int W2, int32_t* cnt, cudaStream_t s) {
    if (n <= 0) return;
    LaunchScope ls("k9_key_count", s, n * 12.0, 0);
    k9_key_count<<<grid_for_count(n), 256, 0, s>>>(codes, n, W2, cnt);
}

void launch_check_offsets(const int32_t* off, int64_t nk, int64_t n, int* status, cudaStream_t s) {
    LaunchScope ls("k9_check_offsets", s, (nk + 1) * 4.0, 0);
    k9_check_offsets<<<grid_for_count(nk + 1), 256, 0, s>>>(off, nk, n, status);
}

void launch_rvq_tables(const float* w1, int W1, const float* w2, int W2, int D, float* n1, float* n2, float* x12,
                       float* w1T, float* w2T, cudaStream_t s) {
    LaunchScope ls("k9_tables", s, (double)(W1 + W2) * D * 12.0 + (double)W1 * W2 * 4.0,
                   (double)(W1 + 1) * (W2 + 1) * D * 2.0);
    k9_tables<<<grid_for_count((int64_t)W1 * W2), 256, 0, s>>>(w1, W1, w2, W2, D, n1, n2, x12, w1T, w2T);
}

int rvq_seed_keys(int probe1, int W2) {
    int P = kSdT;
    while (P < probe1 * W2) P <<= 1;
    return P;
}

size_t rvq_seeds_smem(int probe1, int W2, int D) { return seeds_smem(rvq_seed_keys(probe1, W2), D); }

void launch_rvq_seeds(const float* w1T, int W1, const float* w2T, int W2, int D, const float* n1, const float* n2,
                      const float* x12, const int32_t* off, const int32_t* ids, const float* Q, int64_t m, int probe1,
                      int s_seeds, int32_t* S, const int* status, cudaStream_t s) {
    if (m <= 0) return;
    const int P = rvq_seed_keys(probe1, W2);
    const size_t smem = seeds_smem(P, D);
    // algorithmic bytes: the query, both vocabularies (cached across queries,
    // counted once per query as a bound), the kept rows of w1.w2, the offsets
    // of the candidate keys and the seeds written
    LaunchScope ls("k9_seeds", s,
                   (double)m * (D * 4.0 + (double)(W1 + W2) * D * 4.0 + (double)probe1 * W2 * 12.0 + s_seeds * 8.0),
                   (double)m * (W1 + W2) * D * 2.0);
    cudaFuncSetAttribute(k9_seeds, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k9_seeds<<<(unsigned)m, kSdT, smem, s>>>(w1T, W1, w2T, W2, D, n1, n2, x12, off, ids, Q, probe1, P, s_seeds, S,
                                             status);
}

}  // namespace knng
