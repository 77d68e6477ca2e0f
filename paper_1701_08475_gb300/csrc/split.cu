// split.cu -- K1: one level of the balanced two-means tree (Sec. 3.1: the
// reference set is bisected repeatedly by two-means clustering; Alg. 1
// "apply two means clustering").
//
// Every segment of a level is split at once.  A segment holds its ids in
// ascending order; a split keeps that order on both sides.  One Lloyd
// iteration is
//   project  s_p = x_p . (c1 - c0)          canonical FP32 order (one thread
//                                           per point, dims ascending, fmaf)
//   select   the floor(m/2)-th smallest key (s_p, position) by radix select
//   sums     FP64 sums of the left and right points (fixed reduction order)
//   centroid c0 = mean(left), c1 = mean(right), FP64 divided then rounded
// and the level ends with a final project + select + stable partition.
// With a balanced cut only the order of ||x-c0||^2 - ||x-c1||^2 matters, and
// x . (c1 - c0) has the same order.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdlib>

#include "common.cuh"
#include "kernels.h"

namespace knng {

namespace {

__device__ __forceinline__ uint64_t sel_key(float s, int pos, int pos_bits) {
    return ((uint64_t)ord32(s) << pos_bits) | (uint32_t)pos;
}

// Inclusive/exclusive block scan of one int per thread (blockDim multiple of 32).
__device__ __forceinline__ int block_excl_scan(int v, int* warp_tot, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    const int before = warp ? warp_tot[warp - 1] : 0;
    *total = warp_tot[nw - 1];
    __syncthreads();
    return before + x - v;
}

__device__ __forceinline__ int block_sum(int v, int* warp_tot) {
    int total;
    block_excl_scan(v, warp_tot, &total);
    return total;
}

// Warp 0: digit b with below(b) <= krem < below(b) + hist[b].
// Radix digits of a selection key (ord32(s) << pos_bits | position), from the
// top: the 32 value bits in digits of 11, 11 and 10 bits, then the position
// bits 11 at a time.  `hi` is a digit's upper bound; returns its lower one.
// Once the value digits are done with krem = 0, the selected key is the first
// of its value, so (value << pos_bits) is an equivalent threshold (every key
// of that value goes right) and the position digits are skipped.
__host__ __device__ inline int digit_lo(int hi, int pos_bits) {
    return hi > pos_bits ? (hi - kRadixBits > pos_bits ? hi - kRadixBits : pos_bits)
                         : (hi - kRadixBits > 0 ? hi - kRadixBits : 0);
}

__device__ __forceinline__ void find_digit(const uint32_t* hist, int nb, uint32_t krem, int* out_digit,
                                           uint32_t* out_below) {
    const int lane = threadIdx.x & 31;
    const int per = nb >= 32 ? nb / 32 : 1;
    const int b0 = lane * per;
    uint32_t sum = 0;
    for (int b = b0; b < b0 + per && b < nb; ++b) sum += hist[b];
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t excl = incl - sum;
    if (excl <= krem && krem < incl) {
        uint32_t run = excl;
        for (int b = b0; b < b0 + per && b < nb; ++b) {
            if (krem < run + hist[b]) {
                *out_digit = b;
                *out_below = run;
                break;
            }
            run += hist[b];
        }
    }
}

// find_digit with the whole CTA: thread t sums bins [t per, (t + 1) per), one
// block scan, and the thread whose range holds rank krem walks its bins.
// Called by every thread of the CTA (it synchronises).
__device__ __forceinline__ void block_find_digit(const uint32_t* hist, int nb, uint32_t krem, int* warp_tot,
                                                 int* out_digit, uint32_t* out_below) {
    const int per = nb >= (int)blockDim.x ? nb / (int)blockDim.x : 1;
    const int b0 = (int)threadIdx.x * per;
    uint32_t sum = 0;
    for (int b = b0; b < b0 + per && b < nb; ++b) sum += hist[b];
    int total;
    const uint32_t excl = (uint32_t)block_excl_scan((int)sum, warp_tot, &total);
    if (sum > 0 && excl <= krem && krem < excl + sum) {
        uint32_t run = excl;
        for (int b = b0; b < b0 + per && b < nb; ++b) {
            if (krem < run + hist[b]) {
                *out_digit = b;
                *out_below = run;
                break;
            }
            run += hist[b];
        }
    }
}

__global__ void k1_init(const float* __restrict__ X, int D, const int32_t* __restrict__ perm,
                        const int32_t* __restrict__ seg_off, const int32_t* __restrict__ seg_tile0,
                        const int32_t* __restrict__ seg_local, int level, uint64_t pass_seed,
                        float* __restrict__ W, const int* __restrict__ status) {
    if (*status & kStatusStop) return;  // perm may hold unwritten slots
    const int seg = blockIdx.x;
    if (seg_tile0[seg + 1] == seg_tile0[seg]) return;  // a finished tree's leaf: it does not split
    const int a = seg_off[seg];
    const int m = seg_off[seg + 1] - a;
    // initial centroids: the points at positions h, h2 of the segment, drawn
    // from SplitMix64 of (pass seed, level, segment index in its own tree);
    // h2 != h
    const uint64_t sl = seg_local ? (uint64_t)seg_local[seg] : (uint64_t)seg;
    const uint64_t r1 = splitmix64(splitmix64(splitmix64(pass_seed) ^ (uint64_t)level) ^ sl);
    const uint64_t r2 = splitmix64(r1);
    const int64_t h = (int64_t)(r1 % (uint64_t)m);
    const int64_t h2 = (h + 1 + (int64_t)(r2 % (uint64_t)(m - 1))) % m;
    const float* c0 = X + (int64_t)perm[a + h] * D;
    const float* c1 = X + (int64_t)perm[a + h2] * D;
    for (int j = threadIdx.x; j < D; j += blockDim.x) W[(int64_t)seg * D + j] = __fsub_rn(c1[j], c0[j]);
}

// s_p = x_{perm[p]} . w_seg in the canonical order: one thread owns a point
// and accumulates its dims in ascending order with fmaf.  Rows are staged in
// shared memory 64 dims at a time (a warp loads 32 rows' 256-byte pieces,
// all in flight at once) so that global loads stay coalesced.
// When the 16-bit copy holds every value exactly (flag from the quantize
// kernel), the sweeps read it instead of X: the same FP32 values, half the
// bytes.  qtype: 1 = BF16, 2 = FP16.
__device__ __forceinline__ bool q16_usable(const uint16_t* Xq, const int* qflag) {
    if (Xq == nullptr) return false;
    const int f = *qflag;
    return (f & 1) == 0 && !((f & 2) && (f & 4));
}
template <int Q>  // 1 = BF16, 2 = FP16
__device__ __forceinline__ float q16_to_float(uint32_t h) {
    if (Q == 1) return __uint_as_float(h << 16);
    return __half2float(__ushort_as_half((unsigned short)h));
}

// Byte copy: when every value of X is an integer in [0, 255] (flag from
// k0_bytes), the staged sweeps read one byte per value instead of four (or
// two).  Byte i of `word` as a float, exactly: the byte becomes the low
// mantissa bits of 2^23, which the subtraction then removes.
__device__ __forceinline__ bool u8_usable(const uint8_t* Xb, const int* bflag) {
    return Xb != nullptr && *bflag == 0;
}
__device__ __forceinline__ bool exact_ints(const uint16_t* Xq, const int* qflag, const uint8_t* Xb,
                                          const int* bflag) {
    return u8_usable(Xb, bflag) || q16_usable(Xq, qflag);
}
// Every value of X an integer of magnitude <= 2048 (one of the exact copies is
// usable): then the sums of a tile are exact integers below 2^24 and travel
// as int32 partials, and a segment's sums are int64.
__device__ __forceinline__ bool exact_ints(const uint16_t* Xq, const int* qflag, const uint8_t* Xb,
                                          const int* bflag);
__device__ __forceinline__ float u8_to_float(uint32_t word, int i) {
    return __fsub_rn(__uint_as_float(__byte_perm(word, 0x4B000000u, 0x7540u + (uint32_t)i)), 8388608.f);
}

// Writes the byte copy (rows of Db bytes, zero padded) and sets *bflag when
// some value is not an integer in [0, 255]; once it is set, the remaining
// CTAs return at once.  One warp per row, 4 values per lane and step.
__global__ void __launch_bounds__(256) k0_bytes(const float* __restrict__ X, int64_t n, int D, int Db,
                                                uint8_t* __restrict__ Xb, int* __restrict__ bflag) {
    if (*(volatile int*)bflag) return;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= n) return;
    const int lane = threadIdx.x & 31;
    bool ok = true;
    for (int d0 = lane * 4; d0 < Db; d0 += 128) {
        uint32_t word = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int d = d0 + j;
            const float x = d < D ? X[r * D + d] : 0.f;
            ok &= x == rintf(x) && x >= 0.f && x <= 255.f;
            word |= (uint32_t)(ok ? (int)x : 0) << (8 * j);
        }
        *reinterpret_cast<uint32_t*>(Xb + r * Db + d0) = word;
    }
    if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicOr(bflag, 1);
}

// One sweep tile of the projection.  Q = 0 reads the FP32 rows of X (VEC2:
// as float2), Q = 1 / 2 the BF16 / FP16 copy; every load of a 64-dim slab is
// issued before any value is used.
template <bool VEC2, int Q>
__device__ __forceinline__ void project_tile(const float* __restrict__ X, int D, const uint16_t* __restrict__ Xq,
                                             int Dq, const int32_t* __restrict__ perm, int begin, int end,
                                             const float* __restrict__ w, float* __restrict__ S, float (*xs)[65],
                                             float* ws) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int base = begin; base < end; base += 256) {
        const int cnt = min(256, end - base);
        const int my_row = threadIdx.x < cnt ? perm[base + threadIdx.x] : 0;
        float acc = 0.f;
        for (int d0 = 0; d0 < D; d0 += 64) {
            const int dl = min(64, D - d0);
            if (threadIdx.x < 64) ws[threadIdx.x] = threadIdx.x < dl ? w[d0 + threadIdx.x] : 0.f;
            float2 v[32];
            uint32_t h[32];  // Q != 0: two raw 16-bit values
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int row = __shfl_sync(0xffffffffu, my_row, q);
                const bool live = warp * 32 + q < cnt && 2 * lane < dl;
                v[q] = make_float2(0.f, 0.f);
                h[q] = 0u;
                if (Q != 0) {  // rows padded to Dq: the pair is in bounds
                    if (live) h[q] = __ldg(reinterpret_cast<const uint32_t*>(Xq + (int64_t)row * Dq + d0 + 2 * lane));
                } else {
                    const float* src = X + (int64_t)row * D + d0 + 2 * lane;
                    if (VEC2) {
                        if (live) v[q] = __ldg(reinterpret_cast<const float2*>(src));
                    } else if (live) {
                        v[q].x = __ldg(src);
                        if (2 * lane + 1 < dl) v[q].y = __ldg(src + 1);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                if (Q != 0) v[q] = make_float2(q16_to_float<Q>(h[q] & 0xFFFFu), q16_to_float<Q>(h[q] >> 16));
                xs[warp * 32 + q][2 * lane] = v[q].x;
                xs[warp * 32 + q][2 * lane + 1] = v[q].y;
            }
            __syncthreads();
            if (threadIdx.x < cnt)
                for (int dd = 0; dd < dl; ++dd) acc = __fmaf_rn(xs[threadIdx.x][dd], ws[dd], acc);
            __syncthreads();
        }
        if (threadIdx.x < cnt) S[base + threadIdx.x] = __fadd_rn(acc, 0.f);  // -0 -> +0
    }
}

template <bool VEC2>
__global__ void __launch_bounds__(256) k1_project(const float* __restrict__ X, int D,
                                                  const int32_t* __restrict__ perm,
                                                  const int4* __restrict__ tiles,
                                                  const int32_t* __restrict__ seg_off,
                                                  const float* __restrict__ W, float* __restrict__ S,
                                                  SelState* __restrict__ st, const int* __restrict__ status,
                                                  const uint16_t* __restrict__ Xq, int Dq, int qtype,
                                                  const int* __restrict__ qflag) {
    __shared__ float xs[256][65];
    __shared__ float ws[64];
    if (*status & kStatusStop) return;  // perm may hold unwritten slots
    const int q = q16_usable(Xq, qflag) ? qtype : 0;
    const int4 t = tiles[blockIdx.x];
    const int seg = t.x, begin = t.y, end = t.z;
    if (st != nullptr && t.w && threadIdx.x == 0) {
        const int m = seg_off[seg + 1] - seg_off[seg];
        st[seg].prefix = 0;
        st[seg].krem = (uint32_t)(m / 2);
        st[seg].done = 0;  // set once the selection is done
    }
    const float* w = W + (int64_t)seg * D;
    if (q == 1)
        project_tile<VEC2, 1>(X, D, Xq, Dq, perm, begin, end, w, S, xs, ws);
    else if (q == 2)
        project_tile<VEC2, 2>(X, D, Xq, Dq, perm, begin, end, w, S, xs, ws);
    else
        project_tile<VEC2, 0>(X, D, Xq, Dq, perm, begin, end, w, S, xs, ws);
}

// Rows staged by cp.async, a 128-byte slab at a time (128 dims of the byte
// copy, 64 of the 16-bit copy, or 32 of X), 256 rows per stage.  Staged rows
// are 144 bytes apart, so the 16-byte reads of 8 consecutive threads cover all
// 32 banks once.  Reading X needs 16-byte aligned rows (D a multiple of 4).
constexpr int kPrRows = 256;
constexpr int kPrStride = 144;

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

// Persistent, pipelined projection: CTA b walks the sweep tiles b, b + grid,
// ...; each tile is a run of stages (256 rows by one 128-byte slab of each;
// thread t sums the dims of row t in ascending order, one fmaf per dim, across
// the slabs of its chunk) that flow through a ring of kPpBufs shared-memory
// buffers, so that the copies of the next kPpBufs - 1 stages are in flight
// while one is summed.  The row ids of a stage are loaded into registers one
// iteration before its copies are issued, and the w slab travels with the
// stage's copies.
constexpr int kPpBufs = 3;
constexpr int kPpSmem = kPpBufs * (kPrRows * kPrStride + 128 * 4);

// Walks a CTA's stages: tile t (blockIdx.x + i gridDim.x), chunk c of 256
// rows, slab sl.  Uniform across the CTA.
struct PpIter {
    int t, c, sl, nslab, ntiles;
    int4 tl, tl_next;  // tiles[t], tiles[t + gridDim.x] (loaded ahead)
    __device__ __forceinline__ void init(const int4* __restrict__ tiles, int ntiles_, int nslab_) {
        ntiles = ntiles_;
        nslab = nslab_;
        t = blockIdx.x;
        c = sl = 0;
        tl = t < ntiles ? tiles[t] : make_int4(-1, 0, 0, 0);
        tl_next = t + (int)gridDim.x < ntiles ? tiles[t + gridDim.x] : make_int4(-1, 0, 0, 0);
    }
    __device__ __forceinline__ bool valid() const { return t < ntiles; }
    __device__ __forceinline__ int base() const { return tl.y + c * kPrRows; }
    __device__ __forceinline__ int cnt() const { return min(kPrRows, tl.z - base()); }
    __device__ __forceinline__ void next(const int4* __restrict__ tiles) {
        if (++sl < nslab) return;
        sl = 0;
        if (tl.y + (++c) * kPrRows < tl.z) return;
        c = 0;
        t += gridDim.x;
        tl = tl_next;
        const int t2 = t + (int)gridDim.x;
        tl_next = t2 < ntiles ? tiles[t2] : make_int4(-1, 0, 0, 0);
    }
};

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

template <int Q>  // 0 = FP32 rows of X, 1 / 2 = BF16 / FP16 copy, 3 = byte copy
__device__ __forceinline__ void project_pipe(const float* __restrict__ X, int D, const uint16_t* __restrict__ Xq,
                                             int Dq, const uint8_t* __restrict__ Xb, int Db,
                                             const int32_t* __restrict__ perm, const int4* __restrict__ tiles,
                                             int ntiles, const int32_t* __restrict__ seg_off,
                                             const float* __restrict__ W, float* __restrict__ S,
                                             SelState* __restrict__ st, uint8_t* smem) {
    constexpr int SLAB = Q == 3 ? 128 : Q != 0 ? 64 : 32;  // dims per 128-byte slab
    const int tid = threadIdx.x, piece = tid & 7;
    const int nslab = (D + SLAB - 1) / SLAB;
    // thread tid copies piece (tid & 7) of rows (tid >> 3) + 32 k, k < 8
    int ids[8];
    auto load_ids = [&](const PpIter& it) {
        const int base = it.base(), cnt = it.cnt();
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int r = (tid >> 3) + 32 * k;
            ids[k] = r < cnt ? __ldg(perm + base + r) : 0;
        }
    };
    auto issue = [&](const PpIter& it, int buf) {
        if (it.valid()) {
            const int cnt = it.cnt(), d0 = it.sl * SLAB, seg = it.tl.x;
            uint8_t* b = smem + buf * (kPrRows * kPrStride);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int r = (tid >> 3) + 32 * k;
                if (r >= cnt) break;
                if (Q == 3) {
                    if (d0 + piece * 16 < Db)
                        cp_async16(b + r * kPrStride + piece * 16, Xb + (int64_t)ids[k] * Db + d0 + piece * 16);
                } else if (Q != 0) {
                    cp_async16(b + r * kPrStride + piece * 16, Xq + (int64_t)ids[k] * Dq + d0 + piece * 8);
                } else if (d0 + piece * 4 < D) {
                    cp_async16(b + r * kPrStride + piece * 16, X + (int64_t)ids[k] * D + d0 + piece * 4);
                }
            }
            float* ws = reinterpret_cast<float*>(smem + kPpBufs * (kPrRows * kPrStride)) + buf * 128;
            if (tid < SLAB) {
                if (d0 + tid < D)
                    cp_async4(ws + tid, W + (int64_t)seg * D + d0 + tid);
                else
                    ws[tid] = 0.f;
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    PpIter ic, ii;  // the stage to compute; the next stage to issue
    ic.init(tiles, ntiles, nslab);
    ii = ic;
    // prologue: stages 0 .. kPpBufs - 2
#pragma unroll
    for (int k = 0; k < kPpBufs - 1; ++k) {
        if (ii.valid()) load_ids(ii);
        issue(ii, k);
        if (ii.valid()) ii.next(tiles);
    }
    if (ii.valid()) load_ids(ii);
    float acc = 0.f;
    for (int s = 0; ic.valid(); ++s) {
        issue(ii, (s + kPpBufs - 1) % kPpBufs);  // ids loaded one iteration ago
        if (ii.valid()) {
            ii.next(tiles);
            if (ii.valid()) load_ids(ii);  // consumed by the next iteration's issue
        }
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kPpBufs - 1) : "memory");
        __syncthreads();
        const int buf = s % kPpBufs, cnt = ic.cnt(), d0 = ic.sl * SLAB;
        if (st != nullptr && ic.tl.w && ic.c == 0 && ic.sl == 0 && tid == 0) {  // a segment's first tile
            const int seg = ic.tl.x, m = seg_off[seg + 1] - seg_off[seg];
            st[seg].prefix = 0;
            st[seg].krem = (uint32_t)(m / 2);
            st[seg].done = 0;  // set once the selection is done
        }
        if (tid < cnt) {
            const uint8_t* rowp = smem + buf * (kPrRows * kPrStride) + tid * kPrStride;
            const float* ws = reinterpret_cast<const float*>(smem + kPpBufs * (kPrRows * kPrStride)) + buf * 128;
            const int dl = min(SLAB, D - d0);
            if (dl == SLAB) {  // a full slab: no per-dim guards, w four dims per load
                const float4* w4 = reinterpret_cast<const float4*>(ws);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint4 h = *reinterpret_cast<const uint4*>(rowp + q * 16);
                    const uint32_t hv[4] = {h.x, h.y, h.z, h.w};
                    if (Q == 3) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const float4 wv = w4[q * 4 + u];
                            acc = __fmaf_rn(u8_to_float(hv[u], 0), wv.x, acc);
                            acc = __fmaf_rn(u8_to_float(hv[u], 1), wv.y, acc);
                            acc = __fmaf_rn(u8_to_float(hv[u], 2), wv.z, acc);
                            acc = __fmaf_rn(u8_to_float(hv[u], 3), wv.w, acc);
                        }
                    } else if (Q != 0) {
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const float4 wv = w4[q * 2 + u];
                            acc = __fmaf_rn(q16_to_float<Q>(hv[2 * u] & 0xFFFFu), wv.x, acc);
                            acc = __fmaf_rn(q16_to_float<Q>(hv[2 * u] >> 16), wv.y, acc);
                            acc = __fmaf_rn(q16_to_float<Q>(hv[2 * u + 1] & 0xFFFFu), wv.z, acc);
                            acc = __fmaf_rn(q16_to_float<Q>(hv[2 * u + 1] >> 16), wv.w, acc);
                        }
                    } else {
                        const float4 wv = w4[q];
                        acc = __fmaf_rn(__uint_as_float(hv[0]), wv.x, acc);
                        acc = __fmaf_rn(__uint_as_float(hv[1]), wv.y, acc);
                        acc = __fmaf_rn(__uint_as_float(hv[2]), wv.z, acc);
                        acc = __fmaf_rn(__uint_as_float(hv[3]), wv.w, acc);
                    }
                }
            } else if (Q == 3) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (q * 16 >= dl) break;
                    const uint4 h = *reinterpret_cast<const uint4*>(rowp + q * 16);
                    const uint32_t hv[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
                    for (int t = 0; t < 16; ++t)
                        if (q * 16 + t < dl) acc = __fmaf_rn(u8_to_float(hv[t >> 2], t & 3), ws[q * 16 + t], acc);
                }
            } else if (Q != 0) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (q * 8 >= dl) break;
                    const uint4 h = *reinterpret_cast<const uint4*>(rowp + q * 16);
                    const uint32_t hv[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        if (q * 8 + t < dl) {
                            const uint32_t bits = t & 1 ? hv[t >> 1] >> 16 : hv[t >> 1] & 0xFFFFu;
                            acc = __fmaf_rn(q16_to_float<Q>(bits), ws[q * 8 + t], acc);
                        }
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (q * 4 >= dl) break;
                    const float4 v = *reinterpret_cast<const float4*>(rowp + q * 16);
                    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (q * 4 + t < dl) acc = __fmaf_rn(vv[t], ws[q * 4 + t], acc);
                }
            }
            if (ic.sl == nslab - 1) {
                S[ic.base() + tid] = __fadd_rn(acc, 0.f);  // -0 -> +0
                acc = 0.f;
            }
        }
        __syncthreads();  // buffer s % kPpBufs is refilled by the next issue
        ic.next(tiles);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__global__ void __launch_bounds__(kPrRows, 2) k1_project_pipe(const float* __restrict__ X, int D,
                                                              const int32_t* __restrict__ perm,
                                                              const int4* __restrict__ tiles, int ntiles,
                                                              const int32_t* __restrict__ seg_off,
                                                              const float* __restrict__ W, float* __restrict__ S,
                                                              SelState* __restrict__ st,
                                                              const int* __restrict__ status,
                                                              const uint16_t* __restrict__ Xq, int Dq, int qtype,
                                                              const int* __restrict__ qflag,
                                                              const uint8_t* __restrict__ Xb, int Db,
                                                              const int* __restrict__ bflag) {
    extern __shared__ __align__(16) uint8_t pp_smem[];
    if (*status & kStatusStop) return;  // perm may hold unwritten slots
    const int q = u8_usable(Xb, bflag) ? 3 : q16_usable(Xq, qflag) ? qtype : 0;
    if (q == 3)
        project_pipe<3>(X, D, Xq, Dq, Xb, Db, perm, tiles, ntiles, seg_off, W, S, st, pp_smem);
    else if (q == 1)
        project_pipe<1>(X, D, Xq, Dq, Xb, Db, perm, tiles, ntiles, seg_off, W, S, st, pp_smem);
    else if (q == 2)
        project_pipe<2>(X, D, Xq, Dq, Xb, Db, perm, tiles, ntiles, seg_off, W, S, st, pp_smem);
    else
        project_pipe<0>(X, D, Xq, Dq, Xb, Db, perm, tiles, ntiles, seg_off, W, S, st, pp_smem);
}

int sm_count() {
    static const int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return n;
}

// Small segments: one CTA per segment keeps all keys in shared memory,
// selects the floor(m/2)-th key, and either records it (thr) or, on the
// final cut, partitions the segment stably into perm_out.
__global__ void __launch_bounds__(1024) k1_select_small(const float* __restrict__ S,
                                                        const int32_t* __restrict__ seg_off,
                                                        const int32_t* __restrict__ seg_tile0, int pos_bits,
                                                        uint64_t* __restrict__ thr,
                                                        const int32_t* __restrict__ perm_in,
                                                        int32_t* __restrict__ perm_out, int* __restrict__ status) {
    extern __shared__ uint64_t keys[];
    __shared__ uint32_t hist[1 << kRadixBits];
    __shared__ int sh_digit;
    __shared__ uint32_t sh_below;
    __shared__ int warp_tot[32];
    if (seg_tile0[blockIdx.x + 1] == seg_tile0[blockIdx.x]) return;  // a finished tree's leaf
    const int seg = blockIdx.x, a = seg_off[seg], m = seg_off[seg + 1] - a;
    for (int p = threadIdx.x; p < m; p += blockDim.x) keys[p] = sel_key(S[a + p], p, pos_bits);
    uint64_t prefix = 0;
    uint32_t krem = (uint32_t)(m / 2);
    for (int hi = 32 + pos_bits, lo; hi > 0 && !(hi == pos_bits && krem == 0); hi = lo) {
        lo = digit_lo(hi, pos_bits);
        const int width = hi - lo;
        const uint32_t mask = (1u << width) - 1u;
        for (int b = threadIdx.x; b < (1 << width); b += blockDim.x) hist[b] = 0;
        __syncthreads();
        for (int p = threadIdx.x; p < m; p += blockDim.x) {
            const uint64_t kk = keys[p];
            if ((kk >> hi) == (prefix >> hi)) atomicAdd(&hist[(uint32_t)(kk >> lo) & mask], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 32) find_digit(hist, 1 << width, krem, &sh_digit, &sh_below);
        __syncthreads();
        prefix |= (uint64_t)sh_digit << lo;
        krem -= sh_below;
        __syncthreads();
    }
    if (perm_out == nullptr) {
        if (threadIdx.x == 0) thr[seg] = prefix;
        return;
    }
    const int K = m / 2;
    int left_before = 0;
    for (int base = 0; base < m; base += blockDim.x) {
        const int p = base + threadIdx.x;
        const int isl = (p < m) && keys[p] < prefix;
        int tot;
        const int ex = block_excl_scan(isl, warp_tot, &tot);
        if (p < m) {
            const int lb = left_before + ex;
            const int np = isl ? lb : K + (p - lb);
            if ((isl ? np < K : np < m) && np >= 0)
                perm_out[a + np] = perm_in[a + p];
            else
                atomicOr(status, kStatusInternal);
        }
        left_before += tot;
    }
}

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x / 2); }

// Ascending bitonic sort of 32 R NW keys held by NW warps (R per lane;
// element e = 32 R warp + R lane + r): exchanges within a lane for distances
// below R, across lanes by shuffles up to 32 R, across warps through shared
// memory (xch: 32 R NW keys) above.
template <int R, int NW>
__device__ __forceinline__ void bitonic_sort_keys(uint64_t (&v)[R], uint64_t* xch) {
    const int lane = threadIdx.x & 31, warp = NW > 1 ? (int)(threadIdx.x >> 5) : 0;
    constexpr int LOG = ilog2c(32 * R * NW);
    static_assert((32 * R * NW) == (1 << LOG), "R and NW are powers of two");
    const int e0 = 32 * R * warp + R * lane;  // element of v[0]
#pragma unroll
    for (int lk = 1; lk <= LOG; ++lk) {
#pragma unroll
        for (int lj = LOG - 1; lj >= 0; --lj) {  // constant trip count: unrolls fully
            const int k = 1 << lk, j = 1 << lj;
            if (lj < lk && j >= 32 * R) {
                const int wj = j / (32 * R);
                // the direction bit and the pair are warp bits
                const bool keep_min = ((warp & wj) == 0) == ((e0 & k) == 0);
#pragma unroll
                for (int r = 0; r < R; ++r) xch[r * 32 * NW + threadIdx.x] = v[r];
                __syncthreads();
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint64_t o = xch[r * 32 * NW + (threadIdx.x ^ (32 * wj))];
                    v[r] = keep_min ? (o < v[r] ? o : v[r]) : (o > v[r] ? o : v[r]);
                }
                __syncthreads();
            } else if (lj < lk && j >= R) {
                const int lj2 = j / R;
                // k > j >= R: the direction bit of the pair is a lane or warp bit
                const bool keep_min = ((lane & lj2) == 0) == ((e0 & k) == 0);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint64_t o = shfl_xor64(v[r], lj2);
                    v[r] = keep_min ? (o < v[r] ? o : v[r]) : (o > v[r] ? o : v[r]);
                }
            } else if (lj < lk) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if ((r & j) == 0) {
                        const bool up = ((e0 + r) & k) == 0;
                        const uint64_t x = v[r], y = v[r | j];
                        const bool sw = (x > y) == up;
                        v[r] = sw ? y : x;
                        v[r | j] = sw ? x : y;
                    }
                }
            }
        }
    }
}

// Segments of up to 32 R NW points: NW warps hold a segment's keys in
// registers, sort them and take the floor(m/2)-th smallest.  NW = 1: four
// segments per CTA, one per warp; NW > 1: one segment per CTA.  On the final
// cut each thread takes R consecutive positions, and an exclusive scan of
// the left counts gives every position its place in perm_out (left positions
// first, each side in position order), as k1_select_small does.
template <int R, int NW>
__global__ void __launch_bounds__(NW > 1 ? 32 * NW : 128) k1_select_sort(const float* __restrict__ S,
                                                                        const int32_t* __restrict__ seg_off,
                                                                        const int32_t* __restrict__ seg_tile0,
                                                                        int nseg, int pos_bits,
                                                                        uint64_t* __restrict__ thr,
                                                                        const int32_t* __restrict__ perm_in,
                                                                        int32_t* __restrict__ perm_out,
                                                                        int* __restrict__ status) {
    constexpr int NK = 32 * R * NW;  // keys per segment
    __shared__ uint64_t xch[NW > 1 ? NK : 1];
    __shared__ uint64_t sh_T;
    __shared__ int warp_tot[32];
    const int lane = threadIdx.x & 31;
    const int tid = NW > 1 ? (int)threadIdx.x : lane;  // thread within the segment's group
    const int seg = NW > 1 ? (int)blockIdx.x : (int)(blockIdx.x * 4 + (threadIdx.x >> 5));
    // segment-uniform exits (NW > 1: the whole CTA)
    if (seg >= nseg || seg_tile0[seg + 1] == seg_tile0[seg]) return;  // past the end; a finished tree's leaf
    const int a = seg_off[seg], m = seg_off[seg + 1] - a;
    if (m > NK) {  // the plan sized the kernel from the level's largest segment
        if (tid == 0) atomicOr(status, kStatusInternal);
        return;
    }
    uint64_t v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int p = r * 32 * NW + tid;
        v[r] = p < m ? sel_key(S[a + p], p, pos_bits) : ~0ull;  // padding sorts last
    }
    bitonic_sort_keys<R, NW>(v, xch);
    // element K: register K % R of thread K / R (a masked OR keeps v[] in
    // registers, where a select by a run-time index would not)
    const int K = m / 2;
    uint64_t mine = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) mine |= v[r] & (0ull - (uint64_t)(r == K % R));
    uint64_t T;
    if (NW > 1) {
        if (tid == K / R) sh_T = mine;
        __syncthreads();
        T = sh_T;
    } else {
        T = shfl64(mine, K / R);
    }
    if (perm_out == nullptr) {
        if (tid == 0) thr[seg] = T;
        return;
    }
    const int p0 = tid * R;
    bool isl[R];
    int32_t id[R];
    int cnt = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int p = p0 + r;
        isl[r] = p < m && sel_key(S[a + p], p, pos_bits) < T;
        id[r] = p < m ? perm_in[a + p] : 0;
        cnt += isl[r];
    }
    int lb;  // left positions before p0
    if (NW > 1) {
        int tot;
        lb = block_excl_scan(cnt, warp_tot, &tot);
    } else {
        int x = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        lb = x - cnt;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int p = p0 + r;
        if (p < m) {
            const int np = isl[r] ? lb : K + (p - lb);
            if ((isl[r] ? np < K : np < m) && np >= 0)
                perm_out[a + np] = id[r];
            else
                atomicOr(status, kStatusInternal);
            lb += isl[r];
        }
    }
}

template <int R, int NW>
void launch_select_sort(const LevelPlan& lp, const SplitBuffers& b, const int32_t* perm_in, int32_t* perm_out,
                        cudaStream_t s) {
    const int grid = NW > 1 ? lp.nseg : (lp.nseg + 3) / 4;
    k1_select_sort<R, NW><<<grid, NW > 1 ? 32 * NW : 128, 0, s>>>(b.S, lp.seg_off, lp.seg_tile0, lp.nseg,
                                                                  lp.pos_bits, b.thr, perm_in, perm_out, b.status);
}

// Large segments: one radix pass over bits [hi-11, hi) of the keys.  Every
// tile adds its histogram to the segment's global one; the last tile of the
// segment to finish (ticket) picks the digit and clears the histogram.
__global__ void __launch_bounds__(256) k1_select_pass(const float* __restrict__ S,
                                                      const int4* __restrict__ tiles,
                                                      const int32_t* __restrict__ seg_off,
                                                      const int32_t* __restrict__ seg_tile0, int pos_bits,
                                                      int hi, SelState* __restrict__ st,
                                                      uint32_t* __restrict__ ghist,
                                                      uint32_t* __restrict__ ticket,
                                                      uint64_t* __restrict__ thr) {
    __shared__ uint32_t hist[1 << kRadixBits];
    __shared__ int sh_last, sh_digit;
    __shared__ uint32_t sh_below;
    __shared__ int warp_tot[32];
    const int4 t = tiles[blockIdx.x];
    const int seg = t.x, begin = t.y, end = t.z;
    if (st[seg].done) return;  // selected already (value digits, no tie to the left)
    const int a = seg_off[seg];
    const int lo = digit_lo(hi, pos_bits), width = hi - lo, nb = 1 << width;
    const uint32_t mask = (uint32_t)nb - 1u;
    const uint64_t prefix = st[seg].prefix;
    // the tile's projections first (all loads in flight at once), then the
    // histogram
    constexpr int PER = kTile / 256;
    float sv[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int p = begin + (int)threadIdx.x + 256 * i;
        sv[i] = p < end ? S[p] : 0.f;
    }
    for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int p = begin + (int)threadIdx.x + 256 * i;
        const uint64_t kk = sel_key(sv[i], p - a, pos_bits);
        if (p < end && (kk >> hi) == (prefix >> hi)) atomicAdd(&hist[(uint32_t)(kk >> lo) & mask], 1u);
    }
    __syncthreads();
    uint32_t* gh = ghist + (size_t)seg * (1 << kRadixBits);
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (hist[b]) atomicAdd(&gh[b], hist[b]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t ntile = (uint32_t)(seg_tile0[seg + 1] - seg_tile0[seg]);
        sh_last = atomicAdd(&ticket[seg], 1u) == ntile - 1u;
    }
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = atomicExch(&gh[b], 0u);
    __syncthreads();
    block_find_digit(hist, nb, st[seg].krem, warp_tot, &sh_digit, &sh_below);
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t np = prefix | ((uint64_t)sh_digit << lo);
        const uint32_t kr = st[seg].krem - sh_below;
        st[seg].prefix = np;
        st[seg].krem = kr;
        ticket[seg] = 0;
        if (lo == 0 || (lo == pos_bits && kr == 0)) {
            thr[seg] = np;
            st[seg].done = 1;
        }
    }
}

// Large segments, after the value digits: when the selected value v has ties
// (krem > 0: the key is the krem-th of the keys with value v, in position
// order), one pass finds its position.  Every tile counts its keys with value
// v; the last tile of the segment to finish (ticket) finds the tile that holds
// the krem-th of them from the counts, in tile order, and the position inside
// that tile by ordered ballots.  A segment whose key is known returns at once.
__global__ void __launch_bounds__(256) k1_select_pos(const float* __restrict__ S, const int4* __restrict__ tiles,
                                                     const int32_t* __restrict__ seg_off,
                                                     const int32_t* __restrict__ seg_tile0, int pos_bits,
                                                     SelState* __restrict__ st, int32_t* __restrict__ tcount,
                                                     uint32_t* __restrict__ ticket, uint64_t* __restrict__ thr) {
    __shared__ int warp_tot[32];
    __shared__ int sh_last, sh_tile, sh_before;
    const int4 t = tiles[blockIdx.x];
    const int seg = t.x, begin = t.y, end = t.z;
    if (st[seg].done) return;
    const int a = seg_off[seg];
    const uint32_t v = (uint32_t)(st[seg].prefix >> pos_bits);
    constexpr int PER = kTile / 256;
    int c = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int p = begin + (int)threadIdx.x + 256 * i;
        c += (p < end && ord32(S[p]) == v) ? 1 : 0;
    }
    c = block_sum(c, warp_tot);
    if (threadIdx.x == 0) tcount[blockIdx.x] = c;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t ntile = (uint32_t)(seg_tile0[seg + 1] - seg_tile0[seg]);
        sh_last = atomicAdd(&ticket[seg], 1u) == ntile - 1u;
    }
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    const int krem = (int)st[seg].krem;
    const int t0 = seg_tile0[seg], t1 = seg_tile0[seg + 1];
    // the tile holding the krem-th tied key: warp 0 scans the counts in order
    if (threadIdx.x == 0) sh_tile = -1;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int run = 0;
        for (int q0 = t0; q0 < t1; q0 += 32) {
            const int q = q0 + lane;
            const int cq = q < t1 ? tcount[q] : 0;
            int incl = cq;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int excl = run + incl - cq;
            const unsigned hitb = __ballot_sync(0xffffffffu, q < t1 && excl <= krem && krem < excl + cq);
            if (hitb) {
                const int src = __ffs(hitb) - 1;
                if (lane == src) {
                    sh_tile = q;
                    sh_before = excl;
                }
                break;
            }
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    __syncthreads();
    if (sh_tile < 0) {  // cannot happen (value v has more than krem keys); the cut then reports it
        if (threadIdx.x == 0) ticket[seg] = 0;
        return;
    }
    const int4 tt = tiles[sh_tile];
    int want = krem - sh_before;  // among the tile's tied keys, in position order
    for (int base = tt.y; base < tt.z; base += 256) {
        const int p = base + (int)threadIdx.x;
        const int tied = (p < tt.z && ord32(S[p]) == v) ? 1 : 0;
        int tot;
        const int ex = block_excl_scan(tied, warp_tot, &tot);
        if (tied && ex == want) {
            thr[seg] = ((uint64_t)v << pos_bits) | (uint32_t)(p - a);
            st[seg].done = 1;
        }
        want -= tot;
        if (want < 0) break;  // uniform: tot is the block's
    }
    if (threadIdx.x == 0) ticket[seg] = 0;
}

// FP64 sums of the left and right points of each tile, 128 dims per CTA
// (blockIdx.y).  Warp w owns a contiguous run of the tile's positions; order:
// per warp ascending positions, then warps 0..15, then tiles.
constexpr int kSumsWarps = 16;

// Adds the n rows listed in rows[] (one side of the cut) to the per-lane
// compensated sums (h, l), with the loads of up to U rows in flight.  Q = 0
// reads the FP32 rows of X (VEC: lane l owns dims 4l .. 4l+3, else l, l+32,
// ...), Q = 1 / 2 the BF16 / FP16 copy (dims 4l .. 4l+3).
template <bool VEC, int Q>
__device__ __forceinline__ void sums_side(const float* __restrict__ X, int D, const uint16_t* __restrict__ Xq, int Dq,
                                          const int* rows, int n, int dbase, float* h, float* l) {
    const int lane = threadIdx.x & 31;
    constexpr int U = Q != 0 ? 16 : 8;  // 4 KB per warp in flight
    for (int q0 = 0; q0 < n; q0 += U) {
        float v[U][4];
        uint2 hq[U];  // Q != 0: four raw 16-bit values
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int j = 0; j < 4; ++j) v[u][j] = 0.f;
            hq[u] = make_uint2(0u, 0u);
            if (q0 + u < n) {
                const int row = rows[q0 + u];
                const float* x = X + (int64_t)row * D + dbase;
                if (Q != 0) {  // rows padded to Dq: the four values are in bounds
                    if (dbase + lane * 4 < D)
                        hq[u] = __ldg(reinterpret_cast<const uint2*>(Xq + (int64_t)row * Dq + dbase + 4 * lane));
                } else if (VEC) {
                    if (dbase + lane * 4 < D) {
                        const float4 f = __ldg(reinterpret_cast<const float4*>(x) + lane);
                        v[u][0] = f.x; v[u][1] = f.y; v[u][2] = f.z; v[u][3] = f.w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) v[u][j] = (dbase + lane + 32 * j < D) ? __ldg(x + lane + 32 * j) : 0.f;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (q0 + u >= n) break;
            if (Q != 0) {
                v[u][0] = q16_to_float<Q>(hq[u].x & 0xFFFFu);
                v[u][1] = q16_to_float<Q>(hq[u].x >> 16);
                v[u][2] = q16_to_float<Q>(hq[u].y & 0xFFFFu);
                v[u][3] = q16_to_float<Q>(hq[u].y >> 16);
            }
            if (Q != 0) {
                // exact-mode values are integers of magnitude <= 2048 and a
                // lane adds at most 128 of them per tile: FP32 sums are exact
#pragma unroll
                for (int j = 0; j < 4; ++j) h[j] = __fadd_rn(h[j], v[u][j]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {  // TwoSum: s + err == h + v exactly
                    const float s = __fadd_rn(h[j], v[u][j]);
                    const float bp = __fsub_rn(s, h[j]);
                    const float err = __fadd_rn(__fsub_rn(h[j], __fsub_rn(s, bp)), __fsub_rn(v[u][j], bp));
                    h[j] = s;
                    l[j] = __fadd_rn(l[j], err);
                }
            }
        }
    }
}

// Accumulates the warp's run [w0, w1) of one tile into the sums of two
// lists: full (Sp == nullptr): list 0 = the left positions, list 1 = the
// right ones; delta: list 0 = the positions that moved to the left since the
// previous iteration's cut (projections Sp, key Tp), list 1 = those that moved
// to the right; the rest are not read.  Each chunk of 32 positions is
// compacted by list (rows[]: list 0, then list 1, both in position order), so
// that each list's sums take its rows in ascending positions without per-row
// selects.
template <bool VEC, int Q>
__device__ __forceinline__ void sums_run(const float* __restrict__ X, int D, const uint16_t* __restrict__ Xq, int Dq,
                                         const int32_t* __restrict__ perm, const float* __restrict__ S,
                                         const float* __restrict__ Sp, int a, uint64_t T, uint64_t Tp, int pos_bits,
                                         int w0, int w1, int dbase, int* rows, float* hL, float* lL, float* hR,
                                         float* lR) {
    const int lane = threadIdx.x & 31;
    // ids and projections of the next 32 positions load while this chunk's
    // rows are summed
    int next_row = 0;
    float next_s = 0.f, next_sp = 0.f;
    if (w0 + lane < w1) {
        next_row = perm[w0 + lane];
        next_s = S[w0 + lane];
        if (Sp) next_sp = Sp[w0 + lane];
    }
    for (int c = w0; c < w1; c += 32) {
        const int p = c + lane;
        const int my_row = next_row;
        const bool in = p < w1;
        const bool now_left = in && sel_key(next_s, p - a, pos_bits) < T;
        bool c0 = now_left, c1 = in && !now_left;
        if (Sp) {
            const bool was_left = in && sel_key(next_sp, p - a, pos_bits) < Tp;
            c0 = now_left && !was_left;
            c1 = in && !now_left && was_left;
        }
        if (p + 32 < w1) {
            next_row = perm[p + 32];
            next_s = S[p + 32];
            if (Sp) next_sp = Sp[p + 32];
        }
        const unsigned b0 = __ballot_sync(0xffffffffu, c0), b1 = __ballot_sync(0xffffffffu, c1);
        const unsigned lt = (1u << lane) - 1u;
        const int n0 = __popc(b0);
        __syncwarp();  // the previous chunk's reads of rows[] are done
        if (c0)
            rows[__popc(b0 & lt)] = my_row;
        else if (c1)
            rows[n0 + __popc(b1 & lt)] = my_row;
        __syncwarp();
        sums_side<VEC, Q>(X, D, Xq, Dq, rows, n0, dbase, hL, lL);
        sums_side<VEC, Q>(X, D, Xq, Dq, rows + n0, __popc(b1), dbase, hR, lR);
    }
}

template <bool VEC>
__global__ void __launch_bounds__(32 * kSumsWarps) k1_sums(const float* __restrict__ X, int D,
                                                          const int32_t* __restrict__ perm,
                                                          const int4* __restrict__ tiles,
                                                          const float* __restrict__ S,
                                                          const int32_t* __restrict__ seg_off,
                                                          const uint64_t* __restrict__ thr, int pos_bits,
                                                          double* __restrict__ partial,
                                                          const int* __restrict__ status,
                                                          const uint16_t* __restrict__ Xq, int Dq, int qtype,
                                                          const int* __restrict__ qflag,
                                                          const uint8_t* __restrict__ Xb,
                                                          const int* __restrict__ bflag,
                                                          const float* __restrict__ Sp,
                                                          const uint64_t* __restrict__ thrp) {
    __shared__ double red[kSumsWarps][2][128];
    __shared__ int rows[kSumsWarps][32];
    if (*status & kStatusStop) return;  // perm may hold unwritten slots
    const int q = q16_usable(Xq, qflag) ? qtype : 0;  // then lane l owns dims 4l .. 4l+3
    const bool exact = exact_ints(Xq, qflag, Xb, bflag);
    const int4 t = tiles[blockIdx.x];
    const int seg = t.x, begin = t.y, end = t.z;
    const int dbase = blockIdx.y * 128;
    const int a = seg_off[seg];
    const uint64_t T = thr[seg], Tp = Sp ? thrp[seg] : 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per = (end - begin + kSumsWarps - 1) / kSumsWarps;
    const int w0 = begin + warp * per, w1 = min(end, w0 + per);
    // Per-lane compensated FP32 sums (Knuth's TwoSum: hi + lo carries the
    // exact sum of every addition's rounding error), combined in FP64 below.
    // GB300 issues FP64 at a small fraction of its FP32 rate, so one FP64
    // add per element would bound this sweep far below HBM speed.  For
    // integer-valued data every add is exact and lo stays 0.
    float hL[4] = {0.f, 0.f, 0.f, 0.f}, lL[4] = {0.f, 0.f, 0.f, 0.f};
    float hR[4] = {0.f, 0.f, 0.f, 0.f}, lR[4] = {0.f, 0.f, 0.f, 0.f};
    if (q == 1)
        sums_run<VEC, 1>(X, D, Xq, Dq, perm, S, Sp, a, T, Tp, pos_bits, w0, w1, dbase, rows[warp], hL, lL, hR,
                         lR);
    else if (q == 2)
        sums_run<VEC, 2>(X, D, Xq, Dq, perm, S, Sp, a, T, Tp, pos_bits, w0, w1, dbase, rows[warp], hL, lL, hR,
                         lR);
    else
        sums_run<VEC, 0>(X, D, Xq, Dq, perm, S, Sp, a, T, Tp, pos_bits, w0, w1, dbase, rows[warp], hL, lL, hR,
                         lR);
    if (exact) {  // integer sums below 2^24 per lane and 2^31 per tile: int32 partials
        int(*ired)[2][128] = reinterpret_cast<int(*)[2][128]>(red);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int dl = (VEC || q != 0) ? lane * 4 + j : lane + 32 * j;
            ired[warp][0][dl] = __float2int_rn(hL[j]);
            ired[warp][1][dl] = __float2int_rn(hR[j]);
        }
        __syncthreads();
        if (threadIdx.x < 128 && dbase + threadIdx.x < D) {
            int sL = 0, sR = 0;
#pragma unroll
            for (int w = 0; w < kSumsWarps; ++w) {
                sL += ired[w][0][threadIdx.x];
                sR += ired[w][1][threadIdx.x];
            }
            int32_t* ip = reinterpret_cast<int32_t*>(partial);
            ip[((int64_t)blockIdx.x * 2 + 0) * D + dbase + threadIdx.x] = sL;
            ip[((int64_t)blockIdx.x * 2 + 1) * D + dbase + threadIdx.x] = sR;
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int dl = (VEC || q != 0) ? lane * 4 + j : lane + 32 * j;
        red[warp][0][dl] = (double)hL[j] + (double)lL[j];
        red[warp][1][dl] = (double)hR[j] + (double)lR[j];
    }
    __syncthreads();
    if (threadIdx.x < 128 && dbase + threadIdx.x < D) {
        double sL = 0.0, sR = 0.0;
#pragma unroll
        for (int w = 0; w < kSumsWarps; ++w) {
            sL += red[w][0][threadIdx.x];
            sR += red[w][1][threadIdx.x];
        }
        partial[((int64_t)blockIdx.x * 2 + 0) * D + dbase + threadIdx.x] = sL;
        partial[((int64_t)blockIdx.x * 2 + 1) * D + dbase + threadIdx.x] = sR;
    }
}

// Centroid sums with rows staged like the projection's: a CTA takes one
// select tile (up to kTile positions) and first lists its rows (list 0 in
// ascending positions, then list 1; the lists of sums_run: left and right, or
// moved left and moved right).  The list is staged in chunks of 256 rows, a
// 128-byte slab of each row at a time, by cp.async (double-buffered), and
// each thread sums 4 dims of the slab over a 1/G share of the chunk's rows,
// the two lists apart.  Per thread the rows of a list come in ascending
// positions; the G partial sums of a dim are combined in group order (int32
// for integer data, else FP64).
constexpr int kSuThreads = 256;
constexpr int kSuSmem = 2 * kPrRows * kPrStride + kTile * 4 + 16 * 4 + 2 * 1024 * 8;
static_assert(kTile == 8 * kPrRows && kSuThreads == 256, "one warp lists each 256 positions of a tile");
// Adds 4 dims (quad q) of one staged row to the sums (h, l).
template <int Q>
__device__ __forceinline__ void sums_add(const uint8_t* row, int q, float (&h)[4], float (&l)[4]) {
    float v[4];
    if (Q == 3) {
        const uint32_t b = *reinterpret_cast<const uint32_t*>(row + q * 4);
        // values up to 255, at most kTile / 8 of them per thread, dim and
        // tile: FP32 sums are exact
#pragma unroll
        for (int j = 0; j < 4; ++j) h[j] = __fadd_rn(h[j], u8_to_float(b, j));
    } else if (Q != 0) {
        const uint2 b = *reinterpret_cast<const uint2*>(row + q * 8);
        v[0] = q16_to_float<Q>(b.x & 0xFFFFu);
        v[1] = q16_to_float<Q>(b.x >> 16);
        v[2] = q16_to_float<Q>(b.y & 0xFFFFu);
        v[3] = q16_to_float<Q>(b.y >> 16);
        // exact-mode values are integers of magnitude <= 2048 and a thread
        // adds at most 128 of them per dim and tile: FP32 sums are exact
#pragma unroll
        for (int j = 0; j < 4; ++j) h[j] = __fadd_rn(h[j], v[j]);
    } else {
        const float4 f = *reinterpret_cast<const float4*>(row + q * 16);
        v[0] = f.x;
        v[1] = f.y;
        v[2] = f.z;
        v[3] = f.w;
#pragma unroll
        for (int j = 0; j < 4; ++j) {  // TwoSum: s + err == h + v exactly
            const float s = __fadd_rn(h[j], v[j]);
            const float bp = __fsub_rn(s, h[j]);
            const float err = __fadd_rn(__fsub_rn(h[j], __fsub_rn(s, bp)), __fsub_rn(v[j], bp));
            h[j] = s;
            l[j] = __fadd_rn(l[j], err);
        }
    }
}

// Issues the copies of stage st of a sums tile: dims (st / nchunk) * SLAB ..
// of the rows of chunk st % nchunk, into buffer st & 1.
template <int Q>
__device__ __forceinline__ void sums_issue(const float* __restrict__ X, int D, const uint16_t* __restrict__ Xq,
                                           int Dq, const uint8_t* __restrict__ Xb, int Db, const int* ids, int m,
                                           int nchunk, int st, uint8_t* smem) {
    constexpr int SLAB = Q == 3 ? 128 : Q != 0 ? 64 : 32;
    const int sl = st / nchunk, c = st - sl * nchunk, d0 = sl * SLAB;
    const int cnt = min(kPrRows, m - c * kPrRows);
    uint8_t* buf = smem + (st & 1) * (kPrRows * kPrStride);
    for (int e = threadIdx.x; e < kPrRows * 8; e += kSuThreads) {
        const int r = e >> 3, piece = e & 7;
        if (r >= cnt) break;
        const int row = ids[c * kPrRows + r];
        if (Q == 3) {
            if (d0 + piece * 16 < Db)
                cp_async16(buf + r * kPrStride + piece * 16, Xb + (int64_t)row * Db + d0 + piece * 16);
        } else if (Q != 0) {
            cp_async16(buf + r * kPrStride + piece * 16, Xq + (int64_t)row * Dq + d0 + piece * 8);
        } else if (d0 + piece * 4 < D) {
            cp_async16(buf + r * kPrStride + piece * 16, X + (int64_t)row * D + d0 + piece * 4);
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int Q>
__device__ __forceinline__ void sums_async_tile(const float* __restrict__ X, int D, const uint16_t* __restrict__ Xq,
                                                int Dq, const uint8_t* __restrict__ Xb, int Db,
                                                const int32_t* __restrict__ perm,
                                                const float* __restrict__ S, const float* __restrict__ Sp, int a,
                                                uint64_t T, uint64_t Tp, int pos_bits, int begin, int end,
                                                double* __restrict__ part, int32_t* __restrict__ ipart,
                                                uint8_t* smem) {
    constexpr int SLAB = Q == 3 ? 128 : Q != 0 ? 64 : 32;  // dims per 128-byte slab
    constexpr int QUADS = SLAB / 4;                        // threads per row
    constexpr int G = kSuThreads / QUADS;                  // row groups
    int* ids = reinterpret_cast<int*>(smem + 2 * kPrRows * kPrStride);  // [kTile] row ids, list 0 first
    int* cnt0 = ids + kTile;                                             // [8] list-0 rows per 256 positions
    int* cnt1 = cnt0 + 8;                                                // [8] list-1 rows
    double* red = reinterpret_cast<double*>(cnt1 + 8);                   // [2][G][SLAB], G * SLAB = 1024
    static_assert(G * SLAB == 1024, "the combine buffer holds 2 x 1024 sums");
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = end - begin;
    // warp w lists positions 256 w .. 256 w + 255; their projections and ids
    // load first, all in flight at once
    float sv[8], spv[8];
    int pv[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int p = warp * kPrRows + 32 * i + lane;
        const bool in = p < m;
        sv[i] = in ? S[begin + p] : 0.f;
        spv[i] = in && Sp ? Sp[begin + p] : 0.f;
        pv[i] = in ? perm[begin + p] : 0;
    }
    unsigned bal0[8], bal1[8];
    int n0w = 0, n1w = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int p = warp * kPrRows + 32 * i + lane;
        const bool in = p < m;
        const bool now_left = in && sel_key(sv[i], begin + p - a, pos_bits) < T;
        bool c0 = now_left, c1 = in && !now_left;
        if (Sp) {
            const bool was_left = in && sel_key(spv[i], begin + p - a, pos_bits) < Tp;
            c0 = now_left && !was_left;
            c1 = in && !now_left && was_left;
        }
        bal0[i] = __ballot_sync(0xffffffffu, c0);
        bal1[i] = __ballot_sync(0xffffffffu, c1);
        n0w += __popc(bal0[i]);
        n1w += __popc(bal1[i]);
    }
    if (lane == 0) {
        cnt0[warp] = n0w;
        cnt1[warp] = n1w;
    }
    __syncthreads();
    int NL = 0, N1 = 0, lb0 = 0, lb1 = 0;  // list sizes; list rows of the positions before this warp's
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const int v0 = cnt0[w], v1 = cnt1[w];
        NL += v0;
        N1 += v1;
        lb0 += w < warp ? v0 : 0;
        lb1 += w < warp ? v1 : 0;
    }
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if ((bal0[i] >> lane) & 1u)
            ids[lb0 + __popc(bal0[i] & lt)] = pv[i];
        else if ((bal1[i] >> lane) & 1u)
            ids[NL + lb1 + __popc(bal1[i] & lt)] = pv[i];
        lb0 += __popc(bal0[i]);
        lb1 += __popc(bal1[i]);
    }
    __syncthreads();
    const int mt = NL + N1;  // rows staged
    const int nchunk = (mt + kPrRows - 1) / kPrRows;
    if (nchunk == 0) {  // no rows: zero sums
        for (int d = tid; d < 2 * D; d += kSuThreads) {
            if (Q != 0)
                ipart[d] = 0;
            else
                part[d] = 0.0;
        }
        return;
    }
    const int nslab = (D + SLAB - 1) / SLAB, nstage = nslab * nchunk;
    // stage st: dims (st / nchunk) * SLAB .., rows of chunk st % nchunk
    const int q = tid % QUADS, g = tid / QUADS;
    float hL[4] = {0.f, 0.f, 0.f, 0.f}, lL[4] = {0.f, 0.f, 0.f, 0.f};
    float hR[4] = {0.f, 0.f, 0.f, 0.f}, lR[4] = {0.f, 0.f, 0.f, 0.f};
    sums_issue<Q>(X, D, Xq, Dq, Xb, Db, ids, mt, nchunk, 0, smem);
    for (int st = 0; st < nstage; ++st) {
        if (st + 1 < nstage) {
            sums_issue<Q>(X, D, Xq, Dq, Xb, Db, ids, mt, nchunk, st + 1, smem);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        const int sl = st / nchunk, c = st - sl * nchunk, d0 = sl * SLAB;
        const int cnt = min(kPrRows, mt - c * kPrRows);
        const int nl = min(max(NL - c * kPrRows, 0), cnt);  // the chunk's list-0 rows come first
        const uint8_t* buf = smem + (st & 1) * (kPrRows * kPrStride);
        if (d0 + 4 * q < D) {
            int i = g;
            for (; i < nl; i += G) sums_add<Q>(buf + i * kPrStride, q, hL, lL);
            for (; i < cnt; i += G) sums_add<Q>(buf + i * kPrStride, q, hR, lR);
        }
        if (c == nchunk - 1 && Q != 0) {  // integer data: exact int32 sums of the slab's dims
            int* ired = reinterpret_cast<int*>(red);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                ired[(0 * G + g) * SLAB + 4 * q + j] = __float2int_rn(hL[j]);
                ired[(1 * G + g) * SLAB + 4 * q + j] = __float2int_rn(hR[j]);
                hL[j] = hR[j] = 0.f;
            }
            __syncthreads();
            if (tid < 2 * SLAB) {
                const int side = tid / SLAB, dd = tid - side * SLAB;
                if (d0 + dd < D) {
                    int acc = 0;
                    for (int gg = 0; gg < G; ++gg) acc += ired[(side * G + gg) * SLAB + dd];
                    ipart[(int64_t)side * D + d0 + dd] = acc;
                }
            }
        } else if (c == nchunk - 1) {  // the slab's rows are all in: combine the groups
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                red[(0 * G + g) * SLAB + 4 * q + j] = (double)hL[j] + (double)lL[j];
                red[(1 * G + g) * SLAB + 4 * q + j] = (double)hR[j] + (double)lR[j];
                hL[j] = lL[j] = hR[j] = lR[j] = 0.f;
            }
            __syncthreads();
            if (tid < 2 * SLAB) {
                const int side = tid / SLAB, dd = tid - side * SLAB;
                if (d0 + dd < D) {
                    double acc = 0.0;
                    for (int gg = 0; gg < G; ++gg) acc += red[(side * G + gg) * SLAB + dd];
                    part[(int64_t)side * D + d0 + dd] = acc;
                }
            }
        }
        __syncthreads();  // buffer st & 1 and red are reused
    }
}

__global__ void __launch_bounds__(kSuThreads) k1_sums_async(const float* __restrict__ X, int D,
                                                            const int32_t* __restrict__ perm,
                                                            const int4* __restrict__ tiles,
                                                            const float* __restrict__ S,
                                                            const int32_t* __restrict__ seg_off,
                                                            const uint64_t* __restrict__ thr, int pos_bits,
                                                            double* __restrict__ partial,
                                                            const int* __restrict__ status,
                                                            const uint16_t* __restrict__ Xq, int Dq, int qtype,
                                                            const int* __restrict__ qflag,
                                                            const uint8_t* __restrict__ Xb, int Db,
                                                            const int* __restrict__ bflag,
                                                            const float* __restrict__ Sp,
                                                            const uint64_t* __restrict__ thrp) {
    extern __shared__ __align__(16) uint8_t su_smem[];
    if (*status & kStatusStop) return;  // perm may hold unwritten slots
    const int q = u8_usable(Xb, bflag) ? 3 : q16_usable(Xq, qflag) ? qtype : 0;
    const int4 t = tiles[blockIdx.x];
    const int seg = t.x, begin = t.y, end = t.z;
    const int a = seg_off[seg];
    const uint64_t T = thr[seg], Tp = Sp ? thrp[seg] : 0;
    // this tile's sums: [2][D] FP64, or int32 for integer data (Q != 0)
    double* part = partial + (int64_t)blockIdx.x * 2 * D;
    int32_t* ipart = reinterpret_cast<int32_t*>(partial) + (int64_t)blockIdx.x * 2 * D;
    if (q == 3)
        sums_async_tile<3>(X, D, Xq, Dq, Xb, Db, perm, S, Sp, a, T, Tp, pos_bits, begin, end, part, ipart,
                           su_smem);
    else if (q == 1)
        sums_async_tile<1>(X, D, Xq, Dq, Xb, Db, perm, S, Sp, a, T, Tp, pos_bits, begin, end, part, ipart,
                           su_smem);
    else if (q == 2)
        sums_async_tile<2>(X, D, Xq, Dq, Xb, Db, perm, S, Sp, a, T, Tp, pos_bits, begin, end, part, ipart,
                           su_smem);
    else
        sums_async_tile<0>(X, D, Xq, Dq, Xb, Db, perm, S, Sp, a, T, Tp, pos_bits, begin, end, part, ipart,
                           su_smem);
}

// s / b rounded to nearest (FP64) from inv = RN(1 / b): the FMA residual
// r = s - q0 b of q0 = RN(s inv) is exact, and q0 + r inv rounds to RN(s / b)
// (Markstein's correction).  For integer s and b < 2^52 the quotient is never
// within the correction's error of a rounding boundary, so the result equals
// FP64 division bit for bit; it costs three FP64 operations, where GB300
// issues FP64 at a small fraction of its FP32 rate.
__device__ __forceinline__ double div_by(double s, double b, double inv) {
    const double q0 = __dmul_rn(s, inv);
    const double r = __fma_rn(-q0, b, s);
    return __fma_rn(r, inv, q0);
}

// RN32(S / K) of an integer sum: FP32 division when S and K are exact in FP32
// (no double rounding can separate it from RN32(RN64(S / K)) for K < 2^28:
// the quotient is either an FP32 midpoint, which FP64 holds exactly, or
// farther from one than FP64's rounding error), else FP64 division.
__device__ __forceinline__ float mean_of_ints(long long S, int K) {
    if (S > -16777216LL && S < 16777216LL && K < 16777216) return __fdiv_rn((float)S, (float)K);
    return (float)((double)S / (double)K);
}

// c1 - c0 of one dim from integer sums (int64 in segsum and segleft).  Full
// sweep: s0, s1 are the left and right sums; the segment's total and left sum
// are kept.  Delta sweep: s0, s1 are the sums of the points that moved left
// and right since the last cut, so left = kept left + s0 - s1.
__device__ __forceinline__ void store_w_ints(long long s0, long long s1, int seg, int d, int D, int K, int m,
                                             double* __restrict__ segsum, double* __restrict__ segleft, int delta,
                                             float* __restrict__ W) {
    long long* tot = reinterpret_cast<long long*>(segsum) + (int64_t)seg * D + d;
    long long* lft = reinterpret_cast<long long*>(segleft) + (int64_t)seg * D + d;
    long long sL = s0, sR = s1;
    if (delta) {
        sL = *lft + s0 - s1;
        sR = *tot - sL;
    } else {
        *tot = sL + sR;
    }
    *lft = sL;
    W[(int64_t)seg * D + d] = __fsub_rn(mean_of_ints(sR, m - K), mean_of_ints(sL, K));
}

// The same from FP64 sums: FP64 means rounded to FP32.
__device__ __forceinline__ void store_w(double s0, double s1, int seg, int d, int D, int K, int m, double inv0,
                                        double inv1, double* __restrict__ segsum, double* __restrict__ segleft,
                                        int delta, float* __restrict__ W) {
    double* tot = segsum + (int64_t)seg * D + d;
    double* lft = segleft + (int64_t)seg * D + d;
    double sL = s0, sR = s1;
    if (delta) {
        sL = *lft + s0 - s1;
        sR = *tot - sL;
    } else {
        *tot = sL + sR;
    }
    *lft = sL;
    const float c0 = (float)div_by(sL, (double)K, inv0);
    const float c1 = (float)div_by(sR, (double)(m - K), inv1);
    W[(int64_t)seg * D + d] = __fsub_rn(c1, c0);
}

// New centroids of each segment from its tiles' partial sums; stores
// w = c1 - c0.  A CTA takes 32 dims of one segment; its G warps sum
// interleaved tiles (warp g: tiles t0 + g, t0 + g + G, ... in order), then
// the G sums are added in warp order.  A sweep of both sides stores the
// segment's total (segsum); after a left-only sweep the right sum is that
// total minus the left sum.
template <int G>
__global__ void __launch_bounds__(32 * G) k1_centroids(const double* __restrict__ partial,
                                                       const int32_t* __restrict__ seg_off,
                                                       const int32_t* __restrict__ seg_tile0, int D,
                                                       double* __restrict__ segsum, double* __restrict__ segleft,
                                                       int delta, float* __restrict__ W,
                                                       const uint16_t* __restrict__ Xq,
                                                       const int* __restrict__ qflag,
                                                       const uint8_t* __restrict__ Xb,
                                                       const int* __restrict__ bflag) {
    __shared__ double red[G][2][32];
    __shared__ double inv[2];
    const int seg = blockIdx.x;
    const int m = seg_off[seg + 1] - seg_off[seg];
    const int K = m / 2;
    const int t0 = seg_tile0[seg], t1 = seg_tile0[seg + 1];
    if (t0 == t1) return;  // a finished tree's leaf: no centroids
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int d = blockIdx.y * 32 + lane;
    if (exact_ints(Xq, qflag, Xb, bflag)) {  // int32 partials, int64 sums
        const int32_t* ip = reinterpret_cast<const int32_t*>(partial);
        long long iL = 0, iR = 0;
        if (d < D) {
#pragma unroll 4
            for (int t = t0 + g; t < t1; t += G) {
                iL += ip[((int64_t)t * 2 + 0) * D + d];
                iR += ip[((int64_t)t * 2 + 1) * D + d];
            }
        }
        long long(*ired)[2][32] = reinterpret_cast<long long(*)[2][32]>(red);
        ired[g][0][lane] = iL;
        ired[g][1][lane] = iR;
        __syncthreads();
        if (g == 0 && d < D) {
            iL = ired[0][0][lane];
            iR = ired[0][1][lane];
#pragma unroll
            for (int q = 1; q < G; ++q) {
                iL += ired[q][0][lane];
                iR += ired[q][1][lane];
            }
            store_w_ints(iL, iR, seg, d, D, K, m, segsum, segleft, delta, W);
        }
        return;
    }
    if (threadIdx.x == 0) {
        inv[0] = 1.0 / (double)K;
        inv[1] = 1.0 / (double)(m - K);
    }
    double sL = 0.0, sR = 0.0;
    if (d < D) {
#pragma unroll 4
        for (int t = t0 + g; t < t1; t += G) {
            sL += partial[((int64_t)t * 2 + 0) * D + d];
            sR += partial[((int64_t)t * 2 + 1) * D + d];
        }
    }
    red[g][0][lane] = sL;
    red[g][1][lane] = sR;
    __syncthreads();
    if (g == 0 && d < D) {
        sL = red[0][0][lane];
        sR = red[0][1][lane];
#pragma unroll
        for (int q = 1; q < G; ++q) {
            sL += red[q][0][lane];
            sR += red[q][1][lane];
        }
        store_w(sL, sR, seg, d, D, K, m, inv[0], inv[1], segsum, segleft, delta, W);
    }
}

// Segments of one or two tiles: each warp takes 32 dims of one segment and
// sums its tiles in order.
__global__ void __launch_bounds__(256) k1_centroids_warp(const double* __restrict__ partial,
                                                         const int32_t* __restrict__ seg_off,
                                                         const int32_t* __restrict__ seg_tile0, int nseg, int D,
                                                         double* __restrict__ segsum, double* __restrict__ segleft,
                                                         int delta, float* __restrict__ W,
                                                         const uint16_t* __restrict__ Xq,
                                                         const int* __restrict__ qflag,
                                                         const uint8_t* __restrict__ Xb,
                                                         const int* __restrict__ bflag) {
    const int nch = (D + 31) / 32;
    const int pair = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (pair >= nseg * nch) return;
    const int seg = pair / nch, d = (pair - seg * nch) * 32 + lane;
    const int t0 = seg_tile0[seg], t1 = seg_tile0[seg + 1];
    if (t0 == t1) return;  // a finished tree's leaf: no centroids
    const int m = seg_off[seg + 1] - seg_off[seg];
    const int K = m / 2;
    if (exact_ints(Xq, qflag, Xb, bflag)) {  // int32 partials, int64 sums
        if (d >= D) return;
        const int32_t* ip = reinterpret_cast<const int32_t*>(partial);
        long long iL = 0, iR = 0;
        for (int t = t0; t < t1; ++t) {
            iL += ip[((int64_t)t * 2 + 0) * D + d];
            iR += ip[((int64_t)t * 2 + 1) * D + d];
        }
        store_w_ints(iL, iR, seg, d, D, K, m, segsum, segleft, delta, W);
        return;
    }
    double inv0 = 0.0, inv1 = 0.0;
    if (lane == 0) {
        inv0 = 1.0 / (double)K;
        inv1 = 1.0 / (double)(m - K);
    }
    inv0 = __shfl_sync(0xffffffffu, inv0, 0);
    inv1 = __shfl_sync(0xffffffffu, inv1, 0);
    if (d >= D) return;
    double sL = 0.0, sR = 0.0;
    for (int t = t0; t < t1; ++t) {
        sL += partial[((int64_t)t * 2 + 0) * D + d];
        sR += partial[((int64_t)t * 2 + 1) * D + d];
    }
    store_w(sL, sR, seg, d, D, K, m, inv0, inv1, segsum, segleft, delta, W);
}

template <int G>
void launch_centroids(const LevelPlan& lp, const SplitBuffers& b, int D, int delta, cudaStream_t s) {
    k1_centroids<G><<<dim3(lp.nseg, (D + 31) / 32), 32 * G, 0, s>>>(b.partial, lp.seg_off, lp.seg_tile0, D,
                                                                     b.segsum, b.segleft, delta, b.W, b.Xq,
                                                                     b.qflag, b.Xb, b.bflag);
}

__global__ void __launch_bounds__(256) k1_part_count(const float* __restrict__ S, const int4* __restrict__ tiles,
                                                     const int32_t* __restrict__ seg_off,
                                                     const uint64_t* __restrict__ thr, int pos_bits,
                                                     int32_t* __restrict__ tile_left) {
    __shared__ int warp_tot[32];
    const int4 t = tiles[blockIdx.x];
    const int a = seg_off[t.x];
    const uint64_t T = thr[t.x];
    int c = 0;
    for (int p = t.y + threadIdx.x; p < t.z; p += blockDim.x) c += sel_key(S[p], p - a, pos_bits) < T;
    c = block_sum(c, warp_tot);
    if (threadIdx.x == 0) tile_left[blockIdx.x] = c;
}

__global__ void __launch_bounds__(256) k1_part_scatter(const float* __restrict__ S, const int4* __restrict__ tiles,
                                                       const int32_t* __restrict__ seg_off,
                                                       const int32_t* __restrict__ seg_tile0,
                                                       const uint64_t* __restrict__ thr, int pos_bits,
                                                       const int32_t* __restrict__ tile_left,
                                                       const int32_t* __restrict__ perm_in,
                                                       int32_t* __restrict__ perm_out, int* __restrict__ status) {
    __shared__ int warp_tot[32];
    const int4 t = tiles[blockIdx.x];
    const int seg = t.x;
    const int a = seg_off[seg], m = seg_off[seg + 1] - a, K = m / 2;
    const uint64_t T = thr[seg];
    // the tile's projections and ids first (all loads in flight at once)
    constexpr int PER = kTile / 256;
    float sv[PER];
    int id[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int p = t.y + (int)threadIdx.x + 256 * i;
        sv[i] = p < t.z ? S[p] : 0.f;
        id[i] = p < t.z ? perm_in[p] : 0;
    }
    int lb = 0;
    for (int q = seg_tile0[seg] + threadIdx.x; q < (int)blockIdx.x; q += blockDim.x) lb += tile_left[q];
    lb = block_sum(lb, warp_tot);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int p = t.y + (int)threadIdx.x + 256 * i;
        const int isl = p < t.z && sel_key(sv[i], p - a, pos_bits) < T;
        int tot;
        const int ex = block_excl_scan(isl, warp_tot, &tot);
        if (p < t.z) {
            const int l = lb + ex;
            const int np = isl ? l : K + (p - a - l);
            if ((isl ? np < K : np < m) && np >= 0)
                perm_out[a + np] = id[i];
            else
                atomicOr(status, kStatusInternal);
        }
        lb += tot;
    }
}

}  // namespace

void run_split_level(const float* X, int D, const LevelPlan& lp, int iters, uint64_t pass_seed,
                     const int32_t* perm_in, int32_t* perm_out, const SplitBuffers& b, cudaStream_t s) {
    // algorithmic bytes: a sweep reads every row once plus its id and key
    const double n = lp.n, rows = n * (b.u8_host ? b.Db * 1.0 : b.q16_host ? b.Dq * 2.0 : D * 4.0);
    // the staged kernels read 16-byte pieces of rows: of X (vec) or of the
    // byte copy, whose rows are padded (when the host knows it is usable)
    const bool vec = ((D % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0)) || b.u8_host;
    const bool vec2 = (D % 2 == 0) && ((reinterpret_cast<uintptr_t>(X) & 7) == 0);
    const int dchunks = (D + 127) / 128;
    // finished trees' leaves keep their place: the cut below writes only the
    // segments that split
    if (lp.frozen) cudaMemcpyAsync(perm_out, perm_in, sizeof(int32_t) * (size_t)lp.n, cudaMemcpyDeviceToDevice, s);
    {
        LaunchScope ls("k1_init", s, (double)lp.nseg * 3 * D * 4, 0);
        k1_init<<<lp.nseg, 128, 0, s>>>(X, D, perm_in, lp.seg_off, lp.seg_tile0, lp.seg_local, lp.level, pass_seed,
                                        b.W, b.status);
    }
    for (int it = 0; it <= iters; ++it) {
        const bool last = it == iters;
        // projections and keys alternate between two buffers, so that a
        // sweep can compare this iteration's cut with the previous one
        SplitBuffers bi = b;
        if (it & 1) {
            bi.S = b.S2;
            bi.thr = b.thr2;
        }
        const float* Sp = it > 0 ? ((it & 1) ? b.S : b.S2) : nullptr;
        const uint64_t* Tp = it > 0 ? ((it & 1) ? b.thr : b.thr2) : nullptr;
        {
            LaunchScope ls("k1_project", s, rows + n * 8, 2.0 * n * D);
            SelState* st = lp.small ? nullptr : b.st;
            if (vec) {
                cudaFuncSetAttribute(k1_project_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize, kPpSmem);
                const int grid = std::min(lp.nsweep, 2 * sm_count());
                k1_project_pipe<<<grid, kPrRows, kPpSmem, s>>>(X, D, perm_in, lp.sweep, lp.nsweep, lp.seg_off, b.W,
                                                               bi.S, st, b.status, b.Xq, b.Dq, b.qtype, b.qflag,
                                                               b.Xb, b.Db, b.bflag);
            } else if (vec2)
                k1_project<true><<<lp.nsweep, 256, 0, s>>>(X, D, perm_in, lp.sweep, lp.seg_off, b.W, bi.S, st,
                                                           b.status, b.Xq, b.Dq, b.qtype, b.qflag);
            else
                k1_project<false><<<lp.nsweep, 256, 0, s>>>(X, D, perm_in, lp.sweep, lp.seg_off, b.W, bi.S, st,
                                                            b.status, b.Xq, b.Dq, b.qtype, b.qflag);
        }
        if (lp.small && lp.max_m <= kSortSelectMax) {
            LaunchScope ls("k1_select_sort", s, n * 4 + (last ? n * 8 : 0), 0);
            int32_t* out = last ? perm_out : nullptr;
            if (lp.max_m <= 32)
                launch_select_sort<1, 1>(lp, bi, perm_in, out, s);
            else if (lp.max_m <= 64)
                launch_select_sort<2, 1>(lp, bi, perm_in, out, s);
            else if (lp.max_m <= 128)
                launch_select_sort<4, 1>(lp, bi, perm_in, out, s);
            else if (lp.max_m <= 256)
                launch_select_sort<8, 1>(lp, bi, perm_in, out, s);
            else if (lp.max_m <= 512)
                launch_select_sort<8, 2>(lp, bi, perm_in, out, s);
            else if (lp.max_m <= 1024)
                launch_select_sort<8, 4>(lp, bi, perm_in, out, s);
            else
                launch_select_sort<8, 8>(lp, bi, perm_in, out, s);
            if (last) break;
        } else if (lp.small) {
            const size_t smem = (size_t)lp.max_m * sizeof(uint64_t);
            // one thread per point up to 1024, at least 4 warps
            const int nt = std::min(1024, std::max(128, (lp.max_m + 31) & ~31));
            LaunchScope ls("k1_select_small", s, n * 4 + (last ? n * 8 : 0), 0);
            cudaFuncSetAttribute(k1_select_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k1_select_small<<<lp.nseg, nt, smem, s>>>(bi.S, lp.seg_off, lp.seg_tile0, lp.pos_bits, bi.thr, perm_in,
                                                      last ? perm_out : nullptr, b.status);
            if (last) break;
        } else {
            // every value digit is launched, then the position pass; a
            // segment whose key is known returns at once
            for (int hi = 32 + lp.pos_bits; hi > lp.pos_bits; hi = digit_lo(hi, lp.pos_bits)) {
                LaunchScope ls("k1_select_pass", s, n * 4, 0);
                k1_select_pass<<<lp.ntiles, 256, 0, s>>>(bi.S, lp.tiles, lp.seg_off, lp.seg_tile0, lp.pos_bits, hi,
                                                         b.st, b.ghist, b.ticket, bi.thr);
            }
            {
                LaunchScope ls("k1_select_pos", s, n * 4, 0);
                k1_select_pos<<<lp.ntiles, 256, 0, s>>>(bi.S, lp.tiles, lp.seg_off, lp.seg_tile0, lp.pos_bits, b.st,
                                                        b.tile_left, b.ticket, bi.thr);
            }
            if (last) {
                {
                    LaunchScope ls("k1_part_count", s, n * 4, 0);
                    k1_part_count<<<lp.ntiles, 256, 0, s>>>(bi.S, lp.tiles, lp.seg_off, bi.thr, lp.pos_bits,
                                                            b.tile_left);
                }
                LaunchScope ls("k1_part_scatter", s, n * 12, 0);
                k1_part_scatter<<<lp.ntiles, 256, 0, s>>>(bi.S, lp.tiles, lp.seg_off, lp.seg_tile0, bi.thr,
                                                          lp.pos_bits, b.tile_left, perm_in, perm_out, b.status);
                break;
            }
        }
        // the first sweep sums both sides (and so each segment's total); the
        // later ones read only the points whose side changed at this cut
        // (delta), which Lloyd's iterations make ever fewer
        const int delta = it > 0;
        {
            LaunchScope ls("k1_sums", s, delta ? n * 12 : rows + n * 8, n * D);
            dim3 grid(lp.ntiles, dchunks);
            // the staged sums pay off on an exact narrow copy (when the host
            // does not know, as in a captured build, they decide on the device)
            if (vec && (b.Xq || b.Xb) && (b.u8_host || b.q16_host || b.capture)) {
                cudaFuncSetAttribute(k1_sums_async, cudaFuncAttributeMaxDynamicSharedMemorySize, kSuSmem);
                k1_sums_async<<<lp.ntiles, kSuThreads, kSuSmem, s>>>(X, D, perm_in, lp.tiles, bi.S, lp.seg_off,
                                                                     bi.thr, lp.pos_bits, b.partial, b.status, b.Xq,
                                                                     b.Dq, b.qtype, b.qflag, b.Xb, b.Db, b.bflag, Sp,
                                                                     Tp);
            } else if (vec)
                k1_sums<true><<<grid, 32 * kSumsWarps, 0, s>>>(X, D, perm_in, lp.tiles, bi.S, lp.seg_off, bi.thr,
                                                               lp.pos_bits, b.partial, b.status, b.Xq, b.Dq,
                                                               b.qtype, b.qflag, b.Xb, b.bflag, Sp, Tp);
            else
                k1_sums<false><<<grid, 32 * kSumsWarps, 0, s>>>(X, D, perm_in, lp.tiles, bi.S, lp.seg_off, bi.thr,
                                                                lp.pos_bits, b.partial, b.status, b.Xq, b.Dq,
                                                                b.qtype, b.qflag, b.Xb, b.bflag, Sp, Tp);
        }
        {
            LaunchScope ls("k1_centroids", s, (double)lp.ntiles * 2 * D * 8 + (double)lp.nseg * D * 4, 0);
            // warps per CTA: about one per tile of the largest segment, up to 32
            const int tiles = (lp.max_m + kTile - 1) / kTile + 1;
            if (tiles <= 3) {
                const int64_t pairs = (int64_t)lp.nseg * ((D + 31) / 32);
                k1_centroids_warp<<<(unsigned)((pairs + 7) / 8), 256, 0, s>>>(b.partial, lp.seg_off, lp.seg_tile0,
                                                                               lp.nseg, D, b.segsum, b.segleft, delta,
                                                                               b.W,
                                                                               b.Xq, b.qflag, b.Xb, b.bflag);
            } else if (tiles <= 8)
                launch_centroids<8>(lp, b, D, delta, s);
            else
                launch_centroids<32>(lp, b, D, delta, s);
        }
    }
}

void launch_bytes(const float* X, int64_t n, int D, int Db, uint8_t* Xb, int* bflag, cudaStream_t s) {
    LaunchScope ls("k0_bytes", s, (double)n * (D * 4.0 + Db), 0);
    k0_bytes<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(X, n, D, Db, Xb, bflag);
}

}  // namespace knng
