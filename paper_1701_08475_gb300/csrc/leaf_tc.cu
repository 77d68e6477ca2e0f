// leaf_tc.cu -- the low-precision leaf stage on tcgen05 tensor cores.
//
//   K0 quantize   a BF16 or FP16 copy x^ of every point in leaf order, its
//                 squared norm ||x^||^2 (FP32) and its quantisation error
//                 e = ||x - x^|| (rounded up), plus one flag saying whether
//                 the low-precision arithmetic is exact for this input
//   K2 leaf       per leaf (m <= 128 points): the Gram matrix x^_i . x^_j on
//                 the tensor cores (TMA loads of the leaf's rows into 128-byte
//                 swizzled shared memory, tcgen05.mma with the FP32
//                 accumulator in tensor memory), approximate distances
//                 d^ = ||x^_i||^2 + ||x^_j||^2 - 2 x^_i . x^_j, and per row:
//   K3 re-rank    the k' best approximate candidates get their canonical FP32
//                 distance; the row is certified when no excluded candidate
//                 can beat the row's k-th exact entry by the error bound below,
//                 else it is recomputed exactly over the whole leaf.
//
// With the certificate the graph is identical to the FP32 path's.  When all
// values are integers that the 16-bit type holds exactly and every norm is
// below 2^23, products and sums are exact integers in FP32, d^ is the
// canonical distance itself and no re-rank is needed.
//
// FP8 E4M3 form: each row is scaled first, x~ = s q with s = max|x| / 448 and
// q the E4M3 rounding (nearest even, saturating) of x / s; the tensor cores
// form q_i . q_j (kind::f8f6f4, FP32 accumulation), and
// d^ = ||x~_i||^2 + ||x~_j||^2 - 2 s_i s_j (q_i . q_j).  The bound below then
// holds with x~ in place of x^ and the FP8 accumulation term c8 added to c_D:
// the PTX ISA does not state how many bits the FP8 path keeps while it sums,
// so the certificate assumes at least a 14-bit significand with truncation,
// c8 = D 2^-13 (a previous generation's FP8 path was reported to keep about
// 14 bits); the Gram error the hardware actually makes is measured against
// this assumption by the tests.
//
// Error bound of d^ against the exact distance d of the FP32 points (per row
// i, against every candidate j of the leaf):
//   |sqrt(d) - sqrt(d~)| <= e_i + e_j            (d~: exact distance of x^)
//   |d^ - d~| <= c_D (||x^_i|| + ||x^_j||)^2 + 2^-23 |d^|
// with c_D = (16 D + 8) 2^-24: four times the textbook bound for the FP32
// sums (Higham, Ch. 3) because the tensor cores' summation order and internal
// rounding are not specified.  A candidate excluded with approximate value
// a >= a* can only beat the k-th exact entry t if
//   (sqrt(max(0, a* - eps)) - e_i - e_max)^2 <= t.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace knng {

namespace {

// ---------------------------------------------------------------- K0
template <bool BF16>
__device__ __forceinline__ uint16_t quantize_bits(float x, float* back) {
    if (BF16) {
        const __nv_bfloat16 q = __float2bfloat16_rn(x);
        *back = __bfloat162float(q);
        return __bfloat16_as_ushort(q);
    } else {
        const __half q = __float2half_rn(x);
        *back = __half2float(q);
        return __half_as_ushort(q);
    }
}

// One warp per output row p (= leaf-order position): the row of point
// perm[p], dims padded with zeros to Dp.  Flags in *notexact: 1 = some value
// is not an integer the 16-bit type holds exactly, or some squared norm is
// 2^23 or more; 2 = some value is negative; 4 = some squared norm is 2^22 or
// more.  The 16-bit arithmetic is exact unless flag 1 is set or flags 2 and 4
// both are: then every norm, Gram entry and distance (and every partial sum
// of them) is an integer below 2^24.
template <bool BF16>
__global__ void __launch_bounds__(256) k0_quantize(const float* __restrict__ X, int64_t n, int D, int Dp,
                                                   const int32_t* __restrict__ perm, uint16_t* __restrict__ Xq,
                                                   float* __restrict__ nrm, float* __restrict__ qerr,
                                                   int* __restrict__ notexact) {
    const int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (p >= n) return;
    const int lane = threadIdx.x & 31;
    const int64_t i = perm ? perm[p] : p;
    const float lim = BF16 ? 256.f : 2048.f;
    float sq = 0.f, e2 = 0.f;
    bool exact = true, neg = false;
    for (int d = lane; d < Dp; d += 32) {
        const float x = d < D ? X[i * D + d] : 0.f;
        float b;
        Xq[p * Dp + d] = quantize_bits<BF16>(x, &b);
        sq = __fmaf_rn(b, b, sq);
        const float t = __fsub_rn(x, b);  // exact: b is x rounded to fewer bits
        e2 = __fmaf_rn(t, t, e2);
        exact &= (x == rintf(x)) && fabsf(x) <= lim;
        neg |= x < 0.f;
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        sq += __shfl_xor_sync(0xffffffffu, sq, m);
        e2 += __shfl_xor_sync(0xffffffffu, e2, m);
    }
    exact = __all_sync(0xffffffffu, exact);
    neg = __any_sync(0xffffffffu, neg);
    if (lane == 0) {
        nrm[p] = sq;
        // an upper bound: the FP32 sum of Dp squares is within (Dp + 2) u of
        // the exact sum (Higham, Ch. 3), the square root rounds up
        qerr[p] = e2 > 0.f ? __fsqrt_ru(__fmul_ru(e2, 1.f + (float)(Dp + 8) * 5.9604645e-8f)) : 0.f;
        const int f = ((!exact || sq >= 8388608.f) ? 1 : 0) | (neg ? 2 : 0) | (sq >= 4194304.f ? 4 : 0);
        if (f) atomicOr(notexact, f);
    }
}

// FP8 E4M3 copy with a scale per row (one warp per output row p, dims padded
// with zeros to Dp): s = max|x| / 448 (1 for a row of zeros), q = E4M3(x / s)
// rounded to nearest even and saturated, ||x~||^2 = s^2 sum q^2 and an upper
// bound of e = ||x - s q||.  The FP8 arithmetic is never taken as exact
// (*notexact |= 1).
__global__ void __launch_bounds__(256) k0_quantize_e4m3(const float* __restrict__ X, int64_t n, int D, int Dp,
                                                        const int32_t* __restrict__ perm, uint8_t* __restrict__ Xq,
                                                        float* __restrict__ nrm, float* __restrict__ qerr,
                                                        float* __restrict__ scale, int* __restrict__ notexact) {
    const int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (p >= n) return;
    const int lane = threadIdx.x & 31;
    const int64_t i = perm ? perm[p] : p;
    float amax = 0.f;
    for (int d = lane; d < D; d += 32) amax = fmaxf(amax, fabsf(X[i * D + d]));
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, m));
    // a row whose largest value is tiny keeps the scale 1 (its values round to
    // zero or to subnormals, and e then covers them)
    const float sc = amax >= 1e-30f ? __fdiv_rn(amax, 448.f) : 1.f;
    float sq = 0.f, e2 = 0.f;
    for (int d = lane; d < Dp; d += 32) {
        const float x = d < D ? X[i * D + d] : 0.f;
        const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(__fdiv_rn(x, sc), __NV_SATFINITE, __NV_E4M3);
        Xq[p * Dp + d] = (uint8_t)q;
        const float qf = __half2float(__half(__nv_cvt_fp8_to_halfraw(q, __NV_E4M3)));
        sq = __fmaf_rn(qf, qf, sq);                // products exact: 4-bit significands
        const float t = __fmaf_rn(-sc, qf, x);      // x - s q, rounded once
        e2 = __fmaf_rn(t, t, e2);
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        sq += __shfl_xor_sync(0xffffffffu, sq, m);
        e2 += __shfl_xor_sync(0xffffffffu, e2, m);
    }
    if (lane == 0) {
        nrm[p] = __fmul_rn(__fmul_rn(sc, sc), sq);
        scale[p] = sc;
        // upper bound: the rounding of each difference (1 + u)^2, the FP32 sum
        // of Dp squares (Dp + 2) u (Higham, Ch. 3), the square root rounded up
        qerr[p] = e2 > 0.f ? __fsqrt_ru(__fmul_ru(e2, 1.f + (float)(Dp + 16) * 5.9604645e-8f)) : 0.f;
        if (p == 0) atomicOr(notexact, 1);
    }
}

__device__ __forceinline__ bool lp_exact(int f) { return (f & 1) == 0 && !((f & 2) && (f & 4)); }

// Leaf-order copy gathered from the original-order one: row p of the output
// is row perm[p] of the input (16-byte pieces), with its norm, error and
// (FP8 only) scale.
__global__ void __launch_bounds__(256) k0_permute16(const uint4* __restrict__ Xq, const float* __restrict__ nrm,
                                                    const float* __restrict__ qerr, const float* __restrict__ scale,
                                                    int64_t n, int q_per_row, const int32_t* __restrict__ perm,
                                                    uint4* __restrict__ Xl, float* __restrict__ lnrm,
                                                    float* __restrict__ lerr, float* __restrict__ lscale) {
    const int64_t total = n * q_per_row;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / q_per_row;
        const int q = (int)(e - p * q_per_row);
        const int64_t i = perm[p];
        Xl[e] = __ldg(Xq + i * q_per_row + q);
        if (q == 0) {
            lnrm[p] = nrm[i];
            lerr[p] = qerr[i];
            if (scale) lscale[p] = scale[i];
        }
    }
}

// ---------------------------------------------------------------- K2/K3
constexpr int kTcRows = 128;             // M = N = 128 tile: leaves up to 128 points
constexpr int kTcK = 64;                 // 16-bit elements per 128-byte swizzled row
constexpr int kRowChunk = 128;           // bytes of a row per K chunk (one swizzle span)
constexpr int kStageBytes = kTcRows * kRowChunk;
constexpr int kTcThreads = 128;

struct TcSmem {
    int stages;
    size_t stage_off, dt_off, bar_off, misc_off, scratch_off, total;
};

// MT row tiles of 128 (leaves up to 128 MT points): stages of MT boxes, the
// d^ rows of one tile, barriers, then misc: tmem address, abort flag,
// ids / norms / errors / rounded-up sqrt norms / scales [128 MT] each, two
// maxima; then 32 keys of merge scratch per warp.  Dpb: bytes per row.
__host__ __device__ inline TcSmem tc_smem(int Dpb, int MT) {
    TcSmem L;
    const int nk = Dpb / kRowChunk;
    const int smax = MT == 1 ? 4 : 2;
    L.stages = nk < smax ? nk : smax;
    L.stage_off = 0;
    const size_t stages = (size_t)L.stages * kStageBytes * MT;
    // the d^ rows of half a row tile at a time, over the stages (dead once
    // the product is done): a smaller footprint, more CTAs per SM
    L.dt_off = 0;
    const size_t dt = (size_t)(kTcRows / 2) * (kTcRows * MT + 1) * 4;
    L.bar_off = ((stages > dt ? stages : dt) + 15) & ~(size_t)15;
    L.misc_off = L.bar_off + (size_t)(2 * L.stages + 1) * 8;
    L.scratch_off = L.misc_off + 16 + 5 * (size_t)kTcRows * MT * 4 + 16;
    L.total = L.scratch_off + (kTcThreads / 32) * 32 * 8;
    return L;
}

// the key that lane `src` holds
__device__ __forceinline__ uint64_t lane_key(uint64_t v, int src) { return shfl64(v, src); }

// entry r of a list held lane-major in NO slots (r < 32 * NO)
template <int NO>
__device__ __forceinline__ uint64_t list_at(const uint64_t (&v)[NO], int r) {
    uint64_t mine = v[0];
#pragma unroll
    for (int o = 1; o < NO; ++o)
        if (o == (r >> 5)) mine = v[o];
    return shfl64(mine, r & 31);
}

// QT: 0 FP16, 1 BF16 (kind::f16), 2 FP8 E4M3 (kind::f8f6f4, scaled rows).
// Dpb: bytes per row of the copy; cD: the certificate's coefficient of
// (||x^_i|| + ||x^_j||)^2.  dump (a parity hook; one leaf): the d^ rows are
// written to dump (m x m) and nothing is selected.
template <int QT, int NSG, int MT>
__global__ void __launch_bounds__(kTcThreads, 1) k2_leaf_tc(const __grid_constant__ CUtensorMap tmap, int Dpb,
                                                           float cD, const float* __restrict__ X, int D,
                                                           const int32_t* __restrict__ perm,
                                                           const int32_t* __restrict__ leaf_off,
                                                           const float* __restrict__ nrm,
                                                           const float* __restrict__ qerr,
                                                           const float* __restrict__ scale, int k, int kp,
                                                           uint64_t* __restrict__ G, int* __restrict__ status,
                                                           const int* __restrict__ notexact,
                                                           float* __restrict__ dump) {
    constexpr int RW = kTcRows * MT;      // leaf rows (and Gram columns) held
    constexpr int DTS = RW + 1;           // d^ row stride
    constexpr int SB = kStageBytes * MT;  // one K chunk of all rows
    extern __shared__ uint8_t smem_raw[];
    if (*status & kStatusStop) return;  // whole CTA, before any barrier or tensor memory
    const TcSmem L = tc_smem(Dpb, MT);
    uint8_t* base = smem_raw + ((1024 - (tc::smem_addr(smem_raw) & 1023)) & 1023);
    float* dt = reinterpret_cast<float*>(base + L.dt_off);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + L.bar_off);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + L.misc_off);
    int* abort_flag = reinterpret_cast<int*>(base + L.misc_off + 4);
    int32_t* sid = reinterpret_cast<int32_t*>(base + L.misc_off + 16);
    float* snrm = reinterpret_cast<float*>(sid + RW);
    float* serr = snrm + RW;
    float* srt = serr + RW;   // ||x^|| rounded up
    float* sscl = srt + RW;   // row scales (FP8; 1 otherwise)
    float* smax = sscl + RW;  // [0] max ||x^||, [1] max e

    const int S = L.stages, nk = Dpb / kRowChunk;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // MT = 2: two CTAs per leaf, CTA `tile` takes the leaf's rows
    // 128 tile .. 128 tile + 127 against all of its (up to 256) columns
    const int leaf = blockIdx.x / MT, tile = MT == 1 ? 0 : (int)(blockIdx.x % MT);
    const int a = leaf_off[leaf];
    const int m = leaf_off[leaf + 1] - a;
    if (tile * kTcRows >= m) return;  // a leaf of one tile: nothing for the second CTA
    const uint32_t full0 = tc::smem_addr(bars), empty0 = full0 + 8 * S, done = full0 + 16 * S;
    constexpr uint32_t kCols = kTcRows * MT;  // tensor-memory columns: one row tile against RW columns

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(full0 + 8 * s, 1);
            tc::mbar_init(empty0 + 8 * s, 1);
        }
        tc::mbar_init(done, 1);
        tc::mbar_fence_init();
        *abort_flag = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_addr(tmem_slot), kCols);
        tc::tmem_relinquish();
    }
    for (int r = tid; r < RW; r += kTcThreads) {
        const bool in = r < m;
        sid[r] = in ? perm[a + r] : 0;
        snrm[r] = in ? nrm[a + r] : 0.f;
        serr[r] = in ? qerr[a + r] : 0.f;
        sscl[r] = (in && QT == 2) ? scale[a + r] : 1.f;
    }
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    // ---- producer + MMA issue (one thread): per K chunk, the CTA's row tile
    // of the Gram, A = rows 128 tile .., B = all RW rows (N = RW)
    if (tid == 0) {
        bool ok = true;
        const uint32_t idesc = QT == 2 ? tc::idesc_e4m3(kTcRows, RW) : tc::idesc_f16(QT == 1, kTcRows, RW);
        int issued = 0, consumed = 0;
        auto load_stage = [&](int s, int c) {
            const uint32_t fb = full0 + 8 * s;
            tc::mbar_expect_tx(fb, SB);
#pragma unroll
            for (int t = 0; t < MT; ++t)
                tc::tma_load_2d(tc::smem_addr(base + (size_t)s * SB + (size_t)t * kStageBytes), &tmap,
                                c * (QT == 2 ? kRowChunk : kTcK), a + t * kTcRows, fb);
        };
        for (; issued < S && issued < nk; ++issued) load_stage(issued, issued);
        for (int c = 0; c < nk; ++c) {
            const int s = c % S;
            if (!tc::mbar_wait(full0 + 8 * s, (uint32_t)((c / S) & 1), status)) {
                ok = false;
                break;
            }
            consumed = c + 1;
            const uint64_t d0 = tc::sdesc_k128(tc::smem_addr(base + (size_t)s * SB));
            const uint64_t da = d0 + (uint64_t)(tile * (kStageBytes >> 4));
#pragma unroll
            for (int kk = 0; kk < kRowChunk / 32; ++kk) {  // 32 bytes along the row per instruction
                // (K = 16 16-bit or K = 32 FP8 elements)
                if (QT == 2)
                    tc::mma_f8(tmem, da + 2 * kk, d0 + 2 * kk, idesc, (c | kk) != 0);
                else
                    tc::mma_f16(tmem, da + 2 * kk, d0 + 2 * kk, idesc, (c | kk) != 0);
            }
            tc::mma_commit(empty0 + 8 * s);
            if (c + S < nk) {
                if (!tc::mbar_wait(empty0 + 8 * s, (uint32_t)((c / S) & 1), status)) {
                    ok = false;
                    break;
                }
                load_stage(s, c + S);
                ++issued;
            }
        }
        tc::mma_commit(done);
        if (!ok) {
            *abort_flag = 1;
            // let the loads still in flight land before the CTA can exit
            for (int c = consumed; c < issued; ++c) tc::mbar_wait(full0 + 8 * (c % S), (uint32_t)((c / S) & 1), status);
        }
    }
    __syncwarp();
    // one thread watches the barrier; the others sleep in __syncthreads
    const int mma_ok = tid == 0 ? (tc::mbar_wait(done, 0, status) ? 1 : 0) : 1;
    // uniform over the CTA: the tensor-memory loads below are warp-collective
    const bool ok = __syncthreads_and(mma_ok) && *abort_flag == 0;
    tc::fence_after_sync();
    if (!ok) {
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 0) tc::tmem_dealloc(tmem, kCols);
        return;
    }

    // leaf maxima of ||x^|| and e for the certificate; every ||x^|| rounded up
    for (int r = tid; r < RW; r += kTcThreads) srt[r] = r < m ? __fsqrt_ru(snrm[r]) : 0.f;
    if (warp == 0) {
        float mn = 0.f, me = 0.f;
        for (int r = lane; r < m; r += 32) {
            mn = fmaxf(mn, sqrtf(snrm[r]));
            me = fmaxf(me, serr[r]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn = fmaxf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            me = fmaxf(me, __shfl_xor_sync(0xffffffffu, me, o));
        }
        if (lane == 0) {
            smax[0] = mn * (1.f + 1e-6f);
            smax[1] = me;
        }
    }

    const bool exact = lp_exact(*notexact);
    const bool vec = (D % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    constexpr int NC = RW / 32;
    uint64_t* wscratch = reinterpret_cast<uint64_t*>(base + L.scratch_off) + warp * 32;
    // Two phases: the two halves of the CTA's row tile; dt holds the phase's
    // d^ rows.  dt lies over the operand stages, which the completed product
    // has read through the async proxy.
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    for (int ph = 0; ph < 2; ++ph) {
    const int t = tile;                // row tile
    const int r0 = ph * (kTcRows / 2);  // the phase's first row in the tile
    const int pr = kTcRows / 2;         // rows per phase
    // ---- the phase's d^ rows: thread = TMEM lane = row 128 t + warp * 32 + lane
    if ((warp >> 1) == ph) {
        const int rl = warp * 32 + lane, R = t * kTcRows + rl, rd = rl - r0;
#pragma unroll 1
        for (int cc = 0; cc < RW / 32; ++cc) {
            float v[32];
            tc::tmem_ld_32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), v);
            if (QT == 2) {
                const float s2 = __fmul_rn(2.f, sscl[R]);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = cc * 32 + j;
                    dt[rd * DTS + col] =
                        __fsub_rn(__fadd_rn(snrm[R], snrm[col]), __fmul_rn(__fmul_rn(s2, sscl[col]), v[j]));
                }
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = cc * 32 + j;
                    dt[rd * DTS + col] = __fsub_rn(__fadd_rn(snrm[R], snrm[col]), __fmul_rn(2.f, v[j]));
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (ph == 1 && warp == 0) tc::tmem_dealloc(tmem, kCols);
    const int rows_t = min(r0 + pr, min(kTcRows, m - t * kTcRows));
    if (dump) {  // the parity hook: the phase's d^ rows, nothing selected
        for (int e = tid; e < pr * m; e += kTcThreads) {
            const int r = r0 + e / m, col = e - (e / m) * m;
            if (r < rows_t) dump[(int64_t)(t * kTcRows + r) * m + col] = dt[(r - r0) * DTS + col];
        }
        __syncthreads();
        continue;
    }
    for (int r = r0 + warp; r < rows_t; r += kTcThreads / 32) {
        const int R = t * kTcRows + r;  // the row in the leaf; rd: its d^ row
        const int rd = r - r0;
        const int gi = sid[R];
        uint64_t* grow = G + (int64_t)gi * k;
        uint64_t old[NSG];
#pragma unroll
        for (int s = 0; s < NSG; ++s) old[s] = lane + 32 * s < k ? grow[lane + 32 * s] : kEmptyKey;
        uint64_t res[NSG];
        bool done_row = false;
        if (exact) {
            // d^ is the canonical distance itself
            uint64_t cand[NC + NSG];
#pragma unroll
            for (int s = 0; s < NC; ++s) {
                const int c = lane + 32 * s;
                cand[s] = (c < m && c != R) ? make_key(__fadd_rn(dt[rd * DTS + c], 0.f), (uint32_t)sid[c])
                                            : kEmptyKey;
            }
            if (NSG == 1) {
                // few candidates beat the row's k-th entry after the first pass
                uint64_t few[NC];
#pragma unroll
                for (int s = 0; s < NC; ++s) few[s] = cand[s];
                uint64_t out;
                bool changed;
                if (warp_merge_few<NC>(few, old[0], k, wscratch, out, changed)) {
                    if (changed && lane < k) grow[lane] = out;
                    continue;
                }
                // many survive (the first pass): the lanes' smallest first
#pragma unroll
                for (int s = 0; s < NC; ++s) few[s] = cand[s];
                if (warp_merge_many<NC>(few, old[0], k, wscratch, out, changed)) {
                    if (changed && lane < k) grow[lane] = out;
                    continue;
                }
            }
#pragma unroll
            for (int s = 0; s < NSG; ++s) cand[NC + s] = old[s];
            sort_regs<NC + NSG>(cand);
            warp_select_unique<NC + NSG, NSG>(cand, k, res);
            done_row = true;
        } else if (m - 1 > 0) {
            if (NSG == 1) {
                // Pruned exact re-rank (k <= 32).  With the bound above,
                // evaluated per candidate and rounded so that it stays a lower
                // bound, lb_c = (sqrt(a_c - eps_c) - e_i - e_c)^2 <= d_c; a
                // candidate with lb_c above the row's k-th exact key tau
                // cannot enter.  Batches of the 32 live candidates of least
                // approximate value get canonical distances and merge into the
                // row, which lowers tau; the rest are pruned against it; when
                // at most 32 remain they are evaluated at once.  The row ends
                // as the k best of its list and every candidate, the FP32
                // form's result.
                const uint64_t kth0 = lane_key(old[0], k - 1);
                float tau = kth0 == kEmptyKey ? __int_as_float(0x7f800000) : key_dist(kth0);
                float lbv[NC];
                uint64_t apx[NC];
                bool alive[NC];
#pragma unroll
                for (int s = 0; s < NC; ++s) {
                    const int c = lane + 32 * s;
                    const bool valid = c < m && c != R;
                    apx[s] = kEmptyKey;
                    lbv[s] = __int_as_float(0x7f800000);
                    if (valid) {
                        const float av = dt[rd * DTS + c];
                        apx[s] = make_key(__fadd_rn(av, 0.f), (uint32_t)sid[c]);
                        const float sn = __fadd_ru(srt[R], srt[c]);
                        const float eps =
                            __fadd_ru(__fmul_ru(cD, __fmul_ru(sn, sn)), __fmul_ru(1.1920928955078125e-7f, fabsf(av)));
                        const float lo = __fsub_rd(av, eps);
                        float lb = 0.f;
                        if (lo > 0.f) {
                            const float root = __fsub_rd(__fsub_rd(__fsqrt_rd(lo), serr[R]), serr[c]);
                            if (root > 0.f) lb = __fmul_rd(root, root);
                        }
                        lbv[s] = lb;
                    }
                    alive[s] = valid && lbv[s] <= tau;
                }
                uint64_t list = old[0];
                int batches = 0;
                for (int it = 0; it <= NC; ++it) {
                    unsigned bal[NC];
                    int total = 0;
#pragma unroll
                    for (int s = 0; s < NC; ++s) {
                        bal[s] = __ballot_sync(0xffffffffu, alive[s]);
                        total += __popc(bal[s]);
                    }
                    if (total == 0) break;
                    // into an empty list the first batch is k wide (its k-th
                    // exact key is the first finite tau); later batches 32
                    const int B = (it == 0 && kth0 == kEmptyKey) ? k : 32;
                    uint64_t pick = kEmptyKey;  // this lane's candidate of the batch
                    if (total <= B) {
                        int at = 0;
#pragma unroll
                        for (int s = 0; s < NC; ++s) {
                            if (alive[s]) wscratch[at + __popc(bal[s] & ((1u << lane) - 1u))] = apx[s];
                            at += __popc(bal[s]);
                        }
                        __syncwarp();
                        pick = lane < total ? wscratch[lane] : kEmptyKey;
                        __syncwarp();
                    } else {
                        uint64_t tmp[NC], top[1];
#pragma unroll
                        for (int s = 0; s < NC; ++s) tmp[s] = alive[s] ? apx[s] : kEmptyKey;
                        sort_regs<NC>(tmp);
                        warp_select_unique<NC, 1>(tmp, B, top);
                        pick = top[0];
                    }
                    const uint64_t last = lane_key(pick, B - 1);  // the batch's largest key (lanes below B hold one)
                    uint64_t one[1] = {kEmptyKey};
                    if (pick != kEmptyKey) {
                        const uint32_t cid = key_id(pick);
                        one[0] = make_key(canon_dist(X + (int64_t)gi * D, X + (int64_t)cid * D, D, vec), cid);
                    }
                    uint64_t out;
                    bool changed;
                    if (!warp_merge_few<1>(one, list, k, wscratch, out, changed)) {
                        uint64_t both[2] = {one[0], list};
                        uint64_t res1[1];
                        sort_regs<2>(both);
                        warp_select_unique<2, 1>(both, k, res1);
                        out = res1[0];
                    }
                    list = lane < k ? out : kEmptyKey;
                    ++batches;
                    if (total <= B) break;
                    const uint64_t kth = lane_key(list, k - 1);
                    if (kth != kEmptyKey) tau = key_dist(kth);
#pragma unroll
                    for (int s = 0; s < NC; ++s) alive[s] = alive[s] && apx[s] > last && lbv[s] <= tau;
                }
                if (batches > (kth0 == kEmptyKey ? 2 : 1) && lane == 0)
                    atomicAdd(status + 1, 1);  // rows the approximate order did not settle at once
                if (__any_sync(0xffffffffu, list != old[0]) && lane < k) grow[lane] = list;
                continue;
            }
            // the kp + 1 best approximate candidates (keys unique: distinct ids)
            uint64_t apx[NC];
#pragma unroll
            for (int s = 0; s < NC; ++s) {
                const int c = lane + 32 * s;
                apx[s] = (c < m && c != R) ? make_key(__fadd_rn(dt[rd * DTS + c], 0.f), (uint32_t)sid[c])
                                           : kEmptyKey;
            }
            sort_regs<NC>(apx);
            uint64_t top[2];
            const int want = kp + 1 < m - 1 ? kp + 1 : m - 1;
            warp_select_unique<NC, 2>(apx, want, top);
            const int nre = want < kp ? want : kp;  // re-ranked candidates
            // canonical distances of the re-ranked ones; excluded: from rank kp on
            uint64_t ex[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int j = lane + 32 * s;
                ex[s] = kEmptyKey;
                if (j < nre) {
                    const uint32_t cid = key_id(top[s]);
                    const float d = canon_dist(X + (int64_t)gi * D, X + (int64_t)cid * D, D, vec);
                    ex[s] = make_key(d, cid);
                }
            }
            uint64_t merged[2 + NSG];
            merged[0] = ex[0];
            merged[1] = ex[1];
#pragma unroll
            for (int s = 0; s < NSG; ++s) merged[2 + s] = old[s];
            sort_regs<2 + NSG>(merged);
            warp_select_unique<2 + NSG, NSG>(merged, k, res);
            if (want <= kp) {
                done_row = true;  // nothing excluded
            } else {
                const uint64_t astar_key = list_at<2>(top, kp);
                const uint64_t tau_key = list_at<NSG>(res, k - 1);
                if (tau_key != kEmptyKey) {
                    const double astar = (double)key_dist(astar_key);
                    const double tau = (double)key_dist(tau_key);
                    const double ni = sqrt((double)snrm[R]);
                    const double eps = (double)cD * (ni + smax[0]) * (ni + smax[0]) + 1.1920928955078125e-7 * fabs(astar);
                    const double lo = astar - eps;
                    double root = lo > 0.0 ? sqrt(lo) : 0.0;
                    root -= (double)serr[R] + (double)smax[1];
                    const double lower = root > 0.0 ? root * root : 0.0;
                    done_row = lower * (1.0 - 1e-12) > tau;
                }
            }
        }
        if (!done_row) {
            // not certified: exact distances to the whole leaf
            uint64_t cand[NC + NSG];
#pragma unroll
            for (int s = 0; s < NC; ++s) {
                const int c = lane + 32 * s;
                cand[s] = kEmptyKey;
                if (c < m && c != R)
                    cand[s] = make_key(canon_dist(X + (int64_t)gi * D, X + (int64_t)sid[c] * D, D, vec),
                                       (uint32_t)sid[c]);
            }
#pragma unroll
            for (int s = 0; s < NSG; ++s) cand[NC + s] = old[s];
            sort_regs<NC + NSG>(cand);
            warp_select_unique<NC + NSG, NSG>(cand, k, res);
            if (lane == 0) atomicAdd(status + 1, 1);  // fallback counter (statistics)
        }
#pragma unroll
        for (int s = 0; s < NSG; ++s)
            if (lane + 32 * s < k) grow[lane + 32 * s] = res[s];
    }
    __syncthreads();  // the next phase's d^ rows overwrite dt
    }
}

// The values held by a low-precision copy as FP32, m x D: the 16-bit values
// themselves, or the unscaled E4M3 values q (a parity hook's output).
__global__ void k_lp_to_float(const uint8_t* __restrict__ Xq, int64_t m, int D, int row_bytes, int qt,
                              float* __restrict__ out) {
    const int64_t total = m * D;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / D;
        const int d = (int)(e - r * D);
        const uint8_t* row = Xq + r * row_bytes;
        float v;
        if (qt == 2) {
            v = __half2float(__half(__nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)row[d], __NV_E4M3)));
        } else {
            const uint16_t h = reinterpret_cast<const uint16_t*>(row)[d];
            v = qt == 1 ? __bfloat162float(__ushort_as_bfloat16(h)) : __half2float(__ushort_as_half(h));
        }
        out[e] = v;
    }
}

// ---------------------------------------------------------------- host
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

}  // namespace

int lp_dim(int D) { return (D + kTcK - 1) / kTcK * kTcK; }

int lp_row_bytes(int D, int qt) { return qt == 2 ? (D + kRowChunk - 1) / kRowChunk * kRowChunk : 2 * lp_dim(D); }

float lp_cert_coeff(int D, int qt) {
    const int Dp = qt == 2 ? lp_row_bytes(D, qt) : lp_dim(D);
    const double c16 = (16.0 * Dp + 8.0) * 5.9604644775390625e-8;  // 2^-24
    const double c8 = qt == 2 ? Dp * 1.220703125e-4 : 0.0;          // 2^-13: the FP8 accumulation assumption
    return (float)((c16 + c8) * (1.0 + 1e-6));
}

void launch_quantize(const float* X, int64_t n, int D, const int32_t* perm, int qt, void* Xq, float* nrm,
                     float* qerr, float* scale, int* notexact, cudaStream_t s) {
    const int Dpb = lp_row_bytes(D, qt);
    const int grid = (int)((n * 32 + 255) / 256);
    if (qt == 2) {
        LaunchScope ls("k0_quantize", s, (double)n * (D * 4.0 + Dpb + 12.0), 0);
        k0_quantize_e4m3<<<grid, 256, 0, s>>>(X, n, D, Dpb, perm, static_cast<uint8_t*>(Xq), nrm, qerr, scale,
                                              notexact);
        return;
    }
    const int Dp = lp_dim(D);
    LaunchScope ls("k0_quantize", s, (double)n * (D * 4.0 + Dp * 2.0 + 8.0), 0);
    if (qt == 1)
        k0_quantize<true><<<grid, 256, 0, s>>>(X, n, D, Dp, perm, static_cast<uint16_t*>(Xq), nrm, qerr, notexact);
    else
        k0_quantize<false><<<grid, 256, 0, s>>>(X, n, D, Dp, perm, static_cast<uint16_t*>(Xq), nrm, qerr, notexact);
}

void launch_permute16(const void* Xq, const float* nrm, const float* qerr, const float* scale, int64_t n,
                      int row_bytes, const int32_t* perm, void* Xl, float* lnrm, float* lerr, float* lscale,
                      cudaStream_t s) {
    const int q = row_bytes / 16;
    LaunchScope ls("k0_permute16", s, (double)n * (row_bytes * 2.0 + (scale ? 24.0 : 16.0)), 0);
    int64_t g = (n * q + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    k0_permute16<<<(int)g, 256, 0, s>>>(static_cast<const uint4*>(Xq), nrm, qerr, scale, n, q, perm,
                                        static_cast<uint4*>(Xl), lnrm, lerr, lscale);
}

void launch_lp_to_float(const void* Xq, int64_t m, int D, int qt, float* out, cudaStream_t s) {
    LaunchScope ls("k_lp_to_float", s, (double)m * (lp_row_bytes(D, qt) + D * 4.0), 0);
    int64_t g = (m * D + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    k_lp_to_float<<<(int)(g < 1 ? 1 : g), 256, 0, s>>>(static_cast<const uint8_t*>(Xq), m, D, lp_row_bytes(D, qt), qt,
                                                       out);
}

bool launch_leaf_tc(const void* Xl, int64_t n, const float* X, int D, const int32_t* perm,
                    const int32_t* leaf_off, int nleaf, int max_leaf, const float* nrm, const float* qerr,
                    const float* scale, int k, int kp, int qt, uint64_t* G, int* status, const int* notexact,
                    cudaStream_t s, float* dump) {
    if (max_leaf > 2 * kTcRows) return false;
    const int MT = max_leaf > kTcRows ? 2 : 1;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const int Dpb = lp_row_bytes(D, qt);
    CUtensorMap tmap;
    const cuuint64_t gdim[2] = {(cuuint64_t)(qt == 2 ? Dpb : Dpb / 2), (cuuint64_t)n};
    const cuuint64_t gstride[1] = {(cuuint64_t)Dpb};
    const cuuint32_t box[2] = {(cuuint32_t)(qt == 2 ? kRowChunk : kTcK), (cuuint32_t)kTcRows};
    const cuuint32_t estride[2] = {1, 1};
    const CUtensorMapDataType dtype = qt == 2   ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                      : qt == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    if (enc(&tmap, dtype, 2, const_cast<void*>(Xl), gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const TcSmem L = tc_smem(Dpb, MT);
    const size_t smem = L.total + 1024;
    if (smem > 227 * 1024) return false;
    const float cD = lp_cert_coeff(D, qt);
    const double mm = (double)max_leaf, rw = 128.0 * MT;
    const double elems = qt == 2 ? Dpb : Dpb / 2;
    static const char* names[3] = {"k2_leaf_fp16", "k2_leaf_bf16", "k2_leaf_fp8"};
    LaunchScope ls(names[qt], s, (double)nleaf * mm * (Dpb + 2 * 8.0 * k), (double)nleaf * rw * rw * 2.0 * elems);
#define KNNG_LEAF_TC(Q, NS, T)                                                                                  \
    do {                                                                                                        \
        cudaFuncSetAttribute(k2_leaf_tc<Q, NS, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);     \
        k2_leaf_tc<Q, NS, T><<<nleaf * T, kTcThreads, smem, s>>>(tmap, Dpb, cD, X, D, perm, leaf_off, nrm,   \
                                                             qerr, scale, k, kp, G, status, notexact, dump);    \
    } while (0)
#define KNNG_LEAF_TC_K(Q, T)               \
    do {                                   \
        if (k > 32) KNNG_LEAF_TC(Q, 2, T); \
        else KNNG_LEAF_TC(Q, 1, T);        \
    } while (0)
#define KNNG_LEAF_TC_T(Q)                 \
    do {                                  \
        if (MT == 2) KNNG_LEAF_TC_K(Q, 2); \
        else KNNG_LEAF_TC_K(Q, 1);         \
    } while (0)
    if (qt == 2) KNNG_LEAF_TC_T(2);
    else if (qt == 1) KNNG_LEAF_TC_T(1);
    else KNNG_LEAF_TC_T(0);
#undef KNNG_LEAF_TC_T
#undef KNNG_LEAF_TC_K
#undef KNNG_LEAF_TC
    return true;
}

}  // namespace knng
