// exact.cu -- K7: the exact k nearest neighbours of sampled rows (the
// problem statement of Sec. 1, each sampled point as a query against the
// other n - 1), canonical FP32 distances, ties by id; recall of a graph on
// those rows; and the input check.
#include "common.cuh"
#include "kernels.h"

namespace knng {

namespace {

constexpr int kQR = 64;    // query rows per CTA
constexpr int kCT = 128;   // points per column tile
constexpr int kNT = 256;

__host__ __device__ inline void exact_chunk(int D, int* dch, int* stride) {
    const int d4 = (D + 3) & ~3;
    const int cap = (100 * 1024 / ((kQR + kCT) * 4) - 4) & ~3;
    const int c = d4 < cap ? d4 : cap;
    *dch = c;
    *stride = ((c / 4) & 1) ? c : c + 4;
}

template <int NO>
__global__ void __launch_bounds__(kNT) k7_exact(const float* __restrict__ X, int64_t n, int D, int k,
                                               const int32_t* __restrict__ sample, int64_t s_rows,
                                               uint64_t* __restrict__ out, const int* __restrict__ status) {
    if (*status & kStatusStop) return;  // a sampled id failed its check
    extern __shared__ float4 smem4[];
    int dch, stride;
    exact_chunk(D, &dch, &stride);
    float* qs = reinterpret_cast<float*>(smem4);       // [kQR][stride]
    float* cs = qs + kQR * stride;                     // [kCT][stride]
    float* dt = cs + kCT * stride;                     // [kQR][kCT + 1]
    int64_t* qid = reinterpret_cast<int64_t*>(dt + kQR * (kCT + 1));  // [kQR]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rg = tid % 16, cg = tid / 16;
    const int64_t q0 = (int64_t)blockIdx.x * kQR;
    const int nq = (int)min((int64_t)kQR, s_rows - q0);
    for (int r = tid; r < kQR; r += kNT) qid[r] = r < nq ? (sample ? (int64_t)sample[q0 + r] : q0 + r) : -1;
    __syncthreads();
    const bool one_chunk = dch >= D;
    auto load_rows = [&](float* dst, int rows, int64_t first, bool query, int d0) {
        const int dl = min(dch, D - d0);
        for (int e = tid; e < rows * dch; e += kNT) {
            const int r = e / dch, dd = e - r * dch;
            const int64_t row = query ? qid[r] : first + r;
            float v = 0.f;
            if (row >= 0 && row < n && dd < dl) v = __ldg(X + row * D + d0 + dd);
            dst[r * stride + dd] = v;
        }
    };
    if (one_chunk) load_rows(qs, kQR, 0, true, 0);
    uint64_t run[8][NO];
#pragma unroll
    for (int rr = 0; rr < 8; ++rr)
#pragma unroll
        for (int o = 0; o < NO; ++o) run[rr][o] = kEmptyKey;

    for (int64_t c0 = 0; c0 < n; c0 += kCT) {
        float acc[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
        for (int d0 = 0; d0 < D; d0 += dch) {
            __syncthreads();
            if (!one_chunk) load_rows(qs, kQR, 0, true, d0);
            load_rows(cs, kCT, c0, false, d0);
            __syncthreads();
            const float* rp = qs + rg * stride;
            const float* cp = cs + cg * stride;
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
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) dt[(rg + 16 * i) * (kCT + 1) + cg + 16 * j] = acc[i][j];
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
            const int r = warp * 8 + rr;
            if (r >= nq) continue;
            uint64_t a[4 + NO];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int64_t col = c0 + lane + 32 * s;
                a[s] = (col < n && col != qid[r]) ? make_key(dt[r * (kCT + 1) + lane + 32 * s], (uint32_t)col)
                                                  : kEmptyKey;
            }
            uint64_t mine = run[rr][0];
#pragma unroll
            for (int o = 1; o < NO; ++o)
                if (o == ((k - 1) >> 5)) mine = run[rr][o];
            const uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)mine, (k - 1) & 31);
            const uint32_t hi = __shfl_sync(0xffffffffu, (uint32_t)(mine >> 32), (k - 1) & 31);
            const uint64_t last = ((uint64_t)hi << 32) | lo;
            bool any = false;
#pragma unroll
            for (int s = 0; s < 4; ++s) any |= a[s] < last;
            if (!__any_sync(0xffffffffu, any)) continue;
#pragma unroll
            for (int o = 0; o < NO; ++o) a[4 + o] = run[rr][o];
            sort_regs<4 + NO>(a);
            warp_select_unique<4 + NO, NO>(a, k, run[rr]);
        }
    }
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) {
        const int r = warp * 8 + rr;
        if (r >= nq) continue;
#pragma unroll
        for (int o = 0; o < NO; ++o)
            if (lane + 32 * o < k) out[(q0 + r) * k + lane + 32 * o] = run[rr][o];
    }
}

__global__ void k_recall(const int32_t* __restrict__ ids, const float* __restrict__ d,
                         const int32_t* __restrict__ gt_ids, const float* __restrict__ gt_d,
                         const int32_t* __restrict__ sample, int64_t s_rows, int k,
                         unsigned long long* __restrict__ counts) {
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= s_rows) return;
    const int lane = threadIdx.x & 31;
    const int64_t i = sample[r];
    const float kth = gt_d[r * k + k - 1];
    int hit = 0, tie = 0;
    for (int e = lane; e < k; e += 32) {
        const int32_t g = ids[i * k + e];
        if (g < 0) continue;
        for (int b = 0; b < k; ++b)
            if (gt_ids[r * k + b] == g) {
                ++hit;
                break;
            }
        tie += d[i * k + e] <= kth;
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        hit += __shfl_xor_sync(0xffffffffu, hit, m);
        tie += __shfl_xor_sync(0xffffffffu, tie, m);
    }
    if (lane == 0) {
        atomicAdd(&counts[0], (unsigned long long)hit);
        atomicAdd(&counts[1], (unsigned long long)tie);
    }
}

__global__ void k_check_finite(const float4* __restrict__ X4, int64_t n4, const float* __restrict__ tail,
                               int ntail, int* __restrict__ status) {
    bool bad = false;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n4; e += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = __ldg(X4 + e);
        bad |= !isfinite(v.x) | !isfinite(v.y) | !isfinite(v.z) | !isfinite(v.w);
    }
    if (blockIdx.x == 0 && threadIdx.x < ntail) bad |= !isfinite(tail[threadIdx.x]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStatusNonFinite);
}

}  // namespace

void launch_exact(const float* X, int64_t n, int D, int k, const int32_t* sample, int64_t s_rows, uint64_t* out,
                  const int* status, cudaStream_t s) {
    int dch, stride;
    exact_chunk(D, &dch, &stride);
    const size_t smem = (size_t)(kQR + kCT) * stride * 4 + (size_t)kQR * (kCT + 1) * 4 + kQR * 8;
    const int grid = (int)((s_rows + kQR - 1) / kQR);
    LaunchScope ls("k7_exact", s, (double)grid * n * D * 4.0, (double)s_rows * n * 3.0 * D);
    if (k > 32) {
        cudaFuncSetAttribute(k7_exact<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k7_exact<2><<<grid, kNT, smem, s>>>(X, n, D, k, sample, s_rows, out, status);
    } else {
        cudaFuncSetAttribute(k7_exact<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k7_exact<1><<<grid, kNT, smem, s>>>(X, n, D, k, sample, s_rows, out, status);
    }
}

void launch_recall(const int32_t* ids, const float* d, const int32_t* gt_ids, const float* gt_d,
                   const int32_t* sample, int64_t s_rows, int k, unsigned long long* counts, cudaStream_t s) {
    LaunchScope ls("k_recall", s, (double)s_rows * k * 16.0, 0);
    cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), s);
    if (s_rows == 0) return;
    const int grid = (int)((s_rows * 32 + 255) / 256);
    k_recall<<<grid, 256, 0, s>>>(ids, d, gt_ids, gt_d, sample, s_rows, k, counts);
}

void launch_check_finite(const float* X, int64_t count, int* status, cudaStream_t s) {
    // X may start at any 4-byte boundary: handle the head up to 16 B alignment
    // and the tail with scalar loads
    const uintptr_t addr = reinterpret_cast<uintptr_t>(X);
    const int64_t head = (int64_t)(((16 - (addr & 15)) & 15) / 4);
    const int64_t h = head < count ? head : count;
    LaunchScope ls("k0_check_finite", s, count * 4.0, 0, h > 0 ? 2 : 1);
    if (h > 0) k_check_finite<<<1, 32, 0, s>>>(nullptr, 0, X, (int)h, status);
    const int64_t rest = count - h;
    const int64_t n4 = rest / 4;
    const int ntail = (int)(rest - n4 * 4);
    const int grid = (int)((n4 + 255) / 256 < 152 * 8 ? (n4 + 255) / 256 : 152 * 8);
    k_check_finite<<<grid < 1 ? 1 : grid, 256, 0, s>>>(reinterpret_cast<const float4*>(X + h), n4,
                                                       X + h + n4 * 4, ntail, status);
}

}  // namespace knng
