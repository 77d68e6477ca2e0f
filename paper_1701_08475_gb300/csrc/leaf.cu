// leaf.cu -- K2f: exhaustive comparison inside each cluster (Alg. 1: for
// every pair <i, j>, i != j, of a cluster, update G[i] and G[j] with
// d(x_i, x_j)), in canonical FP32, fused with the merge into the graph.
//
// One CTA per leaf (m <= MC points).  The leaf's rows sit in shared memory
// (DCH dims at a time); each thread accumulates a 4 x 8 block of pairs, dims
// ascending with fmaf, so every distance has the canonical bits.  A row
// block of distances goes to shared memory, and one warp per row selects the
// row's k best of (its G row) + (the leaf) with duplicates merged.  No
// distance matrix reaches HBM; G is updated in place (a point lives in one
// leaf per pass).
#include "common.cuh"
#include "kernels.h"

namespace knng {

namespace {

template <int MC>
struct LeafCfg {
    static constexpr int RB = (MC < 8192 / MC) ? MC : 8192 / MC;  // rows per block
    static constexpr int NT = RB * MC / 32;                        // threads
    static constexpr int RG = RB / 4;                              // row groups
    static constexpr int CG = MC / 8;                              // col groups
};

// dims per chunk and padded stride (stride / 4 odd: conflict-free float4 rows)
__host__ __device__ inline void leaf_chunk(int D, int MC, int* dch, int* stride) {
    const int d4 = (D + 3) & ~3;
    int cap = (72 * 1024 / (MC * 4) - 4) & ~3;
    int c = d4 < cap ? d4 : cap;
    *dch = c;
    *stride = ((c / 4) & 1) ? c : c + 4;
}

template <int MC, int NSG>
__global__ void __launch_bounds__(LeafCfg<MC>::NT) k2_leaf_fp32(const float* __restrict__ X, int D,
                                                                 const int32_t* __restrict__ perm,
                                                                 const int32_t* __restrict__ leaf_off, int k,
                                                                 uint64_t* __restrict__ G,
                                                                 const int* __restrict__ status) {
    using C = LeafCfg<MC>;
    if (*status & kStatusStop) return;  // ids or offsets failed their check
    constexpr int NS = MC / 32 + NSG;
    extern __shared__ float4 smem4[];
    int dch, stride;
    leaf_chunk(D, MC, &dch, &stride);
    float* xs = reinterpret_cast<float*>(smem4);          // [MC][stride]
    float* dt = xs + MC * stride;                          // [RB][MC + 1]
    int32_t* ids = reinterpret_cast<int32_t*>(dt + C::RB * (MC + 1));  // [MC]
    uint64_t* wscratch = reinterpret_cast<uint64_t*>(ids + MC) + (threadIdx.x >> 5) * 32;  // 32 keys per warp

    const int leaf = blockIdx.x;
    const int a = leaf_off[leaf];
    const int m = leaf_off[leaf + 1] - a;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rg = tid % C::RG, cg = tid / C::RG;
    for (int r = tid; r < MC; r += C::NT) ids[r] = r < m ? perm[a + r] : 0;
    __syncthreads();

    const bool one_chunk = dch >= D;
    auto load_chunk = [&](int d0) {
        const int dl = min(dch, D - d0);
        for (int e = tid; e < MC * dch; e += C::NT) {
            const int r = e / dch, dd = e - r * dch;
            float v = 0.f;
            if (r < m && dd < dl) v = __ldg(X + (int64_t)ids[r] * D + d0 + dd);
            xs[r * stride + dd] = v;
        }
    };
    if (one_chunk) {
        load_chunk(0);
        __syncthreads();
    }

    for (int rb = 0; rb * C::RB < m; ++rb) {
        float acc[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
        for (int d0 = 0; d0 < D; d0 += dch) {
            if (!one_chunk) {
                __syncthreads();
                load_chunk(d0);
                __syncthreads();
            }
            const float* rp = xs + (rb * C::RB + rg) * stride;
            const float* cp = xs + cg * stride;
            for (int dq = 0; dq < dch; dq += 4) {
                float4 rv[4], cv[8];
#pragma unroll
                for (int i = 0; i < 4; ++i) rv[i] = *reinterpret_cast<const float4*>(rp + i * C::RG * stride + dq);
#pragma unroll
                for (int j = 0; j < 8; ++j) cv[j] = *reinterpret_cast<const float4*>(cp + j * C::CG * stride + dq);
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
        __syncthreads();  // previous selection done with dt
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) dt[(rg + i * C::RG) * (MC + 1) + cg + j * C::CG] = acc[i][j];
        __syncthreads();
        // one warp per row: k best of G[i] + leaf candidates
        for (int r = warp; r < C::RB; r += C::NT / 32) {
            const int row = rb * C::RB + r;
            if (row >= m) break;
            const int gi = ids[row];
            uint64_t* grow = G + (int64_t)gi * k;
            uint64_t cand[NS];
#pragma unroll
            for (int s = 0; s < MC / 32; ++s) {
                const int c = lane + 32 * s;
                cand[s] = (c < m && c != row) ? make_key(dt[r * (MC + 1) + c], (uint32_t)ids[c]) : kEmptyKey;
            }
            if (NSG == 1) {
                // few candidates beat the row's k-th entry after the first pass
                uint64_t few[MC / 32], out;
                bool changed;
#pragma unroll
                for (int s = 0; s < MC / 32; ++s) few[s] = cand[s];
                const uint64_t cur = lane < k ? grow[lane] : kEmptyKey;
                if (warp_merge_few<MC / 32>(few, cur, k, wscratch, out, changed)) {
                    if (changed && lane < k) grow[lane] = out;
                    continue;
                }
                // many survive (the first pass): the lanes' smallest first
#pragma unroll
                for (int s = 0; s < MC / 32; ++s) few[s] = cand[s];
                if (warp_merge_many<MC / 32>(few, cur, k, wscratch, out, changed)) {  // MC >= 64
                    if (changed && lane < k) grow[lane] = out;
                    continue;
                }
            }
#pragma unroll
            for (int s = 0; s < NSG; ++s) {
                const int e = lane + 32 * s;
                cand[MC / 32 + s] = e < k ? grow[e] : kEmptyKey;
            }
            sort_regs<NS>(cand);
            uint64_t out[NSG];
            warp_select_unique<NS, NSG>(cand, k, out);
#pragma unroll
            for (int s = 0; s < NSG; ++s) {
                const int e = lane + 32 * s;
                if (e < k) grow[e] = out[s];
            }
        }
    }
}

template <int MC, int NSG>
void launch_leaf_t(const float* X, int D, const int32_t* perm, const int32_t* leaf_off, int nleaf, int k,
                   uint64_t* G, const int* status, cudaStream_t s) {
    using C = LeafCfg<MC>;
    int dch, stride;
    leaf_chunk(D, MC, &dch, &stride);
    const size_t smem = (size_t)MC * stride * 4 + (size_t)C::RB * (MC + 1) * 4 + MC * 4 + (C::NT / 32) * 32 * 8;
    cudaFuncSetAttribute(k2_leaf_fp32<MC, NSG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k2_leaf_fp32<MC, NSG><<<nleaf, C::NT, smem, s>>>(X, D, perm, leaf_off, k, G, status);
}

}  // namespace

void launch_leaf_fp32(const float* X, int D, const int32_t* perm, const int32_t* leaf_off, int nleaf,
                      int max_leaf, int k, uint64_t* G, const int* status, cudaStream_t s) {
    // algorithmic work: every leaf row once, every ordered pair once
    const double mm = (double)max_leaf;
    LaunchScope ls("k2_leaf_fp32", s, (double)nleaf * mm * (D * 4.0 + 2 * 8.0 * k),
                   (double)nleaf * mm * (mm - 1) * 3.0 * D);
    const bool two = k > 32;
    if (max_leaf <= 64) {
        if (two) launch_leaf_t<64, 2>(X, D, perm, leaf_off, nleaf, k, G, status, s);
        else launch_leaf_t<64, 1>(X, D, perm, leaf_off, nleaf, k, G, status, s);
    } else if (max_leaf <= 128) {
        if (two) launch_leaf_t<128, 2>(X, D, perm, leaf_off, nleaf, k, G, status, s);
        else launch_leaf_t<128, 1>(X, D, perm, leaf_off, nleaf, k, G, status, s);
    } else {
        if (two) launch_leaf_t<256, 2>(X, D, perm, leaf_off, nleaf, k, G, status, s);
        else launch_leaf_t<256, 1>(X, D, perm, leaf_off, nleaf, k, G, status, s);
    }
}

}  // namespace knng
