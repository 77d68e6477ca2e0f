// join_tc.cu -- the local join (neighbour-of-neighbour refinement, the prior
// art cited in Sec. 1) with the member Gram matrices on tcgen05 tensor cores.
//
// Used when the 16-bit copy makes the arithmetic exact (all values integers
// the 16-bit type holds, every squared norm and distance an integer below
// 2^24): then ||x_u||^2 + ||x_v||^2 - 2 x_u . x_v computed from the tensor
// cores' FP32 accumulator is the canonical distance itself, bit for bit.
// Otherwise the kernel returns at once and the FP32 join (join.cu), launched
// beside it, does the round; the choice is made on the device, so neither
// needs the host to look at the data.
//
// One CTA packs NPC nodes: node j's members N_i = G_old[i] (+ R[i]) occupy
// tile rows j * mcap .. j * mcap + M_j - 1.  Their 16-bit rows are gathered
// into the 128-byte-swizzled K-major layout with cp.async, one thread issues
// the 128 x 128 x Dp Gram on the tensor cores, and in the epilogue each
// node's 2 mcap threads evaluate its pairs.  A node with many pairs goes by
// rows: the two threads of tile row r (= tensor-memory lane r, member s of
// node j) decide the offers to that member, from every other member (quads of
// members alternately; an old member takes the new ones only), with the
// member's k-th entry in a register and one count per target.  A node with
// few pairs (few new members) deals its pairs {u, v} round-robin to its
// threads instead, each pair decided in both directions.
//
// Inside a CTA the groups overlap where they can: the members' thresholds,
// norms and leaf ids travel on cp.async beside the gather and are awaited only
// before the epilogue, and the member lists are double-buffered so that the
// next group's collection runs while this group's offer slots are fetched.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace knng {

namespace {

constexpr int kRows = 128;
constexpr int kKc = 64;                  // 16-bit elements per swizzled row
constexpr int kChunkBytes = kRows * kKc * 2;
constexpr int kThreads = 256;  // two threads per tile row in the epilogue
constexpr int kResident = 4;   // chunks of a row (64 16-bit dims each) held at once
constexpr int kRing = 2;       // chunk buffers for wider rows

__device__ __forceinline__ bool lp_exact_flag(int f) { return (f & 1) == 0 && !((f & 2) && (f & 4)); }

// Row stride (floats) of the Gram rows in shared memory: mcap + 4 is 4 mod 8
// (mcap is a multiple of 8), so the 16-byte accesses of any 8 consecutive
// rows fall in distinct bank quads.
__host__ __device__ __forceinline__ int priv_stride(int mcap) { return mcap + 4; }

// The operand tile, reused after the product for the Gram rows (priv[r][t]:
// row r's entry for member t of its node, row stride priv_stride(mcap); an
// entry that makes an offer is overwritten with the offer's distance); then
// member ids, thresholds, norms, errors and rounded-up norm roots, counts, the
// barrier, the slot.
struct JtSmem {
    size_t tile, priv, mem, thr, nrm, err, srt, lid, cnt, bar, slot, total;
};
__host__ __device__ inline JtSmem jt_smem(int Dp, int mcap, bool cert) {
    JtSmem L;
    L.tile = 0;
    L.priv = 0;  // the operand tile is dead once the MMA has completed
    // rows of up to kResident chunks stay whole in shared memory; wider rows
    // stream through a ring of kRing chunk buffers
    const int nk = Dp / kKc;
    const size_t tile = (size_t)(nk <= kResident ? nk : kRing) * kChunkBytes,
                 pv = (size_t)priv_stride(mcap) * kRows * 4;
    L.mem = tile > pv ? tile : pv;
    L.thr = L.mem + 2 * kRows * 4;  // two member buffers: this group's and the next one's
    L.nrm = L.thr + kRows * 8;
    L.err = L.nrm + kRows * 4;
    L.srt = L.err + (cert ? kRows * 4 : 0);
    L.lid = L.srt + (cert ? kRows * 4 : 0);
    L.cnt = L.lid + kRows * 16;
    L.bar = L.cnt + 2 * 32 * 4;  // member counts, then new-member counts (two buffers)
    L.slot = L.bar + 8 * (1 + kRing);  // the product's barrier, then one per ring buffer
    L.total = L.slot + 8;
    return L;
}

// Flat enumeration of the pairs of a node whose members are nn new ones
// (indices 0 .. nn-1) followed by no old ones.  p < nn * no is the new x old
// pair (p / no, nn + p % no); then the new x new pairs {a, a + 1 + c mod nn}
// for c < (nn - 1) / 2, row by row; then, for even nn, {a, a + nn / 2} with
// a < nn / 2.  Every unordered pair with a new member appears once.
__device__ __forceinline__ int small_div(int p, int d, float rd) {
    // p < 2^15, d <= 128: the estimate is off by at most one
    int q = __float2int_rz((float)p * rd);
    const int rem = p - q * d;
    if (rem < 0) --q;
    else if (rem >= d) ++q;
    return q;
}
struct PairMap {
    int nn, no, H, PO, PC;
    float rno, rH;
    __device__ __forceinline__ void decode(int p, int& a, int& b) const {
        if (p < PO) {
            a = small_div(p, no, rno);
            b = nn + (p - a * no);
        } else if (p - PO < PC) {
            const int q = p - PO;
            a = small_div(q, H, rH);
            const int t = a + 1 + (q - a * H);
            b = t >= nn ? t - nn : t;
        } else {
            a = p - PO - PC;
            b = a + nn / 2;
        }
    }
};
__device__ __forceinline__ PairMap pair_map(int nn, int no) {
    PairMap m;
    m.nn = nn;
    m.no = no;
    m.H = nn > 0 ? (nn - 1) / 2 : 0;
    m.PO = nn * no;
    m.PC = nn * m.H;
    m.rno = no > 0 ? 1.f / (float)no : 0.f;
    m.rH = m.H > 0 ? 1.f / (float)m.H : 0.f;
    return m;
}

// Persistent: CTA b takes node groups b, b + gridDim.x, ...; tensor memory
// and the barrier are set up once.
//
// CERT (the 16-bit copy is not exact): d^ from the Gram only decides which
// pairs need their canonical distance.  With the leaf certificate's bound,
// rounded so that it stays a lower bound, d >= (sqrt(d^ - eps) - e_a - e_b)^2;
// a direction whose target's k-th entry is below that cannot be offered.
// Every other pair gets its canonical FP32 distance from X, and the offers
// are decided on exact keys: the same offers as the FP32 join.
template <bool CERT>
__global__ void __launch_bounds__(kThreads, 4) k5_join_tc(const uint16_t* __restrict__ Xq, int Dp,
                                                         const float* __restrict__ nrm, int k, int rev, int mcap,
                                                         int npc, const uint64_t* __restrict__ Gold,
                                                         const uint64_t* __restrict__ R,
                                                         const int32_t* __restrict__ list,
                                                         const uint64_t* __restrict__ fnew,
                                                         const uint64_t* __restrict__ rnew, int64_t node0,
                                                         int64_t node1, uint32_t* __restrict__ counter, int64_t cap,
                                                         uint32_t* __restrict__ ptgt, uint64_t* __restrict__ pkey,
                                                         int32_t* __restrict__ pcnt, int* __restrict__ status,
                                                         const int* __restrict__ notexact, bool bf16,
                                                         const float* __restrict__ X, int D,
                                                         const float* __restrict__ qerr,
                                                         const int32_t* __restrict__ count_dev,
                                                         const int32_t* __restrict__ leafid, int npass,
                                                         int32_t* __restrict__ ovf_list,
                                                         int32_t* __restrict__ ovf_count) {
    extern __shared__ uint8_t smem_raw[];
    // the exact form runs when the 16-bit copy is exact, the screening form
    // (CERT) when it is not; each returns at once otherwise
    if ((*status & kStatusStop) || (CERT == lp_exact_flag(*notexact))) return;
    if (count_dev && (int64_t)*count_dev < node1) node1 = *count_dev;
    const JtSmem L = jt_smem(Dp, mcap, CERT);
    uint8_t* base = smem_raw + ((1024 - (tc::smem_addr(smem_raw) & 1023)) & 1023);
    float* priv = reinterpret_cast<float*>(base + L.priv);    // [128][PS]: row r's Gram entries
    const int PS = priv_stride(mcap);
    int32_t* mem_buf = reinterpret_cast<int32_t*>(base + L.mem);  // [2][kRows]
    uint64_t* thr = reinterpret_cast<uint64_t*>(base + L.thr);
    float* snrm = reinterpret_cast<float*>(base + L.nrm);
    float* serr = reinterpret_cast<float*>(base + L.err);  // CERT: quantisation errors
    float* srt = reinterpret_cast<float*>(base + L.srt);   // CERT: norm roots, rounded up
    int* cnt_buf = reinterpret_cast<int*>(base + L.cnt);  // [2][32]
    int4* slid = reinterpret_cast<int4*>(base + L.lid);  // [kRows] the members' leaves (npass slots)
    const bool vec = (D % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + L.slot);
    const uint32_t done = tc::smem_addr(base + L.bar);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nk = Dp / kKc;
    const int64_t ngroups = (node1 - node0 + npc - 1) / npc;

    const bool ring = nk > kResident;
    if (tid == 0) {
        tc::mbar_init(done, 1);
        for (int q = 0; q < kRing; ++q) tc::mbar_init(done + 8 * (1 + q), 1);
        tc::mbar_fence_init();
    }
    int uses[kRing] = {0, 0};  // products committed to each ring buffer's barrier so far
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_addr(tmem_slot), kRows);
        tc::tmem_relinquish();
    }
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = tc::idesc_f16(bf16, kRows, kRows);
    int iter = 0;
    bool ok = true;
    const float rmcap = 1.f / (float)mcap;
    // Members of the nodes of the group that starts at position `first`, into
    // mb (member ids; a node's unused slots -1) and cb (member counts, then
    // new-member counts): warp j collects node j, the new members first, then
    // the old ones (flags from the previous round; none = all new).
    auto collect = [&](int64_t first, int32_t* mb, int* cb) {
        int last = 0;  // the last member count (orders later code after the loads)
        for (int j = warp; j < npc; j += kThreads / 32) {
            const int64_t pos = first + j;
            int M = 0, nn = 0;
            if (pos < node1) {
                const int64_t i = list ? (int64_t)list[pos] : pos;
                const uint64_t fb = fnew ? fnew[i] : ~0ull, rb = rnew ? rnew[i] : ~0ull;
                // at most 64 entries: G[i] then R[i] (k <= 32), or G[i] in two
                // halves; both loaded at once, then taken new first, old after
                uint64_t key0, key1;
                bool new0, new1;
                member_keys(Gold, R, i, k, rev, fb, rb, key0, key1, new0, new1);
                const unsigned below = (1u << lane) - 1u;
                // more members than the slot holds (slots smaller than 2k): the
                // node goes to the overflow list, for the launch with full slots
                const int all = __popc(__ballot_sync(0xffffffffu, key0 != kEmptyKey)) +
                                __popc(__ballot_sync(0xffffffffu, key1 != kEmptyKey));
                if (all > mcap) {
                    if (lane == 0) ovf_list[atomicAdd(ovf_count, 1)] = (int32_t)i;
                    key0 = key1 = kEmptyKey;
                }
                for (int want = 1; want >= 0; --want) {
                    const bool t0 = key0 != kEmptyKey && new0 == (want == 1);
                    const unsigned b0 = __ballot_sync(0xffffffffu, t0);
                    if (t0) mb[j * mcap + M + __popc(b0 & below)] = (int32_t)key_id(key0);
                    M += __popc(b0);
                    const bool t1 = key1 != kEmptyKey && new1 == (want == 1);
                    const unsigned b1 = __ballot_sync(0xffffffffu, t1);
                    if (t1) mb[j * mcap + M + __popc(b1 & below)] = (int32_t)key_id(key1);
                    M += __popc(b1);
                    if (want == 1) nn = M;
                }
            }
            for (int t = M + lane; t < mcap; t += 32) mb[j * mcap + t] = -1;
            if (lane == 0) {
                cb[j] = M;
                cb[16 + j] = nn;
            }
            last = M;
        }
        return last;
    };
    // slots past the last node's never hold a member
    for (int r = tid; r < 2 * kRows; r += kThreads) mem_buf[r] = -1;
    __syncthreads();
    if ((int64_t)blockIdx.x < ngroups) collect(node0 + (int64_t)blockIdx.x * npc, mem_buf, cnt_buf);
    __syncthreads();
    for (int64_t grp = blockIdx.x; grp < ngroups && ok; grp += gridDim.x, ++iter) {
        // this group's members (collected before the previous group's offers)
        int32_t* mem = mem_buf + (iter & 1) * kRows;
        const int* mcount = cnt_buf + (iter & 1) * 32;
        // gather the member rows (16-byte pieces) into the swizzled K-major tile;
        // the thresholds and norms below load while these copies are in flight
        // (wide rows: only the first chunk here, the rest in the ring below)
        const int q_per_row = ring ? kKc / 8 : Dp / 8;
        // piece (r, q) goes to chunk q / 8, row r, 16-byte slot (q % 8) ^ (r % 8)
        auto piece = [&](int r, int q, int u) {
            uint8_t* dst = base + (size_t)(q >> 3) * kChunkBytes + r * 128 + (((q & 7) ^ (r & 7)) << 4);
            if (u >= 0) {
                const uint16_t* src = Xq + (int64_t)u * Dp + q * 8;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tc::smem_addr(dst)), "l"(src)
                             : "memory");
            } else {
                *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
            }
        };
        if ((kThreads % q_per_row) == 0) {
            // a power of two: each thread copies piece q of rows r0, r0 + rs, ...
            const int sh = __ffs(q_per_row) - 1;
            const int q = tid & (q_per_row - 1), rs = kThreads >> sh;
#pragma unroll 4
            for (int r = tid >> sh; r < kRows; r += rs) piece(r, q, mem[r]);
        } else {
            // piece e = tid + i * kThreads is (row r, piece q); stepped without a division
            const int r_step = kThreads / q_per_row, q_step = kThreads - r_step * q_per_row;
            for (int r = tid / q_per_row, q = tid - (tid / q_per_row) * q_per_row; r < kRows;) {
                piece(r, q, mem[r]);
                r += r_step;
                q += q_step;
                if (q >= q_per_row) {
                    q -= q_per_row;
                    ++r;
                }
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        // the members' thresholds, norms and leaves: copies of their own,
        // awaited only before the epilogue
        for (int r = tid; r < kRows; r += kThreads) {
            const int u = mem[r];
            if (u >= 0) {
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(tc::smem_addr(thr + r)),
                             "l"(Gold + (int64_t)u * k + k - 1)
                             : "memory");
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(tc::smem_addr(snrm + r)), "l"(nrm + u)
                             : "memory");
                if (npass > 0)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tc::smem_addr(slid + r)),
                                 "l"(reinterpret_cast<const int4*>(leafid) + u)
                                 : "memory");
            } else {
                thr[r] = 0ull;
                snrm[r] = 0.f;
                if (npass > 0) slid[r] = make_int4(-1 - r, -1 - r, -1 - r, -1 - r);
            }
            if (CERT) {
                serr[r] = u >= 0 ? qerr[u] : 0.f;
                srt[r] = u >= 0 ? __fsqrt_ru(nrm[u]) : 0.f;
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        if (!ring) {
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // the tile (the side copies may fly on)
            // the tensor cores read shared memory through the async proxy
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncthreads();
            tc::fence_after_sync();
            if (tid == 0) {
                for (int c = 0; c < nk; ++c) {
                    const uint64_t d0 = tc::sdesc_k128(tc::smem_addr(base + (size_t)c * kChunkBytes));
#pragma unroll
                    for (int kk = 0; kk < kKc / 16; ++kk)
                        tc::mma_f16(tmem, d0 + 2 * kk, d0 + 2 * kk, idesc, (c | kk) != 0);
                }
                tc::mma_commit(done);
            }
        } else {
            // chunk c in ring buffer c % kRing: the copies of chunk c + 1 are
            // in flight while the tensor cores take chunk c; a buffer is
            // refilled only after the product that read it has completed (the
            // first wait also covers the side copies, committed after chunk 0)
            for (int c = 0; c < nk && ok; ++c) {
                if (c + 1 < nk) {
                    const int q1 = (c + 1) % kRing;
                    if (uses[q1] > 0 && !tc::mbar_wait(done + 8 * (1 + q1), (uint32_t)((uses[q1] - 1) & 1), status))
                        ok = false;
                    // pieces of chunk c + 1: row r = e / 8, piece e % 8, 4 per thread
                    for (int e = tid; e < kRows * 8; e += kThreads) {
                        const int r = e >> 3, c16 = e & 7;
                        uint8_t* dst = base + (size_t)q1 * kChunkBytes + r * 128 + ((c16 ^ (r & 7)) << 4);
                        const int u = mem[r];
                        if (u >= 0) {
                            const uint16_t* src = Xq + (int64_t)u * Dp + (c + 1) * kKc + c16 * 8;
                            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tc::smem_addr(dst)),
                                         "l"(src)
                                         : "memory");
                        } else {
                            *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
                        }
                    }
                    asm volatile("cp.async.commit_group;\n" ::: "memory");
                    asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // chunk c has landed
                } else {
                    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
                }
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                ok = __syncthreads_and(ok);
                tc::fence_after_sync();
                if (!ok) break;
                const int q0 = c % kRing;
                if (tid == 0) {
                    const uint64_t d0 = tc::sdesc_k128(tc::smem_addr(base + (size_t)q0 * kChunkBytes));
#pragma unroll
                    for (int kk = 0; kk < kKc / 16; ++kk)
                        tc::mma_f16(tmem, d0 + 2 * kk, d0 + 2 * kk, idesc, (c | kk) != 0);
                    tc::mma_commit(done + 8 * (1 + q0));
                }
                ++uses[q0];
            }
            if (!ok) {
                // copies still in flight land before anything is reused; the
                // products issued so far complete before the CTA frees its
                // tensor memory (below, after the bounded wait on `done`)
                asm volatile("cp.async.wait_all;\n" ::: "memory");
            }
            if (tid == 0) tc::mma_commit(done);
        }
        __syncwarp();
        // one thread watches the barrier; the others sleep in __syncthreads
        const int mma_ok = tid == 0 ? (tc::mbar_wait(done, (uint32_t)(iter & 1), status) ? 1 : 0) : 1;
        asm volatile("cp.async.wait_all;\n" ::: "memory");  // the side copies
        ok = __syncthreads_and(mma_ok && ok);
        tc::fence_after_sync();
        if (!ok) break;

        // ---- epilogue: row r of the tile is member s of node j.  Threads r
        // and r + 128 (warps w and w + 4 read the same tensor-memory lanes)
        // share the row: each copies half of its Gram values to priv[r][t].
        const int r = tid & (kRows - 1), h = tid >> 7;
        const int j = small_div(r, mcap, rmcap), s = r - j * mcap;
        const int Mj = j < npc ? mcount[j] : 0;
        const bool mine = s < Mj;
        // the 32-column chunks that hold the windows of this warp's rows (its
        // first and last row's nodes), alternately to h = 0 and h = 1
        const int wr0 = (warp & 3) * 32;
        const int cmin = small_div(wr0, mcap, rmcap) * mcap,
                  cmax = min((small_div(wr0 + 31, mcap, rmcap) + 1) * mcap, kRows);
#pragma unroll 1
        for (int cc = (cmin >> 5) + h; cc * 32 < cmax; cc += 2) {
            float g[32];
            tc::tmem_ld_32(tmem + ((uint32_t)wr0 << 16) + (uint32_t)(cc * 32), g);
            if (mine) {
                // in aligned quads: j * mcap and cc * 32 are multiples of 8, and
                // a quad that starts below Mj ends below PS
#pragma unroll
                for (int qd = 0; qd < 8; ++qd) {
                    const int t = cc * 32 + 4 * qd - j * mcap;
                    if ((unsigned)t < (unsigned)Mj)
                        *reinterpret_cast<float4*>(priv + r * PS + t) =
                            make_float4(g[4 * qd], g[4 * qd + 1], g[4 * qd + 2], g[4 * qd + 3]);
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        // Bit i of `hit`: by rows, member i is offered to member s; by pairs,
        // the thread's (i / 2)-th pair {a, b} offers b to a (i even) or a to b.
        // An entry of priv that makes an offer is overwritten with its
        // distance (no other thread reads that entry).
        const int nn = j < npc ? mcount[16 + j] : 0, no = Mj - nn;
        const int P = nn * no + nn * (nn - 1) / 2;
        const bool by_rows = 8 * P >= Mj * Mj;
        const int T = 2 * mcap, tix = 2 * s + h, base_row = j * mcap;
        const PairMap pm = pair_map(nn, no);
        uint64_t hit = 0;
        const uint32_t ua = mine ? (uint32_t)mem[r] : 0u;
        if (by_rows && mine) {
            const uint64_t ta = thr[r];
            // the threshold key as (distance, id): an offer (d, ub) is below it
            // when d < ta_d, or d == ta_d and ub < ta_id (d >= 0, never NaN);
            // an empty slot takes everything
            const float ta_d = ta == kEmptyKey ? __int_as_float(0x7f800000) : key_dist(ta);
            const uint32_t ta_id = ta == kEmptyKey ? 0xFFFFFFFFu : key_id(ta);
            const float na = snrm[r];
            const int bend = s < nn ? Mj : nn;
            const int4 la = slid[r];
            float* prow = priv + r * PS;
            if (!CERT) {
                // quads of members, alternately to h = 0 and h = 1: one 16-byte
                // load each of Gram entries, member ids and norms.  Exact
                // arithmetic: s - 2g is an integer below 2^24 however it is
                // rounded, never -0, so its key orders like the distance.
#pragma unroll 1
                for (int b4 = 4 * h; b4 < bend; b4 += 8) {
                    const float4 g4 = *reinterpret_cast<const float4*>(prow + b4);
                    const int4 u4 = *reinterpret_cast<const int4*>(mem + base_row + b4);
                    const float4 n4 = *reinterpret_cast<const float4*>(snrm + base_row + b4);
                    const float gq[4] = {g4.x, g4.y, g4.z, g4.w}, nq[4] = {n4.x, n4.y, n4.z, n4.w};
                    const uint32_t uq[4] = {(uint32_t)u4.x, (uint32_t)u4.y, (uint32_t)u4.z, (uint32_t)u4.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int b = b4 + e;
                        const float d = __fmaf_rn(-2.f, gq[e], __fadd_rn(na, nq[e]));
                        const int4 lb = slid[base_row + b];
                        // member s itself has id ua: the id test skips it
                        const bool off = (b < bend) & (uq[e] != ua) & (make_key(d, uq[e]) < ta) &
                                         !leaf_mates(la, lb, npass);
                        hit |= (uint64_t)off << b;
                        if (off) prow[b] = d;
                    }
                }
            }
            for (int b = h; CERT && b < bend; b += 2) {
                const uint32_t ub = (uint32_t)mem[base_row + b];
                if (b == s || ub == ua) continue;
                // leaf-mates were offered to each other in the leaf stage (with
                // CERT, no canonical distance is needed for them either)
                if (CERT && leaf_mates(la, slid[base_row + b], npass)) continue;
                float d = __fadd_rn(__fsub_rn(__fadd_rn(na, snrm[base_row + b]), __fmul_rn(2.f, prow[b])), 0.f);
                if (CERT) {
                    const float cD = (16.f * Dp + 8.f) * 5.9604644775390625e-8f;  // 2^-24
                    const float sn = __fadd_ru(srt[r], srt[base_row + b]);
                    const float eps = __fadd_ru(__fmul_ru(cD, __fmul_ru(sn, sn)), __fmul_ru(1.1920928955078125e-7f, fabsf(d)));
                    const float lo = __fsub_rd(d, eps);
                    float lb = 0.f;
                    if (lo > 0.f) {
                        const float root = __fsub_rd(__fsub_rd(__fsqrt_rd(lo), serr[r]), serr[base_row + b]);
                        if (root > 0.f) lb = __fmul_rd(root, root);
                    }
                    // an empty slot's key accepts everything
                    if (lb > ta_d) continue;
                    d = canon_dist(X + (int64_t)ua * D, X + (int64_t)ub * D, D, vec);
                }
                if (d < ta_d || (d == ta_d && ub < ta_id)) {
                    hit |= 1ull << b;
                    prow[b] = d;
                }
            }
        } else if (!by_rows) {
            for (int p = tix, i = 0; p < P; p += T, ++i) {
                int a, b;
                pm.decode(p, a, b);
                const uint32_t pa = (uint32_t)mem[base_row + a], pb = (uint32_t)mem[base_row + b];
                if (CERT && (pa == pb || leaf_mates(slid[base_row + a], slid[base_row + b], npass))) continue;
                float d = __fadd_rn(__fsub_rn(__fadd_rn(snrm[base_row + a], snrm[base_row + b]),
                                              __fmul_rn(2.f, priv[(base_row + b) * PS + a])), 0.f);
                const uint64_t ta = thr[base_row + a], tb = thr[base_row + b];
                if (CERT) {
                    const float cD = (16.f * Dp + 8.f) * 5.9604644775390625e-8f;  // 2^-24
                    const float sn = __fadd_ru(srt[base_row + a], srt[base_row + b]);
                    const float eps = __fadd_ru(__fmul_ru(cD, __fmul_ru(sn, sn)), __fmul_ru(1.1920928955078125e-7f, fabsf(d)));
                    const float lo = __fsub_rd(d, eps);
                    float lb = 0.f;
                    if (lo > 0.f) {
                        const float root = __fsub_rd(__fsub_rd(__fsqrt_rd(lo), serr[base_row + a]), serr[base_row + b]);
                        if (root > 0.f) lb = __fmul_rd(root, root);
                    }
                    const bool na = ta == kEmptyKey || !(lb > key_dist(ta));
                    const bool nb = tb == kEmptyKey || !(lb > key_dist(tb));
                    if (!na && !nb) continue;
                    d = canon_dist(X + (int64_t)pa * D, X + (int64_t)pb * D, D, vec);
                }
                // without branches: duplicates of one id and leaf-mates make no offer
                const bool keep = (pa != pb) & !leaf_mates(slid[base_row + a], slid[base_row + b], npass);
                const bool oa = keep & (make_key(d, pb) < ta), ob = keep & (make_key(d, pa) < tb);
                if (oa | ob) priv[(base_row + b) * PS + a] = d;
                hit |= ((uint64_t)oa << (2 * i)) | ((uint64_t)ob << (2 * i + 1));
            }
        }
        // one slot range per warp, then the offers themselves
        const int cnt = __popcll(hit);
        int x = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const int total = __shfl_sync(0xffffffffu, x, 31);
        uint32_t at = 0;
        if (lane == 31 && total > 0) at = atomicAdd(counter, (uint32_t)total);
        // the next group's members are collected (into the other buffers)
        // while the slot range is on its way
        const int64_t nxt = grp + gridDim.x;
        int dep = 0;
        if (nxt < ngroups)
            dep = collect(node0 + nxt * npc, mem_buf + ((iter + 1) & 1) * kRows, cnt_buf + ((iter + 1) & 1) * 32);
        // the slot range is read only here, after the collection's loads
        asm volatile("" : "+r"(at) : "r"(dep));
        at = __shfl_sync(0xffffffffu, at, 31);
        if (total > 0 && (int64_t)at + total > cap) {
            if (lane == 0) atomicOr(status, kStatusOverflow);
            hit = 0;
        }
        uint32_t w = at + x - cnt;
        if (by_rows) {
            if (hit) atomicAdd(&pcnt[ua], cnt);  // one count per target and thread
            while (hit != 0) {
                const int b = __ffsll((long long)hit) - 1;
                hit &= hit - 1;
                ptgt[w] = ua;
                pkey[w] = make_key(priv[r * PS + b], (uint32_t)mem[base_row + b]);
                ++w;
            }
        } else {
            while (hit != 0) {
                const int bit = __ffsll((long long)hit) - 1;
                hit &= hit - 1;
                int a, b;
                pm.decode(tix + (bit >> 1) * T, a, b);
                const uint32_t pa = (uint32_t)mem[base_row + a], pb = (uint32_t)mem[base_row + b];
                const float d = priv[(base_row + b) * PS + a];
                const uint32_t tgt = (bit & 1) ? pb : pa;
                ptgt[w] = tgt;
                pkey[w] = make_key(d, (bit & 1) ? pa : pb);
                ++w;
                atomicAdd(&pcnt[tgt], 1);
            }
        }
        // all tensor-memory reads and shared-memory uses of this group done
        tc::fence_before_sync();
        __syncthreads();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kRows);
}

}  // namespace

namespace {
// One launch of the tensor-core join with member slots of mcap rows (ovf:
// nodes with more members go to b.ovf_list); bytes: its algorithmic bytes.
void join_tc_once(const uint16_t* Xq, int Dp, const float* nrm, int k, bool rev, int mcap, const uint64_t* Gold,
                  const uint64_t* R, int64_t node0, int64_t node1, const JoinBuffers& b, int* status,
                  const int* notexact, bool bf16, cudaStream_t s, bool cert, const float* X, int D, bool ovf,
                  double bytes) {
    const int npc = kRows / mcap;
    const JtSmem L = jt_smem(Dp, mcap, cert);
    // at least 56 KB per CTA: at most 4 CTAs (512 tensor-memory columns) per SM
    size_t smem = L.total + 1024;
    if (smem < 56 * 1024) smem = 56 * 1024;
    const int64_t nodes = node1 - node0;
    const int64_t groups = (nodes + npc - 1) / npc;
    const int per_sm = (int)((227 * 1024) / smem) < 4 ? (int)((227 * 1024) / smem) : 4;
    const int grid = (int)std::max<int64_t>(1, groups < (int64_t)152 * per_sm ? groups : (int64_t)152 * per_sm);
    // certifying: the canonical distances' rows of X are counted per offer
    // written (record_bytes), not here
    LaunchScope ls(cert ? "k5_join_tc_cert" : "k5_join_tc", s, bytes, bytes > 0 ? (double)groups * kRows * kRows * 2.0 * Dp : 0.0);
    int32_t* ol = ovf ? b.ovf_list : nullptr;
    int32_t* oc = ovf ? b.ovf_count : nullptr;
    if (cert) {
        cudaFuncSetAttribute(k5_join_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k5_join_tc<true><<<grid, kThreads, smem, s>>>(Xq, Dp, nrm, k, rev ? 1 : 0, mcap, npc, Gold, R, b.list, b.fnew,
                                                      b.rnew, node0, node1, b.counter, b.cap, b.ptgt, b.pkey, b.pcnt,
                                                      status, notexact, bf16, X, D, b.qerr, b.count_dev, b.leafid,
                                                      b.npass, ol, oc);
    } else {
        cudaFuncSetAttribute(k5_join_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k5_join_tc<false><<<grid, kThreads, smem, s>>>(Xq, Dp, nrm, k, rev ? 1 : 0, mcap, npc, Gold, R, b.list,
                                                       b.fnew, b.rnew, node0, node1, b.counter, b.cap, b.ptgt, b.pkey,
                                                       b.pcnt, status, notexact, bf16, nullptr, 0, nullptr,
                                                       b.count_dev, b.leafid, b.npass, ol, oc);
    }
}
}  // namespace

bool launch_join_tc(const uint16_t* Xq, int D, const float* nrm, int k, bool rev, const uint64_t* Gold,
                    const uint64_t* R, int64_t node0, int64_t node1, const JoinBuffers& b, int* status,
                    const int* notexact, bool bf16, cudaStream_t s, bool cert, const float* X) {
    const int Dp = lp_dim(D);
    const int mcap = ((rev ? 2 * k : k) + 7) & ~7;
    if (mcap > 64) return false;  // a 64-bit mask of offers per tile row
    if (cert && (!X || !b.qerr)) return false;
    const double m = rev ? 2.0 * k : (double)k;
    const double bytes = (double)(node1 - node0) * (m * Dp * 2.0 + 2 * k * 8.0 + m * (cert ? 20.0 : 12.0));
    // With reverse lists a mutual neighbour is one member, so most nodes
    // have far fewer than 2k: slots of four fifths of 2k (rounded to 8) when
    // that packs more nodes into a tile, the nodes that do not fit joined
    // after them with full slots (their count read on the device)
    int small = mcap;
    if (rev && b.ovf_list && b.ovf_count) {
        const int m2 = (mcap * 4 / 5 + 7) & ~7;
        if (m2 >= 8 && kRows / m2 > kRows / mcap) small = m2;
    }
    if (small == mcap) {
        join_tc_once(Xq, Dp, nrm, k, rev, mcap, Gold, R, node0, node1, b, status, notexact, bf16, s, cert, X, D,
                     false, bytes);
        return true;
    }
    cudaMemsetAsync(b.ovf_count, 0, sizeof(int32_t), s);
    join_tc_once(Xq, Dp, nrm, k, rev, small, Gold, R, node0, node1, b, status, notexact, bf16, s, cert, X, D, true,
                 bytes);
    JoinBuffers b2 = b;
    b2.list = b.ovf_list;
    b2.count_dev = b.ovf_count;
    join_tc_once(Xq, Dp, nrm, k, rev, mcap, Gold, R, 0, node1 - node0, b2, status, notexact, bf16, s, cert, X, D,
                 false, 0.0);
    return true;
}

}  // namespace knng
