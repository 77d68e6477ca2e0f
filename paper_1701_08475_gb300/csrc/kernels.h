// kernels.h -- host-side launchers of the kNN-graph kernels (one .cu per stage).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace knng {

// ---------------------------------------------------------------- stats
// Every launcher reports its launch through this hook so that launches,
// algorithmic bytes/flops and (optionally) event-timed device time can be
// summed per kernel name.
struct LaunchScope {
    // `kernels`: how many kernel launches the scope encloses
    LaunchScope(const char* name, cudaStream_t s, double bytes, double flops, int kernels = 1);
    ~LaunchScope();
    const char* name_;
    cudaStream_t s_;
    double bytes_, flops_;
    int slot_;
};
// Reads the event times of the launches timed since the last flush into the
// statistics; call after the stream has been synchronised.
void stats_flush();
// Host-side fault injection for tests (KNNG_FAULT=alloc|launch, read by
// fault_begin at the start of each call): fault_alloc() tells an allocation
// to fail; fault_launch_point(s) issues, once per call, a launch the runtime
// refuses on the host (never on a capturing stream).
void fault_begin();
bool fault_alloc();
void fault_launch_point(cudaStream_t s);
// The first error of a launch made in this call (LaunchScope records it right
// after each launch), else the runtime's last error; both are cleared.
cudaError_t launch_error();

// ---------------------------------------------------------------- prepare (K0)
// Sets *status |= kStatusNonFinite if any of the n*D values is not finite.
void launch_check_finite(const float* X, int64_t count, int* status, cudaStream_t s);

// ---------------------------------------------------------------- two-means split (K1)
struct SelState {
    uint64_t prefix;  // known high bits of the selected key
    uint32_t krem;    // rank still to select among keys matching prefix
    uint32_t done;    // the selected key is known (thr written)
};

struct LevelPlan {
    int level;
    int n;            // points covered by the level (all of them)
    int nseg;
    int ntiles;
    int max_m;        // largest segment size at this level
    int pos_bits;     // bits of a position inside a segment
    bool small;       // one CTA per segment selects and partitions
    int nsweep;       // sweep tiles (project, sums)
    const int32_t* seg_off;    // device [nseg + 1]
    const int4* tiles;         // device [ntiles] select tiles {seg, begin, end, first_of_seg}
    const int32_t* seg_tile0;  // device [nseg + 1] first select tile of each segment
    const int4* sweep;         // device [nsweep] sweep tiles, same layout
    const int32_t* seg_sweep0; // device [nseg + 1] first sweep tile of each segment
    // Forests (independent instances side by side): a segment with no tiles
    // is a finished tree's leaf and does not split (`frozen`: the level has
    // one); seg_local[seg] is the segment's index within its own tree at this
    // level (NULL: the global index, one tree)
    const int32_t* seg_local = nullptr;
    bool frozen = false;
};

struct SplitBuffers {
    float* W;             // [nseg_max][D]  c1 - c0 per segment
    float* S;             // [n] projections (even iterations of a level)
    uint64_t* thr;        // [nseg_max] selected key (first key of the right side)
    float* S2;            // [n], [nseg_max]: the same for odd iterations
    uint64_t* thr2;
    SelState* st;         // [nseg_max]
    uint32_t* ghist;      // [nseg_large][2048]: zeroed once per partition, left zero by each select
    uint32_t* ticket;     // [nseg_large]: same
    int nseg_large;       // segments of the widest level that selects across CTAs
    double* partial;      // [nsweep_max][2][D]
    double* segsum;       // [nseg_max][D] each segment's sum of rows (FP64, or int64 for integer data)
    double* segleft;      // [nseg_max][D] the same for its left side at the last cut
    int32_t* tile_left;   // [ntiles_max]
    int* status;          // device status word
    // 16-bit copy of X (original order, rows of Dq); the sweeps read it
    // instead of X when *qflag says it holds every value exactly
    const uint16_t* Xq = nullptr;
    int Dq = 0, qtype = 0;  // qtype 1 = BF16, 2 = FP16
    const int* qflag = nullptr;
    bool q16_host = false;  // the host's copy of that decision (statistics only)
    // byte copy of X (original order, rows of Db = D rounded up to 16 bytes);
    // the staged sweeps read it first when *bflag == 0 (every value an
    // integer in [0, 255])
    const uint8_t* Xb = nullptr;
    int Db = 0;
    const int* bflag = nullptr;
    bool u8_host = false;   // the host's copy of that decision
    bool capture = false;   // recorded into a CUDA graph: the host knows nothing of the data
};

constexpr int kTile = 2048;         // positions per select/partition tile
constexpr int kSweepTile = 512;     // positions per project/sums tile
constexpr int kSmallMax = 8192;     // segments up to this size select in one CTA
constexpr int kSortSelectMax = 2048; // segments up to this size select by a sort in registers
constexpr int kRadixBits = 11;

// One level of the balanced two-means tree: T Lloyd iterations, then the
// final cut that writes perm_out.
void run_split_level(const float* X, int D, const LevelPlan& lp, int iters, uint64_t pass_seed,
                     const int32_t* perm_in, int32_t* perm_out, const SplitBuffers& b,
                     cudaStream_t s);

// ---------------------------------------------------------------- leaf stage (K2)
// For every leaf l (perm[leaf_off[l] .. leaf_off[l+1]), 2..256 points): all
// pairs, canonical FP32 distances, merged into the key graph G (n x k).
void launch_leaf_fp32(const float* X, int D, const int32_t* perm, const int32_t* leaf_off,
                      int nleaf, int max_leaf, int k, uint64_t* G, const int* status, cudaStream_t s);

// ---------------------------------------------------------------- low precision (K0, K2 tensor cores, K3)
int lp_dim(int D);  // D rounded up to the 64-element rows of the swizzled tiles
// Quantisation types of the low-precision copy: 0 FP16, 1 BF16, 2 FP8 E4M3
// with a scale per row.  Bytes per row of the copy (a multiple of 128).
int lp_row_bytes(int D, int qt);
// The leaf certificate's coefficient of (||x^_i|| + ||x^_j||)^2.
float lp_cert_coeff(int D, int qt);
// Byte copy of X (rows of Db bytes) and its flag: 0 when every value is an
// integer in [0, 255].  The caller clears *bflag; launches over several row
// ranges accumulate into it.
void launch_bytes(const float* X, int64_t n, int D, int Db, uint8_t* Xb, int* bflag, cudaStream_t s);
// Low-precision copy of X (perm: row order; NULL = identity), squared norms
// of the copy, quantisation errors and (FP8) row scales; *notexact |= 1 when
// the low-precision arithmetic is not exact for this input (always for FP8).
void launch_quantize(const float* X, int64_t n, int D, const int32_t* perm, int qt, void* Xq, float* nrm,
                     float* qerr, float* scale, int* notexact, cudaStream_t s);
// Leaf-order gather of a low-precision copy (with its norms, errors and
// scales; scale may be NULL).
void launch_permute16(const void* Xq, const float* nrm, const float* qerr, const float* scale, int64_t n,
                      int row_bytes, const int32_t* perm, void* Xl, float* lnrm, float* lerr, float* lscale,
                      cudaStream_t s);
// Leaf stage on tcgen05 from the leaf-order copy; false when it cannot run
// (leaf above 256 points, no tensor-map encoder) and nothing was launched.
// status[1] counts the rows whose first batch of exact evaluations did not
// settle them.  dump (a parity hook, one leaf of m points): the m x m
// approximate distances are written there and nothing is selected.
// The values of a low-precision copy as FP32 (m x D; FP8: the unscaled q).
void launch_lp_to_float(const void* Xq, int64_t m, int D, int qt, float* out, cudaStream_t s);
bool launch_leaf_tc(const void* Xl, int64_t n, const float* X, int D, const int32_t* perm,
                    const int32_t* leaf_off, int nleaf, int max_leaf, const float* nrm, const float* qerr,
                    const float* scale, int k, int kp, int qt, uint64_t* G, int* status, const int* notexact,
                    cudaStream_t s, float* dump = nullptr);

// ---------------------------------------------------------------- refinement (K4-K6)
struct JoinBuffers {
    int32_t* deg;        // [n + 1]
    int32_t* roff;       // [n + 1]
    int32_t* cur;        // [n]
    uint64_t* rbuf;      // [n * k]
    uint64_t* R;         // [n * k]
    int32_t* pcnt;       // [n + 1]
    int32_t* poff;       // [n + 1]
    int32_t* pcur;       // [n]
    uint32_t* ptgt;      // [cap]
    uint64_t* pkey;      // [cap]
    uint64_t* grouped;   // [cap]
    int64_t cap;         // proposal capacity of one chunk
    uint32_t* counter;   // [1] proposals appended
    int32_t* scan_tmp;   // scan scratch
    unsigned long long* offers_total;  // [1] offers grouped over the whole call (statistics)
    // member flags between rounds: R2 keeps the previous round's reverse
    // lists; fnew_buf / rnew_buf [n] bit e marks entry e of G_old[i] / R[i]
    // new; active [n] lists the nodes with a new member, nactive [1] counts them
    uint64_t* R2 = nullptr;
    uint64_t* fnew_buf = nullptr;
    uint64_t* rnew_buf = nullptr;
    int32_t* active = nullptr;
    int32_t* nactive = nullptr;
    // the current round's view of them (NULL: every node, every member new)
    const int32_t* list = nullptr;
    const uint64_t* fnew = nullptr;
    const uint64_t* rnew = nullptr;
    // capture: no host reads (a CUDA graph records the build): chunks of the
    // worst-case size over all positions, both joins launched with the choice
    // made on the device, and `count_dev` (device) bounding the positions
    bool capture = false;
    const int32_t* count_dev = nullptr;
    // tensor-core join (16-bit copy in original order); used when lp is set
    // and, on the device, only when the copy's arithmetic is exact
    bool lp = false, bf16 = true;
    const uint16_t* Xq = nullptr;
    const float* qnrm = nullptr;
    const float* qerr = nullptr;
    const int* notexact = nullptr;
    // the leaf of every point in the build's last tree passes ([n][4], slots
    // 0 .. npass - 1 used; NULL: none).  Two points that shared a leaf were compared there, and
    // each was offered to the other's list; lists only improve, so offering
    // that pair again could not change either list, and the join skips it.
    const int32_t* leafid = nullptr;
    int npass = 0;
    // the tensor-core join with reverse lists first packs nodes into slots
    // smaller than 2k members (a mutual neighbour is one member, so most
    // nodes have far fewer); a node that does not fit is listed here and joined
    // by a second launch with full slots
    int32_t* ovf_list = nullptr;   // [n]
    int32_t* ovf_count = nullptr;  // [1]
    // sampled rounds: per node a flag mask (bit e: entry e of the list is
    // new) and the mask after this round's sample (NULL: full rounds)
    uint64_t* flags = nullptr;
    uint64_t* flags_post = nullptr;
    // the order in which the rounds take the nodes: the ids in the leaf
    // order of the build's last tree pass (NULL: id order).  Neighbouring
    // nodes of a leaf share most of their members, so taken together their
    // member rows are read once from DRAM and then from L2.  A round's result
    // does not depend on the order.
    const int32_t* order = nullptr;
};

constexpr int kMaxLeafPasses = 4;  // tree passes whose leaves the join remembers

// Did two points with leaf ids a and b (npass slots used) share a leaf?
__device__ __forceinline__ bool leaf_mates(const int4& a, const int4& b, int npass) {
    static_assert(kMaxLeafPasses == 4, "one int4 of leaf ids per point");
    return (npass > 0 && a.x == b.x) || (npass > 1 && a.y == b.y) || (npass > 2 && a.z == b.z) ||
           (npass > 3 && a.w == b.w);
}

// lid[perm[p] * kMaxLeafPasses + slot] = the leaf of position p (leaf_off:
// nleaf + 1 offsets).
void launch_leaf_ids(const int32_t* perm, const int32_t* leaf_off, int nleaf, int64_t n, int slot, int32_t* lid,
                     cudaStream_t s);

// The tensor-core local join of the nodes at positions [node0, node1) of
// b.list (of all nodes when it is NULL); false (nothing launched) when the
// shape is not supported.
// cert: the 16-bit copy is not exact; the Gram only screens pairs and the
// offers use canonical distances from X (b.qerr: quantisation errors).
bool launch_join_tc(const uint16_t* Xq, int D, const float* nrm, int k, bool rev, const uint64_t* Gold,
                    const uint64_t* R, int64_t node0, int64_t node1, const JoinBuffers& b, int* status,
                    const int* notexact, bool bf16, cudaStream_t s, bool cert = false, const float* X = nullptr);

// Adds `items` (algorithmic `bytes`) to the statistics of kernel `name`
// (when statistics are on).
void record_items(const char* name, double items);
void record_bytes(const char* name, double bytes);

void launch_reverse_lists(const uint64_t* G, int64_t n, int k, const JoinBuffers& b, cudaStream_t s);
// `rounds` refinement rounds on G (G2: the second graph buffer); on return
// G points at the result.  Rounds after the first skip the member pairs that
// the previous round already offered.
void run_refine(const float* X, int64_t n, int D, int k, bool rev, uint64_t*& G, uint64_t*& G2,
                const JoinBuffers& b, int64_t nodes_per_chunk, int rounds, int* status, cudaStream_t s);
// `rounds` sampled refinement rounds (nearest-neighbour descent with ms
// samples per list, every entry new before the first): b.flags and
// b.flags_post hold the masks; round r draws with SplitMix64(seed ^ r).
void run_refine_sampled(const float* X, int64_t n, int D, int k, uint64_t*& G, uint64_t*& G2, const JoinBuffers& b,
                        int64_t nodes_per_chunk, int rounds, int ms, uint64_t seed, int* status, cudaStream_t s);

// Exclusive scan of cnt[0..n) into off[0..n], off[n] = total.
void launch_scan(const int32_t* cnt, int32_t* off, int64_t n, int32_t* tmp, cudaStream_t s);
size_t scan_tmp_ints(int64_t n);

// ---------------------------------------------------------------- graph I/O
void launch_fill_empty(uint64_t* G, int64_t count, cudaStream_t s);
// ids outside [-1, n) set kStatusBadInput (and are stored as empty slots)
void launch_pack(const int32_t* ids, const float* d, uint64_t* G, int64_t count, int64_t n, int* status,
                 cudaStream_t s);
// Sets kStatusBadInput if any of ids[0 .. count) lies outside [lo, hi).
void launch_check_ids(const int32_t* ids, int64_t count, int64_t lo, int64_t hi, int* status, cudaStream_t s);
// ids are written as key id - id_offset (an instance's first row in a forest)
void launch_unpack(const uint64_t* G, int32_t* ids, float* d, int64_t count, cudaStream_t s, int64_t id_offset = 0);

// ---------------------------------------------------------------- exact / recall (K7)
// Sampled refinement round (sampled.cu): the sample of every list and of the
// reverse lists, the member view Gm, the masks fm (sampled) and Fp (flags
// after the sample), the sampled reverse rows R with their new-mask rm; and
// the flags after the merge.
void launch_sampled_prepare(const uint64_t* G, uint64_t* F, int64_t n, int k, int ms, uint64_t h0, uint64_t* Gm,
                            uint64_t* fm, uint64_t* Fp, int32_t* deg, int32_t* roff, int32_t* cur, int32_t* scan_tmp,
                            uint64_t* rbuf, uint64_t* R, uint64_t* rm, cudaStream_t s);
void launch_sampled_flags(const uint64_t* Gnew, const uint64_t* Gold, const uint64_t* Fp, int64_t n, int k,
                          uint64_t* F, unsigned long long* entered, cudaStream_t s);

// Residue vector quantisation and its inverted index (rvq.cu, Sec. 4).
// codes of the N vectors v_i = X_i, or X_i - W1[c1[i * c1_stride]] when W1 is
// given, against W <= 256 words: out[i * out_stride].
void launch_rvq_assign(const float* X, int64_t N, int D, const float* W1, const int32_t* c1, int c1_stride,
                       const float* words, int W, int32_t* out, int out_stride, cudaStream_t s);
// Stable sort of the ids in[0..n) (0..n-1 when in is null) by the 8-bit digit
// key[id * kstride] into out.  hist: digit_sort_hist_ints(n) ints; gofs: one
// more; gofs[d * digit_sort_blocks(n)] is where digit d starts.
int digit_sort_blocks(int64_t n);
size_t digit_sort_hist_ints(int64_t n);
void launch_digit_sort(const int32_t* in, int64_t n, const int32_t* key, int kstride, int32_t* out, int32_t* hist,
                       int32_t* gofs, int32_t* scan_tmp, cudaStream_t s);
// words[c] = FP64 mean (ascending vector order) of the vectors of word c, in
// FP32; words without members keep their value.
void launch_rvq_update(const float* X, int64_t N, int D, const float* W1, const int32_t* c1, int c1_stride,
                       const int32_t* order, const int32_t* gofs, int nb, int W, float* words, cudaStream_t s);
void launch_rvq_init(const float* X, int D, const float* W1, const int32_t* c1, int c1_stride, const int64_t* pos,
                     int W, float* words, cudaStream_t s);
// R = X - W1[c1] row by row (FP32): the stage-2 training vectors.
void launch_rvq_residues(const float* X, int64_t N, int D, const float* W1, const int32_t* c1, float* R,
                         cudaStream_t s);
void launch_rvq_key_count(const int32_t* codes, int64_t n, int W2, int32_t* cnt, cudaStream_t s);
void launch_check_offsets(const int32_t* off, int64_t nk, int64_t n, int* status, cudaStream_t s);
void launch_rvq_tables(const float* w1, int W1, const float* w2, int W2, int D, float* n1, float* n2, float* x12,
                       float* w1T, float* w2T, cudaStream_t s);
int rvq_seed_keys(int probe1, int W2);
size_t rvq_seeds_smem(int probe1, int W2, int D);
void launch_rvq_seeds(const float* w1T, int W1, const float* w2T, int W2, int D, const float* n1, const float* n2,
                      const float* x12, const int32_t* off, const int32_t* ids, const float* Q, int64_t m, int probe1,
                      int s_seeds, int32_t* S, const int* status, cudaStream_t s);

// Enhanced hill-climbing search (search.cu): queries [q0, q1) of Q against
// the graph G (n x k ids), seeds S (s per query), t0 iterations, ks <= 32
// results per query; tab: (q1 - q0) << cap_log2 ints of visited tables.
int search_cap_log2(int s, int t0, int ks, int k);
void launch_search(const float* X, int64_t n, int D, const int32_t* G, int k, const float* Q, int64_t q0,
                   int64_t q1, const int32_t* S, int s, int t0, int ks, int32_t* tab, int cap_log2, int32_t* out_ids,
                   float* out_d, cudaStream_t st);

void launch_exact(const float* X, int64_t n, int D, int k, const int32_t* sample, int64_t s_rows,
                  uint64_t* out, const int* status, cudaStream_t s);
void launch_recall(const int32_t* ids, const float* d, const int32_t* gt_ids, const float* gt_d,
                   const int32_t* sample, int64_t s_rows, int k, unsigned long long* counts,
                   cudaStream_t s);

}  // namespace knng
