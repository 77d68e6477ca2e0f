/*
 * knng.h -- C ABI of the GB300 (sm_103a) kNN-graph builder.
 *
 * The library builds an approximate k-nearest-neighbour graph of n points in
 * R^D by the method of Zhao, Yang and Deng, "Scalable Nearest Neighbor Search
 * based on kNN Graph" (arXiv 1701.08475):
 *   - Sec. 3.1 / Alg. 1: I_0 rounds ("tree passes"), each partitioning the
 *     points by recursive two-means bisection into clusters no bigger than a
 *     threshold (leaf_max), then comparing every pair inside each cluster and
 *     updating both endpoints' k-lists;
 *   - Sec. 1 (prior art cited there, nearest-neighbour descent): optional
 *     neighbour-of-neighbour refinement rounds (local join).
 *
 * Conventions shared by every call:
 *   - data is n x D FP32, row-major, rows contiguous (row i at data + i*D).
 *   - A graph is two n x k row-major arrays: ids (int32) and dists (FP32,
 *     squared l2).  Row i is sorted ascending by (dist, id), holds unique ids,
 *     never i itself; an empty slot is (id -1, dist +inf) and sorts last.
 *   - Distances are the canonical FP32 squared l2: acc = 0; for j = 0..D-1:
 *     t = x_j - y_j; acc = fmaf(t, t, acc).  Equal pairs give equal bits.
 *   - Ties are broken by the smaller id.
 *   - Pointers may be device pointers or host pointers (pageable or pinned);
 *     the library detects which.  Host inputs are copied to the device inside
 *     the call and host outputs are copied back before it returns.  The caller
 *     owns every buffer it passes; the library allocates only its own
 *     workspace (stream-ordered, from a library memory pool) and releases it
 *     before returning.
 *   - stream: a cudaStream_t (NULL = the legacy default stream).  Every call
 *     is synchronous: it returns after its work on `stream` has finished.
 *   - Return value: KNNG_OK or a negative KNNG_E* code; knng_last_error()
 *     gives a message (thread-local, valid until the next call on the thread).
 *   - n < 2^31 (ids are int32).  Limits: 1 <= k <= 64, 1 <= D <= 4096,
 *     2 (k + 1) <= leaf_max <= 256.
 */
#ifndef KNNG_H
#define KNNG_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define KNNG_API __attribute__((visibility("default")))
#else
#define KNNG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define KNNG_OK 0
#define KNNG_EINVAL (-1)   /* bad argument (message says which) */
#define KNNG_ENOMEM (-2)   /* device allocation failed */
#define KNNG_ECUDA (-3)    /* a CUDA call or kernel failed */
#define KNNG_ETIMEOUT (-4) /* a bounded device wait gave up */

enum knng_join_mode {
    KNNG_JOIN_FWD = 0,     /* N_i = G[i] */
    KNNG_JOIN_FWD_REV = 1, /* N_i = G[i] + R[i], R[i] the k closest reverse neighbours */
    KNNG_JOIN_SAMPLED = 2  /* nearest-neighbour descent with sampling (Dong, Charikar and Li 2011): per-entry
                              new/old flags, knng_params.sample new entries per list and members per reverse
                              list drawn by a counter-based priority, new x new and new x old pairs joined */
};

enum knng_precision {
    KNNG_FP32 = 0,         /* canonical FP32 everywhere */
    KNNG_BF16 = 1,         /* leaf Gram on tensor cores from a BF16 copy, certified FP32 re-rank */
    KNNG_FP16 = 2,         /* the same from an FP16 copy */
    KNNG_FP8 = 3           /* the same from an FP8 E4M3 copy, each row scaled by max|x| / 448 */
    /* With BF16/FP16 the graph is identical to the FP32 one: every row whose
     * low-precision selection cannot be certified by the error bound is
     * recomputed in FP32.  Leaves above 128 points use the FP32 leaf kernel. */
};

typedef struct knng_params {
    int k;               /* neighbours per point (Alg. 1 "k: scale of k-NN Graph") */
    int leaf_max;        /* cluster-size threshold (Sec. 3.1, e.g. 50) */
    int tree_passes;     /* I_0, the rounds of Alg. 1; each uses a new partition */
    int refine_rounds;   /* neighbour-of-neighbour rounds after the passes */
    int join_mode;       /* enum knng_join_mode */
    int precision;       /* enum knng_precision */
    int twomeans_iters;  /* Lloyd iterations T per two-means split (>= 0) */
    uint64_t seed;       /* partition seed; pass p uses SplitMix64(seed ^ p) */
    int sample;          /* KNNG_JOIN_SAMPLED only: samples per list, 1 <= sample <= k / 2;
                            round r draws member u of node v by the upper 32 bits of
                            SplitMix64(SplitMix64(seed ^ r) ^ (v << 32 | u)), least first, ties by u.
                            Not taken by recorded or batched builds. */
} knng_params;

/* Defaults: k 10, leaf_max 64, tree_passes 1, refine_rounds 0,
 * join_mode FWD_REV, precision FP32, twomeans_iters 4, seed 0, sample 0. */
KNNG_API void knng_default_params(knng_params *p);

/*
 * Build the kNN graph of `data` (Alg. 1, Sec. 3.1): `rounds` tree passes
 * (I_0; the paper calls one partition-and-compare cycle a "round"), each a
 * balanced two-means tree with clusters of at most leaf_max points followed by
 * the all-pairs update inside every cluster; no refinement; FP32; default
 * stream; `seed` fixes the partitions.
 * out_ids, out_dists: n x k, written in full.
 * Errors: KNNG_EINVAL if n <= k, k or D or leaf_max out of range, rounds < 1,
 * a NULL pointer, or non-finite input.
 */
KNNG_API int knng_build(const float *data, int64_t n, int D, int k, int leaf_max, int rounds,
               uint64_t seed, int32_t *out_ids, float *out_dists);

/*
 * Build with every parameter (Sec. 3.1 / Alg. 1, then p->refine_rounds
 * neighbour-of-neighbour rounds, Sec. 1 prior art) on `stream`.
 * Same outputs and errors as knng_build; tree_passes may be 0 only when
 * refine_rounds is 0 too (the graph is then all empty slots).
 */
KNNG_API int knng_build_ex(const float *data, int64_t n, int D, const knng_params *p,
                  int32_t *out_ids, float *out_dists, void *stream);

/* One independent instance of a batched build. */
typedef struct knng_instance {
    const float *data;   /* n x D FP32 row-major, host or device */
    int64_t n;           /* points (> k) */
    int D;               /* dims (1 .. 4096) */
    int leaf_max;        /* this instance's cluster bound; 0: p->leaf_max */
    int32_t *out_ids;    /* n x k, ids local to the instance */
    float *out_dists;    /* n x k */
    int twomeans_iters;  /* this instance's Lloyd iterations per split; 0: p->twomeans_iters.  Instances of
                            one D must agree (KNNG_EINVAL otherwise): they share one forest */
} knng_instance;

/*
 * Many independent graphs in one build (Sec. 3.1 / Alg. 1 and the
 * refinement, per instance; the paper builds one graph at a time, so the
 * batching is this library's).  Instances of equal D run as one forest:
 * every stage is one launch over all their trees (each stops splitting at its
 * own depth, with the seeds it would get alone), then one leaf stage and
 * shared refinement rounds over all their points.  Each instance's result is
 * exactly the one knng_build_ex gives it alone with the same parameters.
 * inst[i].data must not overlap any output.  Errors: as knng_build_ex, for
 * any instance (nothing is written then), or n_inst < 1, or the points of one
 * D together reach 2^31 rows.
 */
KNNG_API int knng_build_batched(int n_inst, const knng_instance *inst, const knng_params *p, void *stream);

/*
 * A build (as knng_build_ex: Sec. 3.1 / Alg. 1, then the refinement rounds of
 * Sec. 1) recorded once into a CUDA graph and replayed at will.  The paper
 * has no counterpart; recording removes the host's part of every launch.
 * data, out_ids and out_dists are device buffers or page-locked host buffers
 * (cudaHostAlloc, cudaMallocHost, cudaHostRegister; pageable memory is refused
 * with KNNG_EINVAL); they are bound at creation, so a replay rebuilds the
 * graph of whatever `data` then holds into the same outputs.  A host buffer
 * gets a workspace copy: each replay copies data in at its start and the lists
 * out at its end, inside the graph, so a replay followed by a wait on the
 * stream leaves the lists in host memory.  The plan owns its workspace
 * (device memory for the whole build; the offer buffer is sized for one chunk
 * per round up to 48 GB, since a graph cannot read offer counts back) until
 * knng_plan_destroy.
 * Recording makes no host reads of the data: every choice the host would make
 * from it (the join kind, the chunk sizes) is made on the device instead, and
 * the result equals knng_build_ex's bit for bit.
 *   knng_plan_create: validates, synchronizes `stream` (so that inputs queued
 *                     on it are ready), allocates, records; *out_plan is NULL
 *                     on error.
 *   knng_plan_launch: enqueues one replay on `stream`.
 *   knng_plan_check:  waits for `stream`, then reports the last replay's
 *                     device status (KNNG_EINVAL for non-finite data, ...).
 *   knng_plan_destroy: frees everything (NULL is ignored).
 * Replays of one plan must not overlap in time (they share the workspace).
 */
typedef struct knng_plan knng_plan;
KNNG_API int knng_plan_create(const float *data, int64_t n, int D, const knng_params *p, int32_t *out_ids,
                              float *out_dists, void *stream, knng_plan **out_plan);
/*
 * The batched form (as knng_build_batched) recorded the same way: one graph
 * for every instance, all instances' data and outputs device buffers bound at
 * creation (the instance array itself is read only while recording).  One
 * replay equals one knng_build_batched call on the same buffers, bit for bit.
 * The offer buffers of the D groups share the 48 GB equally.
 */
KNNG_API int knng_plan_create_batched(int n_inst, const knng_instance *inst, const knng_params *p, void *stream,
                                      knng_plan **out_plan);
KNNG_API int knng_plan_launch(knng_plan *plan, void *stream);
/* Kernel launches one replay makes (the recorded graph's kernel nodes); -1 on error. */
KNNG_API int64_t knng_plan_kernels(knng_plan *plan);
KNNG_API int knng_plan_check(knng_plan *plan, void *stream);
KNNG_API void knng_plan_destroy(knng_plan *plan);

/*
 * Refinement only: p->refine_rounds local-join rounds (Jacobi: every offer of
 * a round comes from the graph as it stood before the round) applied to the
 * graph (ids_inout, dists_inout), which must satisfy the graph conventions and
 * hold canonical distances.  Uses p->k (must equal the graph's k) and
 * p->join_mode.  Also serves to resume a saved graph.
 */
KNNG_API int knng_refine(const float *data, int64_t n, int D, const knng_params *p,
                int32_t *ids_inout, float *dists_inout, void *stream);

/*
 * The partition of tree pass `pass` (Sec. 3.1: recursive two-means
 * bisection), exactly as knng_build_ex computes it for the same seed,
 * leaf_max and twomeans_iters.  out_perm: n ids, the clusters contiguous,
 * ids ascending inside a cluster.  out_leaf_offsets: 2^L + 1 offsets into
 * out_perm, L = the least depth with ceil(n / 2^L) <= leaf_max; cluster c is
 * out_perm[off[c] .. off[c+1]).  Use knng_tree_depth to size it.
 */
KNNG_API int knng_partition(const float *data, int64_t n, int D, int leaf_max, int twomeans_iters,
                   uint64_t seed, int pass, int32_t *out_perm, int64_t *out_leaf_offsets,
                   void *stream);

/* Depth L of the balanced tree for n points and threshold leaf_max (-1 if invalid). */
KNNG_API int knng_tree_depth(int64_t n, int leaf_max);

/*
 * Parity hook of the low-precision leaf stage (Alg. 1's pairwise distances
 * inside one cluster, computed from a low-precision copy): for the m points
 * of `data` (m x D, one cluster of 2..256 points, row-major FP32), the
 * approximate squared distances d^ (out_dhat, m x m row-major FP32, diagonal
 * included) exactly as the tensor-core leaf kernel forms them for
 * `precision` (KNNG_BF16, KNNG_FP16 or KNNG_FP8), and the quantised copy they
 * come from: out_q (m x D FP32) holds the 16-bit values, or for FP8 the
 * unscaled E4M3 values q; out_scale (m) the row scales s (x~ = s q; 1 for the
 * 16-bit forms); out_nrm (m) the FP32 squared norms ||x~||^2 the kernel uses;
 * out_err (m) the upper bounds e >= ||x - x~|| of the certificate.  For
 * tests of the certificate's error bound against the hardware's arithmetic.
 * Pointers host or device (all caller-owned).  KNNG_EINVAL for m outside
 * [2, 256], a non-finite value, or a precision without a low-precision copy;
 * KNNG_ECUDA when the tensor-core kernel cannot run for this D.
 */
KNNG_API int knng_leaf_dhat(const float *data, int64_t m, int D, int precision, float *out_dhat,
                            float *out_q, float *out_scale, float *out_nrm, float *out_err, void *stream);

/*
 * The leaf stage of Alg. 1 on a given partition: for every cluster and every
 * pair <i, j> in it, i != j, update G[i] and G[j] with d(x_i, x_j).
 * perm / leaf_offsets as knng_partition returns them (any partition into
 * clusters of 2..256 points is accepted).  (ids_inout, dists_inout) is the
 * graph G, updated in place.
 */
KNNG_API int knng_leaf_update(const float *data, int64_t n, int D, int k, const int32_t *perm,
                     const int64_t *leaf_offsets, int64_t n_leaves, int32_t *ids_inout,
                     float *dists_inout, void *stream);

/*
 * The enhanced hill-climbing search of Sec. 3.2 (Alg. 2) over a kNN graph, for
 * a batch of m queries.  For query q (row q of `queries`, m x D) the rank list
 * R starts as its seeds (row q of `seeds`, m x s ids; ids outside [0, n) are
 * skipped, repeats count once) with their distances; then, t0 times, every
 * neighbour in `graph_ids` (n x k ids, -1 = empty; e.g. knng_build's output)
 * of the ks first entries of R by (d, id), as R stands at the iteration's
 * start, that has not been visited yet (its distance computed) is visited and
 * added to R.  out_ids, out_dists (m x ks): the ks first entries of R by
 * (d, id), canonical FP32 squared l2, empty slots id -1, d +inf.
 * 1 <= ks <= 32; seeds are the caller's (random ones, as the paper's baseline
 * draws, or any other choice).  Pointers host or device; KNNG_EINVAL on bad
 * sizes or a non-finite input.
 */
KNNG_API int knng_search(const float *data, int64_t n, int D, const int32_t *graph_ids, int k,
                         const float *queries, int64_t m, const int32_t *seeds, int s, int t0, int ks,
                         int32_t *out_ids, float *out_dists, void *stream);

/*
 * Residue vector quantisation vocabularies (Sec. 4.1, Eqn. 1), two stages.
 * Stage 1 (W1 words) is trained on the n points of `data` (n x D FP32,
 * row-major), stage 2 (W2 words) on their residues x - w1[c1(x)] (FP32
 * difference, c1 the nearest stage-1 word after training).  Each stage is
 * Lloyd's k-means for `iters` iterations from W initial words: word c starts
 * as vector p_c, p_c = lo_c + SplitMix64(SplitMix64(seed ^ (stage << 32)) ^ c)
 * mod (hi_c - lo_c) inside the c-th of W equal strata [lo_c, hi_c) of the
 * vectors.  An iteration assigns each vector to its nearest word (canonical
 * FP32 squared l2: dims ascending, t = x - w, acc = fmaf(t, t, acc); ties to
 * the smaller word index) and sets every word with members to the FP64 mean of
 * its members summed in ascending vector order, rounded to FP32; a word
 * without members keeps its value.  1 <= W1, W2 <= 256, both <= n; iters >= 0.
 * Outputs words1 (W1 x D) and words2 (W2 x D), FP32.  Pointers host or
 * device.  KNNG_EINVAL on bad sizes or non-finite data.
 */
KNNG_API int knng_rvq_train(const float *data, int64_t n, int D, int W1, int W2, int iters, uint64_t seed,
                            float *words1, float *words2, void *stream);

/*
 * The inverted index of Sec. 4.2: each point's codes (c1 = nearest stage-1
 * word, c2 = nearest stage-2 word to its residue; same distance and ties as
 * knng_rvq_train) into `codes` (n x 2 int32: c1, c2), and the lists keyed by
 * I = c1 * W2 + c2 as CSR: list I holds list_ids[list_offsets[I] ..
 * list_offsets[I + 1]) in ascending id order (list_offsets: W1 * W2 + 1
 * int32; list_ids: n int32).  1 <= W1, W2 <= 256.  Pointers host or device.
 */
KNNG_API int knng_rvq_index(const float *data, int64_t n, int D, const float *words1, int W1,
                            const float *words2, int W2, int32_t *codes, int32_t *list_offsets,
                            int32_t *list_ids, void *stream);

/*
 * Seeds of the graph search (Alg. 2) from the inverted index (Sec. 4.2,
 * Eqns. 2 and 3), for m queries (m x D).  With canonical dot products
 * (acc = fmaf(a_j, b_j, acc), dims ascending) in FP32:
 *   term1(c1)     = fmaf(-2, q.w1, q.q) + |w1|^2
 *   term2(c1, c2) = fmaf(-2, q.w2, fmaf(2, w1.w2, |w2|^2))
 *   d(q, I)       = term1 + term2          (-0 normalised to +0)
 * the probe1 stage-1 words with the least (term1, c1) are kept (the cascaded
 * pruning), their W2 keys each are ranked by (d, I), and the seeds are the ids
 * of those lists in that order (ascending inside a list), the first s; -1 pads
 * a query whose lists hold fewer.  seeds: m x s int32.  list_offsets /
 * list_ids as knng_rvq_index writes them, n = the number of list ids;
 * offsets that are negative, decreasing or above n give KNNG_EINVAL.
 * 1 <= probe1 <= W1, probe1 * W2 <= 8192, m <= 2^31 - 1 (one CTA per
 * query).  Pointers host or device.
 */
KNNG_API int knng_rvq_seeds(const float *words1, int W1, const float *words2, int W2, int D,
                            const int32_t *list_offsets, const int32_t *list_ids, int64_t n,
                            const float *queries, int64_t m, int probe1, int s, int32_t *seeds, void *stream);

/*
 * Exact k nearest neighbours (the problem statement of Sec. 1, each listed
 * point as a query against the other n - 1) of the s rows listed in `sample`
 * (all rows in order when sample is NULL, then s must equal n), canonical FP32
 * distances, ties by id.  out_ids, out_dists: s x k.  Ground truth for recall.
 */
KNNG_API int knng_exact(const float *data, int64_t n, int D, int k, const int32_t *sample, int64_t s,
               int32_t *out_ids, float *out_dists, void *stream);

/*
 * Recall of a graph (ids, dists: n x k) on the sampled rows against their
 * exact lists (gt_ids, gt_dists: s x k, as knng_exact returns them).
 * out_recall_ids: mean over rows of |G[i] & GT[i]| / k.
 * out_recall_tie: mean over rows of the share of real entries of G[i] whose
 * distance is <= the k-th exact distance of row i (counts any correct
 * neighbour among equal distances).  out_* are host pointers.
 */
KNNG_API int knng_recall(const int32_t *ids, const float *dists, const int32_t *gt_ids,
                const float *gt_dists, const int32_t *sample, int64_t s, int k,
                double *out_recall_ids, double *out_recall_tie, void *stream);

/*
 * knng_exact without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * where they need ground-truth lists -- code running under a memory manager
 * that owns all device memory (a cudaMalloc would fail or escape its
 * accounting), or a latency-bound loop where an allocation's implicit
 * synchronisation is not allowed.
 *
 * Same result as knng_exact for the same arguments.  Differences:
 *   - data, sample, out_ids and out_dists must be device pointers (no host
 *     staging); sample is required (s >= 1);
 *   - s * k must not exceed 262144 (KNNG_EINVAL otherwise): the scratch is a
 *     fixed 2 MiB static device array (plus one status word) that every GPU
 *     loading the library holds until the process exits;
 *   - the first call on each device looks up the scratch's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture on the device;
 *   - every call on a device shares the one scratch: calls whose work
 *     overlaps on the GPU (other streams, other host threads) race and must
 *     be serialised by the caller.  The scratch keeps the last call's
 *     contents; each call clears the status word it needs at zero and
 *     overwrites the lists in full.
 * The call is synchronous with respect to `stream`.
 */
KNNG_API int knng_exact_noalloc(const float *data, int64_t n, int D, int k, const int32_t *sample,
                                int64_t s, int32_t *out_ids, float *out_dists, void *stream);

/* Message of the last failing call on this thread ("" if none). */
KNNG_API const char *knng_last_error(void);

/* Peak device workspace (bytes) knng_build_ex allocates for these arguments. */
KNNG_API size_t knng_workspace_bytes(int64_t n, int D, const knng_params *p);

/*
 * Kernel statistics (process-wide).  While enabled, every kernel launch is
 * counted per kernel name together with its algorithmic bytes and flops (the
 * data the method must move or compute, not what the hardware moved); with
 * timing on, CUDA events on the launching stream bracket each launch and the
 * summed device time is recorded too.
 */
typedef struct knng_kernel_stat {
    char name[32];
    uint64_t launches;
    double ms;       /* summed device time, 0 when timing is off */
    double bytes;    /* summed algorithmic bytes */
    double flops;    /* summed algorithmic flops */
    double items;    /* summed work items where counted (k5_join: offers that passed the filter) */
} knng_kernel_stat;

KNNG_API int knng_stats_enable(int on, int timing);
KNNG_API void knng_stats_reset(void);
KNNG_API int knng_stats_count(void);
KNNG_API int knng_stats_get(int index, knng_kernel_stat *out);

#ifdef __cplusplus
}
#endif

#endif /* KNNG_H */
