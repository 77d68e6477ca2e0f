/*
 * knng_oracle.c -- CPU oracle for kNN-graph construction by two-means-tree
 * partitioning, exhaustive comparison inside each cluster, and
 * neighbour-of-neighbour refinement (Zhao, Yang, Deng, "Scalable Nearest
 * Neighbor Search based on kNN Graph", arXiv 1701.08475, Sec. 3.1, Alg. 1;
 * refinement: the nearest-neighbour-descent prior art cited in Sec. 1, also
 * in its sampled form), and
 * the enhanced hill-climbing search over the built graph (Sec. 3.2, Alg. 2),
 * and the residue-quantisation inverted index that seeds it (Sec. 4).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code,
 * header, table or helper with the CUDA library and never calls it.
 *
 * Plain, slow and single-threaded on purpose.  Build with
 *   gcc -O2 -ffp-contract=off -fPIC -shared
 * so every floating-point operation is the one written here; a fused
 * multiply-add appears only where fmaf() is called explicitly.
 *
 * Readings of the paper used here (the paper leaves these open):
 *  - metric: squared l2 (Sec. 1 allows l1 or l2; squared l2 orders pairs
 *    exactly as l2 does);
 *  - canonical FP32 distance: acc = 0; for j ascending: t = x_j - y_j;
 *    acc = fmaf(t, t, acc).  Symmetric bit for bit, since (x-y)^2 == (y-x)^2;
 *  - ties are broken by the smaller id; lists hold unique ids, sorted by
 *    (d, id); empty slots hold id -1 with d = +inf and sort last;
 *  - two-means split (Sec. 3.1, Alg. 1 "apply two means clustering") is a
 *    balanced Lloyd 2-means: the first floor(m/2) points by (s, id) go left,
 *    where s = x . (c1 - c0) orders points exactly as
 *    ||x - c0||^2 - ||x - c1||^2 does (the two differ by a factor 2 and a
 *    per-segment constant, which a median cut cannot see);
 *  - centroids are FP64 means of FP32 points (summed in ascending id order),
 *    rounded to FP32;
 *  - uniform depth: every segment at a level splits, so leaf sizes are
 *    floor/ceil(n / 2^L), L the least level with ceil(n / 2^L) <= leaf_max;
 *  - initial centroids: the points at positions h and h' of the segment
 *    (segments hold their ids in ascending order), h and h' drawn from a
 *    SplitMix64 hash of (pass seed, level, segment index);
 *  - "visited" pairs (Alg. 1) are not skipped: re-evaluating a pair gives the
 *    same canonical distance and cannot change a list;
 *  - refinement round (Jacobi): reverse lists R[i] capped at the k closest by
 *    (d, id); N_i = G_old[i] (mode 0) or G_old[i] + R[i] (mode 1); every
 *    unordered pair {u, v} of N_i with u != v offers v to u and u to v with
 *    the canonical distance; G_new[u] = first k unique of G_old[u] + offers.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): one output step for  */
/* state z, i.e. advance by the golden-ratio increment, then mix.     */
/* ------------------------------------------------------------------ */
uint64_t orc_splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Seed of tree pass p. */
uint64_t orc_pass_seed(uint64_t seed, int pass)
{
    return orc_splitmix64(seed ^ (uint64_t)pass);
}

/* Positions (h, h2) of the two initial centroids of segment `seg` at
 * `level`, for a segment of m >= 2 points.  h2 != h. */
void orc_init_positions(uint64_t pass_seed, int level, int64_t seg, int64_t m,
                        int64_t *h, int64_t *h2)
{
    uint64_t a = orc_splitmix64(orc_splitmix64(orc_splitmix64(pass_seed) ^ (uint64_t)level) ^ (uint64_t)seg);
    uint64_t b = orc_splitmix64(a);
    *h = (int64_t)(a % (uint64_t)m);
    *h2 = (*h + 1 + (int64_t)(b % (uint64_t)(m - 1))) % m;
}

/* ------------------------------------------------------------------ */
/* Distances                                                          */
/* ------------------------------------------------------------------ */
float orc_dist_f32(const float *x, const float *y, int D)
{
    float acc = 0.0f;
    for (int j = 0; j < D; ++j) {
        float t = x[j] - y[j];
        acc = fmaf(t, t, acc);
    }
    return acc;
}

double orc_dist_f64(const float *x, const float *y, int D)
{
    double acc = 0.0;
    for (int j = 0; j < D; ++j) {
        double t = (double)x[j] - (double)y[j];
        acc += t * t;
    }
    return acc;
}

/* ------------------------------------------------------------------ */
/* Sorted, unique, bounded (d, id) lists                              */
/* ------------------------------------------------------------------ */
/* (d, id) order; an empty slot (id -1, d +inf) is greater than every entry
 * because ids compare as unsigned. */
static int key_less(float da, int32_t ia, float db, int32_t ib)
{
    if (da < db) return 1;
    if (da > db) return 0;
    return (uint32_t)ia < (uint32_t)ib;
}

static void list_clear(int32_t *ids, float *d, int k)
{
    for (int t = 0; t < k; ++t) { ids[t] = -1; d[t] = INFINITY; }
}

/* Offer (cd, cid) to the list: keep the k smallest unique ids by (d, id). */
void orc_list_insert(int32_t *ids, float *d, int k, float cd, int32_t cid)
{
    if (cid < 0) return;
    if (!key_less(cd, cid, d[k - 1], ids[k - 1])) return;
    for (int t = 0; t < k; ++t)
        if (ids[t] == cid) return;
    int pos = 0;
    while (!key_less(cd, cid, d[pos], ids[pos])) ++pos;
    for (int t = k - 1; t > pos; --t) { ids[t] = ids[t - 1]; d[t] = d[t - 1]; }
    ids[pos] = cid;
    d[pos] = cd;
}

static int key_less64(double da, int32_t ia, double db, int32_t ib)
{
    if (da < db) return 1;
    if (da > db) return 0;
    return (uint32_t)ia < (uint32_t)ib;
}

static void list_insert64(int32_t *ids, double *d, int k, double cd, int32_t cid)
{
    if (!key_less64(cd, cid, d[k - 1], ids[k - 1])) return;
    int pos = 0;
    while (!key_less64(cd, cid, d[pos], ids[pos])) ++pos;
    for (int t = k - 1; t > pos; --t) { ids[t] = ids[t - 1]; d[t] = d[t - 1]; }
    ids[pos] = cid;
    d[pos] = cd;
}

/* ------------------------------------------------------------------ */
/* Exact kNN graph (the problem statement of Sec. 1, every point as a  */
/* query against the other n - 1).                                    */
/* ------------------------------------------------------------------ */
/* Rows of `sample` (or all n rows when sample == NULL), canonical FP32
 * distances, ties by id.  out: s x k. */
int orc_exact_f32(const float *X, int64_t n, int D, int k,
                  const int32_t *sample, int64_t s,
                  int32_t *out_ids, float *out_d)
{
    if (!sample) s = n;
    for (int64_t r = 0; r < s; ++r) {
        int64_t i = sample ? sample[r] : r;
        int32_t *li = out_ids + r * k;
        float *ld = out_d + r * k;
        list_clear(li, ld, k);
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            orc_list_insert(li, ld, k, orc_dist_f32(X + i * D, X + j * D, D), (int32_t)j);
        }
    }
    return 0;
}

/* Same with FP64 distances (the error reference). */
int orc_exact_f64(const float *X, int64_t n, int D, int k,
                  const int32_t *sample, int64_t s,
                  int32_t *out_ids, double *out_d)
{
    if (!sample) s = n;
    for (int64_t r = 0; r < s; ++r) {
        int64_t i = sample ? sample[r] : r;
        int32_t *li = out_ids + r * k;
        double *ld = out_d + r * k;
        for (int t = 0; t < k; ++t) { li[t] = -1; ld[t] = INFINITY; }
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            list_insert64(li, ld, k, orc_dist_f64(X + i * D, X + j * D, D), (int32_t)j);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Two-means tree (Sec. 3.1: bisect repeatedly with two-means until    */
/* every cluster is below the threshold; Alg. 1 "apply two means").    */
/* ------------------------------------------------------------------ */
int orc_tree_depth(int64_t n, int leaf_max)
{
    int L = 0;
    while ((n + ((int64_t)1 << L) - 1) / ((int64_t)1 << L) > leaf_max) ++L;
    return L;
}

typedef struct { float s; int32_t id; } proj_t;

static int proj_cmp(const void *a, const void *b)
{
    const proj_t *x = a, *y = b;
    if (x->s < y->s) return -1;
    if (x->s > y->s) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

static int id_cmp(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* FP64 mean of the listed points, rounded to FP32. */
static void mean_of(const float *X, int D, const int32_t *ids, int64_t cnt,
                    double *acc, float *c)
{
    for (int j = 0; j < D; ++j) acc[j] = 0.0;
    for (int64_t t = 0; t < cnt; ++t)
        for (int j = 0; j < D; ++j) acc[j] += (double)X[(int64_t)ids[t] * D + j];
    for (int j = 0; j < D; ++j) c[j] = (float)(acc[j] / (double)cnt);
}

/* Split one segment (ids ascending, m >= 2) into its left half
 * (floor(m/2) ids) and right half, each written back in ascending order. */
static void split_segment(const float *X, int D, int32_t *seg_ids, int64_t m,
                          int iters, uint64_t pass_seed, int level, int64_t seg,
                          proj_t *pr, float *c0, float *c1, float *w, double *acc,
                          int32_t *tmp)
{
    int64_t K = m / 2, h, h2;
    orc_init_positions(pass_seed, level, seg, m, &h, &h2);
    memcpy(c0, X + (int64_t)seg_ids[h] * D, sizeof(float) * D);
    memcpy(c1, X + (int64_t)seg_ids[h2] * D, sizeof(float) * D);
    for (int it = 0; it <= iters; ++it) {
        for (int j = 0; j < D; ++j) w[j] = c1[j] - c0[j];
        for (int64_t t = 0; t < m; ++t) {
            const float *x = X + (int64_t)seg_ids[t] * D;
            float a = 0.0f;
            for (int j = 0; j < D; ++j) a = fmaf(x[j], w[j], a);
            pr[t].s = a + 0.0f;   /* -0 and +0 are one key */
            pr[t].id = seg_ids[t];
        }
        qsort(pr, (size_t)m, sizeof(proj_t), proj_cmp);
        for (int64_t t = 0; t < m; ++t) tmp[t] = pr[t].id;
        qsort(tmp, (size_t)K, sizeof(int32_t), id_cmp);
        qsort(tmp + K, (size_t)(m - K), sizeof(int32_t), id_cmp);
        if (it == iters) break;
        mean_of(X, D, tmp, K, acc, c0);
        mean_of(X, D, tmp + K, m - K, acc, c1);
    }
    memcpy(seg_ids, tmp, sizeof(int32_t) * (size_t)m);
}

/* Partition of tree pass `pass`: out_perm (n ids, leaves contiguous, ids
 * ascending inside a leaf), out_leaf_offsets (2^L + 1 offsets).
 * Returns the depth L, or -1 on bad arguments / allocation failure. */
int orc_partition(const float *X, int64_t n, int D, int leaf_max, int iters,
                  uint64_t seed, int pass, int32_t *out_perm, int64_t *out_leaf_offsets)
{
    if (n < 1 || D < 1 || leaf_max < 2 || iters < 0) return -1;
    int L = orc_tree_depth(n, leaf_max);
    uint64_t ps = orc_pass_seed(seed, pass);
    int64_t nleaf = (int64_t)1 << L;
    int64_t *off = malloc(sizeof(int64_t) * (size_t)(nleaf + 1));
    int64_t *nxt = malloc(sizeof(int64_t) * (size_t)(nleaf + 1));
    proj_t *pr = malloc(sizeof(proj_t) * (size_t)n);
    int32_t *tmp = malloc(sizeof(int32_t) * (size_t)n);
    float *c0 = malloc(sizeof(float) * (size_t)D), *c1 = malloc(sizeof(float) * (size_t)D);
    float *w = malloc(sizeof(float) * (size_t)D);
    double *acc = malloc(sizeof(double) * (size_t)D);
    if (!off || !nxt || !pr || !tmp || !c0 || !c1 || !w || !acc) {
        free(off); free(nxt); free(pr); free(tmp); free(c0); free(c1); free(w); free(acc);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i) out_perm[i] = (int32_t)i;
    off[0] = 0;
    off[1] = n;
    for (int level = 0; level < L; ++level) {
        int64_t nseg = (int64_t)1 << level;
        for (int64_t sg = 0; sg < nseg; ++sg) {
            int64_t a = off[sg], m = off[sg + 1] - off[sg];
            split_segment(X, D, out_perm + a, m, iters, ps, level, sg, pr, c0, c1, w, acc, tmp);
            nxt[2 * sg] = a;
            nxt[2 * sg + 1] = a + m / 2;
        }
        nxt[2 * nseg] = n;
        memcpy(off, nxt, sizeof(int64_t) * (size_t)(2 * nseg + 1));
    }
    memcpy(out_leaf_offsets, off, sizeof(int64_t) * (size_t)(nleaf + 1));
    free(off); free(nxt); free(pr); free(tmp); free(c0); free(c1); free(w); free(acc);
    return L;
}

/* ------------------------------------------------------------------ */
/* Leaf stage (Alg. 1, inner loops): every pair <i, j>, i != j, of a   */
/* cluster updates G[i] and G[j] with d(x_i, x_j).                     */
/* ------------------------------------------------------------------ */
int orc_leaf_update(const float *X, int64_t n, int D, int k,
                    const int32_t *perm, const int64_t *leaf_offsets, int64_t n_leaves,
                    int32_t *ids, float *dists)
{
    (void)n;
    for (int64_t l = 0; l < n_leaves; ++l) {
        for (int64_t a = leaf_offsets[l]; a < leaf_offsets[l + 1]; ++a) {
            for (int64_t b = a + 1; b < leaf_offsets[l + 1]; ++b) {
                int32_t i = perm[a], j = perm[b];
                float d = orc_dist_f32(X + (int64_t)i * D, X + (int64_t)j * D, D);
                orc_list_insert(ids + (int64_t)i * k, dists + (int64_t)i * k, k, d, j);
                orc_list_insert(ids + (int64_t)j * k, dists + (int64_t)j * k, k, d, i);
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Refinement round (neighbour-of-neighbour local join, Jacobi form).  */
/* mode 0: N_i = G_old[i];  mode 1: N_i = G_old[i] + R[i].            */
/* ------------------------------------------------------------------ */
int orc_reverse_lists(int64_t n, int k, const int32_t *ids, const float *dists,
                      int32_t *rev_ids, float *rev_d)
{
    for (int64_t i = 0; i < n; ++i) list_clear(rev_ids + i * k, rev_d + i * k, k);
    for (int64_t j = 0; j < n; ++j)
        for (int t = 0; t < k; ++t) {
            int32_t i = ids[j * k + t];
            if (i < 0) continue;
            orc_list_insert(rev_ids + (int64_t)i * k, rev_d + (int64_t)i * k, k,
                            dists[j * k + t], (int32_t)j);
        }
    return 0;
}

int orc_refine_round(const float *X, int64_t n, int D, int k, int mode,
                     int32_t *ids, float *dists)
{
    size_t nk = (size_t)n * (size_t)k;
    int32_t *old_ids = malloc(sizeof(int32_t) * nk);
    float *old_d = malloc(sizeof(float) * nk);
    int32_t *rev_ids = mode ? malloc(sizeof(int32_t) * nk) : NULL;
    float *rev_d = mode ? malloc(sizeof(float) * nk) : NULL;
    int32_t *memb = malloc(sizeof(int32_t) * (size_t)(2 * k));
    if (!old_ids || !old_d || !memb || (mode && (!rev_ids || !rev_d))) {
        free(old_ids); free(old_d); free(rev_ids); free(rev_d); free(memb);
        return -1;
    }
    memcpy(old_ids, ids, sizeof(int32_t) * nk);
    memcpy(old_d, dists, sizeof(float) * nk);
    if (mode) orc_reverse_lists(n, k, old_ids, old_d, rev_ids, rev_d);
    for (int64_t i = 0; i < n; ++i) {
        int cnt = 0;
        for (int t = 0; t < k; ++t)
            if (old_ids[i * k + t] >= 0) memb[cnt++] = old_ids[i * k + t];
        if (mode)
            for (int t = 0; t < k; ++t)
                if (rev_ids[i * k + t] >= 0) memb[cnt++] = rev_ids[i * k + t];
        for (int a = 0; a < cnt; ++a)
            for (int b = a + 1; b < cnt; ++b) {
                int32_t u = memb[a], v = memb[b];
                if (u == v) continue;
                float d = orc_dist_f32(X + (int64_t)u * D, X + (int64_t)v * D, D);
                orc_list_insert(ids + (int64_t)u * k, dists + (int64_t)u * k, k, d, v);
                orc_list_insert(ids + (int64_t)v * k, dists + (int64_t)v * k, k, d, u);
            }
    }
    free(old_ids); free(old_d); free(rev_ids); free(rev_d); free(memb);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Sampled refinement round: nearest-neighbour descent with sampling,  */
/* the prior art Sec. 1 cites (Dong, Charikar and Li, WWW 2011), in    */
/* Jacobi form.  flags[i*k + t] = 1 marks entry t of G[i] as new (not  */
/* yet joined), 0 as old.                                             */
/*  1. per node v: old[v] = its entries flagged old; new[v] = the ms    */
/*     entries flagged new with the least priority h(v, u) (all of     */
/*     them when fewer), which are then flagged old;                   */
/*  2. reverse lists: rold[u] = {v : u in old[v]}, rnew[u] = {v : u in  */
/*     new[v]}, each cut to the ms members with the least h(u, v);     */
/*  3. per v: Nn = new[v] + rnew[v], No = old[v] + rold[v] without the  */
/*     ids of Nn; every pair of Nn and every pair of Nn x No offers    */
/*     each member to the other with the canonical distance;           */
/*  4. G[u] becomes the first k unique of G[u] and its offers; an id   */
/*     that was not in G[u] enters flagged new, the others keep their  */
/*     flags.                                                          */
/* Priority of member u of node v: the upper 32 bits of                */
/* SplitMix64(SplitMix64(seed ^ round) ^ (v << 32 | u)) above the 32   */
/* bits of u, so one 64-bit key orders by hash, then by id.  Returns   */
/* the entries that entered a list (NN-descent's update count), or < 0 */
/* on bad arguments.                                                   */
/* ------------------------------------------------------------------ */
uint64_t orc_sample_prio(uint64_t seed, int round, int64_t v, int32_t u)
{
    uint64_t h = orc_splitmix64(orc_splitmix64(seed ^ (uint64_t)(uint32_t)round) ^
                                (((uint64_t)v << 32) | (uint32_t)u));
    return (h & 0xFFFFFFFF00000000ull) | (uint32_t)u;
}

typedef struct { uint64_t h; int32_t id; } prio_t;

static int prio_cmp(const void *a, const void *b)
{
    const prio_t *x = (const prio_t *)a, *y = (const prio_t *)b;
    if (x->h != y->h) return x->h < y->h ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* Keep the ms members of ids[0..cnt) with the least h(owner, id). */
static int sample_least(int32_t *ids, int cnt, int ms, uint64_t seed, int round, int64_t owner, prio_t *tmp)
{
    if (cnt <= ms) return cnt;
    for (int a = 0; a < cnt; ++a) {
        tmp[a].h = orc_sample_prio(seed, round, owner, ids[a]);
        tmp[a].id = ids[a];
    }
    qsort(tmp, (size_t)cnt, sizeof(prio_t), prio_cmp);
    for (int a = 0; a < ms; ++a) ids[a] = tmp[a].id;
    return ms;
}

static int has_id(const int32_t *ids, int cnt, int32_t id)
{
    for (int a = 0; a < cnt; ++a)
        if (ids[a] == id) return 1;
    return 0;
}

int64_t orc_refine_sampled(const float *X, int64_t n, int D, int k, int ms, uint64_t seed, int round,
                           int32_t *ids, float *dists, unsigned char *flags)
{
    if (n < 1 || D < 1 || k < 1 || ms < 0) return -1;
    size_t nk = (size_t)n * (size_t)k;
    int32_t *snap = malloc(sizeof(int32_t) * nk);           /* G before the round */
    unsigned char *isnew = malloc(nk);                      /* 1: in new[v] (sampled) */
    int64_t *co = calloc((size_t)n + 1, sizeof(int64_t)), *cn = calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *ro = malloc(sizeof(int32_t) * (nk > 0 ? nk : 1)), *rn = malloc(sizeof(int32_t) * (nk > 0 ? nk : 1));
    int32_t *nn = malloc(sizeof(int32_t) * (size_t)(k + 2 * ms + 1)), *no = malloc(sizeof(int32_t) * (size_t)(k + ms + 1));
    int32_t *buf = malloc(sizeof(int32_t) * (nk > 0 ? nk : 1));
    prio_t *tmp = malloc(sizeof(prio_t) * (nk > 0 ? nk : 1));
    int64_t *fo = malloc(sizeof(int64_t) * ((size_t)n + 1)), *fn = malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!snap || !isnew || !co || !cn || !ro || !rn || !nn || !no || !buf || !tmp || !fo || !fn) {
        free(snap); free(isnew); free(co); free(cn); free(ro); free(rn); free(nn); free(no); free(buf);
        free(tmp); free(fo); free(fn);
        return -2;
    }
    memcpy(snap, ids, sizeof(int32_t) * nk);
    memset(isnew, 0, nk);
    /* 1. samples of the new entries; old[v] = entries flagged old before */
    for (int64_t v = 0; v < n; ++v) {
        int cnt = 0;
        for (int t = 0; t < k; ++t)
            if (snap[v * k + t] >= 0 && flags[v * k + t]) buf[cnt++] = snap[v * k + t];
        cnt = sample_least(buf, cnt, ms, seed, round, v, tmp);
        for (int t = 0; t < k; ++t)
            if (snap[v * k + t] >= 0 && flags[v * k + t] && has_id(buf, cnt, snap[v * k + t])) {
                isnew[v * k + t] = 1;
                flags[v * k + t] = 0;
            }
    }
    /* 2. reverse lists (CSR; cut to ms per node below).  An entry is in
     * new[v] when isnew is set, in old[v] when it is flagged old and was
     * not sampled now, and in neither when it stays new unsampled. */
    for (int64_t v = 0; v < n; ++v)
        for (int t = 0; t < k; ++t) {
            int32_t u = snap[v * k + t];
            if (u < 0) continue;
            if (isnew[v * k + t]) cn[u + 1]++;
            else if (!flags[v * k + t]) co[u + 1]++;
        }
    for (int64_t u = 0; u < n; ++u) { co[u + 1] += co[u]; cn[u + 1] += cn[u]; }
    memcpy(fo, co, sizeof(int64_t) * ((size_t)n + 1));
    memcpy(fn, cn, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t v = 0; v < n; ++v)
        for (int t = 0; t < k; ++t) {
            int32_t u = snap[v * k + t];
            if (u < 0) continue;
            if (isnew[v * k + t]) rn[fn[u]++] = (int32_t)v;
            else if (!flags[v * k + t]) ro[fo[u]++] = (int32_t)v;
        }
    int64_t changed = 0;
    for (int64_t v = 0; v < n; ++v) {
        /* 3. members */
        int cn_ = 0, co_ = 0;
        for (int t = 0; t < k; ++t)
            if (isnew[v * k + t]) nn[cn_++] = snap[v * k + t];
        int rc = (int)(cn[v + 1] - cn[v]);
        memcpy(buf, rn + cn[v], sizeof(int32_t) * (size_t)rc);
        rc = sample_least(buf, rc, ms, seed, round, v, tmp);
        for (int a = 0; a < rc; ++a)
            if (!has_id(nn, cn_, buf[a])) nn[cn_++] = buf[a];
        for (int t = 0; t < k; ++t) {
            int32_t u = snap[v * k + t];
            if (u >= 0 && !isnew[v * k + t] && !flags[v * k + t] && !has_id(nn, cn_, u)) no[co_++] = u;
        }
        rc = (int)(co[v + 1] - co[v]);
        memcpy(buf, ro + co[v], sizeof(int32_t) * (size_t)rc);
        rc = sample_least(buf, rc, ms, seed, round, v, tmp);
        for (int a = 0; a < rc; ++a)
            if (!has_id(nn, cn_, buf[a]) && !has_id(no, co_, buf[a])) no[co_++] = buf[a];
        for (int a = 0; a < cn_; ++a) {
            int32_t u = nn[a];
            for (int b = a + 1; b < cn_ + co_; ++b) {
                int32_t w = b < cn_ ? nn[b] : no[b - cn_];
                float d = orc_dist_f32(X + (int64_t)u * D, X + (int64_t)w * D, D);
                orc_list_insert(ids + (int64_t)u * k, dists + (int64_t)u * k, k, d, w);
                orc_list_insert(ids + (int64_t)w * k, dists + (int64_t)w * k, k, d, u);
            }
        }
    }
    /* 4. flags of the new lists */
    memcpy(isnew, flags, nk);                   /* flags after the sampling, by snapshot slot */
    for (int64_t u = 0; u < n; ++u)
        for (int t = 0; t < k; ++t) {
            int32_t id = ids[u * k + t];
            unsigned char f = 0;
            if (id >= 0) {
                int found = -1;
                for (int s2 = 0; s2 < k; ++s2)
                    if (snap[u * k + s2] == id) { found = s2; break; }
                if (found < 0) { f = 1; ++changed; }
                else f = isnew[u * k + found];
            }
            flags[u * k + t] = f;
        }
    free(snap); free(isnew); free(co); free(cn); free(ro); free(rn); free(nn); free(no); free(buf);
    free(tmp); free(fo); free(fn);
    return changed;
}

/* ------------------------------------------------------------------ */
/* Whole build: "Initialize G", I_0 tree passes (Alg. 1), then the     */
/* refinement rounds.                                                 */
/* ------------------------------------------------------------------ */
int orc_build(const float *X, int64_t n, int D, int k, int leaf_max, int passes,
              int rounds, int iters, int mode, uint64_t seed,
              int32_t *out_ids, float *out_d)
{
    if (n < 2 || k < 1 || D < 1 || leaf_max < 2) return -1;
    for (int64_t i = 0; i < n; ++i) list_clear(out_ids + i * k, out_d + i * k, k);
    int L = orc_tree_depth(n, leaf_max);
    int64_t nleaf = (int64_t)1 << L;
    int32_t *perm = malloc(sizeof(int32_t) * (size_t)n);
    int64_t *off = malloc(sizeof(int64_t) * (size_t)(nleaf + 1));
    if (!perm || !off) { free(perm); free(off); return -1; }
    for (int p = 0; p < passes; ++p) {
        if (orc_partition(X, n, D, leaf_max, iters, seed, p, perm, off) < 0) {
            free(perm); free(off); return -1;
        }
        orc_leaf_update(X, n, D, k, perm, off, nleaf, out_ids, out_d);
    }
    free(perm); free(off);
    for (int r = 0; r < rounds; ++r)
        if (orc_refine_round(X, n, D, k, mode, out_ids, out_d) != 0) return -1;
    return 0;
}

/* Whole build with sampled refinement: the tree passes of orc_build,  */
/* then `rounds` sampled rounds (round r uses priority round r and the */
/* build seed), every entry flagged new before the first.              */
int orc_build_sampled(const float *X, int64_t n, int D, int k, int leaf_max, int passes, int rounds,
                      int iters, int ms, uint64_t seed, int32_t *out_ids, float *out_d)
{
    if (rounds < 0 || ms < 0) return -1;
    int rc = orc_build(X, n, D, k, leaf_max, passes, 0, iters, 1, seed, out_ids, out_d);
    if (rc != 0) return rc;
    unsigned char *flags = malloc((size_t)n * (size_t)k);
    if (!flags) return -2;
    memset(flags, 1, (size_t)n * (size_t)k);
    for (int r = 0; r < rounds && rc == 0; ++r)
        if (orc_refine_sampled(X, n, D, k, ms, seed, r, out_ids, out_d, flags) < 0) rc = -2;
    free(flags);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Recall of a graph against exact lists on sampled rows.             */
/* ids: n x k graph; gt_ids/gt_d: s x k exact lists of sample rows.   */
/* recall_ids: mean over rows of |G[i] & GT[i]| / k.                  */
/* recall_tie: mean over rows of #{real entries of G[i] with          */
/*             d <= d_k of GT[i]} / k.                                */
/* ------------------------------------------------------------------ */
int orc_recall(const int32_t *ids, const float *dists, const int32_t *gt_ids,
               const float *gt_d, const int32_t *sample, int64_t s, int k,
               double *recall_ids, double *recall_tie)
{
    int64_t hit = 0, tie = 0;
    for (int64_t r = 0; r < s; ++r) {
        int64_t i = sample[r];
        float kth = gt_d[r * k + k - 1];
        for (int a = 0; a < k; ++a) {
            int32_t g = ids[i * k + a];
            if (g < 0) continue;
            for (int b = 0; b < k; ++b)
                if (gt_ids[r * k + b] == g) { ++hit; break; }
            if (dists[i * k + a] <= kth) ++tie;
        }
    }
    *recall_ids = s ? (double)hit / ((double)s * k) : 0.0;
    *recall_tie = s ? (double)tie / ((double)s * k) : 0.0;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Enhanced hill-climbing search over a kNN graph (Sec. 3.2, Alg. 2).  */
/* For each query q (m x D) with seeds S[q] (s ids; ids outside [0, n) */
/* are skipped): the rank list R starts as the seeds with d(q, seed);  */
/* then, t0 times, every neighbour (in G, n x k ids, -1 = empty) of     */
/* the ks first entries of R by (d, id) that has not been visited yet  */
/* is visited and added to R.  Visited = its distance was computed     */
/* (seeds included).  Output: the ks first entries of R by (d, id),    */
/* empty slots id -1, d +inf.  d is the canonical FP32 distance.       */
/* ------------------------------------------------------------------ */
typedef struct { float d; int32_t id; } rank_t;

static int rank_cmp(const void *a, const void *b)
{
    const rank_t *x = (const rank_t *)a, *y = (const rank_t *)b;
    if (key_less(x->d, x->id, y->d, y->id)) return -1;
    if (key_less(y->d, y->id, x->d, x->id)) return 1;
    return 0;
}

int orc_search(const float *X, int64_t n, int D, const int32_t *G, int k,
               const float *Q, int64_t m, const int32_t *S, int s, int t0, int ks,
               int32_t *out_ids, float *out_d)
{
    if (n <= 0 || D <= 0 || k <= 0 || s < 0 || t0 < 0 || ks <= 0) return -1;
    unsigned char *visited = (unsigned char *)malloc((size_t)n);
    int32_t *top = (int32_t *)malloc(sizeof(int32_t) * (size_t)ks);
    int64_t cap = (int64_t)s + (int64_t)t0 * ks * k;
    rank_t *R = (rank_t *)malloc(sizeof(rank_t) * (size_t)(cap > 0 ? cap : 1));
    if (!visited || !top || !R) { free(visited); free(top); free(R); return -2; }
    for (int64_t qi = 0; qi < m; ++qi) {
        const float *q = Q + qi * D;
        memset(visited, 0, (size_t)n);
        int64_t nr = 0;
        for (int a = 0; a < s; ++a) {          /* R <- seeds */
            int32_t id = S[qi * s + a];
            if (id < 0 || id >= n || visited[id]) continue;
            visited[id] = 1;
            R[nr].d = orc_dist_f32(X + (int64_t)id * D, q, D);
            R[nr].id = id;
            ++nr;
        }
        for (int t = 0; t < t0; ++t) {
            /* the ks first entries of R as it stands at the iteration's start */
            qsort(R, (size_t)nr, sizeof(rank_t), rank_cmp);
            int ntop = nr < ks ? (int)nr : ks;
            for (int a = 0; a < ntop; ++a) top[a] = R[a].id;
            for (int a = 0; a < ntop; ++a) {
                const int32_t *row = G + (int64_t)top[a] * k;
                for (int e = 0; e < k; ++e) {
                    int32_t nb = row[e];
                    if (nb < 0 || nb >= n || visited[nb]) continue;
                    visited[nb] = 1;
                    R[nr].d = orc_dist_f32(X + (int64_t)nb * D, q, D);
                    R[nr].id = nb;
                    ++nr;
                }
            }
        }
        qsort(R, (size_t)nr, sizeof(rank_t), rank_cmp);
        for (int a = 0; a < ks; ++a) {
            out_ids[qi * ks + a] = a < nr ? R[a].id : -1;
            out_d[qi * ks + a] = a < nr ? R[a].d : INFINITY;
        }
    }
    free(visited);
    free(top);
    free(R);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Residue vector quantisation (Sec. 4.1, Eqn. 1) and the inverted     */
/* index with cascaded pruning (Sec. 4.2, Eqns. 2 and 3).  Two stages. */
/*                                                                    */
/* Readings (the paper names the steps but not these details):         */
/*  - each stage's vocabulary is trained by Lloyd's k-means on that    */
/*    stage's vectors: stage 1 on the points, stage 2 on the residues  */
/*    r = x - w1[c1(x)] (FP32 subtraction), c1 the stage-1 code after  */
/*    training;                                                        */
/*  - initial word c is vector p_c, drawn by SplitMix64 inside the     */
/*    c-th of W equal strata of the N vectors (N >= W);                */
/*  - an iteration assigns every vector to its nearest word (canonical */
/*    FP32 distance, ties to the smaller word index), then sets each   */
/*    word with members to the FP64 mean of its members (summed in     */
/*    ascending vector order), rounded to FP32; a word without members */
/*    keeps its value;                                                 */
/*  - the index key of a point is c1 * W2 + c2; a list holds its ids   */
/*    in ascending order;                                              */
/*  - query-to-key distance, in FP32 with this operation order:        */
/*      term1(c1)     = fmaf(-2, q.w1, q.q) + |w1|^2                   */
/*      term2(c1, c2) = fmaf(-2, q.w2, fmaf(2, w1.w2, |w2|^2))         */
/*      d(q, I)       = term1 + term2                                  */
/*    (Eqn. 3 prints the signs of |w1|^2 and of the two products with  */
/*    w2 garbled; these are the terms of the expansion of Eqn. 2).     */
/*    Dot products and norms are canonical: acc = fmaf(a_j, b_j, acc), */
/*    j ascending, from 0.  -0 is normalised to +0;                    */
/*  - cascaded pruning keeps the probe1 stage-1 words with the least   */
/*    (term1, c1); their keys are ranked by (d, I); the seeds are the  */
/*    ids of the lists in that order, ascending inside a list, the     */
/*    first s of them; -1 pads a query whose lists hold fewer.         */
/* ------------------------------------------------------------------ */
static float dot_f32(const float *a, const float *b, int D)
{
    float acc = 0.0f;
    for (int j = 0; j < D; ++j) acc = fmaf(a[j], b[j], acc);
    return acc;
}

void orc_rvq_init_positions(int64_t N, int W, uint64_t seed, int stage, int64_t *pos)
{
    const uint64_t h0 = orc_splitmix64(seed ^ ((uint64_t)stage << 32));
    for (int c = 0; c < W; ++c) {
        int64_t lo = (int64_t)c * N / W, hi = (int64_t)(c + 1) * N / W;
        uint64_t h = orc_splitmix64(h0 ^ (uint64_t)c);
        pos[c] = lo + (int64_t)(h % (uint64_t)(hi - lo));
    }
}

int orc_rvq_assign(const float *V, int64_t N, int D, const float *words, int W, int32_t *codes)
{
    if (N < 0 || D <= 0 || W <= 0) return -1;
    for (int64_t i = 0; i < N; ++i) {
        float best = INFINITY;
        int32_t bc = 0;
        for (int c = 0; c < W; ++c) {
            float d = orc_dist_f32(V + i * D, words + (int64_t)c * D, D);
            if (d < best) { best = d; bc = c; }
        }
        codes[i] = bc;
    }
    return 0;
}

/* Lloyd's k-means of one stage: W words from the N vectors V. */
static int lloyd(const float *V, int64_t N, int D, int W, int iters, uint64_t seed, int stage,
                 float *words, int32_t *codes)
{
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)W);
    double *acc = (double *)malloc(sizeof(double) * (size_t)W * D);
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)W);
    if (!pos || !acc || !cnt) { free(pos); free(acc); free(cnt); return -2; }
    orc_rvq_init_positions(N, W, seed, stage, pos);
    for (int c = 0; c < W; ++c) memcpy(words + (int64_t)c * D, V + pos[c] * D, sizeof(float) * D);
    for (int it = 0; it < iters; ++it) {
        orc_rvq_assign(V, N, D, words, W, codes);
        memset(acc, 0, sizeof(double) * (size_t)W * D);
        memset(cnt, 0, sizeof(int64_t) * (size_t)W);
        for (int64_t i = 0; i < N; ++i) {        /* ascending vector order */
            double *a = acc + (int64_t)codes[i] * D;
            for (int j = 0; j < D; ++j) a[j] += (double)V[i * D + j];
            cnt[codes[i]] += 1;
        }
        for (int c = 0; c < W; ++c) {
            if (cnt[c] == 0) continue;
            for (int j = 0; j < D; ++j)
                words[(int64_t)c * D + j] = (float)(acc[(int64_t)c * D + j] / (double)cnt[c]);
        }
    }
    free(pos);
    free(acc);
    free(cnt);
    return 0;
}

/* Stage-2 vectors: r_i = x_i - w1[c1_i], FP32. */
static void residues(const float *X, int64_t n, int D, const float *w1, const int32_t *c1, float *R)
{
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < D; ++j) R[i * D + j] = X[i * D + j] - w1[(int64_t)c1[i] * D + j];
}

int orc_rvq_train(const float *X, int64_t n, int D, int W1, int W2, int iters, uint64_t seed,
                  float *w1, float *w2)
{
    if (n <= 0 || D <= 0 || W1 <= 0 || W2 <= 0 || W1 > n || W2 > n || iters < 0) return -1;
    int32_t *codes = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    float *R = (float *)malloc(sizeof(float) * (size_t)n * D);
    if (!codes || !R) { free(codes); free(R); return -2; }
    int rc = lloyd(X, n, D, W1, iters, seed, 1, w1, codes);
    if (rc == 0) {
        orc_rvq_assign(X, n, D, w1, W1, codes);
        residues(X, n, D, w1, codes, R);
        rc = lloyd(R, n, D, W2, iters, seed, 2, w2, codes);
    }
    free(codes);
    free(R);
    return rc;
}

int orc_rvq_index(const float *X, int64_t n, int D, const float *w1, int W1, const float *w2, int W2,
                  int32_t *codes, int32_t *offsets, int32_t *ids)
{
    if (n < 0 || D <= 0 || W1 <= 0 || W2 <= 0) return -1;
    int32_t *c1 = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *c2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    float *R = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1) * D);
    int64_t nk = (int64_t)W1 * W2;
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)nk);
    if (!c1 || !c2 || !R || !fill) { free(c1); free(c2); free(R); free(fill); return -2; }
    orc_rvq_assign(X, n, D, w1, W1, c1);
    residues(X, n, D, w1, c1, R);
    orc_rvq_assign(R, n, D, w2, W2, c2);
    memset(offsets, 0, sizeof(int32_t) * (size_t)(nk + 1));
    for (int64_t i = 0; i < n; ++i) {
        codes[2 * i] = c1[i];
        codes[2 * i + 1] = c2[i];
        offsets[(int64_t)c1[i] * W2 + c2[i] + 1] += 1;
    }
    for (int64_t key = 0; key < nk; ++key) offsets[key + 1] += offsets[key];
    memcpy(fill, offsets, sizeof(int32_t) * (size_t)nk);
    for (int64_t i = 0; i < n; ++i) ids[fill[(int64_t)c1[i] * W2 + c2[i]]++] = (int32_t)i;
    free(c1);
    free(c2);
    free(R);
    free(fill);
    return 0;
}

typedef struct { float d; int32_t key; } keyd_t;

static int keyd_cmp(const void *a, const void *b)
{
    const keyd_t *x = (const keyd_t *)a, *y = (const keyd_t *)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    return (x->key > y->key) - (x->key < y->key);
}

int orc_rvq_seeds(const float *w1, int W1, const float *w2, int W2, int D, const int32_t *offsets,
                  const int32_t *ids, const float *Q, int64_t m, int probe1, int s, int32_t *S)
{
    if (W1 <= 0 || W2 <= 0 || D <= 0 || m < 0 || probe1 <= 0 || s < 0) return -1;
    const int p1 = probe1 < W1 ? probe1 : W1;
    float *n1 = (float *)malloc(sizeof(float) * (size_t)W1);
    float *n2 = (float *)malloc(sizeof(float) * (size_t)W2);
    float *x12 = (float *)malloc(sizeof(float) * (size_t)W1 * W2);
    float *qw2 = (float *)malloc(sizeof(float) * (size_t)W2);
    keyd_t *t1 = (keyd_t *)malloc(sizeof(keyd_t) * (size_t)W1);
    keyd_t *cand = (keyd_t *)malloc(sizeof(keyd_t) * (size_t)p1 * W2);
    if (!n1 || !n2 || !x12 || !qw2 || !t1 || !cand) {
        free(n1); free(n2); free(x12); free(qw2); free(t1); free(cand);
        return -2;
    }
    for (int a = 0; a < W1; ++a) n1[a] = dot_f32(w1 + (int64_t)a * D, w1 + (int64_t)a * D, D);
    for (int b = 0; b < W2; ++b) n2[b] = dot_f32(w2 + (int64_t)b * D, w2 + (int64_t)b * D, D);
    for (int a = 0; a < W1; ++a)
        for (int b = 0; b < W2; ++b)
            x12[(int64_t)a * W2 + b] = dot_f32(w1 + (int64_t)a * D, w2 + (int64_t)b * D, D);
    for (int64_t qi = 0; qi < m; ++qi) {
        const float *q = Q + qi * D;
        const float qq = dot_f32(q, q, D);
        for (int a = 0; a < W1; ++a) {            /* Eqn. 3, term 1 */
            float t = fmaf(-2.0f, dot_f32(q, w1 + (int64_t)a * D, D), qq);
            t1[a].d = (t + n1[a]) + 0.0f;
            t1[a].key = a;
        }
        qsort(t1, (size_t)W1, sizeof(keyd_t), keyd_cmp);
        for (int b = 0; b < W2; ++b) qw2[b] = dot_f32(q, w2 + (int64_t)b * D, D);
        int64_t nc = 0;
        for (int r = 0; r < p1; ++r) {            /* the kept stage-1 words, term 2 */
            const int a = t1[r].key;
            for (int b = 0; b < W2; ++b) {
                float t2 = fmaf(-2.0f, qw2[b], fmaf(2.0f, x12[(int64_t)a * W2 + b], n2[b]));
                cand[nc].d = (t1[r].d + t2) + 0.0f;
                cand[nc].key = a * W2 + b;
                ++nc;
            }
        }
        qsort(cand, (size_t)nc, sizeof(keyd_t), keyd_cmp);
        int cnt = 0;
        for (int64_t e = 0; e < nc && cnt < s; ++e)
            for (int32_t t = offsets[cand[e].key]; t < offsets[cand[e].key + 1] && cnt < s; ++t)
                S[qi * s + cnt++] = ids[t];
        for (; cnt < s; ++cnt) S[qi * s + cnt] = -1;
    }
    free(n1); free(n2); free(x12); free(qw2); free(t1); free(cand);
    return 0;
}
