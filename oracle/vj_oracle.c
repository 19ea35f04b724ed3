/*
 * vj_oracle.c -- plain, slow, single-threaded FP64 CPU oracle of the vector
 * epsilon-join and of the merged-index (MI) join with soft work sharing and
 * the adaptive hybrid expansion.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, helper or constant with
 * the CUDA path.
 *
 * Naming: the paper calls the query set X and the data set Y.  Here the data
 * set is `X` (ids 0..nx-1 in the merged node numbering) and the query set is
 * `Q` (ids nx..nx+nq-1).  "Data node" means id < nx.
 *
 * Every distance is evaluated in FP64 from the FP32 inputs:
 *   L2      dist = sqrt(sum_i (a_i - b_i)^2)                     (Def. 1, Sec. 3.1)
 *   cosine  dist = 1 - <a,b> / (|a| |b|)
 * and a pair is in the join iff dist < eps (strict, Def. 1).
 *
 * Functions and the passages they follow:
 *   vjo_dist          Def. 1 distance
 *   vjo_nlj           nested-loop join, Sec. 3.2 (NLJ)
 *   vjo_knn_rows      exact k nearest other nodes, ties by id (graph-build input)
 *   vjo_build_graph   kNN -> RNG prune -> reverse edges -> entry point
 *                     (RNG rule of App. C; the paper treats the index as a
 *                     black box, so the build steps are this project's reading;
 *                     parity of the pruned graph is unpinned against the paper
 *                     beyond the App. C invariant)
 *   vjo_mst           Prim MST over query nodes plus star edges from the entry
 *                     (Sec. 3.2 WS, Alg. 2)
 *   vjo_ood           d1/d2 > 1.5 OOD predictor (Sec. 4.4; the pair set is this
 *                     project's reading of "2-hop neighbours": parity unpinned
 *                     against the paper beyond hand-computed cases and the
 *                     far-query trend, the paper prints no per-query values)
 *   vjo_join          Alg. 1 VectorJoin with Alg. 2-8 in the paper's order
 *   vjo_nnmap_build   NN-Map witnesses and OOD bits (Sec. NN-Map)
 *   vjo_nnmap_join    the join from the witnesses on the data graph (Sec. NN-Map)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define VJO_L2 0
#define VJO_COSINE 1

/* work_sharing modes (Tab. cfg) */
#define VJO_WS_NONE 0
#define VJO_WS_HARD 1
#define VJO_WS_SOFT 2
#define VJO_WS_SELF 3

/* ------------------------------------------------------------------ */
/* Def. 1 distance                                                     */
/* ------------------------------------------------------------------ */
double vjo_dist(const float *a, const float *b, int d, int metric)
{
    if (metric == VJO_COSINE) {
        double ab = 0.0, aa = 0.0, bb = 0.0;
        for (int i = 0; i < d; i++) {
            ab += (double)a[i] * (double)b[i];
            aa += (double)a[i] * (double)a[i];
            bb += (double)b[i] * (double)b[i];
        }
        if (aa == 0.0 || bb == 0.0) return 1.0;
        return 1.0 - ab / (sqrt(aa) * sqrt(bb));
    }
    double s = 0.0;
    for (int i = 0; i < d; i++) {
        double t = (double)a[i] - (double)b[i];
        s += t * t;
    }
    return sqrt(s);
}

/* row u of the merged node set: data rows first, then query rows */
static const float *node_vec(const float *X, int64_t nx, const float *Q, int d, int64_t u)
{
    return u < nx ? X + (size_t)u * d : Q + (size_t)(u - nx) * d;
}

/* ------------------------------------------------------------------ */
/* NLJ (Sec. 3.2): every (q, x) with dist < eps, per query in data-id order. */
/* Two-pass use: call with ids == NULL to get counts only.             */
/* offsets has nq+1 entries.  Returns total pairs.                      */
/* ------------------------------------------------------------------ */
int64_t vjo_nlj(const float *X, int64_t nx, const float *Q, int64_t nq, int d, int metric,
                double eps, int64_t *offsets, int32_t *ids, double *dists)
{
    int64_t total = 0;
    for (int64_t q = 0; q < nq; q++) {
        if (offsets) offsets[q] = total;
        const float *qv = Q + (size_t)q * d;
        for (int64_t x = 0; x < nx; x++) {
            double dd = vjo_dist(X + (size_t)x * d, qv, d, metric);
            if (dd < eps) {
                if (ids) {
                    ids[total] = (int32_t)x;
                    if (dists) dists[total] = dd;
                }
                total++;
            }
        }
    }
    if (offsets) offsets[nq] = total;
    return total;
}

/* ------------------------------------------------------------------ */
/* (dist, id) ordered lists                                             */
/* ------------------------------------------------------------------ */
typedef struct {
    double d;
    int32_t id;
} cand_t;

static int cand_less(cand_t a, cand_t b)
{
    return a.d < b.d || (a.d == b.d && a.id < b.id);
}

/* insert into an ascending array of length *n (capacity >= *n + 1) */
static void sorted_insert(cand_t *arr, int64_t *n, cand_t c)
{
    int64_t lo = 0, hi = *n;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (cand_less(arr[mid], c)) lo = mid + 1;
        else hi = mid;
    }
    memmove(arr + lo + 1, arr + lo, (size_t)(*n - lo) * sizeof(cand_t));
    arr[lo] = c;
    (*n)++;
}

/* ------------------------------------------------------------------ */
/* exact kNN for a list of rows: the K nearest other nodes of the merged */
/* set by (dist, id).  out_ids/out_d are [nrows][K]; if fewer than K     */
/* other nodes exist the tail is -1 / +inf.                              */
/* ------------------------------------------------------------------ */
void vjo_knn_rows(const float *X, int64_t nx, const float *Q, int64_t nq, int d, int metric, int K,
                  const int64_t *rows, int64_t nrows, int32_t *out_ids, double *out_d)
{
    int64_t n = nx + nq;
    cand_t *best = (cand_t *)malloc((size_t)(K + 1) * sizeof(cand_t));
    for (int64_t r = 0; r < nrows; r++) {
        int64_t u = rows[r];
        const float *uv = node_vec(X, nx, Q, d, u);
        int64_t nb = 0;
        for (int64_t v = 0; v < n; v++) {
            if (v == u) continue;
            cand_t c = {vjo_dist(uv, node_vec(X, nx, Q, d, v), d, metric), (int32_t)v};
            if (nb < K) {
                sorted_insert(best, &nb, c);
            } else if (cand_less(c, best[K - 1])) {
                nb = K - 1;
                sorted_insert(best, &nb, c);
            }
        }
        for (int k = 0; k < K; k++) {
            out_ids[r * K + k] = k < nb ? best[k].id : -1;
            out_d[r * K + k] = k < nb ? best[k].d : INFINITY;
        }
    }
    free(best);
}

/* ------------------------------------------------------------------ */
/* RNG prune (App. C rule, alpha = 1): walk candidates in ascending      */
/* (dist(u,.), id) order; keep v unless an already-kept w is closer to v */
/* than u is (dist(w,v) < dist(u,v)); stop at R kept.                    */
/* ------------------------------------------------------------------ */
static int rng_prune(const float *X, int64_t nx, const float *Q, int d, int metric,
                     const cand_t *cands, int64_t nc, int R, int32_t *kept)
{
    int nk = 0;
    for (int64_t i = 0; i < nc && nk < R; i++) {
        const float *vv = node_vec(X, nx, Q, d, cands[i].id);
        int ok = 1;
        for (int j = 0; j < nk; j++) {
            double dwv = vjo_dist(node_vec(X, nx, Q, d, kept[j]), vv, d, metric);
            if (dwv < cands[i].d) {
                ok = 0;
                break;
            }
        }
        if (ok) kept[nk++] = cands[i].id;
    }
    return nk;
}

/* ------------------------------------------------------------------ */
/* Graph build (this project's reading of the black-box NSG index):     */
/*  1. candidates = exact kNN(K) of every node (given, or computed here) */
/*  2. RNG prune each list to at most R                                   */
/*  3. reverse edges: C(v) = pruned(v) U {u : v in pruned(u)}, ascending  */
/*     (dist(v,.), id); if |C(v)| <= R keep it, else RNG-prune C(v) to R   */
/*  4. entry = node nearest the mean of all nodes, ties by id             */
/* adj is [n][R], -1 padded, each list ascending by (dist, id).          */
/* knn_ids may be NULL (computed here).  pruned_out may be NULL; else it  */
/* receives the step-2 lists ([n][R], -1 padded).                         */
/* ------------------------------------------------------------------ */
int32_t vjo_build_graph(const float *X, int64_t nx, const float *Q, int64_t nq, int d, int metric,
                        int K, int R, const int32_t *knn_ids, int32_t *pruned_out, int32_t *adj)
{
    int64_t n = nx + nq;
    int32_t *knn = (int32_t *)knn_ids;
    int own_knn = 0;
    if (!knn) {
        knn = (int32_t *)malloc((size_t)n * K * sizeof(int32_t));
        double *kd = (double *)malloc((size_t)n * K * sizeof(double));
        int64_t *rows = (int64_t *)malloc((size_t)n * sizeof(int64_t));
        for (int64_t u = 0; u < n; u++) rows[u] = u;
        vjo_knn_rows(X, nx, Q, nq, d, metric, K, rows, n, knn, kd);
        free(kd);
        free(rows);
        own_knn = 1;
    }

    /* step 2 */
    int32_t *pr = (int32_t *)malloc((size_t)n * R * sizeof(int32_t));
    int *npr = (int *)calloc((size_t)n, sizeof(int));
    cand_t *cands = (cand_t *)malloc((size_t)(K + 1) * sizeof(cand_t));
    for (int64_t u = 0; u < n; u++) {
        const float *uv = node_vec(X, nx, Q, d, u);
        int64_t nc = 0;
        for (int k = 0; k < K; k++) {
            int32_t v = knn[u * K + k];
            if (v < 0) continue;
            cand_t c = {vjo_dist(uv, node_vec(X, nx, Q, d, v), d, metric), v};
            sorted_insert(cands, &nc, c);
        }
        npr[u] = rng_prune(X, nx, Q, d, metric, cands, nc, R, pr + u * R);
        for (int k = npr[u]; k < R; k++) pr[u * R + k] = -1;
    }
    if (pruned_out) memcpy(pruned_out, pr, (size_t)n * R * sizeof(int32_t));

    /* step 3: in-lists */
    int *nin = (int *)calloc((size_t)n, sizeof(int));
    for (int64_t u = 0; u < n; u++)
        for (int k = 0; k < npr[u]; k++) nin[pr[u * R + k]]++;
    int64_t *inoff = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    inoff[0] = 0;
    for (int64_t v = 0; v < n; v++) inoff[v + 1] = inoff[v] + nin[v];
    int32_t *inl = (int32_t *)malloc((size_t)(inoff[n] + 1) * sizeof(int32_t));
    int64_t *fill = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    for (int64_t v = 0; v < n; v++) fill[v] = inoff[v];
    for (int64_t u = 0; u < n; u++)
        for (int k = 0; k < npr[u]; k++) inl[fill[pr[u * R + k]]++] = (int32_t)u;

    int maxc = R;
    for (int64_t v = 0; v < n; v++)
        if (R + nin[v] > maxc) maxc = R + nin[v];
    cand_t *un = (cand_t *)malloc((size_t)(maxc + 1) * sizeof(cand_t));
    int32_t *tmp = (int32_t *)malloc((size_t)R * sizeof(int32_t));
    for (int64_t v = 0; v < n; v++) {
        const float *vv = node_vec(X, nx, Q, d, v);
        int64_t nu = 0;
        for (int k = 0; k < npr[v]; k++) {
            int32_t w = pr[v * R + k];
            cand_t c = {vjo_dist(vv, node_vec(X, nx, Q, d, w), d, metric), w};
            sorted_insert(un, &nu, c);
        }
        for (int64_t j = inoff[v]; j < inoff[v + 1]; j++) {
            int32_t w = inl[j];
            int dup = 0;
            for (int64_t t = 0; t < nu; t++)
                if (un[t].id == w) dup = 1;
            if (dup) continue;
            cand_t c = {vjo_dist(vv, node_vec(X, nx, Q, d, w), d, metric), w};
            sorted_insert(un, &nu, c);
        }
        int nk;
        if (nu <= R) {
            nk = (int)nu;
            for (int k = 0; k < nk; k++) tmp[k] = un[k].id;
        } else {
            nk = rng_prune(X, nx, Q, d, metric, un, nu, R, tmp);
        }
        for (int k = 0; k < R; k++) adj[v * R + k] = k < nk ? tmp[k] : -1;
    }

    /* step 4: entry point */
    double *mean = (double *)calloc((size_t)d, sizeof(double));
    for (int64_t u = 0; u < n; u++) {
        const float *uv = node_vec(X, nx, Q, d, u);
        for (int i = 0; i < d; i++) mean[i] += (double)uv[i];
    }
    float *meanf = (float *)malloc((size_t)d * sizeof(float));
    /* distance to the centroid is taken in FP64 against the FP64 centroid */
    int32_t entry = 0;
    double bestd = INFINITY;
    for (int i = 0; i < d; i++) mean[i] /= (double)n;
    for (int64_t u = 0; u < n; u++) {
        const float *uv = node_vec(X, nx, Q, d, u);
        double dd;
        if (metric == VJO_COSINE) {
            double ab = 0, aa = 0, bb = 0;
            for (int i = 0; i < d; i++) {
                ab += (double)uv[i] * mean[i];
                aa += (double)uv[i] * (double)uv[i];
                bb += mean[i] * mean[i];
            }
            dd = (aa == 0.0 || bb == 0.0) ? 1.0 : 1.0 - ab / (sqrt(aa) * sqrt(bb));
        } else {
            double s = 0;
            for (int i = 0; i < d; i++) {
                double t = (double)uv[i] - mean[i];
                s += t * t;
            }
            dd = sqrt(s);
        }
        if (dd < bestd) {
            bestd = dd;
            entry = (int32_t)u;
        }
    }

    free(meanf);
    free(mean);
    free(tmp);
    free(un);
    free(fill);
    free(inl);
    free(inoff);
    free(nin);
    free(cands);
    free(npr);
    free(pr);
    if (own_knn) free(knn);
    return entry;
}

/* ------------------------------------------------------------------ */
/* MST order (Sec. 3.2 WS; Alg. 2).  Undirected graph on {entry} U Q:    */
/*   - every query-query edge of the merged graph (either direction),    */
/*     weight = dist;                                                     */
/*   - a star edge (entry, q) for every query q != entry, weight dist.    */
/* Edges are totally ordered by (weight, min node id, max node id), so   */
/* the MST is unique.  Prim from the entry; parent[qi] is the query       */
/* index of the tree parent, or -1 when the parent is the entry and the   */
/* entry is a data node (or for the entry itself when it is a query).     */
/* order[] receives the query indices in Prim insertion order (a         */
/* topological order of the tree), depth[] the tree depth (entry = 0).    */
/* Returns the MST's total weight.                                        */
/* ------------------------------------------------------------------ */
typedef struct {
    double w;
    int32_t lo, hi; /* edge endpoints as node ids, lo < hi */
    int32_t to;     /* node id being attached */
    int32_t from;   /* node id already in the tree */
} pedge_t;

static int pedge_less(const pedge_t *a, const pedge_t *b)
{
    if (a->w != b->w) return a->w < b->w;
    if (a->lo != b->lo) return a->lo < b->lo;
    return a->hi < b->hi;
}

typedef struct {
    pedge_t *h;
    int64_t n, cap;
} pheap_t;

static void pheap_push(pheap_t *hp, pedge_t e)
{
    if (hp->n == hp->cap) {
        hp->cap = hp->cap ? hp->cap * 2 : 1024;
        hp->h = (pedge_t *)realloc(hp->h, (size_t)hp->cap * sizeof(pedge_t));
    }
    int64_t i = hp->n++;
    hp->h[i] = e;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!pedge_less(&hp->h[i], &hp->h[p])) break;
        pedge_t t = hp->h[i];
        hp->h[i] = hp->h[p];
        hp->h[p] = t;
        i = p;
    }
}

static pedge_t pheap_pop(pheap_t *hp)
{
    pedge_t top = hp->h[0];
    hp->h[0] = hp->h[--hp->n];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < hp->n && pedge_less(&hp->h[l], &hp->h[m])) m = l;
        if (r < hp->n && pedge_less(&hp->h[r], &hp->h[m])) m = r;
        if (m == i) break;
        pedge_t t = hp->h[i];
        hp->h[i] = hp->h[m];
        hp->h[m] = t;
        i = m;
    }
    return top;
}

double vjo_mst(const float *X, int64_t nx, const float *Q, int64_t nq, int d, int metric,
               const int32_t *adj, int R, int32_t entry, int32_t *parent, int32_t *order,
               int32_t *depth)
{
    int64_t n = nx + nq;
    /* undirected query-query adjacency (dedup not needed: duplicates only add */
    /* equal-keyed heap entries)                                              */
    int64_t *deg = (int64_t *)calloc((size_t)nq + 1, sizeof(int64_t));
    for (int64_t qi = 0; qi < nq; qi++) {
        int64_t u = nx + qi;
        for (int k = 0; k < R; k++) {
            int32_t v = adj[u * R + k];
            if (v >= nx && v != u) {
                deg[qi]++;
                deg[v - nx]++;
            }
        }
    }
    int64_t *off = (int64_t *)malloc((size_t)(nq + 1) * sizeof(int64_t));
    off[0] = 0;
    for (int64_t qi = 0; qi < nq; qi++) off[qi + 1] = off[qi] + deg[qi];
    int32_t *nb = (int32_t *)malloc((size_t)(off[nq] + 1) * sizeof(int32_t));
    int64_t *fp = (int64_t *)malloc((size_t)(nq + 1) * sizeof(int64_t));
    for (int64_t qi = 0; qi < nq; qi++) fp[qi] = off[qi];
    for (int64_t qi = 0; qi < nq; qi++) {
        int64_t u = nx + qi;
        for (int k = 0; k < R; k++) {
            int32_t v = adj[u * R + k];
            if (v >= nx && v != u) {
                nb[fp[qi]++] = v;
                nb[fp[v - nx]++] = (int32_t)u;
            }
        }
    }

    char *in_tree = (char *)calloc((size_t)n, 1);
    pheap_t hp = {0, 0, 0};
    const float *sv = node_vec(X, nx, Q, d, entry);
    int entry_is_query = entry >= nx;
    double total = 0.0;
    int64_t placed = 0;

    in_tree[entry] = 1;
    if (entry_is_query) {
        int64_t qs = entry - nx;
        parent[qs] = -1;
        depth[qs] = 0;
        order[placed++] = (int32_t)qs;
    }
    /* edges leaving the entry: all star edges, plus (if the entry is a query) */
    /* its query-query edges (identical endpoints, so they tie with the star   */
    /* edge in weight; either attaches the same node to the same parent)       */
    for (int64_t qi = 0; qi < nq; qi++) {
        int32_t u = (int32_t)(nx + qi);
        if (u == entry) continue;
        pedge_t e;
        e.w = vjo_dist(sv, Q + (size_t)qi * d, d, metric);
        e.lo = entry < u ? entry : u;
        e.hi = entry < u ? u : entry;
        e.to = u;
        e.from = entry;
        pheap_push(&hp, e);
    }
    int32_t *dep_node = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    while (hp.n > 0) {
        pedge_t e = pheap_pop(&hp);
        if (in_tree[e.to]) continue;
        in_tree[e.to] = 1;
        total += e.w;
        int64_t qi = e.to - nx;
        parent[qi] = (e.from == entry && !entry_is_query) ? -1 : (int32_t)(e.from - nx);
        dep_node[e.to] = dep_node[e.from] + 1;
        depth[qi] = dep_node[e.to];
        order[placed++] = (int32_t)qi;
        const float *uv = Q + (size_t)qi * d;
        for (int64_t j = off[qi]; j < off[qi + 1]; j++) {
            int32_t v = nb[j];
            if (in_tree[v]) continue;
            pedge_t f;
            f.w = vjo_dist(uv, Q + (size_t)(v - nx) * d, d, metric);
            f.lo = e.to < v ? e.to : v;
            f.hi = e.to < v ? v : e.to;
            f.to = v;
            f.from = e.to;
            pheap_push(&hp, f);
        }
    }
    free(dep_node);
    free(hp.h);
    free(in_tree);
    free(fp);
    free(nb);
    free(off);
    free(deg);
    return total;
}

/* ------------------------------------------------------------------ */
/* OOD predictor (Sec. 4.4).  N1 = data nodes among the out-neighbours   */
/* of query node u; d1 = mean dist(u, v) over v in N1.  Pairs (v, w) with */
/* v in N1, w a data out-neighbour of v, w not in N(u) and w != u;        */
/* d2 = mean dist(v, w) over those pairs.  OOD iff d1/d2 > 1.5.            */
/* N1 empty -> OOD (flag 1, d1 = d2 = NaN); no pairs -> not OOD.           */
/* ------------------------------------------------------------------ */
int vjo_ood(const float *X, int64_t nx, const float *Q, int d, int metric, const int32_t *adj,
            int R, int64_t u, double *d1_out, double *d2_out)
{
    const float *uv = node_vec(X, nx, Q, d, u);
    double s1 = 0.0, s2 = 0.0;
    int64_t n1 = 0, n2 = 0;
    for (int k = 0; k < R; k++) {
        int32_t v = adj[u * R + k];
        if (v < 0 || v >= nx) continue;
        const float *vv = X + (size_t)v * d;
        s1 += vjo_dist(uv, vv, d, metric);
        n1++;
        for (int j = 0; j < R; j++) {
            int32_t w = adj[(int64_t)v * R + j];
            if (w < 0 || w >= nx || w == u) continue;
            int in_nu = 0;
            for (int t = 0; t < R; t++)
                if (adj[u * R + t] == w) in_nu = 1;
            if (in_nu) continue;
            s2 += vjo_dist(vv, X + (size_t)w * d, d, metric);
            n2++;
        }
    }
    if (n1 == 0) {
        if (d1_out) *d1_out = NAN;
        if (d2_out) *d2_out = NAN;
        return 1;
    }
    double d1 = s1 / (double)n1;
    double d2 = n2 ? s2 / (double)n2 : NAN;
    if (d1_out) *d1_out = d1;
    if (d2_out) *d2_out = d2;
    if (n2 == 0) return 0;
    return d1 / d2 > 1.5;
}

/* ------------------------------------------------------------------ */
/* Alg. 1 VectorJoin on the merged index.                               */
/* ------------------------------------------------------------------ */
typedef struct {
    int work_sharing;     /* VJO_WS_* */
    int force_hybrid;     /* Alg. 6 */
    int adapt_hybrid;     /* Alg. 6 */
    int greedy_beam_size; /* Alg. 4 trim */
    int conv_threshold;   /* Alg. 5 */
    int hybrid_beam_size; /* Alg. 7 trim */
    /* Optional per-query plan (a predictor in place of Alg. 6's rule; not in
     * the paper).  route[qi] != 0: after the greedy phase the query's result
     * is its exact NLJ row (brute-force scan) and no expansion runs; the soft
     * cache is taken over the nodes the greedy phase visited.  beam[qi]: the
     * query runs the hybrid expansion with hybrid_beam_size = beam[qi] when
     * beam[qi] > 0, the plain BFS expansion when beam[qi] == 0, and skips the
     * expansion phase of Alg. 1 when beam[qi] < 0 (an expansion budget of
     * zero: the result is I after the greedy phase; reported as hybrid flag
     * 3).  NULL: unused. */
    const uint8_t *route;
    const int32_t *beam;
    /* 1: separate-index execution (cfg.merged = false, Sec. 3.2 INLJ and its
     * work sharing): `adj` is the data graph G_Y ([nx][R], data ids only),
     * `entry` its entry s_Y, the query is not a graph node, StopGreedy's
     * third rule is off and CheckHybrid ignores adapt_hybrid (Alg. 6).  With
     * hard/soft sharing the order and parents come from the MST over the
     * query graph G_X (Alg. 2).  0: the merged index. */
    int separate;
    /* 1: a hybrid expansion whose greedy phase found no in-range point starts
     * from the closest visited data node instead of returning an empty row
     * (the "seed with the best" variant; the paper's literal reading is 0). */
    int hybrid_seed_best;
} vjo_cfg;

/* per-query outputs of vjo_join */
typedef struct {
    int64_t *offsets; /* [nq+1] CSR over query index, pairs ascending by data id */
    int32_t *ids;     /* [cap] */
    double *dists;    /* [cap] */
    int64_t cap;      /* capacity of ids/dists; pairs beyond are counted only */
    int64_t *steps;   /* [nq] |V| = distance computations of the query */
    int32_t *cache;   /* [nq] C[q] of Alg. 8 (soft): closest visited data node or -1 */
    uint8_t *hybrid;  /* [nq] CheckHybrid outcome */
    int64_t *expansions; /* [nq] nodes popped in the expansion phase */
} vjo_out;

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * order: the processing order (n_order query indices), e.g. from vjo_mst; if
 * NULL the queries are processed 0..nq-1 (Alg. 2 "arbitrary order").  Queries
 * not in the order get empty result rows (sampled runs: the order must then be
 * closed under MST parents when sharing is on).  parent: MST
 * parents (query index or -1), required for hard/soft sharing.
 * Returns the total number of result pairs (may exceed out->cap).
 */
int64_t vjo_join(const float *X, int64_t nx, const float *Q, int64_t nq, int d, int metric,
                 const int32_t *adj, int R, int32_t entry, const int32_t *order, int64_t n_order,
                 const int32_t *parent, const vjo_cfg *cfg, double eps, vjo_out *out)
{
    int64_t n = nx + nq;
    int64_t *stamp = (int64_t *)malloc((size_t)n * sizeof(int64_t)); /* visited marks */
    double *dv = (double *)malloc((size_t)n * sizeof(double));       /* dist to q of visited */
    for (int64_t u = 0; u < n; u++) stamp[u] = -1;
    int64_t qcap = 1024, icap = 1024, vcap = 1024, nvis = 0;
    int32_t *vis = (int32_t *)malloc((size_t)vcap * sizeof(int32_t)); /* visited list */
    cand_t *pq = (cand_t *)malloc((size_t)qcap * sizeof(cand_t)); /* priority queue, ascending */
    int32_t *I = (int32_t *)malloc((size_t)icap * sizeof(int32_t));
    int32_t *fifo = NULL;
    /* hard cache: per-query in-range lists (only for VJO_WS_HARD) */
    int32_t **hard = NULL;
    int64_t *hard_n = NULL;
    if (cfg->work_sharing == VJO_WS_HARD) {
        hard = (int32_t **)calloc((size_t)nq, sizeof(int32_t *));
        hard_n = (int64_t *)calloc((size_t)nq, sizeof(int64_t));
    }
    int32_t *cache = out->cache ? out->cache : (int32_t *)malloc((size_t)nq * sizeof(int32_t));
    for (int64_t qi = 0; qi < nq; qi++) cache[qi] = -1;
    int64_t *counts = (int64_t *)calloc((size_t)nq, sizeof(int64_t));
    int32_t **res = (int32_t **)calloc((size_t)nq, sizeof(int32_t *));
    double **resd = (double **)calloc((size_t)nq, sizeof(double *));

#define VISIT(v, dd)                                                            \
    do {                                                                        \
        stamp[(v)] = qi;                                                        \
        dv[(v)] = (dd);                                                         \
        if (nvis + 1 > vcap) {                                                  \
            vcap *= 2;                                                          \
            vis = (int32_t *)realloc(vis, (size_t)vcap * sizeof(int32_t));      \
        }                                                                       \
        vis[nvis++] = (v);                                                      \
    } while (0)
#define VISITED(v) (stamp[(v)] == qi)
#define PQ_PUSH(c)                                                              \
    do {                                                                        \
        if (npq + 1 > qcap) {                                                   \
            qcap *= 2;                                                          \
            pq = (cand_t *)realloc(pq, (size_t)qcap * sizeof(cand_t));          \
        }                                                                       \
        sorted_insert(pq, &npq, (c));                                           \
    } while (0)
#define I_PUSH(v)                                                               \
    do {                                                                        \
        if (nI + 1 > icap) {                                                    \
            icap *= 2;                                                          \
            I = (int32_t *)realloc(I, (size_t)icap * sizeof(int32_t));          \
        }                                                                       \
        I[nI++] = (v);                                                          \
    } while (0)

    if (!order) n_order = nq;
    for (int64_t t = 0; t < n_order; t++) {
        int64_t qi = order ? order[t] : t;
        int32_t qn = (int32_t)(nx + qi);
        const float *qv = Q + (size_t)qi * d;
        int64_t steps = 0;
        nvis = 0;

        /* --- Alg. 3 SeedPhase.  Merged index: S = {entry}; hard/soft add the */
        /* parent's cache; self adds q.  Reading: under the merged index, soft  */
        /* sharing seeds with q as well (otherwise StopGreedy's third rule ends */
        /* the walk before any neighbourhood is probed).                        */
        const int merged = !cfg->separate;
        int32_t S[2 + 1];
        int nS = 0;
        S[nS++] = entry;
        int32_t *hseed = NULL;
        int64_t nhseed = 0;
        int64_t par = parent ? parent[qi] : -1;
        if (cfg->work_sharing == VJO_WS_SOFT) {
            if (par >= 0 && cache[par] >= 0) S[nS++] = cache[par];
            if (merged) S[nS++] = qn;
        } else if (cfg->work_sharing == VJO_WS_HARD) {
            if (par >= 0) {
                hseed = hard[par];
                nhseed = hard_n[par];
            }
            if (merged) S[nS++] = qn;
        } else if (cfg->work_sharing == VJO_WS_SELF) {
            if (merged) S[nS++] = qn; /* self seeding exists only on the merged index */
        }

        /* --- Alg. 4 GreedySearchPhase */
        int64_t npq = 0, nI = 0;
        /* I <- in-range DATA seeds (reading: the query node itself is never a result) */
        for (int64_t j = 0; j < nS + nhseed; j++) {
            int32_t u = j < nS ? S[j] : hseed[j - nS];
            if (VISITED(u)) continue;
            double dd = vjo_dist(node_vec(X, nx, Q, d, u), qv, d, metric);
            steps++;
            VISIT(u, dd);
            cand_t c = {dd, u};
            PQ_PUSH(c);
            if (u < nx && dd < eps) I_PUSH(u);
        }
        double best_front = INFINITY;
        int64_t no_improve = 0;
        while (npq > 0) {
            /* --- Alg. 5 StopGreedy on the front element */
            cand_t f = pq[0];
            int stop = 0;
            if (f.d < eps && f.id < nx) stop = 1;
            if (!stop) {
                /* reading: "d has not been decreased" counts consecutive checks */
                /* whose front key is not below the best front key seen so far   */
                if (f.d < best_front) {
                    best_front = f.d;
                    no_improve = 0;
                } else {
                    no_improve++;
                }
                if (no_improve >= cfg->conv_threshold) stop = 1;
            }
            if (merged && !stop && f.id != qn) stop = 1; /* merged index: only q's neighbourhood */
            if (stop) break;
            /* pop front */
            int32_t u = f.id;
            memmove(pq, pq + 1, (size_t)(npq - 1) * sizeof(cand_t));
            npq--;
            for (int k = 0; k < R; k++) {
                int32_t v = adj[(int64_t)u * R + k];
                if (v < 0 || VISITED(v)) continue;
                double dd = vjo_dist(node_vec(X, nx, Q, d, v), qv, d, metric);
                steps++;
                VISIT(v, dd);
                cand_t c = {dd, v};
                PQ_PUSH(c);
                if (v < nx && dd < eps) I_PUSH(v);
            }
            if (npq > cfg->greedy_beam_size) npq = cfg->greedy_beam_size;
        }

        /* --- Alg. 6 CheckHybrid (or the per-query plan, when given) */
        int hyb;
        int beam = cfg->hybrid_beam_size;
        const int routed = cfg->route && cfg->route[qi];
        const int no_expansion = cfg->beam && cfg->beam[qi] < 0 && !routed;
        if (cfg->beam) {
            beam = cfg->beam[qi];
            hyb = beam > 0;
        } else if (cfg->adapt_hybrid && merged) {
            hyb = vjo_ood(X, nx, Q, d, metric, adj, R, qn, NULL, NULL);
        } else {
            hyb = cfg->force_hybrid;
        }

        /* --- Alg. 7 ExpansionPhase (merged index: min-priority queue by dist) */
        npq = 0;
        for (int64_t j = 0; j < nI && !routed && !no_expansion; j++) {
            cand_t c = {dv[I[j]], I[j]};
            PQ_PUSH(c);
        }
        if (cfg->hybrid_seed_best && hyb && nI == 0 && !routed) {
            /* no in-range point: start from the closest visited data node */
            int32_t bid = -1;
            double bd = INFINITY;
            for (int64_t j = 0; j < nvis; j++) {
                int32_t v = vis[j];
                if (v >= nx) continue;
                if (dv[v] < bd || (dv[v] == bd && v < bid)) {
                    bd = dv[v];
                    bid = v;
                }
            }
            if (bid >= 0) {
                cand_t c = {bd, bid};
                PQ_PUSH(c);
            }
        }
        int64_t expansions = 0;
        while (npq > 0) {
            int32_t u = pq[0].id;
            memmove(pq, pq + 1, (size_t)(npq - 1) * sizeof(cand_t));
            npq--;
            expansions++;
            for (int k = 0; k < R; k++) {
                int32_t v = adj[(int64_t)u * R + k];
                if (v < 0 || VISITED(v)) continue;
                if (v >= nx) continue; /* merged: skip query nodes, not marked */
                double dd = vjo_dist(X + (size_t)v * d, qv, d, metric);
                steps++;
                VISIT(v, dd);
                cand_t c = {dd, v};
                if (dd < eps) {
                    PQ_PUSH(c);
                    I_PUSH(v);
                } else if (hyb) {
                    PQ_PUSH(c);
                    /* reading of "trim to at most max(beam, |Q|-1)": after an  */
                    /* out-range insert, if |Q| > beam drop the largest key     */
                    if (npq > beam) npq--;
                }
            }
        }

        /* --- Alg. 8 UpdateCache */
        if (cfg->work_sharing == VJO_WS_SOFT || out->cache) {
            /* top-1 closest visited data node, ties by id; recorded for every */
            /* mode so tests can inspect it, used as a seed only in soft mode  */
            int32_t bid = -1;
            double bd = INFINITY;
            for (int64_t j = 0; j < nvis; j++) {
                int32_t v = vis[j];
                if (v >= nx) continue;
                if (dv[v] < bd || (dv[v] == bd && v < bid)) {
                    bd = dv[v];
                    bid = v;
                }
            }
            cache[qi] = bid;
        }
        if (cfg->work_sharing == VJO_WS_HARD) {
            hard[qi] = (int32_t *)malloc((size_t)(nI + 1) * sizeof(int32_t));
            memcpy(hard[qi], I, (size_t)nI * sizeof(int32_t));
            hard_n[qi] = nI;
        }
        if (routed) {
            /* brute-force route: the exact NLJ row replaces the expansion */
            nI = 0;
            for (int64_t x = 0; x < nx; x++) {
                double dd = vjo_dist(X + (size_t)x * d, qv, d, metric);
                if (dd < eps) {
                    dv[x] = dd;
                    I_PUSH((int32_t)x);
                }
            }
            hyb = 2;
        }
        if (no_expansion) hyb = 3;

        /* R <- R U I (sorted by data id for the CSR) */
        qsort(I, (size_t)nI, sizeof(int32_t), cmp_i32);
        counts[qi] = nI;
        res[qi] = (int32_t *)malloc((size_t)(nI + 1) * sizeof(int32_t));
        resd[qi] = (double *)malloc((size_t)(nI + 1) * sizeof(double));
        for (int64_t j = 0; j < nI; j++) {
            res[qi][j] = I[j];
            resd[qi][j] = dv[I[j]];
        }
        if (out->steps) out->steps[qi] = steps;
        if (out->hybrid) out->hybrid[qi] = (uint8_t)hyb;
        if (out->expansions) out->expansions[qi] = expansions;
    }

    int64_t total = 0;
    for (int64_t qi = 0; qi < nq; qi++) {
        if (out->offsets) out->offsets[qi] = total;
        for (int64_t j = 0; j < counts[qi]; j++) {
            if (total + j < out->cap) {
                out->ids[total + j] = res[qi][j];
                if (out->dists) out->dists[total + j] = resd[qi][j];
            }
        }
        total += counts[qi];
        free(res[qi]);
        free(resd[qi]);
    }
    if (out->offsets) out->offsets[nq] = total;

    if (hard) {
        for (int64_t qi = 0; qi < nq; qi++) free(hard[qi]);
        free(hard);
        free(hard_n);
    }
    if (!out->cache) free(cache);
    free(res);
    free(resd);
    free(counts);
    free(fifo);
    free(vis);
    free(I);
    free(pq);
    free(dv);
    free(stamp);
    return total;
#undef VISIT
#undef VISITED
#undef PQ_PUSH
#undef I_PUSH
}

/* ------------------------------------------------------------------ */
/* NN-Map (Sec. NN-Map): a materialised top-1 join index from the       */
/* queries to the data, and the join that expands from it on the data's */
/* own graph G_X (adj: [nx][R] data ids).  Readings as in nnmap.py.     */
/* ------------------------------------------------------------------ */

/* witness[q]: the nearest data vector (ties by id), wdist[q] its distance;
 * ood[q]: d1/d2 > 1.5 with N1 = the R nearest data vectors of q, d1 = their
 * mean distance to q, d2 = the mean length of the G_X edges from N1 to data
 * vectors outside N1 (no such edge: not OOD) */
void vjo_nnmap_build(const float *X, int64_t nx, const float *Q, int64_t nq, int d, int metric,
                     const int32_t *adj, int R, int32_t *witness, double *wdist, uint8_t *ood)
{
    cand_t *nb = (cand_t *)malloc((size_t)(R + 1) * sizeof(cand_t));
    for (int64_t q = 0; q < nq; q++) {
        const float *qv = Q + (size_t)q * d;
        int64_t n1 = 0;
        for (int64_t x = 0; x < nx; x++) {
            cand_t c = {vjo_dist(X + (size_t)x * d, qv, d, metric), (int32_t)x};
            if (n1 < R) {
                sorted_insert(nb, &n1, c);
            } else if (cand_less(c, nb[R - 1])) {
                n1--;
                sorted_insert(nb, &n1, c);
            }
        }
        witness[q] = nb[0].id;
        wdist[q] = nb[0].d;
        double d1 = 0.0, s2 = 0.0;
        int64_t c2 = 0;
        for (int64_t j = 0; j < n1; j++) d1 += nb[j].d;
        d1 /= (double)n1;
        for (int64_t j = 0; j < n1; j++) {
            int32_t v = nb[j].id;
            for (int k = 0; k < R; k++) {
                int32_t u = adj[(int64_t)v * R + k];
                if (u < 0) continue;
                int inside = 0;
                for (int64_t t = 0; t < n1; t++) inside |= nb[t].id == u;
                if (inside) continue;
                s2 += vjo_dist(X + (size_t)v * d, X + (size_t)u * d, d, metric);
                c2++;
            }
        }
        ood[q] = (uint8_t)(c2 > 0 && s2 > 0.0 && d1 / (s2 / (double)c2) > 1.5);
    }
    free(nb);
}

/* hybrid_mode: 0 BFS closure for every query, 1 the OOD bit, 2 hybrid for
 * every query.  A query with wdist >= eps is certainly empty and computes no
 * distance; otherwise Alg. 7 runs from its witness on G_X (min-queue by
 * (dist, id); hybrid: out-range nodes queued, the largest dropped once the
 * queue holds more than `beam`).  steps[q] counts distance computations (the
 * stored witness distance costs none).  Returns the total pair count. */
int64_t vjo_nnmap_join(const float *X, int64_t nx, const float *Q, int64_t nq, int d, int metric,
                       const int32_t *adj, int R, const int32_t *witness, const double *wdist,
                       const uint8_t *ood, int hybrid_mode, int beam, double eps, int64_t *offsets,
                       int32_t *ids, double *dists, int64_t cap, int64_t *steps, uint8_t *hyb_out)
{
    int64_t *stamp = (int64_t *)malloc((size_t)nx * sizeof(int64_t));
    double *dv = (double *)malloc((size_t)nx * sizeof(double));
    for (int64_t u = 0; u < nx; u++) stamp[u] = -1;
    int64_t qcap = 1024, rcap = 1024;
    cand_t *pq = (cand_t *)malloc((size_t)qcap * sizeof(cand_t));
    int32_t *res = (int32_t *)malloc((size_t)rcap * sizeof(int32_t));
    int64_t total = 0;
    for (int64_t q = 0; q < nq; q++) {
        offsets[q] = total;
        steps[q] = 0;
        hyb_out[q] = 0;
        if (wdist[q] >= eps) continue; /* certified empty */
        const float *qv = Q + (size_t)q * d;
        const int hyb = hybrid_mode == 2 || (hybrid_mode == 1 && ood[q]);
        hyb_out[q] = (uint8_t)hyb;
        int64_t npq = 0, nres = 0;
        int32_t s = witness[q];
        stamp[s] = q;
        dv[s] = wdist[q];
        res[nres++] = s;
        cand_t c0 = {wdist[q], s};
        sorted_insert(pq, &npq, c0);
        while (npq > 0) {
            int32_t u = pq[0].id;
            memmove(pq, pq + 1, (size_t)(npq - 1) * sizeof(cand_t));
            npq--;
            for (int k = 0; k < R; k++) {
                int32_t v = adj[(int64_t)u * R + k];
                if (v < 0 || stamp[v] == q) continue;
                double dd = vjo_dist(X + (size_t)v * d, qv, d, metric);
                steps[q]++;
                stamp[v] = q;
                dv[v] = dd;
                if (dd >= eps && !hyb) continue;
                if (npq + 1 > qcap) {
                    qcap *= 2;
                    pq = (cand_t *)realloc(pq, (size_t)qcap * sizeof(cand_t));
                }
                cand_t c = {dd, v};
                sorted_insert(pq, &npq, c);
                if (dd < eps) {
                    if (nres + 1 > rcap) {
                        rcap *= 2;
                        res = (int32_t *)realloc(res, (size_t)rcap * sizeof(int32_t));
                    }
                    res[nres++] = v;
                } else if (npq > beam) {
                    npq--; /* the largest key is out of range */
                }
            }
        }
        qsort(res, (size_t)nres, sizeof(int32_t), cmp_i32);
        for (int64_t j = 0; j < nres; j++) {
            if (total + j < cap) {
                ids[total + j] = res[j];
                dists[total + j] = dv[res[j]];
            }
        }
        total += nres;
    }
    offsets[nq] = total;
    free(res);
    free(pq);
    free(dv);
    free(stamp);
    return total;
}
