/*
 * CPU oracle for exact three-hop top-K path search on a typed knowledge graph.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * definition the CUDA library is checked against.  It shares no code with the
 * library; only tests, the package smoke check and the benchmark's CPU
 * baseline leg may load it.  Build with -ffp-contract=off and without
 * -Ofast / -ffast-math: the floating-point operation order below is the
 * definition of the reference scores.
 *
 * What it computes (paper readings in brackets):
 *   edge weight w(u,r,v), fp64, inputs converted exactly from the stored
 *   float32 or bfloat16 values, j = 0..d-1 in order, no fused multiply-add:
 *     TransE-L1 [Alg. 3 and Alg. 4: score = gamma - sum_j |agg[j] - e_t[j]|
 *                with gamma = 1.0; Sec. 3.1: the TransE relation h + r - t;
 *                Sec. 3.3: the aggregation of head and relation is h + r]
 *        acc += fabs((e_u[j] + w_r[j]) - e_v[j]);   w = gamma - acc
 *     DistMult (a bilinear form for the tensor-core variants; the paper
 *               leaves the generic ComputeScore of Alg. 7 open)
 *        acc += (e_u[j] * w_r[j]) * e_v[j];         w = acc
 *   path s -r1-> u -r2-> v -r3-> t, simple: u not in {s,t}, v not in {s,t,u}
 *     [Alg. 7: a neighbour already on the path is skipped and reaching the
 *      target ends the path]
 *   path score S = (w1 + w2) + w3   (sum of the three edge weights)
 *   result: the K best paths in the total order
 *     score descending, then (u, r1, v, r2, r3) ascending,
 *   kept with a bounded heap of the K best [Sec. 3.3: per-thread k-heaps that
 *   keep only the K highest scores; the "MaxHeap" of Alg. 3/4 is read as the
 *   structure that keeps the K highest scores, evicting the lowest].
 *
 * Tail prediction (Alg. 3, Alg. 4): oracle_tail_topk below scores every
 * candidate vertex of one type against one (head, relation) pair with the same
 * edge weight and keeps the K best (score descending, then vertex ascending).
 * Constrained three-hop queries (Sec. 3.1): oracle_topk_paths_masked, the
 * brute force restricted to allowed relations per hop and vertex types.
 * Generic H-hop search with a per-path beam (Alg. 6, Alg. 7):
 * oracle_beam_paths.
 *
 * Parity pins (tests/): hand-derived examples with dyadic embeddings, closed
 * forms (zero embeddings), the exact rational edge weight within the fp64
 * rounding bound, an independent meet-in-the-middle route in pure Python,
 * brute-force invariants (K = all equals the full sorted enumeration, prefix
 * consistency in K).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef __FAST_MATH__
#error "the oracle must be built without -ffast-math"
#endif
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double score;
    uint32_t u, v;
    uint16_t r1, r2, r3, pad;
} oracle_path;                      /* 24 bytes, same layout as the library's */

typedef struct {
    int64_t deg_s;   /* out-degree of s */
    int64_t deg_t;   /* in-degree of t */
    int64_t n_u;     /* distinct u in N_out(s) \ {s,t} */
    int64_t n_v;     /* distinct v in N_in(t) \ {s,t} */
    int64_t s_f;     /* sum of out-degrees over those u */
    int64_t s_b;     /* sum of in-degrees over those v */
    int64_t hits;    /* middle edges (u,r2,v) with u, v as above and v != u */
    int64_t paths;   /* number of simple s->t three-hop paths */
} oracle_stats;

enum { ORACLE_OK = 0, ORACLE_EINVAL = 1, ORACLE_ENOMEM = 2 };
enum { ORACLE_TRANSE_L1 = 0, ORACLE_DISTMULT = 1 };
enum { ORACLE_F32 = 0, ORACLE_BF16 = 1 };

/* ------------------------------------------------------------------------ */
static double load_elem(const void* tab, int dtype, int64_t row, int d, int j) {
    if (dtype == ORACLE_F32) {
        return (double)((const float*)tab)[row * (int64_t)d + j];
    } else {
        uint32_t bits = (uint32_t)((const uint16_t*)tab)[row * (int64_t)d + j] << 16;
        float f;
        memcpy(&f, &bits, sizeof f);
        return (double)f;
    }
}

double oracle_edge_weight(const void* vemb, const void* remb, int dtype, int d, int fn,
                          double gamma, uint32_t u, uint32_t r, uint32_t v) {
    double acc = 0.0;
    if (fn == ORACLE_TRANSE_L1) {
        for (int j = 0; j < d; ++j) {
            double a = load_elem(vemb, dtype, u, d, j);
            double b = load_elem(remb, dtype, r, d, j);
            double c = load_elem(vemb, dtype, v, d, j);
            double h_plus_r = a + b;
            double diff = h_plus_r - c;
            acc = acc + fabs(diff);
        }
        return gamma - acc;
    } else {
        for (int j = 0; j < d; ++j) {
            double a = load_elem(vemb, dtype, u, d, j);
            double b = load_elem(remb, dtype, r, d, j);
            double c = load_elem(vemb, dtype, v, d, j);
            double ab = a * b;
            double abc = ab * c;
            acc = acc + abc;
        }
        return acc;
    }
}

int oracle_edge_weights(const void* vemb, const void* remb, int dtype, int d, int fn, double gamma,
                        const uint32_t* src, const uint16_t* rel, const uint32_t* dst, int64_t m,
                        double* out) {
    for (int64_t i = 0; i < m; ++i)
        out[i] = oracle_edge_weight(vemb, remb, dtype, d, fn, gamma, src[i], rel[i], dst[i]);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* 1 if p ranks strictly before q in the result order */
static int ranks_before(const oracle_path* p, const oracle_path* q) {
    if (p->score != q->score) return p->score > q->score;
    if (p->u != q->u) return p->u < q->u;
    if (p->r1 != q->r1) return p->r1 < q->r1;
    if (p->v != q->v) return p->v < q->v;
    if (p->r2 != q->r2) return p->r2 < q->r2;
    return p->r3 < q->r3;
}

static int cmp_rank(const void* a, const void* b) {
    const oracle_path* p = (const oracle_path*)a;
    const oracle_path* q = (const oracle_path*)b;
    if (ranks_before(p, q)) return -1;
    if (ranks_before(q, p)) return 1;
    return 0;
}

/* Bounded heap of the K best paths; the root is the worst kept path. */
typedef struct {
    oracle_path* a;
    int64_t size, cap;
} khe;

static void khe_swap(oracle_path* x, oracle_path* y) {
    oracle_path tmp = *x;
    *x = *y;
    *y = tmp;
}

static void khe_push(khe* h, const oracle_path* p) {
    if (h->size < h->cap) {
        int64_t i = h->size++;
        h->a[i] = *p;
        while (i > 0) {                       /* sift up: parent must be worse */
            int64_t par = (i - 1) / 2;
            if (ranks_before(&h->a[par], &h->a[i])) {
                khe_swap(&h->a[par], &h->a[i]);
                i = par;
            } else {
                break;
            }
        }
        return;
    }
    if (!ranks_before(p, &h->a[0])) return;   /* not better than the worst kept */
    h->a[0] = *p;
    int64_t i = 0;
    for (;;) {                                /* sift down: move the worst up */
        int64_t l = 2 * i + 1, r = l + 1, w = i;
        if (l < h->size && ranks_before(&h->a[w], &h->a[l])) w = l;
        if (r < h->size && ranks_before(&h->a[w], &h->a[r])) w = r;
        if (w == i) break;
        khe_swap(&h->a[w], &h->a[i]);
        i = w;
    }
}

/* first index in cols[lo, hi) whose value is >= key (rows are sorted by col) */
static int64_t lower_bound_u32(const uint32_t* cols, int64_t lo, int64_t hi, uint32_t key) {
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (cols[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/*
 * Brute force: every out-edge (s,r1,u), every out-edge (u,r2,v) of u, every
 * edge (v,r3,t) found by binary search in the sorted row of v.
 */
int oracle_topk_paths(const int64_t* offsets, const uint32_t* cols, const uint16_t* rels, int64_t n,
                      const void* vemb, const void* remb, int dtype, int d, int fn, double gamma,
                      uint32_t s, uint32_t t, int64_t K, oracle_path* out, int64_t* n_out,
                      int64_t* hits_out, int64_t* paths_out) {
    if ((int64_t)s >= n || (int64_t)t >= n || s == t || K <= 0) return ORACLE_EINVAL;
    khe h;
    h.a = (oracle_path*)malloc(sizeof(oracle_path) * (size_t)K);
    if (!h.a) return ORACLE_ENOMEM;
    h.size = 0;
    h.cap = K;
    int64_t hits = 0, paths = 0;
    for (int64_t i = offsets[s]; i < offsets[s + 1]; ++i) {
        uint32_t u = cols[i];
        uint16_t r1 = rels[i];
        if (u == s || u == t) continue;
        int first_edge_to_u = (i == offsets[s] || cols[i - 1] != u);   /* rows sorted by col */
        double w1 = oracle_edge_weight(vemb, remb, dtype, d, fn, gamma, s, r1, u);
        for (int64_t j = offsets[u]; j < offsets[u + 1]; ++j) {
            uint32_t v = cols[j];
            uint16_t r2 = rels[j];
            if (v == s || v == t || v == u) continue;
            int64_t k = lower_bound_u32(cols, offsets[v], offsets[v + 1], t);
            if (k >= offsets[v + 1] || cols[k] != t) continue;
            if (first_edge_to_u) ++hits;
            double w2 = oracle_edge_weight(vemb, remb, dtype, d, fn, gamma, u, r2, v);
            for (; k < offsets[v + 1] && cols[k] == t; ++k) {
                uint16_t r3 = rels[k];
                double w3 = oracle_edge_weight(vemb, remb, dtype, d, fn, gamma, v, r3, t);
                oracle_path p;
                p.score = (w1 + w2) + w3;
                p.u = u;
                p.v = v;
                p.r1 = r1;
                p.r2 = r2;
                p.r3 = r3;
                p.pad = 0;
                khe_push(&h, &p);
                ++paths;
            }
        }
    }
    qsort(h.a, (size_t)h.size, sizeof(oracle_path), cmp_rank);
    memcpy(out, h.a, sizeof(oracle_path) * (size_t)h.size);
    *n_out = h.size;
    if (hits_out) *hits_out = hits;
    if (paths_out) *paths_out = paths;
    free(h.a);
    return ORACLE_OK;
}

/*
 * Constrained three-hop query [Sec. 3.1: hop 1 follows the award-winner
 * relation, hop 2 the works-in relation, hop 3 the affiliated-with relation,
 * and the intermediate entities are persons]: the same brute force as above,
 * restricted to paths with rel_ok1[r1], rel_ok2[r2], rel_ok3[r3] (arrays of R
 * flags) and type_ok_u[vtypes[u]], type_ok_v[vtypes[v]] (arrays of 256 flags).
 */
int oracle_topk_paths_masked(const int64_t* offsets, const uint32_t* cols, const uint16_t* rels,
                             int64_t n, const uint8_t* vtypes, const void* vemb, const void* remb,
                             int dtype, int d, int fn, double gamma, uint32_t s, uint32_t t,
                             const uint8_t* rel_ok1, const uint8_t* rel_ok2, const uint8_t* rel_ok3,
                             const uint8_t* type_ok_u, const uint8_t* type_ok_v, int64_t K,
                             oracle_path* out, int64_t* n_out) {
    if ((int64_t)s >= n || (int64_t)t >= n || s == t || K <= 0) return ORACLE_EINVAL;
    khe h;
    h.a = (oracle_path*)malloc(sizeof(oracle_path) * (size_t)K);
    if (!h.a) return ORACLE_ENOMEM;
    h.size = 0;
    h.cap = K;
    for (int64_t i = offsets[s]; i < offsets[s + 1]; ++i) {
        uint32_t u = cols[i];
        uint16_t r1 = rels[i];
        if (u == s || u == t) continue;
        if (!rel_ok1[r1] || !type_ok_u[vtypes[u]]) continue;
        double w1 = oracle_edge_weight(vemb, remb, dtype, d, fn, gamma, s, r1, u);
        for (int64_t j = offsets[u]; j < offsets[u + 1]; ++j) {
            uint32_t v = cols[j];
            uint16_t r2 = rels[j];
            if (v == s || v == t || v == u) continue;
            if (!rel_ok2[r2] || !type_ok_v[vtypes[v]]) continue;
            int64_t k = lower_bound_u32(cols, offsets[v], offsets[v + 1], t);
            if (k >= offsets[v + 1] || cols[k] != t) continue;
            double w2 = oracle_edge_weight(vemb, remb, dtype, d, fn, gamma, u, r2, v);
            for (; k < offsets[v + 1] && cols[k] == t; ++k) {
                uint16_t r3 = rels[k];
                if (!rel_ok3[r3]) continue;
                double w3 = oracle_edge_weight(vemb, remb, dtype, d, fn, gamma, v, r3, t);
                oracle_path p;
                p.score = (w1 + w2) + w3;
                p.u = u;
                p.v = v;
                p.r1 = r1;
                p.r2 = r2;
                p.r3 = r3;
                p.pad = 0;
                khe_push(&h, &p);
            }
        }
    }
    qsort(h.a, (size_t)h.size, sizeof(oracle_path), cmp_rank);
    memcpy(out, h.a, sizeof(oracle_path) * (size_t)h.size);
    *n_out = h.size;
    free(h.a);
    return ORACLE_OK;
}

/* Many queries, independent, in parallel over queries (OpenMP when built with it). */
int oracle_topk_paths_batch(const int64_t* offsets, const uint32_t* cols, const uint16_t* rels,
                            int64_t n, const void* vemb, const void* remb, int dtype, int d, int fn,
                            double gamma, int64_t nq, const uint32_t* S, const uint32_t* T,
                            int64_t K, oracle_path* out, int64_t* n_out, int32_t* status) {
    int any = ORACLE_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nq; ++q) {
        int st = oracle_topk_paths(offsets, cols, rels, n, vemb, remb, dtype, d, fn, gamma, S[q],
                                   T[q], K, out + q * K, &n_out[q], NULL, NULL);
        status[q] = st;
        if (st != ORACLE_OK) {
#pragma omp atomic write
            any = st;
        }
    }
    return any;
}

/* ------------------------------------------------------------------------ */
/*
 * Tail prediction [Alg. 3 scores every person against the aggregated
 * Turing-award embedding; Alg. 4 scores every university for one person]:
 * for a head h and a relation r, every candidate vertex c -- the vertices
 * with vtypes[c] == cand_type, or all vertices when cand_type < 0 -- gets the
 * edge weight w(h, r, c) above, and the K best are kept in the order score
 * descending, then c ascending.  The paper's loops skip no candidate, so the
 * head is a candidate too when its type matches.  The bounded heap of the
 * path search is reused with the candidate in the u field and zero relation
 * fields, which makes its order (score desc, u asc) exactly this order.
 */
typedef struct {
    double score;
    uint32_t v;
    uint32_t pad;
} oracle_tail;                      /* 16 bytes, same layout as the library's */

int oracle_tail_topk(const uint8_t* vtypes, int64_t n, int64_t R, const void* vemb,
                     const void* remb, int dtype, int d, int fn, double gamma, uint32_t h,
                     uint32_t r, int cand_type, int64_t K, oracle_tail* out, int64_t* n_out) {
    if ((int64_t)h >= n || (int64_t)r >= R || K <= 0) return ORACLE_EINVAL;
    khe hp;
    hp.a = (oracle_path*)malloc(sizeof(oracle_path) * (size_t)K);
    if (!hp.a) return ORACLE_ENOMEM;
    hp.size = 0;
    hp.cap = K;
    for (int64_t c = 0; c < n; ++c) {
        if (cand_type >= 0 && (int)vtypes[c] != cand_type) continue;
        oracle_path p;
        memset(&p, 0, sizeof p);
        p.score = oracle_edge_weight(vemb, remb, dtype, d, fn, gamma, h, r, (uint32_t)c);
        p.u = (uint32_t)c;
        khe_push(&hp, &p);
    }
    qsort(hp.a, (size_t)hp.size, sizeof(oracle_path), cmp_rank);
    for (int64_t i = 0; i < hp.size; ++i) {
        out[i].score = hp.a[i].score;
        out[i].v = hp.a[i].u;
        out[i].pad = 0;
    }
    *n_out = hp.size;
    free(hp.a);
    return ORACLE_OK;
}

/* Many tail queries (H[q], Rq[q]), in parallel over queries. */
int oracle_tail_topk_batch(const uint8_t* vtypes, int64_t n, int64_t R, const void* vemb,
                           const void* remb, int dtype, int d, int fn, double gamma, int64_t nq,
                           const uint32_t* H, const uint32_t* Rq, int cand_type, int64_t K,
                           oracle_tail* out, int64_t* n_out, int32_t* status) {
    int any = ORACLE_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nq; ++q) {
        int st = oracle_tail_topk(vtypes, n, R, vemb, remb, dtype, d, fn, gamma, H[q], Rq[q],
                                  cand_type, K, out + q * K, &n_out[q]);
        status[q] = st;
        if (st != ORACLE_OK) {
#pragma omp atomic write
            any = st;
        }
    }
    return any;
}

/* ------------------------------------------------------------------------ */
/*
 * Generic H-hop search with a per-path beam [Alg. 6 and Alg. 7]:
 *   level 0 holds the one-vertex path (s).  At each of the H levels every held
 *   path p, whose last vertex is x, is extended by every out-edge (x, r, y)
 *   with y not already on p [Alg. 7 skips a neighbour already on the path]:
 *     score(p + (r, y)) = score(p) + w(x, r, y)      (fp64, left to right)
 *   - y == t: the extended path is a result [reaching the target ends the
 *     path]; the K best results are kept (one bounded heap for the query);
 *   - otherwise it competes in p's own bounded heap of K extensions, and the
 *     K best of that heap are the paths p contributes to the next level
 *     [UpdateNextPaths in Alg. 7 moves the local heap into the next array].
 *   Paths held after the last level are dropped.  The beam is per path: level
 *   l holds up to K^l paths (the bound Alg. 6 computes for its path arrays).
 * Orders (total, so the result is unique):
 *   within one path's heap: score descending, then (r, y) ascending (the
 *     extensions of one path differ only in their last edge);
 *   results: score descending, then hop count ascending, then the sequence
 *     (y_1, r_1, y_2, r_2, ..., y_{h-1}, r_{h-1}, r_h) ascending, which for
 *     three hops is (u, r1, v, r2, r3) as in the three-hop search.
 * The generic ExtendEmbedding / ComputeScore of Alg. 7 are read as the sum of
 * the edge weights, as in the three-hop search.
 */
#define ORACLE_BEAM_MAX_H 8

typedef struct {
    double score;
    int32_t hops;
    uint32_t v[ORACLE_BEAM_MAX_H + 1];   /* v[0] = s, v[hops] = last vertex */
    uint16_t r[ORACLE_BEAM_MAX_H];       /* r[i]: relation of edge v[i] -> v[i+1] */
} oracle_bpath;

/* 1 if a ranks strictly before b among the results */
static int beam_result_before(const oracle_bpath* a, const oracle_bpath* b) {
    if (a->score != b->score) return a->score > b->score;
    if (a->hops != b->hops) return a->hops < b->hops;
    for (int i = 1; i < a->hops; ++i) {
        if (a->v[i] != b->v[i]) return a->v[i] < b->v[i];
        if (a->r[i - 1] != b->r[i - 1]) return a->r[i - 1] < b->r[i - 1];
    }
    return a->r[a->hops - 1] < b->r[b->hops - 1];
}

/* 1 if a ranks strictly before b among the extensions of one path */
static int beam_ext_before(const oracle_bpath* a, const oracle_bpath* b) {
    if (a->score != b->score) return a->score > b->score;
    const int h = a->hops;
    if (a->r[h - 1] != b->r[h - 1]) return a->r[h - 1] < b->r[h - 1];
    return a->v[h] < b->v[h];
}

typedef int (*bpath_before)(const oracle_bpath*, const oracle_bpath*);

/* bounded heap of the best `cap` paths; the root is the worst kept one */
typedef struct {
    oracle_bpath* a;
    int64_t size, cap;
    bpath_before before;
} bheap;

static void bheap_push(bheap* h, const oracle_bpath* p) {
    oracle_bpath tmp;
    if (h->size < h->cap) {
        int64_t i = h->size++;
        h->a[i] = *p;
        while (i > 0) {
            int64_t par = (i - 1) / 2;
            if (!h->before(&h->a[par], &h->a[i])) break;
            tmp = h->a[par];
            h->a[par] = h->a[i];
            h->a[i] = tmp;
            i = par;
        }
        return;
    }
    if (!h->before(p, &h->a[0])) return;
    h->a[0] = *p;
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, w = i;
        if (l < h->size && h->before(&h->a[w], &h->a[l])) w = l;
        if (r < h->size && h->before(&h->a[w], &h->a[r])) w = r;
        if (w == i) break;
        tmp = h->a[w];
        h->a[w] = h->a[i];
        h->a[i] = tmp;
        i = w;
    }
}

/* pop everything, best first, into out (the heap is emptied) */
static void bheap_drain_sorted(bheap* h, oracle_bpath* out) {
    int64_t n = h->size;
    for (int64_t k = n - 1; k >= 0; --k) {
        out[k] = h->a[0];                    /* the worst remaining */
        h->a[0] = h->a[--h->size];
        int64_t i = 0;
        for (;;) {
            int64_t l = 2 * i + 1, r = l + 1, w = i;
            if (l < h->size && h->before(&h->a[w], &h->a[l])) w = l;
            if (r < h->size && h->before(&h->a[w], &h->a[r])) w = r;
            if (w == i) break;
            oracle_bpath tmp = h->a[w];
            h->a[w] = h->a[i];
            h->a[i] = tmp;
            i = w;
        }
    }
}

int oracle_beam_paths(const int64_t* offsets, const uint32_t* cols, const uint16_t* rels, int64_t n,
                      const void* vemb, const void* remb, int dtype, int d, int fn, double gamma,
                      uint32_t s, uint32_t t, int32_t H, int64_t K, oracle_bpath* out, int64_t* n_out,
                      int64_t* expanded_out) {
    if ((int64_t)s >= n || (int64_t)t >= n || s == t || K <= 0 || H < 1 || H > ORACLE_BEAM_MAX_H)
        return ORACLE_EINVAL;
    /* level l holds at most K^l paths; the caller keeps K^(H-1) within memory */
    double cap_d = 1.0;
    for (int l = 0; l < H - 1; ++l) cap_d *= (double)K;
    if (cap_d > 1e6) return ORACLE_EINVAL;
    const int64_t cap = (int64_t)cap_d;
    oracle_bpath* curr = (oracle_bpath*)calloc((size_t)cap, sizeof(oracle_bpath));
    oracle_bpath* next = (oracle_bpath*)calloc((size_t)cap, sizeof(oracle_bpath));
    bheap res = {(oracle_bpath*)malloc(sizeof(oracle_bpath) * (size_t)K), 0, K, beam_result_before};
    bheap loc = {(oracle_bpath*)malloc(sizeof(oracle_bpath) * (size_t)K), 0, K, beam_ext_before};
    if (!curr || !next || !res.a || !loc.a) {
        free(curr);
        free(next);
        free(res.a);
        free(loc.a);
        return ORACLE_ENOMEM;
    }
    int64_t n_curr = 1, n_next, expanded = 0;
    curr[0].score = 0.0;
    curr[0].hops = 0;
    curr[0].v[0] = s;
    for (int level = 0; level < H; ++level) {
        n_next = 0;
        for (int64_t p = 0; p < n_curr; ++p) {
            const oracle_bpath* path = &curr[p];
            const uint32_t x = path->v[path->hops];
            loc.size = 0;
            ++expanded;
            for (int64_t e = offsets[x]; e < offsets[x + 1]; ++e) {
                const uint32_t y = cols[e];
                int on_path = 0;
                for (int i = 0; i <= path->hops; ++i)
                    if (path->v[i] == y) on_path = 1;
                if (on_path) continue;
                oracle_bpath q = *path;
                q.score = path->score + oracle_edge_weight(vemb, remb, dtype, d, fn, gamma, x, rels[e], y);
                q.r[q.hops] = rels[e];
                q.hops += 1;
                q.v[q.hops] = y;
                if (y == t) bheap_push(&res, &q);
                else bheap_push(&loc, &q);
            }
            if (level + 1 < H) {     /* p's K best extensions go to the next level */
                const int64_t c = loc.size;
                bheap_drain_sorted(&loc, next + n_next);
                n_next += c;
            }
        }
        oracle_bpath* tmp = curr;
        curr = next;
        next = tmp;
        n_curr = n_next;
    }
    const int64_t nr = res.size;
    bheap_drain_sorted(&res, out);
    *n_out = nr;
    if (expanded_out) *expanded_out = expanded;
    free(curr);
    free(next);
    free(res.a);
    free(loc.a);
    return ORACLE_OK;
}

/* Many beam queries, in parallel over queries; out holds K paths per query. */
int oracle_beam_paths_batch(const int64_t* offsets, const uint32_t* cols, const uint16_t* rels, int64_t n,
                            const void* vemb, const void* remb, int dtype, int d, int fn, double gamma,
                            int64_t nq, const uint32_t* S, const uint32_t* T, int32_t H, int64_t K,
                            oracle_bpath* out, int64_t* n_out, int32_t* status) {
    int any = ORACLE_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nq; ++q) {
        int st = oracle_beam_paths(offsets, cols, rels, n, vemb, remb, dtype, d, fn, gamma, S[q], T[q], H, K,
                                   out + q * K, &n_out[q], NULL);
        status[q] = st;
        if (st != ORACLE_OK) {
#pragma omp atomic write
            any = st;
        }
    }
    return any;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Per-query frontier statistics (the counts the library's byte model uses).
 * In-degrees are counted from the edge array directly.
 */
int oracle_query_stats(const int64_t* offsets, const uint32_t* cols, int64_t n, uint32_t s,
                       uint32_t t, oracle_stats* st) {
    if ((int64_t)s >= n || (int64_t)t >= n || s == t) return ORACLE_EINVAL;
    int64_t E = offsets[n];
    int64_t* indeg = (int64_t*)calloc((size_t)n, sizeof(int64_t));
    if (!indeg) return ORACLE_ENOMEM;
    for (int64_t e = 0; e < E; ++e) indeg[cols[e]]++;
    memset(st, 0, sizeof *st);
    st->deg_s = offsets[s + 1] - offsets[s];
    st->deg_t = indeg[t];
    for (int64_t i = offsets[s]; i < offsets[s + 1]; ++i) {
        uint32_t u = cols[i];
        if (u == s || u == t) continue;
        if (i > offsets[s] && cols[i - 1] == u) continue;   /* count each u once */
        st->n_u++;
        st->s_f += offsets[u + 1] - offsets[u];
    }
    for (int64_t v = 0; v < n; ++v) {
        if (v == s || v == t) continue;
        int64_t k = lower_bound_u32(cols, offsets[v], offsets[v + 1], t);
        if (k < offsets[v + 1] && cols[k] == t) {
            st->n_v++;
            st->s_b += indeg[v];
        }
    }
    free(indeg);
    return ORACLE_OK;
}
