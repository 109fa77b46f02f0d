/*
 * mhr.h - C ABI of the GB300 exact three-hop top-K path-search library
 * (libmhr.so, sm_103a).
 *
 * Problem (Sec. 3.1; Sec. 5, Alg. 6 and Alg. 7): given a typed knowledge graph
 * as (h, r, t) triples, an entity embedding table and a relation embedding
 * table, return the K best paths s -r1-> u -r2-> v -r3-> t.
 *   - Edge weight (Alg. 3, Alg. 4): TransE-L1  w = gamma - sum_j |e_u + w_r - e_v|_j
 *     with gamma = 1.0 in the paper, or DistMult w = sum_j e_u[j] w_r[j] e_v[j]
 *     (a bilinear choice for the generic ComputeScore of Alg. 7, which the
 *     paper leaves open).
 *   - Paths are simple: u not in {s, t}, v not in {s, t, u} (Alg. 7 skips a
 *     neighbour already on the path; reaching t ends a path).
 *   - Path score = sum of its three edge weights.
 *   - Result order: score descending, then (u, r1, v, r2, r3) ascending.  This
 *     is a total order, so the result is unique.
 * Every result is exact: candidates are screened in fp32 with a proven error
 * bound and the boundary candidates are rescored in fp64 in a fixed operation
 * order, so scores and order equal an fp64 brute-force enumeration
 * (j = 0..d-1 in order, no fused multiply-add).
 * The library also provides the tail-prediction scan of Alg. 3 / Alg. 4
 * (mhr_tail_topk): the K best candidate vertices of one type for
 * (head, relation) queries, exact in the same way; and the generic H-hop
 * search with a per-path beam of Alg. 6 / Alg. 7 (mhr_beam_paths).
 *
 * Conventions for every entry point:
 *   - Status codes are returned, never raised; mhr_last_error() gives a
 *     thread-local message for the last non-OK status of the calling thread.
 *   - The caller owns every buffer it passes.  mhr_graph_load copies what it
 *     needs; the graph handle owns its device copy until mhr_graph_free.
 *   - cuda_stream is a cudaStream_t (NULL = the legacy default stream).
 *   - The device is the one current on the calling thread when the graph is
 *     loaded; later calls on that graph must use the same device.
 *   - A graph handle keeps per-shape query plans (buffers and captured CUDA
 *     graphs); calls on one handle must not run concurrently from several
 *     host threads.  Different handles are independent.
 */
#ifndef MHR_H
#define MHR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MHR_OK = 0,
    MHR_EINVAL = 1,   /* invalid argument or invalid graph */
    MHR_ENOMEM = 2,   /* host or device allocation failed */
    MHR_ECUDA = 3,    /* a CUDA call or kernel failed */
    MHR_ETIMEOUT = 4, /* a bounded device wait gave up */
    MHR_ERANGE = 5    /* K or a size beyond a documented limit */
} mhr_status;

typedef enum {
    MHR_SCORE_TRANSE_L1 = 0, /* gamma - ||e_u + w_r - e_v||_1 (Alg. 3, Alg. 4) */
    MHR_SCORE_DISTMULT = 1   /* <e_u * w_r, e_v> */
} mhr_score_fn;

typedef enum { MHR_F32 = 0, MHR_BF16 = 1 } mhr_dtype;
typedef enum { MHR_MEM_HOST = 0, MHR_MEM_DEVICE = 1 } mhr_mem;

/* Largest K a query accepts; larger K returns MHR_ERANGE. */
#define MHR_K_MAX 1024

typedef struct mhr_graph mhr_graph; /* opaque; owned by the library */

/*
 * Graph description (Sec. 3.1: edge list, entity embeddings, relation
 * embeddings).  All arrays are borrowed for the duration of mhr_graph_load.
 *   offsets     int64[n_vertices + 1]  CSR row starts by source vertex;
 *               offsets[0] = 0, non-decreasing, offsets[n] = n_edges
 *   cols        uint32[n_edges]        destination of each edge
 *   rels        uint16[n_edges]        relation id of each edge, < n_relations
 *   vtypes      uint8[n_vertices]      vertex type ids (may be NULL: all 0)
 *   vertex_emb  [n_vertices x dim]     row-major, float32 or bfloat16 bits
 *   rel_emb     [n_relations x dim]    row-major, same dtype
 * Each row must be sorted by (col, rel) with no repeated (col, rel) and no
 * self loop; every embedding value must be finite; n_vertices, n_edges < 2^32.
 * mem tells whether the arrays are host or device pointers.
 */
typedef struct {
    int64_t n_vertices;
    int64_t n_edges;
    int32_t n_relations;
    int32_t n_vtypes;
    int32_t dim;
    int32_t reserved0;
    const int64_t* offsets;
    const uint32_t* cols;
    const uint16_t* rels;
    const uint8_t* vtypes;
    const void* vertex_emb;
    const void* rel_emb;
    mhr_dtype emb_dtype;
    mhr_mem mem;
    mhr_score_fn score_fn;
    int32_t reserved1;
    double gamma; /* TransE margin; the paper uses 1.0 */
} mhr_graph_desc;

/* One result path s -r1-> u -r2-> v -r3-> t; score is the fp64 sum of the
 * three edge weights.  24 bytes. */
typedef struct {
    double score;
    uint32_t u, v;
    uint16_t r1, r2, r3, pad;
} mhr_path;

/*
 * Ordering MLP (device pointers): y = w2 . relu(W1 x + b1) + b2 with x the 256
 * bfloat16 features [e_a[0:128]; e_b[0:128]] of two vertices (zero-padded when
 * dim < 128), 256 hidden units.  W1: bfloat16 bits [256 hidden x 256 in],
 * row-major; b1, w2: float[256]; b2: float[1].
 */
typedef struct {
    const uint16_t* W1;
    const float* b1;
    const float* w2;
    const float* b2;
} mhr_mlp;

/*
 * Constraints of a three-hop query (Sec. 3.1): the paper's query follows
 * award-winner, then works-in, then affiliated-with, and both intermediate
 * entities are persons; Alg. 1 extracts those vertex sets by type.  Here each
 * hop has a set of allowed relations and each intermediate vertex a set of
 * allowed vertex types; a path s -r1-> u -r2-> v -r3-> t is a result only when
 * r1, r2, r3 and the types of u and v are all allowed.  Scores, simple-path
 * rules and the result order are those of the unconstrained search.
 *   rel1, rel2, rel3  host arrays of n_relations bytes, nonzero = allowed;
 *                     NULL = every relation
 *   types_u, types_v  host arrays of 256 bytes indexed by vertex type,
 *                     nonzero = allowed; NULL = every type
 * The arrays are read during the call only.  They apply to every query of a
 * batched call.
 */
typedef struct {
    const uint8_t* rel1;
    const uint8_t* rel2;
    const uint8_t* rel3;
    const uint8_t* types_u;
    const uint8_t* types_v;
} mhr_constraints;

/* Query options; a NULL pointer means all defaults (zeros). */
typedef struct {
    int32_t chunk;       /* edges per work item of the middle join: 0 = default (16384), else a
                            multiple of 32 in [32, 32768] (MHR_EINVAL otherwise) */
    int32_t order;       /* order of intermediate vertices: 0 natural, 1 by score
                            bound, 2 by score bound refined inside bound levels by
                            the learned slack prediction of `mlp` */
    int32_t prune;       /* 1 = skip work items, rows and middle edges whose provable
                            score bound cannot reach the kept band (same result) */
    int32_t precision;   /* middle-edge screen: 0 fp32 CUDA cores; 1 bf16 tensor-core
                            contraction with hi/lo split and fp32 accumulation (DistMult,
                            at most 16 relations); the fp64 rescoring keeps results exact */
    const mhr_mlp* mlp;  /* order == 2 only */
    int32_t tile;        /* 32-edge groups each warp of the middle join scans per step:
                            0 = default (4), else 4 or 8 (MHR_EINVAL otherwise) */
    int32_t part_count;  /* vertex partition of the paths (the multi-GPU form of Sec. 3.3's
                            partitioned work): with part_count >= 2 only the paths whose
                            hop-1 vertex u has u % part_count == part_index are searched, so
                            part_count calls (one per GPU) cover every path exactly once and
                            mhr_merge_paths of their lists is the unpartitioned result.
                            0 or 1 = every path.  MHR_EINVAL unless 0 <= part_index <
                            part_count.  Not with mhr_training_labels. */
    const mhr_constraints* constraints;  /* NULL = unconstrained; see mhr_constraints.  The
                            work counters then count the combinations of allowed hop-1 and
                            hop-3 vertices and allowed middle edges, before the hop-1 and
                            hop-3 relation filter.  Not with mhr_training_labels. */
    int32_t part_index;  /* see part_count */
    int32_t reserved;
} mhr_query_opts;

/* Work counters of the last call (optional output). */
typedef struct {
    int64_t edges_scanned; /* middle-join CSR entries streamed */
    int64_t hits;          /* middle edges that joined both frontiers */
    int64_t paths;         /* simple s->t three-hop paths enumerated (scored) */
    int64_t candidates;    /* fp32 candidates kept for the final merge */
    int64_t rescored;      /* candidates rescored in fp64 */
    int64_t pruned_edges;  /* middle edges skipped by provable bounds */
    int64_t dense_queries; /* queries resolved by the exact (tie-heavy) path */
    double ms;             /* wall time of the call (synchronous calls only) */
    double ms_device;      /* device time of the whole launch sequence (CUDA events) */
    double ms_join;        /* device time of the middle-join kernel (CUDA events) */
    double ms_expand;      /* device time of the hop-1 / hop-3 expansion kernel (CUDA events;
                              batched three-hop search only) */
} mhr_stats;

/*
 * Upload a graph and build its device indexes: the reverse CSR (in-edges of
 * each vertex, sorted by (source, relation)) and the norms behind the fp32
 * error bound.  Validates the description (MHR_EINVAL with a message on any
 * violation).  Synchronous; *out is NULL on failure, and a failed load has
 * released every device allocation it made.  A service that must keep the
 * graph within a memory budget sets the environment variable
 * MHR_GRAPH_MEMORY_CAP_BYTES (decimal bytes, read at every load): a load
 * whose resident device arrays would exceed it fails with MHR_ENOMEM.
 */
mhr_status mhr_graph_load(const mhr_graph_desc* desc, mhr_graph** out, void* cuda_stream);

/* Release the device copy.  NULL is accepted. */
mhr_status mhr_graph_free(mhr_graph* g);

/*
 * Sizes of a loaded graph and the proven error bounds its searches screen
 * with.  The paper computes in fp32 (Sec. 4.2 builds with -Ofast) and states
 * no error; these bounds are what keeps the results here exact: an fp32 edge
 * weight is within eps32_edge of the exact one, and the fp32 score of a
 * three-hop path within err_path of its fp64 score (err_path_tc when the
 * middle edge comes from the bf16 tensor-core screen; DistMult only, else 0).
 * All fields are written; out is a host pointer.  MHR_EINVAL on NULL.
 */
typedef struct {
    int64_t n_vertices;
    int64_t n_edges;
    int32_t n_relations;
    int32_t dim;
    int64_t max_out_degree;
    int64_t max_in_degree;
    double eps32_edge;
    double eps64_edge;
    double err_path;
    double epstc_edge;
    double err_path_tc;
} mhr_graph_info;

mhr_status mhr_graph_get_info(const mhr_graph* g, mhr_graph_info* out);

/*
 * Edge weights w(src[i], rel[i], dst[i]) for i < n (Alg. 3, Alg. 4 score form).
 *   precision 0: float32 output, fp32 arithmetic (the screening arithmetic)
 *   precision 2: float64 output, the canonical fp64 operation order
 * src == NULL (then rel and dst must be NULL too): all edges in CSR order and
 * n must equal n_edges.  mem applies to src, rel, dst and out.  Asynchronous
 * on cuda_stream for device memory, synchronous for host memory.
 */
mhr_status mhr_edge_scores(const mhr_graph* g, const uint32_t* src, const uint16_t* rel,
                           const uint32_t* dst, int64_t n, int32_t precision, void* out,
                           mhr_mem mem, void* cuda_stream);

/*
 * One query, synchronous.  out: host array of K paths; *n_out = number
 * written (< K when fewer paths exist).  s, t < n_vertices, s != t,
 * 1 <= K <= MHR_K_MAX (else MHR_EINVAL / MHR_ERANGE).
 */
mhr_status mhr_topk_paths(const mhr_graph* g, uint32_t s, uint32_t t, int32_t K, mhr_path* out,
                          int32_t* n_out, const mhr_query_opts* opts, mhr_stats* stats);

/*
 * nq independent queries (s[i], t[i]) in one batched launch sequence that is
 * captured once into a CUDA graph and replayed.  out: nq*K paths (query i at
 * out[i*K]); n_out[i] = paths written for query i, or -1 when (s[i], t[i]) is
 * invalid (out of range or s == t).  mem applies to s, t, out and n_out.
 * Host memory: synchronous.  Device memory: asynchronous on cuda_stream
 * (the query sizes are read back once, a short synchronisation).  stats, if
 * not NULL, forces a synchronisation at the end.
 */
mhr_status mhr_topk_paths_batched(const mhr_graph* g, int32_t nq, const uint32_t* s,
                                  const uint32_t* t, int32_t K, mhr_path* out, int32_t* n_out,
                                  mhr_mem mem, const mhr_query_opts* opts, mhr_stats* stats,
                                  void* cuda_stream);

/*
 * Merge of partial top-K lists (Alg. 2, ReduceTopKTree: the per-thread K-best
 * lists are merged pairwise in a tree).  Here the lists are the results of
 * disjoint path sets of the same queries -- the parts of a vertex-partitioned
 * search (mhr_query_opts.part_count), one per GPU -- and the merge runs on the
 * GPU: log2(n_parts) rounds, each merging pairs of lists by the result order
 * (score descending, then (u, r1, v, r2, r3) ascending; every list must
 * already be in that order, as the search returns it) and keeping the first K.
 *   parts   n_parts * nq * K paths: part p, query i at parts[(p * nq + i) * K]
 *   n_parts_out  n_parts * nq counts (part p, query i at [p * nq + i]); -1
 *           (an invalid query) in any part makes the output count -1
 *   out     nq * K paths; n_out[i] = min(K, sum of the parts' counts)
 *   mem     where parts, n_parts_out, out and n_out live
 * The parts must not share a path (the result would repeat it).  Host
 * memory: synchronous.  Device memory: asynchronous on cuda_stream.
 * MHR_EINVAL on NULL pointers, nq < 0, n_parts < 1, K outside [1, MHR_K_MAX].
 */
mhr_status mhr_merge_paths(int32_t nq, int32_t K, int32_t n_parts, const mhr_path* parts, const int32_t* n_parts_out,
                           mhr_path* out, int32_t* n_out, mhr_mem mem, void* cuda_stream);

/*
 * Launch-shape autotuner for the batched search (the paper has no
 * counterpart; its OpenMP loops have no tunable shape).  Runs
 * mhr_topk_paths_batched on the nq queries (s, t; mem applies to both) with
 * opts and every combination of
 *   - middle-edge screen: opts->precision, or, when opts->precision < 0, both
 *     0 (fp32 CUDA cores) and 1 (bf16 tensor cores; only for DistMult with at
 *     most 16 relations);
 *   - work-item size chunks[i]: multiples of 32 in [32, 32768] (NULL:
 *     {8192, 16384, 32768}, n_chunks = 3);
 *   - scan tile tiles[j]: 4 or 8 (NULL: {4, 8}, n_tiles = 2).
 * Each combination gets one untimed run, then reps timed runs, timed by CUDA
 * events around the launch sequence on cuda_stream; ms_out (optional, host)
 * receives the fastest time of each combination at
 * [(p * n_chunks + i) * n_tiles + j], p indexing the screens tried in the
 * order above; *best_chunk, *best_tile and *best_precision (optional) (host)
 * = the fastest combination (the first one on ties).  Every run computes the
 * same result (discarded).  Keeps the winner's buffers and releases the
 * others'.  Synchronous.  MHR_EINVAL on bad arguments or candidates.
 */
mhr_status mhr_autotune(const mhr_graph* g, int32_t nq, const uint32_t* s, const uint32_t* t, int32_t K,
                        mhr_mem mem, const mhr_query_opts* opts, const int32_t* chunks, int32_t n_chunks,
                        const int32_t* tiles, int32_t n_tiles, int32_t reps, int32_t* best_chunk,
                        int32_t* best_tile, int32_t* best_precision, float* ms_out, void* cuda_stream);

/*
 * Learned ordering (the paper has no learned component; this implements the
 * ordering proposal of the spec design on top of the exact search).
 * All arrays are device memory; calls are asynchronous on cuda_stream.
 *
 * mhr_training_labels: runs the plain search (no pruning) on nq queries
 * (s, t: host arrays) and writes, for every intermediate vertex x scanned by
 * the join that lies on at least one path, one training row: near_v[i] = x,
 * end_v[i] = the query endpoint on the far side of x (t when x is a hop-1
 * vertex, s when it is a hop-3 vertex), own[i] = the provable upper bound of
 * the fp32 score of any path through x (the row bound the search prunes
 * with), best[i] = the best fp32 path score through x (<= own[i]).  With
 * order 2 a query orders rows by own + min(0, MLP(x, endpoint)), so the
 * network learns the slack best - own.  At most cap
 * rows; *n_written (host) = rows written, or the number needed when > cap
 * (then MHR_ERANGE).  Synchronous.
 */
mhr_status mhr_training_labels(const mhr_graph* g, int32_t nq, const uint32_t* s, const uint32_t* t,
                               int64_t cap, uint32_t* near_v, uint32_t* end_v, float* own, float* best,
                               int64_t* n_written, void* cuda_stream);

/* X[i] = bfloat16 features [e_va[i][0:128]; e_vb[i][0:128]], X is [n x 256]. */
mhr_status mhr_mlp_features(const mhr_graph* g, const uint32_t* va, const uint32_t* vb, int64_t n,
                            uint16_t* X, void* cuda_stream);

/* y[i] = MLP(X[i]); z1 (optional, [n x 256]) receives W1 x + b1. */
mhr_status mhr_mlp_forward(const mhr_mlp* m, const uint16_t* X, int64_t n, float* y, float* z1,
                           void* cuda_stream);

/*
 * Gradients of mean_i (y[i] - target[i])^2 for the y, z1 of mhr_mlp_forward:
 * grads = [dW1 (256x256 row-major) | db1 (256) | dw2 (256) | db2 (1)] fp32;
 * work: n x 256 floats of scratch; loss (optional, device float).
 */
mhr_status mhr_mlp_backward(const mhr_mlp* m, const uint16_t* X, int64_t n, const float* target,
                            const float* y, const float* z1, float* work, float* grads, float* loss,
                            void* cuda_stream);

/* One Adam step on count parameters (step >= 1, bias-corrected). */
mhr_status mhr_mlp_adam(float* params, const float* grads, float* m1, float* m2, int64_t count,
                        float lr, float beta1, float beta2, float eps, int32_t step, void* cuda_stream);

/* dst[i] = bfloat16(src[i]) (round to nearest even). */
mhr_status mhr_mlp_to_bf16(const float* src, uint16_t* dst, int64_t count, void* cuda_stream);

/*
 * mhr_topk_paths_noalloc - one query, like mhr_topk_paths, for callers that
 * cannot allocate device memory.  The paper has no counterpart; this is a
 * deployment entry point.  Callers that cannot allocate: services that must
 * keep a fixed device-memory footprint once started, hosts whose own
 * allocator owns the device memory (a raw allocation would fail or fragment
 * it), and latency-critical sections where the implicit device
 * synchronisation of cudaMalloc/cudaFree is not acceptable.
 *   out    device array of K mhr_path; n_out device pointer to one int32
 *          (paths written).  Same result as mhr_topk_paths (same order,
 *          bit-identical scores).
 *   Asynchronous on cuda_stream.  Allocates nothing: its only scratch is a
 *   fixed device array of about 1 MiB, defined at file scope in the library,
 *   which every GPU that loads the library holds until the process exits.
 *   Limits: out-degree of s and in-degree of t each <= 65536, else
 *   MHR_ERANGE; 1 <= K <= MHR_K_MAX; s, t valid and s != t (MHR_EINVAL).
 *   The first call on each device looks up the device address of that array
 *   and sets the kernel's shared-memory attribute; make that first call
 *   before any stream capture.  Every call on a device shares the array and
 *   it keeps the last call's contents (each call writes every cell it reads),
 *   so calls that overlap on the GPU (other streams, other threads) race:
 *   serialise them.  The looked-up address is kept for the life of the
 *   process; cudaDeviceReset invalidates it, so do not reset a device that
 *   this entry point has run on and then call it again.
 *   Cost: one thread block on one SM walks every middle edge out of the
 *   hop-1 vertices (the sum of their out-degrees), so the time grows with
 *   that sum; a hub source on a power-law graph can make one call take
 *   seconds.  mhr_topk_paths_batched spreads the same work over every SM.
 */
mhr_status mhr_topk_paths_noalloc(const mhr_graph* g, uint32_t s, uint32_t t, int32_t K, mhr_path* out,
                                  int32_t* n_out, void* cuda_stream);

/*
 * Tail prediction (Alg. 3 and Alg. 4): Alg. 3 scores every person against the
 * Turing-award embedding aggregated with the award-winner relation, Alg. 4
 * every university against one person and the affiliation relation; both
 * keep the K best with per-thread heaps merged by a tree (Alg. 2).  Here, for
 * each query i, every candidate vertex c -- the vertices with
 * vtypes[c] == cand_type, or every vertex when cand_type == -1 -- is scored
 * with the graph's edge weight w(h[i], r[i], c) (no edge needs to exist), and
 * the K best are returned in the order score descending, then c ascending
 * (a total order, so the result is unique).  The head itself is a candidate
 * when its type matches: the paper's loops exclude no candidate.  Scores are
 * screened in fp32 with the graph's proven error bound and the boundary
 * candidates are rescored in fp64 in the canonical operation order, so
 * results are bit-identical to an fp64 brute force.
 *   h, r      nq heads (< n_vertices) and relations (< n_relations)
 *   out       nq*K records (query i at out[i*K]); n_out[i] = records written,
 *             min(K, number of candidates)
 *   mem       where h, r, out and n_out live (host or device)
 *   stats     optional (host): edges_scanned = (query, candidate) pairs scored
 *             in fp32 (the sampling pass included), candidates = fp32
 *             survivors of the threshold, rescored = candidates rescored in
 *             fp64, dense_queries = queries whose survivors overflowed the
 *             sized buffer and were rescanned alone, ms = wall time,
 *             ms_device = device time of the call, ms_join = device time of
 *             the full scans; hits, paths and pruned_edges are 0.
 * Synchronous.  MHR_EINVAL: NULL pointers, a head or relation out of range,
 * cand_type outside [-1, 255], K < 1; MHR_ERANGE: K > MHR_TAIL_K_MAX or
 * dim > 16383.  nq == 0 is a no-op.  The first query of a vertex type builds
 * and keeps that type's candidate list on the device (4 bytes per vertex of
 * the type, freed with the graph).
 */
#define MHR_TAIL_K_MAX 4096

/* One tail-prediction result: candidate v with its fp64 score.  16 bytes. */
typedef struct {
    double score;
    uint32_t v;
    uint32_t pad;
} mhr_tail;

mhr_status mhr_tail_topk(const mhr_graph* g, int32_t nq, const uint32_t* h, const uint16_t* r,
                         int32_t cand_type, int32_t K, mhr_tail* out, int32_t* n_out, mhr_mem mem,
                         mhr_stats* stats, void* cuda_stream);

/*
 * Generic H-hop search with a per-path beam (Alg. 6 and Alg. 7), exact.  For
 * each query (s[i], t[i]): level 0 holds the path (s); at each of H levels
 * every held path p ending at x is extended by every out-edge (x, r, y) with y
 * not on p, scored score(p) + w(x, r, y) (fp64, the reference operation
 * order).  y == t makes a result (reaching the target ends a path); otherwise
 * the extension competes in p's own list of K, and p's K best extensions
 * (score desc, then relation, then vertex ascending) are held at the next
 * level, so level l holds up to K^l paths (Alg. 6 sizes its path arrays so).
 * The K best results are returned in the order score descending, hop count
 * ascending, then (y_1, r_1, ..., y_{h-1}, r_{h-1}, r_h) ascending, the vertex
 * and relation sequence after s (for three hops: (u, r1, v, r2, r3)).
 *   out    nq*K records (query i at out[i*K]); n_out[i] = results written
 *   mem    where s, t, out and n_out live
 *   stats  optional: edges_scanned = out-edges scored (fp32 screen),
 *          rescored = extensions and results scored in fp64; ms = wall time
 * Each held path's extensions are screened in fp32 with the graph's proven
 * edge bound: only those within that bound (plus the spacing of the rounded
 * path scores) of the path's K-th fp32 extension are scored in fp64, so every
 * selection is the fp64 one.
 * Synchronous.  MHR_EINVAL: NULL arrays, a vertex out of range, s == t,
 * H outside [1, MHR_BEAM_MAX_H], K < 1; MHR_ERANGE: K > MHR_BEAM_K_MAX or
 * K^(H-1) > 65536.  nq == 0 is a no-op.
 */
#define MHR_BEAM_MAX_H 8
#define MHR_BEAM_K_MAX 64

/* One beam-search result: v[0] = s, v[hops] = t, r[i] the relation of the
 * edge v[i] -> v[i+1].  64 bytes. */
typedef struct {
    double score;
    int32_t hops;
    uint32_t v[MHR_BEAM_MAX_H + 1];
    uint16_t r[MHR_BEAM_MAX_H];
} mhr_beam_path;

mhr_status mhr_beam_paths(const mhr_graph* g, int32_t nq, const uint32_t* s, const uint32_t* t, int32_t H,
                          int32_t K, mhr_beam_path* out, int32_t* n_out, mhr_mem mem, mhr_stats* stats,
                          void* cuda_stream);

/* Thread-local description of the last non-OK status ("" if none). */
const char* mhr_last_error(void);

/* Library version string. */
const char* mhr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MHR_H */
