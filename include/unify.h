/*
 * unify.h - C ABI of the GB300 range-filtered k-NN search over an HSIG.
 *
 * The operation (Definition 1, Section 2.1 of "UNIFY: Unified Index for Range
 * Filtered Approximate Nearest Neighbors Search"): for each query (q, [lo, hi], k)
 * return the k objects v with lo <= v[A] <= hi nearest to q, or all of them when
 * fewer than k exist. Distances are squared L2 (the paper's Euclidean distance,
 * Section 5.1, ranks identically). Ties in distance are broken by id.
 *
 * Search strategies (Section 4.2):
 *   UNIFY_PRE     Strategy A, pre-filtering: exhaustive scan of the in-range
 *                 objects, located through the attribute order. Exact.
 *   UNIFY_HYBRID  Strategy C, hybrid filtering: Algorithm 2's layer scheme with
 *                 Algorithm 7 per layer; only chunks of intersected segments are
 *                 followed, the first ceil(m / S') slots of each (selection S2).
 *   UNIFY_POST    Strategy B, post-filtering: Algorithm 2 with Algorithm 1 over
 *                 the bitmap-marked (global) edges, beam ef_post, then the range
 *                 filter and the first k.
 *   UNIFY_AUTO    Range-aware selection: Y = |{v : lo <= v[A] <= hi}|;
 *                 A if Y <= tau_A, B if Y >= tau_B, otherwise C.
 *
 * Conventions shared by every entry point:
 *   - Return value: UNIFY_OK (0) or a negative UNIFY_E_* code; the message of the
 *     last failure on the calling thread is returned by unify_last_error().
 *   - Device pointers are CUDA device (or managed) memory on the index's device
 *     and stay owned by the caller. Work is enqueued on `stream` (a cudaStream_t,
 *     NULL = the legacy default stream) and is asynchronous unless stated.
 *   - Output rows hold min(k, found) results sorted by (distance, id); the rest of
 *     the row is padded with id -1 and distance +inf. lo > hi is an empty range
 *     (count 0), not an error.
 *   - Attributes are int64; lo and hi are inclusive.
 *   - One index may serve one search at a time: concurrent searches on the same
 *     index from different streams race on its scratch buffers.
 */
#ifndef UNIFY_H
#define UNIFY_H

#include <stdint.h>

#if defined(__GNUC__)
#define UNIFY_API __attribute__((visibility("default")))
#else
#define UNIFY_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct unify_index unify_index_t; /* opaque, library-owned */
typedef struct unify_plan unify_plan_t;   /* opaque: a captured search (CUDA graph) */

typedef enum {
  UNIFY_AUTO = -1,
  UNIFY_PRE = 0,
  UNIFY_HYBRID = 1,
  UNIFY_POST = 2
} unify_strategy_t;

typedef enum {
  UNIFY_FP32 = 0,    /* traversal and scan read the float32 vectors */
  UNIFY_BF16 = 1,    /* read a bfloat16 copy (RNE), FP32 accumulate, FP32 re-rank */
  UNIFY_FP8E4M3 = 2  /* read an FP8 E4M3 copy with a per-vector float32 scale
                        s = max|x| / 448, FP32 accumulate, FP32 re-rank */
} unify_dtype_t;

/* Return codes. */
#define UNIFY_OK 0
#define UNIFY_E_ARG (-1)     /* invalid argument (null pointer, bad size, k < 1, ...) */
#define UNIFY_E_IO (-2)      /* index file missing or unreadable */
#define UNIFY_E_FORMAT (-3)  /* index file malformed or checksum mismatch */
#define UNIFY_E_NOMEM (-4)   /* host or device allocation failed */
#define UNIFY_E_CUDA (-5)    /* a CUDA call failed (message has the CUDA error) */
#define UNIFY_E_LIMIT (-6)   /* a size exceeds a compiled limit (message says which) */

/* Per-query status bits written to out_status. */
#define UNIFY_Q_LIMIT 1u      /* the expansion bound (max_expansions) stopped a layer, or a
                                 wait of the tensor-core scan ran out (empty row) */
#define UNIFY_Q_TRUNCATED 2u  /* the candidate buffer overflowed and dropped its worst
                                 entries; the result is valid but may differ from the
                                 unbounded algorithm */

/* Search parameters. unify_default_params() fills the defaults shown. */
typedef struct {
  int ef;              /* Algorithm 7 layer-0 beam (ann capacity), default 100 */
  int m;               /* hybrid neighbours visited per expanded object, default 16 (S2:
                          ceil(m / S') per intersected chunk; S1: the m nearest) */
  int ef_post;         /* Algorithm 1 layer-0 beam of Strategy B; <= 0 means ef */
  int rerank_mult;     /* BF16/FP8 storage: re-rank rerank_mult * k candidates in FP32 (the
                          tensor-core scan: see tc_scan), default 4 */
  unify_dtype_t dtype; /* storage read by traversal and scan, default UNIFY_FP32 */
  int64_t tau_a;       /* Strategy A when Y <= tau_a; < 0 means floor(0.01 n) */
  int64_t tau_b;       /* Strategy B when Y >= tau_b; < 0 means floor(0.5 n) */
  int cand_cap;        /* candidate buffer entries per query, default 512 (<= 4096) */
  int visited_cap;     /* visited-filter slots per query, power of two, default 2048 */
  int max_expansions;  /* expansions per layer before UNIFY_Q_LIMIT, default 100000 */
  int warps_per_block; /* search warps per CTA (one query or scan item each), 1..4, default 4 */
  int scan_rows;       /* pre-filter rows per scan work item, default 8192 */
  int reg_budget;      /* registers per thread of the search kernel: 128 (16 warps per SM),
                          80 (24 warps) or 64 (32 warps, smaller distance groups); default 128.
                          More resident warps hide more memory latency when shared memory
                          (cand_cap, visited_cap, ef) also fits. */
  int tc_scan;         /* 1: Strategy A queries are scanned on the tensor cores (tcgen05 MMA
                          over TMA-staged row tiles shared by 128 queries; bf16 operands for
                          UNIFY_BF16 storage, tf32 for UNIFY_FP32, E4M3 for UNIFY_FP8E4M3; the
                          top R by that distance re-ranked in FP32, R = rerank_mult * k up
                          to 64 and R = k past that) when d <= 1024, k <= 128 and the rows
                          suit TMA (the padded
                          d a multiple of 8 for BF16, of 16 for FP8); otherwise, and with
                          0 (default), the warp scan. 2: test of the scan's failure path only:
                          the scan's collecting pass waits on a barrier that nothing arrives
                          at, every wait between its roles is limited to 50 ms, the waits run
                          out, and the pre-filter rows come back empty with UNIFY_Q_LIMIT
                          (the call itself succeeds; the next search is unaffected) */
  int selection;       /* hybrid neighbour selection (Section 4.2; Section 5.6 compares the two):
                          2 (default) = S2, the first ceil(m / S') slots of every intersected
                          chunk; 1 = S1, the m neighbours nearest to the expanded object among
                          all slots of the intersected chunks (m <= 64) */
} unify_params_t;

/* Fills *p with the defaults above. */
UNIFY_API void unify_default_params(unify_params_t* p);

/* Reads the serialised HSIG at `path` (written by the host builder), verifies its
 * section checksums and copies it to `device`; the attribute-sorted vector copy
 * and the positions are derived on the device. On success *out owns the device
 * memory until unify_free_index. Synchronous. Errors: UNIFY_E_ARG, UNIFY_E_IO,
 * UNIFY_E_FORMAT, UNIFY_E_NOMEM, UNIFY_E_CUDA. */
UNIFY_API int unify_load_index(const char* path, int device, unify_index_t** out);

/* Releases every device and host buffer of the index (NULL is ignored). The caller
 * must make sure no search on the index is still running. */
UNIFY_API void unify_free_index(unify_index_t* idx);

/* Index sizes; any output pointer may be NULL. */
UNIFY_API int unify_index_info(const unify_index_t* idx, int64_t* n, int* d, int* S, int* M, int* max_level);

/* Range resolution and range-aware selection for nq queries (device pointers):
 *   out_pa[i] = #{v : v[A] < lo[i]}, out_pb[i] = max(pa, #{v : v[A] <= hi[i]})
 *       (the in-range objects are positions [pa, pb) of the attribute order, so
 *        Y = pb - pa; the skip-list descent of Strategy A lands on position pa);
 *   out_mask[i] bit j: segment j holds objects, b_j <= hi and lo < b_{j+1}
 *       (segments are half-open [b_j, b_{j+1}) with b_0 = -inf, b_S = +inf);
 *   out_strategy[i] = UNIFY_PRE / UNIFY_HYBRID / UNIFY_POST by Y vs tau_a, tau_b
 *       (tau < 0 selects the default).
 * Any output may be NULL. Asynchronous on `stream`. */
UNIFY_API int unify_route(unify_index_t* idx, const int64_t* lo, const int64_t* hi, int64_t nq, int64_t tau_a,
                int64_t tau_b, int32_t* out_pa, int32_t* out_pb, uint32_t* out_mask,
                int32_t* out_strategy, void* stream);

/* Searches nq queries with one strategy (UNIFY_AUTO routes per query).
 *   q          nq x d float32, row-major, device
 *   lo, hi     nq int64, device, inclusive ranges
 *   k          results per query, 1 <= k <= 256
 *   ef         overrides p->ef (and ef_post when p->ef_post <= 0); ef >= 1
 *   p          parameters, NULL = defaults
 *   out_ids    nq x k int64, device;  out_dist nq x k float32 (squared L2), device
 *   out_count  nq int32, device: number of valid results in the row
 *   out_status nq uint32 bit set of UNIFY_Q_*, device, may be NULL
 *   out_counters nq x 4 int32, device, may be NULL: distance evaluations (rows scanned
 *              for Strategy A), expansions, and the start and end of the query's work
 *              in microseconds since the search kernel's first work unit started
 * The first call with a larger nq grows the index's scratch buffers (a device
 * allocation), and so does the first call that takes the tensor-core scan (its
 * buffers, about 16 KB per query of capacity, exist only once a search uses it);
 * make those calls before capturing the stream into a CUDA graph. */
UNIFY_API int unify_search(unify_index_t* idx, const float* q, const int64_t* lo, const int64_t* hi, int64_t nq,
                 int k, int ef, unify_strategy_t strategy, const unify_params_t* p, int64_t* out_ids,
                 float* out_dist, int32_t* out_count, uint32_t* out_status, int32_t* out_counters,
                 void* stream);

/* unify_search with a conjunctive predicate on a second attribute (Section 5.9: one
 * single-attribute index per attribute; the index is built on its own attribute A1,
 * and Algorithm 7's push-to-ann test requires both ranges). Query i returns the
 * nearest objects with lo[i] <= A1 <= hi[i] AND lo2[i] <= attr2[id] <= hi2[i]:
 * Strategy A scans the A1 range and keeps the rows that pass A2; Strategy C's
 * layer-0 ann test and entry point test both ranges; Strategy B's final filter tests
 * both. Segments, masks and the router use A1 alone.
 *   attr2      n int64, device: the second attribute of every object, by id; read
 *              during the call (caller-owned, must stay valid until the stream reaches
 *              the end of the search)
 *   lo2, hi2   nq int64, device, inclusive ranges on attr2 (lo2 > hi2 selects nothing)
 * Other arguments and results as unify_search. Returns UNIFY_E_ARG when attr2, lo2 or
 * hi2 is NULL (nq > 0). The tensor-core scan (tc_scan) is not used by this call. */
UNIFY_API int unify_search_conj(unify_index_t* idx, const float* q, const int64_t* lo, const int64_t* hi,
                                const int64_t* attr2, const int64_t* lo2, const int64_t* hi2, int64_t nq, int k,
                                int ef, unify_strategy_t strategy, const unify_params_t* p, int64_t* out_ids,
                                float* out_dist, int32_t* out_count, uint32_t* out_status, int32_t* out_counters,
                                void* stream);

/* unify_search with strategy UNIFY_AUTO (range-aware selection). */
UNIFY_API int unify_search_auto(unify_index_t* idx, const float* q, const int64_t* lo, const int64_t* hi,
                      int64_t nq, int k, int ef, const unify_params_t* p, int64_t* out_ids,
                      float* out_dist, int32_t* out_count, uint32_t* out_status, void* stream);

/* unify_search_auto on HOST buffers (pinned memory is fastest): the inputs are
 * copied to index-owned device staging buffers on `stream`, searched, and the
 * results copied back; returns after the stream has finished that work. */
UNIFY_API int unify_search_auto_host(unify_index_t* idx, const float* q, const int64_t* lo, const int64_t* hi,
                           int64_t nq, int k, int ef, const unify_params_t* p, int64_t* out_ids,
                           float* out_dist, int32_t* out_count, uint32_t* out_status, void* stream);

/* Captures one search of fixed buffers into a CUDA graph: the work-counter reset,
 * the route kernel and the persistent search kernel. Arguments are those of
 * unify_search (device buffers, out_counters not recorded). The call first runs
 * one ordinary search on a private stream (it sizes the scratch and writes the
 * outputs), then captures a second one. Synchronous. Later unify_plan_launch calls
 * replay the search on whatever the buffers hold at launch time (update q, lo, hi
 * in place between launches). While a plan lives, the index refuses searches that
 * would need more scratch (UNIFY_E_LIMIT); plans and searches on one index share
 * its scratch, so they must not run concurrently. */
UNIFY_API int unify_plan_create(unify_index_t* idx, const float* q, const int64_t* lo, const int64_t* hi,
                                int64_t nq, int k, int ef, unify_strategy_t strategy, const unify_params_t* p,
                                int64_t* out_ids, float* out_dist, int32_t* out_count, uint32_t* out_status,
                                unify_plan_t** out);

/* Launches a captured search on `stream` (one cudaGraphLaunch). Asynchronous. */
UNIFY_API int unify_plan_launch(unify_plan_t* plan, void* stream);

/* Releases the graph; the plan's index must still be alive. NULL is ignored. */
UNIFY_API void unify_plan_destroy(unify_plan_t* plan);

/* unify_search without any device allocation. The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc while searching
 * (a fixed device-memory budget, a latency-critical loop that cannot take
 * cudaMalloc's implicit device-wide synchronisation or its failure, a host that
 * must not allocate once running). Arguments are those of unify_search minus
 * out_counters; inputs and outputs are still the caller's device buffers.
 * Scratch comes from one fixed device array of about 8.6 MiB compiled into the
 * library, present on every GPU that loads it until the process exits. Limits:
 * nq <= 1024 and k <= 16 per call; larger sizes return UNIFY_E_LIMIT without
 * running. The first call on a device looks up the array's device address (keep
 * that first call outside any stream capture). All calls share the array and it
 * keeps the last call's contents; each call clears its work counters on `stream`
 * first. Calls whose GPU work overlaps (different streams or threads, or another
 * index on the same device) race on the array and must be serialised. */
UNIFY_API int unify_search_noalloc(unify_index_t* idx, const float* q, const int64_t* lo, const int64_t* hi,
                                   int64_t nq, int k, int ef, unify_strategy_t strategy,
                                   const unify_params_t* p, int64_t* out_ids, float* out_dist,
                                   int32_t* out_count, uint32_t* out_status, void* stream);

/* Per-phase timing of searches with CUDA events recorded on the search stream.
 * While enabled, every search records one event pair around each phase it runs:
 * 0 = route (range bounds, masks, work queues), 1 = the search kernel (hybrid,
 * post-filter and pre-filter work of the batch), 2 = the tensor-core pre-filter scan
 * (when used); 3 is reserved (zero). */
UNIFY_API int unify_timing_enable(unify_index_t* idx, int enable);

/* Waits for the recorded events, writes per phase the summed milliseconds
 * (total_ms[4]) and the number of recorded spans (spans[4]), and clears the
 * records. Either output may be NULL. */
UNIFY_API int unify_timing_collect(unify_index_t* idx, double* total_ms, int64_t* spans);

/* Message of the last failed call on this thread ("" when none). */
UNIFY_API const char* unify_last_error(void);

/* ---- GPU-assisted construction ---------------------------------------------
 * The host builder inserts nodes in id order in batches (HSIGInsert, Algorithm 6;
 * BackboneConnectionsBuild, Algorithm 4). Every node of a batch searches the graph as
 * it stood at the start of the batch. For each segment j it:
 *   - descends the upper layers with ANNSearch (Algorithm 1, ef 1) over the chunks j;
 *   - on its own layers runs ANNSearch with efCons over the chunks j;
 *   - prunes the result to M forward edges with the heuristic of Section 2.2.
 * Then the batch's forward lists are stored, and every forward edge (v -> o) adds the
 * reverse edge (o -> v) to chunk (o's row, seg(v)), re-pruned to M on overflow
 * (Algorithm 4). Reverse edges into one chunk are applied in source-id order.
 *
 * Three callbacks let the GPU take these steps over (context from
 * unify_build_assist_create):
 *   - propose: the searches and pruning of one batch;
 *   - apply: storing the batch's forward lists and applying its reverse edges;
 *   - fetch: copying the finished graph back to the host.
 * With propose alone, the host applies edges itself and lists the chunks it changed in
 * view->dirty. With apply as well, the graph lives on the device from the first
 * proposal on: the host applies nothing, and fetch returns the graph before the host's
 * final passes (skip list, Algorithm 5).
 *
 * The view describes the builder's state at the start of the batch (host memory,
 * read-only during the call). Once the device holds the graph, adj, adjd and cnt
 * are stale. */
typedef struct {
  int64_t n;
  int d, S, M, efc;
  const float* X;            /* n x d float32 vectors, row-major */
  const int32_t* level;      /* n node levels */
  const int64_t* row0;       /* n: first row of each node; its rows are row0[v] + l, l <= level[v] */
  int64_t nrows;
  const int32_t* adj;        /* nrows x S x M neighbour ids, -1 after the chunk's count */
  const float* adjd;         /* nrows x S x M distances to the chunk's owner, 0 after the count */
  const uint8_t* cnt;        /* nrows x S chunk counts */
  const int32_t* entry_seg;  /* S entry nodes (-1: segment still empty) */
  const int32_t* top_seg;    /* S levels of the entry nodes */
  const int64_t* dirty;      /* chunk indices (row * S + j) changed since the previous call */
  int64_t ndirty;
  int64_t first, count;      /* the batch: nodes [first, first + count) */
} unify_build_view_t;

/* Proposal callback: for every node v of the batch, every layer l <= level[v] and
 * every segment j, the pruned forward list of chunk (row0[v] + l, j), written at row
 * row0[v] + l - row0[first]: out_ids / out_dist (rows x S x M, ids and distances to v,
 * ascending by (distance, id)) and out_cnt (rows x S). Returns 0 on success. */
typedef int (*unify_propose_fn)(void* ctx, const unify_build_view_t* view, int32_t* out_ids, float* out_dist,
                                uint8_t* out_cnt);

/* Apply callback, called after propose for the same batch: stores the batch's forward
 * lists (the proposals, non-empty chunks only) and applies the reverse edges. Group g
 * targets chunk group_chunk[g] (row * S + j) and holds edges group_start[g] ..
 * group_start[g + 1] - 1 in source-id order: source rev_v[e] at distance rev_dist[e].
 * Group targets are distinct and belong to nodes inserted before the batch. */
typedef int (*unify_apply_fn)(void* ctx, const unify_build_view_t* view, const int64_t* group_chunk,
                              const int64_t* group_start, int64_t ngroups, const int32_t* rev_v,
                              const float* rev_dist);

/* Fetch callback: writes the whole graph (nrows x S x M ids and distances, nrows x S
 * counts) into host arrays laid out as in the view. */
typedef int (*unify_fetch_fn)(void* ctx, const unify_build_view_t* view, int32_t* adj, float* adjd, uint8_t* cnt);

/* Creates the device state of one GPU-assisted build on `device`; *ctx owns a device
 * mirror of the vectors and the graph until unify_build_assist_destroy (null is a
 * no-op). Errors: UNIFY_E_ARG (null ctx, no such device), UNIFY_E_NOMEM, UNIFY_E_CUDA.
 * The paper builds on the CPU; this is the GPU path of the same batched insertion. */
UNIFY_API int unify_build_assist_create(int device, void** ctx);
UNIFY_API void unify_build_assist_destroy(void* ctx);

/* The unify_propose_fn of the GPU. The first call uploads the vectors and the whole
 * graph; later calls upload only the chunks listed in view->dirty. One warp per
 * (batch node, segment) runs the descent, ANNSearch with the single sorted candidate
 * buffer of the search kernel, and the pruning heuristic.
 * Limits: M <= 32, efc <= 256, d <= 1024, S <= 32 (UNIFY_E_LIMIT otherwise; also
 * when a search exceeds 2^20 expansions). Other errors: UNIFY_E_ARG (null pointers, a
 * batch outside [0, n), a dirty chunk outside nrows x S, a view whose n, nrows, d, S
 * or M differ from the first call's), UNIFY_E_NOMEM, UNIFY_E_CUDA. Distances are
 * float32; on vectors whose squared distances are integers below 2^24 they are exact,
 * and the proposals equal the host builder's. Synchronous: the outputs are complete
 * when it returns. */
UNIFY_API int unify_build_propose(void* ctx, const unify_build_view_t* view, int32_t* out_ids, float* out_dist,
                                  uint8_t* out_cnt);

/* The unify_apply_fn of the GPU: forward lists from the device copy of the last
 * proposals, then one warp per group applying its reverse edges in order (skip an
 * edge already present; insert in (distance, id) order; on overflow re-prune the M + 1
 * candidates with the heuristic of Section 2.2, float32 distances between them).
 * Errors: UNIFY_E_ARG (no preceding propose for view->first, a group chunk outside
 * nrows x S, group_start not ascending or not starting at 0, a source outside
 * [0, n)), UNIFY_E_NOMEM, UNIFY_E_CUDA. Synchronous. */
UNIFY_API int unify_build_apply(void* ctx, const unify_build_view_t* view, const int64_t* group_chunk,
                                const int64_t* group_start, int64_t ngroups, const int32_t* rev_v,
                                const float* rev_dist);

/* The unify_fetch_fn of the GPU. UNIFY_E_ARG before the first propose. Synchronous. */
UNIFY_API int unify_build_fetch(void* ctx, const unify_build_view_t* view, int32_t* adj, float* adjd, uint8_t* cnt);

#ifdef __cplusplus
}
#endif

#endif /* UNIFY_H */
