/*
 * CPU oracle for range-filtered k-NN search over an HSIG.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library. The CUDA search never calls it.
 * It shares no code with the CUDA path (its own index reader, heaps, distance).
 *
 * Paper: "UNIFY: Unified Index for Range Filtered Approximate Nearest Neighbors
 * Search". Two parts:
 *   O1  exact range-filtered k-NN, Definition 1 (Section 2.1), distances in FP64;
 *   O2  a literal HSIG search: range resolution through the skip list, segment
 *       mask, range-aware strategy selection (Section 4.2), Strategy A
 *       (pre-filter), Strategy B (post-filter: Algorithm 2 with Algorithm 1 over
 *       bitmap-marked edges) and Strategy C (hybrid: Algorithm 2's scheme with
 *       Algorithm 7 per layer), with binary heaps and a visited array.
 *
 * Readings of the paper used here (the CUDA path takes the same ones):
 *   R1 Distances are squared L2 (same order as Euclidean); ties are broken by id:
 *      every comparison of two objects compares (distance, id) lexicographically.
 *   R2 Segment j covers [b_j, b_{j+1}) with b_0 = -inf, b_S = +inf; it intersects
 *      the inclusive range [lo, hi] when it holds objects, b_j <= hi and lo < b_{j+1}.
 *   R3 Y = number of objects with lo <= a <= hi; Strategy A when Y <= tau_A,
 *      B when Y >= tau_B, otherwise C (A is tested first).
 *   R4 Algorithm 7: the entry point is pushed to cand and marked visited; it enters
 *      ann only when it passes the ann test. While |ann| < k there is no break and
 *      every unvisited selected neighbour enters cand. ann holds at most k.
 *   R5 Hybrid upper layers (L..1) run Algorithm 7 with k = 1, where the ann test is
 *      "the object lies in an intersected segment"; layer 0 runs it with k = ef and
 *      the test lo <= a <= hi. Start: the global entry point (highest level).
 *      If ann stays empty on a layer, the entry point is kept.
 *   R6 Selection S2 (default): the first ceil(m / S') slots of every intersected
 *      chunk, S' = number of intersected segments, chunks visited in ascending
 *      segment id. Selection S1 (Section 4.2, first strategy; Section 5.6): every
 *      neighbour in the intersected chunks, ordered by (distance to the expanded
 *      object, id) with distances in FP64, and the first m of them. Only distances
 *      to the query count as distance evaluations.
 *   R7 Post-filter: Algorithm 1 over bitmap-marked slots (k = 1 on upper layers,
 *      k = ef_post on layer 0), then the range filter, then the first k.
 *   R8 A result holds min(k, found) entries sorted by (distance, id); the rest of
 *      the row is padded with id -1 and distance +inf.
 *   R9 Conjunctive predicate on a second attribute (Section 5.9, one
 *      single-attribute index per attribute): the index is built on A1; a query adds
 *      lo2 <= A2 <= hi2. Algorithm 7's layer-0 ann test requires both ranges (the
 *      paper's change of its push to ann); by the same reading Strategy A
 *      keeps only rows that satisfy both (rows failing A2 are skipped before any
 *      distance) and Strategy B's final filter tests both. Segments, masks and the
 *      router use A1 alone.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EARG -1
#define ORC_EIO -2
#define ORC_EFORMAT -3
#define ORC_ENOMEM -4

#define STRAT_A 0
#define STRAT_C 1
#define STRAT_B 2

/* ------------------------------------------------------------------ index */

typedef struct {
  int64_t n, n_upper;
  int d, S, M, W, max_level, entry_global;
  float* vectors;
  int64_t* attr;
  int32_t* level;
  int32_t* upper_base;
  int64_t* seg_bounds;
  int64_t* seg_count;
  int32_t* entry_seg;
  int32_t* sorted_ids;
  int32_t* skip_next0;
  int32_t* skip_head;
  int32_t* skip_nextU;
  int32_t* adj0;
  uint32_t* gmask0;
  int32_t* adjU;
  uint32_t* gmaskU;
  unsigned char* blob;
  int64_t blob_size;
} orc_index;

static uint64_t fnv1a_words(const unsigned char* p, uint64_t nbytes) {
  uint64_t h = 0xcbf29ce484222325ull, i = 0, w;
  for (; i + 8 <= nbytes; i += 8) {
    memcpy(&w, p + i, 8);
    h = (h ^ w) * 0x100000001b3ull;
  }
  if (i < nbytes) {
    w = 0;
    memcpy(&w, p + i, nbytes - i);
    h = (h ^ w) * 0x100000001b3ull;
  }
  return h;
}

static void* find_section(orc_index* ix, uint32_t nsec, const char* name, uint32_t want_dtype,
                          uint64_t want_elems, int* err) {
  static const uint64_t esize[7] = {0, 1, 1, 4, 4, 8, 4};
  for (uint32_t s = 0; s < nsec; ++s) {
    const unsigned char* e = ix->blob + 16 + 96 * (uint64_t)s;
    char nm[25];
    memcpy(nm, e, 24);
    nm[24] = 0;
    if (strcmp(nm, name) != 0) continue;
    uint32_t dtype, ndim;
    uint64_t shape[4], off, nbytes, ck, elems = 1;
    memcpy(&dtype, e + 24, 4);
    memcpy(&ndim, e + 28, 4);
    memcpy(shape, e + 32, 32);
    memcpy(&off, e + 64, 8);
    memcpy(&nbytes, e + 72, 8);
    memcpy(&ck, e + 80, 8);
    if (dtype != want_dtype || ndim < 1 || ndim > 4) { *err = 1; return NULL; }
    for (uint32_t k = 0; k < ndim; ++k) elems *= shape[k];
    if (elems * esize[dtype] != nbytes || (want_elems && elems != want_elems)) { *err = 1; return NULL; }
    if (off + nbytes > (uint64_t)ix->blob_size || (off & 63)) { *err = 1; return NULL; }
    if (fnv1a_words(ix->blob + off, nbytes) != ck) { *err = 2; return NULL; }
    return ix->blob + off;
  }
  *err = 1;
  return NULL;
}

int orc_index_open(const char* path, orc_index** out) {
  if (!path || !out) return ORC_EARG;
  *out = NULL;
  FILE* f = fopen(path, "rb");
  if (!f) return ORC_EIO;
  if (fseek(f, 0, SEEK_END) != 0) { fclose(f); return ORC_EIO; }
  long sz = ftell(f);
  if (sz < 16) { fclose(f); return ORC_EFORMAT; }
  rewind(f);
  orc_index* ix = (orc_index*)calloc(1, sizeof(orc_index));
  if (!ix) { fclose(f); return ORC_ENOMEM; }
  ix->blob = (unsigned char*)malloc((size_t)sz);
  ix->blob_size = sz;
  if (!ix->blob) { fclose(f); free(ix); return ORC_ENOMEM; }
  if (fread(ix->blob, 1, (size_t)sz, f) != (size_t)sz) { fclose(f); free(ix->blob); free(ix); return ORC_EIO; }
  fclose(f);
  uint32_t version, nsec;
  memcpy(&version, ix->blob + 8, 4);
  memcpy(&nsec, ix->blob + 12, 4);
  if (memcmp(ix->blob, "UNIFYHSG", 8) != 0 || version != 1 || 16 + 96ull * nsec > (uint64_t)sz) {
    free(ix->blob); free(ix); return ORC_EFORMAT;
  }
  int err = 0;
  int64_t* meta = (int64_t*)find_section(ix, nsec, "meta", 5, 16, &err);
  if (!meta) { free(ix->blob); free(ix); return ORC_EFORMAT; }
  ix->n = meta[0]; ix->d = (int)meta[1]; ix->S = (int)meta[2]; ix->M = (int)meta[3];
  ix->max_level = (int)meta[4]; ix->entry_global = (int)meta[5]; ix->n_upper = meta[6]; ix->W = (int)meta[9];
  if (ix->n < 1 || ix->d < 1 || ix->S < 1 || ix->S > 32 || ix->M < 1 || ix->W != (ix->S * ix->M + 31) / 32) {
    free(ix->blob); free(ix); return ORC_EFORMAT;
  }
  uint64_t n = (uint64_t)ix->n, nu = ix->n_upper > 0 ? (uint64_t)ix->n_upper : 1, SM = (uint64_t)ix->S * ix->M;
  ix->vectors = (float*)find_section(ix, nsec, "vectors", 6, n * ix->d, &err);
  ix->attr = (int64_t*)find_section(ix, nsec, "attr", 5, n, &err);
  ix->level = (int32_t*)find_section(ix, nsec, "level", 3, n, &err);
  ix->upper_base = (int32_t*)find_section(ix, nsec, "upper_base", 3, n, &err);
  ix->seg_bounds = (int64_t*)find_section(ix, nsec, "seg_bounds", 5, ix->S + 1, &err);
  ix->seg_count = (int64_t*)find_section(ix, nsec, "seg_count", 5, ix->S, &err);
  ix->entry_seg = (int32_t*)find_section(ix, nsec, "entry_seg", 3, ix->S, &err);
  ix->sorted_ids = (int32_t*)find_section(ix, nsec, "sorted_ids", 3, n, &err);
  ix->skip_next0 = (int32_t*)find_section(ix, nsec, "skip_next0", 3, n, &err);
  ix->skip_head = (int32_t*)find_section(ix, nsec, "skip_head", 3, ix->max_level + 1, &err);
  ix->skip_nextU = (int32_t*)find_section(ix, nsec, "skip_nextU", 3, nu, &err);
  ix->adj0 = (int32_t*)find_section(ix, nsec, "adj0", 3, n * SM, &err);
  ix->gmask0 = (uint32_t*)find_section(ix, nsec, "gmask0", 4, n * ix->W, &err);
  ix->adjU = (int32_t*)find_section(ix, nsec, "adjU", 3, nu * SM, &err);
  ix->gmaskU = (uint32_t*)find_section(ix, nsec, "gmaskU", 4, nu * ix->W, &err);
  if (err) { free(ix->blob); free(ix); return ORC_EFORMAT; }
  *out = ix;
  return ORC_OK;
}

void orc_index_close(orc_index* ix) {
  if (!ix) return;
  free(ix->blob);
  free(ix);
}

int64_t orc_index_n(const orc_index* ix) { return ix->n; }
int orc_index_d(const orc_index* ix) { return ix->d; }
int orc_index_max_level(const orc_index* ix) { return ix->max_level; }

/* ------------------------------------------------------- distances, keys */

/* Gamma(q, x) = sum_t (q_t - x_t)^2 in FP64, x and q widened from float32. */
static double gamma64(const float* q, const float* x, int d) {
  double s = 0.0;
  for (int t = 0; t < d; ++t) {
    double df = (double)q[t] - (double)x[t];
    s += df * df;
  }
  return s;
}

typedef struct { double d; int64_t id; } key_t_;

static int key_less(key_t_ a, key_t_ b) { return a.d < b.d || (a.d == b.d && a.id < b.id); }

static int key_cmp(const void* pa, const void* pb) {
  key_t_ a = *(const key_t_*)pa, b = *(const key_t_*)pb;
  return key_less(a, b) ? -1 : (key_less(b, a) ? 1 : 0);
}

/* Binary heap of keys. max_heap = 1: the top is the largest (ann);
 * max_heap = 0: the top is the smallest (cand). */
typedef struct { key_t_* a; int64_t n, cap; int max_heap; } heap_t;

static int heap_before(const heap_t* h, key_t_ x, key_t_ y) {
  return h->max_heap ? key_less(y, x) : key_less(x, y);
}

static int heap_push(heap_t* h, key_t_ x) {
  if (h->n == h->cap) {
    int64_t nc = h->cap ? 2 * h->cap : 64;
    key_t_* na = (key_t_*)realloc(h->a, (size_t)nc * sizeof(key_t_));
    if (!na) return -1;
    h->a = na;
    h->cap = nc;
  }
  int64_t i = h->n++;
  h->a[i] = x;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (!heap_before(h, h->a[i], h->a[p])) break;
    key_t_ t = h->a[i]; h->a[i] = h->a[p]; h->a[p] = t;
    i = p;
  }
  return 0;
}

static key_t_ heap_pop(heap_t* h) {
  key_t_ top = h->a[0];
  h->a[0] = h->a[--h->n];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, b = i;
    if (l < h->n && heap_before(h, h->a[l], h->a[b])) b = l;
    if (r < h->n && heap_before(h, h->a[r], h->a[b])) b = r;
    if (b == i) break;
    key_t_ t = h->a[i]; h->a[i] = h->a[b]; h->a[b] = t;
    i = b;
  }
  return top;
}

/* ------------------------------------------------------------------- O1 */

/* Definition 1: R = {i : lo <= a_i <= hi}; rank R by (Gamma(q, x_i), i) in FP64;
 * return the first min(k, |R|). Returns the number written; the rest of the row is
 * padded (R8). */
/* O1 with the R9 predicate: objects with lo <= A <= hi and (A2 NULL or
 * lo2 <= A2 <= hi2). */
static int64_t exact_knn2(const float* X, const int64_t* A, const int64_t* A2, int64_t n, int d, const float* q,
                          int64_t lo, int64_t hi, int64_t lo2, int64_t hi2, int k, int64_t* out_ids,
                          double* out_dist) {
#define IN_R(i) (lo <= A[i] && A[i] <= hi && (!A2 || (lo2 <= A2[i] && A2[i] <= hi2)))
  int64_t r = 0;
  for (int64_t i = 0; i < n; ++i)
    if (IN_R(i)) ++r;
  key_t_* all = (key_t_*)malloc((size_t)(r > 0 ? r : 1) * sizeof(key_t_));
  if (!all) return -1;
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i)
    if (IN_R(i)) {
      all[m].d = gamma64(q, X + i * (int64_t)d, d);
      all[m].id = i;
      ++m;
    }
  qsort(all, (size_t)m, sizeof(key_t_), key_cmp);
  int64_t c = m < k ? m : k;
  for (int64_t t = 0; t < k; ++t) {
    out_ids[t] = t < c ? all[t].id : -1;
    out_dist[t] = t < c ? all[t].d : INFINITY;
  }
  free(all);
  return c;
#undef IN_R
}

int64_t orc_exact_knn(const float* X, const int64_t* A, int64_t n, int d, const float* q,
                      int64_t lo, int64_t hi, int k, int64_t* out_ids, double* out_dist) {
  return exact_knn2(X, A, NULL, n, d, q, lo, hi, 0, 0, k, out_ids, out_dist);
}

/* ------------------------------------------------------------ O2 pieces */

static const int32_t* row_adj(const orc_index* ix, int32_t v, int l) {
  uint64_t SM = (uint64_t)ix->S * ix->M;
  if (l == 0) return ix->adj0 + (uint64_t)v * SM;
  return ix->adjU + ((uint64_t)ix->upper_base[v] + (uint64_t)(l - 1)) * SM;
}

static const uint32_t* row_gmask(const orc_index* ix, int32_t v, int l) {
  if (l == 0) return ix->gmask0 + (uint64_t)v * ix->W;
  return ix->gmaskU + ((uint64_t)ix->upper_base[v] + (uint64_t)(l - 1)) * ix->W;
}

static int32_t skip_next(const orc_index* ix, int32_t v, int l) {
  if (l == 0) return ix->skip_next0[v];
  return ix->skip_nextU[(uint64_t)ix->upper_base[v] + (uint64_t)(l - 1)];
}

/* Segment of attribute value a: the j with b_j <= a < b_{j+1} (R2). */
static int segment_of(const orc_index* ix, int64_t a) {
  int j = 0;
  for (int t = 1; t < ix->S; ++t)
    if (ix->seg_bounds[t] <= a) j = t;
  return j;
}

/* R2: bit j set when segment j holds objects and [b_j, b_{j+1}) meets [lo, hi]. */
uint32_t orc_segment_mask(const orc_index* ix, int64_t lo, int64_t hi) {
  uint32_t mask = 0;
  if (lo > hi) return 0;
  for (int j = 0; j < ix->S; ++j) {
    int lower_ok = (j == 0) || ix->seg_bounds[j] <= hi;
    int upper_ok = (j == ix->S - 1) || lo < ix->seg_bounds[j + 1];
    if (ix->seg_count[j] > 0 && lower_ok && upper_ok) mask |= 1u << j;
  }
  return mask;
}

/* Skip-list descent (Strategy A, Section 4.2): the first object, in attribute order,
 * with attribute >= lo; -1 when there is none. */
int32_t orc_skiplist_first(const orc_index* ix, int64_t lo) {
  int32_t cur = -1;
  for (int l = ix->max_level; l >= 0; --l) {
    int32_t nxt = cur < 0 ? ix->skip_head[l] : skip_next(ix, cur, l);
    while (nxt >= 0 && ix->attr[nxt] < lo) {
      cur = nxt;
      nxt = skip_next(ix, cur, l);
    }
  }
  return cur < 0 ? ix->skip_head[0] : ix->skip_next0[cur];
}

/* Candidate range bounds by their definition: pa = #{a < lo}, pb = #{a <= hi}. */
void orc_range_bounds(const orc_index* ix, int64_t lo, int64_t hi, int64_t* pa, int64_t* pb) {
  int64_t a = 0, b = 0;
  for (int64_t i = 0; i < ix->n; ++i) {
    if (ix->attr[i] < lo) ++a;
    if (ix->attr[i] <= hi) ++b;
  }
  *pa = a;
  *pb = b < a ? a : b;
}

int orc_route(int64_t Y, int64_t tau_a, int64_t tau_b) {
  if (Y <= tau_a) return STRAT_A;
  if (Y >= tau_b) return STRAT_B;
  return STRAT_C;
}

typedef struct {
  heap_t cand, ann;
  unsigned char* visited;
  void* sel;  /* S1 selection buffer, S * M keys */
  const int64_t* a2;  /* second attribute by id, or NULL (R9) */
  int64_t lo2, hi2;
  int64_t n_dist, n_exp;
  int32_t* trace;  /* NULL, or max_level + 1 slots: the entry point each layer starts from */
} scratch_t;

static int sc_init(scratch_t* s, int64_t n) {
  memset(s, 0, sizeof(*s));
  s->ann.max_heap = 1;
  s->visited = (unsigned char*)malloc((size_t)n);
  return s->visited ? 0 : -1;
}

static void sc_free(scratch_t* s) {
  free(s->sel);
  free(s->cand.a);
  free(s->ann.a);
  free(s->visited);
}

/* Strategy A: descend the skip list to the first in-range object, then a linear
 * scan along the layer-0 chain while the attribute is <= hi, keeping the k best. */
/* The second-attribute predicate of R9 (true without a second attribute). */
static int pred2(const scratch_t* s, int64_t v) {
  return !s->a2 || (s->lo2 <= s->a2[v] && s->a2[v] <= s->hi2);
}

static int64_t strategy_pre(const orc_index* ix, const float* q, int64_t lo, int64_t hi, int k,
                            scratch_t* s, key_t_* out) {
  heap_t* ann = &s->ann;
  ann->n = 0;
  if (lo > hi) return 0;
  int32_t v = orc_skiplist_first(ix, lo);
  while (v >= 0 && ix->attr[v] <= hi) {
    if (!pred2(s, v)) {
      v = ix->skip_next0[v];
      continue;
    }
    key_t_ kv = {gamma64(q, ix->vectors + (int64_t)v * ix->d, ix->d), v};
    s->n_dist++;
    if (ann->n < k) {
      if (heap_push(ann, kv)) return -1;
    } else if (key_less(kv, ann->a[0])) {
      heap_pop(ann);
      if (heap_push(ann, kv)) return -1;
    }
    v = ix->skip_next0[v];
  }
  int64_t c = ann->n;
  for (int64_t t = c - 1; t >= 0; --t) out[t] = heap_pop(ann);
  return c;
}

/* Algorithm 1 (ANNSearch) on layer l over bitmap-marked slots (Strategy B). On
 * return s->ann holds the result (a max-heap of at most k keys). */
static int alg1_global(const orc_index* ix, const float* q, int32_t ep, int l, int k, scratch_t* s) {
  heap_t *cand = &s->cand, *ann = &s->ann;
  cand->n = 0;
  ann->n = 0;
  memset(s->visited, 0, (size_t)ix->n);
  key_t_ e = {gamma64(q, ix->vectors + (int64_t)ep * ix->d, ix->d), ep};
  s->n_dist++;
  if (heap_push(cand, e) || heap_push(ann, e)) return -1;
  s->visited[ep] = 1;
  while (cand->n > 0) {
    key_t_ o = heap_pop(cand);
    key_t_ u = ann->a[0];
    if (key_less(u, o)) break;
    s->n_exp++;
    const int32_t* adj = row_adj(ix, (int32_t)o.id, l);
    const uint32_t* gm = row_gmask(ix, (int32_t)o.id, l);
    for (int p = 0; p < ix->S * ix->M; ++p) {
      if (!((gm[p >> 5] >> (p & 31)) & 1u)) continue;
      int32_t v = adj[p];
      if (v < 0 || s->visited[v]) continue;
      s->visited[v] = 1;
      key_t_ kv = {gamma64(q, ix->vectors + (int64_t)v * ix->d, ix->d), v};
      s->n_dist++;
      u = ann->a[0];
      if (key_less(kv, u) || ann->n < k) {
        if (heap_push(cand, kv) || heap_push(ann, kv)) return -1;
        if (ann->n > k) heap_pop(ann);
      }
    }
  }
  return 0;
}

/* Algorithm 7 (HybridFilteringLayer) on layer l with the selection of R6. The ann
 * test is lo <= a <= hi on layer 0 and "in an intersected segment" above (R5). */
/* Selection S1 (R6): the neighbours of o in the intersected chunks, by (FP64
 * distance to o, id); the first m go to sel[0, return value). */
static int select_s1(const orc_index* ix, const int32_t* adj, int32_t o, int m, uint32_t mask, key_t_* sel) {
  int n = 0;
  const float* xo = ix->vectors + (int64_t)o * ix->d;
  for (int i = 0; i < ix->S; ++i) {
    if (!((mask >> i) & 1u)) continue;
    const int32_t* chunk = adj + (int64_t)i * ix->M;
    for (int t = 0; t < ix->M; ++t) {
      int32_t v = chunk[t];
      if (v < 0) break;
      key_t_ kv = {gamma64(xo, ix->vectors + (int64_t)v * ix->d, ix->d), v};
      sel[n++] = kv;
    }
  }
  qsort(sel, (size_t)n, sizeof(key_t_), key_cmp);
  return n < m ? n : m;
}

static int alg7(const orc_index* ix, const float* q, int32_t ep, int l, int k, int m, uint32_t mask,
                int64_t lo, int64_t hi, int selection, scratch_t* s) {
  heap_t *cand = &s->cand, *ann = &s->ann;
  cand->n = 0;
  ann->n = 0;
  memset(s->visited, 0, (size_t)ix->n);
  int Sp = __builtin_popcount(mask);
  if (Sp == 0) return 0;
  int per = (m + Sp - 1) / Sp;
  if (per > ix->M) per = ix->M;
#define ANN_TEST(v) (l == 0 ? (lo <= ix->attr[v] && ix->attr[v] <= hi && pred2(s, v)) \
                            : ((mask >> segment_of(ix, ix->attr[v])) & 1u))
  key_t_ e = {gamma64(q, ix->vectors + (int64_t)ep * ix->d, ix->d), ep};
  s->n_dist++;
  if (heap_push(cand, e)) return -1;
  if (ANN_TEST(ep) && heap_push(ann, e)) return -1;
  s->visited[ep] = 1;
  while (cand->n > 0) {
    key_t_ o = heap_pop(cand);
    if (ann->n >= k && key_less(ann->a[0], o)) break;
    s->n_exp++;
    const int32_t* adj = row_adj(ix, (int32_t)o.id, l);
    /* the selected neighbours, in selection order */
    int nsel = 0;
    if (selection == 1) {
      if (!s->sel) {
        s->sel = malloc((size_t)ix->S * ix->M * sizeof(key_t_));
        if (!s->sel) return -1;
      }
      nsel = select_s1(ix, adj, (int32_t)o.id, m, mask, (key_t_*)s->sel);
    }
    for (int i = 0, t = 0, j = 0;;) {
      int32_t v;
      if (selection == 1) {
        if (j >= nsel) break;
        v = (int32_t)((key_t_*)s->sel)[j++].id;
      } else {
        while (i < ix->S && (!((mask >> i) & 1u) || t >= per || adj[(int64_t)i * ix->M + t] < 0)) {
          ++i;
          t = 0;
        }
        if (i >= ix->S) break;
        v = adj[(int64_t)i * ix->M + t];
        ++t;
      }
      if (s->visited[v]) continue;
      s->visited[v] = 1;
      key_t_ kv = {gamma64(q, ix->vectors + (int64_t)v * ix->d, ix->d), v};
      s->n_dist++;
      if (ann->n < k || key_less(kv, ann->a[0])) {
        if (heap_push(cand, kv)) return -1;
        if (ANN_TEST(v) && heap_push(ann, kv)) return -1;
        if (ann->n > k) heap_pop(ann);
      }
    }
  }
#undef ANN_TEST
  return 0;
}

/* Strategy B (R7). */
static int64_t strategy_post(const orc_index* ix, const float* q, int64_t lo, int64_t hi, int k,
                             int ef_post, scratch_t* s, key_t_* out) {
  int64_t pa, pb;
  orc_range_bounds(ix, lo, hi, &pa, &pb);
  if (pb <= pa) return 0; /* no object in range: the filter would leave nothing */
  int32_t ep = ix->entry_global;
  for (int l = ix->max_level; l >= 1; --l) {
    if (s->trace) s->trace[l] = ep;
    if (alg1_global(ix, q, ep, l, 1, s)) return -1;
    ep = (int32_t)s->ann.a[0].id;
  }
  if (s->trace) s->trace[0] = ep;
  if (alg1_global(ix, q, ep, 0, ef_post, s)) return -1;
  int64_t c = s->ann.n;
  key_t_* tmp = (key_t_*)malloc((size_t)(c > 0 ? c : 1) * sizeof(key_t_));
  if (!tmp) return -1;
  for (int64_t t = c - 1; t >= 0; --t) tmp[t] = heap_pop(&s->ann);
  int64_t w = 0;
  for (int64_t t = 0; t < c && w < k; ++t)
    if (lo <= ix->attr[tmp[t].id] && ix->attr[tmp[t].id] <= hi && pred2(s, tmp[t].id)) out[w++] = tmp[t];
  free(tmp);
  return w;
}

/* Strategy C (R5, R6). */
static int64_t strategy_hybrid(const orc_index* ix, const float* q, int64_t lo, int64_t hi, int k,
                               int ef, int m, int selection, scratch_t* s, key_t_* out) {
  uint32_t mask = orc_segment_mask(ix, lo, hi);
  if (mask == 0) return 0;
  int32_t ep = ix->entry_global;
  for (int l = ix->max_level; l >= 1; --l) {
    if (s->trace) s->trace[l] = ep;
    if (alg7(ix, q, ep, l, 1, m, mask, lo, hi, selection, s)) return -1;
    if (s->ann.n > 0) ep = (int32_t)s->ann.a[0].id;
  }
  if (s->trace) s->trace[0] = ep;
  if (alg7(ix, q, ep, 0, ef, m, mask, lo, hi, selection, s)) return -1;
  int64_t c = s->ann.n;
  key_t_* tmp = (key_t_*)malloc((size_t)(c > 0 ? c : 1) * sizeof(key_t_));
  if (!tmp) return -1;
  for (int64_t t = c - 1; t >= 0; --t) tmp[t] = heap_pop(&s->ann);
  int64_t w = c < k ? c : k;
  for (int64_t t = 0; t < w; ++t) out[t] = tmp[t];
  free(tmp);
  return w;
}

/* ------------------------------------------------------------- batches */

typedef struct {
  const orc_index* ix;
  const float* Q;
  const int64_t *lo, *hi;
  int64_t nq;
  int k, ef, m, ef_post, strategy, selection;
  int64_t tau_a, tau_b;
  const int64_t *a2, *lo2, *hi2;
  int64_t* out_ids;
  double* out_dist;
  int64_t* out_count;
  int32_t* out_strategy;
  int64_t* out_ndist;
  int64_t* out_nexp;
  int32_t* out_eps;
  int64_t next;
  int failed;
  pthread_mutex_t mu;
} batch_t;

static void* search_worker(void* arg) {
  batch_t* b = (batch_t*)arg;
  const orc_index* ix = b->ix;
  scratch_t s;
  key_t_* out = (key_t_*)malloc((size_t)b->k * sizeof(key_t_));
  if (sc_init(&s, ix->n) || !out) {
    pthread_mutex_lock(&b->mu); b->failed = 1; pthread_mutex_unlock(&b->mu);
    free(out); sc_free(&s);
    return NULL;
  }
  for (;;) {
    pthread_mutex_lock(&b->mu);
    int64_t i = b->next++;
    pthread_mutex_unlock(&b->mu);
    if (i >= b->nq) break;
    const float* q = b->Q + i * (int64_t)ix->d;
    int64_t lo = b->lo[i], hi = b->hi[i];
    int st = b->strategy;
    if (st < 0) {
      int64_t pa, pb;
      orc_range_bounds(ix, lo, hi, &pa, &pb);
      st = orc_route(pb - pa, b->tau_a, b->tau_b);
    }
    s.n_dist = 0;
    s.n_exp = 0;
    s.trace = NULL;
    if (b->out_eps) {
      s.trace = b->out_eps + i * (int64_t)(ix->max_level + 1);
      for (int l = 0; l <= ix->max_level; ++l) s.trace[l] = -1;
    }
    s.a2 = b->a2;
    if (b->a2) {
      s.lo2 = b->lo2[i];
      s.hi2 = b->hi2[i];
    }
    int64_t c;
    if (st == STRAT_A) c = strategy_pre(ix, q, lo, hi, b->k, &s, out);
    else if (st == STRAT_B) c = strategy_post(ix, q, lo, hi, b->k, b->ef_post, &s, out);
    else c = strategy_hybrid(ix, q, lo, hi, b->k, b->ef, b->m, b->selection, &s, out);
    if (c < 0) {
      pthread_mutex_lock(&b->mu); b->failed = 1; pthread_mutex_unlock(&b->mu);
      c = 0;
    }
    for (int t = 0; t < b->k; ++t) {
      b->out_ids[i * b->k + t] = t < c ? out[t].id : -1;
      b->out_dist[i * b->k + t] = t < c ? out[t].d : INFINITY;
    }
    b->out_count[i] = c;
    if (b->out_strategy) b->out_strategy[i] = st;
    if (b->out_ndist) b->out_ndist[i] = s.n_dist;
    if (b->out_nexp) b->out_nexp[i] = s.n_exp;
  }
  free(out);
  sc_free(&s);
  return NULL;
}

/* O2 over a batch of queries. strategy: 0 = A, 1 = C, 2 = B, -1 = range-aware (R3);
 * selection: 2 = S2, 1 = S1 (R6) for Strategy C. out_eps (NULL, or nq x (max_level + 1))
 * receives, for Strategies B and C, the entry point each layer l of Algorithm 2's
 * descent starts from at slot l (slot max_level is the global entry point, slot 0 the
 * layer-0 entry); -1 for layers that were not searched.
 * Queries are independent; threads only split the batch. */
int orc_search_batch_tr(const orc_index* ix, const float* Q, const int64_t* lo, const int64_t* hi,
                        int64_t nq, int k, int ef, int m, int ef_post, int strategy, int64_t tau_a,
                        int64_t tau_b, int threads, int64_t* out_ids, double* out_dist,
                        int64_t* out_count, int32_t* out_strategy, int64_t* out_ndist, int64_t* out_nexp,
                        int selection, const int64_t* attr2, const int64_t* lo2, const int64_t* hi2,
                        int32_t* out_eps) {
  if (!ix || !Q || !lo || !hi || nq < 0 || k < 1 || ef < 1 || m < 1 || ef_post < 1 || !out_ids ||
      !out_dist || !out_count || strategy < -1 || strategy > 2 || (selection != 1 && selection != 2) ||
      (attr2 && (!lo2 || !hi2)))
    return ORC_EARG;
  if (threads < 1) threads = 1;
  batch_t b;
  memset(&b, 0, sizeof(b));
  b.ix = ix; b.Q = Q; b.lo = lo; b.hi = hi; b.nq = nq; b.k = k; b.ef = ef; b.m = m;
  b.ef_post = ef_post; b.strategy = strategy; b.tau_a = tau_a; b.tau_b = tau_b; b.selection = selection;
  b.a2 = attr2; b.lo2 = lo2; b.hi2 = hi2;
  b.out_ids = out_ids; b.out_dist = out_dist; b.out_count = out_count;
  b.out_strategy = out_strategy; b.out_ndist = out_ndist; b.out_nexp = out_nexp; b.out_eps = out_eps;
  pthread_mutex_init(&b.mu, NULL);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
  if (!th) return ORC_ENOMEM;
  int started = 0;
  for (int t = 0; t < threads; ++t)
    if (pthread_create(&th[t], NULL, search_worker, &b) == 0) ++started;
  if (started == 0) search_worker(&b);
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  free(th);
  pthread_mutex_destroy(&b.mu);
  return b.failed ? ORC_ENOMEM : ORC_OK;
}

/* O2 without the descent trace. */
int orc_search_batch_ex(const orc_index* ix, const float* Q, const int64_t* lo, const int64_t* hi,
                        int64_t nq, int k, int ef, int m, int ef_post, int strategy, int64_t tau_a,
                        int64_t tau_b, int threads, int64_t* out_ids, double* out_dist,
                        int64_t* out_count, int32_t* out_strategy, int64_t* out_ndist, int64_t* out_nexp,
                        int selection, const int64_t* attr2, const int64_t* lo2, const int64_t* hi2) {
  return orc_search_batch_tr(ix, Q, lo, hi, nq, k, ef, m, ef_post, strategy, tau_a, tau_b, threads, out_ids,
                             out_dist, out_count, out_strategy, out_ndist, out_nexp, selection, attr2, lo2, hi2,
                             NULL);
}

/* O2 with one attribute and the given selection. */
int orc_search_batch_sel(const orc_index* ix, const float* Q, const int64_t* lo, const int64_t* hi,
                         int64_t nq, int k, int ef, int m, int ef_post, int strategy, int64_t tau_a,
                         int64_t tau_b, int threads, int64_t* out_ids, double* out_dist,
                         int64_t* out_count, int32_t* out_strategy, int64_t* out_ndist, int64_t* out_nexp,
                         int selection) {
  return orc_search_batch_ex(ix, Q, lo, hi, nq, k, ef, m, ef_post, strategy, tau_a, tau_b, threads, out_ids,
                             out_dist, out_count, out_strategy, out_ndist, out_nexp, selection, NULL, NULL, NULL);
}

/* O2 with selection S2. */
int orc_search_batch(const orc_index* ix, const float* Q, const int64_t* lo, const int64_t* hi,
                     int64_t nq, int k, int ef, int m, int ef_post, int strategy, int64_t tau_a,
                     int64_t tau_b, int threads, int64_t* out_ids, double* out_dist,
                     int64_t* out_count, int32_t* out_strategy, int64_t* out_ndist, int64_t* out_nexp) {
  return orc_search_batch_sel(ix, Q, lo, hi, nq, k, ef, m, ef_post, strategy, tau_a, tau_b, threads, out_ids,
                              out_dist, out_count, out_strategy, out_ndist, out_nexp, 2);
}

typedef struct {
  const float* X; const int64_t* A; int64_t n; int d;
  const float* Q; const int64_t *lo, *hi; int64_t nq; int k;
  const int64_t *A2, *lo2, *hi2;
  int64_t* out_ids; double* out_dist; int64_t* out_count;
  int64_t next; int failed; pthread_mutex_t mu;
} exact_t;

static void* exact_worker(void* arg) {
  exact_t* b = (exact_t*)arg;
  for (;;) {
    pthread_mutex_lock(&b->mu);
    int64_t i = b->next++;
    pthread_mutex_unlock(&b->mu);
    if (i >= b->nq) break;
    int64_t c = exact_knn2(b->X, b->A, b->A2, b->n, b->d, b->Q + i * (int64_t)b->d, b->lo[i], b->hi[i],
                           b->A2 ? b->lo2[i] : 0, b->A2 ? b->hi2[i] : 0, b->k, b->out_ids + i * b->k,
                           b->out_dist + i * b->k);
    if (c < 0) { pthread_mutex_lock(&b->mu); b->failed = 1; pthread_mutex_unlock(&b->mu); c = 0; }
    b->out_count[i] = c;
  }
  return NULL;
}

/* O1 over a batch of queries (threads only split the batch); A2 (with lo2, hi2)
 * adds the conjunctive predicate of R9, or is NULL. */
int orc_exact_knn_batch2(const float* X, const int64_t* A, const int64_t* A2, int64_t n, int d, const float* Q,
                         const int64_t* lo, const int64_t* hi, const int64_t* lo2, const int64_t* hi2, int64_t nq,
                         int k, int threads, int64_t* out_ids, double* out_dist, int64_t* out_count) {
  if (!X || !A || n < 0 || d < 1 || !Q || !lo || !hi || nq < 0 || k < 1 || !out_ids || !out_dist ||
      !out_count || (A2 && (!lo2 || !hi2)))
    return ORC_EARG;
  if (threads < 1) threads = 1;
  exact_t b;
  memset(&b, 0, sizeof(b));
  b.X = X; b.A = A; b.n = n; b.d = d; b.Q = Q; b.lo = lo; b.hi = hi; b.nq = nq; b.k = k;
  b.A2 = A2; b.lo2 = lo2; b.hi2 = hi2;
  b.out_ids = out_ids; b.out_dist = out_dist; b.out_count = out_count;
  pthread_mutex_init(&b.mu, NULL);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
  if (!th) return ORC_ENOMEM;
  int started = 0;
  for (int t = 0; t < threads; ++t)
    if (pthread_create(&th[t], NULL, exact_worker, &b) == 0) ++started;
  if (started == 0) exact_worker(&b);
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  free(th);
  pthread_mutex_destroy(&b.mu);
  return b.failed ? ORC_ENOMEM : ORC_OK;
}

/* O1 over a batch of queries with one attribute. */
int orc_exact_knn_batch(const float* X, const int64_t* A, int64_t n, int d, const float* Q,
                        const int64_t* lo, const int64_t* hi, int64_t nq, int k, int threads,
                        int64_t* out_ids, double* out_dist, int64_t* out_count) {
  return orc_exact_knn_batch2(X, A, NULL, n, d, Q, lo, hi, NULL, NULL, nq, k, threads, out_ids, out_dist,
                              out_count);
}

/* Routing fields per query by their definitions (R2, R3) plus the skip-list
 * descent result, for checking the CUDA router. */
int orc_route_batch(const orc_index* ix, const int64_t* lo, const int64_t* hi, int64_t nq,
                    int64_t tau_a, int64_t tau_b, int64_t* out_pa, int64_t* out_pb,
                    uint32_t* out_mask, int32_t* out_strategy, int32_t* out_first) {
  if (!ix || !lo || !hi || nq < 0) return ORC_EARG;
  for (int64_t i = 0; i < nq; ++i) {
    int64_t pa, pb;
    orc_range_bounds(ix, lo[i], hi[i], &pa, &pb);
    if (out_pa) out_pa[i] = pa;
    if (out_pb) out_pb[i] = pb;
    if (out_mask) out_mask[i] = orc_segment_mask(ix, lo[i], hi[i]);
    if (out_strategy) out_strategy[i] = orc_route(pb - pa, tau_a, tau_b);
    if (out_first) out_first[i] = orc_skiplist_first(ix, lo[i]);
  }
  return ORC_OK;
}
