// Host-side HSIG builder: produces the serialised index that the search reads.
//
// Implements the construction of Section 4.1 of "UNIFY: Unified Index for Range
// Filtered Approximate Nearest Neighbors Search":
//   * equi-depth attribute segmentation (Section 3.1),
//   * ANNSearch (Algorithm 1) restricted to one segment's sub-graph,
//   * the Prune heuristic (Section 2.2),
//   * BackboneConnectionsBuild (Algorithm 4),
//   * HSIGInsert (Algorithm 6): per-segment descent and layer-wise insertion,
//   * skip-list connections in attribute order (Section 4.1),
//   * GlobalEdgeMasking (Algorithm 5).
//
// Readings taken where the paper is silent:
//   * Segment bounds use all n attributes: b_j = sorted_attr[floor(j*n/S)] for
//     j = 1..S-1, b_0 = -inf, b_S = +inf, segments half-open [b_j, b_{j+1}).
//   * Node levels are floor(-ln(U) * mL) with mL = 1/ln(M), U in (0,1] drawn from
//     a counter-based hash of (seed, id) (the printed formula is garbled).
//   * Every chunk is kept sorted by (distance to its owner, id).
//   * Empty segments are skipped; only a node's own segment can take it as entry.
//   * Nodes are inserted in id order in batches: every node of a batch searches the
//     graph as it stood at the start of the batch, then the batch's edges are
//     applied in id order. The first 1024 nodes go one at a time. This makes the
//     result independent of the thread count.
//   * The skip list and the global-edge bitmaps are derived once all chunks are
//     final: the skip-list level-l chain links the nodes of level >= l in
//     attribute order (ties by id); Algorithm 5 runs per node in id order over the
//     final chunks, so every stored bit position names the slot it was set for.
//
// Distances are float32 squared L2 with a fixed 8-way accumulation order
// (compiled with -ffp-contract=off), so the graph is the same on every host.
//
// The proposal step of a batch (the searches and pruning of every batch node) can be
// handed to a callback (hsig_build_index_ex), e.g. the GPU's unify_build_propose. The
// callback sees the graph as it stood at the start of the batch plus the list of
// chunks changed since its previous call; batches smaller than kAssistMinBatch stay
// on the host. With an apply and a fetch callback as well, the graph moves to the
// callee at the first proposal: from then on every batch is proposed and applied
// there (the host still derives the reverse-edge groups and the entry points), and
// the graph is fetched back before the skip list and Algorithm 5.

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>
#include <queue>
#include <string>
#include <utility>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "../include/unify.h"

namespace {

using Key = std::pair<float, int32_t>;  // (distance, id), compared lexicographically

inline float l2sq(const float* a, const float* b, int d) {
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int t = 0;
  for (; t + 8 <= d; t += 8) {
    for (int u = 0; u < 8; ++u) {
      float df = a[t + u] - b[t + u];
      acc[u] += df * df;
    }
  }
  for (int u = 0; t < d; ++t, ++u) {
    float df = a[t] - b[t];
    acc[u] += df * df;
  }
  return ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
}

inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

struct Visited {
  std::vector<uint32_t> stamp;
  uint32_t cur = 0;
  void reset(size_t n) {
    if (stamp.size() != n) { stamp.assign(n, 0); cur = 0; }
    if (++cur == 0) { std::fill(stamp.begin(), stamp.end(), 0); cur = 1; }
  }
  bool test_set(int32_t v) {
    if (stamp[v] == cur) return true;
    stamp[v] = cur;
    return false;
  }
};

struct Builder {
  int64_t n = 0;
  int d = 0, S = 0, M = 0, efc = 0;
  uint64_t seed = 0;
  const float* X = nullptr;
  const int64_t* A = nullptr;

  std::vector<int64_t> bounds;     // S+1
  std::vector<int64_t> seg_count;  // S
  std::vector<int32_t> seg;        // n
  std::vector<int32_t> level;      // n
  std::vector<int64_t> row0;       // n: first row (layer 0) of node v; rows of v are row0[v] + l
  int64_t nrows = 0;
  // Per row: S chunks of M slots (ids, distances to owner), counts per chunk.
  std::vector<int32_t> adj;
  std::vector<float> adjd;
  std::vector<uint8_t> cnt;
  std::vector<int32_t> entry_seg;  // S, -1 when the segment holds no node yet
  std::vector<int32_t> top_seg;    // S, level of entry_seg
  std::vector<int32_t> order;      // attribute order (ties by id)

  // Proposal callback (null: every batch is proposed on the host); apply and fetch
  // (both null or both set) move edge application to the callee.
  unify_propose_fn propose_fn = nullptr;
  unify_apply_fn apply_fn = nullptr;
  unify_fetch_fn fetch_fn = nullptr;
  void* propose_ctx = nullptr;
  bool device_owns = false;  // the callee holds the current graph
  std::vector<int64_t> g_chunk, g_start;
  std::vector<int32_t> r_v;
  std::vector<float> r_d;
  int propose_rc = 0;
  std::vector<int64_t> dirty;        // chunks changed since the last callback
  std::vector<uint8_t> dirty_flag;   // nrows x S
  std::vector<int32_t> o_ids;
  std::vector<float> o_dist;
  std::vector<uint8_t> o_cnt;
  static constexpr int64_t kAssistMinBatch = 64;
  // Seconds spent per phase (reported on stderr when HSIG_BUILD_TIMING is set).
  double t_propose_host = 0, t_propose_cb = 0, t_apply = 0, t_finalize = 0;

  const float* vec(int64_t v) const { return X + v * (int64_t)d; }
  int64_t row(int32_t v, int l) const { return row0[v] + l; }
  int32_t* chunk(int64_t r, int j) { return adj.data() + (r * S + j) * (int64_t)M; }
  float* chunkd(int64_t r, int j) { return adjd.data() + (r * S + j) * (int64_t)M; }
  uint8_t& chunkn(int64_t r, int j) { return cnt[r * S + j]; }

  // ---- segmentation (Section 3.1) ----
  void segment() {
    order.resize(n);
    for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)i;
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      return A[a] != A[b] ? A[a] < A[b] : a < b;
    });
    bounds.assign(S + 1, 0);
    bounds[0] = std::numeric_limits<int64_t>::min();
    bounds[S] = std::numeric_limits<int64_t>::max();
    for (int j = 1; j < S; ++j) bounds[j] = A[order[(int64_t)j * n / S]];
    seg.resize(n);
    seg_count.assign(S, 0);
    for (int64_t v = 0; v < n; ++v) {
      // segment j with bounds[j] <= a < bounds[j+1]
      int j = (int)(std::upper_bound(bounds.begin() + 1, bounds.begin() + S, A[v]) - (bounds.begin() + 1));
      seg[v] = j;
      seg_count[j]++;
    }
  }

  // ---- levels (the level draw of Algorithm 6) ----
  void assign_levels() {
    level.resize(n);
    row0.resize(n);
    double mL = 1.0 / std::log((double)M);
    int64_t r = 0;
    for (int64_t v = 0; v < n; ++v) {
      uint64_t h = splitmix64(seed * 0x632BE59BD9B4E019ull + (uint64_t)v);
      double u = ((double)(h >> 11) + 1.0) * (1.0 / 9007199254740992.0);  // (0, 1]
      int lv = (int)std::floor(-std::log(u) * mL);
      if (lv > 30) lv = 30;
      level[v] = lv;
      row0[v] = r;
      r += lv + 1;
    }
    nrows = r;
    adj.assign((size_t)nrows * S * M, -1);
    adjd.assign((size_t)nrows * S * M, 0.f);
    cnt.assign((size_t)nrows * S, 0);
    entry_seg.assign(S, -1);
    top_seg.assign(S, -1);
  }

  void prefetch_vec(int32_t v) const {
    const char* p = reinterpret_cast<const char*>(vec(v));
    for (int b = 0; b < d * 4; b += 64) __builtin_prefetch(p + b);
  }

  // ---- Algorithm 1 on the sub-graph of segment j at layer l ----
  // cand_buf / ann_buf are reusable heap storage (min-heap and max-heap).
  void ann_search(const float* q, int32_t ep, int l, int j, int ef, Visited& vis,
                  std::vector<Key>& out, std::vector<Key>& cand_buf, std::vector<Key>& ann_buf) const {
    std::vector<Key>& cand = cand_buf;
    std::vector<Key>& ann = ann_buf;
    cand.clear();
    ann.clear();
    auto cand_push = [&](Key k) { cand.push_back(k); std::push_heap(cand.begin(), cand.end(), std::greater<Key>()); };
    auto ann_push = [&](Key k) { ann.push_back(k); std::push_heap(ann.begin(), ann.end()); };
    Key e{l2sq(q, vec(ep), d), ep};
    cand_push(e);
    ann_push(e);
    vis.test_set(ep);
    int32_t fresh[256];
    while (!cand.empty()) {
      std::pop_heap(cand.begin(), cand.end(), std::greater<Key>());
      Key o = cand.back();
      cand.pop_back();
      if (o > ann.front()) break;
      int64_t r = row0[o.second] + l;
      const int32_t* ch = adj.data() + (r * S + j) * (int64_t)M;
      int c = cnt[r * S + j];
      int nf = 0;
      for (int s = 0; s < c; ++s) {
        int32_t v = ch[s];
        if (vis.test_set(v)) continue;
        fresh[nf++] = v;
        prefetch_vec(v);
      }
      for (int t = 0; t < nf; ++t) {
        int32_t v = fresh[t];
        Key kv{l2sq(q, vec(v), d), v};
        if ((int)ann.size() < ef || kv < ann.front()) {
          cand_push(kv);
          ann_push(kv);
          if ((int)ann.size() > ef) {
            std::pop_heap(ann.begin(), ann.end());
            ann.pop_back();
          }
        }
      }
    }
    out.assign(ann.begin(), ann.end());
    std::sort(out.begin(), out.end());
  }

  // ---- Prune heuristic (Section 2.2) ----
  // cands: (distance to owner, id); returns at most M survivors in ascending order.
  void prune(std::vector<Key>& cands, int Mmax, std::vector<Key>& kept) const {
    std::sort(cands.begin(), cands.end());
    for (size_t t = 0; t < cands.size() && t < 64; ++t) prefetch_vec(cands[t].second);
    kept.clear();
    for (const Key& r : cands) {
      if ((int)kept.size() >= Mmax) break;
      bool drop = false;
      for (const Key& e : kept) {
        if (r.first > l2sq(vec(e.second), vec(r.second), d)) { drop = true; break; }
      }
      if (!drop) kept.push_back(r);
    }
  }

  struct Proposal {  // forward edges of one node: per layer, per segment
    std::vector<std::vector<Key>> fwd;  // index l*S + j
  };

  // Searches of Algorithm 6 for node v against the current (read-only) graph.
  void propose(int32_t v, Visited& vis, Proposal& P, std::vector<Key>& ann,
               std::vector<Key>& tmp) const {
    thread_local std::vector<Key> cand_buf, ann_buf;
    const float* q = vec(v);
    int lv = level[v];
    P.fwd.assign((size_t)(lv + 1) * S, {});
    for (int j = 0; j < S; ++j) {
      int32_t ep = entry_seg[j];
      if (ep < 0) continue;  // empty segment
      int L = top_seg[j];
      for (int l = L; l > lv; --l) {
        vis.reset(n);
        ann_search(q, ep, l, j, 1, vis, ann, cand_buf, ann_buf);
        ep = ann[0].second;
      }
      for (int l = std::min(lv, L); l >= 0; --l) {
        vis.reset(n);
        ann_search(q, ep, l, j, efc, vis, ann, cand_buf, ann_buf);
        tmp = ann;
        prune(tmp, M, P.fwd[(size_t)l * S + j]);
        ep = ann[0].second;
      }
    }
  }

  void set_chunk(int64_t r, int j, const std::vector<Key>& ks) {
    int32_t* ch = chunk(r, j);
    float* cd = chunkd(r, j);
    int c = (int)ks.size();
    for (int s = 0; s < M; ++s) {
      ch[s] = s < c ? ks[s].second : -1;
      cd[s] = s < c ? ks[s].first : 0.f;
    }
    chunkn(r, j) = (uint8_t)c;
  }

  // Algorithm 4, reverse edges: add (o -> v) to G[o][i], re-prune on overflow.
  void add_reverse(int32_t o, int l, int i, Key kv, std::vector<Key>& cands, std::vector<Key>& kept) {
    int64_t r = row(o, l);
    int c = chunkn(r, i);
    const int32_t* ch = chunk(r, i);
    const float* cd = chunkd(r, i);
    cands.clear();
    for (int s = 0; s < c; ++s) {
      if (ch[s] == kv.second) return;  // already present
      cands.push_back({cd[s], ch[s]});
    }
    cands.push_back(kv);
    if ((int)cands.size() <= M) {
      std::sort(cands.begin(), cands.end());
      set_chunk(r, i, cands);
    } else {
      prune(cands, M, kept);
      set_chunk(r, i, kept);
    }
  }

  void mark_dirty(int64_t c) {
    if (!dirty_flag[c]) {
      dirty_flag[c] = 1;
      dirty.push_back(c);
    }
  }

  unify_build_view_t view(int64_t first, int64_t count) {
    unify_build_view_t vw;
    vw.n = n;
    vw.d = d;
    vw.S = S;
    vw.M = M;
    vw.efc = efc;
    vw.X = X;
    vw.level = level.data();
    vw.row0 = row0.data();
    vw.nrows = nrows;
    vw.adj = adj.data();
    vw.adjd = adjd.data();
    vw.cnt = cnt.data();
    vw.entry_seg = entry_seg.data();
    vw.top_seg = top_seg.data();
    vw.dirty = dirty.data();
    vw.ndirty = (int64_t)dirty.size();
    vw.first = first;
    vw.count = count;
    return vw;
  }

  // Proposals of the batch [first, first + count) from the callback.
  bool propose_by_callback(int64_t first, int64_t count, std::vector<Proposal>& props) {
    const int64_t last = first + count - 1;
    const int64_t rf = row0[first];
    const int64_t rows = row0[last] + level[last] + 1 - rf;
    o_ids.resize((size_t)rows * S * M);
    o_dist.resize((size_t)rows * S * M);
    o_cnt.resize((size_t)rows * S);
    unify_build_view_t vw = view(first, count);
    propose_rc = propose_fn(propose_ctx, &vw, o_ids.data(), o_dist.data(), o_cnt.data());
    if (propose_rc != 0) return false;
    for (int64_t c : dirty) dirty_flag[c] = 0;
    dirty.clear();
    for (int64_t t = 0; t < count; ++t) {
      const int32_t v = (int32_t)(first + t);
      Proposal& P = props[t];
      P.fwd.assign((size_t)(level[v] + 1) * S, {});
      for (int l = 0; l <= level[v]; ++l)
        for (int j = 0; j < S; ++j) {
          const int64_t o = (row0[v] + l - rf) * S + j;
          const int c = o_cnt[o];
          if (c > M) { propose_rc = -1; return false; }
          std::vector<Key>& f = P.fwd[(size_t)l * S + j];
          for (int s = 0; s < c; ++s) f.push_back({o_dist[o * M + s], o_ids[o * M + s]});
        }
    }
    return true;
  }

  struct Rev { int32_t o; int32_t l; int32_t i; int32_t v; float dist; };
  std::vector<uint64_t> rev_key, rev_key_tmp;
  std::vector<uint32_t> rev_idx, rev_idx_tmp;
  std::vector<Rev> rev_tmp;
  std::vector<size_t> radix_count;

  // Stable LSD radix sort of revs by target chunk index, 11 bits per pass; leaves the
  // sorted keys in rev_key.
  void sort_by_chunk(std::vector<Rev>& revs) {
    const size_t N = revs.size();
    rev_key.resize(N);
    rev_idx.resize(N);
    uint64_t kmax = 0;
    for (size_t e = 0; e < N; ++e) {
      rev_key[e] = (uint64_t)(row(revs[e].o, revs[e].l) * S + revs[e].i);
      rev_idx[e] = (uint32_t)e;
      kmax = std::max(kmax, rev_key[e]);
    }
    rev_key_tmp.resize(N);
    rev_idx_tmp.resize(N);
    constexpr int kBits = 11;
    radix_count.assign((size_t)1 << kBits, 0);
    for (int shift = 0; shift == 0 || (kmax >> shift) != 0; shift += kBits) {
      std::fill(radix_count.begin(), radix_count.end(), 0);
      for (size_t e = 0; e < N; ++e) radix_count[(rev_key[e] >> shift) & ((1u << kBits) - 1)]++;
      size_t sum = 0;
      for (size_t& c : radix_count) {
        const size_t t = c;
        c = sum;
        sum += t;
      }
      for (size_t e = 0; e < N; ++e) {
        const size_t dst = radix_count[(rev_key[e] >> shift) & ((1u << kBits) - 1)]++;
        rev_key_tmp[dst] = rev_key[e];
        rev_idx_tmp[dst] = rev_idx[e];
      }
      rev_key.swap(rev_key_tmp);
      rev_idx.swap(rev_idx_tmp);
    }
    rev_tmp.resize(N);
    for (size_t e = 0; e < N; ++e) rev_tmp[e] = revs[rev_idx[e]];
    revs.swap(rev_tmp);
  }

  bool build(int threads) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
    int nth = omp_get_max_threads();
#else
    (void)threads;
    int nth = 1;
#endif
    segment();
    assign_levels();
    if (propose_fn) dirty_flag.assign((size_t)nrows * S, 0);
    std::vector<Visited> vis(nth);
    std::vector<std::vector<Key>> ann(nth), tmp(nth), kept(nth);
    std::vector<Proposal> props;
    std::vector<Rev> revs;
    int64_t done = 0;
    while (done < n) {
      int64_t bs = done < 1024 ? 1 : std::min<int64_t>(4096, done / 64);
      int64_t end = std::min<int64_t>(n, done + bs);
      int64_t cntb = end - done;
      props.assign(cntb, {});
      auto t0 = std::chrono::steady_clock::now();
      const bool by_cb = propose_fn && (cntb >= kAssistMinBatch || device_owns);
      if (by_cb) {
        if (!propose_by_callback(done, cntb, props)) return false;
        if (apply_fn) device_owns = true;
      } else {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
        for (int64_t t = 0; t < cntb; ++t) {
#ifdef _OPENMP
          int th = omp_get_thread_num();
#else
          int th = 0;
#endif
          propose((int32_t)(done + t), vis[th], props[t], ann[th], tmp[th]);
        }
      }
      auto t1 = std::chrono::steady_clock::now();
      (by_cb ? t_propose_cb : t_propose_host) += std::chrono::duration<double>(t1 - t0).count();
      // forward edges (batch nodes' own rows) and the reverse-edge list, in id order
      revs.clear();
      for (int64_t t = 0; t < cntb; ++t) {
        int32_t v = (int32_t)(done + t);
        int i = seg[v];
        const Proposal& P = props[t];
        for (int l = 0; l <= level[v]; ++l)
          for (int j = 0; j < S; ++j) {
            const std::vector<Key>& f = P.fwd[(size_t)l * S + j];
            if (f.empty()) continue;
            if (!device_owns) {
              set_chunk(row(v, l), j, f);
              if (propose_fn) mark_dirty(row(v, l) * S + j);
            }
            for (const Key& o : f) revs.push_back({o.second, l, i, v, o.first});
          }
      }
      // reverse edges grouped by target chunk, applied in source-id order: a stable
      // sort by chunk index (row(o, l) * S + i orders as (o, l, i), since a node's rows
      // are contiguous and ascend with its id)
      sort_by_chunk(revs);
      std::vector<size_t> starts;
      for (size_t e = 0; e < revs.size(); ++e)
        if (e == 0 || rev_key[e] != rev_key[e - 1]) starts.push_back(e);
      starts.push_back(revs.size());
      const int64_t ngroups = (int64_t)starts.size() - 1;
      if (device_owns) {
        // the callee stores the forward lists and applies the groups in this order
        g_chunk.resize(ngroups);
        g_start.resize(ngroups + 1);
        r_v.resize(revs.size());
        r_d.resize(revs.size());
        for (int64_t g = 0; g < ngroups; ++g) {
          g_chunk[g] = (int64_t)rev_key[starts[g]];
          g_start[g] = (int64_t)starts[g];
        }
        g_start[ngroups] = (int64_t)revs.size();
        for (size_t e = 0; e < revs.size(); ++e) {
          r_v[e] = revs[e].v;
          r_d[e] = revs[e].dist;
        }
        unify_build_view_t vw = view(done, cntb);
        propose_rc = apply_fn(propose_ctx, &vw, g_chunk.data(), g_start.data(), ngroups, r_v.data(), r_d.data());
        if (propose_rc != 0) return false;
      } else {
        if (propose_fn)
          for (int64_t g = 0; g < ngroups; ++g) {
            const Rev& e = revs[starts[g]];
            mark_dirty(row(e.o, e.l) * S + e.i);
          }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
        for (int64_t g = 0; g < ngroups; ++g) {
#ifdef _OPENMP
          int th = omp_get_thread_num();
#else
          int th = 0;
#endif
          for (size_t e = starts[g]; e < starts[g + 1]; ++e)
            add_reverse(revs[e].o, revs[e].l, revs[e].i, {revs[e].dist, revs[e].v}, tmp[th], kept[th]);
        }
      }
      t_apply += std::chrono::duration<double>(std::chrono::steady_clock::now() - t1).count();
      // entry points (Algorithm 6): only the node's own segment
      for (int64_t t = 0; t < cntb; ++t) {
        int32_t v = (int32_t)(done + t);
        int i = seg[v];
        if (entry_seg[i] < 0 || level[v] > top_seg[i]) {
          entry_seg[i] = v;
          top_seg[i] = level[v];
        }
      }
      done = end;
    }
    if (device_owns) {
      unify_build_view_t vw = view(n, 0);
      propose_rc = fetch_fn(propose_ctx, &vw, adj.data(), adjd.data(), cnt.data());
      if (propose_rc != 0) return false;
    }
    return true;
  }

  // ---- skip list (Section 4.1) and global edge masking (Algorithm 5) ----
  int max_level = 0;
  int32_t entry_global = -1;
  std::vector<int32_t> skip_next;  // per row
  std::vector<int32_t> skip_head;  // per layer
  std::vector<uint32_t> gmask;     // per row, W words
  int W = 0;

  void finalize(int threads) {
    (void)threads;
    max_level = 0;
    for (int64_t v = 0; v < n; ++v) max_level = std::max(max_level, level[v]);
    entry_global = -1;
    for (int64_t v = 0; v < n; ++v)
      if (level[v] == max_level) { entry_global = (int32_t)v; break; }
    // skip list: level-l chain over nodes of level >= l in attribute order
    skip_next.assign(nrows, -1);
    skip_head.assign(max_level + 1, -1);
    std::vector<int32_t> last(max_level + 1, -1);
    for (int64_t p = 0; p < n; ++p) {
      int32_t v = order[p];
      for (int l = 0; l <= level[v]; ++l) {
        if (last[l] < 0) skip_head[l] = v;
        else skip_next[row(last[l], l)] = v;
        last[l] = v;
      }
    }
    // Algorithm 5 over the final chunks.
    W = (S * M + 31) / 32;
    gmask.assign((size_t)nrows * W, 0u);
    // Prune(x, G[x], M) depends only on the final chunks: compute it for every row.
    std::vector<std::vector<int32_t>> keep_pos(nrows);
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
      std::vector<Key> cands, kept;
      std::vector<int32_t> posv;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
      for (int64_t v = 0; v < n; ++v) {
        for (int l = 0; l <= level[v]; ++l) {
          int64_t r = row0[v] + l;
          cands.clear();
          for (int j = 0; j < S; ++j) {
            int c = cnt[r * S + j];
            for (int s = 0; s < c; ++s)
              cands.push_back({adjd[(r * S + j) * M + s], adj[(r * S + j) * M + s]});
          }
          prune(cands, M, kept);
          posv.clear();
          for (const Key& k : kept) {
            int32_t id = k.second;
            int j = seg[id];
            int c = cnt[r * S + j];
            for (int s = 0; s < c; ++s)
              if (adj[(r * S + j) * M + s] == id) { posv.push_back(j * M + s); break; }
          }
          keep_pos[r] = posv;
        }
      }
    }
    auto popc = [&](int64_t r) {
      int c = 0;
      for (int w = 0; w < W; ++w) c += __builtin_popcount(gmask[r * W + w]);
      return c;
    };
    auto set_from = [&](int64_t r) {
      for (int w = 0; w < W; ++w) gmask[r * W + w] = 0;
      for (int32_t p : keep_pos[r]) gmask[r * W + (p >> 5)] |= 1u << (p & 31);
    };
    for (int64_t v = 0; v < n; ++v) {
      for (int l = 0; l <= level[v]; ++l) {
        int64_t r = row0[v] + l;
        set_from(r);
        for (int32_t p : keep_pos[r]) {
          int32_t o = adj[r * S * (int64_t)M + p];
          int64_t ro = row0[o] + l;
          int i = seg[v];
          int c = cnt[ro * S + i];
          int pos = -1;
          for (int s = 0; s < c; ++s)
            if (adj[(ro * S + i) * M + s] == (int32_t)v) { pos = i * M + s; break; }
          if (pos < 0) continue;
          gmask[ro * W + (pos >> 5)] |= 1u << (pos & 31);
          if (popc(ro) > M) set_from(ro);
        }
      }
    }
  }
};

// ---- index file writer ----
// Layout: "UNIFYHSG", u32 version, u32 nsec, then nsec 96-byte entries
// {char name[24]; u32 dtype; u32 ndim; u64 shape[4]; u64 offset; u64 nbytes;
//  u64 checksum; u64 reserved}, then the section payloads at 64-byte aligned
// offsets. dtype: 1 i8, 2 u8, 3 i32, 4 u32, 5 i64, 6 f32. checksum: FNV-1a 64
// over little-endian 8-byte words (the last word zero-padded).
struct Section {
  std::string name;
  uint32_t dtype;
  std::vector<uint64_t> shape;
  const void* data;
  uint64_t nbytes;
};

uint64_t fnv1a_words(const void* p, uint64_t nbytes) {
  const unsigned char* b = (const unsigned char*)p;
  uint64_t h = 0xcbf29ce484222325ull;
  uint64_t i = 0;
  for (; i + 8 <= nbytes; i += 8) {
    uint64_t w;
    std::memcpy(&w, b + i, 8);
    h = (h ^ w) * 0x100000001b3ull;
  }
  if (i < nbytes) {
    uint64_t w = 0;
    std::memcpy(&w, b + i, nbytes - i);
    h = (h ^ w) * 0x100000001b3ull;
  }
  return h;
}

bool write_index(const char* path, const std::vector<Section>& secs, std::string& err) {
  FILE* f = std::fopen(path, "wb");
  if (!f) { err = std::string("cannot open ") + path; return false; }
  const uint32_t version = 1, nsec = (uint32_t)secs.size();
  uint64_t off = 16 + 96ull * nsec;
  off = (off + 63) & ~63ull;
  std::vector<unsigned char> table(96ull * nsec, 0);
  std::vector<uint64_t> offs;
  for (size_t s = 0; s < secs.size(); ++s) {
    unsigned char* e = table.data() + 96 * s;
    std::strncpy((char*)e, secs[s].name.c_str(), 23);
    std::memcpy(e + 24, &secs[s].dtype, 4);
    uint32_t nd = (uint32_t)secs[s].shape.size();
    std::memcpy(e + 28, &nd, 4);
    for (uint32_t k = 0; k < 4; ++k) {
      uint64_t v = k < nd ? secs[s].shape[k] : 0;
      std::memcpy(e + 32 + 8 * k, &v, 8);
    }
    std::memcpy(e + 64, &off, 8);
    std::memcpy(e + 72, &secs[s].nbytes, 8);
    uint64_t ck = fnv1a_words(secs[s].data, secs[s].nbytes);
    std::memcpy(e + 80, &ck, 8);
    offs.push_back(off);
    off += secs[s].nbytes;
    off = (off + 63) & ~63ull;
  }
  bool ok = std::fwrite("UNIFYHSG", 1, 8, f) == 8 && std::fwrite(&version, 4, 1, f) == 1 &&
            std::fwrite(&nsec, 4, 1, f) == 1 && std::fwrite(table.data(), 1, table.size(), f) == table.size();
  uint64_t pos = 16 + table.size();
  static const unsigned char zeros[64] = {0};
  for (size_t s = 0; ok && s < secs.size(); ++s) {
    while (ok && pos < offs[s]) {
      size_t z = (size_t)std::min<uint64_t>(64, offs[s] - pos);
      ok = std::fwrite(zeros, 1, z, f) == z;
      pos += z;
    }
    ok = ok && std::fwrite(secs[s].data, 1, secs[s].nbytes, f) == secs[s].nbytes;
    pos += secs[s].nbytes;
  }
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) err = std::string("write failed: ") + path;
  return ok;
}

}  // namespace

extern "C" {

// Builds the HSIG over X (n x d float32, row-major) with integer attributes A and
// writes it to out_path. Returns 0 on success, a negative code otherwise (message
// in errbuf). threads <= 0 uses every available core. propose (may be null) takes
// over the proposal step of every batch of at least kAssistMinBatch nodes; apply and
// fetch (both null, or both set together with propose) take over edge application
// from the first proposal on; ctx is passed through. -3: a callback returned an
// error (its code in errbuf).
int hsig_build_index_ex(const float* X, const int64_t* A, int64_t n, int d, int S, int M, int efc,
                        uint64_t seed, int threads, const char* out_path, char* errbuf, int errlen,
                        unify_propose_fn propose, unify_apply_fn apply, unify_fetch_fn fetch, void* ctx) {
  auto fail = [&](int code, const std::string& msg) {
    if (errbuf && errlen > 0) {
      std::strncpy(errbuf, msg.c_str(), errlen - 1);
      errbuf[errlen - 1] = 0;
    }
    return code;
  };
  if (!X || !A || !out_path) return fail(-1, "null argument");
  if (n < 1 || n >= (1ll << 30)) return fail(-1, "n must be in [1, 2^30)");
  if (d < 1 || S < 1 || S > 32 || M < 1 || M > 255 || efc < 1) return fail(-1, "bad d/S/M/efc (S <= 32, M <= 255)");
  Builder b;
  b.n = n; b.d = d; b.S = S; b.M = M; b.efc = efc; b.seed = seed; b.X = X; b.A = A;
  if ((apply == nullptr) != (fetch == nullptr) || (apply && !propose))
    return fail(-1, "apply and fetch go together, and need propose");
  b.propose_fn = propose;
  b.apply_fn = apply;
  b.fetch_fn = fetch;
  b.propose_ctx = ctx;
  if (!b.build(threads)) return fail(-3, "build callback failed with code " + std::to_string(b.propose_rc));
  auto tf = std::chrono::steady_clock::now();
  b.finalize(threads);
  b.t_finalize = std::chrono::duration<double>(std::chrono::steady_clock::now() - tf).count();
  if (std::getenv("HSIG_BUILD_TIMING"))
    std::fprintf(stderr, "hsig_build: propose host %.2f s, propose callback %.2f s, apply edges %.2f s, "
                 "skip list + Algorithm 5 %.2f s\n", b.t_propose_host, b.t_propose_cb, b.t_apply, b.t_finalize);

  std::vector<int32_t> upper_base(n, -1);
  int64_t n_upper = 0;
  for (int64_t v = 0; v < n; ++v)
    if (b.level[v] > 0) { upper_base[v] = (int32_t)n_upper; n_upper += b.level[v]; }
  const int64_t SM = (int64_t)S * M;
  const int W = b.W;
  std::vector<int32_t> adj0((size_t)n * SM), adjU((size_t)std::max<int64_t>(1, n_upper) * SM, -1);
  std::vector<uint32_t> gm0((size_t)n * W), gmU((size_t)std::max<int64_t>(1, n_upper) * W, 0);
  std::vector<int32_t> next0(n), nextU((size_t)std::max<int64_t>(1, n_upper), -1);
  for (int64_t v = 0; v < n; ++v) {
    int64_t r = b.row0[v];
    std::memcpy(&adj0[(size_t)v * SM], &b.adj[(size_t)r * SM], SM * 4);
    std::memcpy(&gm0[(size_t)v * W], &b.gmask[(size_t)r * W], W * 4);
    next0[v] = b.skip_next[r];
    for (int l = 1; l <= b.level[v]; ++l) {
      int64_t u = upper_base[v] + l - 1;
      std::memcpy(&adjU[(size_t)u * SM], &b.adj[(size_t)(r + l) * SM], SM * 4);
      std::memcpy(&gmU[(size_t)u * W], &b.gmask[(size_t)(r + l) * W], W * 4);
      nextU[u] = b.skip_next[r + l];
    }
  }
  std::vector<int64_t> meta(16, 0);
  meta[0] = n; meta[1] = d; meta[2] = S; meta[3] = M; meta[4] = b.max_level;
  meta[5] = b.entry_global; meta[6] = n_upper; meta[7] = efc; meta[8] = (int64_t)seed; meta[9] = W;
  uint64_t nu = (uint64_t)std::max<int64_t>(1, n_upper);
  std::vector<Section> secs = {
      {"meta", 5, {16}, meta.data(), 16 * 8},
      {"vectors", 6, {(uint64_t)n, (uint64_t)d}, X, (uint64_t)n * d * 4},
      {"attr", 5, {(uint64_t)n}, A, (uint64_t)n * 8},
      {"level", 3, {(uint64_t)n}, b.level.data(), (uint64_t)n * 4},
      {"upper_base", 3, {(uint64_t)n}, upper_base.data(), (uint64_t)n * 4},
      {"seg_bounds", 5, {(uint64_t)S + 1}, b.bounds.data(), (uint64_t)(S + 1) * 8},
      {"seg_count", 5, {(uint64_t)S}, b.seg_count.data(), (uint64_t)S * 8},
      {"entry_seg", 3, {(uint64_t)S}, b.entry_seg.data(), (uint64_t)S * 4},
      {"sorted_ids", 3, {(uint64_t)n}, b.order.data(), (uint64_t)n * 4},
      {"skip_next0", 3, {(uint64_t)n}, next0.data(), (uint64_t)n * 4},
      {"skip_head", 3, {(uint64_t)b.max_level + 1}, b.skip_head.data(), (uint64_t)(b.max_level + 1) * 4},
      {"skip_nextU", 3, {nu}, nextU.data(), nu * 4},
      {"adj0", 3, {(uint64_t)n, (uint64_t)S, (uint64_t)M}, adj0.data(), (uint64_t)n * SM * 4},
      {"gmask0", 4, {(uint64_t)n, (uint64_t)W}, gm0.data(), (uint64_t)n * W * 4},
      {"adjU", 3, {nu, (uint64_t)S, (uint64_t)M}, adjU.data(), nu * SM * 4},
      {"gmaskU", 4, {nu, (uint64_t)W}, gmU.data(), nu * W * 4},
  };
  std::string err;
  if (!write_index(out_path, secs, err)) return fail(-2, err);
  return 0;
}

int hsig_build_index(const float* X, const int64_t* A, int64_t n, int d, int S, int M, int efc,
                     uint64_t seed, int threads, const char* out_path, char* errbuf, int errlen) {
  return hsig_build_index_ex(X, A, n, d, S, M, efc, seed, threads, out_path, errbuf, errlen, nullptr, nullptr,
                             nullptr, nullptr);
}

}  // extern "C"
