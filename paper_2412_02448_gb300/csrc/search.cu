// The search of one batch in one persistent kernel: hybrid filtering (Strategy
// C), post-filtering (Strategy B) and pre-filtering (Strategy A) of Section 4.2.
//
// Work queue. The router appends every query to a queue per strategy and splits
// each pre-filter query into scan items. One warp takes one work unit at a time
// from a single device counter, in the order: hybrid queries, post-filter queries,
// scan items. The long graph searches start first and the short scan items fill
// the tail, so the batch has one tail instead of one per strategy. A pre-filter
// query split into several items is merged by the warp that completes its last
// item (release/acquire through a per-query counter).
//
// Graph search (Algorithm 2's scheme; Algorithm 1 for B over bitmap-marked
// slots; Algorithm 7 for C over the first ceil(m/S') slots of each intersected
// chunk). One warp per query. Per-warp shared memory holds
//   E    the candidate buffer: every visited object that can still matter, sorted
//        by key (distance, id), with an "expanded" flag; popping the nearest
//        candidate is taking the first unexpanded entry;
//   ann  the result heap of Algorithms 1/7 as a sorted array of capacity ef;
//   vis  a direct-mapped visited filter (ids; a slot may be overwritten).
// Equivalence with the heap formulation: once ann holds ef entries its worst key
// w only decreases, and an object with key > w can neither enter cand or ann nor
// be expanded (the loop stops first), so E keeps exactly the visited objects with
// key <= w (all visited objects while ann is not full). An object the filter
// forgot is re-checked against E and ann by key, which is exact because its
// distance is recomputed bit-identically (fixed per-lane order and a fixed
// reduction tree). The neighbours of one expansion are processed as one batch
// against the ann of the start of the batch; objects the sequential loop would
// have rejected after an earlier insertion of the same batch end above the final
// w and are dropped from E, so the outcome is the same. The visible differences
// are the capacity of E (UNIFY_Q_TRUNCATED) and the expansion bound
// (UNIFY_Q_LIMIT). While an expansion is processed, the adjacency of the next
// candidate is prefetched into L2.
//
// Scan (Strategy A): rows [pa, pb) of the attribute-ordered vectors; a warp
// computes 32 rows per step with coalesced 16-byte loads issued in batches of
// 64 registers and a transposed shuffle reduction that leaves row r's distance
// in lane r; keys beating the current k-th are merged into a sorted top-k.
//
// Bounds (checked by reading, against the buffers the launch receives):
// E[< cand_cap], ann[< ann_cap], vis[< 2^vis_log2], clist[< 32], slots[< 64] as
// uint64 (S1 keys) or as ints (post-filter slots; the hybrid S2 table, < kSlotTable);
// ids come from validated adjacency (0 <= id < n); upper-layer rows exist for
// every object reached on that layer (validated levels); scan rows lie in
// [pa, pb) and loads clamp to the last valid row.
#include "common.cuh"
#include "internal.h"
#include "warp_ops.cuh"

namespace unify {

struct BatchArgs {
  const float* vec;                // float32 rows by id (re-rank, and traversal for FP32)
  const unsigned char* vt;         // traversal rows by id in the storage format
  const unsigned char* vts;        // the same rows in attribute order (scan)
  const float* scale;              // FP8 per-vector scales by id (else null)
  const float* scale_sorted;       // FP8 scales in attribute order
  int row_bytes;                   // bytes per stored row
  int rerank;                      // candidates re-ranked in FP32 (0: FP32 storage, none)
  const int32_t* sorted_ids;
  int dp4, d;
  int S, M, W, max_level, entry_global;
  const int32_t* adj0;
  const uint32_t* gmask0;
  const int32_t* adjU;
  const uint32_t* gmaskU;
  const int32_t* upper_base;
  const int32_t* pos;
  const int32_t* seg_start;
  const float* q;
  const int32_t* pa;
  const int32_t* pb;
  const uint32_t* mask;
  const int32_t* queues;
  int64_t cap_nq;
  const int32_t* nblk;
  const int32_t* qbase;
  int32_t* done;
  const int2* items;
  uint64_t* part;
  int32_t* counters;
  int k, ef_h, ef_p, m, cand_cap, ann_cap, vis_log2, max_exp;
  Conj cj;  // second-attribute predicate (attr2 == nullptr: none)
  int s1;  // hybrid selection S1 (the m neighbours nearest to the expanded object) instead of S2
  int warp_bytes;
  int skip_scan;  // the pre-filter queries were searched by the tensor-core scan
  Outputs o;
};

struct WarpMem {
  uint64_t* E;
  uint64_t* ann;
  int32_t* vis;
  uint8_t* Ef;
  int* R;
  int* clist;
  int* slots;  // post-filter: 64 bitmap-marked slots; hybrid S1: 64 selected keys (uint64)
};

__host__ __device__ inline int flag_cap(int cand_cap, int ann_cap) {
  return ((cand_cap > ann_cap ? cand_cap : ann_cap) + 15) & ~15;
}

constexpr int kSlotTable = 128;  // ints of the per-warp slots array (64 uint64)

__host__ __device__ inline int batch_warp_bytes(int cand_cap, int ann_cap, int vis_log2) {
  int b = cand_cap * 8 + ann_cap * 8 + (4 << vis_log2);
  b += flag_cap(cand_cap, ann_cap);
  b += 32 * 4 + 32 * 4 + 64 * 8;
  return (b + 15) & ~15;
}

__device__ __forceinline__ WarpMem carve(unsigned char* base, const BatchArgs& a) {
  WarpMem w;
  w.E = reinterpret_cast<uint64_t*>(base);
  w.ann = w.E + a.cand_cap;
  w.vis = reinterpret_cast<int32_t*>(w.ann + a.ann_cap);
  w.Ef = reinterpret_cast<uint8_t*>(w.vis + (1 << a.vis_log2));
  w.R = reinterpret_cast<int*>(w.Ef + flag_cap(a.cand_cap, a.ann_cap));
  w.clist = w.R + 32;
  w.slots = w.clist + 32;
  return w;
}

__device__ __forceinline__ uint32_t vis_hash(int id, int log2) {
  return ((uint32_t)id * 0x9E3779B1u) >> (32 - log2);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Microseconds since the first work unit of this launch started (instrumented runs).
__device__ __forceinline__ int us_since_start(int32_t* counters) {
  unsigned long long* t0 = reinterpret_cast<unsigned long long*>(counters + CNT_T0);
  const unsigned long long now = global_ns();
  unsigned long long base = atomicCAS(t0, 0ull, now);
  if (base == 0ull) base = now;
  return (int)((now - base) / 1000ull);
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// The second-attribute predicate for object id (true without a second attribute).
__device__ __forceinline__ bool conj_ok(const BatchArgs& a, int id, int64_t l2, int64_t h2) {
  if (!a.cj.attr2) return true;
  const int64_t v = __ldg(a.cj.attr2 + id);
  return v >= l2 && v <= h2;
}

// Slot (segment * M + s) of the ci-th selected neighbour (hybrid, S2 selection).
__device__ __forceinline__ int hybrid_slot(int ci, int per, uint32_t mask, int M, int* seg) {
  const int kseg = ci / per;
  const int s = ci - kseg * per;
  *seg = (int)__fns(mask, 0, kseg + 1);
  return *seg * M + s;
}

// One layer of Algorithm 1 (post) or Algorithm 7 (hybrid). Returns |ann|; the ann
// array is w.ann for hybrid. For post every candidate push is also an ann push, so
// cand is a subset of ann and one sorted buffer of capacity efl holds both: the
// result is then in w.ann as well (the buffer is w.ann itself).
template <class T, int CH, int G>
__device__ int search_layer(const BatchArgs& a, const WarpMem& w, const float4 (&q)[CH], bool hybrid, int l,
                            int efl, uint64_t ep_key, bool ep_in, uint32_t mask, uint32_t full_mask, int per,
                            int pa, int pb, int64_t l2, int64_t h2, int& n_dist, int& n_exp, uint32_t& status) {
  const int lane = lane_id();
  const int H = 1 << a.vis_log2;
  uint64_t* E = hybrid ? w.E : w.ann;  // candidate buffer
  const int capE = hybrid ? a.cand_cap : efl;
  for (int t = lane; t < H; t += 32) w.vis[t] = -1;
  __syncwarp();
  const int ep = key_id(ep_key);
  if (lane == 0) {
    E[0] = ep_key;
    w.Ef[0] = 0;
    if (hybrid && ep_in) w.ann[0] = ep_key;
    w.vis[vis_hash(ep, a.vis_log2)] = ep;
  }
  __syncwarp();
  int nE = 1, nA = hybrid ? (ep_in ? 1 : 0) : 1, cursor = 0, exp_l = 0;
  bool truncated = false;
  const int Sp = __popc(mask);
  const int SM = a.S * a.M;
  // Hybrid S2 selects the same slots in every expansion of the query: the slot and
  // segment of each selection index are tabled once (up to kSlotTable of them) in
  // the slots array, which S2 does not otherwise use.
  const bool tabled = hybrid && !a.s1 && Sp * per <= kSlotTable;
  if (tabled) {
    for (int ci = lane; ci < Sp * per; ci += 32) {
      int sg;
      const int slot = hybrid_slot(ci, per, mask, a.M, &sg);
      w.slots[ci] = slot | (sg << 16);
    }
    __syncwarp();
  }
  for (;;) {
    // the nearest unexpanded candidate
    while (cursor < nE) {
      const int j = cursor + lane;
      const bool un = j < nE && w.Ef[j] == 0;
      const unsigned bal = __ballot_sync(kFull, un);
      if (bal) {
        cursor += __ffs(bal) - 1;
        break;
      }
      cursor += 32;
    }
    if (cursor >= nE) break;
    if (exp_l >= a.max_exp) {
      status |= UNIFY_Q_LIMIT;
      break;
    }
    const int o = key_id(E[cursor]);
    __syncwarp();
    if (lane == 0) w.Ef[cursor] = 1;
    __syncwarp();
    ++exp_l;
    ++n_exp;
    const int64_t row = (l == 0) ? (int64_t)o : ((int64_t)__ldg(a.upper_base + o) + (l - 1));
    const int32_t* adj = (l == 0 ? a.adj0 : a.adjU) + row * SM;
    int ncand;
    if (hybrid && a.s1) {
      // Selection S1: every neighbour of o in the intersected chunks, by (distance
      // to o, id), the first m (these owner distances are not query distance
      // evaluations and are not counted)
      float4 xo[CH];
      {
        const unsigned char* orow = a.vt + (int64_t)o * a.row_bytes;
        const float sc = a.scale ? __ldg(a.scale + o) : 1.f;
#pragma unroll
        for (int t = 0; t < CH; ++t) {
          const int c = lane + 32 * t;
          xo[t] = c < a.dp4 ? value4<T>(T::load(orow, c, sc), sc) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      uint64_t* selk = reinterpret_cast<uint64_t*>(w.slots);
      const int msel = a.m < 64 ? a.m : 64;
      const int tot = Sp * a.M;
      int ns = 0;
      for (int b0 = 0; b0 < tot; b0 += 32) {
        const int ci = b0 + lane;
        int cid = -1;
        if (ci < tot) {
          const int kseg = ci / a.M;
          const int sl = ci - kseg * a.M;
          const int sg = (int)__fns(mask, 0, kseg + 1);
          cid = __ldg(adj + sg * a.M + sl);
        }
        const float dv = batch_dist<T, CH, G>(xo, cid, a.vt, a.row_bytes, a.scale, a.dp4, w.clist);
        ns = topk_offer(selk, ns, msel, cid >= 0 ? make_key(dv, cid) : kKeyMax, w.R);
      }
      ncand = ns;
    } else if (hybrid) {
      ncand = Sp * per;
    } else {
      // all bitmap words in one round trip, then compaction by ballots
      const uint32_t* gm = (l == 0 ? a.gmask0 : a.gmaskU) + row * a.W;
      int cnt = 0;
      for (int wb = 0; wb < a.W; wb += 32) {
        const uint32_t myword = wb + lane < a.W ? __ldg(gm + wb + lane) : 0u;
        const int nw = a.W - wb < 32 ? a.W - wb : 32;
        for (int wd = 0; wd < nw; ++wd) {
          const uint32_t word = __shfl_sync(kFull, myword, wd);
          const bool has = (word >> lane) & 1u;
          const unsigned bal = __ballot_sync(kFull, has);
          if (has) {
            const int p = cnt + __popc(bal & lanemask_lt());
            if (p < 64) w.slots[p] = (wb + wd) * 32 + lane;
          }
          cnt += __popc(bal);
        }
      }
      __syncwarp();
      ncand = cnt < 64 ? cnt : 64;
    }
    // prefetch the adjacency of the next candidate (layer 0) into L2
    if (l == 0) {
      const int j = cursor + 1 + lane;
      const unsigned bal = __ballot_sync(kFull, j < nE && w.Ef[j] == 0);
      if (bal) {
        const int o2 = key_id(E[cursor + __ffs(bal)]);
        const int32_t* adj2 = a.adj0 + (int64_t)o2 * SM;
        if (hybrid && !a.s1) {
          if (lane < ncand) {
            int sg;
            prefetch_l2(adj2 + (tabled ? (w.slots[lane] & 0xffff) : hybrid_slot(lane, per, mask, a.M, &sg)));
          }
        } else if (hybrid) {
          if (lane * 32 < SM) prefetch_l2(adj2 + lane * 32);
        } else {
          if (lane * 32 < SM) prefetch_l2(adj2 + lane * 32);
          if (lane == 31) prefetch_l2(a.gmask0 + (int64_t)o2 * a.W);
        }
      }
    }
    for (int rb = 0; rb < ncand; rb += 32) {
      const int ci = rb + lane;
      int cid = -1, cseg = 0;
      if (ci < ncand && hybrid && a.s1) {
        cid = key_id(reinterpret_cast<const uint64_t*>(w.slots)[ci]);
        cseg = -1;  // the range test below uses the position
      } else if (ci < ncand) {
        int slot;
        if (tabled) {
          const int e = w.slots[ci];
          slot = e & 0xffff;
          cseg = e >> 16;
        } else if (hybrid) {
          slot = hybrid_slot(ci, per, mask, a.M, &cseg);
        } else {
          slot = w.slots[ci];  // the post-filter tests no range while it traverses
        }
        if (slot < SM) cid = __ldg(adj + slot);
      }
      if (cid >= 0) {
        const uint32_t h = vis_hash(cid, a.vis_log2);
        if (w.vis[h] == cid) cid = -1;
        else w.vis[h] = cid;
      }
      __syncwarp();
      bool need = false;
      int pv = 0;
      if (hybrid && l == 0 && cid >= 0 && (cseg < 0 || !((full_mask >> cseg) & 1u))) {
        need = true;
        pv = __ldg(a.pos + cid);
      }
      const float dist = batch_dist<T, CH, G>(q, cid, a.vt, a.row_bytes, a.scale, a.dp4, w.clist);
      // layer 0 of a hybrid query: the range (by position where the segment is only
      // partly inside) and the second-attribute predicate
      const bool inr = (need ? (pv >= pa && pv < pb) : true) &&
                       (!(hybrid && l == 0 && cid >= 0) || conj_ok(a, cid, l2, h2));
      n_dist += __popc(__ballot_sync(kFull, cid >= 0));
      const uint64_t key = cid >= 0 ? make_key(dist, cid) : kKeyMax;
      const uint64_t thr = nA >= efl ? (hybrid ? w.ann[efl - 1] : E[efl - 1]) : kKeyMax;
      const bool keep = cid >= 0 && key < thr;
      const unsigned kb = __ballot_sync(kFull, keep);
      if (kb == 0) continue;
      int r0;
      bool dropped;
      uint64_t sk = keep ? key : kKeyMax;
      uint32_t fl = (keep && inr) ? 1u : 0u;
      warp_sort_kept(sk, fl, kb);
      int nk = __popc(kb);
      // a visited object the filter forgot is still in E (or, after an overflow of E,
      // possibly only in ann): drop it. Its rank in E is the merge's rank, found once.
      int rk = lane < nk ? lower_bound_u64(E, nE, sk) : nE;
      bool dup = lane < nk && rk < nE && E[rk] == sk;
      if (hybrid && truncated && lane < nk && !dup) dup = contains_u64(w.ann, nA, sk);
      if (__any_sync(kFull, dup)) {
        const unsigned kept = __ballot_sync(kFull, lane < nk && !dup);
        nk = __popc(kept);
        const int src = lane < nk ? (int)__fns(kept, 0, lane + 1) : lane;
        sk = __shfl_sync(kFull, sk, src);
        fl = __shfl_sync(kFull, fl, src);
        rk = __shfl_sync(kFull, rk, src);
        if (lane >= nk) {
          sk = kKeyMax;
          fl = 0u;
        }
        if (nk == 0) continue;
      }
      nE = warp_merge(E, w.Ef, nE, capE, sk, nk, w.R, &r0, &dropped, rk);
      if (r0 < cursor) cursor = r0;
      if (!hybrid) {
        nA = nE;  // cand and ann share the buffer; dropping beyond ef is ann's pop
        if (cursor > nE) cursor = nE;
        continue;
      }
      if (dropped) {
        truncated = true;
        status |= UNIFY_Q_TRUNCATED;
      }
      // in-range keys of the sorted batch, compacted in order
      const unsigned ab = __ballot_sync(kFull, lane < nk && fl != 0u);
      if (ab) {
        const int na = __popc(ab);
        const int src = lane < na ? (int)__fns(ab, 0, lane + 1) : 0;
        const uint64_t v = __shfl_sync(kFull, sk, src);
        nA = warp_merge(w.ann, nullptr, nA, efl, lane < na ? v : kKeyMax, na, w.R, &r0, &dropped);
      }
      if (nA >= efl) {
        nE = upper_bound_u64(E, nE, w.ann[efl - 1]);
        if (cursor > nE) cursor = nE;
      }
    }
  }
  return nA;
}

// FP32 re-rank: exact float32 distances (direct difference against the float32
// rows) of the nc candidates in keys[], the k best written to row qi. tmp holds
// >= k keys and does not overlap keys. Returns the number written.
template <int CH, int G>
__device__ int rerank_write(const BatchArgs& a, const WarpMem& w, const float4 (&q)[CH], const uint64_t* keys,
                            int nc, int64_t qi, uint64_t* tmp) {
  const int lane = lane_id();
  int nt = 0;
  for (int base = 0; base < nc; base += 32) {
    const int t = base + lane;
    const int cid = t < nc ? key_id(keys[t]) : -1;
    const float dist = batch_dist<StoreF32, CH, G>(q, cid, reinterpret_cast<const unsigned char*>(a.vec),
                                                   a.dp4 * 16, nullptr, a.dp4, w.clist);
    const uint64_t key = cid >= 0 ? make_key(dist, cid) : kKeyMax;
    nt = topk_offer(tmp, nt, a.k, key, w.R);
  }
  write_row(tmp, nt, a.k, qi, a.o);
  return nt;
}

template <class T, int CH, int G, int GF>
__device__ void graph_query(const BatchArgs& a, const WarpMem& w, int qi, bool hybrid) {
  const int lane = lane_id();
  int t_start = 0;
  if (a.o.counters && lane == 0) t_start = us_since_start(a.counters);
  const uint32_t mask = a.mask[qi];
  const int pa = a.pa[qi], pb = a.pb[qi];
  const int64_t l2 = a.cj.attr2 ? a.cj.lo2[qi] : 0, h2 = a.cj.attr2 ? a.cj.hi2[qi] : 0;
  uint32_t status = 0;
  int n_dist = 0, n_exp = 0, cnt = 0;
  if (hybrid ? mask != 0 : pb > pa) {  // nothing can be in range otherwise
    float4 q[CH];
    load_query<CH>(q, a.q + (int64_t)qi * a.d, a.d);
    uint32_t full_mask = 0;
    for (int j = 0; j < a.S; ++j)
      if (((mask >> j) & 1u) && __ldg(a.seg_start + j) >= pa && __ldg(a.seg_start + j + 1) <= pb)
        full_mask |= 1u << j;
    const int Sp = __popc(mask);
    int per = Sp > 0 ? (a.m + Sp - 1) / Sp : 0;
    if (per > a.M) per = a.M;
    const int efl0 = hybrid ? (a.ef_h > a.k ? a.ef_h : a.k) : (a.ef_p > a.k ? a.ef_p : a.k);
    // entry point: the first object on the top layer
    const int ep0 = a.entry_global;
    const float d0 = batch_dist<T, CH, G>(q, lane == 0 ? ep0 : -1, a.vt, a.row_bytes, a.scale, a.dp4, w.clist);
    uint64_t ep_key = make_key(__shfl_sync(kFull, d0, 0), ep0);
    n_dist = 1;
    int nA = 0;
    for (int l = a.max_level; l >= 0; --l) {
      const int ep = key_id(ep_key);
      bool ep_in = true;
      if (hybrid) {
        const int p = __ldg(a.pos + ep);
        if (l == 0) {
          ep_in = p >= pa && p < pb && conj_ok(a, ep, l2, h2);
        } else {
          int seg = 0;
          for (int j = 1; j < a.S; ++j)
            if (__ldg(a.seg_start + j) <= p) seg = j;
          ep_in = (mask >> seg) & 1u;
        }
      }
      nA = search_layer<T, CH, G>(a, w, q, hybrid, l, l > 0 ? 1 : efl0, ep_key, ep_in, mask, full_mask, per, pa, pb,
                               l2, h2, n_dist, n_exp, status);
      if (l > 0 && nA > 0) ep_key = w.ann[0];
    }
    if (a.rerank > 0) {
      // reduced-precision storage: re-rank the first rerank_mult * k candidates in FP32
      const uint64_t* src = w.ann;
      int nc = nA;
      if (!hybrid) {
        // Strategy B: the range filter first, compacted into E (free after the search)
        nc = 0;
        for (int base = 0; base < nA && nc < a.rerank; base += 32) {
          const int t = base + lane;
          bool inr = false;
          uint64_t key = kKeyMax;
          if (t < nA) {
            key = w.ann[t];
            const int p = __ldg(a.pos + key_id(key));
            inr = p >= pa && p < pb && conj_ok(a, key_id(key), l2, h2);
          }
          const unsigned bal = __ballot_sync(kFull, inr);
          const int dst = nc + __popc(bal & lanemask_lt());
          if (inr && dst < a.rerank) w.E[dst] = key;
          nc += __popc(bal);
        }
        __syncwarp();
        src = w.E;
      }
      if (nc > a.rerank) nc = a.rerank;
      cnt = rerank_write<CH, GF>(a, w, q, src, nc, qi, hybrid ? w.E : w.ann);
    } else if (hybrid) {
      cnt = nA < a.k ? nA : a.k;
      write_row(w.ann, cnt, a.k, qi, a.o);
    } else {
      // Strategy B: filter ann by the range, keep the first k
      for (int base = 0; base < nA && cnt < a.k; base += 32) {
        const int t = base + lane;
        bool inr = false;
        uint64_t key = kKeyMax;
        if (t < nA) {
          key = w.ann[t];
          const int p = __ldg(a.pos + key_id(key));
          inr = p >= pa && p < pb && conj_ok(a, key_id(key), l2, h2);
        }
        const unsigned bal = __ballot_sync(kFull, inr);
        const int dst = cnt + __popc(bal & lanemask_lt());
        if (inr && dst < a.k) {
          a.o.ids[(int64_t)qi * a.k + dst] = key_id(key);
          a.o.dist[(int64_t)qi * a.k + dst] = key_dist(key);
        }
        cnt += __popc(bal);
      }
      if (cnt > a.k) cnt = a.k;
      for (int t = cnt + lane; t < a.k; t += 32) {
        a.o.ids[(int64_t)qi * a.k + t] = -1;
        a.o.dist[(int64_t)qi * a.k + t] = __int_as_float(0x7f800000);
      }
    }
  } else {
    write_row(w.ann, 0, a.k, qi, a.o);
  }
  if (lane == 0) {
    a.o.count[qi] = cnt;
    if (a.o.status) a.o.status[qi] = status;
    if (a.o.counters) {
      a.o.counters[4 * (int64_t)qi] = n_dist;
      a.o.counters[4 * (int64_t)qi + 1] = n_exp;
      a.o.counters[4 * (int64_t)qi + 2] = t_start;
      a.o.counters[4 * (int64_t)qi + 3] = us_since_start(a.counters);
    }
  }
  __syncwarp();
}

template <class T, int CH, int G, int GF>
__device__ void scan_item(const BatchArgs& a, const WarpMem& w, int it) {
  const int lane = lane_id();
  uint64_t* topk = w.ann;  // ann_cap >= kk
  const int kk = a.rerank > 0 ? a.rerank : a.k;  // keys kept per list
  const int2 item = a.items[it];
  const int qi = item.x, b = item.y;
  if (a.o.counters && lane == 0) atomicMin(&a.o.counters[4 * (int64_t)qi + 2], us_since_start(a.counters));
  const int pa = a.pa[qi], pb = a.pb[qi], nb = a.nblk[qi];
  const int Y = pb - pa;
  const int rpb = (Y + nb - 1) / (nb > 0 ? nb : 1);
  const int r0 = pa + b * rpb;
  const int r1 = min(pb, r0 + rpb);
  const int64_t l2 = a.cj.attr2 ? a.cj.lo2[qi] : 0, h2 = a.cj.attr2 ? a.cj.hi2[qi] : 0;
  float4 q[CH];
  load_query<CH>(q, a.q + (int64_t)qi * a.d, a.d);
  // rows per load batch: all 32 rows of a step where raw narrow chunks are held and
  // rows have at most 128 elements (bfloat16: 64 registers), otherwise 16 / CH (64
  // registers of float32 chunks)
  constexpr int RB = (CH == 1 && T::kRawRegs < 4 && T::kHoldRaw) ? 32 : ((16 / CH) > 2 ? (16 / CH) : 2);
  int nt = 0;
  for (int base = r0; base < r1; base += 32) {
    float part[32];
#pragma unroll
    for (int h = 0; h < 32; h += RB) {
      Held<T> x[RB][CH];
      float sc[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int row = min(base + h + r, r1 - 1);
        const unsigned char* src = a.vts + (int64_t)row * a.row_bytes;
        sc[r] = a.scale_sorted ? __ldg(a.scale_sorted + row) : 1.f;
#pragma unroll
        for (int t = 0; t < CH; ++t) {
          const int c = lane + 32 * t;
          if constexpr (T::kHoldRaw) x[r][t] = c < a.dp4 ? T::load_raw(src, c) : T::zero_raw();
          else x[r][t] = c < a.dp4 ? T::load(src, c, sc[r]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        float s = 0.f;
#pragma unroll
        for (int t = 0; t < CH; ++t) {
          const float4 e = diff4<T>(q[t], unhold<T>(x[r][t]), sc[r]);
          s = fmaf(e.x, e.x, s);
          s = fmaf(e.y, e.y, s);
          s = fmaf(e.z, e.z, s);
          s = fmaf(e.w, e.w, s);
        }
        part[h + r] = s;
      }
    }
    const float dist = warp_transpose_reduce<32>(part);
    const int row = base + lane;
    uint64_t key = kKeyMax;
    if (row < r1) {
      const int32_t id = __ldg(a.sorted_ids + row);
      if (conj_ok(a, id, l2, h2)) key = make_key(dist, id);
    }
    nt = topk_offer(topk, nt, kk, key, w.R);
  }
  if (nb > 1) {
    // split query: publish the partial list; the warp finishing the last item merges
    uint64_t* dst = a.part + (int64_t)it * kk;
    for (int t = lane; t < kk; t += 32) dst[t] = t < nt ? topk[t] : kKeyMax;
    __threadfence();
    __syncwarp();
    int prev = 0;
    if (lane == 0) prev = atomicAdd(&a.done[qi], 1);
    prev = __shfl_sync(kFull, prev, 0);
    if (prev != nb - 1) {
      if (a.o.counters && lane == 0) atomicMax(&a.o.counters[4 * (int64_t)qi + 3], us_since_start(a.counters));
      return;
    }
    __threadfence();
    const uint64_t* src = a.part + (int64_t)a.qbase[qi] * kk;
    const int total = nb * kk;
    nt = 0;
    for (int off = 0; off < total; off += 32) {
      const uint64_t key = (off + lane < total)
                               ? __ldcg(reinterpret_cast<const unsigned long long*>(src) + off + lane)
                               : kKeyMax;
      nt = topk_offer(topk, nt, kk, key, w.R);
    }
    nt = min(nt, Y);
  }
  int cnt;
  if (a.rerank > 0) {
    cnt = rerank_write<CH, GF>(a, w, q, topk, nt, qi, w.E);
  } else {
    cnt = min(nt, a.k);
    write_row(topk, cnt, a.k, qi, a.o);
  }
  if (lane == 0) {
    a.o.count[qi] = cnt;
    if (a.o.status) a.o.status[qi] = 0u;
    if (a.o.counters) atomicMax(&a.o.counters[4 * (int64_t)qi + 3], us_since_start(a.counters));
  }
  __syncwarp();
}

// MINB: minimum resident CTAs of 128 threads per SM the register allocation must
// allow (4 -> 128 registers, 6 -> 80, 8 -> 64).
template <class T, int CH, int G, int GF, int MINB>
__global__ void __launch_bounds__(128, MINB) batch_kernel(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const WarpMem w = carve(smem_raw + (size_t)warp * a.warp_bytes, a);
  const int nC = a.counters[CNT_QC], nB = a.counters[CNT_QB], nI = a.skip_scan ? 0 : a.counters[CNT_ITEMS];
  for (;;) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(&a.counters[CNT_TAKE], 1);
    idx = __shfl_sync(kFull, idx, 0);
    if (idx < nC) {
      graph_query<T, CH, G, GF>(a, w, a.queues[a.cap_nq + idx], true);
    } else if (idx < nC + nB) {
      graph_query<T, CH, G, GF>(a, w, a.queues[2 * a.cap_nq + (idx - nC)], false);
    } else if (idx < nC + nB + nI) {
      scan_item<T, CH, G, GF>(a, w, idx - nC - nB);
    } else {
      break;
    }
  }
}

template <class T, int CH, int G, int GF, int MINB>
static cudaError_t launch_t(const BatchArgs& a, int wpb, int num_sms, cudaStream_t st) {
  const int threads = 32 * wpb;
  const size_t smem = (size_t)wpb * a.warp_bytes;
  cudaError_t e = cudaFuncSetAttribute(batch_kernel<T, CH, G, GF, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<T, CH, G, GF, MINB>, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  batch_kernel<T, CH, G, GF, MINB><<<num_sms * per_sm, threads, smem, st>>>(a);
  return cudaGetLastError();
}

template <class T>
static cudaError_t launch_dt(const BatchArgs& a, int wpb, int regs, int num_sms, cudaStream_t st) {
  // G rows per distance group: G * CH = 16 row chunks in flight (8 under the
  // 64-register budget, and for FP8 rows, decoded when they load, under the 80-register
  // one: 16 decoded rows crowd its registers and measured 13 % slower on GB300); a group
  // of 32 raw bfloat16 or FP8 rows measured no faster. GF rows per group of the float32
  // re-rank, which runs after the traversal.
  const int ch = (a.dp4 + 31) / 32;
  if (ch <= 1) {
    if (regs == 80) {
      if constexpr (T::kHoldRaw) return launch_t<T, 1, 16, 16, 6>(a, wpb, num_sms, st);
      else return launch_t<T, 1, 8, 8, 6>(a, wpb, num_sms, st);
    }
    if (regs == 64) return launch_t<T, 1, 8, 8, 8>(a, wpb, num_sms, st);
    return launch_t<T, 1, 16, 16, 4>(a, wpb, num_sms, st);
  }
  if (ch <= 2) return launch_t<T, 2, 8, 8, 4>(a, wpb, num_sms, st);
  if (ch <= 4) return launch_t<T, 4, 4, 4, 4>(a, wpb, num_sms, st);
  return launch_t<T, 8, 2, 2, 4>(a, wpb, num_sms, st);
}

int rerank_count(const Params& p) { return p.dtype == UNIFY_FP32 ? 0 : p.rerank_mult * p.k; }

int batch_ann_cap(const Params& p) {
  int c = p.ef > p.ef_post ? p.ef : p.ef_post;
  if (c < p.k) c = p.k;
  if (c < rerank_count(p)) c = rerank_count(p);
  return c;
}

int batch_smem_per_warp(const Params& p) { return batch_warp_bytes(p.cand_cap, batch_ann_cap(p), p.vis_log2); }

cudaError_t launch_batch(const DeviceIndex& ix, const Scratch& sc, const float* q, const Params& p,
                         const Outputs& o, cudaStream_t st, bool skip_scan, const Conj* cj) {
  BatchArgs a;
  a.cj = cj ? *cj : Conj{};
  a.skip_scan = skip_scan ? 1 : 0;
  a.vec = ix.vec;
  a.dp4 = ix.dp / 4;
  a.rerank = rerank_count(p);
  if (p.dtype == UNIFY_BF16) {
    a.vt = ix.vt_bf16;
    a.vts = ix.vts_bf16;
    a.scale = a.scale_sorted = nullptr;
    a.row_bytes = a.dp4 * 8;
  } else if (p.dtype == UNIFY_FP8E4M3) {
    a.vt = ix.vt_fp8;
    a.vts = ix.vts_fp8;
    a.scale = ix.scale_fp8;
    a.scale_sorted = ix.scale_fp8_sorted;
    a.row_bytes = a.dp4 * 4;
  } else {
    a.vt = reinterpret_cast<const unsigned char*>(ix.vec);
    a.vts = reinterpret_cast<const unsigned char*>(ix.vec_sorted);
    a.scale = a.scale_sorted = nullptr;
    a.row_bytes = a.dp4 * 16;
  }
  a.sorted_ids = ix.sorted_ids;
  a.d = ix.d;
  a.S = ix.S;
  a.M = ix.M;
  a.W = ix.W;
  a.max_level = ix.max_level;
  a.entry_global = ix.entry_global;
  a.adj0 = ix.adj0;
  a.gmask0 = ix.gmask0;
  a.adjU = ix.adjU;
  a.gmaskU = ix.gmaskU;
  a.upper_base = ix.upper_base;
  a.pos = ix.pos;
  a.seg_start = ix.seg_start;
  a.q = q;
  a.pa = sc.pa;
  a.pb = sc.pb;
  a.mask = sc.mask;
  a.queues = sc.queues;
  a.cap_nq = sc.cap_nq;
  a.nblk = sc.nblk;
  a.qbase = sc.qbase;
  a.done = sc.done;
  a.items = sc.items;
  a.part = sc.part;
  a.counters = sc.counters;
  a.k = p.k;
  a.ef_h = p.ef;
  a.ef_p = p.ef_post;
  a.m = p.m;
  a.s1 = p.selection == 1 ? 1 : 0;
  a.cand_cap = p.cand_cap;
  a.ann_cap = batch_ann_cap(p);
  a.vis_log2 = p.vis_log2;
  a.max_exp = p.max_exp;
  a.warp_bytes = batch_warp_bytes(a.cand_cap, a.ann_cap, a.vis_log2);
  a.o = o;
  const int wpb = p.warps_per_block;
  if (p.dtype == UNIFY_BF16) return launch_dt<StoreBF16>(a, wpb, p.reg_budget, ix.num_sms, st);
  if (p.dtype == UNIFY_FP8E4M3) return launch_dt<StoreFP8>(a, wpb, p.reg_budget, ix.num_sms, st);
  return launch_dt<StoreF32>(a, wpb, p.reg_budget, ix.num_sms, st);
}

}  // namespace unify
