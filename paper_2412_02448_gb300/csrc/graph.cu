// Strategies B (post-filter) and C (hybrid) of Section 4.2: Algorithm 2's layer
// scheme with Algorithm 1 (B, over bitmap-marked edges) or Algorithm 7 (C, over
// the first ceil(m/S') slots of each intersected chunk) on every layer.
//
// One warp per query, persistent over a device queue of query ids. Per-warp
// shared memory holds
//   E    the candidate buffer: every visited object that can still matter, sorted
//        by key (distance, id), with an "expanded" flag. Popping the nearest
//        candidate is taking the first unexpanded entry.
//   ann  the result heap of Algorithms 1/7 as a sorted array of capacity ef.
//   vis  a direct-mapped visited filter (ids; a slot may be overwritten).
// Equivalence with the heap formulation: once ann holds ef entries its worst key w
// only decreases, and an object with key > w can neither enter cand or ann nor be
// expanded (the loop stops first), so E keeps exactly the visited objects with key
// <= w (all visited objects while ann is not full). An object the filter forgot is
// re-checked against E and ann by key, which is exact because its distance is
// recomputed bit-identically. The neighbours of one expansion are processed as one
// batch against the ann of the start of the batch; objects that the sequential
// loop would have rejected after an earlier insertion of the same batch end with a
// key above the final w and are dropped from E, so the outcome is the same. The
// visible differences are the capacity of E (UNIFY_Q_TRUNCATED when it overflowed)
// and the expansion bound (UNIFY_Q_LIMIT).
#include "common.cuh"
#include "internal.h"

namespace unify {

struct GraphArgs {
  const float* vec;
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
  const int32_t* queue;
  int32_t* counters;
  int qcount_idx, take_idx;
  int strategy;
  int k, efl, m, cand_cap, ann_cap, vis_log2, max_exp;
  int warp_bytes;
  Outputs o;
};

struct WarpMem {
  uint64_t* E;
  uint64_t* ann;
  int32_t* vis;
  uint8_t* Ef;
  int* R;
  int* clist;
  int* slots;
};

__host__ __device__ inline int warp_mem_bytes(int cand_cap, int ann_cap, int vis_log2) {
  int b = cand_cap * 8 + ann_cap * 8 + (4 << vis_log2);
  b += (cand_cap + 15) & ~15;
  b += 32 * 4 + 32 * 4 + 64 * 4;
  return (b + 15) & ~15;
}

__device__ __forceinline__ WarpMem carve(unsigned char* base, const GraphArgs& a) {
  WarpMem w;
  w.E = reinterpret_cast<uint64_t*>(base);
  w.ann = w.E + a.cand_cap;
  w.vis = reinterpret_cast<int32_t*>(w.ann + a.ann_cap);
  w.Ef = reinterpret_cast<uint8_t*>(w.vis + (1 << a.vis_log2));
  w.R = reinterpret_cast<int*>(w.Ef + ((a.cand_cap + 15) & ~15));
  w.clist = w.R + 32;
  w.slots = w.clist + 32;
  return w;
}

__device__ __forceinline__ uint32_t vis_hash(int id, int log2) {
  return ((uint32_t)id * 0x9E3779B1u) >> (32 - log2);
}

// Distances of the candidates held by the lanes (cid >= 0), G at a time.
template <int CH, int G>
__device__ __forceinline__ float batch_dist(const float4 (&q)[CH], int cid, const float* vec, int dp4,
                                            int* clist) {
  const int lane = lane_id();
  const unsigned vm = __ballot_sync(kFull, cid >= 0);
  const int nv = __popc(vm);
  const int my = __popc(vm & lanemask_lt());
  if (cid >= 0) clist[my] = cid;
  __syncwarp();
  constexpr int SH = (G == 8) ? 2 : (G == 16 ? 1 : 0);
  float result = 0.f;
  for (int g = 0; g * G < nv; ++g) {
    float part[G];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int c = g * G + u;
      part[u] = (c < nv) ? l2_partial<CH>(q, vec + (int64_t)clist[c] * dp4 * 4, dp4) : 0.f;
    }
    const float red = warp_transpose_reduce<G>(part);
    const int u = my - g * G;
    const bool mine = cid >= 0 && u >= 0 && u < G;
    const float v = __shfl_sync(kFull, red, mine ? (u << SH) : 0);
    if (mine) result = v;
  }
  __syncwarp();
  return result;
}

// One layer of Algorithm 1 (post) or Algorithm 7 (hybrid). Returns |ann|.
template <int CH, int G>
__device__ int search_layer(const GraphArgs& a, const WarpMem& w, const float4 (&q)[CH], int l, int efl,
                            uint64_t ep_key, bool ep_in, uint32_t mask, uint32_t full_mask, int per,
                            int pa, int pb, int& n_dist, int& n_exp, uint32_t& status) {
  const int lane = lane_id();
  const bool hybrid = a.strategy == UNIFY_HYBRID;
  const int H = 1 << a.vis_log2;
  for (int t = lane; t < H; t += 32) w.vis[t] = -1;
  __syncwarp();
  const int ep = key_id(ep_key);
  if (lane == 0) {
    w.E[0] = ep_key;
    w.Ef[0] = 0;
    if (ep_in) w.ann[0] = ep_key;
    w.vis[vis_hash(ep, a.vis_log2)] = ep;
  }
  __syncwarp();
  int nE = 1, nA = ep_in ? 1 : 0, cursor = 0, exp_l = 0;
  const int Sp = __popc(mask);
  const int SM = a.S * a.M;
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
    const int o = key_id(w.E[cursor]);
    __syncwarp();
    if (lane == 0) w.Ef[cursor] = 1;
    __syncwarp();
    ++exp_l;
    ++n_exp;
    const int64_t row = (l == 0) ? (int64_t)o : ((int64_t)__ldg(a.upper_base + o) + (l - 1));
    const int32_t* adj = (l == 0 ? a.adj0 : a.adjU) + row * SM;
    int ncand;
    if (hybrid) {
      ncand = Sp * per;
    } else {
      const uint32_t* gm = (l == 0 ? a.gmask0 : a.gmaskU) + row * a.W;
      int cnt = 0;
      for (int wd = 0; wd < a.W; ++wd) {
        const uint32_t word = __ldg(gm + wd);
        const bool has = (word >> lane) & 1u;
        const unsigned bal = __ballot_sync(kFull, has);
        if (has) {
          const int p = cnt + __popc(bal & lanemask_lt());
          if (p < 64) w.slots[p] = wd * 32 + lane;
        }
        cnt += __popc(bal);
      }
      __syncwarp();
      ncand = cnt < 64 ? cnt : 64;
    }
    for (int rb = 0; rb < ncand; rb += 32) {
      const int ci = rb + lane;
      int cid = -1, cseg = 0;
      if (ci < ncand) {
        int slot;
        if (hybrid) {
          const int kseg = ci / per;
          const int s = ci - kseg * per;
          cseg = (int)__fns(mask, 0, kseg + 1);
          slot = cseg * a.M + s;
        } else {
          slot = w.slots[ci];
          cseg = slot / a.M;
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
      if (hybrid && l == 0 && cid >= 0 && !((full_mask >> cseg) & 1u)) {
        need = true;
        pv = __ldg(a.pos + cid);
      }
      const float dist = batch_dist<CH, G>(q, cid, a.vec, a.dp4, w.clist);
      const bool inr = need ? (pv >= pa && pv < pb) : true;
      n_dist += __popc(__ballot_sync(kFull, cid >= 0));
      const uint64_t key = cid >= 0 ? make_key(dist, cid) : kKeyMax;
      const uint64_t thr = nA >= efl ? w.ann[efl - 1] : kKeyMax;
      bool keep = cid >= 0 && key < thr;
      if (keep && (contains_u64(w.E, nE, key) || contains_u64(w.ann, nA, key))) keep = false;
      const unsigned kb = __ballot_sync(kFull, keep);
      if (kb == 0) continue;
      int r0;
      bool dropped;
      const uint64_t sk = warp_sort_asc(keep ? key : kKeyMax);
      nE = warp_merge(w.E, w.Ef, nE, a.cand_cap, sk, __popc(kb), w.R, &r0, &dropped);
      if (dropped) status |= UNIFY_Q_TRUNCATED;
      if (r0 < cursor) cursor = r0;
      const bool ka = keep && inr;
      const unsigned ab = __ballot_sync(kFull, ka);
      if (ab) {
        const uint64_t sa = warp_sort_asc(ka ? key : kKeyMax);
        nA = warp_merge(w.ann, nullptr, nA, efl, sa, __popc(ab), w.R, &r0, &dropped);
      }
      if (nA >= efl) {
        nE = upper_bound_u64(w.E, nE, w.ann[efl - 1]);
        if (cursor > nE) cursor = nE;
      }
    }
  }
  return nA;
}

template <int CH, int G>
__global__ void __launch_bounds__(256) graph_kernel(GraphArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const WarpMem w = carve(smem_raw + (size_t)warp * a.warp_bytes, a);
  const bool hybrid = a.strategy == UNIFY_HYBRID;
  const int nqs = a.counters[a.qcount_idx];
  for (;;) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(&a.counters[a.take_idx], 1);
    idx = __shfl_sync(kFull, idx, 0);
    if (idx >= nqs) break;
    const int qi = a.queue[idx];
    const uint32_t mask = a.mask[qi];
    const int pa = a.pa[qi], pb = a.pb[qi];
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
      // entry point: the first object on the top layer
      const int ep0 = a.entry_global;
      const float d0 = batch_dist<CH, G>(q, lane == 0 ? ep0 : -1, a.vec, a.dp4, w.clist);
      uint64_t ep_key = make_key(__shfl_sync(kFull, d0, 0), ep0);
      n_dist = 1;
      int nA = 0;
      for (int l = a.max_level; l >= 0; --l) {
        const int ep = key_id(ep_key);
        bool ep_in = true;
        if (hybrid) {
          const int p = __ldg(a.pos + ep);
          if (l == 0) {
            ep_in = p >= pa && p < pb;
          } else {
            int seg = 0;
            for (int j = 1; j < a.S; ++j)
              if (__ldg(a.seg_start + j) <= p) seg = j;
            ep_in = (mask >> seg) & 1u;
          }
        }
        const int efl = l > 0 ? 1 : a.efl;
        nA = search_layer<CH, G>(a, w, q, l, efl, ep_key, ep_in, mask, full_mask, per, pa, pb, n_dist,
                                 n_exp, status);
        if (l > 0 && nA > 0) ep_key = w.ann[0];
      }
      // results
      if (hybrid) {
        cnt = nA < a.k ? nA : a.k;
        for (int t = lane; t < a.k; t += 32) {
          const bool v = t < cnt;
          const uint64_t key = v ? w.ann[t] : kKeyMax;
          a.o.ids[(int64_t)qi * a.k + t] = v ? (int64_t)key_id(key) : (int64_t)-1;
          a.o.dist[(int64_t)qi * a.k + t] = v ? key_dist(key) : __int_as_float(0x7f800000);
        }
      } else {
        // Strategy B: filter ann by the range, keep the first k
        for (int base = 0; base < nA && cnt < a.k; base += 32) {
          const int t = base + lane;
          bool inr = false;
          uint64_t key = kKeyMax;
          if (t < nA) {
            key = w.ann[t];
            const int p = __ldg(a.pos + key_id(key));
            inr = p >= pa && p < pb;
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
      for (int t = lane; t < a.k; t += 32) {
        a.o.ids[(int64_t)qi * a.k + t] = -1;
        a.o.dist[(int64_t)qi * a.k + t] = __int_as_float(0x7f800000);
      }
    }
    if (lane == 0) {
      a.o.count[qi] = cnt;
      if (a.o.status) a.o.status[qi] = status;
      if (a.o.counters) {
        a.o.counters[2 * (int64_t)qi] = n_dist;
        a.o.counters[2 * (int64_t)qi + 1] = n_exp;
      }
    }
    __syncwarp();
  }
}

template <int CH, int G>
static cudaError_t launch_graph_t(const GraphArgs& a, int wpb, int num_sms, cudaStream_t st) {
  const int threads = 32 * wpb;
  const size_t smem = (size_t)wpb * a.warp_bytes;
  cudaError_t e = cudaFuncSetAttribute(graph_kernel<CH, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, graph_kernel<CH, G>, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  graph_kernel<CH, G><<<num_sms * per_sm, threads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_graph(const DeviceIndex& ix, const Scratch& sc, const float* q, int64_t nq,
                         int strategy, const Params& p, const Outputs& o, cudaStream_t st) {
  (void)nq;
  GraphArgs a;
  a.vec = ix.vec;
  a.dp4 = ix.dp / 4;
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
  a.counters = sc.counters;
  a.strategy = strategy;
  if (strategy == UNIFY_HYBRID) {
    a.queue = sc.queues + sc.cap_nq;
    a.qcount_idx = CNT_QC;
    a.take_idx = CNT_TAKE_C;
    a.efl = p.ef > p.k ? p.ef : p.k;
  } else {
    a.queue = sc.queues + 2 * sc.cap_nq;
    a.qcount_idx = CNT_QB;
    a.take_idx = CNT_TAKE_B;
    a.efl = p.ef_post > p.k ? p.ef_post : p.k;
  }
  a.k = p.k;
  a.m = p.m;
  a.cand_cap = p.cand_cap;
  a.ann_cap = a.efl;
  a.vis_log2 = p.vis_log2;
  a.max_exp = p.max_exp;
  a.warp_bytes = warp_mem_bytes(a.cand_cap, a.ann_cap, a.vis_log2);
  a.o = o;
  const int wpb = p.warps_per_block;
  const int ch = (a.dp4 + 31) / 32;
  if (ch <= 1) return launch_graph_t<1, 16>(a, wpb, ix.num_sms, st);
  if (ch <= 2) return launch_graph_t<2, 16>(a, wpb, ix.num_sms, st);
  if (ch <= 4) return launch_graph_t<4, 8>(a, wpb, ix.num_sms, st);
  return launch_graph_t<8, 8>(a, wpb, ix.num_sms, st);
}

}  // namespace unify
