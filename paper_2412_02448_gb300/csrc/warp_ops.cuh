// Warp-level helpers shared by the search kernel and the tensor-core scan:
// writing a result row, grouped distance evaluation and top-k insertion.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace unify {

// Writes keys[0, cnt) as result row qi (ids and distances), padded with -1 / +inf.
__device__ __forceinline__ void write_row(const uint64_t* keys, int cnt, int k, int64_t qi, const Outputs& o) {
  const int lane = lane_id();
  for (int t = lane; t < k; t += 32) {
    const bool v = t < cnt;
    const uint64_t key = v ? keys[t] : kKeyMax;
    o.ids[qi * k + t] = v ? (int64_t)key_id(key) : (int64_t)-1;
    o.dist[qi * k + t] = v ? key_dist(key) : __int_as_float(0x7f800000);
  }
}

// Distances of the candidates held by the lanes (cid >= 0), G at a time, from
// rows of `rows` (row_bytes each) in storage format T (scale: FP8 scales or null).
// All G row loads of a group are issued before any of them is used (slots past
// the last candidate reload the last candidate's row and are discarded), so a
// group costs one memory latency, not G.
template <class T, int CH, int G>
__device__ __forceinline__ float batch_dist(const float4 (&q)[CH], int cid, const unsigned char* rows,
                                            int row_bytes, const float* scale, int dp4, int* clist) {
  const int lane = lane_id();
  const unsigned vm = __ballot_sync(kFull, cid >= 0);
  const int nv = __popc(vm);
  const int my = __popc(vm & lanemask_lt());
  if (cid >= 0) clist[my] = cid;
  __syncwarp();
  constexpr int SH = (G == 32) ? 0 : (G == 16) ? 1 : (G == 8) ? 2 : (G == 4) ? 3 : 4;  // log2(32 / G)
  float result = 0.f;
  for (int g = 0; g * G < nv; ++g) {
    int ids[G];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int c = g * G + u;
      ids[u] = clist[c < nv ? c : nv - 1];
    }
    Held<T> x[G][CH];
    float sc[G];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const unsigned char* row = rows + (int64_t)ids[u] * row_bytes;
      sc[u] = scale ? __ldg(scale + ids[u]) : 1.f;
#pragma unroll
      for (int t = 0; t < CH; ++t) {
        const int c = lane + 32 * t;
        if constexpr (T::kHoldRaw) x[u][t] = c < dp4 ? T::load_raw(row, c) : T::zero_raw();
        else x[u][t] = c < dp4 ? T::load(row, c, sc[u]) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    float part[G];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      float s = 0.f;
#pragma unroll
      for (int t = 0; t < CH; ++t) {
        // chunks past the row are zero in q and x alike, so their difference is zero
        const float4 e = diff4<T>(q[t], unhold<T>(x[u][t]), sc[u]);
        s = fmaf(e.x, e.x, s);
        s = fmaf(e.y, e.y, s);
        s = fmaf(e.z, e.z, s);
        s = fmaf(e.w, e.w, s);
      }
      part[u] = (g * G + u < nv) ? s : 0.f;
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

// Keeps the k smallest keys: merges the lanes' keys that beat the current k-th.
__device__ __forceinline__ int topk_offer(uint64_t* topk, int nt, int k, uint64_t key, int* R) {
  const uint64_t thr = (nt >= k) ? topk[k - 1] : kKeyMax;
  const bool pass = key < thr;
  const unsigned bal = __ballot_sync(kFull, pass);
  if (bal == 0) return nt;
  uint64_t s = warp_sort_kept(pass ? key : kKeyMax, bal);
  int r0;
  bool dropped;
  return warp_merge(topk, nullptr, nt, k, s, __popc(bal), R, &r0, &dropped);
}

}  // namespace unify
