// Strategy A, pre-filtering (Section 4.2): an exhaustive scan of the in-range
// objects, which are the positions [pa, pb) of the attribute order (the bottom
// layer of the fused skip list), keeping the k nearest by (distance, id).
//
// GB300 layout: the vectors are also stored in attribute order (vec_sorted), so a
// query's in-range rows are one contiguous block of HBM. A warp computes 32 row
// distances per step with coalesced 16-byte loads (32 lanes x float4 = one
// 128-float row per instruction) and a transposed shuffle reduction that leaves
// row r's distance in lane r. Long ranges are split into up to 64 work items
// whose partial top-k lists are merged by a second kernel.
#include "common.cuh"
#include "internal.h"

namespace unify {

struct ScanArgs {
  const float* vec_sorted;
  const int32_t* sorted_ids;
  int dp4;  // float4 chunks per row
  int d;
  const float* q;
  const int32_t* pa;
  const int32_t* pb;
  const int32_t* nblk;
  const int32_t* qbase;
  const int32_t* queues;  // queue A = queues[0 .. counters[CNT_QA])
  const int2* items;
  uint64_t* part;
  int32_t* counters;
  int k;
  int warps;
  Outputs o;
};

__device__ __forceinline__ void write_result(const uint64_t* keys, int cnt, int k, int64_t qi,
                                             const Outputs& o) {
  const int lane = lane_id();
  for (int t = lane; t < k; t += 32) {
    bool v = t < cnt;
    uint64_t key = v ? keys[t] : kKeyMax;
    o.ids[qi * k + t] = v ? (int64_t)key_id(key) : (int64_t)-1;
    o.dist[qi * k + t] = v ? key_dist(key) : __int_as_float(0x7f800000);
  }
  if (lane == 0) {
    o.count[qi] = cnt;
    if (o.status) o.status[qi] = 0u;
  }
}

// Keeps the k smallest keys: merges the lanes' keys that beat the current k-th.
__device__ __forceinline__ int topk_offer(uint64_t* topk, int nt, int k, uint64_t key, int* R) {
  const uint64_t thr = (nt >= k) ? topk[k - 1] : kKeyMax;
  const bool pass = key < thr;
  const unsigned bal = __ballot_sync(kFull, pass);
  if (bal == 0) return nt;
  uint64_t s = warp_sort_asc(pass ? key : kKeyMax);
  int r0;
  bool dropped;
  return warp_merge(topk, nullptr, nt, k, s, __popc(bal), R, &r0, &dropped);
}

template <int CH>
__global__ void __launch_bounds__(128) scan_kernel(ScanArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  uint64_t* topk = reinterpret_cast<uint64_t*>(smem_raw) + (size_t)warp * a.k;
  int* R = reinterpret_cast<int*>(reinterpret_cast<uint64_t*>(smem_raw) + (size_t)a.warps * a.k) + warp * 32;
  const int n_items = a.counters[CNT_ITEMS];
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(&a.counters[CNT_TAKE_ITEMS], 1);
    it = __shfl_sync(kFull, it, 0);
    if (it >= n_items) break;
    const int2 item = a.items[it];
    const int qi = item.x, b = item.y;
    const int pa = a.pa[qi], pb = a.pb[qi], nb = a.nblk[qi];
    const int Y = pb - pa;
    const int rpb = (Y + nb - 1) / (nb > 0 ? nb : 1);
    const int r0 = pa + b * rpb;
    const int r1 = min(pb, r0 + rpb);
    float4 q[CH];
    load_query<CH>(q, a.q + (int64_t)qi * a.d, a.d);
    int nt = 0;
    for (int base = r0; base < r1; base += 32) {
      float part[32];
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        const int row = base + r;
        part[r] = (row < r1) ? l2_partial<CH>(q, a.vec_sorted + (int64_t)row * a.dp4 * 4, a.dp4) : 0.f;
      }
      const float dist = warp_transpose_reduce<32>(part);
      const int row = base + lane;
      uint64_t key = kKeyMax;
      if (row < r1) key = make_key(dist, __ldg(a.sorted_ids + row));
      nt = topk_offer(topk, nt, a.k, key, R);
    }
    if (nb == 1) {
      write_result(topk, nt, a.k, qi, a.o);
    } else {
      uint64_t* dst = a.part + (int64_t)it * a.k;
      for (int t = lane; t < a.k; t += 32) dst[t] = t < nt ? topk[t] : kKeyMax;
    }
    __syncwarp();
  }
}

// Merges the partial lists of the pre-filter queries that were split.
__global__ void __launch_bounds__(128) scan_merge_kernel(ScanArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  uint64_t* topk = reinterpret_cast<uint64_t*>(smem_raw) + (size_t)warp * a.k;
  int* R = reinterpret_cast<int*>(reinterpret_cast<uint64_t*>(smem_raw) + (size_t)a.warps * a.k) + warp * 32;
  const int nA = a.counters[CNT_QA];
  for (;;) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(&a.counters[CNT_TAKE_MERGE], 1);
    idx = __shfl_sync(kFull, idx, 0);
    if (idx >= nA) break;
    const int qi = a.queues[idx];
    const int nb = a.nblk[qi];
    if (nb <= 1) continue;
    const uint64_t* src = a.part + (int64_t)a.qbase[qi] * a.k;
    const int total = nb * a.k;
    int nt = 0;
    for (int off = 0; off < total; off += 32) {
      const uint64_t key = (off + lane < total) ? src[off + lane] : kKeyMax;
      nt = topk_offer(topk, nt, a.k, key, R);
    }
    const int Y = a.pb[qi] - a.pa[qi];
    write_result(topk, min(nt, min(Y, a.k)), a.k, qi, a.o);
    __syncwarp();
  }
}

cudaError_t launch_scan(const DeviceIndex& ix, const Scratch& sc, const float* q, int64_t nq,
                        const Params& p, const Outputs& o, cudaStream_t st) {
  (void)nq;
  ScanArgs a;
  a.vec_sorted = ix.vec_sorted;
  a.sorted_ids = ix.sorted_ids;
  a.dp4 = ix.dp / 4;
  a.d = ix.d;
  a.q = q;
  a.pa = sc.pa;
  a.pb = sc.pb;
  a.nblk = sc.nblk;
  a.qbase = sc.qbase;
  a.queues = sc.queues;
  a.items = sc.items;
  a.part = sc.part;
  a.counters = sc.counters;
  a.k = p.k;
  a.warps = 4;
  a.o = o;
  const int threads = 32 * a.warps;
  const size_t smem = (size_t)a.warps * (a.k * 8 + 32 * 4);
  const int ch = (a.dp4 + 31) / 32;
  int per_sm = 0;
  cudaError_t e = cudaSuccess;
#define UNIFY_SCAN_CASE(C)                                                                   \
  case C:                                                                                    \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_kernel<C>, threads, smem); \
    if (e != cudaSuccess) return e;                                                          \
    scan_kernel<C><<<ix.num_sms * (per_sm > 0 ? per_sm : 1), threads, smem, st>>>(a);         \
    break;
  switch (ch <= 1 ? 1 : ch <= 2 ? 2 : ch <= 4 ? 4 : 8) {
    UNIFY_SCAN_CASE(1)
    UNIFY_SCAN_CASE(2)
    UNIFY_SCAN_CASE(4)
    UNIFY_SCAN_CASE(8)
  }
#undef UNIFY_SCAN_CASE
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  scan_merge_kernel<<<ix.num_sms * 4, threads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace unify
