// Range resolution, segment mask and range-aware strategy selection
// (Section 4.2: Strategy A's skip-list descent lands on the first in-range object;
// Algorithm 7: the segments that intersect [l, h]; range-aware selection:
// A if Y <= tau_A, B if Y >= tau_B, otherwise C).
//
// The skip list's bottom layer is the attribute order, so the descent to the first
// object with attribute >= lo is a lower_bound on the attribute-sorted values, and
// the in-range objects are the positions [pa, pb) of that order.
#include "common.cuh"
#include "internal.h"

namespace unify {

__device__ __forceinline__ int64_t lower_bound_i64(const int64_t* a, int64_t n, int64_t x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int64_t upper_bound_i64(const int64_t* a, int64_t n, int64_t x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

struct RouteArgs {
  const int64_t* sorted_attr;
  int64_t n;
  int S;
  const int64_t* lo;
  const int64_t* hi;
  int64_t nq;
  int64_t tau_a, tau_b;
  int forced;        // -1: range-aware, else the strategy for every query
  int scan_rows;
  int build_queues;
  int32_t* pa;
  int32_t* pb;
  uint32_t* mask;
  int32_t* strat;
  int32_t* nblk;
  int32_t* qbase;
  int32_t* done;
  int32_t* queues;
  int64_t cap_nq;
  int2* items;
  int32_t* counters;
  int32_t* out_count;     // may be null (set 0 for empty pre-filter queries handled here)
  int32_t* out_counters;  // may be null
};

__global__ void route_kernel(RouteArgs a, const int64_t* __restrict__ seg_bounds,
                             const int32_t* __restrict__ seg_start) {
  __shared__ int64_t b[kMaxS + 1];
  __shared__ int32_t ss[kMaxS + 1];
  for (int j = threadIdx.x; j <= a.S; j += blockDim.x) {
    b[j] = seg_bounds[j];
    ss[j] = seg_start[j];
  }
  __syncthreads();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.nq) return;
  const int64_t lo = a.lo[i], hi = a.hi[i];
  int64_t p0 = lower_bound_i64(a.sorted_attr, a.n, lo);
  int64_t p1 = upper_bound_i64(a.sorted_attr, a.n, hi);
  if (p1 < p0) p1 = p0;
  uint32_t m = 0;
  if (lo <= hi) {
    for (int j = 0; j < a.S; ++j) {
      bool nonempty = ss[j + 1] > ss[j];
      bool lower_ok = (j == 0) || b[j] <= hi;
      bool upper_ok = (j == a.S - 1) || lo < b[j + 1];
      if (nonempty && lower_ok && upper_ok) m |= 1u << j;
    }
  }
  const int64_t Y = p1 - p0;
  int st = a.forced;
  if (st < 0) st = (Y <= a.tau_a) ? UNIFY_PRE : ((Y >= a.tau_b) ? UNIFY_POST : UNIFY_HYBRID);
  if (a.pa) a.pa[i] = (int32_t)p0;
  if (a.pb) a.pb[i] = (int32_t)p1;
  if (a.mask) a.mask[i] = m;
  if (a.strat) a.strat[i] = st;
  if (!a.build_queues) return;
  const int qi = (st == UNIFY_PRE) ? 0 : (st == UNIFY_HYBRID ? 1 : 2);
  int slot = atomicAdd(&a.counters[CNT_QA + qi], 1);
  a.queues[qi * a.cap_nq + slot] = (int32_t)i;
  if (st == UNIFY_PRE) {
    int64_t nb = (Y + a.scan_rows - 1) / a.scan_rows;
    if (nb < 1) nb = 1;
    if (nb > kMaxScanBlocks) nb = kMaxScanBlocks;
    int base = atomicAdd(&a.counters[CNT_ITEMS], (int)nb);
    a.nblk[i] = (int)nb;
    a.qbase[i] = base;
    a.done[i] = 0;
    for (int t = 0; t < nb; ++t) a.items[base + t] = make_int2((int)i, t);
    if (a.out_counters) {
      a.out_counters[4 * i] = (int32_t)Y;
      a.out_counters[4 * i + 1] = 0;
      a.out_counters[4 * i + 2] = 0x7fffffff;  // earliest item start (atomicMin)
      a.out_counters[4 * i + 3] = 0;           // latest item end (atomicMax)
    }
  }
}

cudaError_t launch_route(const DeviceIndex& ix, const Scratch& sc, const int64_t* lo, const int64_t* hi,
                         int64_t nq, int64_t tau_a, int64_t tau_b, int forced, int scan_rows,
                         int build_queues, int32_t* out_pa, int32_t* out_pb, uint32_t* out_mask,
                         int32_t* out_strat, const Outputs* outs, cudaStream_t st) {
  RouteArgs a;
  a.sorted_attr = ix.sorted_attr;
  a.n = ix.n;
  a.S = ix.S;
  a.lo = lo;
  a.hi = hi;
  a.nq = nq;
  a.tau_a = tau_a;
  a.tau_b = tau_b;
  a.forced = forced;
  a.scan_rows = scan_rows > 0 ? scan_rows : 8192;
  a.build_queues = build_queues;
  a.pa = out_pa;
  a.pb = out_pb;
  a.mask = out_mask;
  a.strat = out_strat;
  a.nblk = sc.nblk;
  a.qbase = sc.qbase;
  a.done = sc.done;
  a.queues = sc.queues;
  a.cap_nq = sc.cap_nq;
  a.items = sc.items;
  a.counters = sc.counters;
  a.out_count = outs ? outs->count : nullptr;
  a.out_counters = outs ? outs->counters : nullptr;
  if (nq == 0) return cudaSuccess;
  const int tpb = 256;
  int64_t blocks = (nq + tpb - 1) / tpb;
  route_kernel<<<(unsigned)blocks, tpb, 0, st>>>(a, ix.seg_bounds, ix.seg_start);
  return cudaGetLastError();
}

}  // namespace unify
