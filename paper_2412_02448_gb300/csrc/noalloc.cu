// unify_search_noalloc: the search of unify_search without any device allocation.
//
// Some callers cannot call cudaMalloc at search time: code that runs under a
// fixed device-memory budget, latency-critical serving loops that cannot accept
// cudaMalloc's implicit device-wide synchronisation or its failure, and hosts
// that must not allocate at all once they have started (for instance inside a
// capture they control). unify_search grows the index's scratch buffers on
// demand; this entry point instead takes its scratch (range bounds, masks,
// strategy queues, scan work items, partial top-k lists, work counters) from one
// file-scope device array of fixed size, so a call allocates nothing.
//
// Limits: at most kNoAllocMaxQueries queries and k <= kNoAllocMaxK per call.
// The array (see kNoAllocBytes) lives on every GPU that loads this library until
// the process exits. Every call shares it and it keeps the previous call's
// contents: the work counters are cleared on the stream at the start of each
// call, and two calls whose work overlaps on the GPU (other streams, other
// threads, other indexes on the same device) race on it.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace unify {
namespace {

constexpr int64_t kNoAllocMaxQueries = 1024;
constexpr int kNoAllocMaxK = 16;
constexpr int kNoAllocMaxDevices = 64;

constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kI32 = al256(kNoAllocMaxQueries * sizeof(int32_t));
constexpr size_t kOffPa = 0;
constexpr size_t kOffPb = kOffPa + kI32;
constexpr size_t kOffMask = kOffPb + kI32;
constexpr size_t kOffStrat = kOffMask + kI32;
constexpr size_t kOffNblk = kOffStrat + kI32;
constexpr size_t kOffQbase = kOffNblk + kI32;
constexpr size_t kOffDone = kOffQbase + kI32;
constexpr size_t kOffQueues = kOffDone + kI32;
constexpr size_t kOffItems = kOffQueues + al256(3 * kNoAllocMaxQueries * sizeof(int32_t));
constexpr size_t kOffPart = kOffItems + al256(kNoAllocMaxQueries * kMaxScanBlocks * sizeof(int2));
constexpr size_t kOffCounters =
    kOffPart + al256((size_t)kNoAllocMaxQueries * kMaxScanBlocks * kNoAllocMaxK * sizeof(uint64_t));
constexpr size_t kNoAllocBytes = kOffCounters + al256(kNumCounters * sizeof(int32_t));  // about 8.6 MiB

}  // namespace

// The shared scratch. In host code this name is only a stand-in for the symbol:
// its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

std::mutex g_mu;
unsigned char* g_addr[kNoAllocMaxDevices] = {};

int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

// Device address of the scratch on `device` (which must be current). The first
// call on a device looks it up once.
int scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kNoAllocMaxDevices) return fail(UNIFY_E_LIMIT, "unify_search_noalloc: device id above 63");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(UNIFY_E_CUDA, std::string("unify_search_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[device] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[device];
  return UNIFY_OK;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(UNIFY_E_CUDA, std::string("unify_search_noalloc: ") + where + ": " + cudaGetErrorString(e));
}

}  // namespace
}  // namespace unify

using namespace unify;

extern "C" int unify_search_noalloc(unify_index_t* idx, const float* q, const int64_t* lo, const int64_t* hi,
                                    int64_t nq, int k, int ef, unify_strategy_t strategy,
                                    const unify_params_t* p, int64_t* out_ids, float* out_dist,
                                    int32_t* out_count, uint32_t* out_status, void* stream) {
  if (!idx) return fail(UNIFY_E_ARG, "unify_search_noalloc: null index");
  if (nq < 0) return fail(UNIFY_E_ARG, "unify_search_noalloc: nq < 0");
  if (nq > kNoAllocMaxQueries)
    return fail(UNIFY_E_LIMIT, "unify_search_noalloc: nq exceeds the fixed scratch limit of 1024 queries per call");
  if (k < 1 || k > kNoAllocMaxK)
    return fail(UNIFY_E_LIMIT, "unify_search_noalloc: k must be in [1, 16] (fixed scratch limit)");
  const int st_code = (int)strategy;
  if (st_code < -1 || st_code > 2) return fail(UNIFY_E_ARG, "unify_search_noalloc: bad strategy");
  Params prm;
  int rc = resolve_search_params(idx->ix, p, k, ef, prm);
  if (rc != UNIFY_OK) return rc;
  if (rerank_count(prm) > kNoAllocMaxK)
    return fail(UNIFY_E_LIMIT, "unify_search_noalloc: rerank_mult * k must be <= 16 (fixed scratch limit)");
  if (nq == 0) return UNIFY_OK;
  if (!q || !lo || !hi || !out_ids || !out_dist || !out_count)
    return fail(UNIFY_E_ARG, "unify_search_noalloc: null query or output pointer");
  cudaStream_t st = (cudaStream_t)stream;
  DeviceGuard guard(idx->ix.device);
  unsigned char* base = nullptr;
  rc = scratch_address(idx->ix.device, &base);
  if (rc != UNIFY_OK) return rc;
  Scratch sc;
  sc.cap_nq = kNoAllocMaxQueries;
  sc.cap_k = kNoAllocMaxK;
  sc.pa = reinterpret_cast<int32_t*>(base + kOffPa);
  sc.pb = reinterpret_cast<int32_t*>(base + kOffPb);
  sc.mask = reinterpret_cast<uint32_t*>(base + kOffMask);
  sc.strat = reinterpret_cast<int32_t*>(base + kOffStrat);
  sc.nblk = reinterpret_cast<int32_t*>(base + kOffNblk);
  sc.qbase = reinterpret_cast<int32_t*>(base + kOffQbase);
  sc.done = reinterpret_cast<int32_t*>(base + kOffDone);
  sc.queues = reinterpret_cast<int32_t*>(base + kOffQueues);
  sc.items = reinterpret_cast<int2*>(base + kOffItems);
  sc.part = reinterpret_cast<uint64_t*>(base + kOffPart);
  sc.counters = reinterpret_cast<int32_t*>(base + kOffCounters);
  cudaError_t e = cudaMemsetAsync(sc.counters, 0, kNumCounters * sizeof(int32_t), st);
  if (e != cudaSuccess) return cuda_fail(e, "counter reset");
  Outputs o{out_ids, out_dist, out_count, out_status, nullptr};
  e = launch_route(idx->ix, sc, lo, hi, nq, prm.tau_a, prm.tau_b, st_code, prm.scan_rows, 1, sc.pa, sc.pb,
                   sc.mask, sc.strat, &o, st);
  if (e != cudaSuccess) return cuda_fail(e, "route kernel");
  e = launch_batch(idx->ix, sc, q, prm, o, st);
  if (e != cudaSuccess) return cuda_fail(e, "search kernel");
  return UNIFY_OK;
}
