// Internal declarations of the CUDA search library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/unify.h"

namespace unify {

constexpr int kMaxS = 32;      // segments (one bit each in a 32-bit mask)
constexpr int kMaxK = 256;     // results per query
constexpr int kMaxCand = 4096; // candidate buffer entries per query
constexpr int kMaxScanBlocks = 64;  // scan work items per pre-filter query

// Device-resident index. Arrays marked (n) are indexed by object id unless noted.
struct DeviceIndex {
  int device = 0;
  int64_t n = 0, n_upper = 0;
  int d = 0, dp = 0;           // dimension and padded row stride (multiple of 4 floats)
  int S = 0, M = 0, W = 0;     // segments, chunk width, bitmap words per row
  int max_level = 0, entry_global = 0;
  int64_t h_seg_bounds[kMaxS + 1];
  int32_t h_seg_start[kMaxS + 1];  // first attribute-order position of each segment
  // device memory
  float* vec = nullptr;         // (n, dp) float32 by id
  float* vec_sorted = nullptr;  // (n, dp) float32 in attribute order
  int32_t* sorted_ids = nullptr;   // attribute order (ties by id)
  int64_t* sorted_attr = nullptr;  // attribute values in attribute order
  int32_t* pos = nullptr;       // (n) position of each id in attribute order
  int32_t* upper_base = nullptr;
  int32_t* adj0 = nullptr;      // (n, S, M), -1 padded
  uint32_t* gmask0 = nullptr;   // (n, W)
  int32_t* adjU = nullptr;      // (n_upper, S, M)
  uint32_t* gmaskU = nullptr;   // (n_upper, W)
  int64_t* seg_bounds = nullptr;  // (S+1)
  int32_t* seg_start = nullptr;   // (S+1)
  // reduced-precision copies (rows of dp/4 chunks of 4 elements): by id and in attribute order
  unsigned char* vt_bf16 = nullptr;   // bfloat16, 8 bytes per chunk
  unsigned char* vts_bf16 = nullptr;
  unsigned char* vt_fp8 = nullptr;    // E4M3 codes of x / scale, 4 bytes per chunk
  unsigned char* vts_fp8 = nullptr;
  float* scale_fp8 = nullptr;         // per-vector scale max|x| / 448 (by id)
  float* scale_fp8_sorted = nullptr;  // the same in attribute order
  float* xn_bf16_sorted = nullptr;    // squared norms of the bfloat16 rows, attribute order
  float* xn_f32_sorted = nullptr;     // squared norms of the float32 rows, attribute order
  float* xn_fp8_sorted = nullptr;     // squared norms of the decoded FP8 rows, attribute order
  int num_sms = 0;
};

// Per-index scratch, grown on demand.
struct Scratch {
  int64_t cap_nq = 0;
  int cap_k = 0;
  int32_t* pa = nullptr;
  int32_t* pb = nullptr;
  uint32_t* mask = nullptr;
  int32_t* strat = nullptr;
  int32_t* nblk = nullptr;     // scan work items of each pre-filter query
  int32_t* qbase = nullptr;    // index of its first work item
  int32_t* done = nullptr;     // completed scan work items of each pre-filter query
  int32_t* queues = nullptr;   // 3 x cap_nq: query ids per strategy (A, C, B)
  int2* items = nullptr;       // cap_nq * kMaxScanBlocks scan work items (query, block)
  uint64_t* part = nullptr;    // cap_nq * kMaxScanBlocks * cap_k partial top-k keys
  int32_t* counters = nullptr; // kNumCounters ints, zeroed per call
  // tensor-core pre-filter scan: queries by position (their queue order), tiles of
  // 128 slots per span of the attribute order, per-query bound and candidate list
  int32_t* tc_aq = nullptr;      // pre-filter query ids by position
  float* tc_aqn = nullptr;       // squared norms of their vectors in the scan's format
  float* tc_aqs = nullptr;       // their FP8 scales
  void* tc_qb = nullptr;         // their vectors in the scan's format, tc_rows x tc_qrow_bytes
  void* tc_qg = nullptr;         // the rows gathered per tile slot, tc_slots x tc_qrow_bytes
  int32_t* tc_slotpos = nullptr;  // per tile slot: query position (-1: none), tc_slots
  int32_t* tc_tiles = nullptr;   // per tile: span, then unit offsets (2 x tc_slots / 128 + 1)
  int32_t* tc_spans = nullptr;   // per span: count, fill cursor, first tile (3 x tc_spans_cap + 1)
  unsigned* tc_gmin = nullptr;   // per query: 128 group minima (float bits)
  uint64_t* tc_qlist = nullptr;  // per query: kTcQCap candidate keys
  int32_t* tc_qcnt = nullptr;    // per query: candidates found
  unsigned long long* tc_thr = nullptr;   // per query: bound key
  unsigned long long* tc_sumy = nullptr;  // total in-range rows of the pre-filter queries
  uint64_t* tc_stage = nullptr;  // per scan CTA and epilogue thread: kTcStage keys of the current unit
  int tc_stage_sms = 0;
  int64_t tc_rows = 0;        // query positions (a multiple of 128)
  int64_t tc_slots = 0;       // tile slots: 16 per query position
  int64_t tc_spans_cap = 0;   // spans: ceil(n / 4096) + 1
  size_t tc_qrow_bytes = 0;
  // host-buffer staging
  int64_t stage_nq = 0;
  int stage_k = 0, stage_d = 0;
  float* s_q = nullptr;
  int64_t* s_lo = nullptr;
  int64_t* s_hi = nullptr;
  int64_t* s_ids = nullptr;
  float* s_dist = nullptr;
  int32_t* s_count = nullptr;
  uint32_t* s_status = nullptr;
};

constexpr int kTcQueryTile = 128;   // pre-filter queries per tensor-core tile
constexpr int kTcRowPad = 256;      // zero entries past row n of the attribute-ordered norms, scales
                                    // and ids (the tensor-core scan copies whole 256-row blocks)
constexpr int kTcQCap = 512;        // candidate keys per query below its bound
constexpr int kTcStage = 96;        // keys an epilogue thread stages per work unit
constexpr int kTcEpiThreads = 256;  // epilogue threads of a tensor-core scan CTA
constexpr int kTcPairsPerQuery = 8;  // (query, span) pairs the scratch holds per query position

// counters[] layout
enum {
  CNT_QA = 0, CNT_QC = 1, CNT_QB = 2,  // queue lengths
  CNT_ITEMS = 3,                       // scan work items
  CNT_TAKE = 4,                        // head of the combined work queue
  CNT_T0 = 8,                          // counters[8..9]: 64-bit global-timer origin of the search kernel
  CNT_TC_ERR = 10,                     // the tensor-core scan timed out on a wait
  CNT_TC_UNITS = 11,                   // work units of the tensor-core scan
  CNT_TC_TAKE = 12,                    // next work unit to claim (tensor-core scan pass)
  CNT_TC_TAKE_B = 13,                  // next work unit to claim (tensor-core bounding pass)
  CNT_TC_L = 14,                       // span length of the tensor-core scan's tiles (rows)
  CNT_TC_TILES = 15,                   // tiles of the tensor-core scan
  kNumCounters = 16
};

struct Params {
  int k, ef, m, ef_post, cand_cap, vis_log2, max_exp, warps_per_block, scan_rows, rerank_mult, reg_budget, tc_scan, selection;
  int64_t tau_a, tau_b;
  unify_dtype_t dtype;
};

// Conjunctive predicate on a second attribute: attr2 holds one value per object
// (by id); query i also requires lo2[i] <= attr2[id] <= hi2[i]. attr2 == nullptr:
// no second attribute.
struct Conj {
  const int64_t* attr2 = nullptr;
  const int64_t* lo2 = nullptr;
  const int64_t* hi2 = nullptr;
};

struct Outputs {
  int64_t* ids;
  float* dist;
  int32_t* count;
  uint32_t* status;
  int32_t* counters;
};

// launchers (return cudaGetLastError())
cudaError_t launch_route(const DeviceIndex& ix, const Scratch& sc, const int64_t* lo, const int64_t* hi,
                         int64_t nq, int64_t tau_a, int64_t tau_b, int forced, int scan_rows,
                         int build_queues, int32_t* out_pa, int32_t* out_pb, uint32_t* out_mask,
                         int32_t* out_strat, const Outputs* outs, cudaStream_t st);
cudaError_t launch_batch(const DeviceIndex& ix, const Scratch& sc, const float* q, const Params& p,
                         const Outputs& o, cudaStream_t st, bool skip_scan = false, const Conj* cj = nullptr);
bool tc_scan_available(const DeviceIndex& ix, const Params& p);
size_t tc_query_row_bytes(int d);  // bytes of one query row of the tensor-core scan, any format
cudaError_t launch_tcscan(const DeviceIndex& ix, const Scratch& sc, const float* q, int64_t nq, const Params& p,
                          const Outputs& o, cudaStream_t st);
int batch_smem_per_warp(const Params& p);
int rerank_count(const Params& p);  // candidates re-ranked in FP32 (0 for FP32 storage)

void set_error(const std::string& msg);
int resolve_search_params(const DeviceIndex& ix, const unify_params_t* up, int k, int ef, Params& p);
void free_scratch(Scratch& sc);

// Makes `dev` current for the lifetime of the guard.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace unify

namespace unify {
// Optional per-phase CUDA-event timing of searches (route, scan, hybrid, post).
constexpr int kPhases = 4;  // 0 route, 1 search kernel, 2 and 3 unused
struct Timing {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> rec[kPhases];
};
}  // namespace unify

struct unify_index {
  unify::DeviceIndex ix;
  unify::Scratch sc;
  unify::Timing tm;
  int live_plans = 0;  // captured graphs that hold pointers into sc
};

struct unify_plan {
  unify_index* idx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};
