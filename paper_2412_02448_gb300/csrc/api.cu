// C ABI entry points: argument checks, parameters, scratch, and the launch
// sequence route -> pre-filter scan (+ merge) -> hybrid search -> post search.
#include <nvtx3/nvToolsExt.h>

#include <cstring>
#include <new>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace unify {

namespace {
thread_local std::string g_last_error;

// NVTX range for one phase of a search (visible in a profiler's timeline; the
// calls do nothing when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(e == cudaErrorMemoryAllocation ? UNIFY_E_NOMEM : UNIFY_E_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

template <typename T>
void release(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_core(Scratch& sc) {
  release(sc.pa);
  release(sc.pb);
  release(sc.mask);
  release(sc.strat);
  release(sc.nblk);
  release(sc.qbase);
  release(sc.done);
  release(sc.queues);
  release(sc.items);
  release(sc.part);
  release(sc.counters);
  sc.cap_nq = 0;
  sc.cap_k = 0;
}

void free_tc(Scratch& sc) {
  release(sc.tc_aq);
  release(sc.tc_aqn);
  release(sc.tc_aqs);
  if (sc.tc_qb) cudaFree(sc.tc_qb);
  sc.tc_qb = nullptr;
  if (sc.tc_qg) cudaFree(sc.tc_qg);
  sc.tc_qg = nullptr;
  release(sc.tc_slotpos);
  release(sc.tc_tiles);
  release(sc.tc_spans);
  release(sc.tc_gmin);
  release(sc.tc_qlist);
  release(sc.tc_qcnt);
  release(sc.tc_thr);
  release(sc.tc_sumy);
  release(sc.tc_stage);
  sc.tc_stage_sms = 0;
  sc.tc_rows = 0;
  sc.tc_slots = 0;
  sc.tc_spans_cap = 0;
  sc.tc_qrow_bytes = 0;
}

void free_stage(Scratch& sc) {
  release(sc.s_q);
  release(sc.s_lo);
  release(sc.s_hi);
  release(sc.s_ids);
  release(sc.s_dist);
  release(sc.s_count);
  release(sc.s_status);
  sc.stage_nq = 0;
  sc.stage_k = 0;
  sc.stage_d = 0;
}

template <typename T>
cudaError_t alloc(T*& p, size_t elems) {
  return cudaMalloc(reinterpret_cast<void**>(&p), (elems > 0 ? elems : 1) * sizeof(T));
}

// Grows the scratch to hold nq queries with k results (device allocation).
cudaError_t ensure_scratch(Scratch& sc, int64_t nq, int k) {
  if (sc.counters && nq <= sc.cap_nq && k <= sc.cap_k) return cudaSuccess;
  int64_t cap = nq > sc.cap_nq ? nq : sc.cap_nq;
  if (cap < 256) cap = 256;
  int kc = k > sc.cap_k ? k : sc.cap_k;
  if (kc < 16) kc = 16;
  free_core(sc);
  cudaError_t e = alloc(sc.pa, cap);
  if (e == cudaSuccess) e = alloc(sc.pb, cap);
  if (e == cudaSuccess) e = alloc(sc.mask, cap);
  if (e == cudaSuccess) e = alloc(sc.strat, cap);
  if (e == cudaSuccess) e = alloc(sc.nblk, cap);
  if (e == cudaSuccess) e = alloc(sc.qbase, cap);
  if (e == cudaSuccess) e = alloc(sc.done, cap);
  if (e == cudaSuccess) e = alloc(sc.queues, 3 * cap);
  if (e == cudaSuccess) e = alloc(sc.items, cap * kMaxScanBlocks);
  if (e == cudaSuccess) e = alloc(sc.part, (size_t)cap * kMaxScanBlocks * kc);
  if (e == cudaSuccess) e = alloc(sc.counters, kNumCounters);
  if (e != cudaSuccess) {
    free_core(sc);
    return e;
  }
  sc.cap_nq = cap;
  sc.cap_k = kc;
  return cudaSuccess;
}

// Tensor-core scan buffers for nq queries of d columns over n rows, allocated only
// when a search uses that scan: per query position its operand row, 16 tile slots
// (each with a gathered operand row), 128 group minima and a list of kTcQCap keys.
bool tc_scratch_fits(const Scratch& sc, int64_t nq, int d, int64_t n, int sms) {
  return sc.tc_qlist && nq <= sc.tc_rows && tc_query_row_bytes(d) <= sc.tc_qrow_bytes &&
         (n + 4095) / 4096 + 1 <= sc.tc_spans_cap && sms <= sc.tc_stage_sms;
}

cudaError_t ensure_tc_scratch(Scratch& sc, int64_t nq, int d, int64_t n, int sms) {
  if (tc_scratch_fits(sc, nq, d, n, sms)) return cudaSuccess;
  const size_t qrow = tc_query_row_bytes(d);  // query rows of any of the scan's formats, K padded
  int64_t cap = nq > sc.tc_rows ? nq : sc.tc_rows;
  const int64_t rows = ((cap + kTcQueryTile - 1) / kTcQueryTile) * kTcQueryTile;
  const int64_t slots = 2 * kTcPairsPerQuery * rows;  // a multiple of 128
  const int64_t spans = (n + 4095) / 4096 + 1;
  free_tc(sc);
  cudaError_t e = alloc(sc.tc_aq, rows);
  if (e == cudaSuccess) e = alloc(sc.tc_aqn, rows);
  if (e == cudaSuccess) e = alloc(sc.tc_aqs, rows);
  if (e == cudaSuccess) e = cudaMalloc(&sc.tc_qb, (size_t)rows * qrow);
  if (e == cudaSuccess) e = cudaMalloc(&sc.tc_qg, (size_t)slots * qrow);
  if (e == cudaSuccess) e = alloc(sc.tc_slotpos, slots);
  if (e == cudaSuccess) e = alloc(sc.tc_tiles, 2 * (slots / kTcQueryTile) + 1);
  if (e == cudaSuccess) e = alloc(sc.tc_spans, 3 * spans + 1);
  if (e == cudaSuccess) e = alloc(sc.tc_gmin, (size_t)rows * 128);
  if (e == cudaSuccess) e = alloc(sc.tc_qlist, (size_t)rows * kTcQCap);
  if (e == cudaSuccess) e = alloc(sc.tc_qcnt, rows);
  if (e == cudaSuccess) e = alloc(sc.tc_thr, rows);
  if (e == cudaSuccess) e = alloc(sc.tc_sumy, 1);
  if (e == cudaSuccess) e = alloc(sc.tc_stage, (size_t)sms * kTcEpiThreads * kTcStage);
  if (e != cudaSuccess) {
    free_tc(sc);
    return e;
  }
  sc.tc_stage_sms = sms;
  sc.tc_rows = rows;
  sc.tc_slots = slots;
  sc.tc_spans_cap = spans;
  sc.tc_qrow_bytes = qrow;
  return cudaSuccess;
}

cudaError_t ensure_stage(Scratch& sc, int64_t nq, int k, int d) {
  if (sc.s_q && nq <= sc.stage_nq && k <= sc.stage_k && d == sc.stage_d) return cudaSuccess;
  int64_t cap = nq > sc.stage_nq ? nq : sc.stage_nq;
  int kc = k > sc.stage_k ? k : sc.stage_k;
  free_stage(sc);
  cudaError_t e = alloc(sc.s_q, (size_t)cap * d);
  if (e == cudaSuccess) e = alloc(sc.s_lo, cap);
  if (e == cudaSuccess) e = alloc(sc.s_hi, cap);
  if (e == cudaSuccess) e = alloc(sc.s_ids, (size_t)cap * kc);
  if (e == cudaSuccess) e = alloc(sc.s_dist, (size_t)cap * kc);
  if (e == cudaSuccess) e = alloc(sc.s_count, cap);
  if (e == cudaSuccess) e = alloc(sc.s_status, cap);
  if (e != cudaSuccess) {
    free_stage(sc);
    return e;
  }
  sc.stage_nq = cap;
  sc.stage_k = kc;
  sc.stage_d = d;
  return cudaSuccess;
}

int resolve(const DeviceIndex& ix, const unify_params_t* up, int k, int ef, Params& p) {
  unify_params_t d;
  unify_default_params(&d);
  if (up) d = *up;
  if (k < 1 || k > kMaxK) return fail(UNIFY_E_ARG, "k must be in [1, 256]");
  p.k = k;
  p.ef = ef > 0 ? ef : d.ef;
  p.ef_post = d.ef_post > 0 ? d.ef_post : p.ef;
  p.m = d.m;
  p.cand_cap = d.cand_cap;
  p.max_exp = d.max_expansions;
  p.warps_per_block = d.warps_per_block;
  p.scan_rows = d.scan_rows;
  p.reg_budget = d.reg_budget;
  p.tc_scan = d.tc_scan;
  p.selection = d.selection;
  p.dtype = d.dtype;
  p.rerank_mult = d.rerank_mult;
  p.tau_a = d.tau_a >= 0 ? d.tau_a : ix.n / 100;
  p.tau_b = d.tau_b >= 0 ? d.tau_b : ix.n / 2;
  if (p.ef < 1 || p.ef > 2048 || p.ef_post < 1 || p.ef_post > 2048) return fail(UNIFY_E_ARG, "ef and ef_post must be in [1, 2048]");
  if (p.m < 1 || p.m > 1024) return fail(UNIFY_E_ARG, "m must be in [1, 1024]");
  if (p.selection != 1 && p.selection != 2) return fail(UNIFY_E_ARG, "selection must be 1 (S1) or 2 (S2)");
  if (p.tc_scan < 0 || p.tc_scan > 2) return fail(UNIFY_E_ARG, "tc_scan must be 0, 1 or 2");
  if (p.tc_scan && (p.rerank_mult < 1 || (long)p.rerank_mult * k > kMaxCand))
    return fail(UNIFY_E_ARG, "rerank_mult must be >= 1 with rerank_mult * k <= 4096");
  if (p.selection == 1 && p.m > 64) return fail(UNIFY_E_ARG, "selection S1 takes m <= 64");
  if (p.cand_cap < 32 || p.cand_cap > kMaxCand) return fail(UNIFY_E_ARG, "cand_cap must be in [32, 4096]");
  if (d.visited_cap < 64 || d.visited_cap > 65536 || (d.visited_cap & (d.visited_cap - 1)))
    return fail(UNIFY_E_ARG, "visited_cap must be a power of two in [64, 65536]");
  p.vis_log2 = 0;
  while ((1 << p.vis_log2) < d.visited_cap) ++p.vis_log2;
  if (p.max_exp < 1) return fail(UNIFY_E_ARG, "max_expansions must be >= 1");
  if (p.warps_per_block < 1 || p.warps_per_block > 4) return fail(UNIFY_E_ARG, "warps_per_block must be in [1, 4]");
  if (p.reg_budget != 128 && p.reg_budget != 80 && p.reg_budget != 64)
    return fail(UNIFY_E_ARG, "reg_budget must be 128, 80 or 64");
  if (p.scan_rows < 32) return fail(UNIFY_E_ARG, "scan_rows must be >= 32");
  if (p.dtype != UNIFY_FP32 && p.dtype != UNIFY_BF16 && p.dtype != UNIFY_FP8E4M3)
    return fail(UNIFY_E_ARG, "dtype must be UNIFY_FP32, UNIFY_BF16 or UNIFY_FP8E4M3");
  if (p.dtype != UNIFY_FP32) {
    if (p.rerank_mult < 1 || (long)p.rerank_mult * k > kMaxCand)
      return fail(UNIFY_E_ARG, "rerank_mult must be >= 1 with rerank_mult * k <= 4096");
    // the re-rank reads its candidates from the candidate buffer
    if (p.cand_cap < rerank_count(p)) p.cand_cap = rerank_count(p);
  }
  const long smem = (long)p.warps_per_block * batch_smem_per_warp(p);
  if (smem > 227 * 1024) return fail(UNIFY_E_LIMIT, "graph search shared memory per CTA exceeds 227 KB; lower warps_per_block, cand_cap, visited_cap or ef");
  return UNIFY_OK;
}

cudaEvent_t take_event(Timing& t) {
  if (!t.pool.empty()) {
    cudaEvent_t e = t.pool.back();
    t.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Records an event pair around one phase when timing is on.
struct PhaseTimer {
  Timing& t;
  int phase;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  PhaseTimer(Timing& t_, int ph, cudaStream_t s) : t(t_), phase(ph), st(s) {
    if (t.on) {
      a = take_event(t);
      cudaEventRecord(a, st);
    }
  }
  ~PhaseTimer() {
    if (t.on && a) {
      cudaEvent_t b = take_event(t);
      cudaEventRecord(b, st);
      t.rec[phase].push_back({a, b});
    }
  }
};

int run_search(unify_index_t* idx, const float* q, const int64_t* lo, const int64_t* hi, int64_t nq, int k,
               int ef, int strategy, const unify_params_t* up, int64_t* out_ids, float* out_dist,
               int32_t* out_count, uint32_t* out_status, int32_t* out_counters, cudaStream_t st,
               const Conj* cj = nullptr) {
  if (!idx) return fail(UNIFY_E_ARG, "null index");
  if (nq < 0 || nq >= (1ll << 31) / kMaxScanBlocks) return fail(UNIFY_E_ARG, "nq out of range");
  if (strategy < -1 || strategy > 2) return fail(UNIFY_E_ARG, "bad strategy");
  Params p;
  int rc = resolve(idx->ix, up, k, ef, p);
  if (rc != UNIFY_OK) return rc;
  if (nq == 0) return UNIFY_OK;
  if (!q || !lo || !hi || !out_ids || !out_dist || !out_count) return fail(UNIFY_E_ARG, "null query or output pointer");
  DeviceGuard guard(idx->ix.device);
  if (idx->live_plans > 0 && (nq > idx->sc.cap_nq || k > idx->sc.cap_k))
    return fail(UNIFY_E_LIMIT, "search larger than the scratch held by a live plan; destroy the plans first");
  const int kk = rerank_count(p) > k ? rerank_count(p) : k;  // keys per partial scan list
  if (idx->live_plans > 0 && kk > idx->sc.cap_k)
    return fail(UNIFY_E_LIMIT, "search larger than the scratch held by a live plan; destroy the plans first");
  cudaError_t e = ensure_scratch(idx->sc, nq, kk);
  if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
  // the tensor-core scan has no second-attribute predicate: conjunctive queries use the warp scan
  const bool tc = !cj && (strategy == UNIFY_PRE || strategy == UNIFY_AUTO) && tc_scan_available(idx->ix, p);
  if (tc) {
    if (idx->live_plans > 0 && !tc_scratch_fits(idx->sc, nq, idx->ix.d, (int64_t)idx->ix.n, idx->ix.num_sms))
      return fail(UNIFY_E_LIMIT, "search larger than the scratch held by a live plan; destroy the plans first");
    e = ensure_tc_scratch(idx->sc, nq, idx->ix.d, (int64_t)idx->ix.n, idx->ix.num_sms);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core scan scratch allocation");
  }
  Scratch& sc = idx->sc;
  e = cudaMemsetAsync(sc.counters, 0, kNumCounters * sizeof(int32_t), st);
  if (e != cudaSuccess) return cuda_fail(e, "counter reset");
  Outputs o{out_ids, out_dist, out_count, out_status, out_counters};
  NvtxRange whole("unify:search");
  {
    NvtxRange r("unify:route");
    PhaseTimer t(idx->tm, 0, st);
    e = launch_route(idx->ix, sc, lo, hi, nq, p.tau_a, p.tau_b, strategy, p.scan_rows, 1, sc.pa, sc.pb, sc.mask,
                     sc.strat, &o, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "route kernel");
  if (tc) {
    NvtxRange r("unify:tensor-core scan");
    PhaseTimer t(idx->tm, 2, st);
    e = launch_tcscan(idx->ix, sc, q, nq, p, o, st);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core pre-filter scan");
  }
  {
    NvtxRange r("unify:search kernel");
    PhaseTimer t(idx->tm, 1, st);
    e = launch_batch(idx->ix, sc, q, p, o, st, tc, cj);
  }
  if (e != cudaSuccess) return cuda_fail(e, "search kernel");
  return UNIFY_OK;
}

}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

int resolve_search_params(const DeviceIndex& ix, const unify_params_t* up, int k, int ef, Params& p) {
  return resolve(ix, up, k, ef, p);
}

void free_scratch(Scratch& sc) {
  free_core(sc);
  free_tc(sc);
  free_stage(sc);
}

}  // namespace unify

using namespace unify;

extern "C" void unify_default_params(unify_params_t* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->ef = 100;
  p->m = 16;
  p->ef_post = 0;
  p->rerank_mult = 4;
  p->dtype = UNIFY_FP32;
  p->tau_a = -1;
  p->tau_b = -1;
  p->cand_cap = 512;
  p->visited_cap = 2048;
  p->max_expansions = 100000;
  p->warps_per_block = 4;
  p->scan_rows = 8192;
  p->reg_budget = 128;
  p->tc_scan = 0;
  p->selection = 2;
}

extern "C" const char* unify_last_error(void) { return g_last_error.c_str(); }

extern "C" int unify_plan_create(unify_index_t* idx, const float* q, const int64_t* lo, const int64_t* hi,
                                 int64_t nq, int k, int ef, unify_strategy_t strategy, const unify_params_t* p,
                                 int64_t* out_ids, float* out_dist, int32_t* out_count, uint32_t* out_status,
                                 unify_plan_t** out) {
  if (!idx || !out) return fail(UNIFY_E_ARG, "unify_plan_create: null argument");
  *out = nullptr;
  if (nq < 1) return fail(UNIFY_E_ARG, "unify_plan_create: nq must be >= 1");
  DeviceGuard guard(idx->ix.device);
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "unify_plan_create: stream");
  // One ordinary search first: it sizes the scratch and sets kernel attributes, so
  // that the captured search enqueues kernels only.
  const bool timing = idx->tm.on;
  idx->tm.on = false;
  int rc = run_search(idx, q, lo, hi, nq, k, ef, (int)strategy, p, out_ids, out_dist, out_count, out_status,
                      nullptr, cs);
  if (rc == UNIFY_OK) {
    e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) rc = cuda_fail(e, "unify_plan_create: first search");
  }
  unify_plan_t* plan = nullptr;
  if (rc == UNIFY_OK) {
    plan = new (std::nothrow) unify_plan_t;
    if (!plan) rc = fail(UNIFY_E_NOMEM, "unify_plan_create: host allocation");
  }
  if (rc == UNIFY_OK) {
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "unify_plan_create: begin capture");
    } else {
      rc = run_search(idx, q, lo, hi, nq, k, ef, (int)strategy, p, out_ids, out_dist, out_count, out_status,
                      nullptr, cs);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(cs, &g);
      if (rc == UNIFY_OK && e != cudaSuccess) rc = cuda_fail(e, "unify_plan_create: end capture");
      plan->graph = g;
      if (rc == UNIFY_OK) {
        e = cudaGraphInstantiate(&plan->exec, g, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "unify_plan_create: instantiate");
      }
    }
  }
  idx->tm.on = timing;
  cudaStreamDestroy(cs);
  if (rc != UNIFY_OK) {
    if (plan) {
      if (plan->exec) cudaGraphExecDestroy(plan->exec);
      if (plan->graph) cudaGraphDestroy(plan->graph);
      delete plan;
    }
    return rc;
  }
  plan->idx = idx;
  idx->live_plans++;
  *out = plan;
  return UNIFY_OK;
}

extern "C" int unify_plan_launch(unify_plan_t* plan, void* stream) {
  if (!plan || !plan->exec) return fail(UNIFY_E_ARG, "unify_plan_launch: null plan");
  DeviceGuard guard(plan->idx->ix.device);
  cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
  return e == cudaSuccess ? UNIFY_OK : cuda_fail(e, "unify_plan_launch");
}

extern "C" void unify_plan_destroy(unify_plan_t* plan) {
  if (!plan) return;
  {
    DeviceGuard guard(plan->idx->ix.device);
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
  }
  plan->idx->live_plans--;
  delete plan;
}

extern "C" int unify_timing_enable(unify_index_t* idx, int enable) {
  if (!idx) return fail(UNIFY_E_ARG, "unify_timing_enable: null index");
  idx->tm.on = enable != 0;
  return UNIFY_OK;
}

extern "C" int unify_timing_collect(unify_index_t* idx, double* total_ms, int64_t* spans) {
  if (!idx) return fail(UNIFY_E_ARG, "unify_timing_collect: null index");
  DeviceGuard guard(idx->ix.device);
  for (int ph = 0; ph < kPhases; ++ph) {
    double sum = 0.0;
    int64_t cnt = 0;
    for (auto& pr : idx->tm.rec[ph]) {
      cudaError_t e = cudaEventSynchronize(pr.second);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pr.first, pr.second);
      if (e != cudaSuccess) return cuda_fail(e, "unify_timing_collect");
      sum += ms;
      ++cnt;
      idx->tm.pool.push_back(pr.first);
      idx->tm.pool.push_back(pr.second);
    }
    idx->tm.rec[ph].clear();
    if (total_ms) total_ms[ph] = sum;
    if (spans) spans[ph] = cnt;
  }
  return UNIFY_OK;
}

extern "C" int unify_route(unify_index_t* idx, const int64_t* lo, const int64_t* hi, int64_t nq, int64_t tau_a,
                           int64_t tau_b, int32_t* out_pa, int32_t* out_pb, uint32_t* out_mask,
                           int32_t* out_strategy, void* stream) {
  if (!idx) return fail(UNIFY_E_ARG, "unify_route: null index");
  if (nq < 0) return fail(UNIFY_E_ARG, "unify_route: nq < 0");
  if (nq == 0) return UNIFY_OK;
  if (!lo || !hi) return fail(UNIFY_E_ARG, "unify_route: null range pointer");
  DeviceGuard guard(idx->ix.device);
  const int64_t ta = tau_a >= 0 ? tau_a : idx->ix.n / 100;
  const int64_t tb = tau_b >= 0 ? tau_b : idx->ix.n / 2;
  cudaError_t e = launch_route(idx->ix, idx->sc, lo, hi, nq, ta, tb, -1, 8192, 0, out_pa, out_pb, out_mask,
                               out_strategy, nullptr, (cudaStream_t)stream);
  return e == cudaSuccess ? UNIFY_OK : cuda_fail(e, "unify_route");
}

extern "C" int unify_search(unify_index_t* idx, const float* q, const int64_t* lo, const int64_t* hi, int64_t nq,
                            int k, int ef, unify_strategy_t strategy, const unify_params_t* p, int64_t* out_ids,
                            float* out_dist, int32_t* out_count, uint32_t* out_status, int32_t* out_counters,
                            void* stream) {
  return run_search(idx, q, lo, hi, nq, k, ef, (int)strategy, p, out_ids, out_dist, out_count, out_status,
                    out_counters, (cudaStream_t)stream);
}

extern "C" int unify_search_conj(unify_index_t* idx, const float* q, const int64_t* lo, const int64_t* hi,
                                 const int64_t* attr2, const int64_t* lo2, const int64_t* hi2, int64_t nq, int k,
                                 int ef, unify_strategy_t strategy, const unify_params_t* p, int64_t* out_ids,
                                 float* out_dist, int32_t* out_count, uint32_t* out_status, int32_t* out_counters,
                                 void* stream) {
  if (nq > 0 && (!attr2 || !lo2 || !hi2))
    return fail(UNIFY_E_ARG, "unify_search_conj: null second-attribute pointer");
  Conj cj;
  cj.attr2 = attr2;
  cj.lo2 = lo2;
  cj.hi2 = hi2;
  return run_search(idx, q, lo, hi, nq, k, ef, (int)strategy, p, out_ids, out_dist, out_count, out_status,
                    out_counters, (cudaStream_t)stream, &cj);
}

extern "C" int unify_search_auto(unify_index_t* idx, const float* q, const int64_t* lo, const int64_t* hi,
                                 int64_t nq, int k, int ef, const unify_params_t* p, int64_t* out_ids,
                                 float* out_dist, int32_t* out_count, uint32_t* out_status, void* stream) {
  return run_search(idx, q, lo, hi, nq, k, ef, UNIFY_AUTO, p, out_ids, out_dist, out_count, out_status, nullptr,
                    (cudaStream_t)stream);
}

extern "C" int unify_search_auto_host(unify_index_t* idx, const float* q, const int64_t* lo, const int64_t* hi,
                                      int64_t nq, int k, int ef, const unify_params_t* p, int64_t* out_ids,
                                      float* out_dist, int32_t* out_count, uint32_t* out_status, void* stream) {
  if (!idx) return fail(UNIFY_E_ARG, "null index");
  if (nq < 0) return fail(UNIFY_E_ARG, "nq < 0");
  if (k < 1 || k > kMaxK) return fail(UNIFY_E_ARG, "k must be in [1, 256]");
  if (nq == 0) return UNIFY_OK;
  if (!q || !lo || !hi || !out_ids || !out_dist || !out_count) return fail(UNIFY_E_ARG, "null query or output pointer");
  cudaStream_t st = (cudaStream_t)stream;
  DeviceGuard guard(idx->ix.device);
  Scratch& sc = idx->sc;
  const int d = idx->ix.d;
  cudaError_t e = ensure_stage(sc, nq, k, d);
  if (e != cudaSuccess) return cuda_fail(e, "staging allocation");
  e = cudaMemcpyAsync(sc.s_q, q, (size_t)nq * d * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sc.s_lo, lo, (size_t)nq * sizeof(int64_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sc.s_hi, hi, (size_t)nq * sizeof(int64_t), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
  int rc = run_search(idx, sc.s_q, sc.s_lo, sc.s_hi, nq, k, ef, UNIFY_AUTO, p, sc.s_ids, sc.s_dist, sc.s_count,
                      sc.s_status, nullptr, st);
  if (rc != UNIFY_OK) return rc;
  e = cudaMemcpyAsync(out_ids, sc.s_ids, (size_t)nq * k * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_dist, sc.s_dist, (size_t)nq * k * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_count, sc.s_count, (size_t)nq * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && out_status)
    e = cudaMemcpyAsync(out_status, sc.s_status, (size_t)nq * sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? UNIFY_OK : cuda_fail(e, "device-to-host copy");
}
