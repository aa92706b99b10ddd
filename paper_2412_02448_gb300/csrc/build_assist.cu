// GPU-assisted construction: the proposal step of the batched HSIG insertion.
//
// The host builder inserts nodes in id order in batches; every node of a batch
// searches the graph as it stood at the start of the batch (HSIGInsert,
// Algorithm 6, with BackboneConnectionsBuild, Algorithm 4). For node v and every
// segment j:
//   * descend from the segment's entry point through the layers above v's level
//     with ANNSearch (Algorithm 1) at ef = 1, following only the chunks j;
//   * on every layer l <= level[v] (and <= the segment's top) run ANNSearch with
//     ef = efCons over the chunks j, then keep at most M forward edges with the
//     pruning heuristic of Section 2.2 (walk the candidates in ascending (distance,
//     id); drop one that is farther from v than from an edge already kept);
//   * the nearest result is the entry point of the next layer.
// Here one warp does this for one (batch node, segment) pair against a device
// mirror of the graph. Either the host uploads the chunks it changed between calls and
// applies the proposals and reverse edges itself, or (apply) the device stores the
// forward lists and applies the reverse edges of Algorithm 4 in its own copy, one warp
// per target chunk, and the host fetches the graph once at the end. Entry points stay
// on the host.
//
// ANNSearch uses the single sorted buffer of the post-filter search: cand is a
// subset of ann (every candidate push is also an ann push), so one array E of
// capacity ef, sorted by key (distance, id) with an "expanded" flag, holds both;
// an object evicted from ann is larger than every object left in it, so when the
// heap version breaks (its nearest candidate was evicted) every object of E has
// been expanded and the loop here ends too. A direct-mapped visited filter may
// forget objects; a forgotten object is re-found in E by its bit-identical key, or
// lies above the threshold. Float32 distances use the fixed lane order and
// reduction tree of the search kernel; on vectors whose squared distances are
// integers below 2^24 they are exact, and the proposals equal the host's.
//
// Bounds (checked against the buffers of each launch): warps cover
// count * S pairs (a warp-uniform early return past the end); neighbour slots are
// read for lane < cnt <= M <= 32; E holds at most ecap >= efc keys; kept at most
// M <= 32 keys; output rows are row0[v] + l - row0[first] < rows of the batch. The
// reverse-edge warps hold at most M + 1 <= 33 candidate keys; group chunks, group
// bounds and sources are validated on the host before upload.
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "warp_ops.cuh"

namespace unify {
namespace {

constexpr int kBuildMaxM = 32;
constexpr int kBuildMaxEf = 256;
constexpr int kBuildMaxS = 32;
constexpr int kBuildVisLog2 = 11;
constexpr int kBuildWarps = 4;
constexpr long long kBuildMaxExpansions = 1ll << 20;

int bfail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

int bcuda_fail(cudaError_t e, const char* where) {
  return bfail(e == cudaErrorMemoryAllocation ? UNIFY_E_NOMEM : UNIFY_E_CUDA,
               std::string(where) + ": " + cudaGetErrorString(e));
}

struct BuildArgs {
  const float* X;  // n x dp, zero-padded rows
  int dp4;
  const int32_t* level;
  const int64_t* row0;
  const int32_t* adj;  // nrows x S x M
  const uint8_t* cnt;  // nrows x S
  int S, M, efc, ecap;
  int32_t entry_seg[kBuildMaxS], top_seg[kBuildMaxS];
  int64_t first, count, row_first;
  int32_t* out_ids;
  float* out_dist;
  uint8_t* out_cnt;
  int32_t* err;  // set when a search hit the expansion bound
};

struct BuildWarp {
  uint64_t* E;
  uint8_t* Ef;
  int32_t* vis;
  int* R;
  int* clist;
  uint64_t* kept;
};

__host__ __device__ inline size_t build_warp_bytes(int ecap) {
  size_t b = (size_t)ecap * 8 + (size_t)((ecap + 15) & ~15) + ((size_t)4 << kBuildVisLog2) + 32 * 4 * 2 + 32 * 8;
  return (b + 15) & ~(size_t)15;
}

__device__ __forceinline__ BuildWarp build_carve(unsigned char* base, int ecap) {
  BuildWarp w;
  w.E = reinterpret_cast<uint64_t*>(base);
  w.Ef = reinterpret_cast<uint8_t*>(w.E + ecap);
  w.vis = reinterpret_cast<int32_t*>(w.Ef + ((ecap + 15) & ~15));
  w.R = reinterpret_cast<int*>(w.vis + (1 << kBuildVisLog2));
  w.clist = w.R + 32;
  w.kept = reinterpret_cast<uint64_t*>(w.clist + 32);
  return w;
}

__device__ __forceinline__ uint32_t build_hash(int id) {
  return ((uint32_t)id * 0x9E3779B1u) >> (32 - kBuildVisLog2);
}

// Row id of X into the lane layout (chunks lane, lane + 32, ...).
template <int CH>
__device__ __forceinline__ void load_row(float4 (&x)[CH], const float* X, int dp4, int64_t id) {
  const int lane = lane_id();
  const float4* r = reinterpret_cast<const float4*>(X) + id * dp4;
#pragma unroll
  for (int t = 0; t < CH; ++t) {
    const int c = lane + 32 * t;
    x[t] = c < dp4 ? __ldg(r + c) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// ANNSearch (Algorithm 1) from ep_key on layer l over the chunks j, capacity ef.
// Returns |E|; E[0, |E|) ascending.
template <int CH, int G>
__device__ int build_search(const BuildArgs& a, const BuildWarp& w, const float4 (&q)[CH], int l, int j, int ef,
                            uint64_t ep_key) {
  const int lane = lane_id();
  for (int t = lane; t < (1 << kBuildVisLog2); t += 32) w.vis[t] = -1;
  __syncwarp();
  const int ep = key_id(ep_key);
  if (lane == 0) {
    w.E[0] = ep_key;
    w.Ef[0] = 0;
    w.vis[build_hash(ep)] = ep;
  }
  __syncwarp();
  int nE = 1, cursor = 0;
  long long nexp = 0;
  for (;;) {
    // the nearest unexpanded candidate
    while (cursor < nE) {
      const int jj = cursor + lane;
      const unsigned bal = __ballot_sync(kFull, jj < nE && w.Ef[jj] == 0);
      if (bal) {
        cursor += __ffs(bal) - 1;
        break;
      }
      cursor += 32;
    }
    if (cursor >= nE) break;
    if (++nexp > kBuildMaxExpansions) {
      if (lane == 0) atomicExch(a.err, 1);
      break;
    }
    const int o = key_id(w.E[cursor]);
    __syncwarp();
    if (lane == 0) w.Ef[cursor] = 1;
    __syncwarp();
    const int64_t row = a.row0[o] + l;
    const int c = a.cnt[row * a.S + j];
    int cid = lane < c ? __ldg(a.adj + (row * a.S + j) * a.M + lane) : -1;
    if (cid >= 0) {
      const uint32_t h = build_hash(cid);
      if (w.vis[h] == cid) cid = -1;
      else w.vis[h] = cid;
    }
    __syncwarp();
    const float dist = batch_dist<StoreF32, CH, G>(q, cid, reinterpret_cast<const unsigned char*>(a.X), a.dp4 * 16,
                                                   nullptr, a.dp4, w.clist);
    const uint64_t key = cid >= 0 ? make_key(dist, cid) : kKeyMax;
    const uint64_t thr = nE >= ef ? w.E[ef - 1] : kKeyMax;
    bool keep = cid >= 0 && key < thr;
    // a visited object the filter forgot is still in E (or above the threshold)
    if (keep && contains_u64(w.E, nE, key)) keep = false;
    const unsigned kb = __ballot_sync(kFull, keep);
    if (kb == 0) continue;
    const uint64_t sk = warp_sort_asc(keep ? key : kKeyMax);
    int r0;
    bool dropped;
    nE = warp_merge(w.E, w.Ef, nE, ef, sk, __popc(kb), w.R, &r0, &dropped);
    if (r0 < cursor) cursor = r0;
  }
  __syncwarp();
  return nE;
}

// Pruning heuristic over E[0, nE): at most M kept keys in w.kept, ascending.
template <int CH, int G>
__device__ int build_prune(const BuildArgs& a, const BuildWarp& w, int nE) {
  const int lane = lane_id();
  int nk = 0;
  for (int i = 0; i < nE && nk < a.M; ++i) {
    const uint64_t r = w.E[i];
    float4 xr[CH];
    load_row<CH>(xr, a.X, a.dp4, key_id(r));
    const int cid = lane < nk ? key_id(w.kept[lane]) : -1;
    // distances from r to the kept objects, one per lane
    const float dk = batch_dist<StoreF32, CH, G>(xr, cid, reinterpret_cast<const unsigned char*>(a.X), a.dp4 * 16,
                                                 nullptr, a.dp4, w.clist);
    const bool drop = __any_sync(kFull, cid >= 0 && key_dist(r) > dk);
    if (!drop) {
      if (lane == 0) w.kept[nk] = r;
      ++nk;
      __syncwarp();
    }
  }
  return nk;
}

template <int CH, int G>
__global__ void __launch_bounds__(32 * kBuildWarps) build_kernel(BuildArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const BuildWarp w = build_carve(smem_raw + (size_t)warp * build_warp_bytes(a.ecap), a.ecap);
  const int64_t wid = (int64_t)blockIdx.x * kBuildWarps + warp;
  if (wid >= a.count * a.S) return;  // whole warps
  const int64_t t = wid / a.S;
  const int j = (int)(wid - t * a.S);
  const int64_t v = a.first + t;
  const int lv = a.level[v];
  const int64_t rb = a.row0[v] - a.row_first;
  if (lane == 0)
    for (int l = 0; l <= lv; ++l) a.out_cnt[(rb + l) * a.S + j] = 0;
  const int ep0 = a.entry_seg[j];
  if (ep0 < 0) return;  // the segment holds no node yet
  const int L = a.top_seg[j];
  float4 q[CH];
  load_row<CH>(q, a.X, a.dp4, v);
  const float d0 = batch_dist<StoreF32, CH, G>(q, lane == 0 ? ep0 : -1, reinterpret_cast<const unsigned char*>(a.X),
                                               a.dp4 * 16, nullptr, a.dp4, w.clist);
  uint64_t ep = make_key(__shfl_sync(kFull, d0, 0), ep0);
  for (int l = L; l > lv; --l) {
    build_search<CH, G>(a, w, q, l, j, 1, ep);
    ep = w.E[0];
    __syncwarp();
  }
  for (int l = (lv < L ? lv : L); l >= 0; --l) {
    const int nE = build_search<CH, G>(a, w, q, l, j, a.efc, ep);
    const int nk = build_prune<CH, G>(a, w, nE);
    const int64_t o = (rb + l) * a.S + j;
    for (int s = lane; s < nk; s += 32) {
      a.out_ids[o * a.M + s] = key_id(w.kept[s]);
      a.out_dist[o * a.M + s] = key_dist(w.kept[s]);
    }
    if (lane == 0) a.out_cnt[o] = (uint8_t)nk;
    ep = w.E[0];
    __syncwarp();
  }
}

// Writes uploaded chunk contents into the device graph.
__global__ void scatter_chunks(const int64_t* __restrict__ idx, const int32_t* __restrict__ ids,
                               const float* __restrict__ dist, const uint8_t* __restrict__ cnt, int64_t nd, int M,
                               int32_t* adj, float* adjd, uint8_t* cnt_dev) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nd * M; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / M;
    const int s = (int)(i - e * M);
    adj[idx[e] * M + s] = ids[i];
    adjd[idx[e] * M + s] = dist[i];
    if (s == 0) cnt_dev[idx[e]] = cnt[e];
  }
}

// Stores the batch's non-empty forward lists (rows x S chunks from row_first on),
// padding slots past the count with id -1 and distance 0 as the host does.
__global__ void store_forward(const int32_t* __restrict__ o_ids, const float* __restrict__ o_dist,
                              const uint8_t* __restrict__ o_cnt, int64_t nchunks, int M, int64_t chunk0,
                              int32_t* adj, float* adjd, uint8_t* cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nchunks * M;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / M;
    const int s = (int)(i - e * M);
    const int c = o_cnt[e];
    if (c == 0) continue;
    const int64_t dst = (chunk0 + e) * M + s;
    adj[dst] = s < c ? o_ids[i] : -1;
    adjd[dst] = s < c ? o_dist[i] : 0.f;
    if (s == 0) cnt[chunk0 + e] = (uint8_t)c;
  }
}

struct RevArgs {
  const float* X;
  int dp4, M;
  int32_t* adj;
  float* adjd;
  uint8_t* cnt;
  const int64_t* g_chunk;
  const int64_t* g_start;
  int64_t ngroups;
  const int32_t* r_v;
  const float* r_d;
};

// Algorithm 4's reverse edges, one warp per target chunk, edges in source-id order:
// an edge already present changes nothing; otherwise it is inserted in (distance, id)
// order and, when the chunk then holds M + 1 keys, the chunk is re-pruned with the
// heuristic of Section 2.2 (candidates ascending; one is dropped when it is farther
// from the owner than from a neighbour already kept).
template <int CH, int G>
__global__ void __launch_bounds__(32 * kBuildWarps) reverse_kernel(RevArgs a) {
  __shared__ uint64_t sK[kBuildWarps][kBuildMaxM + 1];
  __shared__ uint64_t sKept[kBuildWarps][kBuildMaxM];
  __shared__ int sList[kBuildWarps][32];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const int64_t g = (int64_t)blockIdx.x * kBuildWarps + warp;
  if (g >= a.ngroups) return;  // whole warps
  uint64_t* K = sK[warp];
  uint64_t* kept = sKept[warp];
  const int64_t ch = a.g_chunk[g];
  const int M = a.M;
  int c = a.cnt[ch];
  uint64_t key = lane < c ? make_key(a.adjd[ch * M + lane], a.adj[ch * M + lane]) : kKeyMax;
  K[lane] = warp_sort_asc(key);
  __syncwarp();
  const int64_t e1 = a.g_start[g + 1];
  for (int64_t e = a.g_start[g]; e < e1; ++e) {
    const int32_t v = a.r_v[e];
    if (__any_sync(kFull, lane < c && key_id(K[lane]) == v)) continue;
    const uint64_t kv = make_key(a.r_d[e], v);
    const int pos = __popc(__ballot_sync(kFull, lane < c && K[lane] < kv));
    const uint64_t mine = lane < c ? K[lane] : 0;
    __syncwarp();
    if (lane < c && lane >= pos) K[lane + 1] = mine;
    __syncwarp();
    if (lane == 0) K[pos] = kv;
    __syncwarp();
    ++c;
    if (c <= M) continue;
    int nk = 0;
    for (int t = 0; t < c && nk < M; ++t) {
      const uint64_t r = K[t];
      float4 xr[CH];
      load_row<CH>(xr, a.X, a.dp4, key_id(r));
      const int cid = lane < nk ? key_id(kept[lane]) : -1;
      const float dk = batch_dist<StoreF32, CH, G>(xr, cid, reinterpret_cast<const unsigned char*>(a.X), a.dp4 * 16,
                                                   nullptr, a.dp4, sList[warp]);
      if (!__any_sync(kFull, cid >= 0 && key_dist(r) > dk)) {
        if (lane == 0) kept[nk] = r;
        ++nk;
        __syncwarp();
      }
    }
    __syncwarp();
    if (lane < nk) K[lane] = kept[lane];
    __syncwarp();
    c = nk;
  }
  if (lane < M) {
    const bool has = lane < c;
    a.adj[ch * M + lane] = has ? key_id(K[lane]) : -1;
    a.adjd[ch * M + lane] = has ? key_dist(K[lane]) : 0.f;
  }
  if (lane == 0) a.cnt[ch] = (uint8_t)c;
}

template <class T>
cudaError_t grow(T*& p, int64_t& cap, int64_t need) {
  if (need <= cap && p) return cudaSuccess;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), (size_t)(need > 0 ? need : 1) * sizeof(T));
  if (e == cudaSuccess) cap = need;
  return e;
}

}  // namespace

struct BuildCtx {
  int device = 0;
  bool ready = false;
  int64_t n = 0, nrows = 0;
  int d = 0, dp = 0, S = 0, M = 0;
  float* X = nullptr;
  int32_t* level = nullptr;
  int64_t* row0 = nullptr;
  int32_t* adj = nullptr;
  float* adjd = nullptr;
  uint8_t* cnt = nullptr;
  int32_t* err = nullptr;
  int32_t* o_ids = nullptr;
  float* o_dist = nullptr;
  uint8_t* o_cnt = nullptr;
  int64_t o_cap = 0, o_cap_d = 0, o_cap_c = 0;
  int64_t* u_idx = nullptr;
  int32_t* u_ids = nullptr;
  float* u_dist = nullptr;
  uint8_t* u_cnt = nullptr;
  int64_t u_cap = 0, u_cap_i = 0, u_cap_d = 0, u_cap_c = 0;
  std::vector<int64_t> h_idx;
  std::vector<int32_t> h_ids;
  std::vector<float> h_dist;
  std::vector<uint8_t> h_cnt;
  // the last proposals (device buffers o_*): batch and its rows
  int64_t prop_first = -1, prop_rows = 0, prop_row_first = 0;
  // reverse-edge groups of the current batch
  int64_t* g_chunk = nullptr;
  int64_t* g_start = nullptr;
  int32_t* r_v = nullptr;
  float* r_d = nullptr;
  int64_t g_cap = 0, g_cap_s = 0, r_cap = 0, r_cap_d = 0;
  cudaStream_t st = nullptr;
};

namespace {

// Frees every device buffer and the stream, and returns the context to its state
// after creation (same device).
void build_free(BuildCtx* c) {
  void* ptrs[] = {c->X, c->level, c->row0, c->adj, c->adjd, c->cnt, c->err, c->o_ids, c->o_dist, c->o_cnt,
                  c->u_idx, c->u_ids, c->u_dist, c->u_cnt, c->g_chunk, c->g_start, c->r_v, c->r_d};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->st) cudaStreamDestroy(c->st);
  const int dev = c->device;
  *c = BuildCtx();
  c->device = dev;
}

template <int CH, int G>
cudaError_t launch_build(const BuildArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)kBuildWarps * build_warp_bytes(a.ecap);
  cudaError_t e = cudaFuncSetAttribute(build_kernel<CH, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t pairs = a.count * a.S;
  const int64_t blocks = (pairs + kBuildWarps - 1) / kBuildWarps;
  build_kernel<CH, G><<<(unsigned)blocks, 32 * kBuildWarps, smem, st>>>(a);
  return cudaGetLastError();
}

int propose(BuildCtx* c, const unify_build_view_t* v, int32_t* out_ids, float* out_dist, uint8_t* out_cnt) {
  cudaError_t e = cudaSuccess;
  if (!c->ready) {
    c->n = v->n;
    c->nrows = v->nrows;
    c->d = v->d;
    c->dp = (v->d + 3) / 4 * 4;
    c->S = v->S;
    c->M = v->M;
    e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&c->X, (size_t)c->n * c->dp * sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->X, 0, (size_t)c->n * c->dp * sizeof(float), c->st);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(c->X, (size_t)c->dp * 4, v->X, (size_t)c->d * 4, (size_t)c->d * 4, (size_t)c->n,
                            cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMalloc(&c->level, (size_t)c->n * 4);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->level, v->level, (size_t)c->n * 4, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMalloc(&c->row0, (size_t)c->n * 8);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->row0, v->row0, (size_t)c->n * 8, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMalloc(&c->adj, (size_t)c->nrows * c->S * c->M * 4);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->adj, v->adj, (size_t)c->nrows * c->S * c->M * 4, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMalloc(&c->adjd, (size_t)c->nrows * c->S * c->M * 4);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->adjd, v->adjd, (size_t)c->nrows * c->S * c->M * 4, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMalloc(&c->cnt, (size_t)c->nrows * c->S);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->cnt, v->cnt, (size_t)c->nrows * c->S, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMalloc(&c->err, 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, 4, c->st);
    if (e != cudaSuccess) {
      // start clean on a later call: nothing of the partial copy stays allocated
      if (c->st) cudaStreamSynchronize(c->st);
      build_free(c);
      return bcuda_fail(e, "build assist: device copy of the graph");
    }
    c->ready = true;
  } else if (v->ndirty > 0) {
    // the chunks the host changed since the previous batch
    const int64_t nd = v->ndirty;
    c->h_idx.assign(v->dirty, v->dirty + nd);
    c->h_ids.resize((size_t)nd * c->M);
    c->h_dist.resize((size_t)nd * c->M);
    c->h_cnt.resize((size_t)nd);
    for (int64_t i = 0; i < nd; ++i) {
      const int64_t ch = v->dirty[i];
      if (ch < 0 || ch >= c->nrows * c->S) return bfail(UNIFY_E_ARG, "build assist: dirty chunk out of range");
      std::memcpy(&c->h_ids[(size_t)i * c->M], v->adj + ch * c->M, (size_t)c->M * 4);
      std::memcpy(&c->h_dist[(size_t)i * c->M], v->adjd + ch * c->M, (size_t)c->M * 4);
      c->h_cnt[i] = v->cnt[ch];
    }
    e = grow(c->u_idx, c->u_cap, nd);
    if (e == cudaSuccess) e = grow(c->u_ids, c->u_cap_i, nd * c->M);
    if (e == cudaSuccess) e = grow(c->u_dist, c->u_cap_d, nd * c->M);
    if (e == cudaSuccess) e = grow(c->u_cnt, c->u_cap_c, nd);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->u_idx, c->h_idx.data(), nd * 8, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->u_ids, c->h_ids.data(), nd * c->M * 4, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->u_dist, c->h_dist.data(), nd * c->M * 4, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->u_cnt, c->h_cnt.data(), nd, cudaMemcpyHostToDevice, c->st);
    if (e != cudaSuccess) return bcuda_fail(e, "build assist: chunk upload");
    scatter_chunks<<<256, 256, 0, c->st>>>(c->u_idx, c->u_ids, c->u_dist, c->u_cnt, nd, c->M, c->adj, c->adjd,
                                           c->cnt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return bcuda_fail(e, "build assist: chunk scatter");
  }
  if (v->count <= 0) return UNIFY_OK;
  const int64_t last = v->first + v->count - 1;
  const int64_t row_first = v->row0[v->first];
  const int64_t rows = v->row0[last] + v->level[last] + 1 - row_first;
  e = grow(c->o_ids, c->o_cap, rows * c->S * c->M);
  if (e == cudaSuccess) e = grow(c->o_dist, c->o_cap_d, rows * c->S * c->M);
  if (e == cudaSuccess) e = grow(c->o_cnt, c->o_cap_c, rows * c->S);
  if (e != cudaSuccess) return bcuda_fail(e, "build assist: output buffers");
  BuildArgs a;
  a.X = c->X;
  a.dp4 = c->dp / 4;
  a.level = c->level;
  a.row0 = c->row0;
  a.adj = c->adj;
  a.cnt = c->cnt;
  a.S = c->S;
  a.M = c->M;
  a.efc = v->efc;
  a.ecap = v->efc < 1 ? 1 : v->efc;
  for (int j = 0; j < kBuildMaxS; ++j) {
    a.entry_seg[j] = j < c->S ? v->entry_seg[j] : -1;
    a.top_seg[j] = j < c->S ? v->top_seg[j] : -1;
  }
  a.first = v->first;
  a.count = v->count;
  a.row_first = row_first;
  a.out_ids = c->o_ids;
  a.out_dist = c->o_dist;
  a.out_cnt = c->o_cnt;
  a.err = c->err;
  const int ch = (a.dp4 + 31) / 32;
  if (ch <= 1) e = launch_build<1, 16>(a, c->st);
  else if (ch <= 2) e = launch_build<2, 8>(a, c->st);
  else if (ch <= 4) e = launch_build<4, 4>(a, c->st);
  else e = launch_build<8, 2>(a, c->st);
  if (e != cudaSuccess) return bcuda_fail(e, "build assist: proposal kernel");
  int32_t herr = 0;
  e = cudaMemcpyAsync(out_ids, c->o_ids, rows * c->S * c->M * 4, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_dist, c->o_dist, rows * c->S * c->M * 4, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_cnt, c->o_cnt, rows * c->S, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, c->err, 4, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return bcuda_fail(e, "build assist: proposals to the host");
  if (herr) return bfail(UNIFY_E_LIMIT, "build assist: a search hit the expansion bound");
  c->prop_first = v->first;
  c->prop_rows = rows;
  c->prop_row_first = row_first;
  return UNIFY_OK;
}

template <int CH, int G>
cudaError_t launch_reverse(const RevArgs& a, cudaStream_t st) {
  const int64_t blocks = (a.ngroups + kBuildWarps - 1) / kBuildWarps;
  reverse_kernel<CH, G><<<(unsigned)blocks, 32 * kBuildWarps, 0, st>>>(a);
  return cudaGetLastError();
}

int apply(BuildCtx* c, const unify_build_view_t* v, const int64_t* g_chunk, const int64_t* g_start, int64_t ngroups,
          const int32_t* r_v, const float* r_d) {
  if (c->prop_first < 0 || c->prop_first != v->first)
    return bfail(UNIFY_E_ARG, "unify_build_apply: no proposals for this batch");
  if (ngroups < 0 || (ngroups > 0 && (!g_chunk || !g_start)) || !g_start)
    return bfail(UNIFY_E_ARG, "unify_build_apply: bad groups");
  if (g_start[0] != 0) return bfail(UNIFY_E_ARG, "unify_build_apply: group_start[0] must be 0");
  for (int64_t g = 0; g < ngroups; ++g) {
    if (g_chunk[g] < 0 || g_chunk[g] >= c->nrows * c->S)
      return bfail(UNIFY_E_ARG, "unify_build_apply: group chunk out of range");
    if (g_start[g + 1] < g_start[g]) return bfail(UNIFY_E_ARG, "unify_build_apply: group_start not ascending");
  }
  const int64_t nrev = g_start[ngroups];
  if (nrev > 0 && (!r_v || !r_d)) return bfail(UNIFY_E_ARG, "unify_build_apply: null edges");
  for (int64_t i = 0; i < nrev; ++i)
    if (r_v[i] < 0 || r_v[i] >= c->n) return bfail(UNIFY_E_ARG, "unify_build_apply: source out of range");
  // forward lists of the batch from the device copy of its proposals
  store_forward<<<1024, 256, 0, c->st>>>(c->o_ids, c->o_dist, c->o_cnt, c->prop_rows * c->S, c->M,
                                         c->prop_row_first * c->S, c->adj, c->adjd, c->cnt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bcuda_fail(e, "unify_build_apply: forward lists");
  c->prop_first = -1;
  if (ngroups == 0) {
    e = cudaStreamSynchronize(c->st);
    return e == cudaSuccess ? UNIFY_OK : bcuda_fail(e, "unify_build_apply");
  }
  e = grow(c->g_chunk, c->g_cap, ngroups);
  if (e == cudaSuccess) e = grow(c->g_start, c->g_cap_s, ngroups + 1);
  if (e == cudaSuccess) e = grow(c->r_v, c->r_cap, nrev);
  if (e == cudaSuccess) e = grow(c->r_d, c->r_cap_d, nrev);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->g_chunk, g_chunk, ngroups * 8, cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->g_start, g_start, (ngroups + 1) * 8, cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess && nrev > 0) e = cudaMemcpyAsync(c->r_v, r_v, nrev * 4, cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess && nrev > 0) e = cudaMemcpyAsync(c->r_d, r_d, nrev * 4, cudaMemcpyHostToDevice, c->st);
  if (e != cudaSuccess) return bcuda_fail(e, "unify_build_apply: edge upload");
  RevArgs a;
  a.X = c->X;
  a.dp4 = c->dp / 4;
  a.M = c->M;
  a.adj = c->adj;
  a.adjd = c->adjd;
  a.cnt = c->cnt;
  a.g_chunk = c->g_chunk;
  a.g_start = c->g_start;
  a.ngroups = ngroups;
  a.r_v = c->r_v;
  a.r_d = c->r_d;
  const int chn = (a.dp4 + 31) / 32;
  if (chn <= 1) e = launch_reverse<1, 16>(a, c->st);
  else if (chn <= 2) e = launch_reverse<2, 8>(a, c->st);
  else if (chn <= 4) e = launch_reverse<4, 4>(a, c->st);
  else e = launch_reverse<8, 2>(a, c->st);
  if (e != cudaSuccess) return bcuda_fail(e, "unify_build_apply: reverse-edge kernel");
  e = cudaStreamSynchronize(c->st);
  return e == cudaSuccess ? UNIFY_OK : bcuda_fail(e, "unify_build_apply");
}

}  // namespace
}  // namespace unify

using namespace unify;

extern "C" int unify_build_assist_create(int device, void** ctx) {
  if (!ctx) return bfail(UNIFY_E_ARG, "unify_build_assist_create: null ctx");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return bcuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return bfail(UNIFY_E_ARG, "unify_build_assist_create: bad device");
  BuildCtx* c = new (std::nothrow) BuildCtx();
  if (!c) return bfail(UNIFY_E_NOMEM, "unify_build_assist_create: host allocation");
  c->device = device;
  *ctx = c;
  return UNIFY_OK;
}

extern "C" void unify_build_assist_destroy(void* ctx) {
  if (!ctx) return;
  BuildCtx* c = static_cast<BuildCtx*>(ctx);
  DeviceGuard guard(c->device);
  build_free(c);
  delete c;
}

extern "C" int unify_build_apply(void* ctx, const unify_build_view_t* view, const int64_t* group_chunk,
                                 const int64_t* group_start, int64_t ngroups, const int32_t* rev_v,
                                 const float* rev_dist) {
  if (!ctx || !view) return bfail(UNIFY_E_ARG, "unify_build_apply: null pointer");
  BuildCtx* c = static_cast<BuildCtx*>(ctx);
  if (!c->ready) return bfail(UNIFY_E_ARG, "unify_build_apply: no preceding unify_build_propose");
  DeviceGuard guard(c->device);
  return apply(c, view, group_chunk, group_start, ngroups, rev_v, rev_dist);
}

extern "C" int unify_build_fetch(void* ctx, const unify_build_view_t* view, int32_t* adj, float* adjd, uint8_t* cnt) {
  if (!ctx || !view || !adj || !adjd || !cnt) return bfail(UNIFY_E_ARG, "unify_build_fetch: null pointer");
  BuildCtx* c = static_cast<BuildCtx*>(ctx);
  if (!c->ready) return bfail(UNIFY_E_ARG, "unify_build_fetch: no preceding unify_build_propose");
  if (view->nrows != c->nrows || view->S != c->S || view->M != c->M)
    return bfail(UNIFY_E_ARG, "unify_build_fetch: the view changed shape");
  DeviceGuard guard(c->device);
  const size_t slots = (size_t)c->nrows * c->S * c->M;
  cudaError_t e = cudaMemcpyAsync(adj, c->adj, slots * 4, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(adjd, c->adjd, slots * 4, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, c->cnt, (size_t)c->nrows * c->S, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  return e == cudaSuccess ? UNIFY_OK : bcuda_fail(e, "unify_build_fetch");
}

extern "C" int unify_build_propose(void* ctx, const unify_build_view_t* view, int32_t* out_ids, float* out_dist,
                                   uint8_t* out_cnt) {
  if (!ctx || !view || !out_ids || !out_dist || !out_cnt) return bfail(UNIFY_E_ARG, "unify_build_propose: null pointer");
  if (view->M < 1 || view->M > kBuildMaxM || view->efc < 1 || view->efc > kBuildMaxEf || view->d < 1 ||
      view->d > 1024 || view->S < 1 || view->S > kBuildMaxS)
    return bfail(UNIFY_E_LIMIT, "unify_build_propose: needs M <= 32, efc <= 256, d <= 1024, S <= 32");
  if (view->first < 0 || view->count < 0 || view->first + view->count > view->n)
    return bfail(UNIFY_E_ARG, "unify_build_propose: batch out of range");
  BuildCtx* c = static_cast<BuildCtx*>(ctx);
  if (c->ready && (view->n != c->n || view->nrows != c->nrows || view->S != c->S || view->M != c->M || view->d != c->d))
    return bfail(UNIFY_E_ARG, "unify_build_propose: the view changed shape");
  DeviceGuard guard(c->device);
  return propose(c, view, out_ids, out_dist, out_cnt);
}
