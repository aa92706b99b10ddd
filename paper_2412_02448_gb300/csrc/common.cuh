// Warp-level device primitives shared by the search kernels.
//
// Keys: a candidate (distance, id) is packed into one uint64 as
// (bits of the non-negative float32 distance) << 32 | id. For non-negative
// floats the IEEE bit pattern orders like the value, so comparing keys compares
// (distance, id) lexicographically: the tie rule "equal distance -> smaller id".
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace unify {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint64_t kKeyMax = ~0ull;

__device__ __forceinline__ uint64_t make_key(float d, int32_t id) {
  return ((uint64_t)__float_as_uint(d) << 32) | (uint32_t)id;
}
__device__ __forceinline__ float key_dist(uint64_t k) { return __uint_as_float((uint32_t)(k >> 32)); }
__device__ __forceinline__ int32_t key_id(uint64_t k) { return (int32_t)(uint32_t)(k & 0xffffffffu); }

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

// Bitonic sort of one key per lane, ascending across lanes 0..31.
__device__ __forceinline__ uint64_t warp_sort_asc(uint64_t x) {
  const int lane = lane_id();
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      uint64_t y = __shfl_xor_sync(kFull, x, j);
      bool up = (lane & k) == 0;
      bool lower = (lane & j) == 0;
      x = (lower == up) ? (x < y ? x : y) : (x < y ? y : x);
    }
  }
  return x;
}

// The same network carrying a 32-bit payload with each key.
__device__ __forceinline__ void warp_sort_asc_payload(uint64_t& x, uint32_t& f) {
  const int lane = lane_id();
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const uint64_t y = __shfl_xor_sync(kFull, x, j);
      const uint32_t g = __shfl_xor_sync(kFull, f, j);
      const bool up = (lane & k) == 0;
      const bool lower = (lane & j) == 0;
      const bool take = (lower == up) ? (y < x) : (x < y);
      if (take) {
        x = y;
        f = g;
      }
    }
  }
}

// The keys of the lanes in kb (a ballot; the other lanes hold kKeyMax), distinct,
// sorted ascending into lanes 0 .. popc(kb) - 1 with their payloads; the other lanes
// end with kKeyMax and payload 0. Up to four keys take their rank among the kept keys
// by broadcast comparisons and move in one shuffle; more go through the bitonic
// network. Both give the same lanes.
__device__ __forceinline__ void warp_sort_kept(uint64_t& x, uint32_t& f, unsigned kb) {
  const int nk = __popc(kb);
  if (nk > 4) {
    warp_sort_asc_payload(x, f);
    return;
  }
  const int lane = lane_id();
  const bool mine = (kb >> lane) & 1u;
  int rank = 0;
  for (unsigned rest = kb; rest; rest &= rest - 1) {
    const uint64_t y = __shfl_sync(kFull, x, __ffs(rest) - 1);
    rank += y < x;
  }
  int src = lane;
  for (int r = 0; r < nk; ++r) {
    const unsigned b = __ballot_sync(kFull, mine && rank == r);
    if (lane == r) src = __ffs(b) - 1;
  }
  const uint64_t y = __shfl_sync(kFull, x, src);
  const uint32_t g = __shfl_sync(kFull, f, src);
  x = lane < nk ? y : kKeyMax;
  f = lane < nk ? g : 0u;
}

__device__ __forceinline__ uint64_t warp_sort_kept(uint64_t x, unsigned kb) {
  uint32_t f = 0;
  warp_sort_kept(x, f, kb);
  return x;
}

// First index i in a[0, n) with a[i] >= x (per lane).
__device__ __forceinline__ int lower_bound_u64(const uint64_t* a, int n, uint64_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// First index i in a[0, n) with a[i] > x (per lane).
__device__ __forceinline__ int upper_bound_u64(const uint64_t* a, int n, uint64_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ bool contains_u64(const uint64_t* a, int n, uint64_t x) {
  int i = lower_bound_u64(a, n, x);
  return i < n && a[i] == x;
}

// Merges a sorted batch into the sorted array arr[0, n) of capacity cap, in place.
// Every lane of the warp calls it. Lane i < nb holds the i-th smallest batch key
// (distinct from every arr entry); the other lanes hold kKeyMax. Entries that fall
// beyond cap are dropped (the largest ones). flags (may be null) move with their
// keys; new entries get flag 0. R is 32 ints of per-warp shared scratch. rank, when
// given (>= 0 on the lanes < nb), is lower_bound(arr, n, bk), already known.
// Returns the new size; *r0 = rank of the smallest batch key in the old array
// (entries below r0 did not move); *dropped = some entry fell beyond cap.
__device__ __forceinline__ int warp_merge(uint64_t* arr, uint8_t* flags, int n, int cap, uint64_t bk,
                                          int nb, int* R, int* r0_out, bool* dropped, int rank = -1) {
  const int lane = lane_id();
  int r = (lane < nb) ? (rank >= 0 ? rank : lower_bound_u64(arr, n, bk)) : n;
  R[lane] = r;
  __syncwarp();
  const int r0 = __shfl_sync(kFull, r, 0);
  if (n > 0 && nb > 0) {
    for (int base = (n - 1) & ~31; base >= (r0 & ~31); base -= 32) {
      int j = base + lane;
      bool act = j >= r0 && j < n;
      uint64_t v = 0;
      uint8_t f = 0;
      int dst = 0;
      if (act) {
        int a = 0, b = nb;  // number of batch keys with rank <= j
        while (a < b) {
          int mid = (a + b) >> 1;
          if (R[mid] <= j) a = mid + 1; else b = mid;
        }
        dst = j + a;
        v = arr[j];
        if (flags) f = flags[j];
      }
      __syncwarp();
      if (act && dst < cap) {
        arr[dst] = v;
        if (flags) flags[dst] = f;
      }
      __syncwarp();
    }
  }
  if (lane < nb) {
    int dst = r + lane;
    if (dst < cap) {
      arr[dst] = bk;
      if (flags) flags[dst] = 0;
    }
  }
  __syncwarp();
  *r0_out = r0;
  *dropped = (n + nb) > cap;
  return (n + nb) < cap ? (n + nb) : cap;
}

// Transposed warp reduction of V partial values per lane (V in {2, 4, 8, 16, 32}).
// Afterwards the lanes whose index >> log2(32/V) equals u hold the sum over all
// 32 lanes of value u. Every value is summed by the same tree (pairs across lane
// bit 4, then bit 3, ..., bit 0), so a vector's distance does not depend on the
// slot it was computed in.
template <int V>
__device__ __forceinline__ float warp_transpose_reduce(float (&v)[V]) {
  const int lane = lane_id();
  int off = 16;
#pragma unroll
  for (int cnt = V; cnt > 1; cnt >>= 1, off >>= 1) {
    const int half = cnt >> 1;
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      float send = up ? v[i] : v[i + half];
      float keep = up ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(kFull, send, off);
    }
  }
#pragma unroll
  for (; off >= 1; off >>= 1) v[0] += __shfl_xor_sync(kFull, v[0], off);
  return v[0];
}

// Vector storage formats. A row is dp4 chunks of 4 elements; lane L handles chunks
// L, L + 32, ... in every format, so the query registers and the reduction tree
// are the same and only the load width differs (16, 8 or 4 bytes per chunk).
//
// Raw is a chunk as loaded (16, 8 or 4 bytes: 4, 2 or 1 registers); decode() turns it
// into four floats. Distance groups and the pre-filter scan's load batches hold what
// kHoldRaw says: raw bfloat16 chunks, decoded at use, let a scan batch hold all 32
// rows of a step in 64 registers; FP8 rows are decoded at load (measured on GB300:
// raw bfloat16 about 5 % faster on mixed batches, raw FP8 about 6 % slower).
struct StoreF32 {
  static constexpr int kChunkBytes = 16;
  static constexpr bool kScaled = false;
  using Raw = float4;
  static constexpr int kRawRegs = 4;
  static constexpr bool kHoldRaw = true;
  __device__ static __forceinline__ Raw load_raw(const unsigned char* row, int c) {
    return __ldg(reinterpret_cast<const float4*>(row) + c);
  }
  __device__ static __forceinline__ Raw zero_raw() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ static __forceinline__ float4 decode(const Raw& r) { return r; }
  __device__ static __forceinline__ float4 load(const unsigned char* row, int c, float) {
    return __ldg(reinterpret_cast<const float4*>(row) + c);
  }
};
struct StoreBF16 {  // bfloat16, converted from float32 with round-to-nearest-even
  static constexpr int kChunkBytes = 8;
  static constexpr bool kScaled = false;
  using Raw = uint2;
  static constexpr int kRawRegs = 2;
  static constexpr bool kHoldRaw = true;
  __device__ static __forceinline__ Raw load_raw(const unsigned char* row, int c) {
    return __ldg(reinterpret_cast<const uint2*>(row) + c);
  }
  __device__ static __forceinline__ Raw zero_raw() { return make_uint2(0u, 0u); }
  __device__ static __forceinline__ float4 decode(const Raw& u) {
    // a bfloat16 is the upper half of a float32
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
  }
  __device__ static __forceinline__ float4 load(const unsigned char* row, int c, float) {
    return decode(load_raw(row, c));
  }
};
// E4M3 codes of x / s with s = max|x| / 448 per vector. load() returns the decoded
// codes without the scale: the distance loops apply s inside their first FMA
// (q - s x as one fused operation, see diff4), so the scale costs no multiply.
struct StoreFP8 {
  static constexpr int kChunkBytes = 4;
  static constexpr bool kScaled = true;
  using Raw = uint32_t;
  static constexpr int kRawRegs = 1;
  static constexpr bool kHoldRaw = false;
  __device__ static __forceinline__ Raw load_raw(const unsigned char* row, int c) {
    return __ldg(reinterpret_cast<const uint32_t*>(row) + c);
  }
  __device__ static __forceinline__ Raw zero_raw() { return 0u; }
  __device__ static __forceinline__ float4 decode(const Raw& u) {
    const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u & 0xffffu), __NV_E4M3);
    const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u >> 16), __NV_E4M3);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&lo));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&hi));
    return make_float4(a.x, a.y, b.x, b.y);
  }
  __device__ static __forceinline__ float4 load(const unsigned char* row, int c, float) {
    return decode(load_raw(row, c));
  }
};

// A chunk as a distance group holds it (raw, or decoded at load) and its value.
template <class T>
using Held = typename std::conditional<T::kHoldRaw, typename T::Raw, float4>::type;
template <class T>
__device__ __forceinline__ float4 unhold(const Held<T>& h) {
  if constexpr (T::kHoldRaw) return T::decode(h);
  else return h;
}

// q - x for a chunk loaded by T::load: for scaled formats x holds codes and the
// difference is q - scale * code, fused.
template <class T>
__device__ __forceinline__ float4 diff4(const float4& q, const float4& x, float scale) {
  if constexpr (T::kScaled) {
    return make_float4(fmaf(-scale, x.x, q.x), fmaf(-scale, x.y, q.y), fmaf(-scale, x.z, q.z),
                       fmaf(-scale, x.w, q.w));
  } else {
    return make_float4(q.x - x.x, q.y - x.y, q.z - x.z, q.w - x.w);
  }
}

// The value of a chunk loaded by T::load (the scale applied for scaled formats).
template <class T>
__device__ __forceinline__ float4 value4(const float4& x, float scale) {
  if constexpr (T::kScaled) return make_float4(scale * x.x, scale * x.y, scale * x.z, scale * x.w);
  else return x;
}

// Squared-L2 partial of one lane over its chunks of a row in storage format T.
template <class T, int CH>
__device__ __forceinline__ float l2_partial_t(const float4 (&q)[CH], const unsigned char* row, int nchunks,
                                              float scale) {
  const int lane = lane_id();
  float s = 0.f;
#pragma unroll
  for (int t = 0; t < CH; ++t) {
    int c = lane + 32 * t;
    if (c < nchunks) {
      const float4 e = diff4<T>(q[t], T::load(row, c, scale), scale);
      s = fmaf(e.x, e.x, s);
      s = fmaf(e.y, e.y, s);
      s = fmaf(e.z, e.z, s);
      s = fmaf(e.w, e.w, s);
    }
  }
  return s;
}

// Loads the query into the per-lane chunks (zero beyond d).
template <int CH>
__device__ __forceinline__ void load_query(float4 (&q)[CH], const float* qrow, int d) {
  const int lane = lane_id();
#pragma unroll
  for (int t = 0; t < CH; ++t) {
    int c = (lane + 32 * t) * 4;
    q[t].x = c + 0 < d ? qrow[c + 0] : 0.f;
    q[t].y = c + 1 < d ? qrow[c + 1] : 0.f;
    q[t].z = c + 2 < d ? qrow[c + 2] : 0.f;
    q[t].w = c + 3 < d ? qrow[c + 3] : 0.f;
  }
}

}  // namespace unify
