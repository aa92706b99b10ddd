// Index loading: parses the serialised HSIG, validates it so that every index a
// kernel derives from it stays inside its buffer, and places it in device memory.
//
// File layout: "UNIFYHSG", u32 version (1), u32 section count, then 96-byte
// entries {char name[24]; u32 dtype; u32 ndim; u64 shape[4]; u64 offset;
// u64 nbytes; u64 checksum; u64 reserved}; payloads are 64-byte aligned. The
// checksum is FNV-1a (64-bit) over little-endian 8-byte words, the last one
// zero-padded. dtype codes: 1 i8, 2 u8, 3 i32, 4 u32, 5 i64, 6 f32.
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace unify {

namespace {

struct Entry {
  std::string name;
  uint32_t dtype = 0, ndim = 0;
  uint64_t shape[4] = {0, 0, 0, 0};
  uint64_t off = 0, nbytes = 0, ck = 0;
};

uint64_t fnv1a64_words(const unsigned char* p, uint64_t nbytes) {
  uint64_t h = 0xcbf29ce484222325ull;
  uint64_t i = 0;
  for (; i + 8 <= nbytes; i += 8) {
    uint64_t w;
    std::memcpy(&w, p + i, 8);
    h ^= w;
    h *= 0x100000001b3ull;
  }
  if (i < nbytes) {
    uint64_t w = 0;
    std::memcpy(&w, p + i, nbytes - i);
    h ^= w;
    h *= 0x100000001b3ull;
  }
  return h;
}

struct FileView {
  std::vector<unsigned char> bytes;
  std::vector<Entry> entries;

  const Entry* find(const char* name) const {
    for (const Entry& e : entries)
      if (e.name == name) return &e;
    return nullptr;
  }
};

int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

// Returns a pointer to a validated section with the given dtype and element count.
template <typename T>
const T* section(const FileView& f, const char* name, uint32_t dtype, uint64_t elems, std::string& err) {
  const Entry* e = f.find(name);
  if (!e) { err = std::string("missing section ") + name; return nullptr; }
  if (e->dtype != dtype) { err = std::string("bad dtype in section ") + name; return nullptr; }
  uint64_t cnt = 1;
  for (uint32_t k = 0; k < e->ndim; ++k) cnt *= e->shape[k];
  if (cnt != elems || e->nbytes != elems * sizeof(T)) { err = std::string("bad shape in section ") + name; return nullptr; }
  if (e->off % 64 || e->off + e->nbytes > f.bytes.size()) { err = std::string("bad offset in section ") + name; return nullptr; }
  if (fnv1a64_words(f.bytes.data() + e->off, e->nbytes) != e->ck) { err = std::string("checksum mismatch in section ") + name; return nullptr; }
  return reinterpret_cast<const T*>(f.bytes.data() + e->off);
}

__global__ void derive_kernel(const float* __restrict__ vec, const int32_t* __restrict__ sorted_ids,
                              const int64_t* __restrict__ attr, int64_t n, int dp, float* vec_sorted,
                              int64_t* sorted_attr, int32_t* pos) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = sorted_ids[p];
    pos[v] = (int32_t)p;
    sorted_attr[p] = attr[v];
  }
  // rows: one warp per row, float4 copies
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n; p += warps) {
    const int32_t v = sorted_ids[p];
    const float4* src = reinterpret_cast<const float4*>(vec + (int64_t)v * dp);
    float4* dst = reinterpret_cast<float4*>(vec_sorted + p * dp);
    for (int c = lane; c < dp / 4; c += 32) dst[c] = src[c];
  }
}

// Reduced-precision copies, one warp per attribute-order position p (object v):
// bfloat16 by round-to-nearest-even; FP8 E4M3 codes of x / s (saturating,
// round-to-nearest-even) with s = max|x| / 448 (s = 1 for an all-zero vector). Also
// the squared norms, in attribute order, of the bfloat16 rows, the float32 rows and
// the decoded FP8 rows (s * code), which the tensor-core scan of each format uses.
__device__ __forceinline__ float fp8_value(uint32_t code) {
  const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)(code & 0xffu), __NV_E4M3);
  return __half2float(*reinterpret_cast<const __half*>(&h));
}

__global__ void lowp_kernel(const float* __restrict__ vec, const int32_t* __restrict__ sorted_ids, int64_t n,
                            int dp, uint2* bf_id, uint2* bf_sorted, uint32_t* f8_id, uint32_t* f8_sorted,
                            float* sc_id, float* sc_sorted, float* xn_sorted, float* xn32_sorted,
                            float* xn8_sorted) {
  const int lane = threadIdx.x & 31;
  const int dp4 = dp / 4;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n; p += warps) {
    const int32_t v = sorted_ids[p];
    const float4* row = reinterpret_cast<const float4*>(vec + (int64_t)v * dp);
    float mx = 0.f;
    for (int c = lane; c < dp4; c += 32) {
      const float4 x = row[c];
      mx = fmaxf(mx, fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w))));
    }
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    const float s = mx > 0.f ? mx / 448.f : 1.f;
    float nn = 0.f, n32 = 0.f, n8 = 0.f;  // squared norms: bfloat16, float32, decoded FP8 rows
    for (int c = lane; c < dp4; c += 32) {
      const float4 x = row[c];
      uint2 b;
      b.x = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x.x)) |
            ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x.y)) << 16);
      b.y = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x.z)) |
            ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x.w)) << 16);
      const uint32_t f = (uint32_t)__nv_cvt_float_to_fp8(x.x / s, __NV_SATFINITE, __NV_E4M3) |
                         ((uint32_t)__nv_cvt_float_to_fp8(x.y / s, __NV_SATFINITE, __NV_E4M3) << 8) |
                         ((uint32_t)__nv_cvt_float_to_fp8(x.z / s, __NV_SATFINITE, __NV_E4M3) << 16) |
                         ((uint32_t)__nv_cvt_float_to_fp8(x.w / s, __NV_SATFINITE, __NV_E4M3) << 24);
      const float b0 = __uint_as_float(b.x << 16), b1 = __uint_as_float(b.x & 0xffff0000u);
      const float b2 = __uint_as_float(b.y << 16), b3 = __uint_as_float(b.y & 0xffff0000u);
      nn = fmaf(b0, b0, nn);
      nn = fmaf(b1, b1, nn);
      nn = fmaf(b2, b2, nn);
      nn = fmaf(b3, b3, nn);
      n32 = fmaf(x.x, x.x, n32);
      n32 = fmaf(x.y, x.y, n32);
      n32 = fmaf(x.z, x.z, n32);
      n32 = fmaf(x.w, x.w, n32);
      for (int t = 0; t < 4; ++t) {
        const float e = s * fp8_value(f >> (8 * t));
        n8 = fmaf(e, e, n8);
      }
      bf_id[(int64_t)v * dp4 + c] = b;
      bf_sorted[p * dp4 + c] = b;
      f8_id[(int64_t)v * dp4 + c] = f;
      f8_sorted[p * dp4 + c] = f;
    }
    for (int off = 16; off > 0; off >>= 1) {
      nn += __shfl_xor_sync(0xffffffffu, nn, off);
      n32 += __shfl_xor_sync(0xffffffffu, n32, off);
      n8 += __shfl_xor_sync(0xffffffffu, n8, off);
    }
    if (lane == 0) {
      sc_id[v] = s;
      sc_sorted[p] = s;
      xn_sorted[p] = nn;
      xn32_sorted[p] = n32;
      xn8_sorted[p] = n8;
    }
  }
}

void free_device(DeviceIndex& ix) {
  void* ptrs[] = {ix.vec, ix.vec_sorted, ix.sorted_ids, ix.sorted_attr, ix.pos, ix.upper_base, ix.adj0,
                  ix.gmask0, ix.adjU, ix.gmaskU, ix.seg_bounds, ix.seg_start, ix.vt_bf16, ix.vts_bf16,
                  ix.vt_fp8, ix.vts_fp8, ix.scale_fp8, ix.scale_fp8_sorted, ix.xn_bf16_sorted,
                  ix.xn_f32_sorted, ix.xn_fp8_sorted};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  ix.vt_bf16 = ix.vts_bf16 = ix.vt_fp8 = ix.vts_fp8 = nullptr;
  ix.scale_fp8 = ix.scale_fp8_sorted = ix.xn_bf16_sorted = ix.xn_f32_sorted = ix.xn_fp8_sorted = nullptr;
  ix.vec = ix.vec_sorted = nullptr;
  ix.sorted_ids = ix.pos = ix.upper_base = ix.adj0 = ix.adjU = ix.seg_start = nullptr;
  ix.sorted_attr = ix.seg_bounds = nullptr;
  ix.gmask0 = ix.gmaskU = nullptr;
}

template <typename T>
cudaError_t upload(T** dst, const T* src, uint64_t elems) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), elems * sizeof(T) > 0 ? elems * sizeof(T) : 16);
  if (e != cudaSuccess) return e;
  if (elems) e = cudaMemcpy(*dst, src, elems * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

// An attribute-ordered per-row array with kTcRowPad zero entries past the last row.
template <class T>
cudaError_t alloc_rows(T** dst, uint64_t n) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), (n + kTcRowPad) * sizeof(T));
  if (e == cudaSuccess) e = cudaMemset(*dst, 0, (n + kTcRowPad) * sizeof(T));
  return e;
}

}  // namespace

void free_scratch(Scratch& sc);

}  // namespace unify

using namespace unify;

extern "C" int unify_load_index(const char* path, int device, unify_index_t** out) {
  if (!path || !out) return fail(UNIFY_E_ARG, "unify_load_index: null argument");
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return fail(UNIFY_E_ARG, "unify_load_index: no such CUDA device");
  FileView f;
  {
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(UNIFY_E_IO, std::string("cannot open ") + path);
    std::fseek(fp, 0, SEEK_END);
    long sz = std::ftell(fp);
    std::rewind(fp);
    if (sz < 16) { std::fclose(fp); return fail(UNIFY_E_FORMAT, "index file too short"); }
    f.bytes.resize((size_t)sz);
    size_t got = std::fread(f.bytes.data(), 1, (size_t)sz, fp);
    std::fclose(fp);
    if (got != (size_t)sz) return fail(UNIFY_E_IO, "short read of index file");
  }
  uint32_t version = 0, nsec = 0;
  std::memcpy(&version, f.bytes.data() + 8, 4);
  std::memcpy(&nsec, f.bytes.data() + 12, 4);
  if (std::memcmp(f.bytes.data(), "UNIFYHSG", 8) != 0) return fail(UNIFY_E_FORMAT, "bad magic");
  if (version != 1) return fail(UNIFY_E_FORMAT, "unsupported index version");
  if (16 + 96ull * nsec > f.bytes.size()) return fail(UNIFY_E_FORMAT, "truncated section table");
  for (uint32_t s = 0; s < nsec; ++s) {
    const unsigned char* e = f.bytes.data() + 16 + 96ull * s;
    Entry en;
    char nm[25];
    std::memcpy(nm, e, 24);
    nm[24] = 0;
    en.name = nm;
    std::memcpy(&en.dtype, e + 24, 4);
    std::memcpy(&en.ndim, e + 28, 4);
    std::memcpy(en.shape, e + 32, 32);
    std::memcpy(&en.off, e + 64, 8);
    std::memcpy(&en.nbytes, e + 72, 8);
    std::memcpy(&en.ck, e + 80, 8);
    if (en.ndim < 1 || en.ndim > 4) return fail(UNIFY_E_FORMAT, "bad section rank");
    f.entries.push_back(en);
  }
  std::string err;
  const int64_t* meta = section<int64_t>(f, "meta", 5, 16, err);
  if (!meta) return fail(UNIFY_E_FORMAT, err);
  DeviceIndex ix;
  ix.device = device;
  ix.n = meta[0];
  ix.d = (int)meta[1];
  ix.S = (int)meta[2];
  ix.M = (int)meta[3];
  ix.max_level = (int)meta[4];
  ix.entry_global = (int)meta[5];
  ix.n_upper = meta[6];
  ix.W = (int)meta[9];
  if (ix.n < 1 || ix.n >= (1ll << 30)) return fail(UNIFY_E_LIMIT, "n must be in [1, 2^30)");
  if (ix.d < 1 || ix.d > 1024) return fail(UNIFY_E_LIMIT, "d must be in [1, 1024]");
  if (ix.S < 1 || ix.S > kMaxS) return fail(UNIFY_E_LIMIT, "S must be in [1, 32]");
  if (ix.M < 1 || ix.M > 255) return fail(UNIFY_E_LIMIT, "M must be in [1, 255]");
  if (ix.W != (ix.S * ix.M + 31) / 32) return fail(UNIFY_E_FORMAT, "bad bitmap width");
  if (ix.max_level < 0 || ix.max_level > 30 || ix.n_upper < 0) return fail(UNIFY_E_FORMAT, "bad levels");
  if (ix.entry_global < 0 || ix.entry_global >= ix.n) return fail(UNIFY_E_FORMAT, "bad entry point");
  const uint64_t n = (uint64_t)ix.n, SM = (uint64_t)ix.S * ix.M;
  const uint64_t nu = ix.n_upper > 0 ? (uint64_t)ix.n_upper : 1;
  const float* vectors = section<float>(f, "vectors", 6, n * ix.d, err);
  const int64_t* attr = vectors ? section<int64_t>(f, "attr", 5, n, err) : nullptr;
  const int32_t* level = attr ? section<int32_t>(f, "level", 3, n, err) : nullptr;
  const int32_t* upper_base = level ? section<int32_t>(f, "upper_base", 3, n, err) : nullptr;
  const int64_t* seg_bounds = upper_base ? section<int64_t>(f, "seg_bounds", 5, ix.S + 1, err) : nullptr;
  const int64_t* seg_count = seg_bounds ? section<int64_t>(f, "seg_count", 5, ix.S, err) : nullptr;
  const int32_t* sorted_ids = seg_count ? section<int32_t>(f, "sorted_ids", 3, n, err) : nullptr;
  const int32_t* adj0 = sorted_ids ? section<int32_t>(f, "adj0", 3, n * SM, err) : nullptr;
  const uint32_t* gmask0 = adj0 ? section<uint32_t>(f, "gmask0", 4, n * ix.W, err) : nullptr;
  const int32_t* adjU = gmask0 ? section<int32_t>(f, "adjU", 3, nu * SM, err) : nullptr;
  const uint32_t* gmaskU = adjU ? section<uint32_t>(f, "gmaskU", 4, nu * ix.W, err) : nullptr;
  if (!gmaskU) return fail(UNIFY_E_FORMAT, err);

  // --- validation: every id, row and position a kernel derives stays in bounds
  std::vector<unsigned char> seen(n, 0);
  for (uint64_t p = 0; p < n; ++p) {
    int32_t v = sorted_ids[p];
    if (v < 0 || (uint64_t)v >= n || seen[v]) return fail(UNIFY_E_FORMAT, "sorted_ids is not a permutation");
    seen[v] = 1;
    if (p > 0) {
      int32_t u = sorted_ids[p - 1];
      if (attr[u] > attr[v] || (attr[u] == attr[v] && u > v)) return fail(UNIFY_E_FORMAT, "sorted_ids not in attribute order");
    }
  }
  int64_t total = 0;
  ix.h_seg_start[0] = 0;
  for (int j = 0; j < ix.S; ++j) {
    if (seg_count[j] < 0) return fail(UNIFY_E_FORMAT, "negative segment count");
    total += seg_count[j];
    ix.h_seg_start[j + 1] = (int32_t)total;
  }
  if (total != ix.n) return fail(UNIFY_E_FORMAT, "segment counts do not sum to n");
  for (int j = 0; j <= ix.S; ++j) ix.h_seg_bounds[j] = seg_bounds[j];
  for (int j = 1; j <= ix.S; ++j)
    if (seg_bounds[j] < seg_bounds[j - 1]) return fail(UNIFY_E_FORMAT, "segment bounds not sorted");
  for (int j = 0; j < ix.S; ++j)
    for (int64_t p = ix.h_seg_start[j]; p < ix.h_seg_start[j + 1]; ++p) {
      int64_t a = attr[sorted_ids[p]];
      if ((j > 0 && a < seg_bounds[j]) || (j < ix.S - 1 && a >= seg_bounds[j + 1]))
        return fail(UNIFY_E_FORMAT, "segment counts disagree with the bounds");
    }
  int max_lv = 0;
  int64_t upper_rows = 0;
  for (uint64_t v = 0; v < n; ++v) {
    if (level[v] < 0 || level[v] > ix.max_level) return fail(UNIFY_E_FORMAT, "bad node level");
    max_lv = level[v] > max_lv ? level[v] : max_lv;
    if (level[v] > 0) {
      if (upper_base[v] != upper_rows) return fail(UNIFY_E_FORMAT, "upper rows not laid out by id");
      upper_rows += level[v];
    } else if (upper_base[v] != -1) {
      return fail(UNIFY_E_FORMAT, "level-0 node with upper rows");
    }
  }
  if (max_lv != ix.max_level || upper_rows != ix.n_upper || level[ix.entry_global] != ix.max_level)
    return fail(UNIFY_E_FORMAT, "levels disagree with the header");
  for (uint64_t e = 0; e < n * SM; ++e)
    if (adj0[e] < -1 || adj0[e] >= ix.n) return fail(UNIFY_E_FORMAT, "layer-0 neighbour id out of range");
  for (uint64_t v = 0; v < n; ++v)
    for (int l = 1; l <= level[v]; ++l) {
      const int32_t* row = adjU + ((uint64_t)upper_base[v] + l - 1) * SM;
      for (uint64_t s = 0; s < SM; ++s) {
        int32_t x = row[s];
        if (x < -1 || x >= ix.n || (x >= 0 && level[x] < l))
          return fail(UNIFY_E_FORMAT, "upper-layer neighbour id out of range");
      }
    }

  // --- padded float32 rows (16-byte aligned)
  ix.dp = (ix.d + 3) & ~3;
  std::vector<float> padded;
  const float* vsrc = vectors;
  if (ix.dp != ix.d) {
    padded.assign(n * ix.dp, 0.f);
    for (uint64_t v = 0; v < n; ++v) std::memcpy(&padded[v * ix.dp], vectors + v * ix.d, ix.d * 4);
    vsrc = padded.data();
  }
  DeviceGuard guard(device);
  int64_t* d_attr = nullptr;
  cudaError_t e = upload(&ix.vec, vsrc, n * ix.dp);
  if (e == cudaSuccess) e = upload(&d_attr, attr, n);
  if (e == cudaSuccess) e = alloc_rows(&ix.sorted_ids, n);
  if (e == cudaSuccess) e = cudaMemcpy(ix.sorted_ids, sorted_ids, n * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = upload(&ix.upper_base, upper_base, n);
  if (e == cudaSuccess) e = upload(&ix.adj0, adj0, n * SM);
  if (e == cudaSuccess) e = upload(&ix.gmask0, gmask0, n * ix.W);
  if (e == cudaSuccess) e = upload(&ix.adjU, adjU, nu * SM);
  if (e == cudaSuccess) e = upload(&ix.gmaskU, gmaskU, nu * ix.W);
  if (e == cudaSuccess) e = upload(&ix.seg_bounds, ix.h_seg_bounds, (uint64_t)ix.S + 1);
  if (e == cudaSuccess) e = upload(&ix.seg_start, ix.h_seg_start, (uint64_t)ix.S + 1);
  if (e == cudaSuccess) e = cudaMalloc(&ix.vec_sorted, n * ix.dp * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&ix.sorted_attr, n * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc(&ix.pos, n * sizeof(int32_t));
  const uint64_t dp4 = (uint64_t)ix.dp / 4;
  if (e == cudaSuccess) e = cudaMalloc(&ix.vt_bf16, n * dp4 * 8);
  if (e == cudaSuccess) e = cudaMalloc(&ix.vts_bf16, n * dp4 * 8);
  if (e == cudaSuccess) e = cudaMalloc(&ix.vt_fp8, n * dp4 * 4);
  if (e == cudaSuccess) e = cudaMalloc(&ix.vts_fp8, n * dp4 * 4);
  if (e == cudaSuccess) e = cudaMalloc(&ix.scale_fp8, n * sizeof(float));
  if (e == cudaSuccess) e = alloc_rows(&ix.scale_fp8_sorted, n);
  if (e == cudaSuccess) e = alloc_rows(&ix.xn_bf16_sorted, n);
  if (e == cudaSuccess) e = alloc_rows(&ix.xn_f32_sorted, n);
  if (e == cudaSuccess) e = alloc_rows(&ix.xn_fp8_sorted, n);
  if (e == cudaSuccess) {
    derive_kernel<<<1024, 256>>>(ix.vec, ix.sorted_ids, d_attr, ix.n, ix.dp, ix.vec_sorted, ix.sorted_attr, ix.pos);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    lowp_kernel<<<1024, 256>>>(ix.vec, ix.sorted_ids, ix.n, ix.dp, reinterpret_cast<uint2*>(ix.vt_bf16),
                               reinterpret_cast<uint2*>(ix.vts_bf16), reinterpret_cast<uint32_t*>(ix.vt_fp8),
                               reinterpret_cast<uint32_t*>(ix.vts_fp8), ix.scale_fp8, ix.scale_fp8_sorted,
                               ix.xn_bf16_sorted, ix.xn_f32_sorted, ix.xn_fp8_sorted);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (d_attr) cudaFree(d_attr);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ix.num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    free_device(ix);
    return fail(e == cudaErrorMemoryAllocation ? UNIFY_E_NOMEM : UNIFY_E_CUDA,
                std::string("unify_load_index: ") + cudaGetErrorString(e));
  }
  unify_index_t* h = new (std::nothrow) unify_index_t;
  if (!h) {
    free_device(ix);
    return fail(UNIFY_E_NOMEM, "unify_load_index: host allocation failed");
  }
  h->ix = ix;
  *out = h;
  return UNIFY_OK;
}

extern "C" void unify_free_index(unify_index_t* idx) {
  if (!idx) return;
  {
    DeviceGuard guard(idx->ix.device);
    free_device(idx->ix);
    free_scratch(idx->sc);
    for (int ph = 0; ph < kPhases; ++ph)
      for (auto& pr : idx->tm.rec[ph]) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
      }
    for (cudaEvent_t e : idx->tm.pool) cudaEventDestroy(e);
  }
  delete idx;
}

extern "C" int unify_index_info(const unify_index_t* idx, int64_t* n, int* d, int* S, int* M, int* max_level) {
  if (!idx) return fail(UNIFY_E_ARG, "unify_index_info: null index");
  if (n) *n = idx->ix.n;
  if (d) *d = idx->ix.d;
  if (S) *S = idx->ix.S;
  if (M) *M = idx->ix.M;
  if (max_level) *max_level = idx->ix.max_level;
  return UNIFY_OK;
}
