// Strategy A (pre-filtering, Section 4.2) for many queries at once on the 5th-
// generation tensor cores: queries x in-range vectors is a dense contraction.
//
// Tiles per span. The attribute order is cut into spans of L rows (L a multiple of
// 256, at least 4096, grown when the batch's ranges are long; see span_len). Every
// pre-filter query takes one slot in a tile of every span its range [pa, pb) meets,
// and its vector, converted to the scan's operand format (below), is copied into that
// slot's row of a gathered buffer; a span's covering queries fill ceil(count / 128)
// tiles. So each 256-row block is read by about count / 128 tiles, whatever the mix
// of range widths, instead of by every tile of consecutive queries whose union of
// ranges holds it. A tile's span is split into work units of at most 16 blocks. For a
// block, TMA stages 128-byte slices of K of the tile's gathered query rows and of the
// block's attribute-ordered rows (128-byte swizzled), and tcgen05.mma forms D = Q X^T
// (M = 128 query slots, N = 256 rows, 32 bytes of K per instruction, float32
// accumulation in tensor memory, two accumulators so that the epilogue of one block
// overlaps the products of the next). Tensor-memory lane q is slot q of the tile: its
// epilogue threads turn the slot's dot products into squared distances
// ||x||^2 + ||q||^2 - 2 x.q (norms of the operand values) and keep the rows of the
// query's range.
//
// Two passes over the same tiles select, for every query, the R smallest keys
// (distance, id), R = rerank_mult * k up to 64 and k past that (k <= 128), without any
// per-query heap:
//   1. bounding pass: per query, the minimum distance of each of 128 disjoint row
//      groups over its whole range (group = column half x column mod 64 of a 256-row
//      block; every unit min-merges its minima into the query's 128 with atomicMin).
//      A small kernel then takes the R-th smallest of the 128: R distinct rows lie at
//      or below it, so it bounds the query's R-th smallest key (R <= 128);
//   2. collecting pass: every in-range row whose key is below the bound is appended
//      to the query's list in global memory (an atomic count; about 1.5 R rows per
//      query qualify).
// A finishing kernel takes the R smallest keys of each query's list and re-ranks
// them with exact float32 direct-difference distances against the float32 vectors,
// as the other reduced-precision paths do. A list that overflowed (more than kTcQCap
// rows below the bound) sends that query through an exact warp scan of its range
// instead. On integer-valued vectors of at most 8 bits and d <= 128 every term is an
// exact integer below 2^24, so the result equals the exact float32 scan.
//
// Roles in a CTA of 10 warps: warps 0-7 epilogue (warp w reads tensor-memory
// lanes 32 (w % 4).. 32 (w % 4) + 31, the queries it owns, over column half w / 4 of
// each 256-column block, so that two warps share every scheduler's epilogue work),
// warp 8 lane 0 issues TMA loads, warp 9 lane 0 issues the MMAs and owns the
// tensor-memory allocation. Work units are claimed dynamically: the producer takes
// the next unit from a global counter and hands its index to the MMA issuer and the
// epilogue through a small ring in shared memory (index -1 ends the kernel), so CTAs
// that drew cheap units take more of them. Stages of shared memory (query slice
// 16 KB + row slice 32 KB per 128 bytes of K) are handed over with mbarriers. Every
// wait is bounded (a number of polls and an elapsed time); a timeout sets an error
// flag instead of hanging, the waiting warp stops, and the copies and products in
// flight are drained before the CTA releases its tensor memory and exits.
//
// The epilogues read a chunk of 32 columns at a time. When every lane of the warp
// takes either all 32 columns of the chunk or none of them, the chunk runs without a
// per-column range test: a lane without columns adds NaN to its distances, which
// neither fminf nor the bound's comparison lets through; the rows' norms and ids come
// as broadcast vector loads. Only chunks that hold the end of some lane's range take
// the per-column test.
//
// Bounds (checked against the buffers each launch receives): the span length keeps
// the (query, span) pairs within the scratch's pairs and the tiles within its slots
// (span_len; the tile count is checked again, and an overflow raises the error flag);
// a unit's rows start below n and the attribute-ordered norms, scales and ids hold
// 256 zero entries past n, TMA zero-fills rows past n; the query tiles' TMA rows end
// at the scratch's slots; list stores stop at kTcQCap while the count goes on.

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "warp_ops.cuh"

namespace unify {

namespace {

constexpr int kTcQ = kTcQueryTile;  // queries per tile (MMA M = tensor-memory lanes)
constexpr int kTcRows = 256;        // rows per block (MMA N = tensor-memory columns per accumulator)
constexpr int kTcKb = 128;          // bytes of K per stage (one 128-byte swizzle row)
constexpr int kTcStages = 4;
constexpr int kUnitRing = 4;        // claimed work units handed from the producer to the other roles
constexpr int kEpiWarps = kTcEpiThreads / 32;  // 8 epilogue warps: warp w reads lanes 32 (w % 4).. and column half w / 4
constexpr int kTmaWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1;
constexpr int kTcThreads = 32 * (kEpiWarps + 2);
constexpr int kHalfCols = kTcRows / 2;  // columns of a block per epilogue warp
constexpr int kTcRMax = 128;        // candidates kept per query for the re-rank, at most
constexpr int kTcRTight = 64;       // up to here the bound stays near R rows; past it the scan keeps k
constexpr int kStageA = kTcQ * kTcKb;     // 16 KB of queries
constexpr int kStageB = kTcRows * kTcKb;  // 32 KB of rows

// Operand formats of the scan. Every MMA instruction takes 32 bytes of K, so a stage
// holds four of them whatever the element width:
//   bfloat16  (BF16 storage): kind::f16, K = 16 elements, 64 per stage;
//   tf32      (FP32 storage): kind::tf32, the float32 rows and queries as stored, of
//                             which the tensor cores use the top 19 bits; K = 8, 32
//                             per stage;
//   E4M3      (FP8 storage):  kind::f8f6f4, the stored codes of the rows and E4M3 codes
//                             of the queries (per-query scale max|q| / 448); the dot
//                             product of the codes is scaled by s_q * s_x in the
//                             epilogue; K = 32, 128 per stage.
enum TcFmt { kFmtBF16 = 0, kFmtTF32 = 1, kFmtFP8 = 2 };

template <int F>
struct TcTraits;
template <>
struct TcTraits<kFmtBF16> {
  static constexpr int kElemBytes = 2;
  static constexpr bool kScaled = false;
  // instruction descriptor type fields (A and B): bfloat16
  static constexpr uint32_t kAB = (1u << 7) | (1u << 10);
};
template <>
struct TcTraits<kFmtTF32> {
  static constexpr int kElemBytes = 4;
  static constexpr bool kScaled = false;
  static constexpr uint32_t kAB = (2u << 7) | (2u << 10);  // tf32
};
template <>
struct TcTraits<kFmtFP8> {
  static constexpr int kElemBytes = 1;
  static constexpr bool kScaled = true;
  static constexpr uint32_t kAB = (0u << 7) | (0u << 10);  // E4M3
};
constexpr long long kWaitLimit = 1ll << 22;   // polls
constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s of elapsed time
constexpr uint64_t kTestWaitNs = 50000000ull;  // 50 ms: the limit of the timeout test

struct TcSmem {
  // 1024-byte aligned stages first
  uint8_t a[kTcStages][kStageA];
  uint8_t b[kTcStages][kStageB];
  // per accumulator: the block's squared norms, ids and (FP8) scales, copied by the
  // producer when it starts the block's loads; mfull[i] completes when they landed
  float mxn[2][kTcRows];
  int32_t mid[2][kTcRows];
  float mxs[2][kTcRows];
  uint64_t full[kTcStages], empty[kTcStages], accf[2], acce[2], drain, mfull[2];
  uint64_t never;  // no thread arrives on it (the timeout test waits on it)
  uint64_t ufull[kUnitRing], uempty[kUnitRing];
  int uring[kUnitRing];  // claimed unit (-1: no more units)
  uint32_t tmem;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the completion of the phase with the given parity; false on timeout.
// A few immediate polls, then polls with a growing sleep in between, bounded
// both by the number of polls and by limit_ns of elapsed time.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  const uint32_t addr = smem_u32(bar);
#pragma unroll 1
  for (int i = 0; i < 16; ++i)
    if (mbar_try(addr, parity)) return true;
  const uint64_t t0 = global_ns();
  unsigned ns = 32;
#pragma unroll 1
  for (long long i = 0; i < kWaitLimit; ++i) {
    if (mbar_try(addr, parity)) return true;
    __nanosleep(ns);
    if (ns < 512) ns <<= 1;
    if ((i & 63) == 63 && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// Untiled bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// into shared memory, completing on the mbarrier.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(tm), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand in 128-byte swizzled atoms
// (8 rows x 128 bytes, 1024 bytes apart), start address 1024-byte aligned except
// for the 32-byte steps along K inside an atom.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset: 8-row atoms
  d |= (uint64_t)1 << 46;              // descriptor version
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}

// Instruction descriptor: f32 accumulator, the format's A and B types (the same for
// both), K-major A and B, M = 128, N = 256.
template <int F>
__device__ __forceinline__ uint32_t idesc_of() {
  return (1u << 4) | TcTraits<F>::kAB | ((uint32_t)(kTcRows >> 3) << 17) | ((uint32_t)(kTcQ >> 4) << 24);
}

template <int F>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (F == kFmtBF16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else if constexpr (F == kFmtTF32) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive float32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld32(uint32_t addr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Element i (a constant after unrolling) of a vector of four.
__device__ __forceinline__ float f4_at(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
__device__ __forceinline__ int i4_at(const int4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
__device__ __forceinline__ unsigned u4_at(const uint4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

struct TcArgs {
  const int32_t* sorted_ids;
  const float* xn;     // squared norms of the rows as the scan's format holds them, attribute order
  const float* xs;     // FP8: per-row scales in attribute order (else null)
  const float* vec;    // float32 rows by id (re-rank)
  const unsigned char* vt;  // rows by id in the storage format (scan of an overflowed query)
  const float* vscale;      // FP8: per-row scales by id (else null)
  const float* q;      // float32 queries (re-rank)
  int dp4, d, dpq, eb, KC, num_sms;
  int64_t n;
  const int32_t* pa;
  const int32_t* pb;
  int32_t* aq;          // pre-filter query ids by position (the order of their queue)
  float* aqn;           // squared norms of their vectors as the scan's format holds them
  float* aqs;           // FP8: their scales (else null)
  void* qb;             // their vectors in the scan's format, dpq elements a row
  void* qg;             // the same rows gathered per tile slot (TMA source of the query operand)
  int32_t* slotpos;     // per tile slot: the query position it holds, -1 for none
  int32_t* tile_span;   // per tile: its span
  int32_t* unit_off;    // per tile: its first work unit (tiles + 1 entries)
  int32_t* span_cnt;    // per span: queries whose range meets it
  int32_t* span_tile;   // per span: its first tile (spans + 1 entries)
  int32_t* span_fill;   // per span: next free slot (placement cursor)
  unsigned* gmin;       // per query: 128 group minima over its whole range (float bits)
  uint64_t* qlist;      // per query: kTcQCap candidate keys below its bound
  uint64_t* stage;      // per CTA and epilogue thread: kTcStage keys found in the current unit
  int32_t* qcnt;        // per query: candidates found (above kQCap: overflow)
  unsigned long long* sumy;  // total in-range rows of the pre-filter queries
  unsigned long long* qthr;  // per query: key(T, INT_MAX) of its bound T (kKeyMax: none)
  int64_t slot_cap, span_cap, pcap;  // tile slots, spans and (query, span) pairs the scratch holds
  int32_t* counters;
  int k, R;
  uint64_t wait_ns;  // elapsed-time limit of every wait on another role
  int stall;         // timeout test: the collecting epilogue waits on a barrier nobody arrives at
  Outputs o;
};

// Tile of work unit x (the last tile whose first unit is <= x).
__device__ __forceinline__ int unit_tile(const TcArgs& a, int ntiles, int x) {
  int lo = 0, hi = ntiles;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a.unit_off[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// Span length L (rows; a multiple of 256, at least 4096). It keeps the (query, span)
// pairs P within pcap: a query meets at most (Y - 1) / L + 2 spans, so
// L >= sum(Y) / (pcap - 2 nA) gives P <= pcap; and the tiles within slot_cap / 128 =
// pcap / 64: there are at most P / 128 + ceil(n / L) of them, and
// L >= 128 n / (pcap - 128) makes ceil(n / L) <= pcap / 128.
__device__ __forceinline__ int64_t span_len(const TcArgs& a, int nA) {
  const unsigned long long sy = *a.sumy;
  const int64_t room = a.pcap - 2 * (int64_t)nA;  // > 0: pcap is 8 slots per query
  int64_t L = (int64_t)((sy + room - 1) / room);
  const int64_t L2 = (128 * a.n + a.pcap - 129) / (a.pcap - 128);  // pcap >= 1024
  if (L2 > L) L = L2;
  if (L < 4096) L = 4096;
  return (L + kTcRows - 1) / kTcRows * kTcRows;
}

// Rows [r0, r1) of unit u of tile t: its share of the blocks of the tile's span
// (r1 may pass the end of the data; those rows are not used).
__device__ __forceinline__ void tile_unit_rows(const TcArgs& a, int t, int u, int* r0, int* r1) {
  const int64_t L = a.counters[CNT_TC_L];
  const int64_t s0 = (int64_t)a.tile_span[t] * L;
  const int64_t rows = (a.n - s0 < L) ? a.n - s0 : L;
  const int nb = (int)((rows + kTcRows - 1) / kTcRows), U = a.unit_off[t + 1] - a.unit_off[t];
  const int b0 = (int)((int64_t)u * nb / U), b1 = (int)((int64_t)(u + 1) * nb / U);
  *r0 = (int)(s0 + (int64_t)b0 * kTcRows);
  *r1 = (int)(s0 + (int64_t)b1 * kTcRows);
}

// kBound = true: the bounding pass. Its epilogue keeps, per query, the minimum
// distance of 128 disjoint groups of the query's rows in the unit (column half x
// chunk parity x column within the chunk; each of the query's two threads holds its
// half's 64 in registers with static indices). The R-th smallest T of the 128
// minima has R distinct rows at or below it, so key(T, INT_MAX) is above every key
// of the query's top R (R <= 128): it is published into the query's threshold with
// atomicMin before the collecting pass starts.
template <int F, bool kBound>
__global__ void __launch_bounds__(kTcThreads, 1) tc_scan_kernel(const __grid_constant__ CUtensorMap tmX,
                                                          const __grid_constant__ CUtensorMap tmQ, TcArgs a) {
  constexpr bool kSc = TcTraits<F>::kScaled;
  constexpr int kKc = kTcKb / TcTraits<F>::kElemBytes;  // K elements per stage
  constexpr uint32_t kMetaBytes = kTcRows * 4 * (1 + (kBound ? 0 : 1) + (kSc ? 1 : 0));
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  TcSmem& s = *reinterpret_cast<TcSmem*>(smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023));
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const int ntiles = a.counters[CNT_TC_TILES];
  const int nunits = a.counters[CNT_TC_UNITS];
  int* err = a.counters + CNT_TC_ERR;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kTcStages; ++i) {
      mbar_init(&s.full[i], 1);
      mbar_init(&s.empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&s.accf[i], 1);
      mbar_init(&s.acce[i], kEpiWarps * 32);
    }
    mbar_init(&s.drain, 1);
    mbar_init(&s.never, 1);
    for (int i = 0; i < 2; ++i) mbar_init(&s.mfull[i], 1);
    for (int i = 0; i < kUnitRing; ++i) {
      mbar_init(&s.ufull[i], 1);
      mbar_init(&s.uempty[i], 1 + kEpiWarps * 32);  // the MMA issuer and the epilogue threads
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s.tmem)),
                 "r"(2 * kTcRows)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s.tmem;

  if (warp == kTmaWarp) {
    // ---- TMA producer (lane 0 issues; the warp stays converged)
    if (lane == 0) {
      bool ok = true;
      long long it = 0, gb = 0;
      for (long long useq = 0; ok; ++useq) {
        // claim the next unit and hand it to the other roles
        const int us = (int)(useq % kUnitRing);
        const long long uu = useq / kUnitRing;
        if (uu > 0 && !mbar_wait(&s.uempty[us], (uint32_t)((uu - 1) & 1), a.wait_ns)) {
          ok = false;
          break;
        }
        int x = atomicAdd(a.counters + (kBound ? CNT_TC_TAKE_B : CNT_TC_TAKE), 1);
        if (x >= nunits) x = -1;
        s.uring[us] = x;
        mbar_arrive(&s.ufull[us]);
        if (x < 0) break;
        const int t = unit_tile(a, ntiles, x);
        int r0, r1;
        tile_unit_rows(a, t, x - a.unit_off[t], &r0, &r1);
        for (int row0 = r0; row0 < r1 && ok; row0 += kTcRows, ++gb) {
          // the block's norms, ids and scales, once the epilogue is done with the
          // block that used this accumulator before (rows below n + kTcRowPad: the
          // arrays' zero padding covers the last block)
          const int mb = (int)(gb & 1);
          if (gb >= 2 && !mbar_wait(&s.acce[mb], (uint32_t)(((gb >> 1) - 1) & 1), a.wait_ns)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&s.mfull[mb], kMetaBytes);
          bulk_load(s.mxn[mb], a.xn + row0, kTcRows * 4, &s.mfull[mb]);
          if constexpr (!kBound) bulk_load(s.mid[mb], a.sorted_ids + row0, kTcRows * 4, &s.mfull[mb]);
          if constexpr (kSc) bulk_load(s.mxs[mb], a.xs + row0, kTcRows * 4, &s.mfull[mb]);
          for (int kc = 0; kc < a.KC; ++kc, ++it) {
            const int st = (int)(it % kTcStages);
            const long long u = it / kTcStages;
            if (u > 0 && !mbar_wait(&s.empty[st], (uint32_t)((u - 1) & 1), a.wait_ns)) {
              ok = false;
              break;
            }
            mbar_expect_tx(&s.full[st], kStageA + kStageB);
            tma_load_2d(s.a[st], &tmQ, kc * kKc, t * kTcQ, &s.full[st]);
            tma_load_2d(s.b[st], &tmX, kc * kKc, row0, &s.full[st]);
          }
        }
      }
      // no copy may still be landing in shared memory when the CTA leaves: wait
      // (bounded) for the last load issued into every stage
      for (int st = 0; st < kTcStages; ++st) {
        if (it <= st) continue;
        const long long last_use = (it - 1 - st) / kTcStages;
        if (!mbar_wait(&s.full[st], (uint32_t)(last_use & 1), kWaitNs)) ok = false;
      }
      for (int mb = 0; mb < 2; ++mb) {
        if (gb <= mb) continue;
        const long long last_use = (gb - 1 - mb) / 2;
        if (!mbar_wait(&s.mfull[mb], (uint32_t)(last_use & 1), kWaitNs)) ok = false;
      }
      if (!ok) atomicExch(err, 1);
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    // ---- MMA issuer (lane 0 issues; the warp stays converged)
    if (lane == 0) {
      bool ok = true;
      const uint32_t idesc = idesc_of<F>();
      long long it = 0, g = 0;
      for (long long useq = 0; ok; ++useq) {
        const int us = (int)(useq % kUnitRing);
        if (!mbar_wait(&s.ufull[us], (uint32_t)((useq / kUnitRing) & 1), a.wait_ns)) {
          ok = false;
          break;
        }
        const int x = *reinterpret_cast<volatile int*>(&s.uring[us]);
        mbar_arrive(&s.uempty[us]);
        if (x < 0) break;
        const int t = unit_tile(a, ntiles, x);
        int r0, r1;
        tile_unit_rows(a, t, x - a.unit_off[t], &r0, &r1);
        for (int row0 = r0; row0 < r1 && ok; row0 += kTcRows, ++g) {
          const int ab = (int)(g & 1);
          const long long ua = g >> 1;
          if (ua > 0 && !mbar_wait(&s.acce[ab], (uint32_t)((ua - 1) & 1), a.wait_ns)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t d_tmem = tmem + (uint32_t)(ab * kTcRows);
          for (int kc = 0; kc < a.KC; ++kc, ++it) {
            const int st = (int)(it % kTcStages);
            if (!mbar_wait(&s.full[st], (uint32_t)((it / kTcStages) & 1), a.wait_ns)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da = sw128_desc(smem_u32(s.a[st]));
            const uint64_t db = sw128_desc(smem_u32(s.b[st]));
#pragma unroll
            for (int kk = 0; kk < kTcKb / 32; ++kk)  // 32 bytes of K per instruction
              umma<F>(d_tmem, da + 2 * kk, db + 2 * kk, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
            umma_commit(&s.empty[st]);
          }
          if (!ok) break;
          umma_commit(&s.accf[ab]);
        }
      }
      // every product issued has completed before tensor memory is released
      umma_commit(&s.drain);
      if (!mbar_wait(&s.drain, 0, kWaitNs)) ok = false;
      if (!ok) atomicExch(err, 1);
    }
    __syncwarp();
  } else if (kBound) {
    // ---- bounding epilogue (warps 0-7): group minima per query. Warp w holds the
    // queries of tensor-memory lanes 32 (w % 4).. over columns 128 (w / 4).. of each
    // block; group = column mod 64 (chunk parity x column within the chunk). At the
    // end of a unit the column-half-1 warp hands its 64 minima to the half-0 warp of
    // the same lanes, which merges them (a group's minimum over the block is the
    // smaller of its two halves' minima) and publishes the bound.
    const int lq = warp & 3, hh = warp >> 2;
    const int tq = lq * 32 + lane;
    const int cbase = hh * kHalfCols;
    bool failed = false;
    long long g = 0;
    for (long long useq = 0; !failed; ++useq) {
      const int us = (int)(useq % kUnitRing);
      if (!__all_sync(kFull, mbar_wait(&s.ufull[us], (uint32_t)((useq / kUnitRing) & 1), a.wait_ns))) {
        failed = true;
        break;
      }
      const int x = *reinterpret_cast<volatile int*>(&s.uring[us]);
      mbar_arrive(&s.uempty[us]);
      if (x < 0) break;
      const int t = unit_tile(a, ntiles, x);
      int r0, r1;
      tile_unit_rows(a, t, x - a.unit_off[t], &r0, &r1);
      const int qpos = a.slotpos[(int64_t)t * kTcQ + tq];  // query position of this slot, -1: none
      const bool qv = qpos >= 0;
      int pa = 0, pb = 0;
      float qn = 0.f, qs = 1.f;
      if (qv) {
        const int qi = a.aq[qpos];
        pa = a.pa[qi];
        pb = a.pb[qi];
        qn = a.aqn[qpos];
        if constexpr (kSc) qs = a.aqs[qpos];
      }
      const float w2 = 2.f * qs;  // weight of the dot product (times the row's scale for FP8)
      float gm0[32], gm1[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) gm0[j] = gm1[j] = __int_as_float(0x7f800000);
      for (int row0 = r0; row0 < r1; row0 += kTcRows, ++g) {
        const int ab = (int)(g & 1);
        const int c0 = max(pa - row0, 0), c1 = min(pb - row0, kTcRows);  // this query's columns
        if (!__all_sync(kFull, mbar_wait(&s.accf[ab], (uint32_t)((g >> 1) & 1), a.wait_ns) &&
                                   mbar_wait(&s.mfull[ab], (uint32_t)((g >> 1) & 1), a.wait_ns))) {
          failed = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t taddr = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(ab * kTcRows + cbase);
        const float* mxn = s.mxn[ab];
        const float* mxs = s.mxs[ab];
#pragma unroll 1
        for (int cp = 0; cp < kHalfCols / 64; ++cp) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int lc = 2 * cp + h;          // chunk of this warp's half
            const int cb = cbase + 32 * lc;     // its first column in the block
            const bool need = c1 > cb && c0 < cb + 32;
            if (!__any_sync(kFull, need)) continue;
            const bool full = c0 <= cb && c1 >= cb + 32;
            float v[32];
            if (__all_sync(kFull, full || !need)) {
              // every lane takes all 32 columns or none: a lane without columns adds
              // NaN, which fminf ignores
              const float qe = need ? qn : __int_as_float(0x7fc00000);
              float4 x4[8], s4[8];
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                x4[i] = reinterpret_cast<const float4*>(mxn + cb)[i];
                if constexpr (kSc) s4[i] = reinterpret_cast<const float4*>(mxs + cb)[i];
              }
              tmem_ld32(taddr + (uint32_t)(32 * lc), v);
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const float xv = f4_at(x4[j >> 2], j & 3);
                float w = 2.f;
                if constexpr (kSc) w = w2 * f4_at(s4[j >> 2], j & 3);
                const float dist = fmaf(-w, v[j], xv + qe);
                if (h) gm1[j] = fminf(gm1[j], dist);
                else gm0[j] = fminf(gm0[j], dist);
              }
            } else {
              tmem_ld32(taddr + (uint32_t)(32 * lc), v);
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const float xv = mxn[cb + j];
                float w = 2.f;
                if constexpr (kSc) w = w2 * mxs[cb + j];
                const float dist = fmaf(-w, v[j], xv + qn);
                const bool in = cb + j >= c0 && cb + j < c1;
                if (h) gm1[j] = in ? fminf(gm1[j], dist) : gm1[j];
                else gm0[j] = in ? fminf(gm0[j], dist) : gm0[j];
              }
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&s.acce[ab]);
      }
      if (failed) break;
      // the query's 128 group minima over its whole range: group hh * 64 + (column mod
      // 64) of column half hh; every span and block starts on a multiple of 256 rows,
      // so a group is the same set of row residues in every unit of the query, and the
      // minimum over units is the group's minimum over the range. Clamped at 0 (the
      // clamp commutes with min and rank); groups without rows stay +inf.
      // Only minima below the query's current ones take an atomic (a plain read first;
      // a stale read only costs an atomic that changes nothing).
      if (qv) {
        unsigned* gq = a.gmin + (int64_t)qpos * 128 + hh * 64;
        uint4 cur[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) cur[i] = __ldcg(reinterpret_cast<const uint4*>(gq) + i);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const unsigned v0 = __float_as_uint(fmaxf(gm0[j], 0.f)), v1 = __float_as_uint(fmaxf(gm1[j], 0.f));
          if (gm0[j] < __int_as_float(0x7f800000) && v0 < u4_at(cur[j >> 2], j & 3)) atomicMin(gq + j, v0);
          if (gm1[j] < __int_as_float(0x7f800000) && v1 < u4_at(cur[8 + (j >> 2)], j & 3)) atomicMin(gq + 32 + j, v1);
        }
      }
    }
    if (failed) atomicExch(err, 1);
  } else {
    // ---- collecting epilogue (warps 0-7): lane q of warp w is query 32 (w % 4) + q
    // of the tile (its tensor-memory lane) over columns 128 (w / 4).. of each block.
    // Every in-range row whose key is below the query's bound is staged in this
    // thread's area (a predicated store, thread-private count); at the end of the unit
    // the thread reserves room in the query's list with one atomicAdd and copies its
    // keys there. The query's count goes on past kTcQCap (a staging area that filled
    // up adds more than kTcQCap), so that the finishing kernel can see an overflow. The
    // warps run independently; a timed-out wait ends the warp's loop (decided
    // warp-wide).
    const int lq = warp & 3, hh = warp >> 2;
    const int tq = lq * 32 + lane;
    const int cbase = hh * kHalfCols;
    bool failed = false;
    long long g = 0;
    // timeout test: this wait runs out after wait_ns; the producer's and the MMA
    // issuer's waits on the epilogue then run out in turn, and both drain
    if (a.stall && !__all_sync(kFull, mbar_wait(&s.never, 0, a.wait_ns))) failed = true;
    for (long long useq = 0; !failed; ++useq) {
      const int us = (int)(useq % kUnitRing);
      if (!__all_sync(kFull, mbar_wait(&s.ufull[us], (uint32_t)((useq / kUnitRing) & 1), a.wait_ns))) {
        failed = true;
        break;
      }
      const int x = *reinterpret_cast<volatile int*>(&s.uring[us]);
      mbar_arrive(&s.uempty[us]);
      if (x < 0) break;
      const int t = unit_tile(a, ntiles, x);
      int r0, r1;
      tile_unit_rows(a, t, x - a.unit_off[t], &r0, &r1);
      const int qpos = a.slotpos[(int64_t)t * kTcQ + tq];  // query position of this slot, -1: none
      const bool qv = qpos >= 0;
      int pa = 0, pb = 0;
      float qn = 0.f, qs = 1.f;
      uint64_t thr = kKeyMax;
      if (qv) {
        const int qi = a.aq[qpos];
        pa = a.pa[qi];
        pb = a.pb[qi];
        qn = a.aqn[qpos];
        if constexpr (kSc) qs = a.aqs[qpos];
        thr = *reinterpret_cast<volatile unsigned long long*>(a.qthr + qpos);
      }
      const float w2 = 2.f * qs;
      // the bound's distance (+inf without a bound: every row qualifies); the bound is
      // the key (tdist, INT_MAX), so a row's key is below it exactly when its
      // distance is at most tdist
      const float tdist = thr == kKeyMax ? __int_as_float(0x7f800000) : key_dist(thr);
      uint64_t* const stage = a.stage + ((int64_t)blockIdx.x * kTcEpiThreads + threadIdx.x) * kTcStage;
      int cnt = 0;  // keys found in this unit (may pass kTcStage; stores stop there)
      for (int row0 = r0; row0 < r1; row0 += kTcRows, ++g) {
        const int ab = (int)(g & 1);
        const int c0 = max(pa - row0, 0), c1 = min(pb - row0, kTcRows);  // this query's columns
        if (!__all_sync(kFull, mbar_wait(&s.accf[ab], (uint32_t)((g >> 1) & 1), a.wait_ns) &&
                                   mbar_wait(&s.mfull[ab], (uint32_t)((g >> 1) & 1), a.wait_ns))) {
          failed = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t taddr = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(ab * kTcRows + cbase);
        const float* mxn = s.mxn[ab];
        const int32_t* mid = s.mid[ab];
        const float* mxs = s.mxs[ab];
#pragma unroll 1
        for (int lc = 0; lc < kHalfCols / 32; ++lc) {
          const int cb = cbase + 32 * lc;
          const bool need = c1 > cb && c0 < cb + 32;
          if (!__any_sync(kFull, need)) continue;
          const bool full = c0 <= cb && c1 >= cb + 32;
          float v[32];
          if (__all_sync(kFull, (full || !need) && cnt + 32 <= kTcStage)) {
            // every lane takes all 32 columns or none (NaN compares false), and has
            // room for 32 more keys
            const float qe = need ? qn : __int_as_float(0x7fc00000);
            float4 x4[8], s4[8];
            int4 i4[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              x4[i] = reinterpret_cast<const float4*>(mxn + cb)[i];
              i4[i] = reinterpret_cast<const int4*>(mid + cb)[i];
              if constexpr (kSc) s4[i] = reinterpret_cast<const float4*>(mxs + cb)[i];
            }
            tmem_ld32(taddr + (uint32_t)(32 * lc), v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float xv = f4_at(x4[j >> 2], j & 3);
              float w = 2.f;
              if constexpr (kSc) w = w2 * f4_at(s4[j >> 2], j & 3);
              const float dist = fmaf(-w, v[j], xv + qe);
              const bool hit = dist <= tdist;
              if (hit) stage[cnt] = make_key(fmaxf(dist, 0.f), i4_at(i4[j >> 2], j & 3));
              cnt += hit;
            }
          } else {
            tmem_ld32(taddr + (uint32_t)(32 * lc), v);
            // this query's columns of the chunk: [jlo, jhi)
            const int jlo = c0 - cb, jhi = c1 - cb;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float xv = mxn[cb + j];
              float w = 2.f;
              if constexpr (kSc) w = w2 * mxs[cb + j];
              const float dist = fmaf(-w, v[j], xv + qn);
              if (j >= jlo && j < jhi && dist <= tdist) {
                if (cnt < kTcStage) stage[cnt] = make_key(fmaxf(dist, 0.f), mid[cb + j]);
                ++cnt;
              }
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&s.acce[ab]);
      }
      if (failed) break;
      // the unit's keys into the query's list (a staging area that filled up forces
      // the query's overflow: its exact scan)
      if (cnt > 0) {
        const int o = atomicAdd(a.qcnt + qpos, cnt > kTcStage ? kTcQCap + 1 : cnt);
        uint64_t* const list = a.qlist + (int64_t)qpos * kTcQCap;
        if (cnt <= kTcStage)
          for (int i = 0; i < cnt && o + i < kTcQCap; ++i) list[o + i] = stage[i];
      }
    }
    if (failed) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTcRows)
                 : "memory");
  }
}

// Spans of the attribute order met by each pre-filter query: one thread per query
// position counts itself into every span its range [pa, pb) meets.
__global__ void tc_span_count(TcArgs a) {
  const int nA = a.counters[CNT_QA];
  const int64_t L = span_len(a, nA);
  if (blockIdx.x == 0 && threadIdx.x == 0) a.counters[CNT_TC_L] = (int)L;
  for (int pos = blockIdx.x * blockDim.x + threadIdx.x; pos < nA; pos += gridDim.x * blockDim.x) {
    const int qi = a.aq[pos];
    const int pa = a.pa[qi], pb = a.pb[qi];
    if (pb <= pa) continue;
    for (int64_t sp = pa / L; sp <= (pb - 1) / L; ++sp) atomicAdd(&a.span_cnt[sp], 1);
  }
}

// Exclusive prefix sum over the 1024 threads of a CTA; *total gets the sum.
__device__ __forceinline__ int cta_exclusive_scan(int v, int* sm, int* total) {
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int w = threadIdx.x >= off ? sm[threadIdx.x - off] : 0;
    __syncthreads();
    sm[threadIdx.x] += w;
    __syncthreads();
  }
  const int r = sm[threadIdx.x] - v;
  *total = sm[1023];
  __syncthreads();
  return r;
}

// One CTA of 1024 threads: tiles of 128 slots per span (ceil(count / 128)), the first
// tile of every span, the span of every tile, the work units of every tile and the
// placement cursors (every slot was marked empty, -1, before). A unit holds bpu of its span's
// 256-row blocks, bpu in [1, 16] chosen for about four units per SM over the batch
// (all tiles of a span have the same units). Totals go to the counters; tiles past the
// scratch's slots raise the error flag and are dropped.
__global__ void tc_span_scan(TcArgs a) {
  __shared__ int sm[1024];
  __shared__ int carry;
  __shared__ unsigned long long blocks;
  const int64_t L = a.counters[CNT_TC_L];
  const int nspan = (int)((a.n + L - 1) / L);
  const int tile_cap = (int)(a.slot_cap / kTcQ);
  auto span_blocks = [&](int sp) {
    const int64_t rows = (a.n - sp * L < L) ? a.n - sp * L : L;
    return (int)((rows + kTcRows - 1) / kTcRows);
  };
  if (threadIdx.x == 0) {
    carry = 0;
    blocks = 0;
  }
  __syncthreads();
  // sweep 1: tiles per span and their first tile; tile-blocks of the batch
  for (int base = 0; base < nspan; base += 1024) {
    const int sp = base + threadIdx.x;
    const int nt = sp < nspan ? (a.span_cnt[sp] + kTcQ - 1) / kTcQ : 0;
    int tsum;
    const int t0 = carry + cta_exclusive_scan(nt, sm, &tsum);
    if (sp < nspan) {
      a.span_tile[sp] = t0;
      a.span_fill[sp] = t0 * kTcQ;
      if (nt > 0) atomicAdd(&blocks, (unsigned long long)nt * span_blocks(sp));
      for (int i = 0; i < nt && t0 + i < tile_cap; ++i) a.tile_span[t0 + i] = sp;
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += tsum;
    __syncthreads();
  }
  const int tiles = carry;
  const unsigned long long want = 4ull * (unsigned long long)a.num_sms;
  unsigned long long per = (blocks + want - 1) / want;
  const int bpu = per < 1 ? 1 : per > 16 ? 16 : (int)per;
  __syncthreads();
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  // sweep 2: units of every tile
  for (int base = 0; base < nspan; base += 1024) {
    const int sp = base + threadIdx.x;
    int nt = 0, nu = 0;
    if (sp < nspan) {
      nt = (a.span_cnt[sp] + kTcQ - 1) / kTcQ;
      nu = (span_blocks(sp) + bpu - 1) / bpu;
    }
    int usum;
    const int u0 = carry + cta_exclusive_scan(nt * nu, sm, &usum);
    if (sp < nspan) {
      const int t0 = a.span_tile[sp];
      for (int i = 0; i < nt && t0 + i < tile_cap; ++i) a.unit_off[t0 + i] = u0 + i * nu;
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += usum;
    __syncthreads();
  }
  int ntiles = tiles, units = carry;
  if (ntiles > tile_cap) {  // cannot happen with the span length's bounds; kept safe
    ntiles = 0;
    units = 0;
    if (threadIdx.x == 0) atomicExch(&a.counters[CNT_TC_ERR], 1);
  }
  if (threadIdx.x == 0) {
    a.span_tile[nspan] = ntiles;
    a.unit_off[ntiles] = units;
    a.counters[CNT_TC_TILES] = ntiles;
    a.counters[CNT_TC_UNITS] = units;
  }
}

// One warp per pre-filter query position: a slot in one tile of every span its range
// meets, and its operand row copied into that slot's row of the gathered buffer.
__global__ void tc_place(TcArgs a) {
  const int nA = a.counters[CNT_QA];
  const int64_t L = a.counters[CNT_TC_L];
  const int64_t slots = (int64_t)a.counters[CNT_TC_TILES] * kTcQ;
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  const int row16 = a.dpq * a.eb / 16;  // 16-byte words of an operand row
  for (int pos = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; pos < nA; pos += warps) {
    const int qi = a.aq[pos];
    const int pa = a.pa[qi], pb = a.pb[qi];
    if (pb <= pa) continue;
    const int4* src = reinterpret_cast<const int4*>(reinterpret_cast<const unsigned char*>(a.qb) +
                                                    (int64_t)pos * a.dpq * a.eb);
    for (int64_t sp = pa / L; sp <= (pb - 1) / L; ++sp) {
      int gs = 0;
      if (lane == 0) gs = atomicAdd(&a.span_fill[sp], 1);
      gs = __shfl_sync(kFull, gs, 0);
      if (gs >= slots) continue;  // only with dropped tiles (error flag set)
      if (lane == 0) a.slotpos[gs] = pos;
      int4* dst = reinterpret_cast<int4*>(reinterpret_cast<unsigned char*>(a.qg) + (int64_t)gs * a.dpq * a.eb);
      for (int c = lane; c < row16; c += 32) dst[c] = src[c];
    }
  }
}

// One warp per pre-filter query position: its bound, the R-th smallest of its 128
// group minima (the smallest value v with at least R minima <= v, by bisection over
// the float bits, which order like the values for v >= 0). No bound (+inf) when fewer
// than R groups hold rows.
__global__ void tc_bound(TcArgs a) {
  const int nA = a.counters[CNT_QA];
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int pos = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; pos < nA; pos += warps) {
    const uint4 m = reinterpret_cast<const uint4*>(a.gmin + (int64_t)pos * 128)[lane];
    auto count_le = [&](unsigned x) {
      const int c = (m.x <= x) + (m.y <= x) + (m.z <= x) + (m.w <= x);
      int t = c;
      for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(kFull, t, off);
      return t;
    };
    const unsigned kInf = 0x7f800000u;
    if (count_le(kInf - 1) < a.R) continue;  // the threshold stays kKeyMax
    unsigned lo = 0, hi = kInf - 1;  // count_le(hi) >= R
    while (lo < hi) {
      const unsigned mid = lo + (hi - lo) / 2;
      if (count_le(mid) >= a.R) hi = mid;
      else lo = mid + 1;
    }
    if (lane == 0) a.qthr[pos] = make_key(__uint_as_float(lo), 0x7fffffff);
  }
}

// One warp per pre-filter query: takes the R smallest keys of its candidate list,
// re-ranks them with exact float32 distances and writes the result row. A list that
// overflowed (more than kTcQCap candidates below the bound) sends the query through
// an exact warp scan of
// its range instead: the stored rows (format T) against the float32 query, direct
// differences, the same selection as the warp scan of the search kernel. After a
// timed-out wait the rows are empty and flagged.
template <class T, int CH, int G>
__global__ void __launch_bounds__(128) tc_finish(TcArgs a) {
  __shared__ uint64_t top[4][kTcRMax];
  __shared__ uint64_t out[4][kTcRMax];
  __shared__ int R[4][32];
  __shared__ int clist[4][32];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const int nA = a.counters[CNT_QA];
  const bool failed = a.counters[CNT_TC_ERR] != 0;
  const int warps = gridDim.x * 4;
  for (int pos = blockIdx.x * 4 + warp; pos < nA; pos += warps) {
    const int qi = a.aq[pos];
    const int pa = a.pa[qi], pb = a.pb[qi];
    float4 qv[CH];
    load_query<CH>(qv, a.q + (int64_t)qi * a.d, a.d);
    const int c = a.qcnt[pos];
    const bool overflow = c > kTcQCap;
    int nt = 0;
    if (failed || pb <= pa) {
      nt = 0;
    } else if (!overflow) {
      const uint64_t* src = a.qlist + (int64_t)pos * kTcQCap;
      for (int off = 0; off < c; off += 32) {
        const uint64_t key = off + lane < c ? src[off + lane] : kKeyMax;
        nt = topk_offer(top[warp], nt, a.R, key, R[warp]);
      }
    } else {
      for (int base = pa; base < pb; base += 32) {
        int cid = base + lane < pb ? __ldg(a.sorted_ids + base + lane) : -1;
        const float dist = batch_dist<T, CH, G>(qv, cid, a.vt, a.dp4 * T::kChunkBytes, a.vscale, a.dp4, clist[warp]);
        nt = topk_offer(top[warp], nt, a.R, cid >= 0 ? make_key(dist, cid) : kKeyMax, R[warp]);
      }
    }
    int no = 0;
    for (int off = 0; off < nt; off += 32) {
      int cid = off + lane < nt ? key_id(top[warp][off + lane]) : -1;
      if (cid >= a.n) cid = -1;
      const float dist = batch_dist<StoreF32, CH, G>(qv, cid, reinterpret_cast<const unsigned char*>(a.vec),
                                                     a.dp4 * 16, nullptr, a.dp4, clist[warp]);
      no = topk_offer(out[warp], no, a.k, cid >= 0 ? make_key(dist, cid) : kKeyMax, R[warp]);
    }
    write_row(out[warp], no, a.k, qi, a.o);
    if (lane == 0) {
      a.o.count[qi] = no;
      if (a.o.status) a.o.status[qi] = failed ? UNIFY_Q_LIMIT : 0u;
      if (a.o.counters) {
        a.o.counters[4 * (int64_t)qi + 2] = 0;
        a.o.counters[4 * (int64_t)qi + 3] = 0;
      }
    }
    __syncwarp();
  }
}

// One warp per pre-filter query (position = its place in the queue): its vector in
// the scan's format (zero-padded to dpq elements: bfloat16 by round-to-nearest-even;
// float32 as given for tf32; E4M3 codes of q / s_q with s_q = max|q| / 448,
// saturating), the squared norm of those values (for E4M3, of the decoded s_q * code),
// and its bound, group minima and candidate count reset; its in-range row count is
// added to the batch's total.
template <int F>
__global__ void tc_scatter(const int32_t* __restrict__ queues, const int32_t* __restrict__ pa,
                           const int32_t* __restrict__ pb, const float* __restrict__ q, int d, int dpq,
                           int32_t* counters, int32_t* aq, float* aqn, float* aqs, void* qb,
                           unsigned long long* qthr, unsigned* gmin, int32_t* qcnt, unsigned long long* sumy) {
  const int nA = counters[CNT_QA];
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int pos = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; pos < nA; pos += warps) {
    const int qi = queues[pos];
    reinterpret_cast<uint4*>(gmin + (int64_t)pos * 128)[lane] = make_uint4(0x7f800000u, 0x7f800000u, 0x7f800000u,
                                                                          0x7f800000u);
    if (lane == 0) {
      const int y = pb[qi] - pa[qi];
      if (y > 0) atomicAdd(sumy, (unsigned long long)y);
      qcnt[pos] = 0;
    }
    const float* qrow = q + (int64_t)qi * d;
    float ss = 0.f, sq = 1.f;
    if constexpr (F == kFmtBF16) {
      __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(qb) + (int64_t)pos * dpq;
      for (int c = lane; c < dpq; c += 32) {
        const __nv_bfloat16 h = __float2bfloat16_rn(c < d ? qrow[c] : 0.f);
        dst[c] = h;
        const float f = __bfloat162float(h);
        ss = fmaf(f, f, ss);
      }
    } else if constexpr (F == kFmtTF32) {
      float* dst = reinterpret_cast<float*>(qb) + (int64_t)pos * dpq;
      for (int c = lane; c < dpq; c += 32) {
        const float f = c < d ? qrow[c] : 0.f;
        dst[c] = f;
        ss = fmaf(f, f, ss);
      }
    } else {
      float mx = 0.f;
      for (int c = lane; c < d; c += 32) mx = fmaxf(mx, fabsf(qrow[c]));
      for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, off));
      sq = mx > 0.f ? mx / 448.f : 1.f;
      unsigned char* dst = reinterpret_cast<unsigned char*>(qb) + (int64_t)pos * dpq;
      for (int c = lane; c < dpq; c += 32) {
        const __nv_fp8_storage_t code =
            __nv_cvt_float_to_fp8(c < d ? qrow[c] / sq : 0.f, __NV_SATFINITE, __NV_E4M3);
        dst[c] = (unsigned char)code;
        const __half_raw hr = __nv_cvt_fp8_to_halfraw(code, __NV_E4M3);
        const float f = sq * __half2float(*reinterpret_cast<const __half*>(&hr));
        ss = fmaf(f, f, ss);
      }
    }
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(kFull, ss, off);
    if (lane == 0) {
      aq[pos] = qi;
      aqn[pos] = ss;
      if (aqs) aqs[pos] = sq;
      qthr[pos] = kKeyMax;
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult qr;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) ==
            cudaSuccess &&
        qr == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2D tensor map of the scan's format: rows of `cols` elements, `row_bytes` apart,
// boxes of box_cols x box_rows (box_cols elements = 128 bytes) with 128-byte swizzle;
// reads outside the tensor return 0.
bool encode_2d(CUtensorMap* tm, CUtensorMapDataType dt, const void* base, uint64_t cols, uint64_t rows,
               uint64_t row_bytes, uint32_t box_cols, uint32_t box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(tm, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t tc_smem_bytes() { return sizeof(TcSmem) + 1024; }


// Candidates the scan keeps per query for the FP32 re-rank: rerank_mult * k up to
// kTcRTight, and k itself past that (k <= kTcRMax). The bound is the R-th smallest of
// 128 group minima: about -128 ln(1 - R / 128) rows lie below it, 48 at R = 40 and
// 195 at R = 100, while at R = 128 it is the largest minimum and most rows pass.
int tc_rerank_width(const Params& p) {
  return (int)std::max<long>(p.k, std::min<long>((long)p.rerank_mult * p.k, kTcRTight));
}

template <int F>
cudaError_t launch_tc(const DeviceIndex& ix, const Scratch& sc, const float* q, int64_t nq, const Params& p,
                      const Outputs& o, cudaStream_t st) {
  constexpr int eb = TcTraits<F>::kElemBytes;
  constexpr int kKc = kTcKb / eb;  // K elements per stage
  const int dpq = ((ix.d + kKc - 1) / kKc) * kKc;
  const CUtensorMapDataType dt = F == kFmtBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                 : F == kFmtTF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  const void* rows = F == kFmtBF16 ? (const void*)ix.vts_bf16
                     : F == kFmtTF32 ? (const void*)ix.vec_sorted : (const void*)ix.vts_fp8;
  CUtensorMap tmX, tmQ;
  if (!encode_2d(&tmX, dt, rows, (uint64_t)ix.dp, (uint64_t)ix.n, (uint64_t)ix.dp * eb, kKc, kTcRows) ||
      !encode_2d(&tmQ, dt, sc.tc_qg, (uint64_t)dpq, (uint64_t)sc.tc_slots, (uint64_t)dpq * eb, kKc, kTcQ))
    return cudaErrorInvalidValue;
  const int64_t tile_cap = sc.tc_slots / kTcQ;
  TcArgs a;
  a.sorted_ids = ix.sorted_ids;
  a.xn = F == kFmtBF16 ? ix.xn_bf16_sorted : F == kFmtTF32 ? ix.xn_f32_sorted : ix.xn_fp8_sorted;
  a.xs = F == kFmtFP8 ? ix.scale_fp8_sorted : nullptr;
  a.vec = ix.vec;
  a.vt = F == kFmtBF16 ? ix.vt_bf16 : F == kFmtTF32 ? reinterpret_cast<const unsigned char*>(ix.vec) : ix.vt_fp8;
  a.vscale = F == kFmtFP8 ? ix.scale_fp8 : nullptr;
  a.q = q;
  a.dp4 = ix.dp / 4;
  a.d = ix.d;
  a.dpq = dpq;
  a.eb = eb;
  a.KC = dpq / kKc;
  a.num_sms = ix.num_sms;
  a.n = ix.n;
  a.pa = sc.pa;
  a.pb = sc.pb;
  a.aq = sc.tc_aq;
  a.aqn = sc.tc_aqn;
  a.aqs = F == kFmtFP8 ? sc.tc_aqs : nullptr;
  a.qb = sc.tc_qb;
  a.qg = sc.tc_qg;
  a.slotpos = sc.tc_slotpos;
  a.tile_span = sc.tc_tiles;
  a.unit_off = sc.tc_tiles + tile_cap;
  a.span_cnt = sc.tc_spans;
  a.span_fill = sc.tc_spans + sc.tc_spans_cap;
  a.span_tile = sc.tc_spans + 2 * sc.tc_spans_cap;
  a.gmin = sc.tc_gmin;
  a.qlist = sc.tc_qlist;
  a.qcnt = sc.tc_qcnt;
  a.stage = sc.tc_stage;
  a.sumy = sc.tc_sumy;
  a.qthr = sc.tc_thr;
  a.slot_cap = sc.tc_slots;
  a.span_cap = sc.tc_spans_cap;
  a.pcap = kTcPairsPerQuery * sc.tc_rows;
  a.counters = sc.counters;
  a.k = p.k;
  a.R = tc_rerank_width(p);
  a.stall = p.tc_scan == 2 ? 1 : 0;
  a.wait_ns = p.tc_scan == 2 ? kTestWaitNs : kWaitNs;
  a.o = o;
  // queries by position, then spans, tiles, units and slots
  cudaError_t e = cudaMemsetAsync(sc.tc_sumy, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc.tc_spans, 0, (size_t)sc.tc_spans_cap * sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc.tc_slotpos, 0xff, (size_t)sc.tc_slots * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  const int qgrid = (int)std::max<int64_t>(ix.num_sms, (nq + 7) / 8);  // a warp per query, 8 per CTA
  tc_scatter<F><<<qgrid, 256, 0, st>>>(sc.queues, sc.pa, sc.pb, q, ix.d, dpq, sc.counters, sc.tc_aq, sc.tc_aqn,
                                       F == kFmtFP8 ? sc.tc_aqs : nullptr, sc.tc_qb, sc.tc_thr, sc.tc_gmin,
                                       sc.tc_qcnt, sc.tc_sumy);
  tc_span_count<<<(int)std::max<int64_t>(1, (nq + 255) / 256), 256, 0, st>>>(a);
  tc_span_scan<<<1, 1024, 0, st>>>(a);
  tc_place<<<qgrid, 256, 0, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = tc_smem_bytes();
  e = cudaFuncSetAttribute(tc_scan_kernel<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_scan_kernel<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // bounding pass (each query's bound), then the collecting pass
  tc_scan_kernel<F, true><<<ix.num_sms, kTcThreads, smem, st>>>(tmX, tmQ, a);
  tc_bound<<<qgrid, 256, 0, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  tc_scan_kernel<F, false><<<ix.num_sms, kTcThreads, smem, st>>>(tmX, tmQ, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // FP32 re-rank with the row-width variants of the search kernel; an overflowed
  // query scans the stored rows of its format
  using T = typename std::conditional<F == kFmtBF16, StoreBF16,
                                      typename std::conditional<F == kFmtTF32, StoreF32, StoreFP8>::type>::type;
  // one warp per query of the batch (the pre-filter queries are a part of it), so that
  // every query's list merge and re-rank gathers are in flight at once
  const int ch = (a.dp4 + 31) / 32;
  const int fgrid = (int)std::max<int64_t>(ix.num_sms * 4, (nq + 3) / 4);
  if (ch <= 1)
    tc_finish<T, 1, 16><<<fgrid, 128, 0, st>>>(a);
  else if (ch <= 2)
    tc_finish<T, 2, 8><<<fgrid, 128, 0, st>>>(a);
  else if (ch <= 4)
    tc_finish<T, 4, 4><<<fgrid, 128, 0, st>>>(a);
  else
    tc_finish<T, 8, 2><<<fgrid, 128, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool tc_scan_available(const DeviceIndex& ix, const Params& p) {
  if (!p.tc_scan || ix.d > 1024 || encode_fn() == nullptr) return false;
  if (p.rerank_mult < 1 || p.k > kTcRMax) return false;
  // the rows' TMA stride must be a multiple of 16 bytes
  if (p.dtype == UNIFY_BF16) return ix.dp % 8 == 0;
  if (p.dtype == UNIFY_FP32) return true;  // dp is a multiple of 4
  return ix.dp % 16 == 0;                  // FP8: one byte per element
}

size_t tc_query_row_bytes(int d) { return (size_t)((d + kTcKb - 1) / kTcKb) * kTcKb * 4; }

cudaError_t launch_tcscan(const DeviceIndex& ix, const Scratch& sc, const float* q, int64_t nq, const Params& p,
                          const Outputs& o, cudaStream_t st) {
  if (p.dtype == UNIFY_BF16) return launch_tc<kFmtBF16>(ix, sc, q, nq, p, o, st);
  if (p.dtype == UNIFY_FP32) return launch_tc<kFmtTF32>(ix, sc, q, nq, p, o, st);
  return launch_tc<kFmtFP8>(ix, sc, q, nq, p, o, st);
}

}  // namespace unify
