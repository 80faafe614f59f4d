// Shared by the split-precision translation units: tile geometry, work
// descriptors, PTX wrappers (mbarrier, TMA bulk copy, tcgen05), the digit cut
// and the GEMM kernel's helpers. See split.cu for the method.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "split.h"

namespace bg {
namespace splitk {


constexpr int BM = 128, BK = 64;
constexpr int kATileBytes = BM * BK * 2;  // 16 KiB: one A plane of one k-block
constexpr int kLineBytes = BK * 2;        // 128 bytes: one row of a tile
// The A ring holds groups of kAGroup plane slots: the producer fills a group
// with one barrier and the MMA issuer waits on it once and releases it with
// one commit. Each wait, fence and commit in the MMA issue loop stalls the
// tensor pipe for about a hundred clocks (measured on GB300), so one sync
// per plane held a 9-slice k-block about 40% above its MMA time.
constexpr int kAGroup = 3;
constexpr int kMaxAGroups = 4;
// Split GEMM CTA: producer warp, MMA warp, then 4 H epilogue warps.
__host__ __device__ constexpr int gemm_threads(int h) { return 64 + 128 * h; }
constexpr int kMetaStride = 264;  // int32 per block: e[128], R[128] (then padding)
constexpr int kTmemCols = 512;
constexpr int kSliceThreads = 256;
// Largest FP64 footprint of one slicer job (see split_jobs).
constexpr int64_t kSliceJobBytes = 65536;
constexpr int kMaxDynSmem = 232448;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s bound on any single wait

// Tile width (columns of the output tile, rows of a B tile) for s planes:
// the largest multiple of 16 (at most 128) with s * BN <= 512 TMEM columns.
// Output tile width of the split GEMM for s slices. Up to 5 slices the tile's
// s level accumulators fit TMEM twice (2 s BN <= 512 columns): the MMAs of the
// next tile then run while the epilogue empties the other copy. From 6
// slices on one copy fills TMEM and the epilogue empties it level by level
// (a double-buffered 6-slice tile would be 32 wide, which measured slower).
__host__ __device__ constexpr int bn_for(int s) {
  return s <= 2 ? 128 : s <= 4 ? 64 : s == 5 ? 48 : s == 6 ? 48 : s <= 8 ? 64 : s <= 10 ? 48 : 32;
}
__host__ __device__ constexpr bool double_buffered(int s) { return s <= 5; }

struct SInst {
  int64_t a_off, b_off, c_off;  // user element offsets
  int64_t lda, ldb, ldc;        // user elements
  int32_t m, n, k;              // user sizes
  int32_t pad;
};

struct SliceJob {
  int64_t tile0;  // first tile of the block (k-block 0, plane 1)
  int32_t blk;    // block id = meta index
  int32_t pos;    // first position in the order list
  int16_t side;   // 0: A block (rows), 1: B block (columns)
  int16_t g;      // instances stacked in the block
  int16_t span;   // lines per stacked instance (virtual rows of A / columns of B)
  int16_t nkb;    // k-blocks of 64
  int32_t org;    // first line of the block within its instance (big instances)
  int32_t kv;     // virtual k' of the instances
  int16_t l0;     // first line of the block this job cuts
  int16_t nl;     // lines this job cuts (a multiple of 4)
};

struct SplitUnit {
  int64_t a_tile0, b_tile0;  // first tiles (chain mode: a_tile0 is relative to the pool entry)
  int32_t a_blk, b_blk;      // meta blocks (chain mode: a_blk is the row block index)
  int32_t pos;               // order position of the (first) instance
  int16_t g;                 // packed instances (1 = a tile of one instance)
  int16_t nkb;               // k-blocks
  int16_t kmma_last;         // MMA K-steps (16 each) in the last k-block
  int16_t mrow;              // virtual rows per packed instance
  int16_t ncol;              // columns per packed instance
  int16_t pad;
  int32_t r0, c0;            // tile origin in the instance (virtual rows, columns)
};

struct SliceArgs {
  const SliceJob* jobs;
  int64_t njobs;
  const SInst* instA;
  const SInst* instB;
  const int32_t* orderA;
  const int32_t* orderB;
  const double* A;
  const double* B;
  uint8_t* tilesA;
  uint8_t* tilesB;
  int32_t* metaA;
  int32_t* metaB;
  int cplx, s, beta, bn;
  int herk;  // Hermitian update: B lines are rows of A (conjugated), read through the A side
};

struct GemmArgs {
  const SplitUnit* units;
  int64_t nunits;
  const SInst* inst;
  const int32_t* order;
  const uint8_t* tilesA;
  const uint8_t* tilesB;
  const int32_t* metaA;
  const int32_t* metaB;
  double* C;
  const int32_t* idx;         // chain mode: pool index per walker, else nullptr
  const int64_t* pool_tile0;  // chain mode: first tile of each pool entry
  const int32_t* pool_blk0;   // chain mode: first meta block of each pool entry
  const SInst* pool;          // chain mode: pool entries (sizes)
  int32_t pool_count;         // chain mode: number of pool entries
  Scalars sc;
  int cplx, s, beta, skip_product;
  int kpass;                  // k-blocks per exact pass
  int a_groups;               // groups of kAGroup slots in the A ring
  int herk;                   // Hermitian update: store only the lower triangle
  int* err;
};

// Small real instances (m, n, k <= 64) of a split plan: one fused kernel
// (split_small.cu) reads A and B, cuts the digits into shared memory and
// multiplies them with mma.sync. A work item is up to 16 instances of one
// padded edge t (16, 32 or 64) that one CTA's instance groups take together.
constexpr int kSmallMax = 64;                 // largest m, n and k of a small instance
constexpr size_t kSmallSmemMax = 232448;      // dynamic shared memory of one CTA
struct SmallItem {
  int32_t first;  // position in the plan's small-instance list
  int16_t count;  // instances (<= the groups per CTA for this t)
  int16_t t;      // padded edge: 16, 32 or 64
};
struct SmallArgs {
  const SInst* inst;
  const int32_t* ids;  // small-instance list (instance indices)
  const SmallItem* items;
  int64_t nitems;
  const double* A;
  const double* B;
  double* C;
  Scalars sc;
  int skip_product;  // alpha == 0: C = beta C
};

// ---- small device helpers --------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void record_error(int* err, int code, int loc, int detail) {
  if (atomicCAS(err, 0, code) == 0) {
    err[1] = loc;
    err[2] = detail;
  }
  atomicAdd(err + 3, 1);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase with the given parity; gives up (returns false) after
// kWaitNs or when another role has raised the abort flag.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          const volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long deadline = globaltimer_ns() + kWaitNs;
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (globaltimer_ns() > deadline) return false;
  }
  return true;
}

// Waits for the phase with the given parity for at most kWaitNs, ignoring the
// abort flag (used to let in-flight copies and MMAs finish before exit).
__device__ __forceinline__ bool mbar_wait_time(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long deadline = globaltimer_ns() + kWaitNs;
  while (!mbar_try_wait(bar, parity))
    if (globaltimer_ns() > deadline) return false;
  return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (the layout the slicer writes).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // SWIZZLE_128B
  return d;
}

// Instruction descriptor: kind::f16, A = B = BF16, D = FP32, both K-major, M x N.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---- digits --------------------------------------------------------------------------------

// Exponent e with |x| < 2^e for the largest magnitude of a line, from the bit
// pattern of that magnitude (0 for an all-zero line).
__device__ __forceinline__ int line_exponent(unsigned long long maxbits) {
  if (maxbits == 0) return 0;
  const int eb = (int)(maxbits >> 52) & 0x7FF;
  if (eb != 0) return eb - 1022;
  const unsigned long long frac = maxbits & ((1ull << 52) - 1);
  return (64 - __clzll((long long)frac)) - 1074;
}

// Per-kernel constants of the digit cut: digit width beta, half = 2^(beta-1),
// the balancing bias sum_{p=1..S} half 2^(beta (S-p)) and 2^-beta.
struct DigitCtx {
  int beta, half, mask;
  bool narrow;  // S beta <= 60: the fixed-point value fits 64-bit arithmetic
  long long bias64;
  __int128 bias;
  float step;
};

template <int S>
__device__ __forceinline__ DigitCtx digit_ctx(int beta) {
  DigitCtx c;
  c.beta = beta;
  c.half = 1 << (beta - 1);
  c.mask = (1 << beta) - 1;
  c.narrow = S * beta <= 60;
  c.bias = 0;
#pragma unroll
  for (int p = 0; p < S; ++p) c.bias = (c.bias << beta) + c.half;
  c.bias64 = (long long)c.bias;
  c.step = __int_as_float((127 - beta) << 23);
  return c;
}

// Balanced base-2^beta digits of round(x 2^(S beta - e)), most significant
// first: d[0] = d_1 ... d[S-1] = d_S, with |d_1| <= 2^beta and
// -2^(beta-1) <= d_p < 2^(beta-1) for p >= 2. The magnitude is rounded half
// up, then the sign applied; the balanced form comes from adding the bias
// and reading beta-bit fields. Returns the absolute digit weight
// alpha = sum_p |d_p| 2^(-beta (p-1)) (FP32) used for the norm bound.
template <int S>
__device__ __forceinline__ float make_digits(double x, int e, const DigitCtx& c, int* d) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int eb = (int)(bits >> 52) & 0x7FF;
  unsigned long long M = bits & ((1ull << 52) - 1);
  int q;
  if (eb == 0) {
    q = -1074;
  } else {
    M |= 1ull << 52;
    q = eb - 1075;
  }
  const int sh = q - e + S * c.beta;
  const bool neg = (bits >> 63) != 0;
  if (c.narrow) {
    unsigned long long N = 0;
    if (M != 0) {
      if (sh >= 0) N = M << sh;
      else if (sh > -64) N = (M + (1ull << (-sh - 1))) >> (-sh);
    }
    long long Np = (neg ? -(long long)N : (long long)N) + c.bias64;
#pragma unroll
    for (int p = S - 1; p >= 1; --p) {
      d[p] = (int)(Np & c.mask) - c.half;
      Np >>= c.beta;
    }
    d[0] = (int)Np - c.half;
  } else {
    unsigned __int128 N = 0;
    if (M != 0) {
      if (sh >= 0) N = (unsigned __int128)M << sh;
      else if (sh > -64) N = (unsigned __int128)((M + (1ull << (-sh - 1))) >> (-sh));
    }
    __int128 Np = (neg ? -(__int128)N : (__int128)N) + c.bias;
#pragma unroll
    for (int p = S - 1; p >= 1; --p) {
      d[p] = (int)((long long)Np & c.mask) - c.half;
      Np >>= c.beta;
    }
    d[0] = (int)(long long)Np - c.half;
  }
  float alpha = 0.f, w = 1.f;
#pragma unroll
  for (int p = 0; p < S; ++p) {
    alpha = fmaf((float)abs(d[p]), w, alpha);
    w *= c.step;
  }
  return alpha;
}

// BF16 bit pattern of a small integer (|d| <= 256), exact.
__device__ __forceinline__ uint32_t bf16_of_int(int d) {
  const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
  return __float_as_uint(f) >> 16;
}

// round(x 2^(S BETA - e)) + bias as a 64-bit two's-complement value, in its
// two 32-bit halves (S BETA <= 60: the narrow cut); ties round away from zero.
// With |x| = M 2^(q) (M < 2^53 the integer significand), the magnitude is
// M >> r rounded, r = e - S BETA - q: (M + 2^(r-1)) >> r, computed as
// ((M >> (r-1)) + 1) >> 1, and 0 once r > 53. A non-positive r (a line of
// subnormals only) shifts left.
template <int S, int BETA>
__device__ __forceinline__ void biased_fixed(double x, int e, long long bias, uint32_t& lo,
                                             uint32_t& hi) {
  static_assert(S * BETA <= 60, "narrow cut only");
  const uint32_t xh = (uint32_t)__double2hiint(x), xl = (uint32_t)__double2loint(x);
  const int eb = (int)(xh >> 20) & 0x7FF;
  const unsigned long long M =
      (unsigned long long)((xh & 0xFFFFFu) | (eb != 0 ? 0x100000u : 0u)) << 32 | xl;
  // q = max(eb, 1) - 1075
  const int r = e - S * BETA + 1075 - (eb > 1 ? eb : 1);
  unsigned long long N;
  if (r >= 1) {
    N = r <= 53 ? ((M >> (r - 1)) + 1) >> 1 : 0ull;
  } else {
    N = M << (-r);
  }
  const long long Np = ((xh >> 31) ? -(long long)N : (long long)N) + bias;
  lo = (uint32_t)Np;
  hi = (uint32_t)((unsigned long long)Np >> 32);
}

// a - b on two packed BF16 values (round to nearest; exact for the small
// integers used here)
__device__ __forceinline__ uint32_t bf16x2_sub(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("sub.rn.bf16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// The balanced digits of make_digits with S and BETA known at compile time
// and S BETA <= 60 (the cut the slice kernels use for the documented modes),
// read from the two 32-bit halves of the biased 64-bit fixed-point value
// (biased_fixed) with constant shifts: digit p (1-based) is the BETA-bit field
// at bit BETA (S - p), minus HALF, the top one the arithmetic remainder above.
//
// Lower digit p >= 2 (index p - 1 >= 1) for two values at once, packed as the
// BF16 pair the tiles hold: bf16(d(x1)) << 16 | bf16(d(x0)). The digit is
// field - HALF with 0 <= field < 2^BETA <= 128: both fields go under the BF16
// pattern of 128 (0x4300, whose 7 fraction bits then count units), which makes
// 128 + field exactly, and one packed BF16 subtraction of 128 + HALF leaves
// field - HALF, also exact. A field inside one 16-bit window of a 32-bit half
// is gathered for both values with one byte permute and one shift.
template <int S, int BETA>
__device__ __forceinline__ uint32_t lower_digit_pair(int p, uint32_t lo0, uint32_t hi0,
                                                     uint32_t lo1, uint32_t hi1) {
  static_assert(BETA <= 7, "fields must stay below 128");
  constexpr int HALF = 1 << (BETA - 1), MASK = (1 << BETA) - 1;
  constexpr uint32_t kFields = (uint32_t)MASK * 0x10001u;
  constexpr uint32_t kBase = 0x43004300u;                           // (128, 128)
  constexpr uint32_t kSub = (0x4300u + (uint32_t)HALF) * 0x10001u;  // (128 + HALF) twice
  const int off = BETA * (S - 1 - p);
  uint32_t both;
  if (off + BETA <= 32 || off >= 32) {
    const uint32_t w0 = off >= 32 ? hi0 : lo0, w1 = off >= 32 ? hi1 : lo1;
    const int o = off >= 32 ? off - 32 : off;  // field at bits [o, o + BETA) of w
    const int b = o / 8 < 2 ? o / 8 : 2;       // 16-bit window from byte b
    if (o - 8 * b + BETA <= 16) {
      // bytes b, b+1 of w0 below bytes b, b+1 of w1, then one shift for both
      const uint32_t sel = (uint32_t)b | (uint32_t)(b + 1) << 4 | (uint32_t)(b + 4) << 8 |
                           (uint32_t)(b + 5) << 12;
      both = __byte_perm(w0, w1, sel) >> (o - 8 * b);
    } else {
      both = __byte_perm(w0 >> o, w1 >> o, 0x5410);
    }
  } else {
    both = __byte_perm(__funnelshift_r(lo0, hi0, off), __funnelshift_r(lo1, hi1, off), 0x5410);
  }
  return bf16x2_sub((both & kFields) | kBase, kSub);
}

// Top digit d_1 (|d_1| <= 2^BETA, possibly below -HALF) as
// an exact FP32 value, from the biased fixed-point halves.
template <int S, int BETA>
__device__ __forceinline__ float top_digit(uint32_t lo, uint32_t hi) {
  constexpr int HALF = 1 << (BETA - 1);
  constexpr int kMagic = 0x4B400000 - HALF;
  constexpr int off0 = BETA * (S - 1);
  int top;
  if constexpr (off0 >= 32) top = (int)hi >> (off0 - 32);
  else top = (int)__funnelshift_r(lo, hi, off0);
  return __int_as_float(kMagic + top) - 12582912.0f;
}

// Norm exponent: smallest R with sqrt(S) < 2^R (with a margin for the FP32
// rounding of S); -126 for S == 0.
__device__ __forceinline__ int norm_exponent(float S) {
  if (!(S > 0.f)) return -126;
  const float S2 = S * 1.03125f;
  const int E = (int)((__float_as_uint(S2) >> 23) & 0xFF) - 126;
  return (E + 1) >> 1;
}

// Value of the virtual real matrix A' (m' x k') at (r, q); A is real or
// complex (expanded 2x2 per entry).
__device__ __forceinline__ double valA(const double* A, const SInst& in, int cplx, int r, int q) {
  if (!cplx) return __ldg(A + in.a_off + r + (int64_t)q * in.lda);
  const double2 z =
      __ldg(reinterpret_cast<const double2*>(A) + in.a_off + (r >> 1) + (int64_t)(q >> 1) * in.lda);
  const int sel = ((r & 1) << 1) | (q & 1);
  return sel == 0 ? z.x : sel == 1 ? -z.y : sel == 2 ? z.y : z.x;
}

// Value of B' (k' x n) at (q, c): the real view of B.
__device__ __forceinline__ double valB(const double* B, const SInst& in, int cplx, int q, int c) {
  if (!cplx) return __ldg(B + in.b_off + q + (int64_t)c * in.ldb);
  return __ldg(B + 2 * in.b_off + q + (int64_t)c * 2 * in.ldb);
}

// ---- GEMM --------------------------------------------------------------------------------------

struct GemmBars {
  uint64_t b_full[2];
  uint64_t b_empty[2];
  uint64_t a_full[kMaxAGroups];   // A ring group g holds its planes
  uint64_t a_empty[kMaxAGroups];  // the MMAs are done with A ring group g
  uint64_t lvl_full[kMaxSlices];  // entry i: the levels of plane group i are complete
  uint64_t acc_full[2];   // double-buffered TMEM: accumulator copy b holds a finished tile
  uint64_t acc_empty[2];  // double-buffered TMEM: the epilogue has emptied copy b
  uint64_t tmem_free;
  uint64_t mma_done;
  uint32_t tmem_base;
  int abort_flag;
};

// Resolves the tiles and meta block of a unit. In chain mode the A side is
// the pool matrix named by the walker's index for this step; an index out of
// range or naming a matrix of another size makes the unit invalid (returns
// false): every role then skips it and the walker's output is left as is.
__device__ __forceinline__ bool unit_tiles(const GemmArgs& g, const SplitUnit& U, int64_t* at,
                                           int64_t* bt, int* ablk) {
  *bt = U.b_tile0;
  if (g.idx) {
    const int w = g.order[U.pos];
    const int j = g.idx[w];
    if (j < 0 || j >= g.pool_count || g.pool[j].n != g.inst[w].n) {
      *at = 0;
      *ablk = 0;
      return false;
    }
    *at = g.pool_tile0[j] + U.a_tile0;
    *ablk = g.pool_blk0[j] + U.a_blk;
    return true;
  }
  *at = U.a_tile0;
  *ablk = U.a_blk;
  return true;
}

__device__ __forceinline__ int unit_passes(const GemmArgs& g, const SplitUnit& U) {
  if (g.skip_product || U.nkb <= 0) return 0;
  return (U.nkb + g.kpass - 1) / g.kpass;
}

// Out-of-range tail of fixed_to_double (a result below the normal range or
// above it): kept out of line so that the common path stays free of FP64
// instructions (each warp-wide FP64 instruction holds GB300's FP64 pipe for
// about 64 clocks).
static __device__ __noinline__ double fixed_to_double_slow(unsigned long long sign,
                                                    unsigned long long mant, int ex) {
  const double v = scalbn((double)mant, ex - 52);
  return sign ? -v : v;
}

// Exactly rounded FP64 value of a * 2^E (a a 64-bit integer), by integer
// operations (round to nearest even); FP64 scaling only outside the normal
// range.
__device__ __forceinline__ double fixed_to_double(long long a, int E) {
  if (a == 0) return 0.0;
  const unsigned long long sign = a < 0 ? (1ull << 63) : 0ull;
  const unsigned long long u = a < 0 ? (unsigned long long)(-a) : (unsigned long long)a;
  const int lz = __clzll((long long)u);
  const unsigned long long un = u << lz;
  unsigned long long mant = un >> 11;
  const unsigned long long rem = un & 0x7FFull;
  mant += (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) ? 1ull : 0ull;
  int ex = 63 - lz + E;
  if (mant >> 53) {
    mant >>= 1;
    ex += 1;
  }
  const int biased = ex + 1023;
  if (__builtin_expect(biased >= 1 && biased <= 2046, 1))
    return __longlong_as_double((long long)(sign | ((unsigned long long)biased << 52) |
                                            (mant & ((1ull << 52) - 1))));
  return fixed_to_double_slow(sign, mant, ex);
}

// Branch-free form of fixed_to_double for the normal range, so that a group
// of conversions compiles to straight-line code the scheduler can interleave.
// Sets `bad` when the result is not a normal FP64 number (or a == 0 is not
// the case and the exponent is out of range); the caller then redoes that
// element with fixed_to_double. a == 0 gives 0.0 without setting `bad`.
__device__ __forceinline__ double fixed_to_double_fast(long long a, int E, bool& bad) {
  const unsigned long long sign = (unsigned long long)a & (1ull << 63);
  const unsigned long long u = a < 0 ? 0ull - (unsigned long long)a : (unsigned long long)a;
  const int lz = __clzll((long long)u);  // 64 for u == 0
  const unsigned long long un = u << (lz & 63);
  unsigned long long mant = un >> 11;
  const unsigned long long rem = un & 0x7FFull;
  mant += (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) ? 1ull : 0ull;
  const unsigned long long carry = mant >> 53;  // rounding overflowed into bit 53
  mant >>= carry;
  const int biased = 63 - lz + E + 1023 + (int)carry;
  const bool zero = u == 0;
  bad = bad || (!zero && (biased < 1 || biased > 2046));
  const unsigned long long bits =
      sign | ((unsigned long long)(biased & 0x7FF) << 52) | (mant & ((1ull << 52) - 1));
  return zero ? 0.0 : __longlong_as_double((long long)bits);
}

// The small-instance kernel (split_small.cu): slice counts and digit widths it
// has compiled versions for, instances per work item, shared memory, launch.
bool split_small_supported(int s, int beta);
bool split_small_route(int s, int64_t m, int64_t n, int64_t k);  // instance to this kernel?
int split_small_groups(int s, int t);  // instances per item for padded edge t
size_t split_small_smem(int s);
cudaError_t launch_split_small(int s, int grid, cudaStream_t st, const SmallArgs& g);

// GEMM launchers, one per element type (split_gemm_r64.cu, split_gemm_c128.cu).
cudaError_t launch_split_gemm_r64(int s, int grid, size_t smem, cudaStream_t st, const GemmArgs& g);
cudaError_t launch_split_gemm_c128(int s, int grid, size_t smem, cudaStream_t st, const GemmArgs& g);
cudaError_t set_split_gemm_attr_r64(int s);
cudaError_t set_split_gemm_attr_c128(int s);

}  // namespace splitk
}  // namespace bg
