// Split-precision path of Eq. (1): FP64 operands cut into BF16 digit planes,
// multiplied on the 5th-generation tensor cores (tcgen05, accumulators in
// TMEM) with FP32 sums that are exact by construction, recombined exactly
// in integer arithmetic and rounded once to FP64.
//
// The paper computes its GEMMs in complex FP64 through cuBLAS (Sec. 4) and has
// no such mode; it is the GB300 answer to an FP64 pipe that issues only 2
// DFMA per clock per SM. The method, step by step:
//
//  1. Scale. Row i of A gets the exponent e_i with max_p |A_ip| < 2^e_i, column
//     j of B the exponent f_j with max_p |B_pj| < 2^f_j (0 for an all-zero line).
//  2. Cut. a = A_ip 2^(beta - e_i) lies in (-2^beta, 2^beta). Its fixed-point
//     value N = round(a 2^(beta (s-1))) is written in balanced base 2^beta:
//     N = sum_{p=1..s} d_p 2^(beta (s-p)), |d_1| <= 2^beta, |d_p| <= 2^(beta-1)
//     (p >= 2). Every digit is an integer of at most 9 significant bits, hence
//     exact in BF16. Same for B per column.
//  3. Multiply. For each level t = p + q (2 <= t <= s+1, the triangular set of
//     plane pairs), L_t = sum_{p+q=t} D_p^A D_q^B on the tensor cores. The digit
//     width is chosen (host: level_pass()) so that every partial sum of a level
//     stays below 2^24 over a pass of k: the FP32 accumulation is exact; longer
//     k runs in several passes whose FP64 results are summed into C.
//  4. Recombine. G_ij = sum_t L_t 2^(-beta (t-2)) is accumulated per element in
//     a 64-bit fixed-point integer whose frame is set from bounds on the row and
//     column digit norms (so it cannot overflow and keeps >= 60 bits of the
//     result), then converted to FP64 with one correct rounding and scaled by
//     2^(e_i + f_j - 2 beta). alpha and beta of Eq. (1) are applied in FP64.
//
// Complex instances run as real ones through the real representation of a
// complex number: B and C viewed as real matrices with interleaved (re, im)
// rows (k' = 2k, ldb' = 2 ldb; m' = 2m, ldc' = 2 ldc) and each entry a of A
// expanded to [[re a, -im a], [im a, re a]]; exponents are then shared by the
// real and imaginary parts of a row of A / a column of B.
//
// Kernels:
//  * split_slice_kernel: one CTA per line block (128 rows of A, or BN columns
//    of B), or per part of one: exponents, digit planes written as
//    pre-swizzled BF16 tiles of 64 k (the exact SWIZZLE_128B K-major
//    shared-memory image), the s planes of one k-block stored next to each
//    other, per-line norm exponents. Integer arithmetic, plus exact
//    conversions of small integers to FP32 and BF16.
//  * split_gemm_kernel<BN>: persistent, one CTA per SM, warp-specialised.
//    Output tile 128 x BN with BN = the largest multiple of 16 with
//    s BN <= 512, so that the s level accumulators (one per t) all live in
//    TMEM at once. Per k-block, warp 0 copies the s B planes with one 1-D TMA
//    bulk copy (cp.async.bulk) and streams the s A planes through a ring of
//    16 KiB slots; warp 1 issues, for each A plane p, one tcgen05.mma over the
//    N-concatenation of B planes 1..s+1-p, which lands every product of the
//    plane pair (p, q) in the accumulator of its level p + q -- one A tile
//    and one B tile read per plane instead of per plane pair. Warps 2-9 drain
//    each level as soon as its last MMA completes, do the integer
//    recombination, free TMEM and then convert and store while the next tile
//    is already being multiplied.
//    Small instances are packed along the diagonal of a 128 x BN tile.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "split_common.cuh"

namespace bg {

using namespace splitk;

namespace {

// ---- slicer ----------------------------------------------------------------------------------

// Tile layout (A and B alike): the tile of plane p (0-based) and k-block kb
// of a block is tile number tile0 + kb * S + p; tiles are `lines` rows of 128
// bytes (64 BF16 values of k), chunk c of row r stored at chunk c ^ (r & 7).
//
// Work distribution: the (group of 4 lines) x (k-block) items of a block are
// dealt to the CTA's warps; a warp covers 4 lines x 8 chunks of 8 k values,
// so each plane store writes 4 whole 128-byte rows (512 contiguous bytes)
// and every lane keeps 8 values in flight. Line maxima and norm sums meet in
// shared memory through integer atomics (max, and sums of fixed-point
// squares), so the result does not depend on the order of the items.

// Where line l of a job's block starts in its operand, and how far apart its
// consecutive k' values lie; built once per job in shared memory.
//   rows of A, real:    x(k') = A[off + k' ld]
//   rows of A, complex: z = A[off + (k' / 2) ld] in double2 units; row 2r of
//                       the 2 x 2 expansion reads (re, -im), row 2r+1 (im, re)
//   columns of B:       x(k') = B[off + k'] (complex: re, im interleaved)
// off < 0 marks a line beyond its instance. ldx = 2 ld + (odd complex row).
struct LineSrc {
  int64_t off, ldx;
};

__device__ __forceinline__ LineSrc line_src(const SliceArgs& a, const SliceJob& J, bool isA,
                                            int l) {
  LineSrc r{-1, 0};
  const int li = l / J.span;
  const int line = J.org + l % J.span;
  if (li >= J.g) return r;
  const SInst in = isA ? a.instA[a.orderA[J.pos + li]] : a.instB[a.orderB[J.pos + li]];
  if (!(isA ? line < (a.cplx ? 2 * in.m : in.m) : line < in.n)) return r;
  if (isA || a.herk) {
    // Hermitian update, B side: column j of B = A^H is row j of A conjugated,
    // which in the real view is row 2j of A's 2 x 2 expansion (re, -im)
    const int row = isA ? line : (a.cplx ? 2 * line : line);
    r.off = a.cplx ? in.a_off + (row >> 1) : in.a_off + row;
    r.ldx = 2 * in.lda + (a.cplx ? (row & 1) : 0);
  } else {
    r.off = a.cplx ? 2 * in.b_off + (int64_t)line * 2 * in.ldb : in.b_off + (int64_t)line * in.ldb;
    r.ldx = 2;
  }
  return r;
}

// The 8 values x[u] = (line, k' = q0 + u) of the block's operand, 0 beyond
// k' or for a line beyond its instance; rows: the lines are rows of A.
__device__ __forceinline__ void load8(const SliceArgs& a, bool rows, LineSrc src, int q0, int kv,
                                      double (&x)[8]) {
  if (src.off < 0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = 0.0;
    return;
  }
  const int64_t ld = src.ldx >> 1;
  if (rows) {
    if (!a.cplx) {
      const double* p = a.A + src.off + (int64_t)q0 * ld;
      if (q0 + 8 <= kv) {
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = __ldg(p + (int64_t)u * ld);
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = q0 + u < kv ? __ldg(p + (int64_t)u * ld) : 0.0;
      }
    } else {
      const double2* p = reinterpret_cast<const double2*>(a.A) + src.off + (int64_t)(q0 >> 1) * ld;
      const bool im_row = src.ldx & 1;
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        const double2 z = q0 + u < kv ? __ldg(p + (int64_t)(u >> 1) * ld) : make_double2(0.0, 0.0);
        x[u] = im_row ? z.y : z.x;
        x[u + 1] = q0 + u + 1 < kv ? (im_row ? z.x : -z.y) : 0.0;
      }
    }
  } else {
    const double* p = a.B + src.off + q0;
    // 16-byte loads where the column allows them (a real B with an odd ldb or
    // offset puts every other column on an 8-byte boundary)
    const bool vec = (reinterpret_cast<uintptr_t>(p) & 15) == 0;
    if (vec && q0 + 8 <= kv) {
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        const double2 z = __ldg(reinterpret_cast<const double2*>(p + u));
        x[u] = z.x;
        x[u + 1] = z.y;
      }
      return;
    }
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
      if (vec && q0 + u + 1 < kv) {
        const double2 z = __ldg(reinterpret_cast<const double2*>(p + u));
        x[u] = z.x;
        x[u + 1] = z.y;
      } else {
        x[u] = q0 + u < kv ? __ldg(p + u) : 0.0;
        x[u + 1] = q0 + u + 1 < kv ? __ldg(p + u + 1) : 0.0;
      }
    }
  }
}

// Line maximum of the 8 values of a lane, merged over the 8 lanes of the line
// and into s_max. Only line_exponent of the largest |x| is used, and it sees
// the same value in the pair of separate maxima of the 32-bit halves (sign
// cleared): the exponent field sits in the high half, and where every
// exponent is zero, the largest high half, or when those are all zero the
// largest low half, holds the highest fraction bit. Merging such pairs as
// 64-bit values keeps this.
__device__ __forceinline__ void merge_max(const double (&x)[8], int cc, unsigned long long* s_max_l) {
  uint32_t mh = 0, ml = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    mh = max(mh, (uint32_t)__double2hiint(x[u]) & 0x7FFFFFFFu);
    ml = max(ml, (uint32_t)__double2loint(x[u]));
  }
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    mh = max(mh, __shfl_xor_sync(0xFFFFFFFFu, mh, o));
    ml = max(ml, __shfl_xor_sync(0xFFFFFFFFu, ml, o));
  }
  const unsigned long long mx = (unsigned long long)mh << 32 | ml;
  if (cc == 0 && mx) atomicMax(s_max_l, mx);
}

// Digit planes of the 8 values of a lane (chunk cc of a line with exponent e),
// stored at dst (plane p at dst + p tile_bytes); the line's sum of squared
// absolute digit weights is merged into s_n2.
template <int S, int BETA>
__device__ __forceinline__ void cut_item(const double (&x)[8], int e, const DigitCtx& dc,
                                         uint8_t* dst, int tile_bytes, int cc,
                                         unsigned long long* s_n2_l) {
  float n2f = 0.f;
  if constexpr (BETA > 0) {
    // plane by plane from the 8 biased fixed-point values: each plane's 16
    // bytes are stored as soon as they are cut
    uint32_t lo[8], hi[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) biased_fixed<S, BETA>(x[u], e, dc.bias64, lo[u], hi[u]);
    uint32_t w0[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float f0 = top_digit<S, BETA>(lo[2 * v], hi[2 * v]);
      const float f1 = top_digit<S, BETA>(lo[2 * v + 1], hi[2 * v + 1]);
      w0[v] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
      const float al0 = fabsf(f0) + 0.51f, al1 = fabsf(f1) + 0.51f;
      n2f = fmaf(al0, al0, n2f);
      n2f = fmaf(al1, al1, n2f);
    }
    *reinterpret_cast<uint4*>(dst) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
#pragma unroll
    for (int p = 1; p < S; ++p)
      *reinterpret_cast<uint4*>(dst + (int64_t)p * tile_bytes) =
          make_uint4(lower_digit_pair<S, BETA>(p, lo[0], hi[0], lo[1], hi[1]),
                     lower_digit_pair<S, BETA>(p, lo[2], hi[2], lo[3], hi[3]),
                     lower_digit_pair<S, BETA>(p, lo[4], hi[4], lo[5], hi[5]),
                     lower_digit_pair<S, BETA>(p, lo[6], hi[6], lo[7], hi[7]));
  } else {
    uint32_t w[S][4];
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
      int d0[S], d1[S];
      const float al0 = make_digits<S>(x[u], e, dc, d0);
      const float al1 = make_digits<S>(x[u + 1], e, dc, d1);
#pragma unroll
      for (int p = 0; p < S; ++p) w[p][u >> 1] = bf16_of_int(d0[p]) | (bf16_of_int(d1[p]) << 16);
      n2f = fmaf(al0, al0, n2f);
      n2f = fmaf(al1, al1, n2f);
    }
#pragma unroll
    for (int p = 0; p < S; ++p)
      *reinterpret_cast<uint4*>(dst + (int64_t)p * tile_bytes) =
          make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
  }
  // 8 values of at most 257.51^2 each, in units of 2^-8: < 2^28 per lane; 8 lanes < 2^31
  uint32_t n2 = __float2uint_ru(n2f * 256.0f * 1.0001f);
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) n2 += __shfl_xor_sync(0xFFFFFFFFu, n2, o);
  if (cc == 0 && n2) atomicAdd(s_n2_l, (unsigned long long)n2);
}

// Advances a warp's item (group g of 4 lines, k-block kb) by `step` items in
// the group-fastest order, without a division.
__device__ __forceinline__ void next_item(int& g, int& kb, int step, int groups) {
  g += step;
  while (g >= groups) {
    g -= groups;
    ++kb;
  }
}

// BETA > 0: compile-time digit width (S * BETA <= 60); BETA == 0: any width a.beta.
// The compile-time cuts run six CTAs per SM (at most 40 registers a thread):
// the kernel is bound by memory latency, and 48 warps per SM hide it better
// than 40 (measured 3.41 -> 3.35 ms for 9 slices on the 20000-instance size
// mix; seven or eight CTAs, with fewer registers, are slower). The generic cut keeps four,
// where five would spill.
template <int S, int BETA>
__global__ void __launch_bounds__(kSliceThreads, BETA > 0 ? 6 : 4)
    split_slice_kernel(const SliceArgs a) {
  const DigitCtx dc = digit_ctx<S>(BETA > 0 ? BETA : a.beta);
  __shared__ unsigned long long s_max[128];
  __shared__ unsigned long long s_n2[128];  // sum of alpha^2 in units of 2^-8 (rounded up)
  __shared__ int s_e[128];
  __shared__ LineSrc s_src[128];            // the job's lines, job-relative
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int cc = lane & 7;        // chunk of 8 k values inside a 64-wide k-block
  const int lsub = lane >> 3;     // line within the warp's group of 4
  constexpr int kWarps = kSliceThreads / 32;
  for (int64_t jb = blockIdx.x; jb < a.njobs; jb += gridDim.x) {
    const SliceJob J = a.jobs[jb];
    const bool isA = J.side == 0;
    const bool rows = isA || a.herk;
    const int kv = J.kv;
    const int lines = isA ? BM : a.bn;
    const int groups = J.nl / 4;  // the job's lines [l0, l0 + nl) in groups of 4
    if (groups <= 0) continue;    // (the planner makes none; same for every thread)
    const int tile_bytes = lines * kLineBytes;
    uint8_t* tiles = isA ? a.tilesA : a.tilesB;
    if (t < 128) {
      s_max[t] = 0;
      s_n2[t] = 0;
    }
    if (t < J.nl) s_src[t] = line_src(a, J, isA, J.l0 + t);
    __syncthreads();
    // ---- phase 1: line maxima (exponents). Lines beyond their instance only
    // meet discarded outputs: a group of 4 such lines is skipped here and in
    // phase 2 (its tile rows keep whatever finite digits they hold; the
    // planner zeroes them once).
    {
      int g = 0, kb = 0;
      next_item(g, kb, warp, groups);
      while (kb < J.nkb) {
        const int r = g * 4 + lsub;
        const LineSrc src = s_src[r];
        if (__any_sync(0xFFFFFFFFu, src.off >= 0)) {
          double x[8];
          load8(a, rows, src, kb * BK + 8 * cc, kv, x);
          merge_max(x, cc, &s_max[J.l0 + r]);
        }
        next_item(g, kb, kWarps, groups);
      }
    }
    __syncthreads();
    if (t < 128) s_e[t] = line_exponent(s_max[t]);
    __syncthreads();
    // ---- phase 2: digit planes and the norm of the absolute digit weights
    {
      int g = 0, kb = 0;
      next_item(g, kb, warp, groups);
      while (kb < J.nkb) {
        const int r = g * 4 + lsub;
        const LineSrc src = s_src[r];
        if (__any_sync(0xFFFFFFFFu, src.off >= 0)) {
          const int l = J.l0 + r;
          double x[8];
          load8(a, rows, src, kb * BK + 8 * cc, kv, x);
          uint8_t* dst = tiles + (J.tile0 + (int64_t)kb * S) * tile_bytes + l * kLineBytes +
                         ((cc ^ (l & 7)) << 4);
          cut_item<S, BETA>(x, s_e[l], dc, dst, tile_bytes, cc, &s_n2[l]);
        }
        next_item(g, kb, kWarps, groups);
      }
    }
    __syncthreads();
    // ---- phase 3: meta of the job's lines (exponent, norm exponent)
    int32_t* meta = (isA ? a.metaA : a.metaB) + (int64_t)J.blk * kMetaStride;
    if (t >= J.l0 && t < J.l0 + J.nl) {
      meta[t] = s_e[t];
      meta[128 + t] = norm_exponent((float)s_n2[t] * (1.0f / 256.0f));
    }
    __syncthreads();
  }
}

// ---- standalone plane cut (exposed for checking the digit arithmetic) ------------------------

__global__ void planes_exp_kernel(int64_t m, int64_t k, const double* X, int64_t ldx, int axis,
                                  int32_t* exps) {
  const int64_t lines = axis == 0 ? m : k;
  const int64_t len = axis == 0 ? k : m;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < lines;
       l += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long mx = 0;
    for (int64_t i = 0; i < len; ++i) {
      const double x = axis == 0 ? X[l + i * ldx] : X[i + l * ldx];
      const unsigned long long b =
          (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
      mx = b > mx ? b : mx;
    }
    exps[l] = line_exponent(mx);
  }
}

template <int S>
__global__ void planes_digit_kernel(int64_t m, int64_t k, const double* X, int64_t ldx, int axis,
                                    int beta, const int32_t* exps, uint16_t* digits) {
  const DigitCtx dc = digit_ctx<S>(beta);
  const int64_t total = m * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % m, c = e / m;
    int d[S];
    make_digits<S>(X[r + c * ldx], exps[axis == 0 ? r : c], dc, d);
#pragma unroll
    for (int p = 0; p < S; ++p) digits[(int64_t)p * total + e] = (uint16_t)bf16_of_int(d[p]);
  }
}

// Expands the variadic body once per slice count S = 1..12 and runs the one
// matching `s`.
#define BG_DISPATCH_SLICES(s, ...)                      \
  switch (s) {                                          \
    case 1: { constexpr int S = 1; __VA_ARGS__; }       \
    case 2: { constexpr int S = 2; __VA_ARGS__; }       \
    case 3: { constexpr int S = 3; __VA_ARGS__; }       \
    case 4: { constexpr int S = 4; __VA_ARGS__; }       \
    case 5: { constexpr int S = 5; __VA_ARGS__; }       \
    case 6: { constexpr int S = 6; __VA_ARGS__; }       \
    case 7: { constexpr int S = 7; __VA_ARGS__; }       \
    case 8: { constexpr int S = 8; __VA_ARGS__; }       \
    case 9: { constexpr int S = 9; __VA_ARGS__; }       \
    case 10: { constexpr int S = 10; __VA_ARGS__; }     \
    case 11: { constexpr int S = 11; __VA_ARGS__; }     \
    case 12: { constexpr int S = 12; __VA_ARGS__; }     \
    default: return cudaErrorInvalidValue;              \
  }

}  // namespace

cudaError_t launch_split_planes(int64_t m, int64_t k, const double* X, int64_t ldx, int axis,
                                int slices, int beta_bits, int32_t* exps, uint16_t* digits,
                                cudaStream_t st) {
  const int64_t lines = axis == 0 ? m : k;
  planes_exp_kernel<<<(unsigned)std::min<int64_t>((lines + 255) / 256, 4096), 256, 0, st>>>(
      m, k, X, ldx, axis, exps);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::min<int64_t>((m * k + 255) / 256, 65536);
  BG_DISPATCH_SLICES(slices, {
    planes_digit_kernel<S><<<grid, 256, 0, st>>>(m, k, X, ldx, axis, beta_bits, exps, digits);
    count_launch();
    return cudaGetLastError();
  });
}

// ---- host: plans ------------------------------------------------------------------------------

int split_default_beta(int slices) { return slices <= 6 ? 7 : 6; }

// K-blocks of 64 per pass such that every partial sum of a level's digit
// products stays below 2^24 (exact in FP32): with |d_1| <= 2^beta and
// |d_p| <= 2^(beta-1) for p >= 2, the level-t sum of |d_p d_q| per k is at
// most bound_t; the pass length is set by the largest bound. 0 = impossible.
static int level_pass(int s, int beta) {
  double worst = 0;
  for (int t = 2; t <= s + 1; ++t) {
    double bound = 0;
    for (int p = 1; p < t; ++p) {
      const int q = t - p;
      const double bp = p == 1 ? std::ldexp(1.0, beta) : std::ldexp(1.0, beta - 1);
      const double bq = q == 1 ? std::ldexp(1.0, beta) : std::ldexp(1.0, beta - 1);
      bound += bp * bq;
    }
    worst = std::max(worst, bound);
  }
  const double kc = std::floor(16777216.0 / (worst * BK));
  return (int)std::min(kc, 4096.0);
}

struct SplitPlan {
  bg_dtype dt = BG_R64;
  int s = 0, beta = 0, bn = 0, kpass = 0, a_groups = 0;
  size_t smem = 0;
  bool chain = false;
  bool herk = false;       // Hermitian rank-k updates (B = A^H, lower triangle)
  bool small_ok = false;   // real instances with m, n, k <= 64 go to the small-instance kernel
  std::vector<int8_t> route;  // per instance: 0 rule, 1 small where possible, 2 tiles (may be empty)
  int sms = 0;
  int64_t count = 0;
  // device
  SliceJob* d_jobs = nullptr;
  int64_t n_jobs = 0, n_jobs_A = 0;  // A jobs first (chain plans)
  SplitUnit* d_units = nullptr;
  int64_t n_units = 0;
  SInst* d_inst = nullptr;       // instances (chain: walkers)
  SInst* d_pool = nullptr;       // chain: pool entries
  int32_t* d_order = nullptr;    // A side order (== B side order except chain)
  int32_t* d_small = nullptr;    // instances computed by the small-instance kernel
  SmallItem* d_small_items = nullptr;
  int64_t n_small = 0, n_small_items = 0;
  double small_mnk = 0, small_ab = 0;  // sum of m n k and of m k + k n over small instances
  int32_t* d_pool_order = nullptr;
  int64_t* d_pool_tile0 = nullptr;
  int32_t* d_pool_blk0 = nullptr;
  int32_t n_pool = 0;
  uint8_t* tilesA = nullptr;
  uint8_t* tilesB = nullptr;
  int32_t* metaA = nullptr;
  int32_t* metaB = nullptr;
  int64_t bytes = 0;
  int grid_slice = 0, grid_gemm = 0, grid_small = 0;
  std::vector<int64_t> key;  // fixed-size plan cache key
  std::string desc;
};

SplitWorkspace::~SplitWorkspace() {
  for (auto* p : cache) split_plan_destroy(p);
}

static cudaError_t dalloc(void** p, size_t bytes, int64_t* total) {
  *total += (int64_t)bytes;
  return cudaMalloc(p, std::max<size_t>(bytes, 16));
}

template <class T>
static cudaError_t dput(T** d, const std::vector<T>& v, int64_t* total) {
  cudaError_t e = dalloc(reinterpret_cast<void**>(d), v.size() * sizeof(T), total);
  if (e != cudaSuccess) return e;
  if (!v.empty()) e = cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

void split_plan_destroy(SplitPlan* p) {
  if (!p) return;
  cudaFree(p->d_jobs);
  cudaFree(p->d_units);
  cudaFree(p->d_inst);
  cudaFree(p->d_pool);
  cudaFree(p->d_order);
  cudaFree(p->d_small);
  cudaFree(p->d_small_items);
  cudaFree(p->d_pool_order);
  cudaFree(p->d_pool_tile0);
  cudaFree(p->d_pool_blk0);
  cudaFree(p->tilesA);
  cudaFree(p->tilesB);
  cudaFree(p->metaA);
  cudaFree(p->metaB);
  delete p;
}

int64_t split_plan_workspace(const SplitPlan* p) { return p ? p->bytes : 0; }
int split_plan_launches(const SplitPlan* p) {
  return p ? (p->n_jobs > 0) + (p->n_units > 0) + (p->n_small > 0) : 0;
}
int64_t split_plan_items(const SplitPlan* p) { return p ? p->n_units + p->n_small : 0; }
int split_plan_beta_bits(const SplitPlan* p) { return p ? p->beta : 0; }
std::string split_plan_describe(const SplitPlan* p) { return p ? p->desc : "null"; }

static bg_status set_err(std::string* err, bg_status s, const std::string& msg) {
  *err = msg;
  return s;
}

static bg_status cuda_err(std::string* err, cudaError_t e, const char* what) {
  cudaGetLastError();
  *err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? BG_ERR_NOMEM : BG_ERR_CUDA;
}

static bool setup_common(SplitPlan* p, bg_dtype dt, const bg_precision& pr, int sms,
                         std::string* err) {
  p->dt = dt;
  p->s = pr.slices;
  p->beta = pr.beta_bits ? pr.beta_bits : split_default_beta(pr.slices);
  p->bn = bn_for(p->s);
  p->sms = sms;
  p->kpass = level_pass(p->s, p->beta);
  if (p->kpass < 1) {
    *err = "split mode: digit width too large for exact FP32 sums";
    return false;
  }
  const size_t bbytes = 2 * (size_t)p->s * p->bn * kLineBytes;
  const size_t budget = kMaxDynSmem - 1024 - sizeof(GemmBars);
  p->a_groups =
      (int)std::min<size_t>(kMaxAGroups, (budget - bbytes) / ((size_t)kAGroup * kATileBytes));
  if (p->a_groups < 2) {
    *err = "split mode: shared memory too small for this slice count";
    return false;
  }
  p->smem = 1024 + bbytes + (size_t)p->a_groups * kAGroup * kATileBytes + sizeof(GemmBars);
  return true;
}

static int kmma_last_of(int kv) {
  if (kv <= 0) return 0;
  const int rem = kv - ((kv - 1) / BK) * BK;  // 1..64
  return (rem + 15) / 16;
}

// Cuts a block job whose FP64 values exceed kSliceJobBytes into jobs of
// fewer lines (halving while the count stays a multiple of 4). The slicer
// reads a job's values twice (line maxima, then digits); smaller jobs keep
// what all resident CTAs read between the two passes within L2.
static void split_jobs(std::vector<SliceJob>* jobs, int bn) {
  std::vector<SliceJob> out;
  out.reserve(jobs->size() * 2);
  for (const SliceJob& j : *jobs) {
    const int lines = j.side == 0 ? BM : bn;
    const int64_t line_bytes = (int64_t)j.nkb * BK * 8;
    int nl = lines;
    while (nl * line_bytes > kSliceJobBytes && nl % 2 == 0 && (nl / 2) % 4 == 0) nl /= 2;
    for (int l0 = 0; l0 < lines; l0 += nl) {
      SliceJob sj = j;
      sj.l0 = (int16_t)l0;
      sj.nl = (int16_t)nl;
      out.push_back(sj);
    }
  }
  jobs->swap(out);
}

// Host-side schedule of a (non-chain) split plan: instances, order list,
// slice jobs, GEMM units and the sizes of the tile and meta stores.
struct HostTables {
  std::vector<SInst> inst;
  std::vector<int32_t> order;
  std::vector<SliceJob> jobs;
  std::vector<SplitUnit> units;
  std::vector<int32_t> small;  // instances for the small-instance kernel
  std::vector<SmallItem> small_items;
  int64_t tileA = 0, tileB = 0, n_jobs_A = 0;
  int32_t blkA = 0, blkB = 0;
};

static void make_tables(const SplitPlan* p, const std::vector<bg_instance>& table,
                        HostTables* out) {
  const bool cplx = p->dt == BG_C128;
  const int s = p->s, BN = p->bn;
  std::vector<SInst> inst(table.size());
  for (size_t i = 0; i < table.size(); ++i) {
    const bg_instance& t = table[i];
    inst[i] = SInst{t.a_off, t.b_off, t.c_off, t.lda, t.ldb, t.ldc, (int32_t)t.m, (int32_t)t.n,
                    (int32_t)t.k, 0};
  }
  // group instances of identical shape (packing needs equal shapes); small
  // real instances go to their own kernel
  std::map<std::array<int64_t, 3>, std::vector<int32_t>> groups;
  std::vector<int32_t> small;
  for (size_t i = 0; i < table.size(); ++i) {
    const bg_instance& t = table[i];
    if (t.m == 0 || t.n == 0) continue;
    const int8_t r = p->route.empty() ? 0 : p->route[i];
    const bool fits = std::max(t.m, std::max(t.n, t.k)) <= kSmallMax;
    if (p->small_ok && !cplx && !p->herk && fits &&
        (r == 1 || (r == 0 && split_small_route(s, t.m, t.n, t.k)))) {
      small.push_back((int32_t)i);
      continue;
    }
    groups[{t.m, t.n, t.k}].push_back((int32_t)i);
  }
  // small instances by padded edge (64, 32, 16), largest first within an
  // edge; work items of as many instances as the kernel runs side by side
  auto edge = [&](int32_t i) {
    const int64_t e = std::max(table[i].m, std::max(table[i].n, table[i].k));
    return e <= 16 ? 16 : e <= 32 ? 32 : 64;
  };
  std::stable_sort(small.begin(), small.end(), [&](int32_t a, int32_t b) {
    const int ea = edge(a), eb = edge(b);
    if (ea != eb) return ea > eb;
    return table[a].m * table[a].n * table[a].k > table[b].m * table[b].n * table[b].k;
  });
  std::vector<SmallItem> small_items;
  for (size_t i = 0; i < small.size();) {
    const int e = edge(small[i]);
    const int ng = std::max(1, split_small_groups(s, e));
    size_t j = i;
    while (j < small.size() && j - i < (size_t)ng && edge(small[j]) == e) ++j;
    small_items.push_back(SmallItem{(int32_t)i, (int16_t)(j - i), (int16_t)e});
    i = j;
  }
  std::vector<int32_t> order;
  std::vector<SliceJob> jobsA, jobsB;
  std::vector<SplitUnit> units;
  int64_t tileA = 0, tileB = 0;
  int32_t blkA = 0, blkB = 0;
  for (auto& kv : groups) {
    const int64_t m = kv.first[0], n = kv.first[1], k = kv.first[2];
    const int64_t mv = cplx ? 2 * m : m, kvv = cplx ? 2 * k : k;
    const int nkb = (int)((kvv + BK - 1) / BK);
    const auto& ids = kv.second;
    const int gmax = (int)std::min<int64_t>(BM / mv, BN / n);
    if (gmax >= 2) {
      for (size_t s0 = 0; s0 < ids.size(); s0 += gmax) {
        const int gc = (int)std::min<size_t>(gmax, ids.size() - s0);
        const int32_t pos = (int32_t)order.size();
        for (int i = 0; i < gc; ++i) order.push_back(ids[s0 + i]);
        if (nkb > 0) {
          jobsA.push_back(SliceJob{tileA, blkA, pos, 0, (int16_t)gc, (int16_t)mv, (int16_t)nkb, 0,
                                   (int32_t)kvv});
          jobsB.push_back(SliceJob{tileB, blkB, pos, 1, (int16_t)gc, (int16_t)n, (int16_t)nkb, 0,
                                   (int32_t)kvv});
        }
        SplitUnit U{};
        U.a_tile0 = tileA;
        U.b_tile0 = tileB;
        U.a_blk = blkA;
        U.b_blk = blkB;
        U.pos = pos;
        U.g = (int16_t)gc;
        U.nkb = (int16_t)nkb;
        U.kmma_last = (int16_t)kmma_last_of((int)kvv);
        U.mrow = (int16_t)mv;
        U.ncol = (int16_t)n;
        units.push_back(U);
        tileA += (int64_t)s * nkb;
        tileB += (int64_t)s * nkb;
        ++blkA;
        ++blkB;
      }
    } else {
      for (int32_t id : ids) {
        const int32_t pos = (int32_t)order.size();
        order.push_back(id);
        const int64_t rbs = (mv + BM - 1) / BM, cbs = (n + BN - 1) / BN;
        const int64_t tA0 = tileA, tB0 = tileB;
        const int32_t bA0 = blkA, bB0 = blkB;
        for (int64_t rb = 0; rb < rbs; ++rb) {
          if (nkb > 0)
            jobsA.push_back(SliceJob{tileA, blkA, pos, 0, 1, (int16_t)BM, (int16_t)nkb,
                                     (int32_t)(rb * BM), (int32_t)kvv});
          tileA += (int64_t)s * nkb;
          ++blkA;
        }
        for (int64_t cb = 0; cb < cbs; ++cb) {
          if (nkb > 0)
            jobsB.push_back(SliceJob{tileB, blkB, pos, 1, 1, (int16_t)BN, (int16_t)nkb,
                                     (int32_t)(cb * BN), (int32_t)kvv});
          tileB += (int64_t)s * nkb;
          ++blkB;
        }
        // row blocks inner: the units sharing a B block run side by side (L2 reuse)
        for (int64_t cb = 0; cb < cbs; ++cb)
          for (int64_t rb = 0; rb < rbs; ++rb) {
            // Hermitian update: a tile wholly above the diagonal (its last row,
            // counted in complex rows, before its first column) is not needed
            if (p->herk && ((std::min<int64_t>(mv, (rb + 1) * BM) - 1) >> (cplx ? 1 : 0)) < cb * BN)
              continue;
            SplitUnit U{};
            U.a_tile0 = tA0 + rb * s * nkb;
            U.b_tile0 = tB0 + cb * s * nkb;
            U.a_blk = bA0 + (int32_t)rb;
            U.b_blk = bB0 + (int32_t)cb;
            U.pos = pos;
            U.g = 1;
            U.nkb = (int16_t)nkb;
            U.kmma_last = (int16_t)kmma_last_of((int)kvv);
            U.mrow = (int16_t)std::min<int64_t>(mv, 32767);
            U.ncol = (int16_t)std::min<int64_t>(n, 32767);
            U.r0 = (int32_t)(rb * BM);
            U.c0 = (int32_t)(cb * BN);
            units.push_back(U);
          }
      }
    }
  }
  // longest first
  std::stable_sort(units.begin(), units.end(),
                   [](const SplitUnit& a, const SplitUnit& b) { return a.nkb > b.nkb; });
  std::stable_sort(jobsA.begin(), jobsA.end(),
                   [](const SliceJob& a, const SliceJob& b) { return a.nkb > b.nkb; });
  std::stable_sort(jobsB.begin(), jobsB.end(),
                   [](const SliceJob& a, const SliceJob& b) { return a.nkb > b.nkb; });
  std::vector<SliceJob> jobs;
  size_t ia = 0, ib = 0;
  while (ia < jobsA.size() || ib < jobsB.size()) {
    if (ia < jobsA.size()) jobs.push_back(jobsA[ia++]);
    if (ib < jobsB.size()) jobs.push_back(jobsB[ib++]);
  }
  split_jobs(&jobs, BN);
  out->inst = std::move(inst);
  out->order = std::move(order);
  out->jobs = std::move(jobs);
  out->units = std::move(units);
  out->small = std::move(small);
  out->small_items = std::move(small_items);
  out->tileA = tileA;
  out->tileB = tileB;
  out->blkA = blkA;
  out->blkB = blkB;
  out->n_jobs_A = (int64_t)jobsA.size();
}

// Builds jobs and units for instances (non-chain plans) and allocates the
// plan's device tables and workspace.
static bg_status build_instances(SplitPlan* p, const std::vector<bg_instance>& table,
                                 std::string* err) {
  HostTables t;
  make_tables(p, table, &t);
  const int64_t tileA = t.tileA, tileB = t.tileB;
  const int32_t blkA = t.blkA, blkB = t.blkB;
  p->n_jobs = (int64_t)t.jobs.size();
  p->n_jobs_A = t.n_jobs_A;
  p->n_units = (int64_t)t.units.size();
  p->n_small = (int64_t)t.small.size();
  p->n_small_items = (int64_t)t.small_items.size();
  for (int32_t i : t.small) {
    const bg_instance& x = table[i];
    p->small_mnk += (double)x.m * x.n * x.k;
    p->small_ab += (double)x.m * x.k + (double)x.k * x.n;
  }
  p->count = (int64_t)table.size();
  const size_t btile = (size_t)p->bn * kLineBytes;
  cudaError_t e;
  if ((e = dput(&p->d_jobs, t.jobs, &p->bytes)) != cudaSuccess ||
      (e = dput(&p->d_units, t.units, &p->bytes)) != cudaSuccess ||
      (e = dput(&p->d_inst, t.inst, &p->bytes)) != cudaSuccess ||
      (e = dput(&p->d_order, t.order, &p->bytes)) != cudaSuccess ||
      (e = dput(&p->d_small, t.small, &p->bytes)) != cudaSuccess ||
      (e = dput(&p->d_small_items, t.small_items, &p->bytes)) != cudaSuccess ||
      (e = dalloc(reinterpret_cast<void**>(&p->tilesA), (size_t)tileA * kATileBytes, &p->bytes)) !=
          cudaSuccess ||
      (e = dalloc(reinterpret_cast<void**>(&p->tilesB), (size_t)tileB * btile, &p->bytes)) !=
          cudaSuccess ||
      (e = dalloc(reinterpret_cast<void**>(&p->metaA), (size_t)std::max(blkA, 1) * kMetaStride * 4,
                  &p->bytes)) != cudaSuccess ||
      (e = dalloc(reinterpret_cast<void**>(&p->metaB), (size_t)std::max(blkB, 1) * kMetaStride * 4,
                  &p->bytes)) != cudaSuccess)
    return cuda_err(err, e, "split plan allocation");
  // meta of blocks without slice jobs (k == 0) must read as zero lines; tile
  // rows of lines beyond an instance are never written by the slicer and
  // start out as zero digits
  if ((e = cudaMemset(p->metaA, 0, (size_t)std::max(blkA, 1) * kMetaStride * 4)) != cudaSuccess ||
      (e = cudaMemset(p->metaB, 0, (size_t)std::max(blkB, 1) * kMetaStride * 4)) != cudaSuccess ||
      (e = cudaMemset(p->tilesA, 0, (size_t)tileA * kATileBytes)) != cudaSuccess ||
      (e = cudaMemset(p->tilesB, 0, (size_t)tileB * btile)) != cudaSuccess)
    return cuda_err(err, e, "split plan workspace clear");
  return BG_OK;
}

static void finish_desc(SplitPlan* p) {
  char buf[1024];
  snprintf(buf, sizeof buf,
           "{\"slices\": %d, \"beta_bits\": %d, \"pairs\": %d, \"tile\": [%d, %d, %d], "
           "\"kpass_kblocks\": %d, \"a_ring_groups\": %d, \"smem_bytes\": %zu, \"units\": %lld, "
           "\"slice_jobs\": %lld, \"small_instances\": %lld, \"small_items\": %lld, "
           "\"small_mnk\": %.17g, \"small_ab_elems\": %.17g, \"workspace_bytes\": %lld}",
           p->s, p->beta, p->s * (p->s + 1) / 2, BM, p->bn, BK, p->kpass, p->a_groups, p->smem,
           (long long)p->n_units, (long long)p->n_jobs, (long long)p->n_small,
           (long long)p->n_small_items, p->small_mnk, p->small_ab, (long long)p->bytes);
  p->desc = buf;
}

static cudaError_t set_gemm_attr(bg_dtype dt, int s) {
  static bool done[2][kMaxSlices + 1] = {};
  if (s < 1 || s > kMaxSlices) return cudaErrorInvalidValue;
  const int c = dt == BG_C128 ? 1 : 0;
  if (done[c][s]) return cudaSuccess;
  cudaError_t e = c ? set_split_gemm_attr_c128(s) : set_split_gemm_attr_r64(s);
  if (e == cudaSuccess) done[c][s] = true;
  return e;
}

static void grids(SplitPlan* p) {
  set_gemm_attr(p->dt, p->s);
  p->grid_gemm = (int)std::max<int64_t>(1, std::min<int64_t>(p->sms, p->n_units));
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, split_slice_kernel<9, 6>, kSliceThreads, 0);
  if (bps < 1) bps = 1;
  p->grid_slice = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)p->sms * bps, p->n_jobs));
  if (p->n_small_items > 0)
    p->grid_small = (int)std::max<int64_t>(1, std::min<int64_t>(p->sms, p->n_small_items));
}

bg_status split_plan_create(SplitPlan** out, bg_dtype dt, const bg_precision& pr,
                            const std::vector<bg_instance>& table, const int64_t* d_table,
                            int sms, bool autotune, cudaStream_t st, std::string* err,
                            bool herk, bool small_kernel, const std::vector<int8_t>* route) {
  (void)d_table;
  (void)autotune;
  (void)st;
  SplitPlan* p = new SplitPlan();
  if (!setup_common(p, dt, pr, sms, err)) {
    delete p;
    return BG_ERR_INVALID_ARG;
  }
  p->herk = herk;
  p->small_ok = small_kernel && split_small_supported(p->s, p->beta);
  if (route) p->route = *route;
  bg_status s = build_instances(p, table, err);
  if (s != BG_OK) {
    split_plan_destroy(p);
    return s;
  }
  grids(p);
  finish_desc(p);
  *out = p;
  return BG_OK;
}

static cudaError_t launch_slicer(SplitPlan* p, const SliceJob* jobs, int64_t njobs,
                                 const SInst* instA, const SInst* instB, const int32_t* orderA,
                                 const int32_t* orderB, const void* A, const void* B,
                                 cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  SliceArgs a;
  a.jobs = jobs;
  a.njobs = njobs;
  a.instA = instA;
  a.instB = instB;
  a.orderA = orderA;
  a.orderB = orderB;
  a.A = static_cast<const double*>(A);
  a.B = static_cast<const double*>(B);
  a.tilesA = p->tilesA;
  a.tilesB = p->tilesB;
  a.metaA = p->metaA;
  a.metaB = p->metaB;
  a.cplx = p->dt == BG_C128;
  a.s = p->s;
  a.beta = p->beta;
  a.bn = p->bn;
  a.herk = p->herk ? 1 : 0;
  const int grid = (int)std::min<int64_t>(p->grid_slice, njobs);
  // compile-time (slices, digit width) versions for the documented modes
  if (p->s == 3 && p->beta == 7) {
    split_slice_kernel<3, 7><<<grid, kSliceThreads, 0, st>>>(a);
  } else if (p->s == 6 && p->beta == 7) {
    split_slice_kernel<6, 7><<<grid, kSliceThreads, 0, st>>>(a);
  } else if (p->s == 9 && p->beta == 6) {
    split_slice_kernel<9, 6><<<grid, kSliceThreads, 0, st>>>(a);
  } else {
    BG_DISPATCH_SLICES(p->s, {
      split_slice_kernel<S, 0><<<grid, kSliceThreads, 0, st>>>(a);
      count_launch();
      return cudaGetLastError();
    });
  }
  count_launch();
  return cudaGetLastError();
}

// The small-instance kernel reads A and B itself (no slicer pass).
static cudaError_t launch_small(SplitPlan* p, const void* A, const void* B, void* C,
                                const Scalars& sc, cudaStream_t st) {
  if (p->n_small <= 0) return cudaSuccess;
  SmallArgs g;
  g.inst = p->d_inst;
  g.ids = p->d_small;
  g.items = p->d_small_items;
  g.nitems = p->n_small_items;
  g.A = static_cast<const double*>(A);
  g.B = static_cast<const double*>(B);
  g.C = static_cast<double*>(C);
  g.sc = sc;
  g.skip_product = sc.alpha_zero;
  const cudaError_t e = launch_split_small(p->s, p->grid_small, st, g);
  count_launch();
  return e;
}

static cudaError_t launch_gemm(SplitPlan* p, void* C, const Scalars& sc, const int32_t* idx,
                               int* d_err, cudaStream_t st) {
  if (p->n_units <= 0) return cudaSuccess;
  GemmArgs g;
  g.units = p->d_units;
  g.nunits = p->n_units;
  g.inst = p->d_inst;
  g.order = p->d_order;
  g.tilesA = p->tilesA;
  g.tilesB = p->tilesB;
  g.metaA = p->metaA;
  g.metaB = p->metaB;
  g.C = static_cast<double*>(C);
  g.idx = idx;
  g.pool_tile0 = p->d_pool_tile0;
  g.pool_blk0 = p->d_pool_blk0;
  g.pool = p->d_pool;
  g.pool_count = p->n_pool;
  g.sc = sc;
  g.cplx = p->dt == BG_C128;
  g.s = p->s;
  g.beta = p->beta;
  g.skip_product = sc.alpha_zero;
  g.herk = p->herk ? 1 : 0;
  g.kpass = p->kpass;
  g.a_groups = p->a_groups;
  g.err = d_err;
  cudaError_t e = g.cplx ? launch_split_gemm_c128(p->s, p->grid_gemm, p->smem, st, g)
                         : launch_split_gemm_r64(p->s, p->grid_gemm, p->smem, st, g);
  count_launch();
  return e;
}

bg_status split_plan_run(SplitPlan* p, const void* A, const void* B, void* C, const Scalars& s,
                         int* d_err, cudaStream_t st, std::string* err, cudaEvent_t* ev) {
  cudaError_t e;
  if (!s.alpha_zero) {
    e = launch_slicer(p, p->d_jobs, p->n_jobs, p->d_inst, p->d_inst, p->d_order, p->d_order, A, B,
                      st);
    if (e != cudaSuccess) return cuda_err(err, e, "split slicer launch");
  }
  if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return cuda_err(err, e, "event");
  e = launch_small(p, A, B, C, s, st);
  if (e != cudaSuccess) return cuda_err(err, e, "split small-instance launch");
  if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return cuda_err(err, e, "event");
  e = launch_gemm(p, C, s, nullptr, d_err, st);
  if (e != cudaSuccess) return cuda_err(err, e, "split GEMM launch");
  if (ev && (e = cudaEventRecord(ev[2], st)) != cudaSuccess) return cuda_err(err, e, "event");
  return BG_OK;
}

bg_status split_fixed(bg_dtype dt, const bg_precision& pr, int64_t m, int64_t n, int64_t k,
                      const Scalars& s, const void* A, int64_t lda, int64_t sA, const void* B,
                      int64_t ldb, int64_t sB, void* C, int64_t ldc, int64_t sC, int64_t batch,
                      SplitWorkspace* ws, int sms, int* d_err, bool capturing, cudaStream_t st,
                      std::string* err) {
  const int beta = pr.beta_bits ? pr.beta_bits : split_default_beta(pr.slices);
  std::vector<int64_t> key = {(int64_t)dt, m, n, k, lda, ldb, ldc, sA, sB, sC, batch,
                              pr.slices, beta};
  SplitPlan* p = nullptr;
  for (size_t i = 0; i < ws->cache.size(); ++i)
    if (ws->cache[i]->key == key) {
      p = ws->cache[i];
      ws->cache.erase(ws->cache.begin() + i);
      ws->cache.push_back(p);
      break;
    }
  if (!p) {
    if (capturing)
      return set_err(err, BG_ERR_CAPTURE,
                     "first split-mode call of this shape allocates its workspace; the stream "
                     "is being captured");
    std::vector<bg_instance> table((size_t)batch);
    for (int64_t i = 0; i < batch; ++i)
      table[i] = bg_instance{m, n, k, lda, ldb, ldc, i * sA, i * sB, i * sC};
    bg_status rs = split_plan_create(&p, dt, pr, table, nullptr, sms, false, st, err);
    if (rs != BG_OK) return rs;
    p->key = key;
    ws->cache.push_back(p);
    while (ws->cache.size() > 4) {
      // the oldest plan may still be in use by queued work: wait before freeing
      cudaDeviceSynchronize();
      split_plan_destroy(ws->cache.front());
      ws->cache.erase(ws->cache.begin());
    }
  }
  return split_plan_run(p, A, B, C, s, d_err, st, err);
}

// ---- fixed-size split batch in caller-provided device scratch ---------------------------------

// Lays the whole split plan (error word, meta stores, tables, digit tiles) out
// in `scratch` (device memory of the current device, `scratch_bytes` long,
// 256-byte aligned) and runs it. Allocates no device memory; fails with
// BG_ERR_INVALID_ARG when the plan does not fit.
bg_status split_fixed_in_scratch(bg_dtype dt, const bg_precision& pr, int64_t m, int64_t n,
                                 int64_t k, const Scalars& sc, const void* A, int64_t lda,
                                 int64_t sA, const void* B, int64_t ldb, int64_t sB, void* C,
                                 int64_t ldc, int64_t sC, int64_t batch, void* scratch,
                                 size_t scratch_bytes, int sms, cudaStream_t st,
                                 std::string* err) {
  SplitPlan p;  // host object only: every device pointer below points into `scratch`
  if (!setup_common(&p, dt, pr, sms, err)) return BG_ERR_INVALID_ARG;
  p.small_ok = split_small_supported(p.s, p.beta);
  std::vector<bg_instance> table((size_t)batch);
  for (int64_t i = 0; i < batch; ++i)
    table[i] = bg_instance{m, n, k, lda, ldb, ldc, i * sA, i * sB, i * sC};
  HostTables t;
  make_tables(&p, table, &t);
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t meta_a = (size_t)std::max(t.blkA, 1) * kMetaStride * 4;
  const size_t meta_b = (size_t)std::max(t.blkB, 1) * kMetaStride * 4;
  size_t off = 0;
  const size_t o_err = off;    off += up(4 * sizeof(int));
  const size_t o_ma = off;     off += up(meta_a);
  const size_t o_mb = off;     off += up(meta_b);
  const size_t o_jobs = off;   off += up(t.jobs.size() * sizeof(SliceJob) + 1);
  const size_t o_units = off;  off += up(t.units.size() * sizeof(SplitUnit) + 1);
  const size_t o_inst = off;   off += up(t.inst.size() * sizeof(SInst) + 1);
  const size_t o_order = off;  off += up(t.order.size() * sizeof(int32_t) + 1);
  const size_t o_small = off;  off += up(t.small.size() * sizeof(int32_t) + 1);
  const size_t o_items = off;  off += up(t.small_items.size() * sizeof(SmallItem) + 1);
  const size_t o_ta = off;     off += up((size_t)t.tileA * kATileBytes);
  const size_t o_tb = off;     off += up((size_t)t.tileB * p.bn * kLineBytes);
  if (off > scratch_bytes) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "problem needs %zu bytes of split workspace; the static scratch holds %zu",
             off, scratch_bytes);
    return set_err(err, BG_ERR_INVALID_ARG, buf);
  }
  uint8_t* base = static_cast<uint8_t*>(scratch);
  int* d_err = reinterpret_cast<int*>(base + o_err);
  p.metaA = reinterpret_cast<int32_t*>(base + o_ma);
  p.metaB = reinterpret_cast<int32_t*>(base + o_mb);
  p.d_jobs = reinterpret_cast<SliceJob*>(base + o_jobs);
  p.d_units = reinterpret_cast<SplitUnit*>(base + o_units);
  p.d_inst = reinterpret_cast<SInst*>(base + o_inst);
  p.d_order = reinterpret_cast<int32_t*>(base + o_order);
  p.d_small = reinterpret_cast<int32_t*>(base + o_small);
  p.d_small_items = reinterpret_cast<SmallItem*>(base + o_items);
  p.tilesA = base + o_ta;
  p.tilesB = base + o_tb;
  p.n_jobs = (int64_t)t.jobs.size();
  p.n_jobs_A = t.n_jobs_A;
  p.n_units = (int64_t)t.units.size();
  p.n_small = (int64_t)t.small.size();
  p.n_small_items = (int64_t)t.small_items.size();
  p.count = batch;
  cudaError_t e;
  // the scratch keeps the previous call's contents: clear the error word, the
  // meta stores and the digit tiles (rows beyond an instance are not written)
  if ((e = cudaMemsetAsync(base, 0, o_jobs, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(base + o_ta, 0, off - o_ta, st)) != cudaSuccess)
    return cuda_err(err, e, "static scratch clear");
  struct Piece { size_t off; const void* src; size_t bytes; };
  const Piece pieces[] = {{o_jobs, t.jobs.data(), t.jobs.size() * sizeof(SliceJob)},
                          {o_units, t.units.data(), t.units.size() * sizeof(SplitUnit)},
                          {o_inst, t.inst.data(), t.inst.size() * sizeof(SInst)},
                          {o_order, t.order.data(), t.order.size() * sizeof(int32_t)},
                          {o_small, t.small.data(), t.small.size() * sizeof(int32_t)},
                          {o_items, t.small_items.data(), t.small_items.size() * sizeof(SmallItem)}};
  for (const Piece& pc : pieces)
    if (pc.bytes && (e = cudaMemcpyAsync(base + pc.off, pc.src, pc.bytes, cudaMemcpyHostToDevice,
                                         st)) != cudaSuccess)
      return cuda_err(err, e, "static scratch table upload");
  grids(&p);
  return split_plan_run(&p, A, B, C, sc, d_err, st, err);
}

// ---- chain plans -----------------------------------------------------------------------------

bg_status split_chain_create(SplitPlan** out, bg_dtype dt, const bg_precision& pr,
                             const std::vector<int64_t>& wn, const std::vector<int64_t>& woff,
                             const std::vector<int64_t>& pool_n,
                             const std::vector<int64_t>& pool_off, int sms, cudaStream_t st,
                             std::string* err) {
  (void)st;
  SplitPlan* p = new SplitPlan();
  if (!setup_common(p, dt, pr, sms, err)) {
    delete p;
    return BG_ERR_INVALID_ARG;
  }
  p->chain = true;
  const bool cplx = dt == BG_C128;
  const int s = p->s, BN = p->bn;
  // pool entries: A blocks (row blocks), sliced once per chain_step call
  std::vector<SInst> pool(pool_n.size());
  std::vector<int32_t> pool_order(pool_n.size());
  std::vector<int64_t> pool_tile0(pool_n.size());
  std::vector<int32_t> pool_blk0(pool_n.size());
  std::vector<SliceJob> jobsA;
  int64_t tileA = 0;
  int32_t blkA = 0;
  for (size_t j = 0; j < pool_n.size(); ++j) {
    const int64_t n = pool_n[j];
    pool[j] = SInst{pool_off[j], 0, 0, std::max<int64_t>(1, n), 1, 1, (int32_t)n, (int32_t)n,
                    (int32_t)n, 0};
    pool_order[j] = (int32_t)j;
    const int64_t mv = cplx ? 2 * n : n, kvv = mv;
    const int nkb = (int)((kvv + BK - 1) / BK);
    pool_tile0[j] = tileA;
    pool_blk0[j] = blkA;
    for (int64_t rb = 0; rb < (mv + BM - 1) / BM; ++rb) {
      if (nkb > 0)
        jobsA.push_back(SliceJob{tileA, blkA, (int32_t)j, 0, 1, (int16_t)BM, (int16_t)nkb,
                                 (int32_t)(rb * BM), (int32_t)kvv});
      tileA += (int64_t)s * nkb;
      ++blkA;
    }
  }
  // walkers: B blocks (column blocks of the state), sliced every step
  std::vector<SInst> inst(wn.size());
  std::vector<int32_t> order(wn.size());
  std::vector<SliceJob> jobsB;
  std::vector<SplitUnit> units;
  int64_t tileB = 0;
  int32_t blkB = 0;
  for (size_t w = 0; w < wn.size(); ++w) {
    const int64_t n = wn[w];
    inst[w] = SInst{0, woff[w], woff[w], std::max<int64_t>(1, n), std::max<int64_t>(1, n),
                    std::max<int64_t>(1, n), (int32_t)n, (int32_t)n, (int32_t)n, 0};
    order[w] = (int32_t)w;
    if (n == 0) continue;
    const int64_t mv = cplx ? 2 * n : n, kvv = mv;
    const int nkb = (int)((kvv + BK - 1) / BK);
    const int64_t rbs = (mv + BM - 1) / BM, cbs = (n + BN - 1) / BN;
    const int64_t tB0 = tileB;
    const int32_t bB0 = blkB;
    for (int64_t cb = 0; cb < cbs; ++cb) {
      jobsB.push_back(SliceJob{tileB, blkB, (int32_t)w, 1, 1, (int16_t)BN, (int16_t)nkb,
                               (int32_t)(cb * BN), (int32_t)kvv});
      tileB += (int64_t)s * nkb;
      ++blkB;
    }
    for (int64_t cb = 0; cb < cbs; ++cb)
      for (int64_t rb = 0; rb < rbs; ++rb) {
        SplitUnit U{};
        U.a_tile0 = rb * s * nkb;  // relative to the pool entry's first tile
        U.b_tile0 = tB0 + cb * s * nkb;
        U.a_blk = (int32_t)rb;     // relative to the pool entry's first block
        U.b_blk = bB0 + (int32_t)cb;
        U.pos = (int32_t)w;
        U.g = 1;
        U.nkb = (int16_t)nkb;
        U.kmma_last = (int16_t)kmma_last_of((int)kvv);
        U.mrow = (int16_t)std::min<int64_t>(mv, 32767);
        U.ncol = (int16_t)std::min<int64_t>(n, 32767);
        U.r0 = (int32_t)(rb * BM);
        U.c0 = (int32_t)(cb * BN);
        units.push_back(U);
      }
  }
  std::stable_sort(units.begin(), units.end(),
                   [](const SplitUnit& a, const SplitUnit& b) { return a.nkb > b.nkb; });
  // pool jobs first, then walker jobs (the chain step slices the two parts separately)
  split_jobs(&jobsA, BN);
  split_jobs(&jobsB, BN);
  std::vector<SliceJob> jobs = jobsA;
  jobs.insert(jobs.end(), jobsB.begin(), jobsB.end());
  p->n_jobs = (int64_t)jobs.size();
  p->n_jobs_A = (int64_t)jobsA.size();
  p->n_units = (int64_t)units.size();
  p->count = (int64_t)wn.size();
  p->n_pool = (int32_t)pool_n.size();
  const size_t btile = (size_t)BN * kLineBytes;
  cudaError_t e;
  if ((e = dput(&p->d_jobs, jobs, &p->bytes)) != cudaSuccess ||
      (e = dput(&p->d_units, units, &p->bytes)) != cudaSuccess ||
      (e = dput(&p->d_inst, inst, &p->bytes)) != cudaSuccess ||
      (e = dput(&p->d_pool, pool, &p->bytes)) != cudaSuccess ||
      (e = dput(&p->d_order, order, &p->bytes)) != cudaSuccess ||
      (e = dput(&p->d_pool_order, pool_order, &p->bytes)) != cudaSuccess ||
      (e = dput(&p->d_pool_tile0, pool_tile0, &p->bytes)) != cudaSuccess ||
      (e = dput(&p->d_pool_blk0, pool_blk0, &p->bytes)) != cudaSuccess ||
      (e = dalloc(reinterpret_cast<void**>(&p->tilesA), (size_t)tileA * kATileBytes, &p->bytes)) !=
          cudaSuccess ||
      (e = dalloc(reinterpret_cast<void**>(&p->tilesB), (size_t)tileB * btile, &p->bytes)) !=
          cudaSuccess ||
      (e = dalloc(reinterpret_cast<void**>(&p->metaA), (size_t)std::max(blkA, 1) * kMetaStride * 4,
                  &p->bytes)) != cudaSuccess ||
      (e = dalloc(reinterpret_cast<void**>(&p->metaB), (size_t)std::max(blkB, 1) * kMetaStride * 4,
                  &p->bytes)) != cudaSuccess) {
    bg_status rs = cuda_err(err, e, "split chain plan allocation");
    split_plan_destroy(p);
    return rs;
  }
  cudaMemset(p->metaA, 0, (size_t)std::max(blkA, 1) * kMetaStride * 4);
  cudaMemset(p->metaB, 0, (size_t)std::max(blkB, 1) * kMetaStride * 4);
  cudaMemset(p->tilesA, 0, (size_t)tileA * kATileBytes);
  cudaMemset(p->tilesB, 0, (size_t)tileB * btile);
  grids(p);
  finish_desc(p);
  *out = p;
  return BG_OK;
}

bg_status split_chain_prepare_pool(SplitPlan* p, const void* U, int* d_err, cudaStream_t st,
                                   std::string* err) {
  (void)d_err;
  cudaError_t e = launch_slicer(p, p->d_jobs, p->n_jobs_A, p->d_pool, p->d_inst, p->d_pool_order,
                                p->d_order, U, nullptr, st);
  if (e != cudaSuccess) return cuda_err(err, e, "split pool slicer launch");
  return BG_OK;
}

bg_status split_chain_step(SplitPlan* p, const void* U, const int32_t* idx_row, const void* Cin,
                           void* Cout, int* d_err, cudaStream_t st, std::string* err) {
  (void)U;
  cudaError_t e = launch_slicer(p, p->d_jobs + p->n_jobs_A, p->n_jobs - p->n_jobs_A, p->d_pool,
                                p->d_inst, p->d_pool_order, p->d_order, nullptr, Cin, st);
  if (e != cudaSuccess) return cuda_err(err, e, "split state slicer launch");
  Scalars sc;
  sc.alpha_re = 1.0;
  sc.alpha_im = 0.0;
  sc.beta_re = 0.0;
  sc.beta_im = 0.0;
  sc.alpha_zero = 0;
  sc.beta_zero = 1;
  e = launch_gemm(p, Cout, sc, idx_row, d_err, st);
  if (e != cudaSuccess) return cuda_err(err, e, "split chain GEMM launch");
  return BG_OK;
}

}  // namespace bg
