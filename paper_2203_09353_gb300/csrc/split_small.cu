// Split-precision GEMM for small real instances (m, n, k <= 64): the same
// method as split.cu (row / column exponents, balanced base-2^beta digits,
// exact FP32 level sums, 64-bit fixed-point recombination, one rounding to
// FP64), fused into one kernel, without digit planes in HBM.
//
// The tensor-core kernel of split_gemm.cuh works on 128 x BN output tiles
// that are k-blocks of 64 deep; a 16 x 16 instance fills a sliver of such a
// tile and still pays for a full chain of copies, MMAs and a level drain.
// Here an instance is handled by a group of warps sized to its padded edge
// T (16, 32 or 64): (T / 16)^2 warps, each owning one 16 x 16 output block,
// so that a CTA of 16 warps runs 16, 4 or 1 instances side by side. A group:
//  1. loads its operands into registers (each thread: four pairs of
//     neighbouring k values, of one row of A and of four columns of B),
//     takes the line exponents of A's rows and B's columns, and asks L2 for
//     the operands of the CTA's next work item;
//  2. cuts every value into its digits straight into shared memory: S planes
//     of A (T rows x T k, BF16) and of B^T (T columns x T k), rows padded by
//     8 values so that ldmatrix reads are free of bank conflicts, and sums
//     the per-line digit-norm bounds that set the fixed-point frame;
//  3. forms the level sums L_t = sum_{p+q=t} D_p^A D_q^B with mma.sync
//     m16n8k16 (BF16 in, FP32 accumulate, exact: every partial sum is an
//     integer below 2^24), three levels at a time, each folded into 64-bit
//     integers;
//  4. converts exactly to FP64, applies alpha and beta of Eq. (1), stores.
// mma.sync runs at a quarter of the tcgen05 rate on this part, which is
// ample for instances this small. Work items (built by the planner) hold the
// instances that one CTA's groups take together; all of an item's instances
// have the same T.
#include <cuda_runtime.h>

#include <climits>

#include "split_common.cuh"

namespace bg {
namespace splitk {
namespace {

constexpr int kSmallThreads = 512;  // 16 warps

template <int S, int T>
struct SmallShape {
  static constexpr int NW = (T / 16) * (T / 16);  // warps per instance
  static constexpr int GT = NW * 32;              // threads per instance
  static constexpr int PAD = T + 8;               // BF16 per shared-memory row
  static constexpr int ROWB = PAD * 2;
  static constexpr int PLANE = T * ROWB;
  // per group: S planes of A, S planes of B^T, then the line data (exponents
  // of A's rows and B's columns, their digit-norm sums)
  static constexpr int META = (4 * T + 4) * 4;
  static constexpr int GROUP_BYTES = 2 * S * PLANE + META;
  static constexpr int NG_FIT = (int)(kSmallSmemMax / GROUP_BYTES);
  static constexpr int NG = 16 / NW < NG_FIT ? 16 / NW : NG_FIT;  // groups per CTA
  static_assert(PLANE % 16 == 0 && META % 16 == 0, "16-byte aligned planes");
  static_assert(NG >= 1, "one instance group must fit");
};

__device__ __forceinline__ void ldm_x4(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Barrier over the threads of one instance group (named barrier 1 + gid).
template <int NW>
__device__ __forceinline__ void group_sync(int gid) {
  if constexpr (NW == 1) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + gid), "r"(NW * 32) : "memory");
  }
}

// Exponent e with |x| < 2^e; INT_MIN for x == 0 (the identity of the max).
__device__ __forceinline__ int value_exponent(double x) {
  const unsigned long long b =
      (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
  return b ? line_exponent(b) : INT_MIN;
}

// Line exponent from the max of value exponents (0 for an all-zero line).
__device__ __forceinline__ int line_e(int v) { return v == INT_MIN ? 0 : v; }

// Digits of two values of one line (neighbouring k, the same line exponent e)
// into the planes at `dst` (plane p at dst + p PLANE), one 32-bit word per
// plane: BF16 of the first value low, of the second high. Returns the bounds
// |d_1| + 0.51 of their absolute digit weights.
template <int S, int BETA, int PLANE>
__device__ __forceinline__ float2 cut_pair(double x0, double x1, int e, long long bias,
                                           uint8_t* dst) {
  uint32_t lo0, hi0, lo1, hi1;
  biased_fixed<S, BETA>(x0, e, bias, lo0, hi0);
  biased_fixed<S, BETA>(x1, e, bias, lo1, hi1);
  const float t0 = top_digit<S, BETA>(lo0, hi0), t1 = top_digit<S, BETA>(lo1, hi1);
  *reinterpret_cast<uint32_t*>(dst) = __byte_perm(__float_as_uint(t0), __float_as_uint(t1), 0x7632);
#pragma unroll
  for (int p = 1; p < S; ++p)
    *reinterpret_cast<uint32_t*>(dst + p * PLANE) = lower_digit_pair<S, BETA>(p, lo0, hi0, lo1, hi1);
  return make_float2(fabsf(t0) + 0.51f, fabsf(t1) + 0.51f);
}

// al^2 in units of 2^-8, rounded up (integer sums do not depend on their order)
__device__ __forceinline__ uint32_t norm_units(float al) {
  return __float2uint_ru(al * al * 256.0f * 1.0001f);
}

// L2 prefetch of the operands of the next work item's instances (those this
// group would take: gid, gid + NG, ...), issued while the current instance's
// loads are in flight; the instance records on the way are then in L2 too.
template <int GT>
__device__ __forceinline__ void prefetch_next(const SmallArgs& g, int64_t next, int gid, int ng,
                                              int tg) {
  if (next < 0 || g.skip_product) return;  // alpha == 0: A and B are not touched
  const SmallItem nx = g.items[next];
  for (int q = gid; q < nx.count; q += ng) {
    const SInst ni = g.inst[g.ids[nx.first + q]];
    const int ca = (ni.m + 15) >> 4, cb = (ni.k + 15) >> 4;  // 128-byte pieces per column
    const int na = ni.k * ca, nb = ni.n * cb;
    for (int x = tg; x < na + nb; x += GT) {
      const double* p;
      if (x < na) {
        p = g.A + ni.a_off + (int64_t)(x / ca) * ni.lda + min(16 * (x % ca), ni.m - 1);
      } else {
        const int y = x - na;
        p = g.B + ni.b_off + (int64_t)(y / cb) * ni.ldb + min(16 * (y % cb), ni.k - 1);
      }
      asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
    }
  }
}

// alpha and beta of Eq. (1) and the store of a thread's outputs. A1: alpha ==
// 1, BZ: beta == 0, both compile-time so that no FP64 instruction runs that
// the case does not need (a runtime test compiles to the multiply and a
// select; on this part a warp-wide FP64 instruction holds the FP64 pipe for
// about 64 clocks).
template <bool A1, bool BZ>
__device__ __forceinline__ void small_store(const SmallArgs& g, const double (&xs)[2][2][2],
                                            const double (&cold)[2][2][2], double* Cb, int64_t ldc,
                                            const int (&rows)[2], int m, int n, int c0, int tq) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = rows[h];
    if (i >= m) continue;
#pragma unroll
    for (int nh = 0; nh < 2; ++nh)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int j = c0 + 8 * nh + 2 * tq + c;
        if (j >= n) continue;
        double v = xs[h][nh][c];
        if constexpr (!A1) v = g.sc.alpha_re * v;
        if constexpr (!BZ) v = fma(g.sc.beta_re, cold[h][nh][c], v);
        Cb[i + (int64_t)j * ldc] = v;
      }
  }
}

// One instance on one group of (T / 16)^2 warps; tg = thread within the group.
template <int S, int BETA, int T>
__device__ __forceinline__ void small_instance(const SmallArgs& g, const SInst& in, uint8_t* gsm,
                                               int gid, int tg, const DigitCtx& dc, int64_t next) {
  using SH = SmallShape<S, T>;
  constexpr int NW = SH::NW, GT = SH::GT, ROWB = SH::ROWB, PLANE = SH::PLANE;
  // A warp covers RW lines x KW k of A (rows) and of B^T (columns), each
  // thread four pairs of neighbouring k: a warp's 32-bit digit stores then
  // hit 32 distinct banks on both sides
  constexpr int KW = T < 32 ? T : 32;  // k per warp
  constexpr int RW = 256 / KW;         // lines per warp
  constexpr int NRB = T / RW;          // line blocks per instance
  constexpr int POFF = 32 / RW;        // A: lanes sharing a row, stride of a thread's pairs
  constexpr int PL = KW / 2;           // B: lanes sharing a column
  constexpr int CPW = 32 / PL;         // B: columns per lane set
  uint8_t* planesA = gsm;
  uint8_t* planesB = gsm + S * PLANE;
  int* eA = reinterpret_cast<int*>(gsm + 2 * S * PLANE);
  int* eB = eA + T;
  uint32_t* n2A = reinterpret_cast<uint32_t*>(eB + T);
  uint32_t* n2B = n2A + T;
  const int lane = tg & 31, wg = tg >> 5;
  const int m = in.m, n = in.n, k = in.k;
  const bool prod = !g.skip_product;
  for (int x = tg; x < T; x += GT) {
    eA[x] = INT_MIN;
    eB[x] = INT_MIN;
    n2A[x] = 0;
    n2B[x] = 0;
  }
  // ---- 1. operands into registers. A: row ia, k = ka0 + 2 POFF r (+1);
  // B: column jb0 + CPW r, k = kb (+1). Neighbouring lanes read neighbouring
  // addresses (A is column-major: rows; B: k).
  const int blk = wg % NRB, kblk = wg / NRB;
  const int ia = RW * blk + lane % RW, ka0 = KW * kblk + 2 * (lane / RW);
  const int jb0 = RW * blk + lane / PL, kb = KW * kblk + 2 * (lane % PL);
  double va[8], vb[8];
  {
    const double* A = g.A + in.a_off;
    const double* B = g.B + in.b_off;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int kk = ka0 + 2 * POFF * r, j = jb0 + CPW * r;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        va[2 * r + h] =
            (prod && ia < m && kk + h < k) ? __ldg(A + ia + (int64_t)(kk + h) * in.lda) : 0.0;
        vb[2 * r + h] =
            (prod && kb + h < k && j < n) ? __ldg(B + kb + h + (int64_t)j * in.ldb) : 0.0;
      }
    }
  }
  prefetch_next<GT>(g, next, gid, SH::NG, tg);
  group_sync<NW>(gid);  // line data initialised
  {
    int ea = INT_MIN;
#pragma unroll
    for (int r = 0; r < 8; ++r) ea = max(ea, value_exponent(va[r]));
#pragma unroll
    for (int o = RW; o < 32; o <<= 1) ea = max(ea, __shfl_xor_sync(0xFFFFFFFFu, ea, o));
    if (lane < RW && ea != INT_MIN) atomicMax(&eA[ia], ea);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int eb = max(value_exponent(vb[2 * r]), value_exponent(vb[2 * r + 1]));
#pragma unroll
      for (int o = PL / 2; o > 0; o >>= 1) eb = max(eb, __shfl_xor_sync(0xFFFFFFFFu, eb, o));
      if (lane % PL == 0 && eb != INT_MIN) atomicMax(&eB[jb0 + CPW * r], eb);
    }
  }
  group_sync<NW>(gid);
  // ---- 2. digits into shared memory (zero digits outside the instance, where
  // the MMAs read padding); digit-norm sums of the instance's values
  {
    const int e_a = line_e(eA[ia]);
    uint32_t sa = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int kk = ka0 + 2 * POFF * r;
      const float2 al = cut_pair<S, BETA, PLANE>(va[2 * r], va[2 * r + 1], e_a, dc.bias64,
                                                 planesA + ia * ROWB + kk * 2);
      if (ia < m && kk < k) sa += norm_units(al.x);
      if (ia < m && kk + 1 < k) sa += norm_units(al.y);
    }
#pragma unroll
    for (int o = RW; o < 32; o <<= 1) sa += __shfl_xor_sync(0xFFFFFFFFu, sa, o);
    if (lane < RW && ia < m && sa) atomicAdd(&n2A[ia], sa);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int j = jb0 + CPW * r;
      const float2 al = cut_pair<S, BETA, PLANE>(vb[2 * r], vb[2 * r + 1], line_e(eB[j]),
                                                 dc.bias64, planesB + j * ROWB + kb * 2);
      uint32_t sb = 0;
      if (j < n && kb < k) sb += norm_units(al.x);
      if (j < n && kb + 1 < k) sb += norm_units(al.y);
#pragma unroll
      for (int o = PL / 2; o > 0; o >>= 1) sb += __shfl_xor_sync(0xFFFFFFFFu, sb, o);
      if (lane % PL == 0 && sb) atomicAdd(&n2B[j], sb);
    }
  }
  group_sync<NW>(gid);
  // ---- 3. level sums on the tensor cores, folded into 64-bit fixed point.
  // Warp wg takes row block wg / (T/16) and a column block chosen so that the
  // warps of an instance fall on distinct SM sub-partitions (warp w runs on
  // sub-partition w mod 4).
  constexpr int BS = T / 16;
  const int rb = wg / BS;
  const int cb = BS == 4 ? ((wg - 2 * rb) & 3) : (wg % BS);
  const int r0 = 16 * rb, c0 = 16 * cb;
  if (r0 >= m || c0 >= n) return;
  const int gi = lane >> 2, tq = lane & 3;
  const int rows[2] = {r0 + gi, r0 + gi + 8};
  // the frame: a row's norm exponent plus the largest one of the columns
  int RB = -126;
  for (int j = lane; j < n; j += 32) RB = max(RB, norm_exponent((float)n2B[j] * (1.0f / 256.0f)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) RB = max(RB, __shfl_xor_sync(0xFFFFFFFFu, RB, o));
  int F[2];
#pragma unroll
  for (int h = 0; h < 2; ++h)
    F[h] = norm_exponent((float)n2A[min(rows[h], T - 1)] * (1.0f / 256.0f)) + RB + 1;
  // C at this thread's outputs, read ahead of the MMAs
  double cold[2][2][2];
  double* Cb = g.C + in.c_off;
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int nh = 0; nh < 2; ++nh)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int i = rows[h], j = c0 + 8 * nh + 2 * tq + c;
        cold[h][nh][c] = (!g.sc.beta_zero && i < m && j < n) ? Cb[i + (int64_t)j * in.ldc] : 0.0;
      }
  long long accI[2][2][2] = {};  // [row half][n half][column pair]
  if (prod) {
    const int kp = (k + 15) & ~15;  // k padded to the MMA's 16
    const uint32_t aBase = smem_u32(planesA) +
                           (uint32_t)((r0 + (lane & 7) + 8 * ((lane >> 3) & 1)) * ROWB +
                                      16 * (lane >> 4));
    const uint32_t bBase = smem_u32(planesB) +
                           (uint32_t)((c0 + (lane & 7) + 8 * (lane >> 4)) * ROWB +
                                      16 * ((lane >> 3) & 1));
    // levels in groups of three (g3 .. g3 + 2); per k-step the A digits of
    // every plane the group needs stay in registers and each B plane is read
    // once, so that shared-memory reads grow with the planes, not the pairs
#pragma unroll
    for (int g3 = 0; g3 < S; g3 += 3) {
      constexpr int kMaxP = S;
      const int np = g3 + 3 < S ? g3 + 3 : S;  // planes 0 .. np - 1 take part
      float acc[3][2][4] = {};
#pragma unroll 1
      for (int ks = 0; ks < kp; ks += 16) {
        uint32_t a[kMaxP][4];
#pragma unroll
        for (int p = 0; p < kMaxP; ++p)
          if (p < np) ldm_x4(aBase + p * PLANE + ks * 2, a[p]);
#pragma unroll
        for (int q = 0; q < kMaxP; ++q) {
          if (q >= np) break;
          uint32_t b[4];
          ldm_x4(bBase + q * PLANE + ks * 2, b);
#pragma unroll
          for (int l = 0; l < 3; ++l) {
            const int p = g3 + l - q;
            if (p < 0 || p >= S || g3 + l >= S) continue;
            mma_bf16(acc[l][0], a[p], b[0], b[1]);
            mma_bf16(acc[l][1], a[p], b[2], b[3]);
          }
        }
      }
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const int lvl = g3 + l;
        if (lvl >= S) break;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          int sh = 62 - F[h] - BETA * lvl;
          sh = max(-63, min(62, sh));
          const int lsh = sh > 0 ? sh : 0, rsh = sh < 0 ? -sh : 0;
          const long long rnd = rsh > 0 ? (1ll << (rsh - 1)) : 0ll;
#pragma unroll
          for (int nh = 0; nh < 2; ++nh)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              const long long L = (long long)__float2int_rn(acc[l][nh][2 * h + c]);
              accI[h][nh][c] += ((L << lsh) + rnd) >> rsh;
            }
        }
      }
    }
  }
  // ---- 4. exact conversion, then alpha and beta, store
  double xs[2][2][2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = min(rows[h], T - 1);
    const int Ebase = F[h] - 62 + line_e(eA[i]) - 2 * BETA;
#pragma unroll
    for (int nh = 0; nh < 2; ++nh)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int j = min(c0 + 8 * nh + 2 * tq + c, T - 1);
        xs[h][nh][c] = 0.0;
        if (prod) {
          const int E = Ebase + line_e(eB[j]);
          bool bad = false;
          xs[h][nh][c] = fixed_to_double_fast(accI[h][nh][c], E, bad);
          if (bad) xs[h][nh][c] = fixed_to_double(accI[h][nh][c], E);
        }
      }
  }
  const bool alpha_one = g.sc.alpha_re == 1.0;
  if (alpha_one) {
    if (g.sc.beta_zero) small_store<true, true>(g, xs, cold, Cb, in.ldc, rows, m, n, c0, tq);
    else small_store<true, false>(g, xs, cold, Cb, in.ldc, rows, m, n, c0, tq);
  } else {
    if (g.sc.beta_zero) small_store<false, true>(g, xs, cold, Cb, in.ldc, rows, m, n, c0, tq);
    else small_store<false, false>(g, xs, cold, Cb, in.ldc, rows, m, n, c0, tq);
  }
}

template <int S, int BETA, int T>
__device__ __forceinline__ void small_item(const SmallArgs& g, const SmallItem& item, int64_t next,
                                           uint8_t* sm, const DigitCtx& dc) {
  using SH = SmallShape<S, T>;
  const int gid = threadIdx.x / SH::GT, tg = threadIdx.x % SH::GT;
  if (gid >= SH::NG || gid >= item.count) return;
  const SInst in = g.inst[g.ids[item.first + gid]];
  small_instance<S, BETA, T>(g, in, sm + gid * SH::GROUP_BYTES, gid, tg, dc, next);
}

template <int S, int BETA>
__global__ void __launch_bounds__(kSmallThreads, 1) split_small_kernel(const SmallArgs g) {
  extern __shared__ __align__(16) uint8_t sm[];
  const DigitCtx dc = digit_ctx<S>(BETA);
  for (int64_t it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const SmallItem item = g.items[it];
    const int64_t next = it + gridDim.x < g.nitems ? it + gridDim.x : -1;
    if (item.t == 16) small_item<S, BETA, 16>(g, item, next, sm, dc);
    else if (item.t == 32) small_item<S, BETA, 32>(g, item, next, sm, dc);
    else small_item<S, BETA, 64>(g, item, next, sm, dc);
    __syncthreads();  // the next item may lay the shared memory out differently
  }
}

template <int S>
constexpr size_t small_smem_of() {
  const size_t a = (size_t)SmallShape<S, 16>::NG * SmallShape<S, 16>::GROUP_BYTES;
  const size_t b = (size_t)SmallShape<S, 32>::NG * SmallShape<S, 32>::GROUP_BYTES;
  const size_t c = (size_t)SmallShape<S, 64>::NG * SmallShape<S, 64>::GROUP_BYTES;
  return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

}  // namespace

bool split_small_supported(int s, int beta) {
  return (s == 3 && beta == 7) || (s == 6 && beta == 7) || (s == 9 && beta == 6);
}

// Which small instances the kernel takes. Edges up to 32 always (measured
// 0.21-0.49x the time of the tile kernels on uniform batches of n = 16, 24,
// 32 at 3, 6 and 9 slices). Edges 33..64 run padded to 64 here, one instance
// per CTA; they come here only where that measured faster than the tiles
// (whose column width is 48 at 6 and 9 slices, 64 at 3): above 48 at 9
// slices (n = 56, 64: 0.67-0.69x; n = 40, 48: 1.00x), above 40 at 6 slices
// (n = 48..64: 0.57-0.87x; n = 40: 1.00x), always at 3 slices (n = 40..64:
// 0.76-0.79x).
bool split_small_route(int s, int64_t m, int64_t n, int64_t k) {
  const int64_t e = m > n ? (m > k ? m : k) : (n > k ? n : k);
  if (e > kSmallMax) return false;
  if (e <= 32) return true;
  return e > (s == 9 ? 48 : s == 6 ? 40 : 32);
}

int split_small_groups(int s, int t) {
  switch (s) {
#define BG_SMALL_NG(SV)                                                      \
  case SV:                                                                   \
    return t == 16 ? SmallShape<SV, 16>::NG                                  \
                   : t == 32 ? SmallShape<SV, 32>::NG : SmallShape<SV, 64>::NG;
    BG_SMALL_NG(3)
    BG_SMALL_NG(6)
    BG_SMALL_NG(9)
#undef BG_SMALL_NG
    default:
      return 0;
  }
}

size_t split_small_smem(int s) {
  return s == 3 ? small_smem_of<3>() : s == 6 ? small_smem_of<6>() : s == 9 ? small_smem_of<9>() : 0;
}

cudaError_t launch_split_small(int s, int grid, cudaStream_t st, const SmallArgs& g) {
  const size_t smem = split_small_smem(s);
  cudaError_t e;
  switch (s) {
#define BG_SMALL_LAUNCH(SV, BV)                                                       \
  case SV:                                                                            \
    e = cudaFuncSetAttribute(split_small_kernel<SV, BV>,                              \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                   \
    split_small_kernel<SV, BV><<<grid, kSmallThreads, smem, st>>>(g);                 \
    break;
    BG_SMALL_LAUNCH(3, 7)
    BG_SMALL_LAUNCH(6, 7)
    BG_SMALL_LAUNCH(9, 6)
#undef BG_SMALL_LAUNCH
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace splitk
}  // namespace bg
