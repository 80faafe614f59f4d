// The split-precision tensor-core GEMM kernel (see split.cu for the method),
// included by the per-type instantiation units.
#pragma once

#include "split_common.cuh"

namespace bg {
namespace splitk {

// Final stage of the epilogue for 8 columns of one row: exact conversion of
// the fixed-point sums, alpha and beta of Eq. (1), store. The 8 old C values
// and column exponents are loaded first, so that all loads are in flight
// together; the conversions are straight-line code and the rare value
// outside the normal FP64 range is redone exactly afterwards.
// A1: alpha == 1 (no multiply). CM: 0 = C is alpha x (C not read), 1 = alpha
// x + beta C, 2 = alpha x + C (a later pass of a long k adds to C). Both are
// compile-time so that no FP64 instruction runs that the case does not need:
// on this part a warp-wide FP64 instruction holds the FP64 pipe for about 64
// clocks, and a runtime test here compiles to the multiply plus a select.
template <bool CPLX, bool FASTCONV, bool A1, int CM>
__device__ __forceinline__ void epi_store8(const GemmArgs& g, const long long (&acc)[8],
                                           const int32_t* mb, int colb, bool rvalid, int cmin,
                                           int cmax, int coff, int64_t cbase, int64_t ldcv,
                                           int Ebase, int rr, int dcol) {
  double cv[8];
  int fj[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int col = colb + j;
    const bool valid = rvalid && col >= cmin && col < cmax;
    fj[j] = __ldg(mb + col);
    cv[j] = (CM != 0 && valid) ? g.C[cbase + (int64_t)(col + coff) * ldcv] : 0.0;
  }
  double xs[8];
  if constexpr (FASTCONV) {
    bool bad = false;
#pragma unroll
    for (int j = 0; j < 8; ++j) xs[j] = fixed_to_double_fast(acc[j], Ebase + fj[j], bad);
    if (__builtin_expect(bad, 0)) {
#pragma unroll
      for (int j = 0; j < 8; ++j) xs[j] = fixed_to_double(acc[j], Ebase + fj[j]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) xs[j] = fixed_to_double(acc[j], Ebase + fj[j]);
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int col = colb + j;
    const bool valid = rvalid && col >= cmin && col < cmax;
    const double x = valid ? xs[j] : 0.0;
    double* cp = g.C + cbase + (int64_t)(col + coff) * ldcv;
    if constexpr (!CPLX) {
      if (valid) {
        double v = x;
        if constexpr (!A1) v = g.sc.alpha_re * x;
        if constexpr (CM == 2) v += cv[j];
        if constexpr (CM == 1) v = fma(g.sc.beta_re, cv[j], v);
        *cp = v;
      }
    } else {
      double xp = 0.0, cpn = 0.0;
      if constexpr (!A1) xp = __shfl_xor_sync(0xFFFFFFFFu, x, 1);
      if constexpr (CM == 1) cpn = __shfl_xor_sync(0xFFFFFFFFu, cv[j], 1);
      if (valid) {
        const double sgn = (rr & 1) ? 1.0 : -1.0;  // im row: +, re row: -
        double v = x;
        if constexpr (!A1) v = fma(g.sc.alpha_re, x, sgn * g.sc.alpha_im * xp);
        if constexpr (CM == 2) v += cv[j];
        if constexpr (CM == 1) v = fma(g.sc.beta_re, cv[j], fma(sgn * g.sc.beta_im, cpn, v));
        if (col == dcol) v = 0.0;  // Hermitian update: real diagonal
        *cp = v;
      }
    }
  }
}

// epi_store8 for the warp-uniform case at hand.
template <bool CPLX, bool FASTCONV>
__device__ __forceinline__ void epi_store8_for(const GemmArgs& g, const long long (&acc)[8],
                                               const int32_t* mb, int colb, bool rvalid, int cmin,
                                               int cmax, int coff, int64_t cbase, int64_t ldcv,
                                               int Ebase, bool first_pass, bool alpha_one, int rr,
                                               int dcol) {
  const int cm = first_pass ? (g.sc.beta_zero ? 0 : 1) : 2;
#define BG_EPI(A, C)                                                                        \
  epi_store8<CPLX, FASTCONV, A, C>(g, acc, mb, colb, rvalid, cmin, cmax, coff, cbase, ldcv, \
                                   Ebase, rr, dcol)
  if (alpha_one) {
    if (cm == 0) BG_EPI(true, 0);
    else if (cm == 1) BG_EPI(true, 1);
    else BG_EPI(true, 2);
  } else {
    if (cm == 0) BG_EPI(false, 0);
    else if (cm == 1) BG_EPI(false, 1);
    else BG_EPI(false, 2);
  }
#undef BG_EPI
}

// SF > 0: the slice count is the compile-time constant SF (the MMA issue loop
// unrolls completely); SF == 0: any slice count g.s with this tile width.
// CPLX: complex instances (compile-time, so that each version carries only
// its own epilogue).
// DB: two TMEM copies of the level accumulators (2 s BN <= 512), the
// epilogue takes a finished tile whole while the MMAs fill the other copy.
// H: epilogue warps per TMEM lane quadrant; each owns BN / H of the tile's
// columns (more warps hide more of the epilogue's latency, fewer registers
// per thread).
template <int BN, int SF, bool CPLX, bool DB, int H>
__global__ void __launch_bounds__(gemm_threads(H), 1) split_gemm_kernel(const GemmArgs g) {
  static_assert(BN % (8 * H) == 0, "epilogue column groups of 8");
  constexpr int COLS = BN / H;  // output columns per epilogue thread
  constexpr int kEpi = 4 * H;   // epilogue warps
  // The 6-slice tile (40 accumulators per thread) is register-bound: it keeps
  // the compact conversion and drains one level at a time.
  constexpr bool kFastConv = SF != 6;
  constexpr bool kMayPair = SF != 6;
  constexpr int BTILE = BN * kLineBytes;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  const int s = SF > 0 ? SF : g.s;
  const int bplanes_bytes = s * BTILE;
  uint8_t* bbuf = smem;                          // 2 x s B tiles
  uint8_t* aring = smem + 2 * bplanes_bytes;     // a_groups x kAGroup x 16 KiB
  GemmBars& S = *reinterpret_cast<GemmBars*>(aring + g.a_groups * kAGroup * kATileBytes);
  volatile int* abort_flag = &S.abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NG = g.a_groups;
  const int ngroups = (s + kAGroup - 1) / kAGroup;  // plane groups per k-block

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&S.b_full[i], 1);
      mbar_init(&S.b_empty[i], 1);
    }
    for (int i = 0; i < NG; ++i) {
      mbar_init(&S.a_full[i], 1);
      mbar_init(&S.a_empty[i], 1);
    }
    for (int i = 0; i < s; ++i) mbar_init(&S.lvl_full[i], 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&S.acc_full[i], 1);
      mbar_init(&S.acc_empty[i], kEpi);
    }
    mbar_init(&S.tmem_free, kEpi);
    mbar_init(&S.mma_done, 1);
    S.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&S.tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = S.tmem_base;

  if (warp == 0) {
    // ---------------- producer: one TMA bulk copy of the s B planes per k-block, and
    // the s A planes of the k-block through the A ring, kAGroup planes per group
    if (lane == 0) {
      uint32_t kbc = 0, gfill = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; u < g.nunits && ok; u += gridDim.x) {
        const SplitUnit U = g.units[u];
        int64_t at, bt;
        int ablk;
        if (!unit_tiles(g, U, &at, &bt, &ablk)) continue;
        const int npass = unit_passes(g, U);
        for (int c = 0; c < npass && ok; ++c) {
          const int kb_lo = c * g.kpass, kb_hi = min((int)U.nkb, kb_lo + g.kpass);
          for (int kb = kb_lo; kb < kb_hi && ok; ++kb, ++kbc) {
            const int buf = kbc & 1;
            const uint32_t use = kbc >> 1;
            if (use > 0 && !mbar_wait(&S.b_empty[buf], (use - 1) & 1, abort_flag)) {
              record_error(g.err, BG_ERR_TIMEOUT, ERRLOC_SPLIT_EMPTY_BARRIER, (int)u);
              *abort_flag = 1;
              ok = false;
              break;
            }
            mbar_arrive_expect_tx(&S.b_full[buf], (uint32_t)bplanes_bytes);
            bulk_g2s(bbuf + buf * bplanes_bytes, g.tilesB + (bt + (int64_t)kb * s) * BTILE,
                     (uint32_t)bplanes_bytes, &S.b_full[buf]);
            for (int gi = 0; gi < ngroups; ++gi, ++gfill) {
              const int grp = gfill % NG;
              const uint32_t guse = gfill / NG;
              const int p0 = gi * kAGroup, gs = min(kAGroup, s - p0);
              if (guse > 0 && !mbar_wait(&S.a_empty[grp], (guse - 1) & 1, abort_flag)) {
                record_error(g.err, BG_ERR_TIMEOUT, ERRLOC_SPLIT_EMPTY_BARRIER, (int)u);
                *abort_flag = 1;
                ok = false;
                break;
              }
              mbar_arrive_expect_tx(&S.a_full[grp], (uint32_t)(gs * kATileBytes));
              for (int j = 0; j < gs; ++j)
                bulk_g2s(aring + (grp * kAGroup + j) * kATileBytes,
                         g.tilesA + (at + (int64_t)kb * s + p0 + j) * kATileBytes, kATileBytes,
                         &S.a_full[grp]);
            }
          }
        }
      }
      // let every copy this thread started land before the CTA can exit
      for (uint32_t j = kbc > 2 ? kbc - 2 : 0; j < kbc; ++j)
        mbar_wait_time(&S.b_full[j & 1], (j >> 1) & 1);
      for (uint32_t j = gfill > (uint32_t)NG ? gfill - NG : 0; j < gfill; ++j)
        mbar_wait_time(&S.a_full[j % NG], (j / NG) & 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: one N-concatenated MMA per A plane and K-step
    if (lane == 0) {
      uint32_t kbc = 0, passc = 0;
      int grp = 0;
      uint32_t gphase = 0;
      bool ok = true;
      const uint32_t bbase = smem_u32(bbuf);
      const uint32_t abase = smem_u32(aring);
      for (int64_t u = blockIdx.x; u < g.nunits && ok; u += gridDim.x) {
        const SplitUnit U = g.units[u];
        int64_t at_, bt_;
        int ablk_;
        if (!unit_tiles(g, U, &at_, &bt_, &ablk_)) continue;
        const int npass = unit_passes(g, U);
        for (int c = 0; c < npass && ok; ++c, ++passc) {
          // accumulator copy of this pass (always 0 without double buffering)
          const uint32_t buf_off = DB ? (passc & 1) * (uint32_t)(s * BN) : 0u;
          bool free_ok = true;
          if constexpr (DB) {
            if (passc >= 2)
              free_ok = mbar_wait(&S.acc_empty[passc & 1], ((passc >> 1) - 1) & 1, abort_flag);
          } else {
            if (passc > 0) free_ok = mbar_wait(&S.tmem_free, (passc - 1) & 1, abort_flag);
          }
          if (!free_ok) {
            record_error(g.err, BG_ERR_TIMEOUT, ERRLOC_SPLIT_ACC_EMPTY, (int)u);
            *abort_flag = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const int kb_lo = c * g.kpass, kb_hi = min((int)U.nkb, kb_lo + g.kpass);
          for (int kb = kb_lo; kb < kb_hi && ok; ++kb, ++kbc) {
            const int buf = kbc & 1;
            if (!mbar_wait(&S.b_full[buf], (kbc >> 1) & 1, abort_flag)) {
              record_error(g.err, BG_ERR_TIMEOUT, ERRLOC_SPLIT_FULL_BARRIER, (int)u);
              *abort_flag = 1;
              ok = false;
              break;
            }
            const uint64_t bdesc = sw128_desc(bbase + buf * bplanes_bytes);
            const int nk = (kb == U.nkb - 1) ? U.kmma_last : 4;
            const bool last_kb = kb == kb_hi - 1;
            uint32_t acc0 = kb == kb_lo ? 0u : 1u;  // the first MMA of a pass initialises TMEM
#pragma unroll
            for (int p = 0; p < (SF > 0 ? SF : kMaxSlices); ++p) {
              if (SF == 0 && p >= s) break;
              const int j = p % kAGroup;  // plane within its ring group
              if (j == 0) {
                if (!mbar_wait(&S.a_full[grp], gphase, abort_flag)) {
                  record_error(g.err, BG_ERR_TIMEOUT, ERRLOC_SPLIT_FULL_BARRIER, (int)u);
                  *abort_flag = 1;
                  ok = false;
                  break;
                }
                tc_fence_after();
              }
              const uint64_t adesc = sw128_desc(abase + (grp * kAGroup + j) * kATileBytes);
              // B planes 1..s-p (levels p+2 .. s+1) as one N range, cut in pieces of <= 256
              const int ncat = (s - p) * BN;
              const int n1 = ncat > 256 ? ncat - 256 : 0;
              const uint32_t id0 = make_idesc(BM, ncat > 256 ? 256 : ncat);
              const uint32_t id1 = make_idesc(BM, n1 > 0 ? n1 : 16);
              const uint32_t d0 = tmem_base + buf_off + p * BN;
              constexpr uint64_t kB256 = (256 * kLineBytes) >> 4;
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                if (kk < nk) {
                  const uint32_t acc = kk == 0 ? acc0 : 1u;
                  umma_bf16(d0, adesc + 2 * kk, bdesc + 2 * kk, id0, acc);
                  if (n1 > 0) umma_bf16(d0 + 256, adesc + 2 * kk, bdesc + kB256 + 2 * kk, id1, acc);
                }
              }
              acc0 = 1u;
              if (j == kAGroup - 1 || p == s - 1) {
                // the group's planes are done: release its slots; in the last k-block of
                // the pass every level up to p is complete
                umma_commit(&S.a_empty[grp]);
                if (!DB && last_kb) umma_commit(&S.lvl_full[p / kAGroup]);
                if (++grp == NG) {
                  grp = 0;
                  gphase ^= 1;
                }
              }
            }
            if (!ok) break;
            umma_commit(&S.b_empty[buf]);
            if (DB && last_kb) umma_commit(&S.acc_full[passc & 1]);  // the whole tile is done
          }
        }
      }
      // all MMAs issued by this thread are complete once mma_done fires
      umma_commit(&S.mma_done);
      mbar_wait_time(&S.mma_done, 0);
    }
  } else {
    // ---------------- epilogue: drain levels, recombine, free TMEM, store
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;  // column group of this warp within its quadrant
    const int row = quad * 32 + lane;
    const int col0 = half * COLS;
    const uint32_t tq = tmem_base + ((uint32_t)(quad * 32) << 16) + col0;
    const bool alpha_one = g.sc.alpha_re == 1.0 && g.sc.alpha_im == 0.0;
    uint32_t passc = 0;
    bool ok = true;
    for (int64_t u = blockIdx.x; u < g.nunits && ok; u += gridDim.x) {
      const SplitUnit U = g.units[u];
      int64_t at, bt;
      int ablk;
      if (!unit_tiles(g, U, &at, &bt, &ablk)) {
        if (warp == 2 && lane == 0)
          record_error(g.err, BG_ERR_INVALID_ARG, ERRLOC_CHAIN_INDEX, (int)g.order[U.pos]);
        continue;
      }
      const int32_t* ma = g.metaA + (int64_t)ablk * kMetaStride;
      const int32_t* mb = g.metaB + (int64_t)U.b_blk * kMetaStride;
      const int e_i = ma[row];
      // frame: the row's norm exponent plus the largest one of the B block
      int rbmax = -126;
      for (int c = lane; c < BN; c += 32) rbmax = max(rbmax, mb[128 + c]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) rbmax = max(rbmax, __shfl_xor_sync(0xFFFFFFFFu, rbmax, o));
      const int F = ma[128 + row] + rbmax + 1;
      // output rows/columns of this thread
      int rr, inst_pos, cmin, cmax, coff;
      bool rvalid;
      if (U.g > 1) {
        const int li = row / U.mrow;
        rr = row - li * U.mrow;
        rvalid = li < U.g;
        inst_pos = U.pos + (rvalid ? li : 0);
        cmin = li * U.ncol;
        cmax = cmin + U.ncol;
        coff = -cmin;
      } else {
        rr = U.r0 + row;
        inst_pos = U.pos;
        rvalid = true;
        cmin = 0;
        cmax = BN;
        coff = U.c0;
      }
      const SInst in = g.inst[g.order[inst_pos]];
      const int mv = CPLX ? 2 * in.m : in.m;
      rvalid = rvalid && rr < mv;
      if (U.g == 1) cmax = min(cmax, in.n - U.c0);
      // Hermitian update: only columns up to the diagonal (instance row >=
      // instance column, in complex rows for complex data); the diagonal of
      // complex data is real
      int dcol = -1;
      if (g.herk) {
        const int row_inst = CPLX ? rr >> 1 : rr;
        cmax = min(cmax, row_inst - coff + 1);
        if (CPLX && (rr & 1)) dcol = row_inst - coff;
      }
      const int64_t cbase = (CPLX ? 2 * in.c_off : in.c_off) + rr;
      const int64_t ldcv = CPLX ? 2 * in.ldc : in.ldc;
      const int Ebase = F - 62 + e_i - 2 * g.beta;
      const int npass = unit_passes(g, U);
      if constexpr (DB) {
        // ---- double-buffered TMEM: take the finished tile whole, 8 columns at a time
        for (int c = 0; c < max(npass, 1) && ok; ++c) {
          const uint32_t b = passc & 1;
          if (npass > 0) {
            bool got = true;
            if (lane == 0) got = mbar_wait(&S.acc_full[b], (passc >> 1) & 1, abort_flag);
            got = __shfl_sync(0xFFFFFFFFu, got ? 1 : 0, 0) != 0;
            if (!got) {
              if (lane == 0) {
                record_error(g.err, BG_ERR_TIMEOUT, ERRLOC_SPLIT_ACC_FULL, (int)u);
                *abort_flag = 1;
              }
              ok = false;
              break;
            }
            tc_fence_after();
          }
          const uint32_t tb = tq + b * (uint32_t)(s * BN);
#pragma unroll 1
          for (int j0 = 0; j0 < COLS; j0 += 8) {
            long long acc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = 0;
            if (npass > 0) {
              // all levels of the 8 columns in flight at once (compile-time slice
              // counts), then the exact fixed-point sum
              constexpr int NV = SF > 0 ? SF : 1;
              uint32_t v[NV][8];
              if constexpr (SF > 0) {
#pragma unroll
                for (int lv = 0; lv < SF; ++lv) tmem_ld8(tb + lv * BN + j0, v[lv]);
                tmem_ld_wait();
              }
#pragma unroll
              for (int lv = 0; lv < (SF > 0 ? SF : kMaxSlices); ++lv) {
                if (SF == 0 && lv >= s) break;
                uint32_t(&vl)[8] = v[SF > 0 ? lv : 0];
                if constexpr (SF == 0) {
                  tmem_ld8(tb + lv * BN + j0, vl);
                  tmem_ld_wait();
                }
                int sh = 62 - F - g.beta * lv;
                sh = max(-63, min(62, sh));
                const int lsh = sh > 0 ? sh : 0, rsh = sh < 0 ? -sh : 0;
                const long long rnd = rsh > 0 ? (1ll << (rsh - 1)) : 0ll;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  const long long L = (long long)__float2int_rn(__uint_as_float(vl[j]));
                  acc[j] += ((L << lsh) + rnd) >> rsh;
                }
              }
            }
            epi_store8_for<CPLX, kFastConv>(g, acc, mb, col0 + j0, rvalid, cmin, cmax, coff, cbase, ldcv, Ebase,
                             c == 0, alpha_one, rr, dcol);
          }
          if (npass > 0) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.acc_empty[b]);
            ++passc;
          }
        }
      } else {
        for (int c = 0; c < max(npass, 1) && ok; ++c) {
          long long acc[COLS];
#pragma unroll
          for (int j = 0; j < COLS; ++j) acc[j] = 0;
          if (npass > 0) {
            // Levels are drained as they complete. With beta <= 6 two adjacent
            // levels first combine exactly in 32 bits (|L_t 2^beta + L_t+1| <
            // 2^30 + 2^24), which halves the 64-bit shifts and adds.
            const bool pairs = kMayPair && g.beta <= 6;
#pragma unroll 1
            for (int lv = 0; lv < s;) {
              const int nlv = (pairs && lv + 1 < s) ? 2 : 1;
              bool got = true;
              // level t is complete once its plane group (t / kAGroup) is
              if (lane == 0)
                got = mbar_wait(&S.lvl_full[(lv + nlv - 1) / kAGroup], passc & 1, abort_flag);
              got = __shfl_sync(0xFFFFFFFFu, got ? 1 : 0, 0) != 0;
              if (!got) {
                if (lane == 0) {
                  record_error(g.err, BG_ERR_TIMEOUT, ERRLOC_SPLIT_ACC_FULL, (int)u);
                  *abort_flag = 1;
                }
                ok = false;
                break;
              }
              tc_fence_after();
              const int lvl = lv + nlv - 1;  // the combined value sits at this level's weight
              int sh = 62 - F - g.beta * lvl;
              sh = max(-63, min(62, sh));
              const int lsh = sh > 0 ? sh : 0, rsh = sh < 0 ? -sh : 0;
              const long long rnd = rsh > 0 ? (1ll << (rsh - 1)) : 0ll;
#pragma unroll
              for (int j0 = 0; j0 < COLS; j0 += 8) {
                uint32_t v0[8], v1[8];
                tmem_ld8(tq + lv * BN + j0, v0);
                if (nlv == 2) tmem_ld8(tq + (lv + 1) * BN + j0, v1);
                tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  int L = __float2int_rn(__uint_as_float(v0[j]));
                  if (nlv == 2) L = (L << g.beta) + __float2int_rn(__uint_as_float(v1[j]));
                  acc[j0 + j] += (((long long)L << lsh) + rnd) >> rsh;
                }
              }
              lv += nlv;
            }
            if (!ok) break;
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.tmem_free);
            ++passc;
          }
          // ---- exact conversion, alpha/beta, store (TMEM already free: overlaps the next MMAs).
          for (int j0 = 0; j0 < COLS; j0 += 8) {
            epi_store8_for<CPLX, kFastConv>(g, *reinterpret_cast<const long long(*)[8]>(acc), mb, col0 + j0,
                             rvalid, cmin, cmax, coff, cbase, ldcv, Ebase, c == 0, alpha_one, rr, dcol);
            // rotate the next 8 accumulators into place (keeps the loop body small)
#pragma unroll
            for (int j = 0; j + 8 < COLS; ++j) acc[j] = acc[j + 8];
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kTmemCols));
  }
}


// Same for the GEMM kernel template arguments: the tile width BN (from s)
// and the compile-time slice count (3, 6 and 9 have unrolled versions).
#define BG_DISPATCH_GEMM(s, ...)                                                    \
  switch (s) {                                                                      \
    case 3: { constexpr int BNV = bn_for(3), SFV = 3, HV = 4; constexpr bool DBV = true; __VA_ARGS__; } \
    case 6: { constexpr int BNV = bn_for(6), SFV = 6, HV = 3; constexpr bool DBV = false; __VA_ARGS__; } \
    case 9: { constexpr int BNV = bn_for(9), SFV = 9, HV = 3; constexpr bool DBV = false; __VA_ARGS__; } \
    case 1: case 2: { constexpr int BNV = 128, SFV = 0, HV = 2; constexpr bool DBV = true; __VA_ARGS__; } \
    case 4: { constexpr int BNV = 64, SFV = 0, HV = 2; constexpr bool DBV = true; __VA_ARGS__; }   \
    case 5: { constexpr int BNV = 48, SFV = 0, HV = 2; constexpr bool DBV = true; __VA_ARGS__; }   \
    case 7: case 8: { constexpr int BNV = 64, SFV = 0, HV = 2; constexpr bool DBV = false; __VA_ARGS__; } \
    case 10: { constexpr int BNV = 48, SFV = 0, HV = 2; constexpr bool DBV = false; __VA_ARGS__; } \
    case 11: case 12: { constexpr int BNV = 32, SFV = 0, HV = 2; constexpr bool DBV = false; __VA_ARGS__; } \
    default: return cudaErrorInvalidValue;                                          \
  }

template <bool CPLX>
cudaError_t launch_gemm_t(int s, int grid, size_t smem, cudaStream_t st, const GemmArgs& g) {
  BG_DISPATCH_GEMM(s, {
    split_gemm_kernel<BNV, SFV, CPLX, DBV, HV><<<grid, gemm_threads(HV), smem, st>>>(g);
    return cudaGetLastError();
  });
}

template <bool CPLX>
cudaError_t set_attr_t(int s) {
  BG_DISPATCH_GEMM(s, {
    return cudaFuncSetAttribute(split_gemm_kernel<BNV, SFV, CPLX, DBV, HV>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
  });
}

}  // namespace splitk
}  // namespace bg
