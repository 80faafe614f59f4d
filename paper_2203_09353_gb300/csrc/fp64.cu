// FP64 / complex128 path of Eq. (1) (Sec. 2): C_i = alpha A_i B_i + beta C_i.
//
// One persistent kernel walks a list of work items; each item runs one of
// the tile programs below on one tile (or one group of small instances):
//  * small programs: one warp per instance, several instances per CTA (the
//    tiny-matrix idea the paper cites in Sec. 2: several small C per block);
//  * tile programs: a 2-D output tile per CTA (the tiling of Sec. 2), operands
//    staged through shared memory in double-buffered k-slices.
// On GB300 the FP64 pipe issues 2 DFMA per clock per SM (measured 1.19
// TFLOP/s chip-wide, DMMA 1.05), i.e. one warp-wide DFMA per 64 clocks per
// SM sub-partition, so every program here is FP64-issue-bound long before
// memory matters: the design goal is only to keep DFMAs flowing on every SM
// with few non-FMA instructions.
#include <algorithm>

#include "bgemm_internal.h"

namespace bg {

// ---- instance sources ---------------------------------------------------------

struct Desc {
  const double* A;  // complex: interleaved pairs
  const double* B;
  double* C;
  int m, n, k;
  int64_t lda, ldb, ldc;  // elements
  // Hermitian rank-k update (Sec. 3, rho = Psi Psi^H): B is A^H (A^T when
  // real), read from A; only outputs on or below the diagonal are stored,
  // and a complex diagonal gets a zero imaginary part.
  int herm;
};

// Element (p, c) of B (real).
__device__ __forceinline__ double ld_b(const Desc& d, int p, int c) {
  return d.herm ? __ldg(d.A + c + (int64_t)p * d.lda) : __ldg(d.B + p + (int64_t)c * d.ldb);
}

// Element (p, c) of B (complex).
__device__ __forceinline__ double2 ld_bc(const Desc& d, int p, int c) {
  if (d.herm) {
    double2 v = __ldg(reinterpret_cast<const double2*>(d.A) + c + (int64_t)p * d.lda);
    v.y = -v.y;
    return v;
  }
  return __ldg(reinterpret_cast<const double2*>(d.B) + p + (int64_t)c * d.ldb);
}

// Whether output (r, c) is stored (Hermitian updates keep the lower triangle).
__device__ __forceinline__ bool keep_out(const Desc& d, int r, int c) { return !d.herm || r >= c; }

// Fixed-size batch: instance i at constant strides.
struct FixedSrc {
  const double* A;
  const double* B;
  double* C;
  int m, n, k;
  int64_t lda, ldb, ldc, sA, sB, sC;
  int esz;  // doubles per element (1 real, 2 complex)
  __device__ Desc desc(int64_t i) const {
    Desc d;
    d.A = A + i * sA * esz;
    d.B = B + i * sB * esz;
    d.C = C + i * sC * esz;
    d.m = m; d.n = n; d.k = k;
    d.lda = lda; d.ldb = ldb; d.ldc = ldc;
    d.herm = 0;
    return d;
  }
  __device__ int64_t small_inst(int64_t pos) const { return pos; }
};

// Variable-size batch: rows of a device table (m, n, k, lda, ldb, ldc, a_off, b_off, c_off).
struct TableSrc {
  const int64_t* table;
  const int32_t* order;
  const double* A;
  const double* B;
  double* C;
  int esz;
  int herm;  // plan of Hermitian rank-k updates (B unused)
  __device__ Desc desc(int64_t i) const {
    const int64_t* t = table + 9 * i;
    Desc d;
    d.m = (int)t[0]; d.n = (int)t[1]; d.k = (int)t[2];
    d.lda = t[3]; d.ldb = t[4]; d.ldc = t[5];
    d.A = A + t[6] * esz;
    d.B = herm ? d.A : B + t[7] * esz;
    d.C = C + t[8] * esz;
    d.herm = herm;
    return d;
  }
  __device__ int64_t small_inst(int64_t pos) const { return order[pos]; }
};

// One step of the chain: walker w computes U[idx[w]] * Cin_w into Cout_w.
struct ChainSrc {
  const int64_t* wn;
  const int64_t* woff;
  const int64_t* pool_off;
  const int64_t* pool_n;
  int32_t pool_count;
  const int32_t* order;
  const int32_t* idx;
  const double* U;
  const double* Cin;
  double* Cout;
  int esz;
  // An index out of range, or naming a pool matrix of another size, turns the
  // walker's step into a no-op (its output is left as is).
  __device__ Desc desc(int64_t w) const {
    int n = (int)wn[w];
    const int j = idx[w];
    const bool ok = j >= 0 && j < pool_count && pool_n[j] == n;
    if (!ok) n = 0;
    Desc d;
    d.m = d.n = d.k = n;
    d.lda = d.ldb = d.ldc = n > 0 ? n : 1;
    d.A = U + (ok ? pool_off[j] : 0) * esz;
    d.B = Cin + woff[w] * esz;
    d.C = Cout + woff[w] * esz;
    d.herm = 0;
    return d;
  }
  __device__ int64_t small_inst(int64_t pos) const { return order[pos]; }
};

// ---- schedules ------------------------------------------------------------------

struct FixedSched {
  int prog;
  int tm, tn;
  int g;  // small programs: instances per item
  int64_t tiles_m, tiles_n, batch;
  __device__ WorkItem get(int64_t it) const {
    WorkItem w;
    w.prog = (int16_t)prog;
    if (tm == 0) {
      w.inst = (int32_t)(it * g);
      const int64_t left = batch - it * g;
      w.count = (int16_t)(left < g ? left : g);
      w.r0 = kSmallPerCta / g;  // warps per instance
      w.c0 = 0;
    } else {
      const int64_t per = tiles_m * tiles_n;
      w.inst = (int32_t)(it / per);
      const int64_t t = it - (it / per) * per;
      w.r0 = (int32_t)((t % tiles_m) * tm);
      w.c0 = (int32_t)((t / tiles_m) * tn);
      w.count = 1;
    }
    return w;
  }
};

struct TableSched {
  const WorkItem* items;
  __device__ WorkItem get(int64_t it) const { return items[it]; }
};

// ---- real tile program: 64x64 outputs, BK = 16, DFMA ----------------------------

constexpr int TR = 64, BKR = 16;

struct SmemR64 {
  double a[2][BKR][TR];  // a[s][kk][row]
  double b[2][BKR][TR];  // b[s][kk][col]
};

__device__ __forceinline__ void tile_r64(const Desc& d, int r0, int c0, const Scalars& s,
                                         SmemR64& sm) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int K = s.alpha_zero ? 0 : d.k;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  // global -> register staging: A 64 rows x 16 k, B 16 k x 64 cols
  const int ar = tid & 63, ak = tid >> 6;  // row, k (+4j)
  const int bk = tid & 15, bc = tid >> 4;  // k, col (+16j)
  double ra[4], rb[4];
  auto gload = [&](int k0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ar, kk = k0 + ak + 4 * j;
      ra[j] = (r < d.m && kk < K) ? __ldg(d.A + r + (int64_t)kk * d.lda) : 0.0;
      const int kb = k0 + bk, c = c0 + bc + 16 * j;
      rb[j] = (kb < K && c < d.n) ? ld_b(d, kb, c) : 0.0;
    }
  };
  auto sstore = [&](int st) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      sm.a[st][ak + 4 * j][ar] = ra[j];
      sm.b[st][bk][bc + 16 * j] = rb[j];
    }
  };

  if (K > 0) {
    gload(0);
    sstore(0);
  }
  __syncthreads();
  int st = 0;
  for (int k0 = 0; k0 < K; k0 += BKR) {
    const bool more = k0 + BKR < K;
    if (more) gload(k0 + BKR);
#pragma unroll
    for (int kk = 0; kk < BKR; ++kk) {
      const double2 a01 = *reinterpret_cast<const double2*>(&sm.a[st][kk][ty * 4]);
      const double2 a23 = *reinterpret_cast<const double2*>(&sm.a[st][kk][ty * 4 + 2]);
      const double2 b01 = *reinterpret_cast<const double2*>(&sm.b[st][kk][tx * 4]);
      const double2 b23 = *reinterpret_cast<const double2*>(&sm.b[st][kk][tx * 4 + 2]);
      const double a[4] = {a01.x, a01.y, a23.x, a23.y};
      const double b[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (more) sstore(st ^ 1);
    __syncthreads();
    st ^= 1;
  }

#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = c0 + tx * 4 + j;
    if (c >= d.n) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + ty * 4 + i;
      if (r >= d.m || !keep_out(d, r, c)) continue;
      double* cp = d.C + r + (int64_t)c * d.ldc;
      double v = s.alpha_re * acc[i][j];
      if (!s.beta_zero) v = fma(s.beta_re, *cp, v);
      *cp = v;
    }
  }
}

// ---- real tile program on the FP64 tensor cores: mma.sync m8n8k4 -----------------
// 8 warps as 2 (rows) x 4 (cols); each warp owns 32x16 outputs = 4x2 fragments.
// Fragment layout (PTX ISA, mma .f64 m8n8k4, row.col): lane = 4*g + t;
// A(g, t), B(t, g), C(g, 2t + {0,1}).

__device__ __forceinline__ void dmma_884(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

__device__ __forceinline__ void tile_r64_dmma(const Desc& d, int r0, int c0, const Scalars& s,
                                              SmemR64& sm) {
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 1, wn = warp >> 1;
  const int g = lane >> 2, t = lane & 3;
  const int K = s.alpha_zero ? 0 : d.k;
  double acc[4][2][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

  const int ar = tid & 63, ak = tid >> 6;
  const int bk = tid & 15, bc = tid >> 4;
  double ra[4], rb[4];
  auto gload = [&](int k0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ar, kk = k0 + ak + 4 * j;
      ra[j] = (r < d.m && kk < K) ? __ldg(d.A + r + (int64_t)kk * d.lda) : 0.0;
      const int kb = k0 + bk, c = c0 + bc + 16 * j;
      rb[j] = (kb < K && c < d.n) ? ld_b(d, kb, c) : 0.0;
    }
  };
  auto sstore = [&](int st) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      sm.a[st][ak + 4 * j][ar] = ra[j];
      sm.b[st][bk][bc + 16 * j] = rb[j];
    }
  };
  if (K > 0) {
    gload(0);
    sstore(0);
  }
  __syncthreads();
  int st = 0;
  for (int k0 = 0; k0 < K; k0 += BKR) {
    const bool more = k0 + BKR < K;
    if (more) gload(k0 + BKR);
#pragma unroll
    for (int k4 = 0; k4 < BKR; k4 += 4) {
      double a[4], b[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sm.a[st][k4 + t][wm * 32 + i * 8 + g];
#pragma unroll
      for (int j = 0; j < 2; ++j) b[j] = sm.b[st][k4 + t][wn * 16 + j * 8 + g];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) dmma_884(acc[i][j][0], acc[i][j][1], a[i], b[j]);
    }
    if (more) sstore(st ^ 1);
    __syncthreads();
    st ^= 1;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + wm * 32 + i * 8 + g;
    if (r >= d.m) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = c0 + wn * 16 + j * 8 + 2 * t + h;
        if (c >= d.n || !keep_out(d, r, c)) continue;
        double* cp = d.C + r + (int64_t)c * d.ldc;
        double v = s.alpha_re * acc[i][j][h];
        if (!s.beta_zero) v = fma(s.beta_re, *cp, v);
        *cp = v;
      }
  }
}

// ---- complex tile program: 32x32 complex outputs, BK = 16 ---------------------------

constexpr int TC = 32, BKC = 16;

struct SmemC128 {
  double2 a[2][BKC][TC];
  double2 b[2][BKC][TC];
};

__device__ __forceinline__ void cmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

__device__ __forceinline__ double2 c_epilogue(double2 acc, const double2* cp, const Scalars& s) {
  double2 v;
  v.x = s.alpha_re * acc.x - s.alpha_im * acc.y;
  v.y = s.alpha_re * acc.y + s.alpha_im * acc.x;
  if (!s.beta_zero) {
    const double2 c = *cp;
    v.x = fma(s.beta_re, c.x, fma(-s.beta_im, c.y, v.x));
    v.y = fma(s.beta_re, c.y, fma(s.beta_im, c.x, v.y));
  }
  return v;
}

__device__ __forceinline__ void tile_c128(const Desc& d, int r0, int c0, const Scalars& s,
                                          SmemC128& sm) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int K = s.alpha_zero ? 0 : d.k;
  const double2* A = reinterpret_cast<const double2*>(d.A);
  double2 acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0.0, 0.0);

  const int ar = tid & 31, ak = tid >> 5;  // row, k (+8j)
  const int bk = tid & 15, bc = tid >> 4;  // k, col (+16j)
  double2 ra[2], rb[2];
  const double2 z = make_double2(0.0, 0.0);
  auto gload = [&](int k0) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int r = r0 + ar, kk = k0 + ak + 8 * j;
      ra[j] = (r < d.m && kk < K) ? __ldg(A + r + (int64_t)kk * d.lda) : z;
      const int kb = k0 + bk, c = c0 + bc + 16 * j;
      rb[j] = (kb < K && c < d.n) ? ld_bc(d, kb, c) : z;
    }
  };
  auto sstore = [&](int st) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      sm.a[st][ak + 8 * j][ar] = ra[j];
      sm.b[st][bk][bc + 16 * j] = rb[j];
    }
  };
  if (K > 0) {
    gload(0);
    sstore(0);
  }
  __syncthreads();
  int st = 0;
  for (int k0 = 0; k0 < K; k0 += BKC) {
    const bool more = k0 + BKC < K;
    if (more) gload(k0 + BKC);
#pragma unroll
    for (int kk = 0; kk < BKC; ++kk) {
      const double2 a0 = sm.a[st][kk][ty * 2], a1 = sm.a[st][kk][ty * 2 + 1];
      const double2 b0 = sm.b[st][kk][tx * 2], b1 = sm.b[st][kk][tx * 2 + 1];
      cmac(acc[0][0], a0, b0);
      cmac(acc[0][1], a0, b1);
      cmac(acc[1][0], a1, b0);
      cmac(acc[1][1], a1, b1);
    }
    if (more) sstore(st ^ 1);
    __syncthreads();
    st ^= 1;
  }
  double2* C = reinterpret_cast<double2*>(d.C);
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int c = c0 + tx * 2 + j;
    if (c >= d.n) continue;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r = r0 + ty * 2 + i;
      if (r >= d.m || !keep_out(d, r, c)) continue;
      double2* cp = C + r + (int64_t)c * d.ldc;
      double2 v = c_epilogue(acc[i][j], cp, s);
      if (d.herm && r == c) v.y = 0.0;
      *cp = v;
    }
  }
}

// ---- small programs: W warps per instance (real), one warp (complex) ----------
// Thread t (0 <= t < 32 W) of an instance owns outputs o = t + 32 W j
// (j < MAXOUT) of the m*n outputs in column-major order, i.e. (r, c) =
// (o mod m, o div m). When m divides 32 the row is the same for every j and
// the column steps by 32 W / m, so one A load feeds MAXOUT DFMAs; otherwise
// every output loads its own A element.

template <int MAXOUT, int W>
__device__ __forceinline__ void small_r64(const Desc& d, const Scalars& s, int t) {
  const int lane = t;  // thread of the instance
  constexpr int stride = 32 * W;
  const int m = d.m, n = d.n, mn = m * n;
  const int K = s.alpha_zero ? 0 : d.k;
  double acc[MAXOUT];
#pragma unroll
  for (int j = 0; j < MAXOUT; ++j) acc[j] = 0.0;
  if (m > 0 && (32 % m) == 0) {
    const int r = lane % m, c0 = lane / m, cstep = stride / m;
    const double* ap = d.A + r;
    const double* bp = d.B + (int64_t)c0 * d.ldb;
    const int64_t bstep = (int64_t)cstep * d.ldb;
    for (int p = 0; p < K; ++p) {
      const double a = __ldg(ap + (int64_t)p * d.lda);
#pragma unroll
      for (int j = 0; j < MAXOUT; ++j)
        if (c0 + j * cstep < n)
          acc[j] = fma(a, d.herm ? ld_b(d, p, c0 + j * cstep) : __ldg(bp + p + j * bstep), acc[j]);
    }
#pragma unroll
    for (int j = 0; j < MAXOUT; ++j) {
      const int c = c0 + j * cstep;
      if (c < n && keep_out(d, r, c)) {
        double* cp = d.C + r + (int64_t)c * d.ldc;
        double v = s.alpha_re * acc[j];
        if (!s.beta_zero) v = fma(s.beta_re, *cp, v);
        *cp = v;
      }
    }
  } else {
    for (int p = 0; p < K; ++p) {
#pragma unroll
      for (int j = 0; j < MAXOUT; ++j) {
        const int o = lane + stride * j;
        if (o < mn) {
          const int r = o % m, c = o / m;
          acc[j] = fma(__ldg(d.A + r + (int64_t)p * d.lda), ld_b(d, p, c), acc[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < MAXOUT; ++j) {
      const int o = lane + stride * j;
      if (o < mn) {
        const int r = o % m, c = o / m;
        if (!keep_out(d, r, c)) continue;
        double* cp = d.C + r + (int64_t)c * d.ldc;
        double v = s.alpha_re * acc[j];
        if (!s.beta_zero) v = fma(s.beta_re, *cp, v);
        *cp = v;
      }
    }
  }
}

template <int MAXOUT>
__device__ __forceinline__ void small_c128(const Desc& d, const Scalars& s) {
  const int lane = threadIdx.x & 31;
  const int m = d.m, n = d.n, mn = m * n;
  const int K = s.alpha_zero ? 0 : d.k;
  const double2* A = reinterpret_cast<const double2*>(d.A);
  const double2* B = reinterpret_cast<const double2*>(d.B);
  double2* C = reinterpret_cast<double2*>(d.C);
  double2 acc[MAXOUT];
#pragma unroll
  for (int j = 0; j < MAXOUT; ++j) acc[j] = make_double2(0.0, 0.0);
  if (m > 0 && (32 % m) == 0) {
    const int r = lane % m, c0 = lane / m, cstep = 32 / m;
    const int64_t bstep = (int64_t)cstep * d.ldb;
    const double2* bp = B + (int64_t)c0 * d.ldb;
    for (int p = 0; p < K; ++p) {
      const double2 a = __ldg(A + r + (int64_t)p * d.lda);
#pragma unroll
      for (int j = 0; j < MAXOUT; ++j)
        if (c0 + j * cstep < n)
          cmac(acc[j], a, d.herm ? ld_bc(d, p, c0 + j * cstep) : __ldg(bp + p + j * bstep));
    }
#pragma unroll
    for (int j = 0; j < MAXOUT; ++j) {
      const int c = c0 + j * cstep;
      if (c < n && keep_out(d, r, c)) {
        double2* cp = C + r + (int64_t)c * d.ldc;
        double2 v = c_epilogue(acc[j], cp, s);
        if (d.herm && r == c) v.y = 0.0;
        *cp = v;
      }
    }
  } else {
    for (int p = 0; p < K; ++p) {
#pragma unroll
      for (int j = 0; j < MAXOUT; ++j) {
        const int o = lane + 32 * j;
        if (o < mn) {
          const int r = o % m, c = o / m;
          cmac(acc[j], __ldg(A + r + (int64_t)p * d.lda), ld_bc(d, p, c));
        }
      }
    }
#pragma unroll
    for (int j = 0; j < MAXOUT; ++j) {
      const int o = lane + 32 * j;
      if (o < mn) {
        const int r = o % m, c = o / m;
        if (!keep_out(d, r, c)) continue;
        double2* cp = C + r + (int64_t)c * d.ldc;
        double2 v = c_epilogue(acc[j], cp, s);
        if (d.herm && r == c) v.y = 0.0;
        *cp = v;
      }
    }
  }
}

// Small-program limits (outputs per warp).
constexpr int kSmallR64Fast = 1024, kSmallR64Gen = 512;   // MAXOUT 32 / 16
constexpr int kSmallC128Fast = 512, kSmallC128Gen = 256;  // MAXOUT 16 / 8

// ---- the persistent kernel ---------------------------------------------------------

union SmemFp64 {
  SmemR64 r;
  SmemC128 c;
};

template <class Src, class Sched>
__global__ void __launch_bounds__(kFp64Threads, 1)
    fp64_persistent(Src src, Sched sched, int64_t n_items, Scalars s) {
  __shared__ __align__(16) SmemFp64 sm;
  const int warp = threadIdx.x >> 5;
  for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
    const WorkItem w = sched.get(it);
    switch (w.prog) {
      case PROG_R64_TILE:
        tile_r64(src.desc(w.inst), w.r0, w.c0, s, sm.r);
        break;
      case PROG_R64_DMMA:
        tile_r64_dmma(src.desc(w.inst), w.r0, w.c0, s, sm.r);
        break;
      case PROG_C128_TILE:
        tile_c128(src.desc(w.inst), w.r0, w.c0, s, sm.c);
        break;
      case PROG_R64_SMALL: {
        const int W = w.r0 > 0 ? w.r0 : 1;  // warps per instance
        const int slot = warp / W;
        if (slot < w.count) {
          const Desc d = src.desc(src.small_inst((int64_t)w.inst + slot));
          const int t = (warp - slot * W) * 32 + (threadIdx.x & 31);
          const bool fast = d.m > 0 && (32 % d.m) == 0;
          // outputs per thread: at most 1024 (fast) or 512 (other shapes) per instance
          if (W == 1) fast ? small_r64<32, 1>(d, s, t) : small_r64<16, 1>(d, s, t);
          else fast ? small_r64<4, 8>(d, s, t) : small_r64<2, 8>(d, s, t);
        }
        break;
      }
      case PROG_C128_SMALL:
        if (warp < w.count) {
          const Desc d = src.desc(src.small_inst((int64_t)w.inst + warp));
          if (d.m > 0 && (32 % d.m) == 0) small_c128<16>(d, s);
          else small_c128<8>(d, s);
        }
        break;
      default:
        break;
    }
  }
}

// ---- host side -----------------------------------------------------------------------

bool prog_is_small(int prog) { return prog == PROG_R64_SMALL || prog == PROG_C128_SMALL; }

void prog_tile(int prog, int* tm, int* tn) {
  switch (prog) {
    case PROG_R64_TILE:
    case PROG_R64_DMMA: *tm = TR; *tn = TR; break;
    case PROG_C128_TILE: *tm = TC; *tn = TC; break;
    default: *tm = 0; *tn = 0; break;
  }
}

bool prog_fits(int prog, bg_dtype dt, int64_t m, int64_t n) {
  const int64_t mn = m * n;
  const bool div32 = m > 0 && (32 % m) == 0;
  switch (prog) {
    case PROG_R64_SMALL: return dt == BG_R64 && (div32 ? mn <= kSmallR64Fast : mn <= kSmallR64Gen);
    case PROG_C128_SMALL: return dt == BG_C128 && (div32 ? mn <= kSmallC128Fast : mn <= kSmallC128Gen);
    case PROG_R64_TILE:
    case PROG_R64_DMMA: return dt == BG_R64;
    case PROG_C128_TILE: return dt == BG_C128;
    default: return false;
  }
}

int default_prog(bg_dtype dt, int64_t m, int64_t n, int64_t k) {
  (void)k;
  if (dt == BG_R64) return prog_fits(PROG_R64_SMALL, dt, m, n) ? PROG_R64_SMALL : PROG_R64_TILE;
  return prog_fits(PROG_C128_SMALL, dt, m, n) ? PROG_C128_SMALL : PROG_C128_TILE;
}

static int g_bps[2] = {0, 0};

int fp64_blocks_per_sm(bg_dtype dt) {
  int& v = g_bps[dt == BG_C128 ? 1 : 0];
  if (v == 0) {
    int b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &b, fp64_persistent<TableSrc, TableSched>, kFp64Threads, 0);
    v = (e == cudaSuccess && b > 0) ? b : 1;
  }
  return v;
}

static int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

cudaError_t launch_fp64_fixed(bg_dtype dt, int prog, int64_t m, int64_t n, int64_t k,
                              const Scalars& s, const void* A, int64_t lda, int64_t sA,
                              const void* B, int64_t ldb, int64_t sB, void* C, int64_t ldc,
                              int64_t sC, int64_t batch, int grid_cap, cudaStream_t st) {
  FixedSrc src;
  src.A = static_cast<const double*>(A);
  src.B = static_cast<const double*>(B);
  src.C = static_cast<double*>(C);
  src.m = (int)m; src.n = (int)n; src.k = (int)k;
  src.lda = lda; src.ldb = ldb; src.ldc = ldc;
  src.sA = sA; src.sB = sB; src.sC = sC;
  src.esz = dt == BG_C128 ? 2 : 1;
  FixedSched sched;
  sched.prog = prog;
  prog_tile(prog, &sched.tm, &sched.tn);
  sched.batch = batch;
  int64_t n_items;
  int64_t grid = (int64_t)sm_count() * fp64_blocks_per_sm(dt);
  if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
  sched.g = kSmallPerCta;
  if (sched.tm == 0) {
    // the real small program spreads small batches over more CTAs
    if (prog == PROG_R64_SMALL) sched.g = small_group(batch, grid);
    sched.tiles_m = sched.tiles_n = 1;
    n_items = (batch + sched.g - 1) / sched.g;
  } else {
    sched.tiles_m = (m + sched.tm - 1) / sched.tm;
    sched.tiles_n = (n + sched.tn - 1) / sched.tn;
    n_items = batch * sched.tiles_m * sched.tiles_n;
  }
  if (n_items <= 0) return cudaSuccess;
  if (grid > n_items) grid = n_items;
  fp64_persistent<FixedSrc, FixedSched><<<(unsigned)grid, kFp64Threads, 0, st>>>(src, sched,
                                                                                 n_items, s);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_fp64_table(bg_dtype dt, const int64_t* d_table, const int32_t* d_order,
                              const WorkItem* d_items, int64_t n_items, const void* A,
                              const void* B, void* C, const Scalars& s, int grid,
                              cudaStream_t st, bool herm) {
  if (n_items <= 0) return cudaSuccess;
  TableSrc src;
  src.herm = herm ? 1 : 0;
  src.table = d_table;
  src.order = d_order;
  src.A = static_cast<const double*>(A);
  src.B = static_cast<const double*>(B);
  src.C = static_cast<double*>(C);
  src.esz = dt == BG_C128 ? 2 : 1;
  TableSched sched{d_items};
  if (grid <= 0) grid = sm_count() * fp64_blocks_per_sm(dt);
  if (grid > n_items) grid = (int)n_items;
  fp64_persistent<TableSrc, TableSched><<<grid, kFp64Threads, 0, st>>>(src, sched, n_items, s);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_fp64_chain(bg_dtype dt, const int64_t* d_wn, const int64_t* d_woff,
                              const int64_t* d_pool_off, const int64_t* d_pool_n,
                              int32_t pool_count, const int32_t* d_order,
                              const int32_t* d_idx_row, const WorkItem* d_items, int64_t n_items,
                              const void* U, const void* Cin, void* Cout, int grid,
                              cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  ChainSrc src;
  src.wn = d_wn;
  src.woff = d_woff;
  src.pool_off = d_pool_off;
  src.pool_n = d_pool_n;
  src.pool_count = pool_count;
  src.order = d_order;
  src.idx = d_idx_row;
  src.U = static_cast<const double*>(U);
  src.Cin = static_cast<const double*>(Cin);
  src.Cout = static_cast<double*>(Cout);
  src.esz = dt == BG_C128 ? 2 : 1;
  Scalars s;
  s.alpha_re = 1.0; s.alpha_im = 0.0; s.beta_re = 0.0; s.beta_im = 0.0;
  s.alpha_zero = 0; s.beta_zero = 1;
  TableSched sched{d_items};
  if (grid <= 0) grid = sm_count() * fp64_blocks_per_sm(dt);
  if (grid > n_items) grid = (int)n_items;
  fp64_persistent<ChainSrc, TableSched><<<grid, kFp64Threads, 0, st>>>(src, sched, n_items, s);
  count_launch();
  return cudaGetLastError();
}

}  // namespace bg
