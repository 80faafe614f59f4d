// Entanglement entropy of a batch of states (Alg. 1, "Calculate Entropy";
// Sec. 3): for each walker, the K x K Gram matrix G = X X^H of the state seen
// as the column-major K x M matrix X (K = 2^split rows: the lower spins), whose
// nonzero eigenvalues are those of rho = Psi Psi^H; then p_i = lambda_i /
// sum(lambda) and S = -sum p_i ln p_i.
//
// G comes from the library's Hermitian rank-k update (a grouped plan with
// BG_PLAN_HERK, FP64 or split precision), lower triangle. Then, one CTA per
// walker (one SM each):
//  * the Householder reduction of G to a real symmetric tridiagonal matrix
//    (d, e) in FP64, the steps of LAPACK's zhetd2 for the lower triangle:
//    for column j, the reflector H = I - tau v v^H that maps G[j+1:, j] to
//    (beta, 0, ..., 0) (beta real), then G22 <- G22 - v w^H - w v^H with
//    p = tau G22 v, w = p - (tau/2)(p^H v) v. tridiag_kernel runs it column
//    by column on the lower triangle; tridiag_small_kernel does the same
//    for K <= 64 (and the blocked path's last 64 columns) in shared memory.
//    Split-precision plans with K > 64 take the blocked form (zlatrd's
//    steps): tri_panel_kernel reduces 16 columns at a time, keeping their
//    rank-2 updates as [V W], and the trailing update C -= [V W][W V]^H
//    runs as a grouped GEMM in the plan's precision between panels.
//  * bisect_kernel: every eigenvalue of the tridiagonal matrix by bisection
//    on the Sturm count (the number of eigenvalues below x), one thread per
//    eigenvalue, then the entropy by a block reduction.
// All of these are bound by the FP64 pipe (about 2 DFMA per clock per SM on
// this part), not by memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>

#include "bgemm_internal.h"

namespace bg {
namespace {

constexpr int kEntThreads = 256;  // bisection
// Warps per walker of the two reductions. Measured at K = 256 (128
// walkers): 8 warps beat 4, 12 and 16 in both (the tiled product holds 32
// column sums per lane, about 196 registers).
constexpr int kRedWarps = 8;
constexpr int kPanelWarps = 8;
constexpr int kPanelMax = 64;  // widest panel of the blocked reduction

// A kernel's dynamic shared-memory limit is a property of the device: set it
// once per device (at every call for ordinals beyond the table).
constexpr int kAttrDevices = 64;
template <typename Kernel>
cudaError_t smem_limit(Kernel kernel, int bytes, bool (&done)[kAttrDevices]) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool tracked = dev >= 0 && dev < kAttrDevices;
  if (tracked && done[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && tracked) done[dev] = true;
  return e;
}

struct Z {
  double re, im;
};
__device__ __forceinline__ Z zmul(Z a, Z b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ Z zadd(Z a, Z b) { return {a.re + b.re, a.im + b.im}; }

// Sum of v over the block (all threads call it; the result reaches every thread).
// red: one double per warp.
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();  // red[] may still be read by a previous call
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];  // fixed order: same value in every thread
  return s;
}

// Sums of a and b over the block at once (one pair of barriers); red: one
// double2 per warp.
__device__ void block_sum2(double& a, double& b, double2* red) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
    b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = make_double2(a, b);
  __syncthreads();
  a = 0.0;
  b = 0.0;
  for (int i = 0; i < nw; ++i) {
    a += red[i].x;
    b += red[i].y;
  }
}

__device__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = red[0];
  for (int i = 1; i < nw; ++i) s = fmax(s, red[i]);
  return s;
}

// acc + a b and acc + conj(a) b as four FP64 fused multiply-adds each
__device__ __forceinline__ Z zfma(Z a, Z b, Z acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
__device__ __forceinline__ Z zfma_conj(Z a, Z b, Z acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}


// Partial products of y = A v for the m x m Hermitian matrix A (lower
// triangle, leading dimension ld; the upper triangle is never read): warp w
// adds its share into part[w m + i], which must be zero on entry, so that y
// is the sum over the warps. The lower triangle is cut into stripes of
// TJ = 32 columns, and each stripe into 32 x 32 tiles whose rows start at
// the stripe's diagonal. A lane takes one row i of a tile: it adds
// A[i, j] v[j] over the tile's columns into its row's sum (stored once per
// tile), and conj(A[i, j]) v[i] into one accumulator per column j. The tiles,
// in stripe order, are dealt to the warps in equal contiguous runs; a warp
// forms its column sums over the lanes when it leaves a stripe, by a
// butterfly in which each step halves the values a lane keeps (31 complex
// additions for the 32 columns), so that the FP64 pipe spends almost all
// its issue slots on the products.
template <int WARPS>
__device__ __forceinline__ void herm_matvec(const double2* A, int ld, int m, const Z* v, Z* part) {
  constexpr int TJ = 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = (m + TJ - 1) / TJ;
  auto chunks = [&](int s) { return (m - TJ * s + 31) >> 5; };  // tiles of stripe s
  int total = 0;
  for (int s = 0; s < S; ++s) total += chunks(s);
  const int t0 = (int)((int64_t)total * warp / WARPS);
  const int t1 = (int)((int64_t)total * (warp + 1) / WARPS);
  if (t0 >= t1) return;
  int s = 0, first = 0;
  while (first + chunks(s) <= t0) first += chunks(s++);
  int k = t0 - first;
  Z* pw = part + warp * m;
  Z acc[TJ];
#pragma unroll
  for (int jj = 0; jj < TJ; ++jj) acc[jj] = {0.0, 0.0};
  for (int tile = t0; tile < t1; ++tile) {
    const int j0 = TJ * s, i0 = j0 + 32 * k;
    const int i = i0 + lane;
    const bool row_ok = i < m;
    const Z vi = row_ok ? v[i] : Z{0.0, 0.0};
    const double2* arow = A + i + (size_t)j0 * ld;
    Z y0 = {0.0, 0.0}, y1 = {0.0, 0.0};
    if (i0 > j0 && i0 + 32 <= m) {  // a whole tile below the diagonal
#pragma unroll
      for (int jj = 0; jj < TJ; ++jj) {
        const double2 a2 = arow[(size_t)jj * ld];
        const Z a = {a2.x, a2.y};
        if (jj & 1) y1 = zfma(a, v[j0 + jj], y1);
        else y0 = zfma(a, v[j0 + jj], y0);
        acc[jj] = zfma_conj(a, vi, acc[jj]);
      }
    } else {  // the diagonal tile, or the ragged last one
#pragma unroll
      for (int jj = 0; jj < TJ; ++jj) {
        const int j = j0 + jj;
        Z a = {0.0, 0.0};
        if (row_ok && j < m && i >= j) {
          const double2 a2 = arow[(size_t)jj * ld];
          a = {a2.x, a2.y};
        }
        const Z vj = j < m ? v[j] : Z{0.0, 0.0};
        if (jj & 1) y1 = zfma(a, vj, y1);
        else y0 = zfma(a, vj, y0);
        const Z at = i > j ? a : Z{0.0, 0.0};
        acc[jj] = zfma_conj(at, vi, acc[jj]);
      }
    }
    if (row_ok) pw[i] = zadd(pw[i], zadd(y0, y1));
    if (++k == chunks(s) || tile + 1 == t1) {
      // lane l ends with the sum over the lanes of acc[l]: at the step of
      // offset o, a lane whose bit o is set keeps the upper half of its live
      // accumulators and receives its partner's upper half
#pragma unroll
      for (int o = TJ / 2; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int kk = 0; kk < o; ++kk) {
          const Z send = up ? acc[kk] : acc[kk + o];
          const Z keep = up ? acc[kk + o] : acc[kk];
          Z recv;
          recv.re = __shfl_xor_sync(0xFFFFFFFFu, send.re, o);
          recv.im = __shfl_xor_sync(0xFFFFFFFFu, send.im, o);
          acc[kk] = zadd(keep, recv);
        }
      }
      __syncwarp();
      if (j0 + lane < m) pw[j0 + lane] = zadd(pw[j0 + lane], acc[0]);
      __syncwarp();
#pragma unroll
      for (int jj = 0; jj < TJ; ++jj) acc[jj] = {0.0, 0.0};
      ++s;
      k = 0;
    }
  }
}

// Householder tridiagonalisation of n x n Hermitian matrices: for walker w,
// rows and columns off .. off + n - 1 of its ld x ld matrix at G + w ld ld
// (lower triangle, column-major; only the lower triangle is read or
// written). Writes d[w ld + off + i] (diagonal) and e[w ld + off + i]
// (sub-diagonal, i < n - 1; e of the last row is set to 0). The product
// p = G22 v comes from herm_matvec; the rank-2 update then rewrites the lower
// triangle, a warp per column with its lanes down the column (coalesced).
// Dynamic shared memory: v, w and the warps' partial products, (2 + WARPS) n
// complex.
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) tridiag_kernel(double2* G, int n, int ld, int off,
                                                             double* d, double* e) {
  constexpr int kEntWarps = WARPS;
  extern __shared__ double2 sm[];
  Z* v = reinterpret_cast<Z*>(sm);
  Z* w = v + n;
  Z* part = w + n;  // kEntWarps x n
  __shared__ double red[kEntWarps];
  __shared__ double2 red2[kEntWarps];
  __shared__ double s_beta, s_tau_re, s_tau_im, s_sc_re, s_sc_im;
  __shared__ int s_skip;
  double2* A = G + (size_t)blockIdx.x * ld * ld + off + (size_t)off * ld;
  double* dw = d + (size_t)blockIdx.x * ld + off;
  double* ew = e + (size_t)blockIdx.x * ld + off;
  const int t = threadIdx.x, T = blockDim.x, warp = t >> 5, lane = t & 31;
  auto at = [&](int r, int c) -> double2& { return A[r + (size_t)c * ld]; };

  for (int j = 0; j < n - 1; ++j) {
    const int m = n - j - 1;  // order of the trailing matrix G22 = A[j+1:, j+1:]
    double2* A22 = A + (j + 1) + (size_t)(j + 1) * ld;
    // ---- reflector of the column below the diagonal (zlarfg)
    double xn2 = 0.0;
    for (int i = 1 + t; i < m; i += T) {
      const double2 x = at(j + 1 + i, j);
      xn2 = fma(x.x, x.x, fma(x.y, x.y, xn2));
    }
    xn2 = block_sum(xn2, red);
    if (t == 0) {
      const double2 a = at(j + 1, j);
      dw[j] = at(j, j).x;
      if (xn2 == 0.0 && a.y == 0.0) {
        s_skip = 1;  // already reduced: H = I
        s_beta = a.x;
      } else {
        s_skip = 0;
        const double beta = -copysign(sqrt(a.x * a.x + a.y * a.y + xn2), a.x);
        s_beta = beta;
        const double rb = 1.0 / beta;
        s_tau_re = (beta - a.x) * rb;
        s_tau_im = -a.y * rb;
        // 1 / (alpha - beta)
        const double dr = a.x - beta, di = a.y, rden = 1.0 / (dr * dr + di * di);
        s_sc_re = dr * rden;
        s_sc_im = -di * rden;
      }
      ew[j] = s_beta;
    }
    __syncthreads();
    if (s_skip) continue;
    const Z tau = {s_tau_re, s_tau_im}, sc = {s_sc_re, s_sc_im};
    for (int i = t; i < m; i += T) {
      Z vi = {1.0, 0.0};
      if (i > 0) {
        const double2 x = at(j + 1 + i, j);
        vi = zmul({x.x, x.y}, sc);
      }
      v[i] = vi;
    }
    for (int i = t; i < kEntWarps * m; i += T) part[i] = {0.0, 0.0};
    __syncthreads();
    // ---- partial products of p = G22 v from the lower triangle
    herm_matvec<kEntWarps>(A22, ld, m, v, part);
    __syncthreads();
    // ---- p = tau sum of the partials, alpha2 = -tau/2 (p^H v), w = p + alpha2 v
    double pr = 0.0, pi_ = 0.0;
    for (int i = t; i < m; i += T) {
      Z acc = {0.0, 0.0};
#pragma unroll
      for (int q = 0; q < kEntWarps; ++q) acc = zadd(acc, part[q * m + i]);
      const Z p = zmul(tau, acc);
      w[i] = p;
      const Z pv = zfma_conj(p, v[i], {0.0, 0.0});
      pr += pv.re;
      pi_ += pv.im;
    }
    block_sum2(pr, pi_, red2);
    const Z alpha2 = zmul({-0.5 * tau.re, -0.5 * tau.im}, {pr, pi_});
    for (int i = t; i < m; i += T) w[i] = zfma(alpha2, v[i], w[i]);
    __syncthreads();
    // ---- G22 <- G22 - v w^H - w v^H on the lower triangle, a warp per column
    for (int c = warp; c < m; c += kEntWarps) {
      double2* col = A22 + (size_t)c * ld;
      const Z wc = {-w[c].re, w[c].im}, vc = {-v[c].re, v[c].im};  // -conj(w[c]), -conj(v[c])
      for (int i = c + lane; i < m; i += 32) {
        Z a = {col[i].x, col[i].y};
        a = zfma(v[i], wc, a);
        a = zfma(w[i], vc, a);
        col[i] = make_double2(a.re, a.im);
      }
    }
    __syncthreads();
  }
  if (t == 0) {
    dw[n - 1] = at(n - 1, n - 1).x;
    ew[n - 1] = 0.0;
  }
}

// Partial products of y = A v for an m x m complex matrix stored in full
// (leading dimension ld), with S = Re A + Im A beside it (same layout) and
// vs = Re v + Im v: three real products per element instead of four,
//   Re y = sum Re A Re v - sum Im A Im v,
//   Im y = sum S vs - sum Re A Re v - sum Im A Im v
// (Gauss's form; its error is bounded normwise, c u |A| |v| with a small c,
// which is what the reduction's backward stability needs). Warp w takes the
// columns m w / W .. m (w + 1) / W - 1 and writes its share of every row
// i < m to part[w m + i], so that y is the sum over the warps. A lane takes
// the rows lane, lane + 32, ... (up to kDenseRows of them at a time,
// independent sums), down each column; the next column's elements are
// loaded while the current one is multiplied, so that the memory latency
// overlaps the FP64 work.
constexpr int kDenseRows = 8;
template <int WARPS>
__device__ __forceinline__ void dense_matvec(const double2* A, const double* S, int ld, int m,
                                             const Z* v, const double* vs, Z* part) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j0 = m * warp / WARPS, j1 = m * (warp + 1) / WARPS;
  Z* pw = part + warp * m;
  for (int r0 = 0; r0 < m; r0 += 32 * kDenseRows) {
    double t1[kDenseRows], t2[kDenseRows], t3[kDenseRows];
    double2 na[kDenseRows];
    double ns[kDenseRows];
#pragma unroll
    for (int c = 0; c < kDenseRows; ++c) {
      t1[c] = t2[c] = t3[c] = 0.0;
      na[c] = make_double2(0.0, 0.0);
      ns[c] = 0.0;
    }
    const double2* abase = A + r0 + lane;
    const double* sbase = S + r0 + lane;
    auto fetch = [&](int j) {
      const double2* acol = abase + (size_t)j * ld;
      const double* scol = sbase + (size_t)j * ld;
#pragma unroll
      for (int c = 0; c < kDenseRows; ++c)
        if (r0 + 32 * c + lane < m) {
          na[c] = acol[32 * c];
          ns[c] = scol[32 * c];
        }
    };
    if (j0 < j1) fetch(j0);
    for (int j = j0; j < j1; ++j) {
      double2 ca[kDenseRows];
      double cs[kDenseRows];
#pragma unroll
      for (int c = 0; c < kDenseRows; ++c) {
        ca[c] = na[c];
        cs[c] = ns[c];
      }
      if (j + 1 < j1) fetch(j + 1);
      const Z vj = v[j];
      const double vsj = vs[j];
#pragma unroll
      for (int c = 0; c < kDenseRows; ++c) {
        t1[c] = fma(ca[c].x, vj.re, t1[c]);
        t2[c] = fma(ca[c].y, vj.im, t2[c]);
        t3[c] = fma(cs[c], vsj, t3[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < kDenseRows; ++c)
      if (r0 + 32 * c + lane < m)
        pw[r0 + 32 * c + lane] = {t1[c] - t2[c], t3[c] - t1[c] - t2[c]};
  }
}

// The unblocked reduction for n <= kSmallRed with the matrix held in shared
// memory: the same steps as tridiag_kernel (rows and columns off .. off +
// n - 1 of walker w's ld x ld matrix, lower triangle; d and e as there), a
// CTA of 256 threads per walker. The Hermitian product gives each row four
// threads (a quarter of the columns each, summed by two shuffles); the
// rank-2 update gives each thread the rows r and m - 1 - r of one in eight
// columns, so that every thread holds the same number of elements. The
// global matrix is only read.
constexpr int kSmallRed = 64;
constexpr int kSmallLd = kSmallRed + 1;  // shared-memory leading dimension
__global__ void __launch_bounds__(256) tridiag_small_kernel(const double2* G, int n, int ld,
                                                            int off, double* d, double* e) {
  extern __shared__ double2 sm_small[];  // kSmallRed x kSmallLd complex
  Z* As = reinterpret_cast<Z*>(sm_small);
  __shared__ Z v[kSmallRed], w[kSmallRed];
  __shared__ double red[8];
  __shared__ double2 red2[8];
  __shared__ double s_beta, s_tau_re, s_tau_im, s_sc_re, s_sc_im;
  __shared__ int s_skip;
  const double2* A = G + (size_t)blockIdx.x * ld * ld + off + (size_t)off * ld;
  double* dw = d + (size_t)blockIdx.x * ld + off;
  double* ew = e + (size_t)blockIdx.x * ld + off;
  const int t = threadIdx.x, T = blockDim.x;
  for (int idx = t; idx < n * n; idx += T) {
    const int r = idx % n, c = idx / n;
    if (r >= c) {
      const double2 x = A[r + (size_t)c * ld];
      As[r + c * kSmallLd] = {x.x, x.y};
    }
  }
  __syncthreads();
  auto at = [&](int r, int c) -> Z& { return As[r + c * kSmallLd]; };
  for (int j = 0; j < n - 1; ++j) {
    const int m = n - j - 1;
    const int b0 = j + 1;  // first row and column of G22
    double xn2 = 0.0;
    for (int i = 1 + t; i < m; i += T) {
      const Z x = at(b0 + i, j);
      xn2 = fma(x.re, x.re, fma(x.im, x.im, xn2));
    }
    xn2 = block_sum(xn2, red);
    if (t == 0) {
      const Z a = at(b0, j);
      dw[j] = at(j, j).re;
      if (xn2 == 0.0 && a.im == 0.0) {
        s_skip = 1;
        s_beta = a.re;
      } else {
        s_skip = 0;
        const double beta = -copysign(sqrt(a.re * a.re + a.im * a.im + xn2), a.re);
        s_beta = beta;
        const double rb = 1.0 / beta;
        s_tau_re = (beta - a.re) * rb;
        s_tau_im = -a.im * rb;
        const double dr = a.re - beta, di = a.im, rden = 1.0 / (dr * dr + di * di);
        s_sc_re = dr * rden;
        s_sc_im = -di * rden;
      }
      ew[j] = s_beta;
    }
    __syncthreads();
    if (s_skip) continue;
    const Z tau = {s_tau_re, s_tau_im}, sc = {s_sc_re, s_sc_im};
    for (int i = t; i < m; i += T) v[i] = i == 0 ? Z{1.0, 0.0} : zmul(at(b0 + i, j), sc);
    __syncthreads();
    // p = G22 v: row r, a quarter q of the columns
    const int r = t >> 2, q = t & 3;
    Z y = {0.0, 0.0};
    if (r < m) {
      for (int cc = q; cc < m; cc += 4) {
        if (cc <= r) y = zfma(at(b0 + r, b0 + cc), v[cc], y);
        else y = zfma_conj(at(b0 + cc, b0 + r), v[cc], y);
      }
    }
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
      y.re += __shfl_xor_sync(0xFFFFFFFFu, y.re, o);
      y.im += __shfl_xor_sync(0xFFFFFFFFu, y.im, o);
    }
    double pr = 0.0, pi_ = 0.0;
    Z p = {0.0, 0.0};
    if (r < m && q == 0) {
      p = zmul(tau, y);
      const Z pv = zfma_conj(p, v[r], {0.0, 0.0});
      pr = pv.re;
      pi_ = pv.im;
    }
    block_sum2(pr, pi_, red2);
    const Z alpha2 = zmul({-0.5 * tau.re, -0.5 * tau.im}, {pr, pi_});
    if (r < m && q == 0) w[r] = zfma(alpha2, v[r], p);
    __syncthreads();
    // G22 <- G22 - v w^H - w v^H on the lower triangle: thread (pair h,
    // column group g) takes rows h and m - 1 - h, columns g, g + 8, ... up to
    // the row
    const int h = t & 31, g = t >> 5;
    for (int s = 0; s < 2; ++s) {
      const int rr = s == 0 ? h : m - 1 - h;
      if (h > m - 1 - h || (s == 1 && rr == h)) continue;  // the pair's lower row takes both
      const Z vr = v[rr], wr = w[rr];
      for (int cc = g; cc <= rr; cc += 8) {
        const Z wc = {-w[cc].re, w[cc].im}, vc = {-v[cc].re, v[cc].im};
        Z a = at(b0 + rr, b0 + cc);
        a = zfma(vr, wc, a);
        a = zfma(wr, vc, a);
        at(b0 + rr, b0 + cc) = a;
      }
    }
    __syncthreads();
  }
  if (t == 0) {
    dw[n - 1] = at(n - 1, n - 1).re;
    ew[n - 1] = 0.0;
  }
}

// ---- blocked reduction (panels of nb columns; the trailing rank-2nb update
// runs as a batched GEMM on the tensor-core split path, see batched_entropy)
//
// One panel of the Householder reduction of each walker's G (lower triangle,
// leading dimension n), columns c = p0 .. p0 + nbp - 1. The panel's rank-2
// updates are not applied to the trailing matrix; they are kept as the
// columns of V and W (walker w's V at P + w pstride, its W nbp columns
// further, column t at + t n, rows below the column's diagonal), so that
// [V W] is the first operand of the trailing update. For column c of the
// panel:
//  (a) column c (rows c..n-1) first receives this panel's earlier updates,
//      A[r, c] -= sum_t V[r, t] conj(W[c, t]) + W[r, t] conj(V[c, t]);
//  (b) the reflector of A[c+1:, c] gives d[c], e[c], tau and v, as in the
//      unblocked kernel;
//  (c) y = A22 v from the trailing matrix as it is in memory, corrected by
//      the panel's earlier updates: y -= V2 (W2^H v) + W2 (V2^H v). The
//      blocked path keeps both triangles of the trailing matrix (the Gram
//      matrix is mirrored once, and the trailing updates write whole
//      squares), so that this product runs over the full matrix;
//  (d) w = tau y - (tau / 2) (w^H v) v is stored with v.
// The panel ends before the matrix does (p0 + nbp <= n - 1), so every
// column of it has rows below its diagonal.
template <int WARPS, bool VWS>
__global__ void __launch_bounds__(WARPS * 32) tri_panel_kernel(double2* G, const double* Sg, int n,
                                                               int p0, int nbp, double2* P,
                                                               int64_t pstride, double* d,
                                                               double* e) {
  extern __shared__ double2 sm[];
  Z* v = reinterpret_cast<Z*>(sm);
  Z* y = v + n;
  double* vs = reinterpret_cast<double*>(y);  // Re v + Im v, while y is not in use
  Z* part = y + n;  // WARPS x n
  __shared__ Z s1[kPanelMax], s2[kPanelMax];
  __shared__ double red[WARPS];
  __shared__ double2 red2[WARPS];
  __shared__ double s_beta, s_tau_re, s_tau_im, s_sc_re, s_sc_im;
  __shared__ int s_skip;
  double2* A = G + (size_t)blockIdx.x * n * n;
  double2* V = P + (size_t)blockIdx.x * pstride;
  double2* W = V + (size_t)nbp * n;
  // the panel's V and W as the corrections read them: a copy of rows
  // p0 .. n-1 in shared memory (VWS), else the global arrays themselves
  const int ldl = VWS ? n - p0 : n, rb = VWS ? p0 : 0;
  double2* Vl = VWS ? reinterpret_cast<double2*>(part + WARPS * n) : V;
  double2* Wl = VWS ? Vl + (size_t)nbp * ldl : W;
  auto vl = [&](int q, int r) -> double2& { return Vl[(size_t)q * ldl + r - rb]; };
  auto wl = [&](int q, int r) -> double2& { return Wl[(size_t)q * ldl + r - rb]; };
  double* dw = d + (size_t)blockIdx.x * n;
  double* ew = e + (size_t)blockIdx.x * n;
  const int t = threadIdx.x, T = blockDim.x, warp = t >> 5, lane = t & 31;
  auto at = [&](int r, int c) -> double2& { return A[r + (size_t)c * n]; };
  for (int i = 0; i < nbp; ++i) {
    const int c = p0 + i;
    const int m = n - c - 1;  // rows below the diagonal
    // ---- (a) this panel's earlier rank-2 updates, applied to column c,
    // with the squared norm of its rows c+2.. for the reflector
    double xn2 = 0.0;
    if (i > 0) {
      for (int r = c + t; r < n; r += T) {
        Z a = {at(r, c).x, at(r, c).y}, b = {0.0, 0.0};  // two independent sums
#pragma unroll 4
        for (int q = 0; q < i; ++q) {
          const double2 vr = vl(q, r), wr = wl(q, r), wc = wl(q, c), vc = vl(q, c);
          a = zfma({-vr.x, -vr.y}, {wc.x, -wc.y}, a);
          b = zfma({-wr.x, -wr.y}, {vc.x, -vc.y}, b);
        }
        const double2 x = make_double2(a.re + b.re, a.im + b.im);
        at(r, c) = x;
        if (r >= c + 2) xn2 = fma(x.x, x.x, fma(x.y, x.y, xn2));
      }
    } else {
      for (int r = c + 2 + t; r < n; r += T) {
        const double2 x = at(r, c);
        xn2 = fma(x.x, x.x, fma(x.y, x.y, xn2));
      }
    }
    // ---- (b) reflector of the column below the diagonal (the block sum's
    // barriers also publish column c)
    xn2 = block_sum(xn2, red);
    if (t == 0) {
      const double2 a = at(c + 1, c);
      dw[c] = at(c, c).x;
      if (xn2 == 0.0 && a.y == 0.0) {
        s_skip = 1;
        s_beta = a.x;
      } else {
        s_skip = 0;
        const double beta = -copysign(sqrt(a.x * a.x + a.y * a.y + xn2), a.x);
        s_beta = beta;
        const double rb = 1.0 / beta;
        s_tau_re = (beta - a.x) * rb;
        s_tau_im = -a.y * rb;
        const double dr = a.x - beta, di = a.y, rden = 1.0 / (dr * dr + di * di);
        s_sc_re = dr * rden;
        s_sc_im = -di * rden;
      }
      ew[c] = s_beta;
    }
    __syncthreads();
    if (s_skip) {  // H = I: v = w = 0 for this column
      for (int r = c + 1 + t; r < n; r += T) {
        V[(size_t)i * n + r] = make_double2(0.0, 0.0);
        W[(size_t)i * n + r] = make_double2(0.0, 0.0);
        if (VWS) vl(i, r) = wl(i, r) = make_double2(0.0, 0.0);
      }
      __syncthreads();
      continue;
    }
    const Z tau = {s_tau_re, s_tau_im}, sc = {s_sc_re, s_sc_im};
    for (int ii = t; ii < m; ii += T) {
      Z vi = {1.0, 0.0};
      if (ii > 0) {
        const double2 x = at(c + 1 + ii, c);
        vi = zmul({x.x, x.y}, sc);
      }
      v[ii] = vi;
      vs[ii] = vi.re + vi.im;
    }
    __syncthreads();
    // ---- (c) y = A22 v over the full trailing matrix, after the
    // corrections' coefficients W2^H v and V2^H v (a warp per panel column)
    for (int q = warp; q < i; q += WARPS) {
      Z a1 = {0.0, 0.0}, a2 = {0.0, 0.0};
      for (int ii = lane; ii < m; ii += 32) {
        const double2 wr = wl(q, c + 1 + ii), vr = vl(q, c + 1 + ii);
        a1 = zfma_conj({wr.x, wr.y}, v[ii], a1);
        a2 = zfma_conj({vr.x, vr.y}, v[ii], a2);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a1.re += __shfl_xor_sync(0xFFFFFFFFu, a1.re, o);
        a1.im += __shfl_xor_sync(0xFFFFFFFFu, a1.im, o);
        a2.re += __shfl_xor_sync(0xFFFFFFFFu, a2.re, o);
        a2.im += __shfl_xor_sync(0xFFFFFFFFu, a2.im, o);
      }
      if (lane == 0) {
        s1[q] = a1;
        s2[q] = a2;
      }
    }
    dense_matvec<WARPS>(A + (c + 1) + (size_t)(c + 1) * n,
                        Sg + (size_t)blockIdx.x * n * n + (c + 1) + (size_t)(c + 1) * n, n, m, v,
                        vs, part);
    __syncthreads();
    // ---- (d) w = tau (y - V2 s1 - W2 s2), alpha2 = -tau/2 (w^H v), w += alpha2 v
    double pr = 0.0, pi_ = 0.0;
    for (int ii = t; ii < m; ii += T) {
      Z acc = {0.0, 0.0};
#pragma unroll
      for (int q = 0; q < WARPS; ++q) acc = zadd(acc, part[q * m + ii]);
      const int r = c + 1 + ii;
      Z acc2 = {0.0, 0.0};
#pragma unroll 4
      for (int q = 0; q < i; ++q) {
        const double2 vr = vl(q, r), wr = wl(q, r);
        acc = zfma({-vr.x, -vr.y}, s1[q], acc);
        acc2 = zfma({-wr.x, -wr.y}, s2[q], acc2);
      }
      acc = zadd(acc, acc2);
      const Z p = zmul(tau, acc);
      y[ii] = p;
      const Z pv = zfma_conj(p, v[ii], {0.0, 0.0});
      pr += pv.re;
      pi_ += pv.im;
    }
    block_sum2(pr, pi_, red2);
    const Z alpha2 = zmul({-0.5 * tau.re, -0.5 * tau.im}, {pr, pi_});
    for (int ii = t; ii < m; ii += T) {
      const Z wv = zfma(alpha2, v[ii], y[ii]);
      W[(size_t)i * n + c + 1 + ii] = make_double2(wv.re, wv.im);
      V[(size_t)i * n + c + 1 + ii] = make_double2(v[ii].re, v[ii].im);
      if (VWS) {
        wl(i, c + 1 + ii) = make_double2(wv.re, wv.im);
        vl(i, c + 1 + ii) = make_double2(v[ii].re, v[ii].im);
      }
    }
    __syncthreads();
  }
}

// Copies the lower triangle of every walker's n x n matrix into its upper
// triangle, A[j, i] = conj(A[i, j]) for i > j, a 32 x 32 tile per block
// (blockIdx.x = tile of the lower triangle in row order, blockIdx.y =
// walker) through shared memory, so that reads and writes are coalesced.
__global__ void __launch_bounds__(256) tri_mirror_kernel(double2* G, double* Sg, int n) {
  __shared__ double2 tile[32][33];
  int idx = blockIdx.x, bi = 0;
  while (idx > bi) idx -= ++bi;  // tile row bi holds bi + 1 tiles
  const int bj = idx, i0 = 32 * bi, j0 = 32 * bj;
  double2* A = G + (size_t)blockIdx.y * n * n;
  double* S = Sg + (size_t)blockIdx.y * n * n;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int k = ty; k < 32; k += 8) {
    const int r = i0 + tx, c = j0 + k;
    if (r < n && c < n) {
      const double2 x = A[r + (size_t)c * n];
      tile[k][tx] = x;
      if (r >= c) S[r + (size_t)c * n] = x.x + x.y;
    }
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int r = j0 + tx, c = i0 + k;  // (r, c) above the diagonal takes conj(A[c, r])
    if (r < n && c < n && c > r) {
      const double2 x = tile[tx][k];
      A[r + (size_t)c * n] = make_double2(x.x, -x.y);
      S[r + (size_t)c * n] = x.x - x.y;
    }
  }
}

// S = Re A + Im A on rows and columns q .. n-1 of every walker's matrix
// (after a trailing update), a thread per element, coalesced down columns.
__global__ void __launch_bounds__(256) tri_sum_kernel(const double2* G, double* Sg, int n, int q) {
  const int mt = n - q;
  const double2* A = G + (size_t)blockIdx.y * n * n + q + (size_t)q * n;
  double* S = Sg + (size_t)blockIdx.y * n * n + q + (size_t)q * n;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < mt * mt;
       idx += gridDim.x * blockDim.x) {
    const int r = idx % mt, c = idx / mt;
    const double2 x = A[r + (size_t)c * n];
    S[r + (size_t)c * n] = x.x + x.y;
  }
}

// The second operand of the trailing update C -= [V2 W2] [W2 V2]^H, where V2
// and W2 are rows q..n-1 of the panel's V and W (mt = n - q rows; the first
// operand is [V W] itself, rows from q, leading dimension n): WVh is
// 2 nbp x mt, column-major with leading dimension 2 nbp, walker w at
// w mt 2 nbp; WVh[t, r] = conj(W[q + r, t]) for t < nbp and
// conj(V[q + r, t - nbp]) above. A thread per (r, t) pair, t fastest, so
// that the stores are coalesced.
__global__ void tri_pack_kernel(const double2* P, int64_t pstride, int n, int q, int nbp,
                                double2* WVh) {
  const int mt = n - q, k2 = 2 * nbp;
  const size_t w = blockIdx.y;
  const double2* V = P + w * pstride;
  const double2* W = V + (size_t)nbp * n;
  double2* out = WVh + w * (size_t)mt * k2;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < mt * k2;
       idx += gridDim.x * blockDim.x) {
    const int tt = idx % k2, r = idx / k2;
    const double2 x = tt < nbp ? W[(size_t)tt * n + q + r] : V[(size_t)(tt - nbp) * n + q + r];
    out[idx] = make_double2(x.x, -x.y);
  }
}

// 1/q for a normal q: the hardware's approximate reciprocal, then two
// Newton-Raphson steps r <- r + r (1 - q r), each of which squares the
// relative error (to well below 2^-80, so r is within an ulp or so of 1/q).
// On this part an FP64 instruction is slow; this takes five of them where
// an IEEE division takes about twice as many.
__device__ __forceinline__ double recip_nr(double q) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(q));
  double e = fma(-q, r, 1.0);
  r = fma(r, e, r);
  e = fma(-q, r, 1.0);
  return fma(r, e, r);
}

// Number of eigenvalues of the symmetric tridiagonal (d, e2 = e^2) below x:
// the negative pivots of T - x I (a pivot smaller than pivmin in magnitude
// is replaced by -pivmin, as in LAPACK's dstebz). The pivot recurrence
// q_i = (d_i - x) - e2_{i-1} / q_{i-1} is backward stable: the count is exact
// for entries perturbed by a few ulps, which also covers a quotient formed
// with a reciprocal that is not correctly rounded. The sign and the pivmin
// test read the bit pattern (integer compares of |q|'s bits order like the
// magnitudes), so that they stay off the FP64 pipe.
__device__ __forceinline__ int sturm_count(const double* d, const double* e2, int n, double x,
                                           double pivmin) {
  const long long pmin_bits = __double_as_longlong(pivmin);
  const double neg_pmin = -pivmin;
  double q = d[0] - x;
  long long qb = __double_as_longlong(q);
  if ((qb & 0x7FFFFFFFFFFFFFFFll) < pmin_bits) {
    q = neg_pmin;
    qb = __double_as_longlong(q);
  }
  int cnt = (int)((unsigned long long)qb >> 63);
  for (int i = 1; i < n; ++i) {
    q = fma(-e2[i - 1], recip_nr(q), d[i] - x);
    qb = __double_as_longlong(q);
    if ((qb & 0x7FFFFFFFFFFFFFFFll) < pmin_bits) {
      q = neg_pmin;
      qb = __double_as_longlong(q);
    }
    cnt += (int)((unsigned long long)qb >> 63);
  }
  return cnt;
}

// The same count by the three-term recurrence of the leading principal
// minors, p_0 = 1, p_1 = d_0 - x, p_i = (d_{i-1} - x) p_{i-1} - e_{i-2}^2
// p_{i-2}: the number of sign changes along p_0 .. p_n is the number of
// negative pivots q_i = p_i / p_{i-1}, that is, of eigenvalues below x. No
// division: a DADD, a DMUL and a DFMA a step, with the sign and zero tests
// on the bit pattern. For the matrix scaled into [-1, 1] (|d - x| <= 3,
// e^2 <= 1) a step changes |p| by a factor of at most 4 upwards, and a
// cancellation leaves at least an ulp of its terms. A zero p_i is replaced
// by -2^-60 p_{i-1} (the pivot -2^-60, below an ulp of the scaled entries:
// the pivot form's rule for a zero pivot), an exact change of the sign and
// exponent. Every 8 steps p and p_{i-1} are rescaled together by 2^-500 or
// 2^500 when p's binary exponent has left [-500, 500]: in between, no p
// leaves the normal range, and no sign changes. Each step is exact for
// d - x and e^2 perturbed by a few ulps (the rounding factors of the p's
// cancel in the ratios), so the count is exact for a matrix within a few
// ulps of the scaled one.
__device__ __forceinline__ void sturm3_step(double dx, double e2, double& p, double& pm,
                                            long long& pb, int& neg, int& cnt) {
  const double pn = fma(-e2, pm, dx * p);
  long long nb = __double_as_longlong(pn);
  if ((nb << 1) == 0) nb = (pb ^ (long long)0x8000000000000000ull) - (60ll << 52);  // -2^-60 p
  const int s = (int)((unsigned long long)nb >> 63);
  cnt += s ^ neg;
  neg = s;
  pm = p;
  pb = nb;
  p = __longlong_as_double(nb);
}

__device__ __forceinline__ int sturm_count3(const double* d, const double* e2, int n, double x) {
  double pm = 1.0, p = d[0] - x;
  long long pb = __double_as_longlong(p);
  if ((pb << 1) == 0) pb = __double_as_longlong(-0x1p-60);
  p = __longlong_as_double(pb);
  int neg = (int)((unsigned long long)pb >> 63);
  int cnt = neg;
  int i = 1;
  for (; i + 8 <= n; i += 8) {
#pragma unroll 1
    for (int u = 0; u < 8; ++u) sturm3_step(d[i + u] - x, e2[i + u - 1], p, pm, pb, neg, cnt);
    const int ex = (int)((pb >> 52) & 0x7FF) - 1023;
    if (ex > 500) {
      p *= 0x1p-500;
      pm *= 0x1p-500;
      pb = __double_as_longlong(p);
    } else if (ex < -500) {
      p *= 0x1p500;
      pm *= 0x1p500;
      pb = __double_as_longlong(p);
    }
  }
  for (; i < n; ++i) sturm3_step(d[i] - x, e2[i - 1], p, pm, pb, neg, cnt);
  return cnt;
}

// The same recurrence in FP32 on the float copy of the scaled matrix, the
// rescaling by 2^-60 / 2^60 checked at every step and a zero p_i replaced
// by -2^-24 p_{i-1}. Its backward error, a few FP32 ulps of the scaled
// entries, stays below the 32 x 2^-24 by which the FP32 brackets are
// widened.
__device__ __forceinline__ int sturm_count3f(const float* d, const float* e2, int n, float x) {
  float pm = 1.0f, p = d[0] - x;
  if (p == 0.0f) p = -0x1p-24f;
  bool neg = p < 0.0f;
  int cnt = neg;
  for (int i = 1; i < n; ++i) {
    float pn = fmaf(-e2[i - 1], pm, (d[i] - x) * p);
    if (pn == 0.0f) pn = -0x1p-24f * p;
    const bool s = pn < 0.0f;
    cnt += s != neg;
    neg = s;
    pm = p;
    p = pn;
    const int ex = (int)((__float_as_uint(p) >> 23) & 0xFF) - 127;
    if (ex > 60) {
      p *= 0x1p-60f;
      pm *= 0x1p-60f;
    } else if (ex < -60) {
      p *= 0x1p60f;
      pm *= 0x1p60f;
    }
  }
  return cnt;
}

// Eigenvalues of each walker's tridiagonal matrix by bisection, then
// S = -sum p ln p with p = lambda / sum(lambda) over p > 0. The matrix is
// scaled by a power of two into [-1, 1] and counted by the three-term
// recurrence; the brackets are first narrowed in FP32: from there a bracket
// [a, b] with count32(a) <= k < count32(b) holds lambda_k within
// [a - del, b + del] (del = 32 x 2^-24, above the FP32 count's error
// bound), and FP64 bisection takes it on to the tolerance. That saves about
// 10 of the 45 FP64 Sturm counts per eigenvalue, and the recurrence halves
// the FP64 instructions of a count. Matrices whose scale lies outside
// [2^-1000, 2^1000] take the pivot form unscaled, in FP64 only. Dynamic
// shared memory: d, e^2 and the eigenvalues (3 n doubles), T + 1 int
// counts, then d and e^2 as scaled floats (2 n).
__global__ void __launch_bounds__(kEntThreads) bisect_kernel(const double* d, const double* e,
                                                             int n, double* entropy,
                                                             double* eigs) {
  extern __shared__ double sb[];
  double* sd = sb;
  double* se2 = sb + n;
  double* lam = sb + 2 * n;
  __shared__ double red[kEntThreads / 32];
  const int t = threadIdx.x, T = blockDim.x;
  const double* dw = d + (size_t)blockIdx.x * n;
  const double* ew = e + (size_t)blockIdx.x * n;
  double lo = DBL_MAX, hi = -DBL_MAX, e2max = 0.0;
  for (int i = t; i < n; i += T) {
    sd[i] = dw[i];
    const double ei = i + 1 < n ? ew[i] : 0.0;
    se2[i] = ei * ei;
    e2max = fmax(e2max, ei * ei);
    // Gershgorin interval of row i
    const double r = fabs(ei) + (i > 0 ? fabs(ew[i - 1]) : 0.0);
    lo = fmin(lo, dw[i] - r);
    hi = fmax(hi, dw[i] + r);
  }
  lo = -block_max(-lo, red);
  hi = block_max(hi, red);
  e2max = block_max(e2max, red);
  const double pivmin = DBL_MIN * fmax(1.0, e2max);
  const double scale = fmax(fabs(lo), fabs(hi));
  const double tol = 2.0 * DBL_EPSILON * scale + 2.0 * pivmin;
  lo -= tol;
  hi += tol;
  int* cnt = reinterpret_cast<int*>(lam + n);  // T + 1 counts
  float* d32 = reinterpret_cast<float*>(cnt + T + 1);
  float* e32 = d32 + n;
  int ex = 0;
  frexp(scale, &ex);
  const bool use32 = scale > 0x1p-1000 && scale < 0x1p1000;
  const double sc = ldexp(1.0, -ex);  // scale x sc in [0.5, 1)
  if (use32) {  // the scaled matrix, in place of d and e^2, and as floats
    for (int i = t; i < n; i += T) {
      sd[i] *= sc;
      const double es = (i + 1 < n ? ew[i] : 0.0) * sc;
      se2[i] = es * es;
      d32[i] = (float)sd[i];
      e32[i] = (float)se2[i];
    }
  }
  __syncthreads();
  // multisection: one Sturm count per thread on an even grid gives every
  // eigenvalue a bracket T times narrower to start from (the ends widened
  // by twice the FP32 bound, so that the counts there are 0 and n)
  const float del32 = 32.0f * 0x1p-24f;
  const float lo32 = (float)(lo * sc) - 2.0f * del32, hi32 = (float)(hi * sc) + 2.0f * del32;
  const float h32 = (hi32 - lo32) / (float)T;
  const double hstep = (hi - lo) / T;
  auto grid32 = [&](int j) { return __fmaf_rn((float)j, h32, lo32); };
  auto grid64 = [&](int j) { return fma((double)j, hstep, lo); };
  if (use32) cnt[t + 1] = t + 1 < T ? sturm_count3f(d32, e32, n, grid32(t + 1)) : n;
  else cnt[t + 1] = t + 1 < T ? sturm_count(sd, se2, n, grid64(t + 1), pivmin) : n;
  if (t == 0) cnt[0] = 0;
  __syncthreads();
  for (int k = t; k < n; k += T) {
    // the k-th smallest eigenvalue: count(a) <= k < count(b)
    int g = 0;  // a grid cell with cnt[g] <= k < cnt[g + 1]
    int lo_i = 0, hi_i = T;
    while (hi_i - lo_i > 1) {
      const int mid = (lo_i + hi_i) >> 1;
      if (cnt[mid] <= k) lo_i = mid;
      else hi_i = mid;
    }
    g = lo_i;
    double a, b;
    if (use32) {
      float a32 = grid32(g), b32 = g + 1 < T ? grid32(g + 1) : hi32;
      for (int it = 0; it < 40 && b32 - a32 > del32; ++it) {
        const float mid = 0.5f * (a32 + b32);
        if (sturm_count3f(d32, e32, n, mid) <= k) a32 = mid;
        else b32 = mid;
      }
      // in scaled units from here
      a = (double)a32 - (double)del32;
      b = (double)b32 + (double)del32;
      const double tol_s = tol * sc;
      for (int it = 0; it < 200 && b - a > tol_s; ++it) {
        const double mid = 0.5 * (a + b);
        if (sturm_count3(sd, se2, n, mid) <= k) a = mid;
        else b = mid;
      }
      lam[k] = 0.5 * (a + b) / sc;  // dividing by a power of two: exact
    } else {
      a = grid64(g);
      b = g + 1 < T ? grid64(g + 1) : hi;
      for (int it = 0; it < 200 && b - a > tol; ++it) {
        const double mid = 0.5 * (a + b);
        if (sturm_count(sd, se2, n, mid, pivmin) <= k) a = mid;
        else b = mid;
      }
      lam[k] = 0.5 * (a + b);
    }
  }
  __syncthreads();
  double tot = 0.0;
  for (int k = t; k < n; k += T) tot += lam[k];
  tot = block_sum(tot, red);
  double s = 0.0;
  for (int k = t; k < n; k += T) {
    if (eigs) eigs[(size_t)blockIdx.x * n + k] = lam[k];
    const double p = tot > 0.0 ? lam[k] / tot : 0.0;
    if (p > 0.0) s -= p * log(p);
  }
  s = block_sum(s, red);
  if (t == 0) entropy[blockIdx.x] = s;
}

// The unblocked reduction of the n x n matrices at rows and columns
// off .. off + n - 1 of every walker's ld x ld matrix.
cudaError_t launch_tridiag(double2* gram, int64_t walkers, int n, int ld, int off, double* d,
                           double* e, cudaStream_t st) {
  if (n <= kSmallRed) {
    const size_t sm = (size_t)kSmallRed * kSmallLd * sizeof(double2);
    static bool attr_small[kAttrDevices] = {};
    const cudaError_t err = smem_limit(tridiag_small_kernel, (int)sm, attr_small);
    if (err != cudaSuccess) return err;
    tridiag_small_kernel<<<(unsigned)walkers, 256, sm, st>>>(gram, n, ld, off, d, e);
    count_launch();
    return cudaGetLastError();
  }
  const size_t sm = (2 + (size_t)kRedWarps) * n * sizeof(double2);
  static bool attr[kAttrDevices] = {};
  const cudaError_t err = smem_limit(tridiag_kernel<kRedWarps>, 200 * 1024, attr);
  if (err != cudaSuccess) return err;
  tridiag_kernel<kRedWarps><<<(unsigned)walkers, kRedWarps * 32, sm, st>>>(gram, n, ld, off, d, e);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_entropy_eig(double2* gram, int64_t walkers, int n, double* d, double* e,
                               double* entropy, double* eigs, cudaStream_t st) {
  if (walkers <= 0) return cudaSuccess;
  cudaError_t err = launch_tridiag(gram, walkers, n, n, 0, d, e, st);
  if (err != cudaSuccess) return err;
  return launch_entropy_bisect(d, e, walkers, n, entropy, eigs, st);
}

namespace {
constexpr size_t kPanelSmemMax = 220 * 1024;  // dynamic shared memory of the panel kernel
template <int WARPS, bool VWS>
cudaError_t panel_launch(double2* gram, const double* S, int64_t walkers, int n, int p0, int nbp,
                         double2* P, int64_t pstride, double* d, double* e, size_t sm,
                         cudaStream_t st) {
  static bool attr[kAttrDevices] = {};
  const cudaError_t err = smem_limit(tri_panel_kernel<WARPS, VWS>, (int)kPanelSmemMax, attr);
  if (err != cudaSuccess) return err;
  tri_panel_kernel<WARPS, VWS><<<(unsigned)walkers, WARPS * 32, sm, st>>>(gram, S, n, p0, nbp, P,
                                                                           pstride, d, e);
  return cudaSuccess;
}
}  // namespace

cudaError_t launch_tri_panel(double2* gram, const double* S, int64_t walkers, int n, int p0,
                             int nbp, double2* P, int64_t pstride, double* d, double* e,
                             cudaStream_t st) {
  if (walkers <= 0) return cudaSuccess;
  if (nbp < 1 || nbp > kPanelMax || p0 < 0 || p0 + nbp > n - 1 || pstride < 2 * (int64_t)nbp * n)
    return cudaErrorInvalidValue;
  // v, y and the warps' partial products; then, where they fit, the panel's
  // V and W rows p0 .. n-1
  const size_t base = (2 + (size_t)kPanelWarps) * n * sizeof(double2);
  const size_t vw = 2 * (size_t)nbp * (n - p0) * sizeof(double2);
  if (base > kPanelSmemMax) return cudaErrorInvalidValue;
  const cudaError_t err =
      base + vw <= kPanelSmemMax
          ? panel_launch<kPanelWarps, true>(gram, S, walkers, n, p0, nbp, P, pstride, d, e,
                                            base + vw, st)
          : panel_launch<kPanelWarps, false>(gram, S, walkers, n, p0, nbp, P, pstride, d, e, base,
                                             st);
  if (err != cudaSuccess) return err;
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_tri_pack(const double2* P, int64_t pstride, int64_t walkers, int n, int q,
                            int nbp, double2* wvh, cudaStream_t st) {
  if (walkers <= 0 || q >= n) return cudaSuccess;
  const int64_t elems = (int64_t)(n - q) * 2 * nbp;
  const unsigned bx = (unsigned)std::min<int64_t>((elems + 255) / 256, 64);
  tri_pack_kernel<<<dim3(bx, (unsigned)walkers), 256, 0, st>>>(P, pstride, n, q, nbp, wvh);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_tri_mirror(double2* gram, double* S, int64_t walkers, int n, cudaStream_t st) {
  if (walkers <= 0) return cudaSuccess;
  const int T = (n + 31) / 32;
  tri_mirror_kernel<<<dim3((unsigned)(T * (T + 1) / 2), (unsigned)walkers), 256, 0, st>>>(gram, S,
                                                                                         n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_tri_sum(const double2* gram, double* S, int64_t walkers, int n, int q,
                           cudaStream_t st) {
  if (walkers <= 0 || q >= n) return cudaSuccess;
  const int64_t elems = (int64_t)(n - q) * (n - q);
  const unsigned bx = (unsigned)std::min<int64_t>((elems + 255) / 256, 64);
  tri_sum_kernel<<<dim3(bx, (unsigned)walkers), 256, 0, st>>>(gram, S, n, q);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_tri_tail(double2* gram, int64_t walkers, int n, int p0, double* d, double* e,
                            cudaStream_t st) {
  if (walkers <= 0) return cudaSuccess;
  if (p0 < 0 || p0 >= n) return cudaErrorInvalidValue;
  return launch_tridiag(gram, walkers, n - p0, n, p0, d, e, st);
}

cudaError_t launch_entropy_bisect(const double* d, const double* e, int64_t walkers, int n,
                                  double* entropy, double* eigs, cudaStream_t st) {
  if (walkers <= 0) return cudaSuccess;
  static bool attr[kAttrDevices] = {};
  const cudaError_t err = smem_limit(bisect_kernel, 96 * 1024, attr);
  if (err != cudaSuccess) return err;
  const size_t sm2 = 3 * (size_t)n * sizeof(double) + (kEntThreads + 1) * sizeof(int) +
                     2 * (size_t)n * sizeof(float);
  bisect_kernel<<<(unsigned)walkers, kEntThreads, sm2, st>>>(d, e, n, entropy, eigs);
  count_launch();
  return cudaGetLastError();
}

}  // namespace bg
