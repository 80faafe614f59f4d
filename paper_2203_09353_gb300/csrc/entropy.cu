// Entanglement entropy of a batch of states (Alg. 1, "Calculate Entropy";
// Sec. 3): for each walker, the K x K Gram matrix G = X X^H of the state seen
// as the column-major K x M matrix X (K = 2^split rows: the lower spins), whose
// nonzero eigenvalues are those of rho = Psi Psi^H; then p_i = lambda_i /
// sum(lambda) and S = -sum p_i ln p_i.
//
// G comes from the library's Hermitian rank-k update (a grouped plan with
// BG_PLAN_HERK, FP64 or split precision), lower triangle. Two kernels follow,
// one CTA per walker:
//  * tridiag_kernel: Householder reduction of G to a real symmetric
//    tridiagonal matrix (d, e) in FP64, the steps of LAPACK's zhetd2 for the
//    lower triangle: for column j, the reflector H = I - tau v v^H that maps
//    G[j+1:, j] to (beta, 0, ..., 0) (beta real), then
//    G22 <- G22 - v w^H - w v^H with p = tau G22 v, w = p - (tau/2)(p^H v) v.
//    Only the lower triangle is touched: a warp per column of the trailing
//    matrix, its lanes down the column (coalesced).
//  * bisect_kernel: every eigenvalue of the tridiagonal matrix by bisection
//    on the Sturm count (the number of negative pivots of T - x I), one thread
//    per eigenvalue, then the entropy by a block reduction.
// Both are FP64-pipe bound; the tridiagonal step holds a walker's G in
// global memory (L2), one SM per walker.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>

#include "bgemm_internal.h"

namespace bg {
namespace {

constexpr int kEntThreads = 256;      // bisection; reduction for n > 512
constexpr int kEntMaxThreads = 512;   // reduction for n <= 512

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


// Householder tridiagonalisation of the n x n Hermitian matrices G_w (lower
// triangle, column-major, leading dimension n, walker w at G + w n n; only the
// lower triangle is read or written). Writes d[w n + i] (diagonal) and
// e[w n + i] (sub-diagonal, i < n - 1). Each warp takes whole columns of the
// trailing matrix (its lanes run down the column, coalesced): the Hermitian
// product p = G22 v from the lower triangle alone adds G22[i, c] v[c] into
// the warp's own partial vector for rows i >= c and conj(G22[i, c]) v[i]
// into the column's dot product for row c; the rank-2 update then rewrites
// the lower triangle. Dynamic shared memory: v, w and the warps' partial
// products, (2 + WARPS) n complex.
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) tridiag_kernel(double2* G, int n, double* d,
                                                             double* e) {
  constexpr int kEntWarps = WARPS;
  extern __shared__ double2 sm[];
  Z* v = reinterpret_cast<Z*>(sm);
  Z* w = v + n;
  Z* part = w + n;  // kEntWarps x n
  __shared__ double red[kEntWarps];
  __shared__ double s_beta, s_tau_re, s_tau_im, s_sc_re, s_sc_im;
  __shared__ int s_skip;
  double2* A = G + (size_t)blockIdx.x * n * n;
  double* dw = d + (size_t)blockIdx.x * n;
  double* ew = e + (size_t)blockIdx.x * n;
  const int t = threadIdx.x, T = blockDim.x, warp = t >> 5, lane = t & 31;
  auto at = [&](int r, int c) -> double2& { return A[r + (size_t)c * n]; };

  for (int j = 0; j < n - 1; ++j) {
    const int m = n - j - 1;  // order of the trailing matrix G22 = A[j+1:, j+1:]
    double2* A22 = A + (j + 1) + (size_t)(j + 1) * n;
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
        s_tau_re = (beta - a.x) / beta;
        s_tau_im = -a.y / beta;
        // 1 / (alpha - beta)
        const double dr = a.x - beta, di = a.y, den = dr * dr + di * di;
        s_sc_re = dr / den;
        s_sc_im = -di / den;
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
    // ---- partial products of p = G22 v from the lower triangle, a warp per column
    Z* pw = part + warp * m;
    for (int c = warp; c < m; c += kEntWarps) {
      const double2* col = A22 + (size_t)c * n;
      const Z vc = v[c];
      Z dot = {0.0, 0.0};
      for (int i = c + lane; i < m; i += 32) {
        const double2 a2 = col[i];
        const Z a = {a2.x, a2.y};
        pw[i] = zfma(a, vc, pw[i]);                // G22[i, c] v[c], row i
        if (i > c) dot = zfma_conj(a, v[i], dot);  // conj(G22[i, c]) v[i], row c
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        dot.re += __shfl_xor_sync(0xFFFFFFFFu, dot.re, o);
        dot.im += __shfl_xor_sync(0xFFFFFFFFu, dot.im, o);
      }
      __syncwarp();
      if (lane == 0) pw[c] = zadd(pw[c], dot);
      __syncwarp();
    }
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
    pr = block_sum(pr, red);
    pi_ = block_sum(pi_, red);
    const Z alpha2 = zmul({-0.5 * tau.re, -0.5 * tau.im}, {pr, pi_});
    for (int i = t; i < m; i += T) w[i] = zfma(alpha2, v[i], w[i]);
    __syncthreads();
    // ---- G22 <- G22 - v w^H - w v^H on the lower triangle, a warp per column
    for (int c = warp; c < m; c += kEntWarps) {
      double2* col = A22 + (size_t)c * n;
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

// Eigenvalues of each walker's tridiagonal matrix by bisection, then
// S = -sum p ln p with p = lambda / sum(lambda) over p > 0. Dynamic shared
// memory: d, e^2 and the eigenvalues, 3 n doubles, then T + 1 int counts.
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
  __syncthreads();
  // multisection: one Sturm count per thread on an even grid of [lo, hi]
  // gives every eigenvalue a bracket T times narrower to start from
  int* cnt = reinterpret_cast<int*>(lam + n);  // T + 1 counts
  const double hstep = (hi - lo) / T;
  cnt[t + 1] = t + 1 < T ? sturm_count(sd, se2, n, lo + (t + 1) * hstep, pivmin) : n;
  if (t == 0) cnt[0] = 0;
  __syncthreads();
  for (int k = t; k < n; k += T) {
    // the k-th smallest eigenvalue: count(a) <= k < count(b)
    int g = 0;  // last grid point with count <= k (counts are nondecreasing)
    int lo_i = 0, hi_i = T;
    while (hi_i - lo_i > 1) {
      const int mid = (lo_i + hi_i) >> 1;
      if (cnt[mid] <= k) lo_i = mid;
      else hi_i = mid;
    }
    g = lo_i;
    double a = lo + g * hstep, b = g + 1 < T ? lo + (g + 1) * hstep : hi;
    for (int it = 0; it < 200 && b - a > tol; ++it) {
      const double mid = 0.5 * (a + b);
      if (sturm_count(sd, se2, n, mid, pivmin) <= k) a = mid;
      else b = mid;
    }
    lam[k] = 0.5 * (a + b);
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

}  // namespace

cudaError_t launch_entropy_eig(double2* gram, int64_t walkers, int n, double* d, double* e,
                               double* entropy, double* eigs, cudaStream_t st) {
  if (walkers <= 0) return cudaSuccess;
  const int warps = n <= 512 ? kEntMaxThreads / 32 : kEntThreads / 32;
  const size_t sm1 = (2 + (size_t)warps) * n * sizeof(double2);
  const size_t sm2 = 3 * (size_t)n * sizeof(double) + (kEntThreads + 1) * sizeof(int);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tridiag_kernel<kEntMaxThreads / 32>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(tridiag_kernel<kEntThreads / 32>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(bisect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    attr = true;
  }
  if (warps == kEntMaxThreads / 32)
    tridiag_kernel<kEntMaxThreads / 32><<<(unsigned)walkers, kEntMaxThreads, sm1, st>>>(gram, n, d, e);
  else
    tridiag_kernel<kEntThreads / 32><<<(unsigned)walkers, kEntThreads, sm1, st>>>(gram, n, d, e);
  count_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  bisect_kernel<<<(unsigned)walkers, kEntThreads, sm2, st>>>(d, e, n, entropy, eigs);
  count_launch();
  return cudaGetLastError();
}

}  // namespace bg
