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
//    The matrix is first mirrored to both triangles so that the Hermitian
//    product and the rank-2 update read and write whole columns (coalesced).
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

constexpr int kEntThreads = 256;

struct Z {
  double re, im;
};
__device__ __forceinline__ Z zmul(Z a, Z b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ Z zconj(Z a) { return {a.re, -a.im}; }
__device__ __forceinline__ Z zadd(Z a, Z b) { return {a.re + b.re, a.im + b.im}; }

// Sum of v over the block (all threads call it; the result reaches every thread).
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

// Householder tridiagonalisation of the n x n Hermitian matrices G_w (lower
// triangle given; column-major, leading dimension n, walker w at G + w n n).
// Writes d[w n + i] (diagonal) and e[w n + i] (sub-diagonal, i < n - 1). G is
// overwritten. Dynamic shared memory: v and w, 2 n complex.
__global__ void __launch_bounds__(kEntThreads) tridiag_kernel(double2* G, int n, double* d,
                                                              double* e) {
  extern __shared__ double2 sm[];
  Z* v = reinterpret_cast<Z*>(sm);
  Z* w = v + n;
  __shared__ double red[kEntThreads / 32];
  __shared__ double s_beta, s_tau_re, s_tau_im, s_sc_re, s_sc_im;
  __shared__ int s_skip;
  double2* A = G + (size_t)blockIdx.x * n * n;
  double* dw = d + (size_t)blockIdx.x * n;
  double* ew = e + (size_t)blockIdx.x * n;
  const int t = threadIdx.x, T = blockDim.x;
  auto at = [&](int r, int c) -> double2& { return A[r + (size_t)c * n]; };

  // mirror the lower triangle into the upper one; real diagonal
  for (int c = 0; c < n; ++c)
    for (int r = c + t; r < n; r += T) {
      double2 x = at(r, c);
      if (r == c) {
        x.y = 0.0;
        at(r, c) = x;
      } else {
        at(c, r) = make_double2(x.x, -x.y);
      }
    }
  __syncthreads();

  for (int j = 0; j < n - 1; ++j) {
    const int m = n - j - 1;  // order of the trailing matrix G22 = A[j+1:, j+1:]
    // ---- reflector of the column below the diagonal (zlarfg)
    double xn2 = 0.0;
    for (int i = 1 + t; i < m; i += T) {
      const double2 x = at(j + 1 + i, j);
      xn2 += x.x * x.x + x.y * x.y;
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
      Z vi;
      if (i == 0) {
        vi = {1.0, 0.0};
      } else {
        const double2 x = at(j + 1 + i, j);
        vi = zmul({x.x, x.y}, sc);
      }
      v[i] = vi;
    }
    __syncthreads();
    // ---- p = tau G22 v (rows of this thread), then alpha2 = -tau/2 (p^H v)
    double pr = 0.0, pi_ = 0.0;  // p^H v, partial
    for (int i = t; i < m; i += T) {
      Z acc = {0.0, 0.0};
      for (int c = 0; c < m; ++c) {
        const double2 a = at(j + 1 + i, j + 1 + c);
        acc = zadd(acc, zmul({a.x, a.y}, v[c]));
      }
      const Z p = zmul(tau, acc);
      w[i] = p;
      const Z pv = zmul(zconj(p), v[i]);
      pr += pv.re;
      pi_ += pv.im;
    }
    pr = block_sum(pr, red);
    pi_ = block_sum(pi_, red);
    const Z alpha2 = zmul({-0.5 * tau.re, -0.5 * tau.im}, {pr, pi_});
    for (int i = t; i < m; i += T) w[i] = zadd(w[i], zmul(alpha2, v[i]));
    __syncthreads();
    // ---- G22 <- G22 - v w^H - w v^H (whole columns, both triangles)
    for (int c = 0; c < m; ++c) {
      const Z wc = zconj(w[c]), vc = zconj(v[c]);
      for (int i = t; i < m; i += T) {
        double2& a = at(j + 1 + i, j + 1 + c);
        const Z u = zadd(zmul(v[i], wc), zmul(w[i], vc));
        a.x -= u.re;
        a.y -= u.im;
      }
    }
    __syncthreads();
  }
  if (t == 0) {
    dw[n - 1] = at(n - 1, n - 1).x;
    ew[n - 1] = 0.0;
  }
}

// Number of eigenvalues of the symmetric tridiagonal (d, e2 = e^2) below x:
// the negative pivots of T - x I (a pivot smaller than pivmin in magnitude
// is replaced by -pivmin, as in LAPACK's dstebz).
__device__ __forceinline__ int sturm_count(const double* d, const double* e2, int n, double x,
                                           double pivmin) {
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  int cnt = q < 0.0;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

// Eigenvalues of each walker's tridiagonal matrix by bisection, then
// S = -sum p ln p with p = lambda / sum(lambda) over p > 0. Dynamic shared
// memory: d, e^2 and the eigenvalues, 3 n doubles.
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
  for (int k = t; k < n; k += T) {
    // the k-th smallest eigenvalue: count(a) <= k < count(b)
    double a = lo, b = hi;
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
  const size_t sm1 = 2 * (size_t)n * sizeof(double2);
  const size_t sm2 = 3 * (size_t)n * sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tridiag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(bisect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    attr = true;
  }
  tridiag_kernel<<<(unsigned)walkers, kEntThreads, sm1, st>>>(gram, n, d, e);
  count_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  bisect_kernel<<<(unsigned)walkers, kEntThreads, sm2, st>>>(d, e, n, entropy, eigs);
  count_launch();
  return cudaGetLastError();
}

}  // namespace bg
