// Local two-spin gate of the annealing step (Sec. 2 and Alg. 1, "Apply Local
// Gate"): a 4 x 4 unitary U_w on spins (j, j+1) of each walker's state vector
// psi_w of 2^S complex amplitudes, in place:
//
//   psi_w'[x] = sum_{c=0..3} U_w[a(x), c] psi_w[x - a(x) 2^j + c 2^j],
//   a(x) = b_j(x) + 2 b_{j+1}(x),  b_i(x) = bit i of x (spin i).
//
// The 2^S amplitudes fall into 2^(S-2) independent groups of four (the basis
// states that differ only in spins j and j+1). One thread owns one group:
// it reads the four amplitudes, multiplies by U_w held in registers, and
// writes the four results back, so every amplitude is read and written once
// and no two threads touch the same one. Group g starts at x0 = g with two
// zero bits inserted at bit j; consecutive threads take consecutive g, which
// for j >= 5 makes each of the four loads 32 neighbouring amplitudes.
//
// Bound: FP64 arithmetic on this part, not memory. Each amplitude costs 16
// real multiply-adds against 32 bytes moved; at 2 DFMA per clock per SM that
// is about 39 G amplitudes/s, against 210 G/s for the copy bandwidth.
#include <algorithm>

#include "bgemm_internal.h"

namespace bg {

namespace {

constexpr int kGateThreads = 256;

// Same protocol as the other kernels' error word: the first code wins, the
// count keeps growing.
__device__ __forceinline__ void gate_error(int* err, int walker) {
  if (atomicCAS(err, 0, (int)BG_ERR_INVALID_ARG) == 0) {
    err[1] = ERRLOC_GATE_SITE;
    err[2] = walker;
  }
  atomicAdd(err + 3, 1);
}

__global__ void __launch_bounds__(kGateThreads) local_gate_kernel(int64_t walkers, int spins,
                                                                 const int32_t* sites,
                                                                 const double2* gates,
                                                                 double2* states, int64_t stride,
                                                                 int* err) {
  const int64_t w = blockIdx.y + (int64_t)blockIdx.z * gridDim.y;
  if (w >= walkers) return;
  const int j = __ldg(sites + w);
  if (j < 0 || j > spins - 2) {
    if (blockIdx.x == 0 && threadIdx.x == 0) gate_error(err, (int)w);
    return;
  }
  double2 u[16];  // U_w column-major: u[a + 4 c] = U[a, c]
#pragma unroll
  for (int e = 0; e < 16; ++e) u[e] = __ldg(gates + 16 * w + e);
  double2* psi = states + w * stride;
  const int64_t groups = (int64_t)1 << (spins - 2);
  const int64_t low = ((int64_t)1 << j) - 1;
  const int64_t step = (int64_t)1 << j;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x0 = ((g & ~low) << 2) | (g & low);
    double2 v[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = psi[x0 + c * step];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double2 uc = u[a + 4 * c];
        re = fma(uc.x, v[c].x, fma(-uc.y, v[c].y, re));
        im = fma(uc.x, v[c].y, fma(uc.y, v[c].x, im));
      }
      psi[x0 + a * step] = make_double2(re, im);
    }
  }
}

}  // namespace

cudaError_t launch_local_gate(int64_t walkers, int spins, const int32_t* sites, const void* gates,
                              void* states, int64_t stride, int* d_err, int sms,
                              cudaStream_t st) {
  if (walkers <= 0) return cudaSuccess;
  const int64_t groups = (int64_t)1 << (spins - 2);
  // enough blocks per walker to fill the GPU a few times over, the rest by striding
  const int64_t want = std::max<int64_t>(1, (int64_t)sms * 8 / std::max<int64_t>(1, walkers));
  const int64_t gx = std::min<int64_t>((groups + kGateThreads - 1) / kGateThreads,
                                       std::max<int64_t>(want, 1));
  const int64_t gy = std::min<int64_t>(walkers, 65535);
  const int64_t gz = (walkers + gy - 1) / gy;
  if (gz > 65535) return cudaErrorInvalidConfiguration;
  local_gate_kernel<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), kGateThreads, 0, st>>>(
      walkers, spins, sites, static_cast<const double2*>(gates), static_cast<double2*>(states),
      stride, d_err);
  count_launch();
  return cudaGetLastError();
}

}  // namespace bg
