// The Metropolis decision of the annealing step (Alg. 1, "M.A") and the copy
// of accepted proposals over the walkers' current states.
//
// metropolis_decide_kernel: one thread per walker, in FP64: the move from
// energy e_cur to e_new is accepted when delta = direction (e_new - e_cur)
// <= 0, or else when the walker's uniform u satisfies u < exp(-delta / T)
// (T = 0 gives exp(-inf) = 0: uphill moves are refused; a NaN energy fails
// both tests). Accepted walkers take the new energy.
// metropolis_commit_kernel: the accepted walkers' proposed states are copied
// over their current ones, 16-byte loads and stores, grid (chunks, walkers).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "bgemm_internal.h"

namespace bg {
namespace {

__global__ void metropolis_decide_kernel(int64_t walkers, double T, double dir, const double* u,
                                         const double* e_new, double* e_cur, int32_t* acc) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < walkers;
       w += (int64_t)gridDim.x * blockDim.x) {
    const double en = e_new[w], ec = e_cur[w];
    const double delta = dir * (en - ec);
    const bool down = delta <= 0.0;
    const bool accept = down || u[w] < exp(-delta / T);
    if (accept) e_cur[w] = en;
    acc[w] = accept ? 1 : 0;
  }
}

__global__ void metropolis_commit_kernel(const int32_t* acc, const double2* prop, int64_t pstride,
                                         double2* cur, int64_t cstride, int64_t amps) {
  const int64_t w = blockIdx.y;
  if (!acc[w]) return;
  const double2* src = prop + w * pstride;
  double2* dst = cur + w * cstride;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < amps;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

}  // namespace

cudaError_t launch_metropolis(int64_t walkers, double T, int direction, const double* u,
                              const double* e_new, double* e_cur, int32_t* acc,
                              const void* prop, int64_t pstride, void* cur, int64_t cstride,
                              int64_t amps, int sms, cudaStream_t st) {
  if (walkers <= 0) return cudaSuccess;
  const int threads = 256;
  const unsigned grid = (unsigned)std::min<int64_t>((walkers + threads - 1) / threads, 4096);
  metropolis_decide_kernel<<<grid, threads, 0, st>>>(walkers, T, (double)direction, u, e_new,
                                                     e_cur, acc);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || amps <= 0) return e;
  // enough blocks per walker to cover the chip a few times over
  int64_t per = std::max<int64_t>(1, (int64_t)sms * 8 / std::max<int64_t>(walkers, 1));
  per = std::min<int64_t>(per, (amps + threads - 1) / threads);
  for (int64_t w0 = 0; w0 < walkers; w0 += 65535) {
    const int64_t nw = std::min<int64_t>(walkers - w0, 65535);
    metropolis_commit_kernel<<<dim3((unsigned)per, (unsigned)nw), threads, 0, st>>>(
        acc + w0, static_cast<const double2*>(prop) + w0 * pstride, pstride,
        static_cast<double2*>(cur) + w0 * cstride, cstride, amps);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace bg
