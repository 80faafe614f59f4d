// Real (FP64) instantiations of the split-precision GEMM kernel.
#include "split_gemm.cuh"

namespace bg {
namespace splitk {

cudaError_t launch_split_gemm_r64(int s, int grid, size_t smem, cudaStream_t st,
                                  const GemmArgs& g) {
  return launch_gemm_t<false>(s, grid, smem, st, g);
}

cudaError_t set_split_gemm_attr_r64(int s) { return set_attr_t<false>(s); }

}  // namespace splitk
}  // namespace bg
