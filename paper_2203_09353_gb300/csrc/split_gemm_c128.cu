// Complex (complex128, through the real 2x2 expansion) instantiations of the split-precision GEMM kernel.
#include "split_gemm.cuh"

namespace bg {
namespace splitk {

cudaError_t launch_split_gemm_c128(int s, int grid, size_t smem, cudaStream_t st,
                                  const GemmArgs& g) {
  return launch_gemm_t<true>(s, grid, smem, st, g);
}

cudaError_t set_split_gemm_attr_c128(int s) { return set_attr_t<true>(s); }

}  // namespace splitk
}  // namespace bg
