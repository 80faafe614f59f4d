// Split-precision (BF16 digit planes on the tensor cores) path: host-side
// interface used by the C ABI layer. See split.cu for the method.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "bgemm.h"
#include "bgemm_internal.h"

namespace bg {

constexpr int kMaxSlices = 12;

struct SplitPlan;

// Library-owned cache of fixed-size split plans (per device).
struct SplitWorkspace {
  std::vector<SplitPlan*> cache;  // most recent last
  ~SplitWorkspace();
};

// Digit width used for `slices` planes when the caller passes beta_bits = 0.
int split_default_beta(int slices);

namespace splitk {
// Slice counts and digit widths the small-instance kernel has versions for.
bool split_small_supported(int s, int beta);
}  // namespace splitk

bg_status split_plan_create(SplitPlan** out, bg_dtype dt, const bg_precision& pr,
                            const std::vector<bg_instance>& table, const int64_t* d_table,
                            int sms, bool autotune, cudaStream_t st, std::string* err, bool herk = false,
                            bool small_kernel = true, const std::vector<int8_t>* route = nullptr);
// route (optional, one entry per table instance): 0 = the small-instance
// kernel where split_small_route says so, 1 = the small-instance kernel for
// every instance it can take (real, m, n, k <= 64), 2 = the tile kernels.
bg_status split_chain_create(SplitPlan** out, bg_dtype dt, const bg_precision& pr,
                             const std::vector<int64_t>& wn, const std::vector<int64_t>& woff,
                             const std::vector<int64_t>& pool_n,
                             const std::vector<int64_t>& pool_off, int sms, cudaStream_t st,
                             std::string* err);
void split_plan_destroy(SplitPlan* p);
int64_t split_plan_workspace(const SplitPlan* p);
int split_plan_launches(const SplitPlan* p);
int64_t split_plan_items(const SplitPlan* p);
int split_plan_beta_bits(const SplitPlan* p);
std::string split_plan_describe(const SplitPlan* p);

// `ev` (optional): three events recorded after the slicer, after the
// small-instance kernel and after the tile GEMM.
bg_status split_plan_run(SplitPlan* p, const void* A, const void* B, void* C, const Scalars& s,
                         int* d_err, cudaStream_t st, std::string* err,
                         cudaEvent_t* ev = nullptr);

bg_status split_fixed(bg_dtype dt, const bg_precision& pr, int64_t m, int64_t n, int64_t k,
                      const Scalars& s, const void* A, int64_t lda, int64_t sA, const void* B,
                      int64_t ldb, int64_t sB, void* C, int64_t ldc, int64_t sC, int64_t batch,
                      SplitWorkspace* ws, int sms, int* d_err, bool capturing, cudaStream_t st,
                      std::string* err);

// Runs a fixed-size split batch with every workspace inside `scratch`
// (device memory, 256-byte aligned, scratch_bytes long); allocates nothing.
bg_status split_fixed_in_scratch(bg_dtype dt, const bg_precision& pr, int64_t m, int64_t n,
                                 int64_t k, const Scalars& s, const void* A, int64_t lda,
                                 int64_t sA, const void* B, int64_t ldb, int64_t sB, void* C,
                                 int64_t ldc, int64_t sC, int64_t batch, void* scratch,
                                 size_t scratch_bytes, int sms, cudaStream_t st,
                                 std::string* err);

bg_status split_chain_prepare_pool(SplitPlan* p, const void* U, int* d_err, cudaStream_t st,
                                   std::string* err);
bg_status split_chain_step(SplitPlan* p, const void* U, const int32_t* idx_row, const void* Cin,
                           void* Cout, int* d_err, cudaStream_t st, std::string* err);

cudaError_t launch_split_planes(int64_t m, int64_t k, const double* X, int64_t ldx, int axis,
                                int slices, int beta_bits, int32_t* exps, uint16_t* digits,
                                cudaStream_t st);

}  // namespace bg
