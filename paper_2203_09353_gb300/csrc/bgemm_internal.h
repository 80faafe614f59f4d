// Internal declarations shared by the library's translation units.
// Nothing here is part of the public ABI (include/bgemm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "bgemm.h"

namespace bg {

// ---- work description --------------------------------------------------------

// Tile programs of the FP64 path. A work item names one program and the part
// of the batch it covers.
enum Prog : int16_t {
  PROG_R64_SMALL = 0,   // a warp per instance (8 per CTA), or 8 warps on one instance
  PROG_R64_TILE = 1,    // 64x64 output tile, DFMA, 4x4 outputs per thread
  PROG_R64_DMMA = 2,    // 64x64 output tile, FP64 tensor-core mma.sync m8n8k4
  PROG_C128_SMALL = 3,  // one warp per complex instance
  PROG_C128_TILE = 4,   // 32x32 complex output tile, DFMA, 2x2 per thread
  PROG_COUNT = 5
};

// One unit of work of the persistent FP64 kernel (16 bytes).
//  - tile programs: `inst` = instance id, (r0, c0) = first row/col of the tile
//  - small programs: `inst` = first position in the class-ordered instance
//    list, `count` = number of consecutive instances (<= 8), r0 = c0 = 0
struct WorkItem {
  int32_t inst;
  int16_t prog;
  int16_t count;
  int32_t r0;
  int32_t c0;
};
static_assert(sizeof(WorkItem) == 16, "WorkItem must stay 16 bytes");

constexpr int kSmallPerCta = 8;   // warps (instances) per CTA in the small programs
// Real small-program work items hold g instances that the CTA's 8 warps
// share: g = 8 (a warp each), or g = 1 (all 8 warps on one instance) for
// batches too small to give every resident CTA an item of 8; WorkItem.r0
// carries the warps per instance (0 reads as 1).
inline int small_group(int64_t instances, int64_t grid) {
  return (instances + kSmallPerCta - 1) / kSmallPerCta >= grid ? kSmallPerCta : 1;
}
constexpr int kFp64Threads = 256;

struct Scalars {
  double alpha_re, alpha_im, beta_re, beta_im;
  int alpha_zero, beta_zero;
};

// Program picked for a size (FP64 path) when no tuned choice exists.
int default_prog(bg_dtype dt, int64_t m, int64_t n, int64_t k);
// Output-tile extent of a tile program (rows, cols); small programs return 0.
void prog_tile(int prog, int* tm, int* tn);
bool prog_is_small(int prog);
bool prog_fits(int prog, bg_dtype dt, int64_t m, int64_t n);

// ---- FP64 launchers (fp64.cu) ---------------------------------------------------

cudaError_t launch_fp64_fixed(bg_dtype dt, int prog, int64_t m, int64_t n, int64_t k,
                              const Scalars& s, const void* A, int64_t lda, int64_t sA,
                              const void* B, int64_t ldb, int64_t sB, void* C, int64_t ldc,
                              int64_t sC, int64_t batch, int grid_cap, cudaStream_t st);

// herm: the plan's instances are Hermitian rank-k updates (B = A^H, lower
// triangle stored).
cudaError_t launch_fp64_table(bg_dtype dt, const int64_t* d_table, const int32_t* d_order,
                              const WorkItem* d_items, int64_t n_items, const void* A,
                              const void* B, void* C, const Scalars& s, int grid,
                              cudaStream_t st, bool herm = false);

cudaError_t launch_fp64_chain(bg_dtype dt, const int64_t* d_wn, const int64_t* d_woff,
                              const int64_t* d_pool_off, const int64_t* d_pool_n,
                              int32_t pool_count, const int32_t* d_order,
                              const int32_t* d_idx_row, const WorkItem* d_items, int64_t n_items,
                              const void* U, const void* Cin, void* Cout, int grid,
                              cudaStream_t st);

// Resident CTAs per SM of the persistent FP64 kernel (for grid sizing).
int fp64_blocks_per_sm(bg_dtype dt);

// ---- split-BF16 path (split.cu) ---------------------------------------------------

struct SplitParams;  // defined in split.cu

// ---- measurement and diagnostics (util.cu) ------------------------------------------

cudaError_t launch_rel_err(bg_dtype dt, int64_t count, const int64_t* d_table, const void* A,
                           const void* B, const void* Ct, const void* Cr, double* out,
                           cudaStream_t st);
cudaError_t launch_drift(bg_dtype dt, int64_t count, const int64_t* d_n, const int64_t* d_off,
                         const void* C, double* out, cudaStream_t st);
cudaError_t launch_bounded_wait(int64_t spin_limit, int* d_err, cudaStream_t st);
cudaError_t run_fp64_peak_probe(int mma_kind, int sms, double* tflops, cudaStream_t st);
// Local two-spin gate on a batch of complex128 state vectors (gate.cu).
cudaError_t launch_local_gate(int64_t walkers, int spins, const int32_t* sites, const void* gates,
                              void* states, int64_t stride, int* d_err, int sms, cudaStream_t st);

// Device error word layout: [0] = first error code, [1] = location id,
// [2] = detail, [3] = count of events.
enum DevErrLoc : int {
  ERRLOC_NONE = 0,
  ERRLOC_TEST_WAIT = 1,
  ERRLOC_SPLIT_FULL_BARRIER = 2,
  ERRLOC_SPLIT_EMPTY_BARRIER = 3,
  ERRLOC_SPLIT_ACC_FULL = 4,
  ERRLOC_SPLIT_ACC_EMPTY = 5,
  ERRLOC_SPLIT_TMEM_ALLOC = 6,
  ERRLOC_CHAIN_INDEX = 7,
  ERRLOC_GATE_SITE = 8
};

// Host bookkeeping.
void count_launch(int n = 1);

// ---- static scratch (noalloc.cu) ----
// Capacity of the per-device static scratch array, in bytes.
size_t static_scratch_capacity();
// Address of the static scratch on the current device (looked up once per device).
bg_status static_scratch(void** out, size_t* bytes, std::string* err);

// Tridiagonalisation and eigenvalues of each walker's Hermitian n x n Gram
// matrix (lower triangle, overwritten), then the entanglement entropy
// (entropy.cu). eigs: optional device [walkers][n], ascending.
cudaError_t launch_entropy_eig(double2* gram, int64_t walkers, int n, double* d, double* e,
                               double* entropy, double* eigs, cudaStream_t st);

// The blocked form of the same reduction (entropy.cu). Panels of nb columns:
// launch_tri_panel reduces columns p0 .. p0 + nbp - 1 (p0 + nbp <= n - 1) of
// every walker, keeping the panel's rank-2 updates as [V W] (walker w at
// P + w pstride, 2 nbp columns of n, pstride >= 2 nbp n). launch_tri_pack
// writes the trailing update's second operand [W2 V2]^H for the rows from
// q = p0 + nbp (walker w at wvh + w (n - q) 2 nbp), after which the caller
// applies C[q:, q:] -= [V2 W2] [W2 V2]^H as a batched GEMM. launch_tri_tail
// reduces the trailing matrix from row and column p0 unblocked, and
// launch_entropy_bisect takes the tridiagonal matrices to eigenvalues and
// entropies.
// Panel width of the blocked reduction (at most 64): at K = 256 (128
// walkers), 16 columns beat 8 (more trailing GEMMs) and 32 (the corrections
// grow with the width). The last kTriTail columns are reduced unblocked.
constexpr int kTriPanelWidth = 16;
constexpr int kTriTail = 64;
cudaError_t launch_tri_panel(double2* gram, const double* S, int64_t walkers, int n, int p0,
                             int nbp, double2* P, int64_t pstride, double* d, double* e,
                             cudaStream_t st);
cudaError_t launch_tri_tail(double2* gram, int64_t walkers, int n, int p0, double* d, double* e,
                            cudaStream_t st);
// Copies each walker's lower triangle into its upper triangle (conjugated):
// the blocked panels read the trailing matrix in full, together with
// S = Re G + Im G (walkers x n x n doubles, same layout), which the mirror
// writes whole and launch_tri_sum rewrites on rows and columns q.. after
// each trailing update.
cudaError_t launch_tri_mirror(double2* gram, double* S, int64_t walkers, int n, cudaStream_t st);
cudaError_t launch_tri_sum(const double2* gram, double* S, int64_t walkers, int n, int q,
                           cudaStream_t st);
cudaError_t launch_tri_pack(const double2* P, int64_t pstride, int64_t walkers, int n, int q,
                            int nbp, double2* wvh, cudaStream_t st);
cudaError_t launch_entropy_bisect(const double* d, const double* e, int64_t walkers, int n,
                                  double* entropy, double* eigs, cudaStream_t st);

// Metropolis decision per walker and copy of the accepted proposals over the
// current states (anneal.cu). prop / cur may be null when amps == 0.
cudaError_t launch_metropolis(int64_t walkers, double T, int direction, const double* u,
                              const double* e_new, double* e_cur, int32_t* acc,
                              const void* prop, int64_t pstride, void* cur, int64_t cstride,
                              int64_t amps, int sms, cudaStream_t st);

}  // namespace bg
