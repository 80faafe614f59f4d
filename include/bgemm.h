/*
 * bgemm.h -- C ABI of the GB300 batched small-GEMM library.
 *
 * The library computes the batched matrix product of Eq. (1), Sec. 2 of
 * "Batched matrix operations on distributed GPUs with application in
 * theoretical physics" (arXiv 2203.09353):
 *
 *     C_i = alpha * A_i * B_i + beta * C_i,        i = 1..N,
 *
 * for thousands of small independent instances, in real FP64 or complex128
 * (the complex matrices of Sec. 2), with one process submitting the whole
 * batch to one GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Layout: every matrix is column-major; element (r, c) of a matrix with
 *    leading dimension ld is at element offset r + c * ld. Only the
 *    non-transposed product is provided (Eq. 1 has no transposes).
 *  - Element types: BG_R64 = double; BG_C128 = interleaved (re, im) double
 *    pair, 16 bytes. Offsets, leading dimensions and strides are counted in
 *    ELEMENTS of that type, never in bytes.
 *  - Scalars alpha and beta are HOST pointers: one double (BG_R64) or two
 *    doubles {re, im} (BG_C128). When beta == 0 the old C is not read (NaN
 *    or Inf there do not propagate); when alpha == 0, A and B are not read.
 *  - Matrix buffers (A, B, C, U pools, states, tables marked "device") are
 *    caller-owned DEVICE memory of the current CUDA device; the library never
 *    frees them and never keeps a pointer to them past the call, except a
 *    plan's captured graph (see batched_gemm_grouped).
 *  - Alignment: every matrix base pointer must be 8-byte aligned (BG_R64) or
 *    16-byte aligned (BG_C128), otherwise BG_ERR_INVALID_ARG.
 *  - Streams: every compute call is asynchronous on the given stream (NULL
 *    = legacy default stream) and returns after enqueueing its work. A call
 *    that would allocate device memory while the stream is being captured
 *    returns BG_ERR_CAPTURE instead.
 *  - Errors: functions return a bg_status; nothing throws, traps or exits.
 *    Empty problems (batch or count 0, or any of m, n, k equal to 0 with the
 *    BLAS meaning) return BG_OK. bg_last_error() gives a message for the
 *    last failure on the calling host thread. Device-side failures (a bounded
 *    wait that ran out) are recorded in a device error word that
 *    bg_check_device_errors() reads; kernels never trap.
 *  - Precision: BG_MODE_FP64 computes every product and sum in FP64. The
 *    split mode (BG_MODE_SPLIT_BF16) cuts each FP64 operand into `slices`
 *    BF16 digit planes scaled by a power-of-two exponent per row of A and
 *    per column of B, multiplies the planes on the tensor cores with FP32
 *    accumulation that is exact by construction, and recombines the plane
 *    products exactly before one rounding to FP64. The paper itself has no
 *    such mode (its GEMMs are cuBLAS complex FP64, Sec. 4); the normwise
 *    error ||C - C_exact||_F / (||A||_F ||B||_F) falls with `slices`.
 */
#ifndef BGEMM_H
#define BGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL means the legacy default stream. */
typedef struct CUstream_st* bg_stream_t;

typedef enum {
  BG_OK = 0,
  BG_ERR_INVALID_ARG = 1,  /* bad size, null pointer, misalignment, bad enum */
  BG_ERR_UNSUPPORTED = 2,  /* valid request that this build does not implement */
  BG_ERR_CUDA = 3,         /* a CUDA runtime call failed (message in bg_last_error) */
  BG_ERR_NOMEM = 4,        /* device or host allocation failed */
  BG_ERR_CAPTURE = 5,      /* would allocate while the stream is being captured */
  BG_ERR_TIMEOUT = 6       /* a bounded device-side wait gave up */
} bg_status;

typedef enum { BG_R64 = 0, BG_C128 = 1 } bg_dtype;

typedef enum { BG_MODE_FP64 = 0, BG_MODE_SPLIT_BF16 = 1 } bg_mode;

/* Precision request. mode = bg_mode. slices = number of BF16 digit planes
 * per operand in split mode (1..12; 3, 6 and 9 are the documented modes),
 * ignored in FP64 mode. beta_bits = digit width in bits (2..8), 0 = chosen
 * by the library from k so that the FP32 tensor-core sums stay exact.
 * A NULL bg_precision pointer means FP64 mode. */
typedef struct {
  int32_t mode;
  int32_t slices;
  int32_t beta_bits;
  int32_t reserved; /* must be 0 */
} bg_precision;

/* One instance of a variable-size batch (Sec. 2, the variable-size batch of
 * Abdelfattah et al. the paper discusses): sizes, leading dimensions and
 * element offsets of A_i, B_i and C_i from the base pointers passed at run
 * time. Requires m, n, k >= 0, lda >= max(1, m), ldb >= max(1, k),
 * ldc >= max(1, m), offsets >= 0. */
typedef struct {
  int64_t m, n, k;
  int64_t lda, ldb, ldc;
  int64_t a_off, b_off, c_off;
} bg_instance;

typedef struct bg_plan bg_plan;

/* Plan flags. */
enum {
  BG_PLAN_AUTOTUNE = 1u,      /* time candidates per size class and keep the fastest: the FP64
                                 tile programs; in split mode also the split path (for real
                                 classes up to 64 on a side: on the small-instance kernel and
                                 on the tile kernels, separately), each class then computed by
                                 the fastest (the FP64 path is never less accurate) */
  BG_PLAN_USE_CACHE = 2u,     /* read/write autotune results in the JSON file cache_path */
  BG_PLAN_CAPTURE_GRAPH = 4u, /* batched_gemm_grouped replays a captured CUDA graph */
  BG_PLAN_PROFILE = 8u,       /* record CUDA events around each kernel (bg_plan_kernel_times) */
  BG_PLAN_HERK = 16u,         /* Hermitian rank-k updates instead of Eq. (1), see below */
  BG_PLAN_SPLIT_TILES = 32u   /* split mode: compute every instance with the digit-plane tile
                                 kernels, also the small real ones (m, n, k <= 64) that
                                 otherwise go to the fused small-instance kernel; results of
                                 both stay within the split mode's error bound */
};

/* BG_PLAN_HERK. Sec. 3 builds the density matrix rho = Psi Psi^H of each
 * state: a product of a matrix with its own conjugate transpose. A plan made
 * with this flag computes, per instance,
 *   C_i = alpha A_i A_i^H + beta C_i    (A_i A_i^T for real data),
 * with A_i n x k (m_i must equal n_i). Conventions:
 *  - The B fields of the table (ldb, b_off) and B_base are not used; B_base
 *    may be NULL.
 *  - alpha and beta must be real: a non-zero imaginary part is
 *    BG_ERR_INVALID_ARG.
 *  - Only the lower triangle of C_i, diagonal included, is read and
 *    written. For complex128 the diagonal's imaginary parts are set to 0.
 *  - Tiles wholly above the diagonal are not computed, which is about half
 *    the work of the general product.
 * Both precision modes support it; chain plans do not. */

/* ---- Eq. (1), fixed-size batch -------------------------------------------
 * Sec. 2: the batch in which all instances have the same size and sit at a
 * constant stride. Instance i (0 <= i < batch) uses A + i*strideA,
 * B + i*strideB, C + i*strideC (element strides, each >= 0). Requires
 * lda >= max(1,m), ldb >= max(1,k), ldc >= max(1,m). C instances must not
 * overlap each other or A/B. One launch in FP64 mode; the split mode adds
 * the exponent and slicing passes and uses library-owned workspace that is
 * grown (cudaMalloc) on first use of a larger size, so the first split call
 * of a given size must not be made while the stream is being captured. */
bg_status batched_gemm_fixed(bg_dtype dtype, int64_t m, int64_t n, int64_t k,
                             const void* alpha, const void* A, int64_t lda, int64_t strideA,
                             const void* B, int64_t ldb, int64_t strideB, const void* beta,
                             void* C, int64_t ldc, int64_t strideC, int64_t batch,
                             const bg_precision* precision, bg_stream_t stream);

/* ---- fixed-size batch without any device allocation -----------------------
 * No counterpart in the paper: a library service. Same operation, arguments,
 * layout and checks as batched_gemm_fixed, split mode only (precision->mode
 * must be BG_MODE_SPLIT_BF16, else BG_ERR_INVALID_ARG). It is meant for
 * callers that must not allocate device memory while they run: a process
 * whose device memory is already handed out to another allocator (a caching
 * allocator holding the whole GPU), or a latency-critical loop in which a
 * cudaMalloc/cudaFree would stall or synchronise the device.
 *  - Workspace: every buffer the split path needs (digit tiles, line
 *    exponents, work tables, the device error word) is laid out inside one
 *    static device array of 64 MiB per device (67108864 bytes), part of the
 *    library image. Nothing is allocated or freed, by this library or any
 *    other, on any call. A batch whose workspace does not fit is rejected
 *    with BG_ERR_INVALID_ARG before any work is queued, the message giving
 *    the bytes it needs.
 *  - Set-up: the first call on each device looks up the array's address on
 *    that device (the CUDA runtime loads the module holding it then).
 *  - Each call clears what must start at zero (error word, exponent stores)
 *    and uploads its work tables from host memory on `stream`. That host
 *    memory is released on return, so a call made while `stream` is being
 *    captured into a CUDA graph is refused with BG_ERR_CAPTURE.
 *  - Concurrency: all calls on one device share the one array. Calls queued
 *    on the same stream are ordered and safe; calls whose work overlaps in
 *    time (other streams, other host threads) race on the array and give
 *    wrong results.
 *  - A device-side wait that runs out of time (see bg_check_device_errors)
 *    leaves its code only in the array's error word, which the next call
 *    clears; this entry point does not read it back. */
bg_status batched_gemm_fixed_static(bg_dtype dtype, int64_t m, int64_t n, int64_t k,
                                    const void* alpha, const void* A, int64_t lda,
                                    int64_t strideA, const void* B, int64_t ldb, int64_t strideB,
                                    const void* beta, void* C, int64_t ldc, int64_t strideC,
                                    int64_t batch, const bg_precision* precision,
                                    bg_stream_t stream);

/* ---- Eq. (1), variable-size batch: plan -----------------------------------
 * Sec. 2 (variable-size batches, per-size tiling strategies): builds the
 * schedule for `count` instances described by the HOST array `host_table`
 * (copied; the caller may free it on return). The plan sorts instances into
 * size classes, picks a tile program per class (timed when
 * BG_PLAN_AUTOTUNE is set; such timing runs on `stream` on scratch buffers
 * the plan allocates), builds the device-side work table in
 * longest-first order and allocates every workspace the grouped call needs.
 * With BG_PLAN_USE_CACHE the per-class choices are read from / appended to
 * the JSON file at `cache_path` (keyed by GPU name, dtype, mode and class).
 * *out receives a plan owned by the caller (bg_plan_destroy). Must not be
 * called while `stream` is being captured (BG_ERR_CAPTURE). */
bg_status batched_gemm_plan(bg_plan** out, bg_dtype dtype, int64_t count,
                            const bg_instance* host_table, const bg_precision* precision,
                            uint32_t flags, const char* cache_path, bg_stream_t stream);

/* ---- Eq. (1), variable-size batch: run ------------------------------------
 * Computes every instance of the plan with A_base + a_off etc. (element
 * offsets from the plan's table). FP64 mode: one persistent launch that
 * walks the device work table. Split mode: the slicing pass (line exponents
 * and digit planes), one persistent tensor-core launch over the digit tiles
 * and, for the real instances with m, n, k <= 64 (unless
 * BG_PLAN_SPLIT_TILES), one fused small-instance launch that cuts the digits
 * into shared memory itself; instances that an autotuned plan routed to the
 * FP64 path add the FP64 launch. With BG_PLAN_CAPTURE_GRAPH the launches
 * are captured once into a CUDA graph keyed by (A_base, B_base, C_base,
 * alpha, beta) and replayed; a call with other pointers or scalars
 * re-captures. Calls on one plan must not overlap on the GPU (they share the
 * plan's workspace). */
bg_status batched_gemm_grouped(const bg_plan* plan, const void* A_base, const void* B_base,
                               void* C_base, const void* alpha, const void* beta,
                               bg_stream_t stream);

/* ---- chained products (Alg. 1, the step loop) -------------------------------
 * Sec. 3 / Alg. 1: each Monte Carlo procedure multiplies its state by a new
 * operator every step, strictly in sequence, while procedures are
 * independent. chain_plan describes W walkers and a pool of P operators:
 * walker w holds a walker_n[w] x walker_n[w] state at element offset
 * state_off[w] of each state buffer; pool entry j is a pool_n[j] x pool_n[j]
 * matrix at element offset pool_off[j] of U_pool. All arrays are HOST
 * arrays, copied. Leading dimensions equal the sizes. */
bg_status chain_plan(bg_plan** out, bg_dtype dtype, int32_t walkers, const int64_t* walker_n,
                     const int64_t* state_off, int32_t pool_count, const int64_t* pool_n,
                     const int64_t* pool_off, const bg_precision* precision, uint32_t flags,
                     bg_stream_t stream);

/* Runs `steps` steps t = 0..steps-1 of C_w <- U[idx[t][w]] * C_w for every
 * walker w, where idx = U_index is a DEVICE int32 array [steps][walkers]
 * whose entries must name pool matrices of the walker's size. States
 * ping-pong between the two buffers: the input is read from C_ping, step t
 * writes the buffer it did not read, so the result ends in C_ping when
 * `steps` is even and in C_pong when it is odd. The states never leave the
 * device. In split mode the pool's digit planes are cut once per call. */
bg_status chain_step(const bg_plan* plan, const void* U_pool, const int32_t* U_index,
                     void* C_ping, void* C_pong, int32_t steps, bg_stream_t stream);

void bg_plan_destroy(bg_plan* plan);

/* ---- local two-spin gate (Alg. 1, "Apply Local Gate") ----------------------
 * Sec. 2: every Monte Carlo step first applies a unitary to a neighbouring
 * pair of spins of the state. For W state vectors of 2^spins amplitudes, in
 * place:
 *   psi_w'[x] = sum_{c=0..3} U_w[a(x), c] * psi_w[x - a(x) 2^j + c 2^j],
 *   a(x) = b_j(x) + 2 b_{j+1}(x),
 * where b_i(x) is bit i of the basis index x (spin i) and j = sites[w].
 * dtype: BG_C128 only (BG_ERR_UNSUPPORTED otherwise); 2 <= spins <= 40.
 * states: DEVICE, walker w's amplitudes at states + w * stride complex
 *   elements (stride >= 2^spins), interleaved (re, im), 16-byte aligned.
 * sites: DEVICE int32 [walkers], 0 <= sites[w] <= spins - 2. A walker whose
 *   site lies outside that range is left unchanged, and the device error word
 *   records BG_ERR_INVALID_ARG (read it with bg_check_device_errors).
 * gates: DEVICE, 16 complex per walker, U_w column-major (U[a, c] at a + 4 c).
 * Caller-owned memory, nothing allocated; asynchronous on `stream`. */
bg_status apply_local_gate(bg_dtype dtype, int64_t walkers, int32_t spins, const int32_t* sites,
                           const void* gates, void* states, int64_t stride, bg_stream_t stream);

/* ---- entanglement entropy (Alg. 1, "Calculate Entropy"; Sec. 3) -----------
 * Each Monte Carlo step of the paper computes the entanglement entropy of the
 * new state: the state is reshaped across a cut of the chain, multiplied by
 * its own conjugate transpose (the GEMM of Sec. 3, with the shapes M = 2^(S -
 * floor(S/2)), K = 2^floor(S/2)), and the eigenvalues p_i of the normalised
 * density matrix give S = -sum_i p_i ln p_i.
 *  - The cut: spin i is bit i of the basis index x (as for apply_local_gate);
 *    the lower `split` spins (x mod K, K = 2^split) are one side, the upper
 *    spins (x div K, M = 2^(spins - split) values) the other. The state
 *    vector of walker w is, without a copy, the column-major K x M matrix X_w
 *    (leading dimension K), and G_w = X_w X_w^H (K x K) has the nonzero
 *    eigenvalues of rho_w = Psi Psi^H. p_i = lambda_i(G_w) / sum_j lambda_j.
 *  - entropy_plan: `walkers` complex128 states of 2^spins amplitudes, walker w
 *    at element w * stride (stride >= 2^spins); 2 <= spins <= 30,
 *    1 <= split <= min(spins - 1, 10). precision (NULL = FP64) selects the
 *    precision of G_w: it is formed by a Hermitian-update plan
 *    (BG_PLAN_HERK) in that mode. The eigenvalues come from a Householder
 *    reduction of G_w to a real tridiagonal matrix, then bisection on its
 *    Sturm sequence, in FP64. In split mode with K > 64 the reduction is
 *    blocked: panels of 16 columns in FP64, each followed by its rank-32
 *    trailing update as a grouped complex GEMM in the plan's precision (a
 *    panel kernel, a pack kernel and that GEMM's launches), and the last 64
 *    columns unblocked. flags: 0 or BG_PLAN_PROFILE (slot 0 of
 *    bg_plan_kernel_times: G; slot 1: the eigenvalues and the entropy). The
 *    plan owns a workspace of walkers x K x K complex128 plus 2 walkers x K
 *    doubles, and for the blocked reduction the panels' vectors (walkers x
 *    32 K complex128), the packed operand, walkers x K x K doubles of
 *    Re G + Im G and the GEMM plans' workspace (bg_plan_get_info). Must not
 *    be called during stream capture.
 *  - batched_entropy: states: DEVICE, 16-byte aligned; entropy: DEVICE
 *    double [walkers] (natural logarithm); eigenvalues: DEVICE double
 *    [walkers][K] or NULL: the K eigenvalues of each G_w, ascending, not
 *    normalised. Asynchronous on `stream`; calls on one plan must not overlap. */
bg_status entropy_plan(bg_plan** out, int64_t walkers, int32_t spins, int32_t split,
                       int64_t stride, const bg_precision* precision, uint32_t flags,
                       bg_stream_t stream);

bg_status batched_entropy(const bg_plan* plan, const void* states, double* entropy,
                          double* eigenvalues, bg_stream_t stream);

/* ---- the Metropolis decision and the whole annealing step (Alg. 1) ---------
 * Sec. 3: after the local gate and the new entanglement entropy, each Monte
 * Carlo procedure decides by the Metropolis algorithm ("M.A") whether to keep
 * the new state or the current one, then repeats from the chosen state. The
 * paper names the rule and no more; this library's reading: the energy is
 * the entanglement entropy (or any per-walker energy the caller supplies),
 * and a proposal moving the energy from E_cur to E_new is accepted when
 *   delta = direction * (E_new - E_cur) <= 0,  or else when  u < exp(-delta / T),
 * u being the walker's uniform in [0, 1) drawn by the caller, T >= 0 the
 * temperature of the annealing schedule (T = 0 refuses every uphill move;
 * a NaN energy is never accepted), direction = +1 to lower the energy or
 * -1 to raise it. Computed in FP64.
 *
 * metropolis_select: the decision for `walkers` walkers. uniforms, e_new:
 * DEVICE double [walkers]; e_cur: DEVICE double [walkers], set to e_new where
 * accepted; accepted: DEVICE int32 [walkers], 1 or 0. With amplitudes > 0,
 * the accepted walkers' proposals (DEVICE complex128, walker w at proposals
 * + w * proposal_stride) are copied over their states (states + w *
 * state_stride); amplitudes = 0 decides only (proposals and states may then
 * be NULL). Temperature < 0, direction other than +-1 or a stride below
 * `amplitudes` is BG_ERR_INVALID_ARG. Asynchronous on `stream`. */
bg_status metropolis_select(int64_t walkers, double temperature, int32_t direction,
                            const double* uniforms, const double* e_new, double* e_cur,
                            int32_t* accepted, const void* proposals, int64_t proposal_stride,
                            void* states, int64_t state_stride, int64_t amplitudes,
                            bg_stream_t stream);

/* anneal_plan / anneal_step: one whole step of Alg. 1 for `walkers` complex128
 * states of 2^spins amplitudes (walker w at states + w * stride): each
 * walker's proposal is its state with its local gate applied (as
 * apply_local_gate), the proposal's entanglement entropy across the cut
 * after the lower `split` spins is computed (as batched_entropy, the Gram
 * matrices in `precision`), and metropolis_select keeps or replaces the
 * state. energy: DEVICE double [walkers], the current states' entropies
 * (from batched_entropy before the first step), updated in place; sites:
 * DEVICE int32 [walkers]; gates: DEVICE complex128 [walkers][16] (column-major
 * 4 x 4); uniforms: DEVICE double [walkers]; accepted: DEVICE int32 [walkers].
 * The plan owns the entropy plan and a proposal buffer of walkers x 2^spins
 * complex128. Argument ranges as for entropy_plan and metropolis_select;
 * flags: 0 or BG_PLAN_PROFILE. Asynchronous; calls on one plan must not
 * overlap. */
bg_status anneal_plan(bg_plan** out, int64_t walkers, int32_t spins, int32_t split,
                      int64_t stride, const bg_precision* precision, uint32_t flags,
                      bg_stream_t stream);

bg_status anneal_step(const bg_plan* plan, void* states, double* energy, const int32_t* sites,
                      const void* gates, const double* uniforms, double temperature,
                      int32_t direction, int32_t* accepted, bg_stream_t stream);

/* ---- spreading independent work over GPUs (Sec. 4.B, Table 1) --------------
 * The paper runs its independent Monte Carlo procedures on several GPUs and
 * reports near-linear scaling (Sec. 4.B, Table 1). This host-only call splits
 * `count` independent work items -- GEMM instances of a batch, or whole
 * walkers of a chain -- with costs host_cost[i] >= 0 (e.g. 2 m n k flops of
 * an instance, or steps x 8 n^3 for a complex walker) over `parts` processes
 * by longest processing time first: the items in decreasing cost (equal
 * costs: lower index first) each go to the part with the smallest load so
 * far (equal loads: lower part). The result depends only on the inputs, so
 * every rank computes the same partition. No part's load exceeds the mean
 * load plus the largest single cost.
 * host_cost: HOST double [count]; out_part: HOST int32 [count], the part
 * (0..parts-1) of each item; out_load: HOST double [parts] or NULL, each
 * part's summed cost. A negative or non-finite cost, parts < 1 or a NULL
 * array with count > 0 is BG_ERR_INVALID_ARG. No device work. */
bg_status bg_partition_lpt(int64_t count, const double* host_cost, int32_t parts,
                           int32_t* out_part, double* out_load);

/* Plan introspection: number of instances, of device work items per grouped
 * call, of kernel launches per grouped call (or per chain step), workspace
 * bytes, and the size classes. */
typedef struct {
  int64_t count;
  int64_t work_items;
  int32_t launches_per_call;
  int32_t classes;
  int64_t workspace_bytes;
  int32_t slices;       /* split mode: planes per operand, else 0 */
  int32_t beta_bits;    /* split mode: digit width chosen, else 0 */
} bg_plan_info;

bg_status bg_plan_get_info(const bg_plan* plan, bg_plan_info* out);

/* JSON text describing the per-class programs chosen (autotuned or default)
 * and, when timed, their measured milliseconds. Writes at most `len` bytes
 * including the terminating NUL into `buf`; returns BG_ERR_INVALID_ARG when
 * it does not fit (the required length is then in *needed, if non-NULL). */
bg_status bg_plan_describe(const bg_plan* plan, char* buf, size_t len, size_t* needed);

/* Per-kernel device time of the grouped calls of a plan made with
 * BG_PLAN_PROFILE (Sec. 4 reports per-GEMM performance; this is the
 * library's own per-kernel timing, from CUDA events recorded on the call's
 * stream around each launch). Synchronises on the recorded events and writes,
 * for each kernel slot of one call (slot 0: the FP64 kernel, or the slicer in
 * split mode; slot 1: the split tensor-core tile GEMM, plus the FP64 launch
 * of classes an autotuned split plan gave to the FP64 path; slot 2: the
 * split mode's small-instance kernel), the summed milliseconds over all calls
 * since the last reset into total_ms[0..2] (an array of 3 doubles; unused
 * slots read 0) and the number of calls into *calls. reset = 1 clears the
 * sums after reading. Graph capture is not used while profiling. */
bg_status bg_plan_kernel_times(const bg_plan* plan, int32_t reset, double* total_ms,
                               int64_t* calls);

/* ---- measurement (results of runs; not part of the timed path) --------------
 * Per-instance normwise error of Eq. (1) results, the tolerance measure used
 * for every mode: out[i] = ||C_test_i - C_ref_i||_F / (||A_i||_F ||B_i||_F)
 * (0/0 reported as the numerator). d_table is a DEVICE int64 array
 * [count][9] laid out as bg_instance. Computed in FP64; d_out is a DEVICE
 * double array [count]. */
bg_status bg_rel_err(bg_dtype dtype, int64_t count, const int64_t* d_table, const void* A,
                     const void* B, const void* C_test, const void* C_ref, double* d_out,
                     bg_stream_t stream);

/* Unitarity drift of chained states (the products of Alg. 1 stay unitary in
 * exact arithmetic): out[w] = ||C_w^H C_w - I||_F for each square matrix w of
 * size n[w] at element offset off[w] of C. d_n, d_off: DEVICE int64 [count];
 * d_out: DEVICE double [count]. Computed in FP64. */
bg_status bg_unitarity_drift(bg_dtype dtype, int64_t count, const int64_t* d_n,
                             const int64_t* d_off, const void* C, double* d_out,
                             bg_stream_t stream);

/* ---- split-mode building blocks, exposed so they can be checked alone -------
 * Cuts one real m x k column-major matrix X (leading dimension ldx) into
 * `slices` digit planes, the operand split used by BG_MODE_SPLIT_BF16:
 * axis = 0 scales each ROW r by 2^-e[r] (the A side), axis = 1 each COLUMN c
 * by 2^-e[c] (the B side), e = the exponent of the largest magnitude in that
 * row/column (so that every scaled entry is below 1 in magnitude; 0 for an
 * all-zero line). digits[p] (p = 0..slices-1) is an m x k column-major
 * array of BF16 bit patterns (uint16) at digits + p*m*k holding integers d
 * with |d| <= 2^beta_bits, such that
 *   X[r,c] ~= sum_p d_p[r,c] * 2^(e - beta_bits*(p+1)),
 * the remainder being at most half a unit of the last digit. exps: DEVICE
 * int32 [m] (axis 0) or [k] (axis 1). beta_bits must be 2..8. */
bg_status bg_split_planes(int64_t m, int64_t k, const double* X, int64_t ldx, int32_t axis,
                          int32_t slices, int32_t beta_bits, int32_t* exps, uint16_t* digits,
                          bg_stream_t stream);

/* ---- diagnostics ------------------------------------------------------------
 * Synchronises `stream`, reads and clears the library's device error word of
 * the current device. Returns BG_ERR_TIMEOUT if a bounded wait gave up since
 * the last check (the code of the first such event, with the kernel's
 * location, is in bg_last_error()). */
bg_status bg_check_device_errors(bg_stream_t stream);

/* Launches a kernel that waits on a device flag nobody sets, with a wait
 * bound of `spin_limit` polls; the kernel gives up, records BG_ERR_TIMEOUT in
 * the device error word and exits. Used to test the bounded-wait path. */
bg_status bg_test_bounded_wait(int64_t spin_limit, bg_stream_t stream);

/* Measures this GPU's sustained FP64 arithmetic rate (DFMA, and FP64
 * tensor-core mma when mma_kind = 1) with a register-only kernel on all SMs:
 * the FP64 peak that the paper quotes for its A100 (Sec. 4) is the
 * denominator of the FP64 roofline. Writes TFLOP/s to *tflops (host). */
bg_status bg_probe_fp64_peak(int32_t mma_kind, double* tflops, bg_stream_t stream);

/* Number of kernels this library launched on the current host thread since
 * the last reset (reset = 1 clears it after reading). */
int64_t bg_launch_count(int32_t reset);

const char* bg_status_string(bg_status s);
const char* bg_last_error(void);
const char* bg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BGEMM_H */
