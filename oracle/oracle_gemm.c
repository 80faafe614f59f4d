/*
 * CPU oracle for the batched GEMM of Eq. (1) (Sec. 2):
 *
 *     C_i = alpha * A_i * B_i + beta * C_i,   i = 1..N,
 *     A_i in F^{m x k}, B_i in F^{k x n}, C_i in F^{m x n},  F = R (FP64) or C (complex128).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * definition against which the GPU library is checked. Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * library never calls it, and it shares no code, header or constant with the
 * GPU path.
 *
 * Conventions (the definition written out, nothing more):
 *  - every matrix is column-major: element (r, c) of a matrix with leading
 *    dimension ld sits at offset r + c * ld (in elements);
 *  - complex128 is interleaved (re, im), so element e of a complex array is
 *    the double pair [2e], [2e+1];
 *  - the inner sum runs over p = 0, 1, ..., k-1 in increasing order, one
 *    multiply and one add per term (built with -ffp-contract=off, so no
 *    fused multiply-add can change the rounding);
 *  - complex products use the classical four real products:
 *    (ar*br - ai*bi, ar*bi + ai*br), the two parts accumulated separately;
 *  - BLAS scalar rules: when beta == 0 the old C is not read (so NaN/Inf in
 *    C do not propagate); when alpha == 0 neither A nor B is read.
 *
 * The loop over instances is shared out over OpenMP threads; this changes no
 * arithmetic (each output element is computed by one thread in the order
 * above).
 *
 * Planted mistakes: compiling with -DORACLE_MUTANT=<n> (n = 1..8) swaps in one
 * deliberate error. Only the oracle's own pin tests build these variants, to
 * show that each kind of slip is caught by at least one pin.
 */
#include <stdint.h>
#include <stddef.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

/* Index of element (r, c) in a column-major matrix with leading dimension ld. */
static inline int64_t cm(int64_t r, int64_t c, int64_t ld) {
#if ORACLE_MUTANT == 3
  /* planted: operands read transposed */
  return c + r * ld;
#else
  return r + c * ld;
#endif
}

/* One real instance of Eq. (1). */
static void gemm_r64_one(int64_t m, int64_t n, int64_t k, double alpha,
                         const double* A, int64_t lda, const double* B, int64_t ldb,
                         double beta, double* C, int64_t ldc) {
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < m; ++i) {
      double r = 0.0;
      if (alpha != 0.0) {
        double acc = 0.0;
#if ORACLE_MUTANT == 1
        /* planted: last term of the inner sum dropped */
        for (int64_t p = 0; p + 1 < k; ++p) acc += A[cm(i, p, lda)] * B[cm(p, j, ldb)];
#else
        for (int64_t p = 0; p < k; ++p) acc += A[cm(i, p, lda)] * B[cm(p, j, ldb)];
#endif
#if ORACLE_MUTANT == 6
        r = acc; /* planted: alpha ignored */
#else
        r = alpha * acc;
#endif
      }
#if ORACLE_MUTANT == 4
      /* planted: beta term ignored */
#else
      if (beta != 0.0) r += beta * C[i + j * ldc];
#endif
      C[i + j * ldc] = r;
    }
  }
}

/* One complex instance of Eq. (1); all scalars and arrays interleaved (re, im). */
static void gemm_c128_one(int64_t m, int64_t n, int64_t k, const double alpha[2],
                          const double* A, int64_t lda, const double* B, int64_t ldb,
                          const double beta[2], double* C, int64_t ldc) {
  const int alpha_zero = (alpha[0] == 0.0 && alpha[1] == 0.0);
  const int beta_zero = (beta[0] == 0.0 && beta[1] == 0.0);
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < m; ++i) {
      double rr = 0.0, ri = 0.0;
      if (!alpha_zero) {
        double acc_re = 0.0, acc_im = 0.0;
        for (int64_t p = 0; p < k; ++p) {
          const int64_t ea = cm(i, p, lda), eb = cm(p, j, ldb);
          const double ar = A[2 * ea], ai = A[2 * ea + 1];
          const double br = B[2 * eb], bi = B[2 * eb + 1];
#if ORACLE_MUTANT == 2
          const double t_re = ar * br - ai * bi;
          const double t_im = ar * bi - ai * br; /* planted: wrong sign */
#elif ORACLE_MUTANT == 5
          const double t_re = ar * br + ai * bi; /* planted: conjugated operand */
          const double t_im = ar * bi + ai * br;
#elif ORACLE_MUTANT == 7
          const double t_re = ar * br; /* planted: imaginary-imaginary term dropped */
          const double t_im = ar * bi + ai * br;
#else
          const double t_re = ar * br - ai * bi;
          const double t_im = ar * bi + ai * br;
#endif
          acc_re += t_re;
          acc_im += t_im;
        }
#if ORACLE_MUTANT == 8
        rr = alpha[0] * acc_re; /* planted: imaginary part of alpha ignored */
        ri = alpha[0] * acc_im;
#else
        rr = alpha[0] * acc_re - alpha[1] * acc_im;
        ri = alpha[0] * acc_im + alpha[1] * acc_re;
#endif
      }
      if (!beta_zero) {
        const double cr = C[2 * (i + j * ldc)], ci = C[2 * (i + j * ldc) + 1];
        rr += beta[0] * cr - beta[1] * ci;
        ri += beta[0] * ci + beta[1] * cr;
      }
      C[2 * (i + j * ldc)] = rr;
      C[2 * (i + j * ldc) + 1] = ri;
    }
  }
}

/* ---- exported entry points (ctypes) ---------------------------------------- */

/* Number of threads the instance loop may use (OpenMP), 1 without OpenMP. */
int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* Fixed-size batch (Sec. 2, the contiguous equal-size batch): instance i uses
 * A + i*strideA, B + i*strideB, C + i*strideC (strides in elements). */
void oracle_gemm_r64(int64_t m, int64_t n, int64_t k, double alpha,
                     const double* A, int64_t lda, int64_t strideA,
                     const double* B, int64_t ldb, int64_t strideB, double beta,
                     double* C, int64_t ldc, int64_t strideC, int64_t batch) {
  int64_t b;
#pragma omp parallel for schedule(dynamic, 1)
  for (b = 0; b < batch; ++b)
    gemm_r64_one(m, n, k, alpha, A + b * strideA, lda, B + b * strideB, ldb, beta,
                 C + b * strideC, ldc);
}

void oracle_gemm_c128(int64_t m, int64_t n, int64_t k, const double* alpha,
                      const double* A, int64_t lda, int64_t strideA,
                      const double* B, int64_t ldb, int64_t strideB, const double* beta,
                      double* C, int64_t ldc, int64_t strideC, int64_t batch) {
  int64_t b;
#pragma omp parallel for schedule(dynamic, 1)
  for (b = 0; b < batch; ++b)
    gemm_c128_one(m, n, k, alpha, A + 2 * b * strideA, lda, B + 2 * b * strideB, ldb, beta,
                  C + 2 * b * strideC, ldc);
}

/* Variable-size batch (Sec. 2, the "vbatched" form): row i of `table` holds
 * nine int64 values m, n, k, lda, ldb, ldc, a_off, b_off, c_off (offsets in
 * elements from the three base pointers). */
void oracle_gemm_grouped_r64(int64_t count, const int64_t* table, double alpha,
                             const double* A, const double* B, double beta, double* C) {
  int64_t i;
#pragma omp parallel for schedule(dynamic, 1)
  for (i = 0; i < count; ++i) {
    const int64_t* t = table + 9 * i;
    gemm_r64_one(t[0], t[1], t[2], alpha, A + t[6], t[3], B + t[7], t[4], beta, C + t[8], t[5]);
  }
}

void oracle_gemm_grouped_c128(int64_t count, const int64_t* table, const double* alpha,
                              const double* A, const double* B, const double* beta,
                              double* C) {
  int64_t i;
#pragma omp parallel for schedule(dynamic, 1)
  for (i = 0; i < count; ++i) {
    const int64_t* t = table + 9 * i;
    gemm_c128_one(t[0], t[1], t[2], alpha, A + 2 * t[6], t[3], B + 2 * t[7], t[4], beta,
                  C + 2 * t[8], t[5]);
  }
}
