/*
 * CPU oracle for the local two-spin gate of the annealing step (Sec. 2,
 * "Apply Local Gate": a unitary on a neighbouring pair of spins of the
 * state). The paper names the operation without writing it out; the reading
 * used here is the usual action of a two-site unitary on a state vector:
 *
 *     psi'[x] = sum_{c=0..3} U[a(x), c] * psi[x - a(x) 2^j + c 2^j],
 *     a(x) = b_j(x) + 2 b_{j+1}(x),
 *
 * with b_i(x) bit i of the basis index x (spin i), j the lower spin of the
 * pair (0 <= j <= S - 2) and psi of 2^S amplitudes. U is 4 x 4 complex,
 * column-major (U[a, c] at a + 4 c), interleaved (re, im).
 *
 * TEST INFRASTRUCTURE ONLY, like oracle_gemm.c: the plain definition, a loop
 * over x with the c sum in increasing order, one multiply and one add per real
 * term (built with -ffp-contract=off). It shares no code with the GPU path.
 *
 * Planted mistakes (ORACLE_MUTANT): 9 reads U transposed, 10 takes the two
 * spins in the opposite order, 11 conjugates U.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

/* Local index of spins (j, j+1) in x, and the index of the basis state with
 * those two spins set to local value c. */
static inline int local_index(int64_t x, int j) {
#if ORACLE_MUTANT == 10
  return 2 * (int)((x >> j) & 1) + (int)((x >> (j + 1)) & 1);
#else
  return (int)((x >> j) & 1) + 2 * (int)((x >> (j + 1)) & 1);
#endif
}

static inline int64_t with_local(int64_t x, int j, int c) {
  const int64_t cleared = x & ~((int64_t)3 << j);
#if ORACLE_MUTANT == 10
  return cleared | ((int64_t)(c >> 1) << j) | ((int64_t)(c & 1) << (j + 1));
#else
  return cleared | ((int64_t)c << j);
#endif
}

/* Element U[a, c] of the column-major 4 x 4 gate (as re, im). */
static inline void gate_elem(const double* u, int a, int c, double* re, double* im) {
#if ORACLE_MUTANT == 9
  const int e = c + 4 * a;
#else
  const int e = a + 4 * c;
#endif
  *re = u[2 * e];
#if ORACLE_MUTANT == 11
  *im = -u[2 * e + 1];
#else
  *im = u[2 * e + 1];
#endif
}

/* One walker: psi (2^S complex amplitudes) updated in place. Returns 0, or -1
 * for a site outside 0..S-2 or an allocation failure (psi untouched). */
static int gate_one(int S, int j, const double* u, double* psi) {
  if (S < 2 || S > 40 || j < 0 || j > S - 2) return -1;
  const int64_t dim = (int64_t)1 << S;
  double* old = (double*)malloc((size_t)(2 * dim) * sizeof(double));
  if (!old) return -1;
  memcpy(old, psi, (size_t)(2 * dim) * sizeof(double));
  for (int64_t x = 0; x < dim; ++x) {
    const int a = local_index(x, j);
    double sr = 0.0, si = 0.0;
    for (int c = 0; c < 4; ++c) {
      const int64_t xc = with_local(x, j, c);
      double ur, ui;
      gate_elem(u, a, c, &ur, &ui);
      const double pr = old[2 * xc], pi = old[2 * xc + 1];
      sr += ur * pr - ui * pi;
      si += ur * pi + ui * pr;
    }
    psi[2 * x] = sr;
    psi[2 * x + 1] = si;
  }
  free(old);
  return 0;
}

/* Batch of walkers: walker w's state starts at psi + 2 w stride (stride in
 * complex elements, >= 2^S), its lower spin is site[w] and its gate is
 * gates + 32 w. Returns the number of walkers it refused (bad site). */
int64_t oracle_two_site_gate_c128(int64_t walkers, int32_t S, const int32_t* site,
                                  const double* gates, double* psi, int64_t stride) {
  int64_t bad = 0;
  int64_t w;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
  for (w = 0; w < walkers; ++w)
    if (gate_one(S, site[w], gates + 32 * w, psi + 2 * w * stride) != 0) ++bad;
  return bad;
}
