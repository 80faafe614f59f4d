"""Hermitian rank-k updates (plan flag BG_PLAN_HERK): C_i = alpha A_i A_i^H + beta C_i,
the rho = Psi Psi^H product of Sec. 3, lower triangle only.

The oracle computes the full Eq. (1) product with B_i = A_i^H written out
(conjugate transpose is exact), and the test compares the lower triangle; the
strict upper triangle must be left bit for bit as it was, and a complex
diagonal must come out with an imaginary part of exactly zero.
"""
import numpy as np
import pytest

import paper_2203_09353_gb300 as bg
from paper_2203_09353_gb300 import synth

from gpu_util import TOL_FP64, TOL_SPLIT, dev, host, oracle_batch

pytestmark = pytest.mark.gpu

# (n, k) per instance: packed small ones, ragged sizes, the Sec. 3 shape for
# S = 15 spins (M = N = 256, K = 128) and a k long enough for several exact passes
SHAPES = [(16, 16)] * 5 + [(24, 40), (40, 24), (64, 64), (100, 37), (130, 200), (256, 128),
                           (300, 300), (96, 1100)]


def herk_batch(dtype, seed):
    rng = np.random.default_rng(seed)
    shapes = [(n, n, k) for n, k in SHAPES]
    table, la, lb, lc = synth.pack_table(shapes)
    cplx = dtype == "c128"

    def fill(size):
        x = rng.uniform(-1, 1, size)
        return x + 1j * rng.uniform(-1, 1, size) if cplx else x

    A, C = fill(la), fill(lc)
    # B_i = A_i^H, written out for the oracle
    B = np.zeros(lb, dtype=A.dtype)
    for i, (m, n, k, lda, ldb, ldc, ao, bo, co) in enumerate(table):
        a = A[ao:ao + lda * k].reshape(k, lda).T[:m, :]          # m x k
        bh = np.conj(a).T if cplx else a.T                       # k x m
        B[bo:bo + ldb * n] = np.asfortranarray(bh).ravel(order="F")
    return table, A, B, C


def lower_mask(n):
    return np.tril(np.ones((n, n), dtype=bool))


@pytest.mark.parametrize("dtype", ["r64", "c128"])
@pytest.mark.parametrize("mode,s", [("fp64", 0), ("split", 3), ("split", 6), ("split", 9)])
def test_herk_matches_oracle(gpu, dtype, mode, s):
    table, A, B, C = herk_batch(dtype, 11 if dtype == "r64" else 12)
    alpha, beta = 0.75, -0.5
    b = synth.Batch("herk", dtype, table, A, B, C, alpha, beta)
    ref = oracle_batch(b)
    plan = bg.batched_gemm_plan(dtype, table, bg.precision(mode, s), bg.BG_PLAN_HERK)
    Cd = dev(C)
    bg.batched_gemm_grouped(plan, dev(A), None, Cd, alpha, beta)
    got = host(Cd)
    tol = TOL_FP64 if mode == "fp64" else TOL_SPLIT[s]
    for i, (m, n, k, lda, ldb, ldc, ao, bo, co) in enumerate(table):
        g = got[co:co + ldc * n].reshape(n, ldc).T[:m, :]
        r = ref[co:co + ldc * n].reshape(n, ldc).T[:m, :].copy()
        if dtype == "c128":
            # a Hermitian update keeps the diagonal real (its old imaginary parts
            # are taken as zero), where the plain product scales them by beta
            r[np.diag_indices(n)] = np.real(np.diag(r))
        c0 = C[co:co + ldc * n].reshape(n, ldc).T[:m, :]
        low = lower_mask(n)
        a = A[ao:ao + lda * k].reshape(k, lda).T[:m, :]
        err = np.linalg.norm((g - r)[low]) / max(np.linalg.norm(a) ** 2, 1e-300)
        assert err <= tol, (i, n, k, err)
        # strict upper triangle untouched
        assert np.array_equal(g[~low], c0[~low]), i
        if dtype == "c128":
            assert np.all(np.imag(np.diag(g)) == 0.0), i
    plan.close()


def test_herk_rejects_complex_scalars_and_rectangles(gpu):
    table, A, B, C = herk_batch("c128", 3)
    plan = bg.batched_gemm_plan("c128", table, None, bg.BG_PLAN_HERK)
    with pytest.raises(bg.BgemmError) as ei:
        bg.batched_gemm_grouped(plan, dev(A), None, dev(C), 1.0 + 0.5j, 0.0)
    assert ei.value.status == 1
    plan.close()
    bad = table.copy()
    bad[0, 1] += 1  # m != n
    with pytest.raises(bg.BgemmError) as ei:
        bg.batched_gemm_plan("c128", bad, None, bg.BG_PLAN_HERK)
    assert ei.value.status == 1
