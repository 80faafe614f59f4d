"""Pins for the CPU oracle of Eq. (1) (Sec. 2): C_i = alpha A_i B_i + beta C_i.

Nothing here retypes the oracle's formula. Each pin compares it with a value
fixed by something else: exact integer brute force, identity and permutation
matrices, the Pauli multiplication table (the spin operators of Sec. 3,
tests/golden/pauli_products.txt), (AB)^T = B^T A^T, the Kronecker mixed
product, the unitarity of Haar matrices, the BLAS alpha/beta rules and an
independent library (numpy.matmul). ``test_planted_mistakes`` rebuilds the
oracle with one deliberate slip at a time and shows that some pin catches
each one.
"""
import os
import random

import numpy as np
import pytest

import oracle
from paper_2203_09353_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

PAULI = {
    "I": np.eye(2, dtype=np.complex128),
    "x": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


# ---- helpers -------------------------------------------------------------------

def _flat(M):
    return np.asfortranarray(M).ravel(order="F")


def _brute_int(A, B, alpha, beta, C, m, n, k):
    """alpha A B + beta C with Python integers (complex: Gaussian integers)."""
    out = [[None] * n for _ in range(m)]
    for i in range(m):
        for j in range(n):
            s = 0
            for p in range(k):
                s += A[i][p] * B[p][j]
            out[i][j] = alpha * s + beta * C[i][j]
    return out


def _rand_int_matrix(rng, r, c, cplx):
    if cplx:
        return [[complex(rng.randint(-8, 8), rng.randint(-8, 8)) for _ in range(c)] for _ in range(r)]
    return [[rng.randint(-8, 8) for _ in range(c)] for _ in range(r)]


def _to_np(M, r, c, dt):
    a = np.zeros((r, c), dtype=dt)
    for i in range(r):
        for j in range(c):
            a[i, j] = M[i][j]
    return a


# ---- pins: each returns normally or raises AssertionError ----------------------

def pin_brute_force_fixed(lib):
    """Exact integer brute force, fixed-size batches with padded leading dimensions."""
    rng = random.Random(1234)
    for cplx in (False, True):
        dt = np.complex128 if cplx else np.float64
        for trial in range(40):
            m, n, k = rng.randint(0, 4), rng.randint(0, 4), rng.randint(0, 4)
            batch = rng.randint(1, 3)
            lda, ldb, ldc = m + rng.randint(1, 2), k + rng.randint(1, 2), m + rng.randint(1, 2)
            sa, sb, sc = lda * max(k, 1) + 3, ldb * max(n, 1) + 1, ldc * max(n, 1) + 2
            if cplx:
                alpha = complex(rng.randint(-3, 3), rng.randint(-3, 3))
                beta = complex(rng.randint(-3, 3), rng.randint(-3, 3))
            else:
                alpha, beta = rng.randint(-3, 3), rng.randint(-3, 3)
            if trial % 7 == 0:
                alpha = 0
            if trial % 5 == 0:
                beta = 0
            A = np.full(sa * batch, 7777, dtype=dt)
            B = np.full(sb * batch, 7777, dtype=dt)
            C = np.full(sc * batch, 7777, dtype=dt)
            expect = []
            for b in range(batch):
                Ai, Bi, Ci = (_rand_int_matrix(rng, m, k, cplx), _rand_int_matrix(rng, k, n, cplx),
                              _rand_int_matrix(rng, m, n, cplx))
                for M, X, off, ld, r, c in ((Ai, A, b * sa, lda, m, k), (Bi, B, b * sb, ldb, k, n),
                                            (Ci, C, b * sc, ldc, m, n)):
                    for i in range(r):
                        for j in range(c):
                            X[off + i + j * ld] = M[i][j]
                expect.append(_brute_int(Ai, Bi, alpha, beta, Ci, m, n, k))
            C_before = C.copy()
            oracle.gemm_fixed(m, n, k, alpha, A, lda, sa, B, ldb, sb, beta, C, ldc, sc, batch, lib=lib)
            for b in range(batch):
                for i in range(m):
                    for j in range(n):
                        got = C[b * sc + i + j * ldc]
                        assert got == expect[b][i][j], (cplx, trial, b, i, j, got, expect[b][i][j])
            # padding rows (ld > m) and inter-instance gaps are untouched
            mask = np.ones(C.size, dtype=bool)
            for b in range(batch):
                for j in range(n):
                    mask[b * sc + j * ldc: b * sc + j * ldc + m] = False
            assert np.array_equal(C[mask], C_before[mask])


def pin_brute_force_grouped(lib):
    """Exact integer brute force through the variable-size (grouped) entry points."""
    rng = random.Random(99)
    for cplx in (False, True):
        dt = np.complex128 if cplx else np.float64
        shapes = [(rng.randint(0, 5), rng.randint(0, 5), rng.randint(0, 5)) for _ in range(25)]
        table, la, lb, lc = synth.pack_table(shapes, align=3)
        A, B, C = (np.zeros(x, dtype=dt) for x in (la, lb, lc))
        alpha = complex(2, -1) if cplx else 3
        beta = complex(-1, 2) if cplx else -2
        expect = []
        for idx, (m, n, k) in enumerate(shapes):
            Ai, Bi, Ci = (_rand_int_matrix(rng, m, k, cplx), _rand_int_matrix(rng, k, n, cplx),
                          _rand_int_matrix(rng, m, n, cplx))
            _, _, _, lda, ldb, ldc, ao, bo, co = table[idx]
            for M, X, off, ld, r, c in ((Ai, A, ao, lda, m, k), (Bi, B, bo, ldb, k, n),
                                        (Ci, C, co, ldc, m, n)):
                for i in range(r):
                    for j in range(c):
                        X[off + i + j * ld] = M[i][j]
            expect.append(_brute_int(Ai, Bi, alpha, beta, Ci, m, n, k))
        oracle.gemm_grouped(table, alpha, A, B, beta, C, lib=lib)
        for idx, (m, n, k) in enumerate(shapes):
            ldc, co = table[idx, 5], table[idx, 8]
            for i in range(m):
                for j in range(n):
                    assert C[co + i + j * ldc] == expect[idx][i][j]


def pin_identity_permutation(lib):
    """A I = A, I B = B and P B = B with rows permuted, bit for bit (real and complex)."""
    rng = np.random.default_rng(5)
    for dt in (np.float64, np.complex128):
        for n in (1, 3, 8, 33):
            A = rng.standard_normal((n, n))
            if dt == np.complex128:
                A = A + 1j * rng.standard_normal((n, n))
            I = np.eye(n, dtype=dt)
            assert np.array_equal(oracle.matmul(A, I, lib=lib), A)
            assert np.array_equal(oracle.matmul(I, A, lib=lib), A)
            perm = rng.permutation(n)
            P = I[perm]
            assert np.array_equal(oracle.matmul(P, A, lib=lib), A[perm])
            assert np.array_equal(oracle.matmul(A, P.T, lib=lib), A[:, perm])
            # a rectangular slice of the identity selects columns
            if n > 2:
                E = I[:, :2]
                assert np.array_equal(oracle.matmul(A, E, lib=lib), A[:, :2])


def _golden_pauli():
    rows = []
    with open(os.path.join(GOLDEN, "pauli_products.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            lhs, rhs = line.split("=")
            a, b = lhs.split()
            coef, res = rhs.split()
            re, im = (float(x) for x in coef.split(","))
            rows.append((a, b, complex(re, im), res))
    return rows


def pin_pauli(lib):
    """sigma_a sigma_b from the golden table, and its Kronecker lifts to 2^N, exactly."""
    rows = _golden_pauli()
    assert len(rows) == 9
    for a, b, coef, res in rows:
        got = oracle.matmul(PAULI[a], PAULI[b], lib=lib)
        assert np.array_equal(got, coef * PAULI[res]), (a, b, got)
    # lifts to a 3-spin chain: (s_a x s_b x I)(s_c x s_d x s_e) = (s_a s_c) x (s_b s_d) x s_e
    table = {(a, b): (coef, res) for a, b, coef, res in rows}
    for (a, b, c, d) in (("x", "y", "y", "z"), ("z", "x", "x", "x"), ("y", "y", "z", "x"),
                         ("x", "z", "y", "y")):
        lhs = np.kron(np.kron(PAULI[a], PAULI[b]), PAULI["I"])
        for e in ("x", "y", "z"):
            rhs = np.kron(np.kron(PAULI[c], PAULI[d]), PAULI[e])
            c1, r1 = table[(a, c)]
            c2, r2 = table[(b, d)]
            want = (c1 * c2) * np.kron(np.kron(PAULI[r1], PAULI[r2]), PAULI[e])
            assert np.array_equal(oracle.matmul(lhs, rhs, lib=lib), want)


def pin_transpose(lib):
    """(A B)^T == B^T A^T bit for bit on random rectangular operands."""
    rng = np.random.default_rng(7)
    for dt in (np.float64, np.complex128):
        for (m, n, k) in ((5, 7, 3), (16, 9, 31), (1, 4, 2)):
            A = rng.uniform(-1, 1, (m, k))
            B = rng.uniform(-1, 1, (k, n))
            if dt == np.complex128:
                A = A + 1j * rng.uniform(-1, 1, (m, k))
                B = B + 1j * rng.uniform(-1, 1, (k, n))
            left = oracle.matmul(A, B, lib=lib).T
            right = oracle.matmul(B.T.copy(), A.T.copy(), lib=lib)
            assert np.array_equal(left, right)


def pin_kronecker(lib):
    """(A x B)(C x D) = (AC) x (BD): exact on integers, 1e-15 relative on floats."""
    rng = np.random.default_rng(11)
    for dt in (np.float64, np.complex128):
        A, C = rng.integers(-5, 6, (3, 4)), rng.integers(-5, 6, (4, 2))
        B, D = rng.integers(-5, 6, (2, 3)), rng.integers(-5, 6, (3, 5))
        if dt == np.complex128:
            A = A + 1j * rng.integers(-5, 6, (3, 4))
            D = D + 1j * rng.integers(-5, 6, (3, 5))
        lhs = oracle.matmul(np.kron(A, B).astype(dt), np.kron(C, D).astype(dt), lib=lib)
        rhs = np.kron(oracle.matmul(A.astype(dt), C.astype(dt), lib=lib),
                      oracle.matmul(B.astype(dt), D.astype(dt), lib=lib))
        assert np.array_equal(lhs, rhs)
        Af, Bf, Cf, Df = (rng.uniform(-1, 1, s) for s in ((4, 4), (3, 3), (4, 4), (3, 3)))
        lhs = oracle.matmul(np.kron(Af, Bf), np.kron(Cf, Df), lib=lib)
        rhs = np.kron(oracle.matmul(Af, Cf, lib=lib), oracle.matmul(Bf, Df, lib=lib))
        assert np.linalg.norm(lhs - rhs) <= 1e-15 * np.linalg.norm(rhs) * 4


def pin_unitary(lib):
    """Q^H Q = I to 1e-14 for Haar unitaries of the chain workload."""
    rng = np.random.default_rng(13)
    for n in (2, 16, 64):
        for Q in synth.haar_unitary(rng, n, 3):
            assert oracle.unitarity_drift(Q, lib=lib) <= 1e-14 * n
        assert oracle.unitarity_drift(2.0 * synth.haar_unitary(rng, n, 1)[0], lib=lib) > 1.0


def pin_alpha_beta_rules(lib):
    """beta == 0 never reads C (NaN stays out); alpha == 0 never reads A or B."""
    rng = np.random.default_rng(17)
    for dt in (np.float64, np.complex128):
        m, n, k = 4, 3, 5
        A = _flat(rng.uniform(-1, 1, (m, k)).astype(dt))
        B = _flat(rng.uniform(-1, 1, (k, n)).astype(dt))
        C = np.full(m * n, np.nan, dtype=dt)
        oracle.gemm_fixed(m, n, k, 2.0, A, m, m * k, B, k, k * n, 0.0, C, m, m * n, 1, lib=lib)
        assert np.all(np.isfinite(C))
        want = 2.0 * oracle.matmul(A.reshape((k, m)).T, B.reshape((n, k)).T, lib=lib)
        assert np.array_equal(C.reshape((n, m)).T, want)
        An = np.full(m * k, np.nan, dtype=dt)
        Bn = np.full(k * n, np.inf, dtype=dt)
        C2 = _flat(rng.uniform(-1, 1, (m, n)).astype(dt))
        C2_before = C2.copy()
        oracle.gemm_fixed(m, n, k, 0.0, An, m, m * k, Bn, k, k * n, 0.5, C2, m, m * n, 1, lib=lib)
        assert np.array_equal(C2, 0.5 * C2_before)


def pin_numpy_crosscheck(lib):
    """Normwise agreement with numpy.matmul (an independent BLAS) to 1e-14."""
    rng = np.random.default_rng(19)
    for dt in (np.float64, np.complex128):
        for (m, n, k) in ((32, 32, 32), (17, 40, 63), (64, 8, 128)):
            A = rng.uniform(-1, 1, (m, k))
            B = rng.uniform(-1, 1, (k, n))
            if dt == np.complex128:
                A = A + 1j * rng.uniform(-1, 1, (m, k))
                B = B + 1j * rng.uniform(-1, 1, (k, n))
            err = np.linalg.norm(oracle.matmul(A, B, lib=lib) - A @ B)
            assert err <= 1e-14 * np.linalg.norm(A) * np.linalg.norm(B)


PINS = [pin_brute_force_fixed, pin_brute_force_grouped, pin_identity_permutation, pin_pauli,
        pin_transpose, pin_kronecker, pin_unitary, pin_alpha_beta_rules, pin_numpy_crosscheck]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin, oracle_lib):
    pin(oracle_lib)


@pytest.mark.parametrize("mutant", list(range(1, 9)))
def test_planted_mistakes(mutant, tmp_path):
    """Each planted mistake in the oracle makes at least one pin fail."""
    lib = oracle.load(mutant=mutant, out_dir=str(tmp_path))
    failed = []
    for pin in PINS:
        try:
            pin(lib)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"mutant {mutant} passed every pin"


def test_shape_formula_sec3():
    """Operator sizes of Sec. 3: M = N = 2^(S - floor(S/2)), K = 2^floor(S/2).

    S = 15 gives the 256 x 128 operands quoted in Sec. 4.A; the synthetic
    configurations use square powers of two of the same family."""
    def shape(S):
        return 2 ** (S - S // 2), 2 ** (S // 2)
    assert shape(15) == (256, 128)
    assert shape(21) == (2048, 1024)
    assert shape(23) == (4096, 2048)


def test_synth_config_shapes():
    b1 = synth.fixed_real_n32()
    assert b1.count == 64 and b1.fixed_shape() == (32, 32, 32, 64)
    assert np.all(np.abs(b1.A) <= 1.0)
    b2 = synth.hermitian_unitary_c128(batch=8)
    for i in range(8):
        A = b2.instance(i, "A")
        assert np.array_equal(A, np.conj(A.T))
        U = b2.instance(i, "B")
        assert np.linalg.norm(np.conj(U.T) @ U - np.eye(64)) < 1e-13
    b3 = synth.size_mix_uniform(count=300)
    ns = b3.table[:, 0]
    assert set(np.unique(ns)).issubset(set(synth.SIZE_MIX_SIZES))
    assert np.all(b3.table[:, 6] % synth.ALIGN_ELEMS == 0)
    b4 = synth.size_mix_loguniform(count=50)
    mags = np.abs(b4.A[b4.A != 0])
    assert mags.min() >= 1e-4 * (1 - 1e-12) and mags.max() <= 1e4 * (1 + 1e-12)
    assert (b4.A < 0).any() and (b4.A > 0).any()
    ch = synth.annealing_chain(walkers_small=3, walkers_large=1, n_small=8, n_large=16, steps=5,
                       pool_small=4, pool_large=2)
    assert ch.idx.shape == (5, 4)
    assert ch.idx[:, :3].max() < 4 and ch.idx[:, 3].max() < 2


def test_chain_layout_round_trip():
    """The packed chain (pool, states, global index table) gives back every
    pool entry, start state and per-step operator it was built from."""
    ch = synth.annealing_chain(walkers_small=3, walkers_large=2, n_small=8, n_large=16, steps=4,
                               pool_small=5, pool_large=3)
    pool, pool_n, pool_off, states, state_off, gidx = synth.chain_layout(ch)
    assert gidx.shape == ch.idx.shape and gidx.dtype == np.int32
    assert pool.size == int(np.sum(pool_n * pool_n)) and states.size == int(np.sum(ch.n_walker ** 2))

    def entry(j):
        n = int(pool_n[j])
        return pool[pool_off[j]:pool_off[j] + n * n].reshape(n, n).T

    for w in range(ch.walkers):
        n = int(ch.n_walker[w])
        got = states[state_off[w]:state_off[w] + n * n].reshape(n, n).T
        assert np.array_equal(got, ch.C0[w])
        for t in range(ch.steps):
            j = int(gidx[t, w])
            assert pool_n[j] == n
            assert np.array_equal(entry(j), ch.pools[n][ch.idx[t, w]])
