"""Pins of the oracle for the local two-spin gate (Sec. 2, "Apply Local Gate").

The oracle (oracle/oracle_gate.c) applies a 4 x 4 unitary U to spins (j, j+1)
of each walker's state vector: psi'[x] = sum_c U[a(x), c] psi[x with the two
spins set to c], a(x) = b_j + 2 b_{j+1}. These pins fix it against things it
does not compute itself:

* the dense operator I (x) U (x) I built with numpy.kron and applied with
  numpy's matmul (an independent library), for every site of small chains;
* permutation gates, bit for bit: the identity, SWAP (exchanges spins j and
  j+1), and X on either spin (flips that bit of every basis index);
* U followed by U^H gives the state back, and a Haar U keeps the norm;
* a site outside 0..S-2 is refused.

Each planted mistake of ``ORACLE_MUTANT`` 9-11 (U transposed, the two spins in
the opposite order, U conjugated) fails at least one pin.
"""
import numpy as np
import pytest

import oracle

X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
I2 = np.eye(2, dtype=np.complex128)
SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


def _haar4(rng):
    z = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def _states(rng, W, S):
    return rng.standard_normal((W, 1 << S)) + 1j * rng.standard_normal((W, 1 << S))


def pin_dense_kronecker(lib):
    """Every site of chains of 2..7 spins against (I (x) U (x) I) psi from numpy."""
    rng = np.random.default_rng(31)
    for S in range(2, 8):
        sites = np.arange(S - 1, dtype=np.int32)
        W = len(sites)
        psi = _states(rng, W, S)
        U = rng.standard_normal((W, 4, 4)) + 1j * rng.standard_normal((W, 4, 4))
        got = oracle.two_site_gate(psi, S, sites, U, lib=lib)
        for w, j in enumerate(sites):
            M = np.kron(np.kron(np.eye(1 << (S - j - 2)), U[w]), np.eye(1 << j))
            want = M @ psi[w]
            assert np.linalg.norm(got[w] - want) <= 1e-14 * np.linalg.norm(U[w]) * np.linalg.norm(psi[w])


def pin_permutation_gates(lib):
    """Identity, SWAP and X on either spin move amplitudes without arithmetic."""
    rng = np.random.default_rng(32)
    S = 6
    x = np.arange(1 << S)
    for j in range(S - 1):
        psi = _states(rng, 1, S)
        same = oracle.two_site_gate(psi, S, [j], np.eye(4)[None], lib=lib)
        assert np.array_equal(same, psi)
        bj, bk = (x >> j) & 1, (x >> (j + 1)) & 1
        swapped = x - (bj << j) - (bk << (j + 1)) + (bk << j) + (bj << (j + 1))
        got = oracle.two_site_gate(psi, S, [j], SWAP[None], lib=lib)
        assert np.array_equal(got[0], psi[0][swapped])
        # X on spin j+1: U = X (x) I in the local basis a = b_j + 2 b_{j+1}
        got = oracle.two_site_gate(psi, S, [j], np.kron(X, I2)[None], lib=lib)
        assert np.array_equal(got[0], psi[0][x ^ (1 << (j + 1))])
        got = oracle.two_site_gate(psi, S, [j], np.kron(I2, X)[None], lib=lib)
        assert np.array_equal(got[0], psi[0][x ^ (1 << j)])


def pin_unitary_round_trip(lib):
    """U then U^H restores the state; a Haar U keeps its norm."""
    rng = np.random.default_rng(33)
    S, W = 9, 5
    psi = _states(rng, W, S)
    sites = rng.integers(0, S - 1, W).astype(np.int32)
    U = np.stack([_haar4(rng) for _ in range(W)])
    once = oracle.two_site_gate(psi, S, sites, U, lib=lib)
    back = oracle.two_site_gate(once, S, sites, np.conj(U.transpose(0, 2, 1)), lib=lib)
    for w in range(W):
        n0 = np.linalg.norm(psi[w])
        assert abs(np.linalg.norm(once[w]) - n0) <= 1e-14 * n0
        assert np.linalg.norm(back[w] - psi[w]) <= 1e-14 * n0


def pin_bad_site(lib):
    """A site outside 0..S-2 is refused, not applied."""
    psi = np.ones((1, 8), dtype=np.complex128)
    for j in (-1, 2, 7):
        with pytest.raises(ValueError):
            oracle.two_site_gate(psi, 3, [j], np.eye(4)[None], lib=lib)


PINS = [pin_dense_kronecker, pin_permutation_gates, pin_unitary_round_trip, pin_bad_site]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_gate_pin(pin, oracle_lib):
    pin(oracle_lib)


@pytest.mark.parametrize("mutant", [9, 10, 11])
def test_gate_planted_mistakes(mutant, tmp_path):
    """Each planted mistake in the gate oracle makes at least one pin fail."""
    lib = oracle.load(mutant=mutant, out_dir=str(tmp_path))
    failed = []
    for pin in PINS:
        try:
            pin(lib)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"mutant {mutant} passed every pin"
