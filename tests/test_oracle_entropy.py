"""Pins of the entropy oracle (Sec. 2, Alg. 1 "Calculate Entropy"):
rho = Psi Psi^H of the state reshaped across the cut, its spectrum, and
-sum p ln p. The pins use what fixes the entropy without the oracle's route:

* states built from chosen Schmidt coefficients, Psi = U diag(sqrt(p)) V^H
  with Haar U and V: the entropy is -sum p ln p of the chosen p;
* product states have entropy 0, maximally entangled ones ln(min(M, K));
* local unitaries on either side leave it unchanged, and so does the
  normalisation of the state;
* the singular values of Psi (numpy's SVD, another library routine) give
  the same value.
"""
import numpy as np

import oracle


def haar(rng, n):
    z = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def from_schmidt(rng, p, M, K):
    """State whose M x K reshape has squared singular values p (sum 1)."""
    r = len(p)
    U = haar(rng, M)[:, :r]
    V = haar(rng, K)[:, :r]
    P = U @ np.diag(np.sqrt(p)) @ np.conj(V.T)
    return P.reshape(-1)


def test_schmidt_spectrum_closed_form():
    rng = np.random.default_rng(60)
    for S in (2, 5, 8, 11):
        M, K = 1 << (S - S // 2), 1 << (S // 2)
        r = min(M, K)
        p = rng.random(r) ** 3
        p /= p.sum()
        psi = from_schmidt(rng, p, M, K)
        want = float(-np.sum(p * np.log(p)))
        assert abs(oracle.entanglement_entropy(psi, S) - want) <= 1e-12 * max(1.0, want)


def test_product_and_maximally_entangled():
    rng = np.random.default_rng(61)
    S = 8
    M, K = 1 << (S - S // 2), 1 << (S // 2)
    a = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    b = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    assert abs(oracle.entanglement_entropy(np.outer(a, b).reshape(-1), S)) <= 1e-12
    psi = from_schmidt(rng, np.full(min(M, K), 1.0 / min(M, K)), M, K)
    assert abs(oracle.entanglement_entropy(psi, S) - np.log(min(M, K))) <= 1e-12


def test_local_unitaries_and_scale_leave_it_unchanged():
    rng = np.random.default_rng(62)
    S = 9
    M, K = 1 << (S - S // 2), 1 << (S // 2)
    psi = rng.standard_normal(M * K) + 1j * rng.standard_normal(M * K)
    s0 = oracle.entanglement_entropy(psi, S)
    P = psi.reshape(M, K)
    moved = (haar(rng, M) @ P @ haar(rng, K)).reshape(-1)
    assert abs(oracle.entanglement_entropy(moved, S) - s0) <= 1e-11
    assert abs(oracle.entanglement_entropy(3.5 * psi, S) - s0) <= 1e-11


def test_matches_singular_values():
    rng = np.random.default_rng(63)
    for S, split in ((6, 3), (7, 2), (10, 5)):
        M, K = 1 << (S - split), 1 << split
        psi = rng.standard_normal(M * K) + 1j * rng.standard_normal(M * K)
        sv = np.linalg.svd(psi.reshape(M, K), compute_uv=False)
        p = sv ** 2 / np.sum(sv ** 2)
        p = p[p > 0]
        want = float(-np.sum(p * np.log(p)))
        assert abs(oracle.entanglement_entropy(psi, S, split) - want) <= 1e-11


def test_cut_position_for_odd_spin_count():
    """Odd S: the two halvings differ, and the oracle takes the cut between spins
    split-1 and split (split = floor(S/2); lower spins = low bits of the basis
    index). A Bell pair on spins 1 and 2 of a 5-spin product state straddles
    that cut (entropy ln 2) but not the other halving, between spins 2 and 3
    (entropy 0). Built amplitude by amplitude, without the oracle's route."""
    rng = np.random.default_rng(64)
    S = 5
    one = [rng.standard_normal(2) + 1j * rng.standard_normal(2) for _ in range(3)]
    one = [v / np.linalg.norm(v) for v in one]
    psi = np.zeros(1 << S, dtype=np.complex128)
    for x in range(1 << S):
        b = [(x >> i) & 1 for i in range(S)]
        if b[1] == b[2]:
            psi[x] = one[0][b[0]] * one[1][b[3]] * one[2][b[4]] / np.sqrt(2.0)
    assert abs(oracle.entanglement_entropy(psi, S) - np.log(2.0)) <= 1e-12
    # the other halving (3 lower spins) is the product cut
    assert abs(oracle.entanglement_entropy(psi, S, split=3)) <= 1e-12
    # the column-major K x M view of the vector is Psi^T: same spectrum of X X^H
    K, M = 1 << (S // 2), 1 << (S - S // 2)
    X = psi.reshape(M, K).T
    lam = np.linalg.eigvalsh(X @ np.conj(X.T))
    assert np.allclose(np.sort(lam)[-2:], [0.5, 0.5], atol=1e-12)


def test_schmidt_spectrum_at_the_blocked_sizes():
    """The closed form at the cut sizes the GPU's blocked reduction is tested
    on (K = 256 and 512 columns of the Gram matrix), with a full and a
    rank-deficient spectrum."""
    rng = np.random.default_rng(61)
    for S, split in ((17, 8), (19, 9)):
        M, K = 1 << (S - split), 1 << split
        for r in (K, K // 3):
            p = rng.random(r) ** 2
            p /= p.sum()
            psi = from_schmidt(rng, p, M, K)
            want = float(-np.sum(p * np.log(p)))
            assert abs(oracle.entanglement_entropy(psi, S, split) - want) <= 1e-11 * max(1.0, want)
