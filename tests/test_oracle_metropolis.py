"""Pins of the Metropolis decision and the whole annealing step of the oracle
(Alg. 1: "Apply Local Gate", "Calculate Entropy", "M.A").

The decision accepts a move that does not raise the energy and an uphill move
(delta > 0) with probability exp(-delta / T). Pins that fix it without its own
formula:

* a table of hand-worked cases (energies, uniform, temperature, direction);
* threshold cases delta = T ln 2 (probability 1/2) and delta = T ln 4 (1/4):
  uniforms on either side decide, and over a million seeded uniforms the
  accepted fraction matches 1/4 within five standard deviations;
* T = 0 accepts only downhill and flat moves, a huge T accepts everything,
  NaN energies are rejected; direction = -1 is the decision on negated
  energies.

Each planted mistake (``_mutant`` 1-4: sign of delta, T ignored, delta = 0
treated as uphill, the comparison reversed) fails at least one pin.

The annealing step is pinned through states whose entropies are known: a gate
acting on one side of the cut keeps the entropy (a flat move, always
accepted, the new state equal to the gated one); a CNOT across the cut turns
a product state into one with a Bell pair across it (entropy ln 2), which a
minimising walker at T = 0 rejects and a maximising one accepts.
"""
import math

import numpy as np
import pytest

import oracle

# (e_cur, e_new, u, T, direction, accepted), worked by hand
TABLE = [
    (0.5, 0.7, 0.8, 0.2, +1, False),    # delta 0.2, exp(-1) = 0.3679 < 0.8
    (0.5, 0.7, 0.3, 0.2, +1, True),     # 0.3 < 0.3679
    (0.5, 0.2, 0.99, 0.1, +1, True),    # downhill
    (0.5, 0.2, 0.5, 0.1, -1, False),    # maximising: delta 0.3, exp(-3) = 0.0498 < 0.5
    (0.5, 0.2, 0.04, 0.1, -1, True),    # 0.04 < 0.0498
    (1.0, 1.0, 0.999, 0.0, +1, True),   # flat move at T = 0
    (1.0, 1.1, 0.0, 0.0, +1, False),    # uphill at T = 0: exp(-inf) = 0, u = 0 is not below it
    (2.0, 3.0, 0.3, 1.0, +1, True),     # exp(-1) = 0.3679 > 0.3
    (2.0, 3.0, 0.37, 1.0, +1, False),   # 0.37 > 0.3679
    (0.0, 1e-3, 0.99, 1.0, +1, True),   # exp(-0.001) = 0.9990 > 0.99
]


def pin_table(mutant):
    for e0, e1, u, T, d, want in TABLE:
        got = bool(oracle.metropolis_accept([e0], [e1], [u], T, d, _mutant=mutant)[0])
        assert got == want, (e0, e1, u, T, d)


def pin_thresholds(mutant):
    T = 0.37
    for p, lo, hi in ((0.5, 0.25, 0.75), (0.25, 0.2, 0.3)):
        delta = -T * math.log(p)
        acc = oracle.metropolis_accept([1.0, 1.0], [1.0 + delta] * 2, [lo, hi], T, _mutant=mutant)
        assert acc.tolist() == [True, False]
    rng = np.random.default_rng(120)
    n = 1_000_000
    u = rng.random(n)
    delta = T * math.log(4.0)
    frac = float(np.mean(oracle.metropolis_accept(np.zeros(n), np.full(n, delta), u, T,
                                                  _mutant=mutant)))
    assert abs(frac - 0.25) <= 5 * math.sqrt(0.25 * 0.75 / n)


def pin_limits(mutant):
    rng = np.random.default_rng(121)
    e0 = rng.standard_normal(1000)
    e1 = rng.standard_normal(1000)
    u = rng.random(1000)
    cold = oracle.metropolis_accept(e0, e1, u, 0.0, _mutant=mutant)
    assert np.array_equal(cold, e1 <= e0)
    hot = oracle.metropolis_accept(e0, e1, u, 1e300, _mutant=mutant)
    assert hot.all()
    nan = oracle.metropolis_accept([0.0, np.nan], [np.nan, 0.0], [0.0, 0.0], 1.0, _mutant=mutant)
    assert not nan.any()
    T = 0.7
    assert np.array_equal(oracle.metropolis_accept(e0, e1, u, T, -1, _mutant=mutant),
                          oracle.metropolis_accept(-e0, -e1, u, T, +1, _mutant=mutant))


PINS = [pin_table, pin_thresholds, pin_limits]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_metropolis_pin(pin):
    pin(0)


@pytest.mark.parametrize("mutant", [1, 2, 3, 4])
def test_metropolis_planted_mistakes(mutant):
    failed = []
    for pin in PINS:
        try:
            pin(mutant)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"mutant {mutant} passed every pin"


CNOT = np.array([[1, 0, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0], [0, 1, 0, 0]], dtype=np.complex128)


def _product_plus_zero(S):
    """|+> on every spin except spin split = S // 2, which is |0>."""
    plus = np.array([1.0, 1.0]) / math.sqrt(2.0)
    zero = np.array([1.0, 0.0])
    psi = np.ones(1)
    for i in reversed(range(S)):  # spin i is bit i: kron puts the high spin first
        psi = np.kron(psi, zero if i == S // 2 else plus)
    return psi.astype(np.complex128)


def test_anneal_step_flat_move_is_accepted():
    rng = np.random.default_rng(122)
    S = 8  # cut between spins 3 and 4
    W = 4
    psi = rng.standard_normal((W, 1 << S)) + 1j * rng.standard_normal((W, 1 << S))
    e0 = np.array([oracle.entanglement_entropy(p, S) for p in psi])
    q, r = np.linalg.qr(rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)))
    U = np.stack([q] * W)
    sites = np.array([0, 1, 2, 5], dtype=np.int32)  # pairs (0,1), (1,2), (2,3), (5,6): one side
    # the entropy changes only by rounding (|delta| ~ 1e-15): with T = 1e-3 any
    # such delta is accepted for u = 0.5 (exp(-1e-12) > 0.5)
    out, e1, acc = oracle.anneal_step(psi, e0, S, sites, U, np.full(W, 0.5), 1e-3)
    assert acc.all()
    assert np.allclose(e1, e0, atol=1e-12, rtol=0)
    assert np.array_equal(out, oracle.two_site_gate(psi, S, sites, U))


def test_anneal_step_entangling_move():
    S = 6
    split = S // 2
    psi = _product_plus_zero(S)[None]
    # CNOT on spins (split - 1, split): control = spin split-1 (local bit 0), target spin split
    # local index a = b_j + 2 b_{j+1}; CNOT flips b_{j+1} when b_j = 1: a=1 <-> a=3
    e0 = np.array([oracle.entanglement_entropy(psi[0], S)])
    assert abs(e0[0]) <= 1e-12
    sites = np.array([split - 1], dtype=np.int32)
    out, e1, acc = oracle.anneal_step(psi, e0, S, sites, CNOT[None], [0.5], 0.0, +1)
    assert not acc[0] and np.array_equal(out, psi) and e1[0] == e0[0]
    out, e1, acc = oracle.anneal_step(psi, e0, S, sites, CNOT[None], [0.5], 0.0, -1)
    assert acc[0] and abs(e1[0] - math.log(2.0)) <= 1e-12
    assert np.array_equal(out, oracle.two_site_gate(psi, S, sites, CNOT[None]))
