"""GPU parity of the Metropolis decision (metropolis_select) and of whole
annealing steps (anneal_plan / anneal_step; Alg. 1: local gate, entropy,
"M.A") against the oracle.

The decision is an integer outcome taken in FP64 on both sides from the same
energies and uniforms, so it must agree exactly; the only exception would be a
uniform within a rounding of exp(-delta / T) (exp is not correctly rounded),
and the tests check that none of their cases comes that close. In the
composed step the energies come from each side's own entropy (equal within
TOL_ENT), so decisions are compared where the oracle's margin |u - exp(-delta/T)|
exceeds 1e-6; states follow the gate's FP64 tolerance, energies TOL_ENT.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2203_09353_gb300 as bg

from gpu_util import TOL_FP64, host
from test_gpu_entropy import TOL_ENT

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def haar4(rng):
    z = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def gpu_decide(e0, e1, u, T, d):
    e_cur = dev(np.asarray(e0, dtype=np.float64))
    acc = torch.zeros(len(e0), dtype=torch.int32, device="cuda")
    bg.metropolis_select(T, d, dev(np.asarray(u, dtype=np.float64)),
                         dev(np.asarray(e1, dtype=np.float64)), e_cur, acc)
    return host(acc).astype(bool), host(e_cur)


def test_decisions_match_oracle_exactly(gpu):
    rng = np.random.default_rng(130)
    n = 100_000
    e0, e1 = rng.standard_normal(n), rng.standard_normal(n)
    u = rng.random(n)
    for T, d in ((0.3, 1), (0.3, -1), (2.0, 1), (0.0, 1), (1e-3, -1)):
        want = oracle.metropolis_accept(e0, e1, u, T, d)
        with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
            margin = np.abs(u - np.exp(-(d * (e1 - e0)) / T))
        assert margin[(d * (e1 - e0)) > 0].min() > 1e-13  # no case at a rounding of the threshold
        got, ecur = gpu_decide(e0, e1, u, T, d)
        assert np.array_equal(got, want)
        assert np.array_equal(ecur, np.where(want, e1, e0))


def test_hand_worked_table(gpu):
    from test_oracle_metropolis import TABLE
    for e0, e1, u, T, d, want in TABLE:
        got, _ = gpu_decide([e0], [e1], [u], T, d)
        assert bool(got[0]) == want, (e0, e1, u, T, d)
    got, _ = gpu_decide([0.0, np.nan], [np.nan, 0.0], [0.0, 0.0], 1.0, 1)
    assert not got.any()


def test_accepted_states_are_copied(gpu):
    rng = np.random.default_rng(131)
    W, amps, ps, ss = 37, 1000, 1008, 1024
    prop = rng.standard_normal((W, ps)) + 1j * rng.standard_normal((W, ps))
    cur = rng.standard_normal((W, ss)) + 1j * rng.standard_normal((W, ss))
    e0, e1, u = rng.standard_normal(W), rng.standard_normal(W), rng.random(W)
    want = oracle.metropolis_accept(e0, e1, u, 0.5, 1)
    dprop, dcur = dev(prop.ravel()), dev(cur.ravel())
    e_cur = dev(e0)
    acc = torch.zeros(W, dtype=torch.int32, device="cuda")
    bg.metropolis_select(0.5, 1, dev(u), dev(e1), e_cur, acc, dprop, dcur, amps, ps, ss)
    got = host(dcur).reshape(W, ss)
    assert np.array_equal(host(acc).astype(bool), want)
    for w in range(W):
        ref = prop[w, :amps] if want[w] else cur[w, :amps]
        assert np.array_equal(got[w, :amps], ref)
        assert np.array_equal(got[w, amps:], cur[w, amps:])  # padding untouched


def run_steps(mode, S, W, steps, T, d, seed):
    rng = np.random.default_rng(seed)
    psi = rng.standard_normal((W, 1 << S)) + 1j * rng.standard_normal((W, 1 << S))
    e0 = np.array([oracle.entanglement_entropy(p, S) for p in psi])
    prec = None if mode == "fp64" else bg.precision("split", 9)
    plan = bg.anneal_plan(W, S, prec=prec)
    st, en = dev(psi.ravel()), dev(e0)
    acc = torch.zeros(W, dtype=torch.int32, device="cuda")
    ref_psi, ref_e = psi.copy(), e0.copy()
    checked = 0
    for t in range(steps):
        sites = rng.integers(0, S - 1, W).astype(np.int32)
        U = np.stack([haar4(rng) for _ in range(W)])
        u = rng.random(W)
        bg.anneal_step(plan, st, en, dev(sites), dev(U.transpose(0, 2, 1).ravel()), dev(u), T, d,
                       acc)
        got_acc = host(acc).astype(bool)
        # the oracle step from the GPU's previous state, so that one differing
        # decision does not carry over into later steps
        prev_psi, prev_e = ref_psi, ref_e
        ref_psi, ref_e, ref_acc = oracle.anneal_step(prev_psi, prev_e, S, sites, U, u, T, d)
        prop = oracle.two_site_gate(prev_psi, S, sites, U)
        e_new = np.array([oracle.entanglement_entropy(p, S) for p in prop])
        delta = d * (e_new - prev_e)
        with np.errstate(divide="ignore", over="ignore"):
            margin = np.where(delta <= 0, np.inf, np.abs(u - np.exp(-delta / T)))
        gpu_psi = host(st).reshape(W, 1 << S)
        gpu_e = host(en)
        for w in range(W):
            if margin[w] > 1e-6:  # else the two sides' entropies may decide differently
                assert got_acc[w] == ref_acc[w], (t, w)
            if got_acc[w] != ref_acc[w]:
                continue
            n0 = np.linalg.norm(prev_psi[w])
            assert np.linalg.norm(gpu_psi[w] - ref_psi[w]) <= 4 * TOL_FP64 * n0
            assert abs(gpu_e[w] - ref_e[w]) <= TOL_ENT
            checked += 1
        ref_psi, ref_e = gpu_psi.copy(), gpu_e.copy()
    return checked


@pytest.mark.parametrize("mode", ["fp64", "split9"])
def test_anneal_steps_match_oracle(gpu, mode):
    """8 walkers of 10 spins, 6 steps at T = 0.05: every decision, state and
    energy against the oracle's step from the same previous state."""
    assert run_steps(mode, 10, 8, 6, 0.05, 1, 140) == 48


def test_anneal_step_entangling_move(gpu):
    """CNOT across the cut on a product state: rejected when minimising at T = 0,
    accepted (entropy ln 2) when maximising."""
    S = 6
    split = S // 2
    plus, zero = np.array([1.0, 1.0]) / math.sqrt(2.0), np.array([1.0, 0.0])
    psi = np.ones(1)
    for i in reversed(range(S)):
        psi = np.kron(psi, zero if i == split else plus)
    psi = psi.astype(np.complex128)
    cnot = np.array([[1, 0, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0], [0, 1, 0, 0]], dtype=np.complex128)
    plan = bg.anneal_plan(2, S)
    st = dev(np.concatenate([psi, psi]))
    en = torch.zeros(2, dtype=torch.float64, device="cuda")
    acc = torch.zeros(2, dtype=torch.int32, device="cuda")
    g = dev(np.concatenate([cnot.T.ravel()] * 2))
    sites = dev(np.array([split - 1, split - 1], dtype=np.int32))
    bg.anneal_step(plan, st, en, sites, g, dev(np.array([0.5, 0.5])), 0.0, 1, acc)
    assert host(acc).tolist() == [0, 0] and np.array_equal(host(st)[:1 << S], psi)
    bg.anneal_step(plan, st, en, sites, g, dev(np.array([0.5, 0.5])), 0.0, -1, acc)
    assert host(acc).tolist() == [1, 1]
    assert np.all(np.abs(host(en) - math.log(2.0)) <= TOL_ENT)


def test_argument_checks(gpu):
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    a = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(bg.BgemmError):
        bg.metropolis_select(-1.0, 1, x, x, x, a)
    with pytest.raises(bg.BgemmError):
        bg.metropolis_select(1.0, 2, x, x, x, a)
    with pytest.raises(ValueError):
        bg.metropolis_select(1.0, 1, x, x, x, a.to(torch.int64))
    lib = bg.load_library()
    import ctypes
    h = ctypes.c_void_p()
    assert lib.anneal_plan(ctypes.byref(h), 4, 8, 4, 255, None, 0, None) == 1  # stride < 2^S
    assert lib.anneal_plan(ctypes.byref(h), 4, 8, 9, 256, None, 0, None) == 1  # split > S - 1
