"""GPU parity of the entanglement entropy (entropy_plan / batched_entropy;
Alg. 1 "Calculate Entropy", Sec. 3) against the oracle and closed forms.

Tolerance. G = X X^H is formed to a normwise error e_G (about 1e-16 in FP64
and with 9 slices); Householder reduction and bisection in FP64 perturb each
eigenvalue of the normalised spectrum by at most about n (n u + e_G)
(n = K <= 256, u = 2^-53), and -p ln p changes by at most |dp| (|ln max(p, dp)| + 1)
for each eigenvalue. With dp <= 256 x 1e-13 that sums to well under 1e-9 for
n <= 256; TOL_ENT = 1e-9 (absolute, natural log) keeps that worst case and
is about four orders of magnitude above what the GPU reaches. For K = 512
and 1024 the test asserts every eigenvalue to 1e-12 of the largest first;
then |dp| <= 2e-12 and the entropy moves by at most K x 2e-12 x
(ln(1 / 2e-12) + 1) < K x 6e-11, the tolerance used there.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2203_09353_gb300 as bg

from gpu_util import host

pytestmark = pytest.mark.gpu

TOL_ENT = 1e-9


def haar(rng, n):
    z = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def schmidt_state(rng, p, S, split):
    """psi with the reshape Psi (M x K, row = upper spins) = U diag(sqrt(p)) V^H."""
    M, K = 1 << (S - split), 1 << split
    r = len(p)
    P = haar(rng, M)[:, :r] @ np.diag(np.sqrt(p)) @ np.conj(haar(rng, K)[:, :r].T)
    return P.reshape(-1)


def run(states, S, split=None, prec=None, stride=None, eig=False):
    W = len(states)
    dim = 1 << S
    stride = dim if stride is None else stride
    buf = np.zeros((W, stride), dtype=np.complex128)
    for w, psi in enumerate(states):
        buf[w, :dim] = psi
    dst = torch.from_numpy(buf.ravel()).cuda()
    plan = bg.entropy_plan(W, S, split, stride, prec)
    out = torch.zeros(W, dtype=torch.float64, device="cuda")
    K = 1 << (S // 2 if split is None else split)
    ev = torch.zeros(W * K, dtype=torch.float64, device="cuda") if eig else None
    bg.batched_entropy(plan, dst, out, ev)
    bg.check_device_errors()
    res = host(out)
    return (res, host(ev).reshape(W, K)) if eig else res


@pytest.mark.parametrize("S", [2, 5, 8, 9, 12])
def test_schmidt_spectra_closed_form(gpu, S):
    rng = np.random.default_rng(70 + S)
    split = S // 2
    M, K = 1 << (S - split), 1 << split
    states, want = [], []
    for j in range(4):
        r = min(M, K) if j < 3 else max(1, min(M, K) // 2)  # the last one rank-deficient
        p = rng.random(r) ** (j + 1)
        p /= p.sum()
        states.append(schmidt_state(rng, p, S, split) * (0.5 + j))  # any norm
        want.append(float(-np.sum(p * np.log(p))))
    got = run(states, S)
    assert np.max(np.abs(got - np.array(want))) <= TOL_ENT


def test_product_and_maximally_entangled(gpu):
    rng = np.random.default_rng(80)
    S = 10
    M, K = 1 << (S - S // 2), 1 << (S // 2)
    a = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    b = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    prod = np.outer(a, b).reshape(-1)
    maxent = schmidt_state(rng, np.full(K, 1.0 / K), S, S // 2)
    got = run([prod, maxent], S)
    assert abs(got[0]) <= TOL_ENT
    assert abs(got[1] - np.log(K)) <= TOL_ENT


def test_odd_spin_count_cut(gpu):
    """A Bell pair on spins 1 and 2 of a 5-spin product state straddles the cut
    between spins split-1 = 1 and split = 2: entropy ln 2; with split = 3 the
    pair lies on one side: entropy 0."""
    rng = np.random.default_rng(81)
    S = 5
    one = [v / np.linalg.norm(v) for v in
           (rng.standard_normal(2) + 1j * rng.standard_normal(2) for _ in range(3))]
    psi = np.zeros(1 << S, dtype=np.complex128)
    for x in range(1 << S):
        b = [(x >> i) & 1 for i in range(S)]
        if b[1] == b[2]:
            psi[x] = one[0][b[0]] * one[1][b[3]] * one[2][b[4]] / np.sqrt(2.0)
    assert abs(run([psi], S)[0] - np.log(2.0)) <= TOL_ENT
    assert abs(run([psi], S, split=3)[0]) <= TOL_ENT


@pytest.mark.parametrize("S", [13, 15, 17])
@pytest.mark.parametrize("mode", ["fp64", "split9"])
def test_random_states_match_oracle(gpu, S, mode):
    """Random complex states at the paper's Sec. 3 sizes (K x M = 64 x 128,
    128 x 256, 256 x 512); the Gram matrix in FP64 or with 9 slices."""
    rng = np.random.default_rng(90 + S)
    W = 3
    states = [rng.standard_normal(1 << S) + 1j * rng.standard_normal(1 << S) for _ in range(W)]
    prec = None if mode == "fp64" else bg.precision("split", 9)
    got, eig = run(states, S, prec=prec, eig=True)
    for w in range(W):
        want = oracle.entanglement_entropy(states[w], S)
        assert abs(got[w] - want) <= TOL_ENT, (w, got[w], want)
        # the Gram spectrum: sum = ||psi||^2, ascending, nonnegative up to rounding
        n2 = float(np.vdot(states[w], states[w]).real)
        assert abs(eig[w].sum() - n2) <= 1e-12 * n2
        assert np.all(np.diff(eig[w]) >= 0) and eig[w][0] >= -1e-12 * n2
        # each eigenvalue against a library eigensolver on the same Gram matrix
        # (the K x M column-major view X of the state, G = X X^H): Householder
        # reduction and bisection in FP64 stay within a small multiple of
        # n u ||G||
        K = 1 << (S // 2)
        X = states[w].reshape(-1, K).T
        lam = np.linalg.eigvalsh(X @ X.conj().T)
        assert np.max(np.abs(eig[w] - lam)) <= 1e-12 * lam[-1], (w, np.max(np.abs(eig[w] - lam)))


def test_padded_stride_and_many_walkers(gpu):
    rng = np.random.default_rng(95)
    S, W, pad = 8, 40, 16
    states = [rng.standard_normal(1 << S) + 1j * rng.standard_normal(1 << S) for _ in range(W)]
    got = run(states, S, stride=(1 << S) + pad)
    want = np.array([oracle.entanglement_entropy(p, S) for p in states])
    assert np.max(np.abs(got - want)) <= TOL_ENT


def test_argument_checks(gpu):
    lib = bg.load_library()
    import ctypes
    h = ctypes.c_void_p()
    assert lib.entropy_plan(ctypes.byref(h), 4, 8, 0, 256, None, 0, None) == 1   # split 0
    assert lib.entropy_plan(ctypes.byref(h), 4, 8, 8, 256, None, 0, None) == 1   # split = spins
    assert lib.entropy_plan(ctypes.byref(h), 4, 8, 4, 255, None, 0, None) == 1   # stride < 2^S
    assert lib.entropy_plan(ctypes.byref(h), 4, 8, 4, 256, None, 1, None) == 1   # bad flag
    plan = bg.entropy_plan(2, 6)
    st = torch.zeros(128, dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):
        bg.batched_entropy(plan, st, torch.zeros(2, dtype=torch.float32, device="cuda"))
    with pytest.raises(bg.BgemmError) as ei:
        bg.batched_gemm_grouped(plan, st, None, st, 1.0, 0.0)
    assert ei.value.status == 1


@pytest.mark.parametrize("S,split,mode", [(14, 7, "split9"), (19, 9, "split9"), (21, 10, "split9"),
                                          (14, 7, "fp64"), (19, 9, "fp64")])
def test_blocked_reduction(gpu, S, split, mode):
    """Split-precision plans with K > 64 reduce G in panels, the trailing
    updates running as batched GEMMs (K = 128: 4 panels; K = 512: 28 panels,
    whose V and W leave shared memory for the wider ones; K = 1024: 60
    panels); FP64 plans take the unblocked reduction at the same sizes. A
    diagonal G (every reflector the identity), a rank-deficient Schmidt
    spectrum and a random state, each against its closed form or the oracle,
    eigenvalue by eigenvalue against a library eigensolver."""
    rng = np.random.default_rng(110 + S)
    M, K = 1 << (S - split), 1 << split
    p_diag = rng.random(K) + 0.1
    p_diag /= p_diag.sum()
    P = np.zeros((M, K), dtype=np.complex128)
    P[np.arange(K), np.arange(K)] = np.sqrt(p_diag)
    p_low = rng.random(K // 3) ** 2
    p_low /= p_low.sum()
    states = [P.reshape(-1), schmidt_state(rng, p_low, S, split),
              rng.standard_normal(1 << S) + 1j * rng.standard_normal(1 << S)]
    want = [float(-np.sum(p_diag * np.log(p_diag))), float(-np.sum(p_low * np.log(p_low))),
            oracle.entanglement_entropy(states[2], S, split)]
    prec = None if mode == "fp64" else bg.precision("split", 9)
    got, eig = run(states, S, split=split, prec=prec, eig=True)
    for w, psi in enumerate(states):
        X = psi.reshape(-1, K).T
        lam = np.linalg.eigvalsh(X @ X.conj().T)
        assert np.max(np.abs(eig[w] - lam)) <= 1e-12 * lam[-1], (w, np.max(np.abs(eig[w] - lam)))
    tol = TOL_ENT if K <= 256 else K * 6e-11
    assert np.max(np.abs(got - np.array(want))) <= tol, (got, want)
    assert np.allclose(eig[0], np.sort(p_diag), rtol=0, atol=1e-15)
