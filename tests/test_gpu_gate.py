"""GPU parity of the local two-spin gate (apply_local_gate; Sec. 2, Alg. 1
"Apply Local Gate") against the oracle.

The kernel contracts each complex product into FMAs, so general gates match
the oracle within FP64 rounding (TOL_FP64, relative to ||U|| ||psi||);
permutation gates move amplitudes without arithmetic and must match bit for
bit (checked against numpy index permutations, not the oracle).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2203_09353_gb300 as bg

from gpu_util import TOL_FP64, host

pytestmark = pytest.mark.gpu

X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
I2 = np.eye(2, dtype=np.complex128)
SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


def haar4(rng):
    z = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def states(rng, W, S):
    return rng.standard_normal((W, 1 << S)) + 1j * rng.standard_normal((W, 1 << S))


def to_dev(psi, sites, U, stride=None):
    W, dim = psi.shape
    stride = dim if stride is None else stride
    buf = np.zeros((W, stride), dtype=np.complex128)
    buf[:, :dim] = psi
    st = torch.from_numpy(buf.ravel()).cuda()
    s = torch.from_numpy(np.asarray(sites, dtype=np.int32)).cuda()
    g = torch.from_numpy(np.ascontiguousarray(np.asarray(U).transpose(0, 2, 1)).ravel()).cuda()
    return st, s, g


@pytest.mark.parametrize("S", [2, 3, 5, 8, 12, 16])
def test_gate_matches_oracle(gpu, S):
    rng = np.random.default_rng(40 + S)
    W = 6
    sites = np.array([w % (S - 1) for w in range(W)], dtype=np.int32)
    sites[-1] = S - 2
    psi = states(rng, W, S)
    U = np.stack([haar4(rng) if w % 2 else rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
                  for w in range(W)])
    st, s, g = to_dev(psi, sites, U)
    bg.apply_local_gate(st, S, s, g)
    got = host(st).reshape(W, 1 << S)
    ref = oracle.two_site_gate(psi, S, sites, U)
    for w in range(W):
        err = np.linalg.norm(got[w] - ref[w])
        assert err <= TOL_FP64 * np.linalg.norm(U[w]) * np.linalg.norm(psi[w]), (w, err)
    bg.check_device_errors()


def test_gate_permutations_bitwise(gpu):
    rng = np.random.default_rng(50)
    S = 9
    x = np.arange(1 << S)
    for j in range(S - 1):
        bj, bk = (x >> j) & 1, (x >> (j + 1)) & 1
        swapped = x - (bj << j) - (bk << (j + 1)) + (bk << j) + (bj << (j + 1))
        cases = [(np.eye(4, dtype=np.complex128), x), (SWAP, swapped),
                 (np.kron(X, I2), x ^ (1 << (j + 1))), (np.kron(I2, X), x ^ (1 << j))]
        psi = states(rng, len(cases), S)
        U = np.stack([c[0] for c in cases])
        st, s, g = to_dev(psi, [j] * len(cases), U)
        bg.apply_local_gate(st, S, s, g)
        got = host(st).reshape(len(cases), 1 << S)
        for w, (_, perm) in enumerate(cases):
            assert np.array_equal(got[w], psi[w][perm]), (j, w)


def test_gate_many_walkers_padded_stride(gpu):
    """300 walkers with their own sites and gates, states spaced by a stride
    with padding that must stay untouched."""
    rng = np.random.default_rng(51)
    S, W, pad = 10, 300, 24
    psi = states(rng, W, S)
    sites = rng.integers(0, S - 1, W).astype(np.int32)
    U = np.stack([haar4(rng) for _ in range(W)])
    stride = (1 << S) + pad
    st, s, g = to_dev(psi, sites, U, stride)
    fill = torch.full((W, pad), 7.0 + 3.0j, dtype=torch.complex128, device="cuda")
    st.view(W, stride)[:, 1 << S:] = fill
    bg.apply_local_gate(st, S, s, g, stride=stride)
    out = host(st).reshape(W, stride)
    ref = oracle.two_site_gate(psi, S, sites, U)
    assert np.all(out[:, 1 << S:] == 7.0 + 3.0j)
    for w in range(W):
        assert np.linalg.norm(out[w, :1 << S] - ref[w]) <= TOL_FP64 * 2.0 * np.linalg.norm(psi[w])


def test_gate_bad_site_is_reported_and_skipped(gpu):
    rng = np.random.default_rng(52)
    S, W = 6, 4
    psi = states(rng, W, S)
    sites = np.array([0, S - 1, 2, -1], dtype=np.int32)  # walkers 1 and 3 out of range
    U = np.stack([haar4(rng) for _ in range(W)])
    bg.check_device_errors()
    st, s, g = to_dev(psi, sites, U)
    bg.apply_local_gate(st, S, s, g)
    with pytest.raises(bg.BgemmError) as ei:
        bg.check_device_errors()
    assert ei.value.status == 1
    bg.check_device_errors()  # the check cleared the word
    got = host(st).reshape(W, 1 << S)
    assert np.array_equal(got[1], psi[1]) and np.array_equal(got[3], psi[3])
    ref = oracle.two_site_gate(psi[[0, 2]], S, sites[[0, 2]], U[[0, 2]])
    for i, w in enumerate((0, 2)):
        assert np.linalg.norm(got[w] - ref[i]) <= TOL_FP64 * 2.0 * np.linalg.norm(psi[w])


def test_gate_argument_checks(gpu):
    lib = bg.load_library()
    st = torch.zeros(64, dtype=torch.complex128, device="cuda")
    s = torch.zeros(1, dtype=torch.int32, device="cuda")
    g = torch.zeros(16, dtype=torch.complex128, device="cuda")
    p = st.data_ptr()
    assert lib.apply_local_gate(bg.BG_R64, 1, 6, s.data_ptr(), g.data_ptr(), p, 64, None) == 2
    assert lib.apply_local_gate(bg.BG_C128, 1, 1, s.data_ptr(), g.data_ptr(), p, 64, None) == 1
    assert lib.apply_local_gate(bg.BG_C128, 1, 6, s.data_ptr(), g.data_ptr(), p, 63, None) == 1
    assert lib.apply_local_gate(bg.BG_C128, -1, 6, s.data_ptr(), g.data_ptr(), p, 64, None) == 1
    bg.launch_count(reset=True)
    assert lib.apply_local_gate(bg.BG_C128, 0, 6, s.data_ptr(), g.data_ptr(), p, 64, None) == 0
    assert bg.launch_count(reset=True) == 0  # no walkers: nothing launched


def test_wrapper_rejects_bad_tensors_before_launch(gpu):
    """The Python binding checks element types and sizes of torch tensors before
    the call: an int64 sites tensor (torch's default integer type) would be read
    as int32 halves, and undersized states or gates would be written or read out
    of bounds. Each raises ValueError and launches nothing."""
    S, W = 6, 3
    st = torch.zeros(W << S, dtype=torch.complex128, device="cuda")
    s32 = torch.zeros(W, dtype=torch.int32, device="cuda")
    g = torch.zeros(16 * W, dtype=torch.complex128, device="cuda")
    bad = [
        dict(states=st, sites=s32.to(torch.int64), gates=g),
        dict(states=st[: (W << S) - 1], sites=s32, gates=g),
        dict(states=st, sites=s32, gates=g[: 16 * W - 1]),
        dict(states=st.to(torch.complex64), sites=s32, gates=g),
        dict(states=st.view(W, 1 << S).t(), sites=s32, gates=g),
    ]
    bg.launch_count(reset=True)
    for kw in bad:
        with pytest.raises(ValueError):
            bg.apply_local_gate(kw["states"], S, kw["sites"], kw["gates"])
    assert bg.launch_count(reset=True) == 0
    with pytest.raises(ValueError):
        bg.apply_local_gate(st, S, s32, g, stride=(1 << S) + 1)  # 3 strides overrun the buffer
    assert bg.launch_count(reset=True) == 0
