"""CPU oracle for the batched GEMM of Eq. (1) (Sec. 2) -- TEST INFRASTRUCTURE ONLY.

C_i = alpha * A_i * B_i + beta * C_i over N independent instances, in FP64
and complex128, written out as a plain triple loop in C (``oracle_gemm.c``);
the local two-spin gate of the annealing step (Sec. 2, "Apply Local
Gate") on a batch of state vectors (``oracle_gate.c``); and the entanglement
entropy of Alg. 1's "Calculate Entropy" (``entanglement_entropy``: the oracle
GEMM for rho = Psi Psi^H, then numpy's Hermitian eigensolver as a library step);
the Metropolis decision of Alg. 1's "M.A" (``metropolis_accept``) and one
whole annealing step built from these (``anneal_step``).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The GPU library never calls it and the
two share no code: the oracle has its own C source, its own build and its own
loader.

Parity status: pinned. ``tests/test_oracle.py`` checks every entry point
against brute force on small integer inputs, identity and permutation
matrices, the Pauli algebra, (AB)^T = B^T A^T, the Kronecker mixed-product
rule, the BLAS alpha/beta rules and an independent library (numpy.matmul),
and shows that each of the planted mistakes selectable with ``ORACLE_MUTANT``
fails at least one of those pins.

Array convention of this wrapper: every operand is a flat 1-D numpy array
(float64, or complex128 for the complex entry points) holding column-major
instances; offsets, leading dimensions and strides are in elements.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle_gemm.c")
_SRCS = (_SRC, os.path.join(_HERE, "oracle_gate.c"))
_LIB_NAME = "liboracle.so"
_lock = threading.Lock()
_libs: dict[str, ctypes.CDLL] = {}

_CFLAGS = ["-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp"]


def build(out_dir: str | None = None, mutant: int = 0, force: bool = False) -> str:
    """Compile ``oracle_gemm.c`` with gcc and return the path of the shared library.

    ``mutant`` > 0 builds a variant with one planted mistake (pin tests only).
    """
    out_dir = out_dir or _HERE
    name = _LIB_NAME if mutant == 0 else f"liboracle_mutant{mutant}.so"
    path = os.path.join(out_dir, name)
    if force or not os.path.exists(path) or \
            os.path.getmtime(path) < max(os.path.getmtime(f) for f in _SRCS):
        cmd = ["gcc", *_CFLAGS, f"-DORACLE_MUTANT={int(mutant)}", *_SRCS, "-o", path + ".tmp"]
        subprocess.run(cmd, check=True)
        os.replace(path + ".tmp", path)
    return path


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    i64, dbl, vp = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    lib.oracle_gemm_r64.argtypes = [i64, i64, i64, dbl, vp, i64, i64, vp, i64, i64, dbl, vp,
                                    i64, i64, i64]
    lib.oracle_gemm_c128.argtypes = [i64, i64, i64, vp, vp, i64, i64, vp, i64, i64, vp, vp,
                                     i64, i64, i64]
    lib.oracle_gemm_grouped_r64.argtypes = [i64, vp, dbl, vp, vp, dbl, vp]
    lib.oracle_gemm_grouped_c128.argtypes = [i64, vp, vp, vp, vp, vp, vp]
    for f in ("oracle_gemm_r64", "oracle_gemm_c128", "oracle_gemm_grouped_r64",
              "oracle_gemm_grouped_c128"):
        getattr(lib, f).restype = None
    lib.oracle_two_site_gate_c128.argtypes = [i64, ctypes.c_int32, vp, vp, vp, i64]
    lib.oracle_two_site_gate_c128.restype = i64
    lib.oracle_max_threads.restype = ctypes.c_int
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    return lib


def load(mutant: int = 0, out_dir: str | None = None) -> ctypes.CDLL:
    """Load (building first if needed) the oracle library, or a planted-mistake variant."""
    key = f"{out_dir}:{mutant}"
    with _lock:
        if key not in _libs:
            _libs[key] = _bind(ctypes.CDLL(build(out_dir=out_dir, mutant=mutant)))
        return _libs[key]


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"] or a.ndim == 1
    return a.ctypes.data


def max_threads(lib: ctypes.CDLL | None = None) -> int:
    return int((lib or load()).oracle_max_threads())


def set_threads(t: int, lib: ctypes.CDLL | None = None) -> None:
    (lib or load()).oracle_set_threads(int(t))


def gemm_fixed(m, n, k, alpha, A, lda, strideA, B, ldb, strideB, beta, C, ldc, strideC,
               batch, lib: ctypes.CDLL | None = None) -> np.ndarray:
    """Eq. (1) over a fixed-size batch; updates ``C`` in place and returns it.

    Real when ``C`` is float64, complex when it is complex128 (then alpha and
    beta are complex scalars).
    """
    lib = lib or load()
    if C.dtype == np.complex128:
        for x in (A, B):
            assert x.dtype == np.complex128
        al = np.array([complex(alpha).real, complex(alpha).imag], dtype=np.float64)
        be = np.array([complex(beta).real, complex(beta).imag], dtype=np.float64)
        lib.oracle_gemm_c128(m, n, k, _ptr(al), _ptr(A), lda, strideA, _ptr(B), ldb, strideB,
                             _ptr(be), _ptr(C), ldc, strideC, batch)
    else:
        for x in (A, B, C):
            assert x.dtype == np.float64
        lib.oracle_gemm_r64(m, n, k, float(alpha), _ptr(A), lda, strideA, _ptr(B), ldb,
                            strideB, float(beta), _ptr(C), ldc, strideC, batch)
    return C


def gemm_grouped(table: np.ndarray, alpha, A, B, beta, C,
                 lib: ctypes.CDLL | None = None) -> np.ndarray:
    """Eq. (1) over a variable-size batch.

    ``table`` is int64 [count, 9]: m, n, k, lda, ldb, ldc, a_off, b_off, c_off.
    Updates ``C`` in place and returns it.
    """
    lib = lib or load()
    table = np.ascontiguousarray(table, dtype=np.int64)
    assert table.ndim == 2 and table.shape[1] == 9
    count = table.shape[0]
    if C.dtype == np.complex128:
        al = np.array([complex(alpha).real, complex(alpha).imag], dtype=np.float64)
        be = np.array([complex(beta).real, complex(beta).imag], dtype=np.float64)
        lib.oracle_gemm_grouped_c128(count, _ptr(table), _ptr(al), _ptr(A), _ptr(B), _ptr(be),
                                     _ptr(C))
    else:
        lib.oracle_gemm_grouped_r64(count, _ptr(table), float(alpha), _ptr(A), _ptr(B),
                                    float(beta), _ptr(C))
    return C


def matmul(A: np.ndarray, B: np.ndarray, lib: ctypes.CDLL | None = None) -> np.ndarray:
    """Single product A @ B of two 2-D arrays through the oracle (alpha=1, beta=0)."""
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    dt = np.complex128 if (A.dtype == np.complex128 or B.dtype == np.complex128) else np.float64
    a = np.asfortranarray(A, dtype=dt).ravel(order="F")
    b = np.asfortranarray(B, dtype=dt).ravel(order="F")
    c = np.zeros(m * n, dtype=dt)
    gemm_fixed(m, n, k, 1.0, a, max(m, 1), m * k, b, max(k, 1), k * n, 0.0, c, max(m, 1), m * n,
               1, lib=lib)
    return c.reshape((m, n), order="F")


def unitarity_drift(C: np.ndarray, lib: ctypes.CDLL | None = None) -> float:
    """||C^H C - I||_F for one square matrix, the product C^H C taken by the oracle."""
    n = C.shape[0]
    G = matmul(np.conj(C.T), C, lib=lib)
    return float(np.sqrt(np.sum(np.abs(G - np.eye(n)) ** 2)))


def two_site_gate(states: np.ndarray, S: int, sites, gates: np.ndarray,
                  lib: ctypes.CDLL | None = None) -> np.ndarray:
    """The local two-spin gate on a batch of state vectors; returns the new states.

    ``states``: complex128 [walkers, 2^S] (walker w's amplitude of basis state
    x, spin i being bit i of x). ``sites``: the lower spin j of each walker's
    pair (0 <= j <= S - 2). ``gates``: complex128 [walkers, 4, 4], gate[w][a, c]
    acting on the local index a = b_j + 2 b_{j+1}. Raises ValueError for a bad site.
    """
    lib = lib or load()
    st = np.ascontiguousarray(states, dtype=np.complex128).copy()
    W = st.shape[0]
    assert st.shape == (W, 1 << S)
    sites = np.ascontiguousarray(sites, dtype=np.int32)
    assert sites.shape == (W,)
    g = np.ascontiguousarray(np.asarray(gates, dtype=np.complex128).transpose(0, 2, 1))
    assert g.shape == (W, 4, 4)  # column-major 4 x 4 per walker
    bad = lib.oracle_two_site_gate_c128(W, int(S), _ptr(sites), _ptr(g), _ptr(st), 1 << S)
    if bad:
        raise ValueError(f"{bad} walker(s) with a site outside 0..S-2")
    return st


def entanglement_entropy(psi: np.ndarray, S: int, split: int | None = None) -> float:
    """Entanglement entropy of a pure state of S spins across a cut (Sec. 2,
    Alg. 1 "Calculate Entropy"), following the paper's steps: Psi is the state
    reshaped to M x K (M = 2^(S - split) rows for the upper spins, K = 2^split
    columns for the lower ones, split = floor(S/2) by default, Sec. 3's
    shapes); rho = Psi Psi^H is formed by the oracle GEMM; its eigenvalues
    (numpy.linalg.eigvalsh, a library step) give p_i = lambda_i / sum(lambda);
    the entropy is -sum p_i ln p_i over p_i > 0 (natural log).

    The cut: spin i is bit i of the basis index x (as for the local gate);
    the lower spins 0..split-1 (x mod K) index the columns of Psi and the
    upper spins split..S-1 (x div K) its rows, so the cut lies between spins
    split-1 and split. In the library's column-major convention the state
    vector itself is, without a copy, the K x M matrix X = Psi^T (row = lower
    spins); X X^H = conj(Psi^H Psi) has the nonzero spectrum of rho, which
    is the route a GPU path takes. (Viewing the vector as a column-major
    M x K matrix instead would cut between spins S-split-1 and S-split: the
    same cut only for even S.)
    """
    split = S // 2 if split is None else int(split)
    M, K = 1 << (S - split), 1 << split
    psi = np.asarray(psi, dtype=np.complex128).reshape(-1)
    assert psi.size == M * K
    # amplitude of basis state x = upper * K + lower sits at row upper, column lower
    P = psi.reshape(M, K)
    rho = matmul(P, np.conj(P.T))
    lam = np.linalg.eigvalsh(rho)
    total = float(np.sum(lam))
    p = lam / total
    p = p[p > 0]
    return float(-np.sum(p * np.log(p)))


def metropolis_accept(e_cur, e_new, u, temperature: float, direction: int = 1, *,
                      _mutant: int = 0) -> np.ndarray:
    """The Metropolis decision of Alg. 1 ("M.A"), per walker, in FP64.

    The move from energy e_cur to e_new is accepted when it does not raise the
    energy, delta = direction * (e_new - e_cur) <= 0, and otherwise with
    probability exp(-delta / T): accepted when u < exp(-delta / T) for the
    walker's uniform u in [0, 1). direction = +1 lowers the energy (here the
    entanglement entropy), -1 raises it. T = 0 accepts only moves with
    delta <= 0; a NaN energy is never accepted. ``_mutant`` plants a mistake
    for the pin tests only (1: sign of delta flipped, 2: T ignored, 3: delta = 0
    treated as uphill, 4: the comparison with u reversed).
    """
    e_cur = np.asarray(e_cur, dtype=np.float64)
    e_new = np.asarray(e_new, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    T = float(temperature)
    delta = float(direction) * (e_new - e_cur)
    if _mutant == 1:
        delta = -delta
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        x = -delta if _mutant == 2 else -delta / T
        thresh = np.exp(x)
    down = delta < 0 if _mutant == 3 else delta <= 0
    up = u >= thresh if _mutant == 4 else u < thresh
    return down | (~down & up)


def anneal_step(states: np.ndarray, e_cur, S: int, sites, gates: np.ndarray, u,
                temperature: float, direction: int = 1, split: int | None = None,
                lib: ctypes.CDLL | None = None):
    """One step of Alg. 1 for every walker: the local gate on a copy of the
    state (``two_site_gate``), the new entanglement entropy
    (``entanglement_entropy``), the Metropolis decision (``metropolis_accept``);
    an accepted walker takes the new state and energy, a rejected one keeps
    both. Returns (states, energies, accepted)."""
    states = np.asarray(states, dtype=np.complex128)
    prop = two_site_gate(states, S, sites, gates, lib=lib)
    e_new = np.array([entanglement_entropy(prop[w], S, split) for w in range(prop.shape[0])])
    acc = metropolis_accept(e_cur, e_new, u, temperature, direction)
    out = np.where(acc[:, None], prop, states)
    e_out = np.where(acc, e_new, np.asarray(e_cur, dtype=np.float64))
    return out, e_out, acc
