"""Seeded synthetic batches for the batched GEMM C_i = alpha A_i B_i + beta C_i (Eq. 1).

This module only draws inputs: it holds none of the GEMM arithmetic, and
both the GPU tests/benchmark and the CPU oracle take their inputs from here.
Everything is host-side numpy (``numpy.random.default_rng(seed)``).

The paper runs no public dataset; its operands are the 2^S-sized complex
operators of an S-spin transverse-field Ising chain (Sec. 3). These batches
stand in for them with the same shapes (square powers of two) and the
structure the workload has (Hermitian operators, unitary gates, a mix of
sizes), one recipe per workload:

* ``fixed_real_n32``: 64 real instances, n = 32, entries U[-1, 1] (seed 0), alpha=1, beta=0.
* ``hermitian_unitary_c128``: 4096 complex instances, n = 64; A_i Hermitian, (G + G^H)/2 with
  G = X + iY, X, Y standard normal; B_i Haar unitary (QR of a complex Gaussian,
  columns multiplied by the phases of diag(R)); seed 1, alpha=1, beta=0.
* ``size_mix_uniform``: 20000 real instances, n drawn from {16,...,512} with weights
  {.3,.25,.2,.15,.07,.03}, entries U[-1, 1], alpha=1, beta=0.5, seed 2.
* ``size_mix_loguniform``: the same size mix drawn with seed 3, entries of magnitude
  10^U(-4, 4) with a random sign (A, B and C), alpha=1, beta=0.5.
* ``annealing_chain``: chained products C <- U_t C: a pool of Haar unitaries, a
  [steps, walkers] pool-index table and a Haar-unitary start state per walker.

Draw order (fixed so that every run sees the same numbers): sizes first
(``rng.choice``); then for a grouped batch the whole packed A array in one
draw (instances in table order, each column-major), then all of B, then all
of C; a log-uniform array draws all its magnitudes, then its signs (as random
bits); a complex Gaussian draws its real part before its imaginary part.
Alignment gaps between packed instances are zero.

Memory layout of a batch: every instance is column-major and packed
back-to-back in three flat arrays (A, B, C) at offsets that are multiples of
``ALIGN_ELEMS`` elements; ``table`` holds one int64 row per instance:
m, n, k, lda, ldb, ldc, a_off, b_off, c_off (elements).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ALIGN_ELEMS = 32  # 256 B for FP64, 512 B for complex128

SIZE_MIX_SIZES = (16, 32, 64, 128, 256, 512)
SIZE_MIX_WEIGHTS = (0.30, 0.25, 0.20, 0.15, 0.07, 0.03)


@dataclass
class Batch:
    """A synthetic batch of independent GEMM instances (column-major, packed)."""

    name: str
    dtype: str                 # "r64" or "c128"
    table: np.ndarray          # int64 [count, 9]
    A: np.ndarray              # flat float64 / complex128
    B: np.ndarray
    C: np.ndarray
    alpha: complex
    beta: complex
    meta: dict = field(default_factory=dict)

    @property
    def count(self) -> int:
        return int(self.table.shape[0])

    @property
    def np_dtype(self):
        return np.complex128 if self.dtype == "c128" else np.float64

    def flops(self) -> float:
        """Algorithmic flops: 2mnk per real instance, 8mnk per complex one."""
        t = self.table
        per = 8.0 if self.dtype == "c128" else 2.0
        return float(per * np.sum(t[:, 0].astype(np.float64) * t[:, 1] * t[:, 2]))

    def bytes_moved(self) -> float:
        """Algorithmic bytes: read A and B, write C, read C when beta != 0."""
        t = self.table.astype(np.float64)
        esz = 16.0 if self.dtype == "c128" else 8.0
        c_passes = 2.0 if complex(self.beta) != 0 else 1.0
        return float(esz * np.sum(t[:, 0] * t[:, 2] + t[:, 2] * t[:, 1]
                                  + c_passes * t[:, 0] * t[:, 1]))

    def instance(self, i: int, which: str) -> np.ndarray:
        """View of operand ``which`` ('A', 'B' or 'C') of instance i as a 2-D array."""
        m, n, k, lda, ldb, ldc, ao, bo, co = (int(x) for x in self.table[i])
        if which == "A":
            return self.A[ao:ao + lda * k].reshape((k, lda)).T[:m, :]
        if which == "B":
            return self.B[bo:bo + ldb * n].reshape((n, ldb)).T[:k, :]
        return self.C[co:co + ldc * n].reshape((n, ldc)).T[:m, :]

    def fixed_shape(self):
        """(m, n, k, batch) when every instance has the same shape and stride, else None."""
        return self.meta.get("fixed")


def _round_up(x: int, a: int) -> int:
    return (x + a - 1) // a * a


def pack_table(shapes, align: int = ALIGN_ELEMS) -> tuple[np.ndarray, int, int, int]:
    """Build a packed instance table for (m, n, k) shapes; returns (table, lenA, lenB, lenC)."""
    rows = []
    ao = bo = co = 0
    for (m, n, k) in shapes:
        lda, ldb, ldc = max(m, 1), max(k, 1), max(m, 1)
        rows.append((m, n, k, lda, ldb, ldc, ao, bo, co))
        ao = _round_up(ao + lda * k, align)
        bo = _round_up(bo + ldb * n, align)
        co = _round_up(co + ldc * n, align)
    table = np.array(rows, dtype=np.int64).reshape(-1, 9)
    return table, max(ao, 1), max(bo, 1), max(co, 1)


# ---- element distributions --------------------------------------------------

def _uniform(rng, out: np.ndarray) -> None:
    """U[-1, 1] into a float64 view: -1 + 2 r, r = rng.random()."""
    rng.random(out=out)
    out *= 2.0
    out -= 1.0


_LOG2_10 = float(np.log2(10.0))


def _log_uniform_signed(rng, size: int) -> np.ndarray:
    """Magnitude 10^U(-4, 4) = 2^(log2(10) (8u - 4)) with a random sign (p = 1/2):
    magnitudes first, then sign bits."""
    x = rng.random(size)
    x *= 8.0 * _LOG2_10
    x -= 4.0 * _LOG2_10
    np.exp2(x, out=x)
    bits = np.unpackbits(rng.integers(0, 256, (size + 7) // 8, dtype=np.uint8))[:size]
    np.negative(x, out=x, where=bits.view(bool))
    return x


def complex_gaussian(rng, shape) -> np.ndarray:
    """X + iY with X, Y i.i.d. standard normal (real part drawn first)."""
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return re + 1j * im


def haar_unitary(rng, n: int, count: int = 1) -> np.ndarray:
    """``count`` Haar-distributed n x n unitaries, shape [count, n, n].

    QR of a complex Gaussian matrix, then each column of Q multiplied by the
    phase of the matching diagonal entry of R so that the law is Haar
    (Mezzadri, Notices AMS 54 (2007) 592).
    """
    Z = complex_gaussian(rng, (count, n, n)) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R, axis1=1, axis2=2)
    ph = d / np.abs(d)
    return Q * ph[:, None, :]


def hermitian(rng, n: int, count: int = 1) -> np.ndarray:
    """(G + G^H) / 2 with G a complex Gaussian matrix; shape [count, n, n]."""
    G = complex_gaussian(rng, (count, n, n))
    return 0.5 * (G + np.conj(np.swapaxes(G, 1, 2)))


def _col_major_flat(M: np.ndarray) -> np.ndarray:
    """[count, r, c] stack -> flat array of column-major instances."""
    return np.ascontiguousarray(np.swapaxes(M, 1, 2)).reshape(-1)


# ---- batches ------------------------------------------------------------------

def fixed_uniform(batch: int, m: int, n: int, k: int, seed: int, dtype: str = "r64",
                  alpha=1.0, beta=0.0, name: str | None = None) -> Batch:
    """Fixed-size batch with U[-1, 1] entries (complex: independent real and imaginary parts)."""
    rng = np.random.default_rng(seed)
    table, la, lb, lc = pack_table([(m, n, k)] * batch, align=1)
    dt = np.complex128 if dtype == "c128" else np.float64
    A, B, C = (np.zeros(x, dtype=dt) for x in (la, lb, lc))
    for i in range(batch):
        for X, off, size in ((A, table[i, 6], m * k), (B, table[i, 7], k * n),
                             (C, table[i, 8], m * n)):
            view = X[off:off + size].view(np.float64)
            _uniform(rng, view)
    return Batch(name or f"fixed_{dtype}_{batch}x{m}x{n}x{k}", dtype, table, A, B, C,
                 alpha, beta, meta={"fixed": (m, n, k, batch)})


def fixed_real_n32() -> Batch:
    """64 real instances of n = 32, U[-1, 1] entries, seed 0, C = A B."""
    b = fixed_uniform(64, 32, 32, 32, seed=0, dtype="r64", alpha=1.0, beta=0.0,
                      name="fixed_r64_64x32")
    return b


def hermitian_unitary_c128(batch: int = 4096, n: int = 64) -> Batch:
    """Complex fixed batch: A_i Hermitian, B_i Haar unitary, seed 1, C = A B."""
    rng = np.random.default_rng(1)
    A = hermitian(rng, n, batch)
    B = haar_unitary(rng, n, batch)
    table, la, lb, lc = pack_table([(n, n, n)] * batch, align=1)
    return Batch(f"hermitian_unitary_c128_{batch}x{n}", "c128", table, _col_major_flat(A),
                 _col_major_flat(B), np.zeros(lc, dtype=np.complex128), 1.0, 0.0,
                 meta={"fixed": (n, n, n, batch)})


def draw_sizes(rng, count: int, sizes=SIZE_MIX_SIZES, weights=SIZE_MIX_WEIGHTS) -> np.ndarray:
    return rng.choice(np.asarray(sizes, dtype=np.int64), size=count, p=np.asarray(weights))


def _gap_mask(table: np.ndarray, length: int, rows: int, cols: int, ld: int, off: int):
    """Boolean mask of the elements that belong to some instance of a packed array."""
    keep = np.zeros(length, dtype=bool)
    for t in table:
        r, c, l, o = int(t[rows]), int(t[cols]), int(t[ld]), int(t[off])
        if r == l:
            keep[o:o + r * c] = True
        else:
            for j in range(c):
                keep[o + j * l:o + j * l + r] = True
    return keep


def mixed_batch(seed: int, count: int, values: str, alpha=1.0, beta=0.5, sizes=SIZE_MIX_SIZES,
                weights=SIZE_MIX_WEIGHTS, name: str | None = None) -> Batch:
    """Grouped real batch of square instances with sizes drawn from ``sizes``.

    ``values`` is "uniform" (U[-1, 1]) or "loguniform" (10^U(-4,4), random sign).
    """
    rng = np.random.default_rng(seed)
    ns = draw_sizes(rng, count, sizes, weights)
    return batch_of_sizes(rng, ns, values, alpha, beta,
                          name or f"mixed_{values}_{count}_seed{seed}")


def batch_of_sizes(rng, ns, values: str, alpha=1.0, beta=0.5, name: str = "sized") -> Batch:
    """Square real instances of the given sizes, packed, values drawn from ``rng``
    (A, then B, then C, as in ``mixed_batch``)."""
    ns = np.asarray(ns, dtype=np.int64)
    table, la, lb, lc = pack_table([(int(n), int(n), int(n)) for n in ns])
    out = []
    for length, (rows, cols, ld, off) in ((la, (0, 2, 3, 6)), (lb, (2, 1, 4, 7)),
                                          (lc, (0, 1, 5, 8))):
        if values == "uniform":
            X = np.empty(length)
            _uniform(rng, X)
        else:
            X = _log_uniform_signed(rng, length)
        dense = int(np.sum(table[:, rows] * table[:, cols]))
        if dense != length:
            X[~_gap_mask(table, length, rows, cols, ld, off)] = 0.0
        out.append(X)
    A, B, C = out
    return Batch(name, "r64", table, A, B, C, alpha, beta, meta={"sizes": ns})



def size_mix_uniform(count: int = 20000) -> Batch:
    return mixed_batch(2, count, "uniform", 1.0, 0.5, name=f"size_mix_uniform_{count}")


def size_mix_loguniform(count: int = 20000) -> Batch:
    return mixed_batch(3, count, "loguniform", 1.0, 0.5, name=f"size_mix_loguniform_{count}")


@dataclass
class Chain:
    """Chained products C_w <- U_{idx[t, w]} C_w (annealing-shaped workload)."""

    n_walker: np.ndarray        # int64 [W]: matrix size of each walker
    pools: dict                 # n -> complex128 [P_n, n, n] unitaries
    idx: np.ndarray             # int32 [T, W]: index into the walker's size pool
    C0: list                    # per walker complex128 [n, n] start state

    @property
    def steps(self) -> int:
        return int(self.idx.shape[0])

    @property
    def walkers(self) -> int:
        return int(self.idx.shape[1])


def annealing_chain(walkers_small: int = 960, walkers_large: int = 64, n_small: int = 256,
            n_large: int = 1024, steps: int = 200, pool_small: int = 64,
            pool_large: int = 16) -> Chain:
    """Seed-4 chain: Haar pools, a uniform pool-index table, Haar start states.

    Draw order: pool of n_small, pool of n_large, index table for all walkers
    (row t, walkers in order; each index uniform over its size's pool), start
    states of the small walkers, start states of the large walkers.
    """
    rng = np.random.default_rng(4)
    pools = {}
    if walkers_small:
        pools[n_small] = haar_unitary(rng, n_small, pool_small)
    if walkers_large:
        pools[n_large] = haar_unitary(rng, n_large, pool_large)
    nw = np.array([n_small] * walkers_small + [n_large] * walkers_large, dtype=np.int64)
    hi = np.array([pool_small] * walkers_small + [pool_large] * walkers_large, dtype=np.int64)
    idx = (rng.random((steps, nw.size)) * hi[None, :]).astype(np.int32)
    idx = np.minimum(idx, (hi - 1)[None, :].astype(np.int32))
    C0 = []
    if walkers_small:
        C0 += list(haar_unitary(rng, n_small, walkers_small))
    if walkers_large:
        C0 += list(haar_unitary(rng, n_large, walkers_large))
    return Chain(nw, pools, idx, C0)


def chain_layout(chain: Chain):
    """Packs a chain for chain_plan / chain_step: the pool (all sizes, column-major,
    back to back) with each entry's size and offset, the walkers' start states
    with their offsets, and the [steps, walkers] table of global pool indices.
    Returns (pool, pool_n, pool_off, states, state_off, gidx)."""
    sizes = sorted(chain.pools)
    pool_n, pool_off, chunks, base = [], [], [], {}
    off = 0
    for n in sizes:
        base[n] = len(pool_n)
        for U in chain.pools[n]:
            pool_n.append(n)
            pool_off.append(off)
            chunks.append(np.asfortranarray(U).ravel(order="F"))
            off += n * n
    state_off, st = [], []
    off = 0
    for C in chain.C0:
        state_off.append(off)
        st.append(np.asfortranarray(C).ravel(order="F"))
        off += C.shape[0] ** 2
    first = np.array([base[int(n)] for n in chain.n_walker], dtype=np.int64)
    gidx = (chain.idx.astype(np.int64) + first[None, :]).astype(np.int32)
    return (np.concatenate(chunks), np.array(pool_n, dtype=np.int64),
            np.array(pool_off, dtype=np.int64), np.concatenate(st),
            np.array(state_off, dtype=np.int64), gidx)
