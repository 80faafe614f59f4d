"""Parity at the full benchmark sizes, in the launch configuration bench.py times.

* 4096 complex instances of n = 64 (Hermitian A, Haar-unitary B): every
  instance against the oracle, FP64 and all split modes (fixed-size call).
* 20000 real instances, n in {16..512}, U[-1,1], beta = 0.5: autotuned FP64
  plan; a sample of instances against the oracle, computed one by one.
* 20000 real instances of the same size mix with log-uniform magnitudes
  1e-4..1e4: FP64 and 3/6/9-slice plans; a sample against the oracle and
  every instance against the FP64 path (device-side error kernel).
* 960 + 64 complex walkers (n = 256 and 1024) with their Haar pools: two
  chained steps, sampled walkers step-locally against the oracle, and the
  unitarity drift of every walker.
* the rectangular operator shapes of Sec. 3 (S = 13, 15, 17 spins).
"""
import numpy as np
import pytest

import oracle
import paper_2203_09353_gb300 as bg
from paper_2203_09353_gb300 import synth

from gpu_util import TOL_FP64, TOL_SPLIT, dev, errors, host, oracle_batch, oracle_subset, \
    subset_errors

pytestmark = pytest.mark.gpu


def _sample(count: int, every: int, seed: int) -> np.ndarray:
    """Every `every`-th instance from a random start: table order is random, so all
    size classes appear."""
    start = int(np.random.default_rng(seed).integers(0, every))
    return np.arange(start, count, every)


def test_complex_hermitian_unitary_4096_all_instances(gpu):
    b = synth.hermitian_unitary_c128()
    assert b.count == 4096 and b.fixed_shape() == (64, 64, 64, 4096)
    ref = oracle_batch(b)
    A, B = dev(b.A), dev(b.B)
    for prec, tol in ((None, TOL_FP64), (bg.precision("split", 3), TOL_SPLIT[3]),
                      (bg.precision("split", 6), TOL_SPLIT[6]),
                      (bg.precision("split", 9), TOL_SPLIT[9])):
        C = dev(b.C)
        bg.batched_gemm_fixed("c128", 64, 64, 64, b.alpha, A, 64, 64 * 64, B, 64, 64 * 64,
                              b.beta, C, 64, 64 * 64, b.count, prec)
        e = errors(b, host(C), ref)
        assert e.max() <= tol, (prec and prec.slices, e.max())


def test_uniform_size_mix_20000_fp64_autotuned(gpu, tmp_path):
    b = synth.size_mix_uniform()
    assert b.count == 20000
    flags = bg.BG_PLAN_AUTOTUNE | bg.BG_PLAN_USE_CACHE
    plan = bg.batched_gemm_plan("r64", b.table, None, flags, str(tmp_path / "tune.json"))
    C = dev(b.C)
    bg.batched_gemm_grouped(plan, dev(b.A), dev(b.B), C, b.alpha, b.beta)
    ids = _sample(b.count, 40, 1)
    e = subset_errors(b, host(C), oracle_subset(b, ids))
    assert e.max() <= TOL_FP64, e.max()
    bg.check_device_errors()


@pytest.fixture(scope="module")
def loguniform_20000():
    return synth.size_mix_loguniform()


def test_loguniform_size_mix_20000_all_modes(gpu, loguniform_20000):
    import torch
    b = loguniform_20000
    assert b.count == 20000
    A, B, C0 = dev(b.A), dev(b.B), dev(b.C)
    dtab = torch.from_numpy(b.table).cuda()
    ids = _sample(b.count, 40, 2)
    ref = oracle_subset(b, ids)
    out = {}
    for mode in ("fp64", "split3", "split6", "split9"):
        prec = None if mode == "fp64" else bg.precision("split", int(mode[5:]))
        flags = bg.BG_PLAN_PROFILE | (bg.BG_PLAN_AUTOTUNE if mode == "fp64" else 0)
        plan = bg.batched_gemm_plan("r64", b.table, prec, flags)
        C = C0.clone()
        bg.batched_gemm_grouped(plan, A, B, C, b.alpha, b.beta)
        e = subset_errors(b, host(C), ref)
        tol = TOL_FP64 if mode == "fp64" else TOL_SPLIT[int(mode[5:])]
        assert e.max() <= tol, (mode, e.max())
        out[mode] = C
        plan.close()
    bg.check_device_errors()
    err = torch.zeros(b.count, dtype=torch.float64, device="cuda")
    for s in (3, 6, 9):
        bg.rel_err("r64", dtab, A, B, out[f"split{s}"], out["fp64"], err, b.count)
        assert float(err.max()) <= TOL_SPLIT[s] + TOL_FP64, (s, float(err.max()))


@pytest.mark.parametrize("S", [13, 15, 17])
def test_sec3_rectangular_shapes(gpu, S):
    """The operator shapes of Sec. 3 for S spins: M = N = 2^(S - floor(S/2)),
    K = 2^floor(S/2), complex, in one grouped call per mode."""
    rng = np.random.default_rng(S)
    M = N = 2 ** (S - S // 2)
    K = 2 ** (S // 2)
    shapes = [(M, N, K)] * 3
    table, la, lb, lc = synth.pack_table(shapes)
    A = synth.complex_gaussian(rng, la)
    B = synth.complex_gaussian(rng, lb)
    C = synth.complex_gaussian(rng, lc)
    b = synth.Batch(f"sec3_S{S}", "c128", table, A, B, C, 1.0 + 0.5j, 0.5)
    ref = oracle_batch(b)
    for prec, tol in ((None, TOL_FP64), (bg.precision("split", 3), TOL_SPLIT[3]),
                      (bg.precision("split", 6), TOL_SPLIT[6]),
                      (bg.precision("split", 9), TOL_SPLIT[9])):
        plan = bg.batched_gemm_plan("c128", table, prec)
        Cd = dev(C)
        bg.batched_gemm_grouped(plan, dev(A), dev(B), Cd, b.alpha, b.beta)
        e = errors(b, host(Cd), ref)
        assert e.max() <= tol, (S, prec and prec.slices, e.max())
        plan.close()


def test_chain_1024_walkers_two_steps(gpu):
    import torch
    from test_gpu_chain import layout
    ch = synth.annealing_chain()
    assert ch.walkers == 1024 and ch.steps == 200
    pool, pn, po, states, wo, gidx = layout(ch)
    dpool = dev(pool)
    small = [w for w in _sample(960, 120, 3)]
    large = [960 + int(np.random.default_rng(4).integers(0, 64))]
    for mode, s in (("fp64", 0), ("split", 9)):
        plan = bg.chain_plan("c128", ch.n_walker, wo, pn, po, bg.precision(mode, s))
        cur = states
        for t in range(2):
            ping, pong = dev(cur), dev(np.zeros_like(cur))
            bg.chain_step(plan, dpool, dev(gidx[t:t + 1]), ping, pong, 1)
            nxt = host(pong)
            for w in small + (large if t == 0 else []):
                n = int(ch.n_walker[w])
                prev = cur[wo[w]:wo[w] + n * n].reshape(n, n).T
                U = ch.pools[n][ch.idx[t, w]]
                got = nxt[wo[w]:wo[w] + n * n].reshape(n, n).T
                e = np.linalg.norm(got - oracle.matmul(U, prev)) / (
                    np.linalg.norm(U) * np.linalg.norm(prev))
                assert e <= (TOL_FP64 if mode == "fp64" else TOL_SPLIT[9]), (mode, t, w, e)
            cur = nxt
        dn = torch.tensor(ch.n_walker, dtype=torch.int64, device="cuda")
        do = torch.tensor(wo, dtype=torch.int64, device="cuda")
        drift = torch.zeros(ch.walkers, dtype=torch.float64, device="cuda")
        bg.unitarity_drift("c128", dn, do, dev(cur), drift, ch.walkers)
        # ||C^H C - I||_F of a product of numerically unitary factors grows like
        # n^1.5 eps per factor; a 3-slice-level error would show as ~1e-6
        scaled = host(drift) / ch.n_walker.astype(np.float64) ** 1.5
        assert scaled.max() < 1e-13, (mode, float(scaled.max()))
        plan.close()
