"""GPU parity of the FP64 / complex128 path of Eq. (1) against the CPU oracle.

Tolerance: per-instance ||C - C_ref||_F / (||A||_F ||B||_F) <= 1e-14 (both
sides round differently: the kernels use FMA and their own summation order).
"""
import numpy as np
import pytest

import paper_2203_09353_gb300 as bg
from paper_2203_09353_gb300 import synth

from gpu_util import TOL_FP64, dev, errors, host, oracle_batch, run_fixed, run_grouped

pytestmark = pytest.mark.gpu


def test_fixed_real_n32(gpu):
    b = synth.fixed_real_n32()
    C = host(run_fixed(b))
    e = errors(b, C, oracle_batch(b))
    assert e.max() <= TOL_FP64, e.max()


def test_hermitian_unitary_c128_reduced(gpu):
    b = synth.hermitian_unitary_c128(batch=96)
    C = host(run_fixed(b))
    e = errors(b, C, oracle_batch(b))
    assert e.max() <= TOL_FP64, e.max()


@pytest.mark.parametrize("dtype", ["r64", "c128"])
@pytest.mark.parametrize("mnk", [(1, 1, 1), (3, 5, 7), (17, 17, 17), (33, 31, 29), (100, 64, 37),
                                 (257, 130, 65), (16, 512, 16), (512, 16, 8), (5, 3, 0)])
def test_fixed_ragged_shapes(gpu, dtype, mnk):
    m, n, k = mnk
    b = synth.fixed_uniform(5, m, n, k, seed=m * 1000 + n * 10 + k, dtype=dtype, alpha=1.5,
                            beta=-0.25)
    C = host(run_fixed(b))
    e = errors(b, C, oracle_batch(b))
    assert e.max() <= TOL_FP64, e.max()


@pytest.mark.parametrize("dtype", ["r64", "c128"])
def test_padded_leading_dims_and_gaps(gpu, dtype):
    """ld > rows and instance strides with gaps: padding must stay untouched."""
    rng = np.random.default_rng(3)
    m, n, k, batch = 19, 23, 29, 7
    lda, ldb, ldc = m + 5, k + 2, m + 3
    sA, sB, sC = lda * k + 11, ldb * n + 4, ldc * n + 9
    dt = np.complex128 if dtype == "c128" else np.float64

    def fill(size):
        x = rng.uniform(-1, 1, size)
        if dtype == "c128":
            x = x + 1j * rng.uniform(-1, 1, size)
        return x.astype(dt)

    A, B, C0 = fill(sA * batch), fill(sB * batch), fill(sC * batch)
    alpha = 0.75 - 0.5j if dtype == "c128" else 0.75
    beta = 1.25 + 0.25j if dtype == "c128" else 1.25
    Cd = dev(C0)
    bg.batched_gemm_fixed(dtype, m, n, k, alpha, dev(A), lda, sA, dev(B), ldb, sB, beta, Cd, ldc,
                          sC, batch)
    got = host(Cd)
    ref = C0.copy()
    import oracle
    oracle.gemm_fixed(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, ref, ldc, sC, batch)
    mask = np.zeros(ref.size, dtype=bool)
    for i in range(batch):
        for j in range(n):
            mask[i * sC + j * ldc: i * sC + j * ldc + m] = True
    assert np.array_equal(got[~mask], C0[~mask])
    for i in range(batch):
        a = A[i * sA:i * sA + lda * k].reshape(k, lda).T[:m]
        bb = B[i * sB:i * sB + ldb * n].reshape(n, ldb).T[:k]
        g = got[i * sC:i * sC + ldc * n].reshape(n, ldc).T[:m]
        r = ref[i * sC:i * sC + ldc * n].reshape(n, ldc).T[:m]
        assert np.linalg.norm(g - r) <= TOL_FP64 * np.linalg.norm(a) * np.linalg.norm(bb)


@pytest.mark.parametrize("dtype", ["r64", "c128"])
def test_alpha_beta_rules(gpu, dtype):
    """beta = 0 never reads C (NaN stays out); alpha = 0 never reads A or B."""
    b = synth.fixed_uniform(9, 20, 20, 20, seed=4, dtype=dtype, alpha=2.0, beta=0.0)
    Cn = np.full_like(b.C, np.nan)
    C = host(run_fixed(b, C=Cn))
    assert np.all(np.isfinite(C))
    e = errors(b, C, oracle_batch(b, C0=np.zeros_like(b.C)))
    assert e.max() <= TOL_FP64
    m, n, k, cnt = b.fixed_shape()
    An = dev(np.full_like(b.A, np.nan))
    Bn = dev(np.full_like(b.B, np.inf))
    Cd = dev(b.C)
    bg.batched_gemm_fixed(dtype, m, n, k, 0.0, An, m, m * k, Bn, k, k * n, 0.5, Cd, m, m * n, cnt)
    assert np.array_equal(host(Cd), 0.5 * b.C)


def test_empty_batch_is_noop(gpu):
    b = synth.fixed_uniform(3, 4, 4, 4, seed=1)
    Cd = dev(b.C)
    for (m, n, k, cnt) in ((0, 4, 4, 3), (4, 0, 4, 3), (4, 4, 4, 0)):
        bg.batched_gemm_fixed("r64", m, n, k, 1.0, dev(b.A), 4, 16, dev(b.B), 4, 16, 0.0, Cd, 4, 16,
                              cnt)
    assert np.array_equal(host(Cd), b.C)


@pytest.mark.parametrize("values", ["uniform", "loguniform"])
def test_grouped_mixed_sizes_reduced(gpu, values):
    """The size mix (all six classes present), U[-1, 1] and log-uniform values, at a
    reduced count, one persistent launch."""
    b = synth.size_mix_uniform(count=160) if values == "uniform" else synth.size_mix_loguniform(count=160)
    assert set(np.unique(b.table[:, 0])) == set(synth.SIZE_MIX_SIZES)
    C, plan = run_grouped(b)
    assert plan.info()["launches_per_call"] == 1
    e = errors(b, host(C), oracle_batch(b))
    assert e.max() <= TOL_FP64, e.max()


@pytest.mark.parametrize("dtype", ["r64", "c128"])
def test_grouped_ragged_and_degenerate(gpu, dtype):
    """Arbitrary shapes, zero sizes, k = 0 and padded leading dimensions in one plan."""
    rng = np.random.default_rng(21)
    shapes = [(int(rng.integers(0, 70)), int(rng.integers(0, 70)), int(rng.integers(0, 70)))
              for _ in range(60)] + [(0, 0, 0), (7, 9, 0), (1, 300, 2), (300, 1, 2), (129, 65, 200)]
    table, la, lb, lc = synth.pack_table(shapes, align=7)
    table[:, 3] += 2  # lda padding
    table[:, 5] += 1  # ldc padding
    ao = bo = co = 0
    for i, (m, n, k) in enumerate(shapes):
        table[i, 6], table[i, 7], table[i, 8] = ao, bo, co
        ao += table[i, 3] * max(k, 1) + 3
        bo += table[i, 4] * max(n, 1) + 5
        co += table[i, 5] * max(n, 1) + 1
    dt = np.complex128 if dtype == "c128" else np.float64

    def fill(size):
        x = rng.uniform(-1, 1, size)
        return (x + 1j * rng.uniform(-1, 1, size)).astype(dt) if dtype == "c128" else x

    b = synth.Batch("ragged", dtype, table, fill(ao + 8), fill(bo + 8), fill(co + 8),
                    (1.0 - 2.0j) if dtype == "c128" else -1.5, (0.5 + 0.5j) if dtype == "c128" else 0.5)
    C, _ = run_grouped(b)
    e = errors(b, host(C), oracle_batch(b))
    assert e.max() <= TOL_FP64, e.max()


def test_graph_replay_is_bitwise_deterministic(gpu):
    b = synth.size_mix_uniform(count=80)
    plan = bg.batched_gemm_plan("r64", b.table, None, bg.BG_PLAN_CAPTURE_GRAPH)
    A, B = dev(b.A), dev(b.B)
    outs = []
    for _ in range(3):
        C = dev(b.C)
        bg.batched_gemm_grouped(plan, A, B, C, b.alpha, b.beta)
        outs.append(host(C))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
    e = errors(b, outs[0], oracle_batch(b))
    assert e.max() <= TOL_FP64


def test_autotune_and_cache(gpu, tmp_path):
    b = synth.size_mix_uniform(count=120)
    cache = str(tmp_path / "tune.json")
    flags = bg.BG_PLAN_AUTOTUNE | bg.BG_PLAN_USE_CACHE
    plan = bg.batched_gemm_plan("r64", b.table, None, flags, cache)
    import json
    desc = json.loads(plan.describe())
    assert any(c["tried"] for c in desc["classes"])
    saved = json.load(open(cache))
    assert len(saved) >= 1
    plan2 = bg.batched_gemm_plan("r64", b.table, None, flags, cache)
    assert json.loads(plan2.describe())["classes"][0]["program"] == desc["classes"][0]["program"]
    C, _ = run_grouped(b, plan=plan)
    e = errors(b, host(C), oracle_batch(b))
    assert e.max() <= TOL_FP64


def test_dmma_program_matches_oracle(gpu):
    """The FP64 tensor-core (mma.sync m8n8k4) tile program, forced through the cache."""
    import json
    import os
    import tempfile
    b = synth.size_mix_uniform(count=60)
    plan0 = bg.batched_gemm_plan("r64", b.table)
    keys = []
    for c in json.loads(plan0.describe())["classes"]:
        keys.append(c["bucket"])
    d = tempfile.mkdtemp()
    cache = os.path.join(d, "force_dmma.json")
    import torch
    gpu_name = torch.cuda.get_device_name(0).replace('"', "_")
    with open(cache, "w") as f:
        f.write("{\n")
        lines = []
        for (km, kn, kk) in keys:
            prog = 2 if km * kn > 1024 else 0
            lines.append(f'  "{gpu_name}|r64|fp640|{km}x{kn}x{kk}": {{"prog": {prog}, "ms": 0}}')
        f.write(",\n".join(lines) + "\n}\n")
    plan = bg.batched_gemm_plan("r64", b.table, None, bg.BG_PLAN_USE_CACHE, cache)
    progs = {c["program"] for c in json.loads(plan.describe())["classes"]}
    assert "r64_tile64_dmma" in progs, progs
    C, _ = run_grouped(b, plan=plan)
    e = errors(b, host(C), oracle_batch(b))
    assert e.max() <= TOL_FP64, e.max()
