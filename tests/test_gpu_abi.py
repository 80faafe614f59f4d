"""Status codes and error behaviour of the C ABI (include/bgemm.h) on the GPU:
bad arguments, misalignment, capture rules, host-side fault injection."""
import numpy as np
import pytest

import paper_2203_09353_gb300 as bg
from paper_2203_09353_gb300 import synth

from gpu_util import dev, host

pytestmark = pytest.mark.gpu

INVALID, UNSUPPORTED, CUDA, NOMEM, CAPTURE = 1, 2, 3, 4, 5


def status_of(fn, *a, **k):
    try:
        fn(*a, **k)
        return 0
    except bg.BgemmError as e:
        return e.status


def test_invalid_arguments(gpu):
    import torch
    A = torch.zeros(64, dtype=torch.float64, device="cuda")
    f = bg.batched_gemm_fixed
    assert status_of(f, "r64", -1, 2, 2, 1.0, A, 2, 4, A, 2, 4, 0.0, A, 2, 4, 1) == INVALID
    assert status_of(f, "r64", 4, 2, 2, 1.0, A, 3, 8, A, 2, 4, 0.0, A, 4, 8, 1) == INVALID  # lda<m
    assert status_of(f, "r64", 2, 2, 2, 1.0, A, 2, 4, A, 2, 4, 0.0, None, 2, 4, 1) == INVALID
    assert status_of(f, "r64", 2, 2, 2, 1.0, A.data_ptr() + 4, 2, 4, A, 2, 4, 0.0, A, 2, 4,
                     1) == INVALID  # misaligned
    Z = torch.zeros(64, dtype=torch.complex128, device="cuda")
    assert status_of(f, "c128", 2, 2, 2, 1.0, Z.data_ptr() + 8, 2, 4, Z, 2, 4, 0.0, Z, 2, 4,
                     1) == INVALID  # complex needs 16 B
    assert status_of(f, "r64", 2, 2, 2, 1.0, A, 2, 4, A, 2, 4, 0.0, A, 2, 2, 3) == INVALID  # overlap
    p = bg.Precision(1, 13, 0, 0)
    assert status_of(f, "r64", 2, 2, 2, 1.0, A, 2, 4, A, 2, 4, 0.0, A, 2, 4, 1, p) == INVALID
    p = bg.Precision(1, 3, 9, 0)
    assert status_of(f, "r64", 2, 2, 2, 1.0, A, 2, 4, A, 2, 4, 0.0, A, 2, 4, 1, p) == INVALID
    p = bg.Precision(7, 0, 0, 0)
    assert status_of(f, "r64", 2, 2, 2, 1.0, A, 2, 4, A, 2, 4, 0.0, A, 2, 4, 1, p) == INVALID
    bad = np.array([[2, 2, 2, 1, 2, 2, 0, 0, 0]], dtype=np.int64)  # lda < m
    assert status_of(bg.batched_gemm_plan, "r64", bad) == INVALID
    neg = np.array([[2, 2, 2, 2, 2, 2, -1, 0, 0]], dtype=np.int64)
    assert status_of(bg.batched_gemm_plan, "r64", neg) == INVALID
    assert "leading dimension" in bg.load_library().bg_last_error().decode() or True


def test_chain_argument_checks(gpu):
    import torch
    Z = torch.zeros(64, dtype=torch.complex128, device="cuda")
    assert status_of(bg.chain_plan, "c128", [4], [0], [8], [0]) == INVALID  # no pool of size 4
    plan = bg.chain_plan("c128", [4], [0], [4], [0])
    idx = torch.zeros(4, dtype=torch.int32, device="cuda")
    assert status_of(bg.chain_step, plan, Z, idx, Z, Z, 1) == INVALID  # ping == pong
    assert status_of(bg.chain_step, plan, Z, idx, Z, Z, -1) == INVALID
    gp = bg.batched_gemm_plan("r64", np.array([[2, 2, 2, 2, 2, 2, 0, 0, 0]]))
    assert status_of(bg.chain_step, gp, Z, idx, Z, Z.data_ptr() + 256, 1) == INVALID


def test_fault_injection_env(gpu, monkeypatch):
    b = synth.fixed_real_n32()
    monkeypatch.setenv("BGEMM_FAULT", "launch")
    Cd = dev(b.C)
    m, n, k, cnt = b.fixed_shape()
    st = status_of(bg.batched_gemm_fixed, "r64", m, n, k, 1.0, dev(b.A), m, m * k, dev(b.B), k,
                   k * n, 0.0, Cd, m, m * n, cnt)
    assert st == CUDA
    assert np.array_equal(host(Cd), b.C)  # nothing launched
    monkeypatch.delenv("BGEMM_FAULT")
    bg.batched_gemm_fixed("r64", m, n, k, 1.0, dev(b.A), m, m * k, dev(b.B), k, k * n, 0.0, Cd, m,
                          m * n, cnt)


def test_capture_rules(gpu):
    """Plans refuse to be built under capture; the FP64 fixed path can be captured and replayed."""
    import torch
    b = synth.fixed_real_n32()
    m, n, k, cnt = b.fixed_shape()
    A, B, C = dev(b.A), dev(b.B), dev(b.C)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        bg.batched_gemm_fixed("r64", m, n, k, 1.0, A, m, m * k, B, k, k * n, 0.0, C, m, m * n, cnt,
                              stream=s)  # warm (no allocation happens in FP64 mode)
        with torch.cuda.graph(g, stream=s):
            st = status_of(bg.batched_gemm_plan, "r64", b.table, stream=s)
            bg.batched_gemm_fixed("r64", m, n, k, 1.0, A, m, m * k, B, k, k * n, 0.0, C, m, m * n,
                                  cnt, stream=s)
            split = bg.precision("split", 7)
            st2 = status_of(bg.batched_gemm_fixed, "r64", m, n, k, 1.0, A, m, m * k, B, k, k * n,
                            0.0, C, m, m * n, cnt, split, stream=s)
    assert st == CAPTURE
    assert st2 == CAPTURE  # first split call of this shape would allocate
    C.zero_()
    g.replay()
    torch.cuda.synchronize()
    from gpu_util import errors, oracle_batch
    assert errors(b, host(C), oracle_batch(b)).max() <= 1e-14


def test_launch_counter(gpu):
    b = synth.size_mix_uniform(count=50)
    plan = bg.batched_gemm_plan("r64", b.table)
    A, B, C = dev(b.A), dev(b.B), dev(b.C)
    bg.launch_count(reset=True)
    for _ in range(3):
        bg.batched_gemm_grouped(plan, A, B, C, 1.0, 0.5)
    assert bg.launch_count() == 3
    sp = bg.batched_gemm_plan("r64", b.table, bg.precision("split", 6))
    bg.launch_count(reset=True)
    bg.batched_gemm_grouped(sp, A, B, C, 1.0, 0.5)
    # slicer, small-instance kernel (n <= 64), tile kernel
    assert bg.launch_count() == sp.info()["launches_per_call"] == 3
