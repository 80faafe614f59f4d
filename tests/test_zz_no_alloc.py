"""The allocation-free split entry point (C ABI batched_gemm_fixed_static).

Its results must match batched_gemm_fixed in the same split mode, call after
call, although every call reuses the one static device array for all of its
workspace (the second call finds the first one's leftovers there). A batch
whose workspace exceeds the array is refused before any work is queued. The
file is named to be collected last, so that it also runs after every other
GPU test in one process; it passes on its own as well.
"""
import numpy as np
import pytest

import paper_2203_09353_gb300 as bg
from paper_2203_09353_gb300 import synth

from gpu_util import TOL_SPLIT, dev, errors, host, oracle_batch, run_fixed

pytestmark = pytest.mark.gpu

STATIC_SCRATCH_BYTES = 64 << 20


def run_static(batch, prec):
    m, n, k, count = batch.fixed_shape()
    A, B, C = dev(batch.A), dev(batch.B), dev(batch.C)
    bg.batched_gemm_fixed_static(batch.dtype, m, n, k, batch.alpha, A, max(m, 1), m * k, B,
                                 max(k, 1), k * n, batch.beta, C, max(m, 1), m * n, count, prec)
    return C


def cases():
    return [
        (synth.fixed_uniform(200, 40, 33, 47, seed=21, dtype="r64", alpha=0.5, beta=0.25),
         bg.precision("split", 9, 0)),
        (synth.fixed_uniform(100, 20, 24, 30, seed=22, dtype="c128", alpha=0.5 + 1j,
                             beta=0.25 - 1j),
         bg.precision("split", 6, 0)),
    ]


def test_two_calls_match_fixed_entry(gpu):
    """Two calls in a row (different dtype, shape and slice count) each agree with
    batched_gemm_fixed and with the oracle within the split tolerance."""
    for b, prec in cases():
        got = host(run_static(b, prec))
        ref_fixed = host(run_fixed(b, prec))
        s = prec.slices
        assert errors(b, got, ref_fixed).max() <= TOL_SPLIT[s]
        assert errors(b, got, oracle_batch(b)).max() <= TOL_SPLIT[s]


def test_repeat_allocates_no_device_memory(gpu):
    """After the first call on the device (set-up, module load), further calls of
    new sizes leave the device's free memory unchanged."""
    import torch
    first, prec = cases()[0]
    run_static(first, prec)
    b = synth.fixed_uniform(100, 24, 40, 70, seed=23, dtype="r64", alpha=1.0, beta=0.5)
    m, n, k, count = b.fixed_shape()
    A, B, C = dev(b.A), dev(b.B), dev(b.C)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        bg.batched_gemm_fixed_static("r64", m, n, k, 1.0, A, m, m * k, B, k, k * n, 0.5, C, m,
                                     m * n, count, prec)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    # beta = 0.5 applied twice on the same C
    b2 = synth.Batch(b.name, b.dtype, b.table, b.A, b.B, oracle_batch(b), 1.0, 0.5)
    assert errors(b2, host(C), oracle_batch(b2)).max() <= TOL_SPLIT[9]


def test_oversize_batch_is_refused(gpu):
    b = synth.fixed_uniform(400, 128, 128, 128, seed=24, dtype="r64", alpha=1.0, beta=0.0)
    m, n, k, count = b.fixed_shape()
    A, B, C = dev(b.A), dev(b.B), dev(b.C)
    with pytest.raises(bg.BgemmError) as ei:
        bg.batched_gemm_fixed_static("r64", m, n, k, 1.0, A, m, m * k, B, k, k * n, 0.0, C, m,
                                     m * n, count, bg.precision("split", 9, 0))
    assert ei.value.status == 1
    assert str(STATIC_SCRATCH_BYTES) in str(ei.value)
    assert np.array_equal(host(C), b.C)


def test_fp64_mode_is_refused(gpu):
    b = synth.fixed_uniform(4, 8, 8, 8, seed=25, dtype="r64", alpha=1.0, beta=0.0)
    with pytest.raises(bg.BgemmError) as ei:
        run_static(b, bg.precision("fp64"))
    assert ei.value.status == 1


def test_capture_is_refused(gpu):
    """The call uploads host tables that it frees on return, so a call inside a
    stream capture is refused (BG_ERR_CAPTURE) before anything is queued."""
    import torch
    b, prec = cases()[0]
    m, n, k, count = b.fixed_shape()
    A, B, C = dev(b.A), dev(b.B), dev(b.C)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    status = None
    with torch.cuda.graph(g):
        try:
            bg.batched_gemm_fixed_static(b.dtype, m, n, k, b.alpha, A, m, m * k, B, k, k * n,
                                         b.beta, C, m, m * n, count, prec)
        except bg.BgemmError as e:
            status = e.status
    assert status == 5
    torch.cuda.synchronize()
    assert np.array_equal(host(C), b.C)
