"""Argument checks of the Python binding that run before any device work, so
they hold on a machine without a GPU: wrong element types and undersized
buffers of the local gate are refused with ValueError."""
import pytest
import torch

import paper_2203_09353_gb300 as bg


def test_gate_wrapper_rejects_bad_types_and_sizes():
    S, W = 5, 2
    st = torch.zeros(W << S, dtype=torch.complex128)
    s32 = torch.zeros(W, dtype=torch.int32)
    g = torch.zeros(16 * W, dtype=torch.complex128)
    cases = {
        "sites must be torch.int32": dict(states=st, sites=s32.to(torch.int64), gates=g),
        "states holds": dict(states=st[:-1], sites=s32, gates=g),
        "gates holds": dict(states=st, sites=s32, gates=g[:-1]),
        "states must be torch.complex128": dict(states=st.to(torch.complex64), sites=s32, gates=g),
    }
    for msg, kw in cases.items():
        with pytest.raises(ValueError, match=msg):
            bg.apply_local_gate(kw["states"], S, kw["sites"], kw["gates"])
    # well-formed host tensors pass the type and size checks and stop at the device check
    with pytest.raises(ValueError, match="current CUDA device"):
        bg.apply_local_gate(st, S, s32, g)
