"""Helpers shared by the GPU parity tests: move seeded batches to the device,
run the library through its C ABI, compute the oracle's answer on the CPU."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2203_09353_gb300 as bg
from conftest import rel_err_instances

TOL_FP64 = 1e-14
TOL_SPLIT = {3: 1e-6, 6: 1e-12, 9: 1e-12}


def dev(x: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t) -> np.ndarray:
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def oracle_batch(batch, C0=None) -> np.ndarray:
    """Oracle result of Eq. (1) for a packed batch (CPU, test infrastructure)."""
    C = (batch.C if C0 is None else C0).copy()
    oracle.gemm_grouped(batch.table, batch.alpha, batch.A, batch.B, batch.beta, C)
    return C


def oracle_subset(batch, ids) -> dict:
    """Oracle result for selected instances only: {i: 2-D array}."""
    out = {}
    for i in ids:
        A = np.asfortranarray(batch.instance(i, "A"))
        B = np.asfortranarray(batch.instance(i, "B"))
        C = np.asfortranarray(batch.instance(i, "C")).copy()
        m, n, k = (int(x) for x in batch.table[i, :3])
        a, b, c = (np.ravel(X, order="F") for X in (A, B, C))
        c = c.copy()
        oracle.gemm_fixed(m, n, k, batch.alpha, a, max(m, 1), m * k, b, max(k, 1), k * n,
                          batch.beta, c, max(m, 1), m * n, 1)
        out[i] = c.reshape((n, m)).T if m * n else np.zeros((m, n), dtype=batch.np_dtype)
    return out


def subset_errors(batch, C_test: np.ndarray, ref: dict) -> np.ndarray:
    errs = []
    for i, cr in ref.items():
        m, n, k, lda, ldb, ldc, ao, bo, co = (int(x) for x in batch.table[i])
        ct = C_test[co:co + ldc * n].reshape((n, ldc)).T[:m, :]
        den = np.linalg.norm(batch.instance(i, "A")) * np.linalg.norm(batch.instance(i, "B"))
        num = np.linalg.norm(ct - cr)
        errs.append(num / den if den > 0 else num)
    return np.array(errs)


def run_fixed(batch, prec=None, C=None):
    """batched_gemm_fixed on a fixed-shape batch; returns the device C tensor."""
    m, n, k, count = batch.fixed_shape()
    A, B = dev(batch.A), dev(batch.B)
    Cd = dev(batch.C if C is None else C)
    lda, ldb, ldc = max(m, 1), max(k, 1), max(m, 1)
    bg.batched_gemm_fixed(batch.dtype, m, n, k, batch.alpha, A, lda, m * k, B, ldb, k * n,
                          batch.beta, Cd, ldc, m * n, count, prec)
    return Cd


def run_grouped(batch, prec=None, flags=0, C=None, plan=None, cache_path=None):
    """batched_gemm_plan + batched_gemm_grouped; returns (device C, plan)."""
    if plan is None:
        plan = bg.batched_gemm_plan(batch.dtype, batch.table, prec, flags, cache_path)
    A, B = dev(batch.A), dev(batch.B)
    Cd = dev(batch.C if C is None else C)
    bg.batched_gemm_grouped(plan, A, B, Cd, batch.alpha, batch.beta)
    return Cd, plan


def errors(batch, C_test: np.ndarray, C_ref: np.ndarray) -> np.ndarray:
    return rel_err_instances(batch, C_test, C_ref)
