"""GB300-native batched small-GEMM library: Python binding of the C ABI in include/bgemm.h.

The library computes Eq. (1) of the paper (Sec. 2), C_i = alpha A_i B_i + beta C_i,
over thousands of independent instances in one launch, in FP64/complex128 or in
the split-BF16 tensor-core mode. This module only marshals arguments: every
step of the computation runs in the CUDA kernels of ``libbgemm.so``. There is
no CPU fallback: when the shared library is missing every call raises.

Entry points keep the C names: ``batched_gemm_fixed``, ``batched_gemm_plan``,
``batched_gemm_grouped``, ``chain_plan``, ``chain_step``, plus the measurement
calls ``rel_err`` and ``unitarity_drift`` and the checks ``split_planes``,
``check_device_errors``, ``test_bounded_wait`` and ``probe_fp64_peak``.
Tensors are torch CUDA tensors (float64 or complex128, contiguous storage in
the column-major convention of the C ABI); raw integer device pointers are
accepted as well. ``stream`` defaults to torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbgemm.so")

BG_R64, BG_C128 = 0, 1
BG_MODE_FP64, BG_MODE_SPLIT_BF16 = 0, 1
BG_PLAN_AUTOTUNE, BG_PLAN_USE_CACHE, BG_PLAN_CAPTURE_GRAPH, BG_PLAN_PROFILE = 1, 2, 4, 8
BG_PLAN_HERK = 16  # Hermitian rank-k updates C = alpha A A^H + beta C (lower triangle)
BG_PLAN_SPLIT_TILES = 32  # split mode: no small-instance kernel (every instance on the tile kernels)

STATUS = {0: "BG_OK", 1: "BG_ERR_INVALID_ARG", 2: "BG_ERR_UNSUPPORTED", 3: "BG_ERR_CUDA",
          4: "BG_ERR_NOMEM", 5: "BG_ERR_CAPTURE", 6: "BG_ERR_TIMEOUT"}

# Every symbol include/bgemm.h declares (the loader checks they are all exported).
EXPORTS = ("batched_gemm_fixed", "batched_gemm_fixed_static", "batched_gemm_plan", "batched_gemm_grouped", "chain_plan",
           "chain_step", "bg_plan_destroy", "bg_plan_get_info", "bg_plan_describe",
           "bg_plan_kernel_times", "bg_rel_err",
           "bg_unitarity_drift", "bg_split_planes", "bg_check_device_errors",
           "bg_test_bounded_wait", "bg_probe_fp64_peak", "bg_launch_count", "bg_status_string",
           "bg_last_error", "bg_version", "apply_local_gate", "bg_partition_lpt",
           "entropy_plan", "batched_entropy", "metropolis_select", "anneal_plan",
           "anneal_step")


class BgemmError(RuntimeError):
    """A library call returned a status other than BG_OK."""

    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Precision(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("slices", ctypes.c_int32),
                ("beta_bits", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Instance(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("m", "n", "k", "lda", "ldb", "ldc", "a_off",
                                               "b_off", "c_off")]


class PlanInfo(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64), ("work_items", ctypes.c_int64),
                ("launches_per_call", ctypes.c_int32), ("classes", ctypes.c_int32),
                ("workspace_bytes", ctypes.c_int64), ("slices", ctypes.c_int32),
                ("beta_bits", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    i32, i64, u32, vp, dbl = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p,
                              ctypes.c_double)
    P = ctypes.POINTER
    sig = {
        "batched_gemm_fixed": [i32, i64, i64, i64, vp, vp, i64, i64, vp, i64, i64, vp, vp, i64,
                               i64, i64, P(Precision), vp],
        "batched_gemm_fixed_static": [i32, i64, i64, i64, vp, vp, i64, i64, vp, i64, i64, vp, vp,
                                      i64, i64, i64, P(Precision), vp],
        "batched_gemm_plan": [P(vp), i32, i64, P(Instance), P(Precision), u32, ctypes.c_char_p,
                              vp],
        "batched_gemm_grouped": [vp, vp, vp, vp, vp, vp, vp],
        "chain_plan": [P(vp), i32, i32, P(i64), P(i64), i32, P(i64), P(i64), P(Precision), u32,
                       vp],
        "chain_step": [vp, vp, vp, vp, vp, i32, vp],
        "bg_plan_get_info": [vp, P(PlanInfo)],
        "bg_plan_describe": [vp, ctypes.c_char_p, ctypes.c_size_t, P(ctypes.c_size_t)],
        "bg_plan_kernel_times": [vp, i32, P(dbl), P(i64)],
        "bg_rel_err": [i32, i64, vp, vp, vp, vp, vp, vp, vp],
        "bg_unitarity_drift": [i32, i64, vp, vp, vp, vp, vp],
        "bg_split_planes": [i64, i64, vp, i64, i32, i32, i32, vp, vp, vp],
        "bg_check_device_errors": [vp],
        "bg_test_bounded_wait": [i64, vp],
        "bg_probe_fp64_peak": [i32, P(dbl), vp],
        "apply_local_gate": [i32, i64, i32, vp, vp, vp, i64, vp],
        "bg_partition_lpt": [i64, P(dbl), i32, P(i32), P(dbl)],
        "entropy_plan": [P(vp), i64, i32, i32, i64, P(Precision), u32, vp],
        "batched_entropy": [vp, vp, vp, vp, vp],
        "metropolis_select": [i64, dbl, i32, vp, vp, vp, vp, vp, i64, vp, i64, i64, vp],
        "anneal_plan": [P(vp), i64, i32, i32, i64, P(Precision), u32, vp],
        "anneal_step": [vp, vp, vp, vp, vp, vp, dbl, i32, vp, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.bg_plan_destroy.argtypes = [vp]
    lib.bg_plan_destroy.restype = None
    lib.bg_launch_count.argtypes = [i32]
    lib.bg_launch_count.restype = i64
    lib.bg_status_string.argtypes = [ctypes.c_int]
    lib.bg_status_string.restype = ctypes.c_char_p
    lib.bg_last_error.restype = ctypes.c_char_p
    lib.bg_version.restype = ctypes.c_char_p
    return lib


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libbgemm.so (built by ``paper_2203_09353_gb300.build``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(
                    f"libbgemm.so not found at {p}: build it with "
                    "`python -m paper_2203_09353_gb300.build` (there is no CPU fallback)")
            lib = ctypes.CDLL(p)
            missing = [s for s in EXPORTS if not hasattr(lib, s)]
            if missing:
                raise RuntimeError(f"libbgemm.so lacks symbols: {missing}")
            _lib = _bind(lib)
        return _lib


def _check(status: int) -> None:
    if status != 0:
        raise BgemmError(status, load_library().bg_last_error().decode(errors="replace"))


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_cuda") and not x.is_cuda:
            raise ValueError("the library takes CUDA device tensors")
        return x.data_ptr()
    raise TypeError(f"expected a torch CUDA tensor or an int pointer, got {type(x)}")


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def dtype_code(x) -> int:
    """BG_R64 / BG_C128 from 'r64'/'c128', a torch dtype, a numpy dtype or a tensor."""
    if isinstance(x, int):
        return x
    if isinstance(x, str):
        return {"r64": BG_R64, "c128": BG_C128}[x]
    name = str(getattr(x, "dtype", x))
    if "complex128" in name:
        return BG_C128
    if "float64" in name:
        return BG_R64
    raise ValueError(f"unsupported dtype {name}: FP64 or complex128 only")


def precision(mode: str = "fp64", slices: int = 0, beta_bits: int = 0) -> Precision:
    """Precision request: mode 'fp64' or 'split' (BF16 digit planes, `slices` per operand)."""
    m = {"fp64": BG_MODE_FP64, "split": BG_MODE_SPLIT_BF16}[mode]
    return Precision(m, int(slices), int(beta_bits), 0)


def _scalar(dt: int, v):
    c = complex(v)
    arr = (ctypes.c_double * 2)(c.real, c.imag)
    if dt == BG_R64 and c.imag != 0:
        raise ValueError("complex scalar for a real problem")
    return arr


def batched_gemm_fixed(dtype, m, n, k, alpha, A, lda, strideA, B, ldb, strideB, beta, C, ldc,
                       strideC, batch, prec: Precision | None = None, stream=None) -> None:
    """Eq. (1) over a fixed-size batch at constant element strides (C ABI batched_gemm_fixed)."""
    lib = load_library()
    dt = dtype_code(dtype)
    _check(lib.batched_gemm_fixed(dt, m, n, k, _scalar(dt, alpha), _ptr(A), lda, strideA, _ptr(B),
                                  ldb, strideB, _scalar(dt, beta), _ptr(C), ldc, strideC, batch,
                                  ctypes.byref(prec) if prec is not None else None,
                                  _stream(stream)))


def batched_gemm_fixed_static(dtype, m, n, k, alpha, A, lda, strideA, B, ldb, strideB, beta, C,
                              ldc, strideC, batch, prec: Precision, stream=None) -> None:
    """The split-mode fixed-size batch with its whole workspace in the library's static
    64 MiB device array: allocates no device memory, for callers that must not (C ABI
    batched_gemm_fixed_static). Calls that overlap in time on one device race on that
    array; calls queued on one stream are safe."""
    lib = load_library()
    dt = dtype_code(dtype)
    _check(lib.batched_gemm_fixed_static(dt, m, n, k, _scalar(dt, alpha), _ptr(A), lda, strideA,
                                         _ptr(B), ldb, strideB, _scalar(dt, beta), _ptr(C), ldc,
                                         strideC, batch,
                                         ctypes.byref(prec) if prec is not None else None,
                                         _stream(stream)))


def _instances(table) -> ctypes.Array:
    t = np.ascontiguousarray(np.asarray(table, dtype=np.int64).reshape(-1, 9))
    arr = (Instance * max(1, t.shape[0]))()
    if t.shape[0]:
        ctypes.memmove(arr, t.ctypes.data, t.nbytes)
    return arr, t.shape[0]


class Plan:
    """Owns a bg_plan (batched_gemm_plan or chain_plan); destroyed with the object."""

    def __init__(self, handle: int, dtype: int, kind: str):
        self.handle = handle
        self.dtype = dtype
        self.kind = kind

    def info(self) -> dict:
        inf = PlanInfo()
        _check(load_library().bg_plan_get_info(self.handle, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in PlanInfo._fields_}

    def describe(self) -> str:
        lib = load_library()
        need = ctypes.c_size_t(0)
        lib.bg_plan_describe(self.handle, None, 0, ctypes.byref(need))
        buf = ctypes.create_string_buffer(need.value)
        _check(lib.bg_plan_describe(self.handle, buf, need.value, None))
        return buf.value.decode()

    def kernel_times(self, reset: bool = False) -> tuple[list[float], int]:
        """Summed per-kernel ms and call count (plans made with BG_PLAN_PROFILE): slot 0
        the slicer (FP64 mode: the FP64 kernel), slot 1 the tile GEMM, slot 2 the
        small-instance kernel."""
        ms = (ctypes.c_double * 3)()
        calls = ctypes.c_int64(0)
        _check(load_library().bg_plan_kernel_times(self.handle, 1 if reset else 0, ms,
                                                   ctypes.byref(calls)))
        return [ms[0], ms[1], ms[2]], calls.value

    def close(self) -> None:
        if self.handle:
            load_library().bg_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batched_gemm_plan(dtype, table, prec: Precision | None = None, flags: int = 0,
                      cache_path: str | None = None, stream=None) -> Plan:
    """Schedule for a variable-size batch; ``table`` is int64 [count, 9] (bg_instance rows)."""
    lib = load_library()
    dt = dtype_code(dtype)
    arr, count = _instances(table)
    h = ctypes.c_void_p()
    _check(lib.batched_gemm_plan(ctypes.byref(h), dt, count, arr,
                                 ctypes.byref(prec) if prec is not None else None, flags,
                                 cache_path.encode() if cache_path else None, _stream(stream)))
    return Plan(h.value, dt, "grouped")


def batched_gemm_grouped(plan: Plan, A, B, C, alpha, beta, stream=None) -> None:
    """Runs every instance of ``plan`` on base pointers A, B, C (C ABI batched_gemm_grouped)."""
    lib = load_library()
    _check(lib.batched_gemm_grouped(plan.handle, _ptr(A), _ptr(B), _ptr(C),
                                    _scalar(plan.dtype, alpha), _scalar(plan.dtype, beta),
                                    _stream(stream)))


def chain_plan(dtype, walker_n, state_off, pool_n, pool_off, prec: Precision | None = None,
               flags: int = 0, stream=None) -> Plan:
    """Plan for chained products C_w <- U[idx[t][w]] C_w (C ABI chain_plan)."""
    lib = load_library()
    dt = dtype_code(dtype)
    wn = np.ascontiguousarray(walker_n, dtype=np.int64)
    wo = np.ascontiguousarray(state_off, dtype=np.int64)
    pn = np.ascontiguousarray(pool_n, dtype=np.int64)
    po = np.ascontiguousarray(pool_off, dtype=np.int64)
    P = ctypes.POINTER(ctypes.c_int64)
    h = ctypes.c_void_p()
    _check(lib.chain_plan(ctypes.byref(h), dt, wn.size, wn.ctypes.data_as(P),
                          wo.ctypes.data_as(P), pn.size, pn.ctypes.data_as(P),
                          po.ctypes.data_as(P), ctypes.byref(prec) if prec is not None else None,
                          flags, _stream(stream)))
    return Plan(h.value, dt, "chain")


def chain_step(plan: Plan, U_pool, U_index, C_ping, C_pong, steps: int, stream=None) -> None:
    """Runs ``steps`` chained steps; the result ends in C_ping if steps is even, else C_pong."""
    lib = load_library()
    _check(lib.chain_step(plan.handle, _ptr(U_pool), _ptr(U_index), _ptr(C_ping), _ptr(C_pong),
                          int(steps), _stream(stream)))


def entropy_plan(walkers: int, spins: int, split: int | None = None, stride: int | None = None,
                 prec: Precision | None = None, flags: int = 0, stream=None) -> Plan:
    """Plan for the entanglement entropy of ``walkers`` complex128 states of ``spins``
    spins, cut after the lower ``split`` spins (default floor(spins/2)) (C ABI entropy_plan)."""
    split = spins // 2 if split is None else int(split)
    stride = (1 << spins) if stride is None else int(stride)
    h = ctypes.c_void_p()
    _check(load_library().entropy_plan(ctypes.byref(h), int(walkers), int(spins), split, stride,
                                       ctypes.byref(prec) if prec is not None else None,
                                       int(flags), _stream(stream)))
    return Plan(h.value, BG_C128, "entropy")


def batched_entropy(plan: Plan, states, entropy, eigenvalues=None, stream=None) -> None:
    """Entropy of every walker's state into the float64 device tensor ``entropy``
    (optionally the ascending Gram eigenvalues into ``eigenvalues``) (C ABI batched_entropy)."""
    import torch
    tens = {"states": states, "entropy": entropy, "eigenvalues": eigenvalues}
    want = {"states": torch.complex128, "entropy": torch.float64, "eigenvalues": torch.float64}
    for name, x in tens.items():
        if isinstance(x, torch.Tensor):
            if x.dtype != want[name]:
                raise ValueError(f"batched_entropy: {name} must be {want[name]}, got {x.dtype}")
            if not x.is_contiguous():
                raise ValueError(f"batched_entropy: {name} must be contiguous")
    _check(load_library().batched_entropy(plan.handle, _ptr(states), _ptr(entropy),
                                          _ptr(eigenvalues), _stream(stream)))


def _require(name: str, x, dtype) -> None:
    import torch
    if isinstance(x, torch.Tensor):
        if x.dtype != dtype:
            raise ValueError(f"{name} must be {dtype}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")


def metropolis_select(temperature: float, direction: int, uniforms, e_new, e_cur, accepted,
                      proposals=None, states=None, amplitudes: int = 0,
                      proposal_stride: int | None = None, state_stride: int | None = None,
                      walkers: int | None = None, stream=None) -> None:
    """The Metropolis decision of Alg. 1 ("M.A") per walker; with ``amplitudes`` > 0
    the accepted proposals are copied over the states (C ABI metropolis_select)."""
    import torch
    for name, x, dt in (("uniforms", uniforms, torch.float64), ("e_new", e_new, torch.float64),
                        ("e_cur", e_cur, torch.float64), ("accepted", accepted, torch.int32),
                        ("proposals", proposals, torch.complex128),
                        ("states", states, torch.complex128)):
        _require(name, x, dt)
    if walkers is None:
        walkers = int(e_cur.numel())
    ps = amplitudes if proposal_stride is None else int(proposal_stride)
    ss = amplitudes if state_stride is None else int(state_stride)
    _check(load_library().metropolis_select(int(walkers), float(temperature), int(direction),
                                            _ptr(uniforms), _ptr(e_new), _ptr(e_cur),
                                            _ptr(accepted), _ptr(proposals), ps, _ptr(states), ss,
                                            int(amplitudes), _stream(stream)))


def anneal_plan(walkers: int, spins: int, split: int | None = None, stride: int | None = None,
                prec: Precision | None = None, flags: int = 0, stream=None) -> Plan:
    """Plan for whole annealing steps of Alg. 1 (C ABI anneal_plan)."""
    split = spins // 2 if split is None else int(split)
    stride = (1 << spins) if stride is None else int(stride)
    h = ctypes.c_void_p()
    _check(load_library().anneal_plan(ctypes.byref(h), int(walkers), int(spins), split, stride,
                                      ctypes.byref(prec) if prec is not None else None,
                                      int(flags), _stream(stream)))
    return Plan(h.value, BG_C128, "anneal")


def anneal_step(plan: Plan, states, energy, sites, gates, uniforms, temperature: float,
                direction: int, accepted, stream=None) -> None:
    """One step of Alg. 1 for every walker: local gate, entropy, Metropolis (C ABI anneal_step)."""
    import torch
    for name, x, dt in (("states", states, torch.complex128), ("energy", energy, torch.float64),
                        ("sites", sites, torch.int32), ("gates", gates, torch.complex128),
                        ("uniforms", uniforms, torch.float64),
                        ("accepted", accepted, torch.int32)):
        _require(name, x, dt)
    _check(load_library().anneal_step(plan.handle, _ptr(states), _ptr(energy), _ptr(sites),
                                      _ptr(gates), _ptr(uniforms), float(temperature),
                                      int(direction), _ptr(accepted), _stream(stream)))


def rel_err(dtype, d_table, A, B, C_test, C_ref, out, count: int, stream=None) -> None:
    """Per-instance ||C_test - C_ref||_F / (||A||_F ||B||_F) into the device tensor ``out``."""
    _check(load_library().bg_rel_err(dtype_code(dtype), count, _ptr(d_table), _ptr(A), _ptr(B),
                                     _ptr(C_test), _ptr(C_ref), _ptr(out), _stream(stream)))


def unitarity_drift(dtype, d_n, d_off, C, out, count: int, stream=None) -> None:
    """||C_w^H C_w - I||_F per square matrix into the device tensor ``out``."""
    _check(load_library().bg_unitarity_drift(dtype_code(dtype), count, _ptr(d_n), _ptr(d_off),
                                             _ptr(C), _ptr(out), _stream(stream)))


def _check_gate_args(states, spins: int, sites, gates, walkers: int, stride: int) -> None:
    """Argument checks of apply_local_gate for torch tensors (raw integer pointers
    are passed through unchecked): element types, contiguity, sizes against the
    walker count and stride, then the device. Raises ValueError before any launch."""
    import torch
    tens = {"states": states, "sites": sites, "gates": gates}
    if not all(isinstance(x, torch.Tensor) for x in tens.values()):
        return
    want = {"states": torch.complex128, "sites": torch.int32, "gates": torch.complex128}
    for name, x in tens.items():
        if x.dtype != want[name]:
            raise ValueError(f"apply_local_gate: {name} must be {want[name]}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError(f"apply_local_gate: {name} must be contiguous")
    if walkers < 0 or walkers > sites.numel():
        raise ValueError(f"apply_local_gate: {walkers} walkers but {sites.numel()} sites")
    if gates.numel() < 16 * walkers:
        raise ValueError(f"apply_local_gate: gates holds {gates.numel()} entries, "
                         f"{16 * walkers} needed (16 per walker)")
    if not 2 <= spins <= 40:
        raise ValueError(f"apply_local_gate: spins = {spins} outside 2..40")
    if stride < (1 << spins):
        raise ValueError(f"apply_local_gate: stride {stride} below 2^spins = {1 << spins}")
    need = (walkers - 1) * stride + (1 << spins) if walkers > 0 else 0
    if states.numel() < need:
        raise ValueError(f"apply_local_gate: states holds {states.numel()} amplitudes, "
                         f"{need} needed")
    if walkers > 0:
        cur = torch.cuda.current_device() if torch.cuda.is_available() else None
        for name, x in tens.items():
            if not x.is_cuda or x.device.index != cur:
                raise ValueError(f"apply_local_gate: {name} must be on the current CUDA device")


def apply_local_gate(states, spins: int, sites, gates, walkers: int | None = None,
                     stride: int | None = None, stream=None) -> None:
    """The local two-spin gate (Alg. 1, "Apply Local Gate") on device state vectors, in place.

    ``states``: complex128 device tensor, walker w's 2^spins amplitudes at
    element w * stride (default stride 2^spins); ``sites``: int32 device tensor
    [walkers], the lower spin j of each pair; ``gates``: complex128 device
    tensor of 16 entries per walker, U_w column-major (U[a, c] at a + 4 c) for
    the local index a = b_j + 2 b_{j+1}. A bad site is reported through the
    device error word (check_device_errors)."""
    stride = (1 << spins) if stride is None else int(stride)
    if walkers is None:
        walkers = int(sites.numel())
    _check_gate_args(states, int(spins), sites, gates, int(walkers), stride)
    _check(load_library().apply_local_gate(dtype_code("c128"), int(walkers), int(spins),
                                           _ptr(sites), _ptr(gates), _ptr(states), stride,
                                           _stream(stream)))


def partition_lpt(costs, parts: int) -> tuple[np.ndarray, np.ndarray]:
    """Longest-processing-time-first split of independent items over ``parts``
    processes (C ABI bg_partition_lpt): returns (part of each item, load per part)."""
    c = np.ascontiguousarray(costs, dtype=np.float64).reshape(-1)
    part = np.zeros(c.size, dtype=np.int32)
    load = np.zeros(max(1, int(parts)), dtype=np.float64)
    P = ctypes.POINTER
    _check(load_library().bg_partition_lpt(c.size, c.ctypes.data_as(P(ctypes.c_double)),
                                           int(parts), part.ctypes.data_as(P(ctypes.c_int32)),
                                           load.ctypes.data_as(P(ctypes.c_double))))
    return part, load[:int(parts)]


def instance_flops(table, dtype) -> np.ndarray:
    """Algorithmic flops per instance of a bg_instance table: 2 m n k (8 m n k complex)."""
    t = np.asarray(table, dtype=np.int64).reshape(-1, 9).astype(np.float64)
    per = 8.0 if dtype_code(dtype) == BG_C128 else 2.0
    return per * t[:, 0] * t[:, 1] * t[:, 2]


def split_planes(m, k, X, ldx, axis, slices, beta_bits, exps, digits, stream=None) -> None:
    """Exponents and BF16 digit planes of one real matrix (the split mode's operand cut)."""
    _check(load_library().bg_split_planes(m, k, _ptr(X), ldx, axis, slices, beta_bits,
                                          _ptr(exps), _ptr(digits), _stream(stream)))


def check_device_errors(stream=None) -> None:
    """Synchronises and raises if a bounded device-side wait gave up since the last check."""
    _check(load_library().bg_check_device_errors(_stream(stream)))


def test_bounded_wait(spin_limit: int, stream=None) -> None:
    _check(load_library().bg_test_bounded_wait(int(spin_limit), _stream(stream)))


def probe_fp64_peak(mma: bool = False, stream=None) -> float:
    """Measured FP64 TFLOP/s of this GPU (DFMA, or FP64 mma.sync when ``mma``)."""
    v = ctypes.c_double(0)
    _check(load_library().bg_probe_fp64_peak(1 if mma else 0, ctypes.byref(v), _stream(stream)))
    return v.value


def launch_count(reset: bool = False) -> int:
    """Kernels this library launched on the calling thread (since the last reset)."""
    return int(load_library().bg_launch_count(1 if reset else 0))


def version() -> str:
    return load_library().bg_version().decode()
