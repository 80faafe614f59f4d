#!/usr/bin/env python3
"""Benchmark of the batched GEMM hot path (Eq. 1, Sec. 2) on one GB300 per rank.

One step = one grouped call of the library on the whole synthetic batch (one
persistent launch for FP64; slicer + tensor-core GEMM for split-BF16). The
default workload is the log-uniform size mix: 20000 square FP64 instances
with n drawn from {16, 32, 64, 128, 256, 512} (weights .3/.25/.2/.15/.07/.03),
entries of magnitude 10^U(-4,4) with random signs, alpha = 1, beta = 0.5,
seed 3. Every mode runs on the same batch: plain FP64 and split-BF16 with 3,
6 and 9 slices. The headline value is the 9-slice mode (whose error matches
the FP64 path's), in FP64-equivalent TFLOP/s (2 m n k per instance); the FP64
mode and the others are reported beside it with their errors against the CPU
oracle on a sample.

Prints ONE JSON line (rank 0). ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "batched GEMM TFLOP/s & roofline %: FP64 vs split-BF16 at same error"
# the seeded synthetic workloads: a fixed n = 32 real batch, a complex n = 64
# Hermitian x unitary batch, and the 20000-instance size mixes (U[-1,1] and
# log-uniform magnitudes)
WORKLOADS = ("fixed-n32", "complex-n64", "mix-uniform", "mix-loguniform")
UNIT = "TFLOP/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch from one
# single-metric ncu capture of the headline batch itself (20000-instance
# log-uniform size mix, seed 3, 9 slices; profiles/), divided by that batch's
# Eq. (1) bytes (10314440704): a launch's traffic is this ratio times its own
# batch's Eq. (1) bytes (exactly the captured figure for the headline batch).
# Valid only while the split kernel sources hash to NCU_SOURCES_SHA; otherwise
# the traffic is reported as null.
NCU_EQ1_BYTES = 10314440704.0
NCU_TRAFFIC_PER_BYTE = {"split9": {"gemm": (13589957376 + 2374727168) / NCU_EQ1_BYTES,
                                   "slicer": (7149745920 + 10727013376) / NCU_EQ1_BYTES,
                                   "small": (560837632 + 155502080) / NCU_EQ1_BYTES}}
NCU_SOURCES = ("split.cu", "split_common.cuh", "split_gemm.cuh", "split_gemm_r64.cu",
               "split_small.cu")
NCU_SOURCES_SHA = "39867e7f115557e5"


def split_sources_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in NCU_SOURCES:
        with open(os.path.join(ROOT, "paper_2203_09353_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse_args():
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=WORKLOADS, default="mix-loguniform")
    p.add_argument("--count", type=int, default=20000, help="instances (the size mixes)")
    p.add_argument("--mode", default="split9", help="headline mode: fp64 or splitS")
    p.add_argument("--modes", default="fp64,split3,split6,split9")
    p.add_argument("--fp64-steps", type=int, default=0,
                   help="timed steps of the FP64 mode (0: as --steps)")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--e2e-chunks", type=int, default=4, help="instance ranges of the e2e pipeline")
    p.add_argument("--no-library-baseline", action="store_true",
                   help="skip timing one cuBLAS DGEMM per instance (the paper's design)")
    p.add_argument("--no-gate", action="store_true",
                   help="skip the local two-spin gate line")
    p.add_argument("--no-herk", action="store_true",
                   help="skip the Hermitian-update line (rho = Psi Psi^H, Sec. 3 shapes)")
    p.add_argument("--no-chain", action="store_true",
                   help="skip the chained-product line (1024 walkers, Alg. 1 step loop)")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the fixed-size and uniform-mix workloads (configs 1-3)")
    p.add_argument("--no-entropy", action="store_true",
                   help="skip the entanglement-entropy line (128 states of 17 spins)")
    p.add_argument("--no-anneal", action="store_true",
                   help="skip the whole-annealing-step line (gate, entropy, Metropolis)")
    p.add_argument("--no-ablation", action="store_true",
                   help="skip the tasked-vs-batched ablation (N streams of plans vs one launch)")
    p.add_argument("--no-cpu", action="store_true")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


def lpt_shard(seed: int, count: int, world: int, rank: int, values: str):
    """Rank ``rank``'s share of ONE size-mix batch of ``world * count`` instances.
    The sizes of the whole batch are drawn once from ``seed`` (every rank draws
    the same ones); the instances are split by the library's longest-first
    partition of their flops (bg_partition_lpt), which every rank computes
    identically; the values of this rank's instances are drawn from
    seed + 1000 rank. Returns (batch, ids of the whole batch this rank holds)."""
    import paper_2203_09353_gb300 as bg
    from paper_2203_09353_gb300 import synth
    ns = synth.draw_sizes(np.random.default_rng(seed), world * count)
    part, _ = bg.partition_lpt(2.0 * ns.astype(np.float64) ** 3, world)
    ids = np.flatnonzero(part == rank)
    b = synth.batch_of_sizes(np.random.default_rng(seed + 1000 * rank), ns[ids], values, 1.0, 0.5,
                             f"size_mix_{values}_{world * count}_part{rank}of{world}")
    return b, ids


def make_batch(workload: str, count: int, rank: int, world: int = 1):
    from paper_2203_09353_gb300 import synth
    if workload.startswith("mix-") and world > 1:
        values = workload[4:]
        seed = 2 if values == "uniform" else 3
        b, ids = lpt_shard(seed, count, world, rank, values)
        return b, (f"part {rank} of {world} (longest-first flop split) of one batch of "
                   f"{world * count} real FP64 instances n in {{16..512}} (w .3/.25/.2/.15/.07/.03), "
                   f"{'U[-1,1]' if values == 'uniform' else '|x| = 10^U(-4,4) random sign'}, "
                   f"alpha=1, beta=0.5, sizes seed {seed}, values seed {seed + 1000 * rank}; "
                   f"{b.count} instances here")
    if workload == "fixed-n32":
        return synth.fixed_real_n32(), "64 real FP64 instances n=32, U[-1,1], seed 0, C=AB"
    if workload == "complex-n64":
        return synth.hermitian_unitary_c128(), ("4096 complex128 instances n=64, A Hermitian, "
                                 "B Haar unitary, seed 1, C=AB")
    if workload == "mix-uniform":
        seed = 2 + 1000 * rank
        b = synth.mixed_batch(seed, count, "uniform", 1.0, 0.5, name=f"size_mix_uniform_{count}")
        return b, (f"{count} real FP64 instances n in {{16..512}} "
                   f"(w .3/.25/.2/.15/.07/.03), U[-1,1], alpha=1, beta=0.5, seed {seed}")
    seed = 3 + 1000 * rank
    b = synth.mixed_batch(seed, count, "loguniform", 1.0, 0.5, name=f"size_mix_loguniform_{count}")
    return b, (f"{count} real FP64 instances n in {{16..512}} "
               f"(w .3/.25/.2/.15/.07/.03), |x| = 10^U(-4,4) random sign, alpha=1, beta=0.5, "
               f"seed {seed}")


def sample_ids(batch, frac_flops: float) -> np.ndarray:
    """Every j-th instance (table order is random, so all size classes appear)."""
    t = batch.table
    fl = 2.0 * t[:, 0].astype(np.float64) * t[:, 1] * t[:, 2]
    target = frac_flops * fl.sum()
    step = max(1, int(round(fl.sum() / max(target, 1.0))))
    ids = np.arange(0, batch.count, step)
    return ids


def oracle_on(batch, ids):
    """Runs the CPU oracle on the chosen instances; returns ({id: C}, seconds, flops, threads)."""
    import oracle
    from paper_2203_09353_gb300 import synth
    shapes = [tuple(int(x) for x in batch.table[i, :3]) for i in ids]
    table, la, lb, lc = synth.pack_table(shapes)
    A = np.zeros(la, dtype=batch.np_dtype)
    B = np.zeros(lb, dtype=batch.np_dtype)
    C = np.zeros(lc, dtype=batch.np_dtype)
    for j, i in enumerate(ids):
        m, n, k = shapes[j]
        A[table[j, 6]:table[j, 6] + m * k] = np.ravel(batch.instance(i, "A"), order="F")
        B[table[j, 7]:table[j, 7] + k * n] = np.ravel(batch.instance(i, "B"), order="F")
        C[table[j, 8]:table[j, 8] + m * n] = np.ravel(batch.instance(i, "C"), order="F")
    lib = oracle.load()
    threads = oracle.max_threads(lib)
    t0 = time.perf_counter()
    oracle.gemm_grouped(table, batch.alpha, A, B, batch.beta, C, lib=lib)
    dt = time.perf_counter() - t0
    out = {}
    for j, i in enumerate(ids):
        m, n, k = shapes[j]
        out[int(i)] = C[table[j, 8]:table[j, 8] + m * n].reshape((n, m)).T.copy()
    flops = float(np.sum([(8.0 if batch.dtype == "c128" else 2.0) * m * n * k
                          for (m, n, k) in shapes]))
    return out, dt, flops, threads


def calibrated_sample(batch, seconds: float):
    """Oracle sample sized to take about `seconds` on this host's cores."""
    ids = sample_ids(batch, 0.05)
    _, dt, fl, _ = oracle_on(batch, ids)
    rate = fl / max(dt, 1e-6)
    frac = min(1.0, seconds * rate / (2.0 * batch.table[:, 0].astype(np.float64)
                                       @ (batch.table[:, 1] * batch.table[:, 2].astype(np.float64))
                                       * (4.0 if batch.dtype == "c128" else 1.0)))
    return sample_ids(batch, max(frac, 0.0005))


def sample_errors(batch, C_host: np.ndarray, ref: dict) -> float:
    worst = 0.0
    for i, cr in ref.items():
        m, n, k, lda, ldb, ldc, ao, bo, co = (int(x) for x in batch.table[i])
        ct = C_host[co:co + ldc * n].reshape((n, ldc)).T[:m, :]
        den = np.linalg.norm(batch.instance(i, "A")) * np.linalg.norm(batch.instance(i, "B"))
        e = np.linalg.norm(ct - cr) / den if den > 0 else np.linalg.norm(ct - cr)
        worst = max(worst, float(e))
    return worst


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.path = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            sel = ["-i", f"GPU-{uuid}" if not uuid.startswith("GPU-") else uuid]
        except Exception:
            sel = []
        self.sel = sel

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", *self.sel, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = np.array([num(r[0]) for r in rows])
        mx = np.nanmax([num(r[1]) for r in rows])
        power = np.array([num(r[2]) for r in rows])
        loaded = sm[power >= np.nanmedian(power)] if len(sm) > 2 else sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4)
                          if r[4 + j].lower().startswith("active")})
        return {"sm_mhz": float(np.nanmedian(loaded)), "sm_max_mhz": float(mx),
                "reasons": reasons, "samples": len(rows),
                "power_w_max": float(np.nanmax(power))}


_T0 = time.time()


def log(msg: str) -> None:
    sys.stderr.write(f"[bench {time.time() - _T0:7.1f}s] {msg}\n")
    sys.stderr.flush()


def bind_near_gpu(local: int) -> str:
    """Pins this process to the CPU cores next to its GPU (the PCI device's
    local_cpulist), so that the pinned host buffers of the end-to-end step are
    allocated on the memory node wired to that GPU. Returns what was done."""
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout.split()
        if not out:
            return "unbound (no bus id)"
        bus = out[min(local, len(out) - 1)].strip().lower()
        dom, rest = bus.split(":", 1)
        path = f"/sys/bus/pci/devices/{int(dom, 16):04x}:{rest}/local_cpulist"
        cpus = set()
        with open(path) as fh:
            for part in fh.read().strip().split(","):
                lo, _, hi = part.partition("-")
                cpus.update(range(int(lo), int(hi or lo) + 1))
        cpus &= os.sched_getaffinity(0)
        if not cpus:
            return "unbound (no local cores available)"
        os.sched_setaffinity(0, cpus)
        return f"bound to {len(cpus)} cores local to GPU {bus}"
    except Exception as e:  # the binding is an optimisation only
        return f"unbound ({type(e).__name__})"


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v: float) -> float:
    if pg is None:
        return v
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, v: float) -> float:
    if pg is None:
        return v
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def cublas_per_instance(batch, A, B, C0, steps: int, warmup: int, branches: int = 8):
    """The paper's design on this GPU: one library GEMM per instance (its MPI
    ranks each multiply one matrix through cuBLAS), here cuBLAS DGEMM through
    torch.addmm on column-major views, C^T = beta C^T + alpha B^T A^T, issued
    round-robin on `branches` concurrent streams and replayed as one CUDA
    graph so that host launch overhead is not counted. Real FP64 batches only.
    Returns (ms per step, the resulting C)."""
    import torch
    t = batch.table
    C = C0.clone()
    views = []
    for i in range(batch.count):
        m, n, k, lda, ldb, ldc, ao, bo, co = (int(x) for x in t[i])
        if m == 0 or n == 0:
            continue
        At = A[ao:ao + lda * k].view(k, lda)[:, :m]     # A^T, k x m
        Bt = B[bo:bo + ldb * n].view(n, ldb)[:, :k]     # B^T, n x k
        Ct = C[co:co + ldc * n].view(n, ldc)[:, :m]     # C^T, n x m
        views.append((At, Bt, Ct))
    streams = [torch.cuda.Stream() for _ in range(branches)]

    def issue():
        # fork from and join into the stream current at call time (the capture
        # stream while the graph is recorded)
        cur = torch.cuda.current_stream()
        for sb in streams:
            sb.wait_stream(cur)
        for j, (At, Bt, Ct) in enumerate(views):
            with torch.cuda.stream(streams[j % branches]):
                torch.addmm(Ct, Bt, At, beta=float(batch.beta), alpha=float(batch.alpha), out=Ct)
        for sb in streams:
            cur.wait_stream(sb)

    issue()  # warm cuBLAS up outside the capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        issue()
    for _ in range(max(1, warmup)):
        graph.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    C.copy_(C0)  # every replay updated C in place: one more from the start for the check
    graph.replay()
    torch.cuda.synchronize()
    return ms, C


def herk_line(bg, steps: int, warmup: int, S: int = 17, count: int = 128):
    """rho = Psi Psi^H of Sec. 3 for `count` complex states of S spins: Psi is
    M x K with M = 2^(S - floor(S/2)), K = 2^floor(S/2); lower triangle through
    plans with BG_PLAN_HERK, FP64 and 9 slices. Flops: 4 K M (M + 1) per
    instance (the Hermitian half of 8 M M K)."""
    import torch
    from paper_2203_09353_gb300 import synth
    M, K = 2 ** (S - S // 2), 2 ** (S // 2)
    rng = np.random.default_rng(17)
    table, la, lb, lc = synth.pack_table([(M, M, K)] * count)
    A = torch.from_numpy(synth.complex_gaussian(rng, la)).cuda()
    C0 = torch.zeros(lc, dtype=torch.complex128, device="cuda")
    flops = count * 4.0 * K * M * (M + 1)
    out, res = {}, {"workload": f"{count} complex Psi of {M} x {K} (S = {S}), C = Psi Psi^H",
                    "gflop": flops / 1e9}
    for mode in ("fp64", "split9"):
        prec = None if mode == "fp64" else bg.precision("split", 9)
        plan = bg.batched_gemm_plan("c128", table, prec, bg.BG_PLAN_HERK)
        C = C0.clone()
        for _ in range(max(1, warmup)):
            bg.batched_gemm_grouped(plan, A, None, C, 1.0, 0.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            bg.batched_gemm_grouped(plan, A, None, C, 1.0, 0.0)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[mode] = {"ms_per_step": ms, "value": flops / (ms * 1e-3) / 1e12, "unit": UNIT}
        out[mode] = C
        plan.close()
    # lower triangle of the 9-slice result against the FP64 one (normwise, max over instances)
    worst = 0.0
    for i in range(count):
        co = int(table[i, 8])
        # row-major views of column-major matrices: the lower triangle is the views' upper one
        a = out["fp64"][co:co + M * M].view(M, M)
        b = out["split9"][co:co + M * M].view(M, M)
        d = torch.triu(a - b).abs().pow(2).sum().sqrt() / torch.triu(a).abs().pow(2).sum().sqrt()
        worst = max(worst, float(d))
    res["split9_vs_fp64_lower_rel"] = worst
    return res


def gate_line(bg, fp64_peak, hbm_peak, hbm_src, steps: int = 20, S: int = 17,
              walkers: int = 1024):
    """The local two-spin gate of Alg. 1 ("Apply Local Gate") on `walkers` complex
    state vectors of S spins (2 GB for 1024 walkers of 17 spins, well above L2):
    every step applies a fresh Haar gate per walker on a random neighbouring pair.
    Algorithmic work per amplitude: 4 complex multiply-adds (32 FP64 flops) and
    32 bytes (read and write once). The norm of every state is checked after the
    last step (the gates are unitary)."""
    import torch
    rng = np.random.default_rng(23)
    dim = 1 << S
    gen = torch.Generator(device="cuda").manual_seed(23)
    psi = torch.randn(walkers * dim, dtype=torch.complex128, device="cuda", generator=gen)
    norm0 = psi.view(walkers, dim).abs().pow(2).sum(dim=1).sqrt()
    z = rng.standard_normal((steps, walkers, 4, 4)) + 1j * rng.standard_normal((steps, walkers, 4, 4))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    haar = q * (d / np.abs(d))[..., None, :]
    # column-major 4 x 4 per walker
    gates = torch.from_numpy(np.ascontiguousarray(haar.transpose(0, 1, 3, 2))).cuda()
    sites = torch.from_numpy(rng.integers(0, S - 1, (steps, walkers)).astype(np.int32)).cuda()
    for t in range(min(3, steps)):
        bg.apply_local_gate(psi, S, sites[t], gates[t])
    torch.cuda.synchronize()
    bg.launch_count(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for t in range(steps):
        bg.apply_local_gate(psi, S, sites[t], gates[t])
    e1.record()
    torch.cuda.synchronize()
    launches = bg.launch_count(reset=True)
    bg.check_device_errors()
    ms = e0.elapsed_time(e1) / steps
    amps = float(walkers) * dim
    tflops = 32.0 * amps / (ms * 1e-3) / 1e12
    gbs = 32.0 * amps / (ms * 1e-3) / 1e9
    drift = float(((psi.view(walkers, dim).abs().pow(2).sum(dim=1).sqrt() - norm0).abs() / norm0).max())
    return {"workload": f"{walkers} complex states of {S} spins, a Haar two-spin gate per walker "
                        f"and step on a random neighbouring pair",
            "steps": steps, "ms_per_step": ms, "value": amps / (ms * 1e-3) / 1e9,
            "unit": "G amplitudes/s", "fp64_tflops": tflops, "hbm_gbs": gbs,
            "roofline": {"bound": "alu", "achieved": tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": tflops / fp64_peak if fp64_peak else None,
                         "peak_source": "DFMA probe measured live (bg_probe_fp64_peak)"},
            "hbm_frac_of_copy_peak": gbs / hbm_peak,
            "hbm_peak": {"value": hbm_peak, "unit": "GB/s", "source": hbm_src},
            "gpu_launches": launches,
            "max_norm_drift": drift}


def chain_line(bg, fp64_steps: int = 10, split_steps: int = 200):
    """The annealing-shaped chain: 960 complex walkers of n = 256 and 64 of
    n = 1024, each multiplied by a pool unitary per step (Alg. 1 step loop),
    through chain_step with the step loop captured in a CUDA graph. 9 slices
    run all 200 steps; FP64, 50 times slower, a bounded number. The unitarity
    drift ||C^H C - I||_F of every walker is reported after the last step."""
    import torch
    from paper_2203_09353_gb300 import synth
    ch = synth.annealing_chain()
    pool, pn, po, states, wo, gidx = synth.chain_layout(ch)
    dpool = torch.from_numpy(pool).cuda()
    didx = torch.from_numpy(gidx).cuda()
    dn = torch.from_numpy(ch.n_walker.astype(np.int64)).cuda()
    do = torch.from_numpy(wo).cuda()
    step_flops = float(np.sum(8.0 * ch.n_walker.astype(np.float64) ** 3))
    res = {"workload": f"{ch.walkers} complex walkers (960 x n=256, 64 x n=1024), pool of "
                       f"{len(pn)} Haar unitaries, C <- U_t C", "gflop_per_step": step_flops / 1e9}
    for mode, steps in (("fp64", fp64_steps), ("split9", split_steps)):
        prec = None if mode == "fp64" else bg.precision("split", 9)
        plan = bg.chain_plan("c128", ch.n_walker, wo, pn, po, prec, bg.BG_PLAN_CAPTURE_GRAPH)
        ping = torch.from_numpy(states).cuda()
        pong = torch.empty_like(ping)
        # warm-up with the timed arguments: captures the step loop's graph
        bg.chain_step(plan, dpool, didx[:steps], ping, pong, steps)
        ping.copy_(torch.from_numpy(states))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bg.chain_step(plan, dpool, didx[:steps], ping, pong, steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out = ping if steps % 2 == 0 else pong
        drift = torch.zeros(ch.walkers, dtype=torch.float64, device="cuda")
        bg.unitarity_drift("c128", dn, do, out, drift, ch.walkers)
        res[mode] = {"steps": steps, "ms": ms, "ms_per_step": ms / steps,
                     "value": step_flops * steps / (ms * 1e-3) / 1e12, "unit": UNIT,
                     "max_unitarity_drift": float(drift.max())}
        if steps < split_steps:
            # a bounded number of the 200 steps, timed; the whole run extrapolated linearly
            res[mode]["extrapolated"] = {"steps": split_steps, "ms": ms / steps * split_steps,
                                         "from_timed_steps": steps}
        plan.close()
    return res


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _time_calls(fn, steps: int, warmup: int, flush=None) -> float:
    """Mean device ms of fn() over `steps` calls after `warmup`, CUDA events on the
    current stream. With `flush`, each call is timed alone and flush() (a write
    larger than L2) runs between calls outside the timed pairs."""
    import torch
    for _ in range(max(1, warmup)):
        fn()
    torch.cuda.synchronize()
    if flush is None:
        e0, e1 = _events()
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps
    total = 0.0
    for _ in range(steps):
        flush()
        e0, e1 = _events()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    return total / steps


def configs_line(bg, pk, fp64_peak, steps: int, warmup: int, cpu_seconds: float, cache: str):
    """The three workloads besides the log-uniform headline mix: 64 real n = 32
    instances, 4096 complex n = 64 Hermitian x Haar-unitary instances, and the
    20000-instance U[-1,1] size mix (alpha = 1, beta = 0.5) -- the last as one
    autotuned persistent launch replayed from a captured CUDA graph, with a
    per-size-class FP64 rate. Each in FP64 and with 9 slices; the roofline of
    the FP64 path is min(FP64 peak, intensity x copy bandwidth)."""
    import torch
    from paper_2203_09353_gb300 import synth
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    for name, make in (("fixed-n32", synth.fixed_real_n32), ("complex-n64",
                       synth.hermitian_unitary_c128), ("mix-uniform", synth.size_mix_uniform)):
        b = make()
        flops, nbytes = b.flops(), b.bytes_moved()
        inten = flops / nbytes
        roof = min(fp64_peak, inten * pk["hbm_gbs"] / 1e3)
        A, B, C0 = (torch.from_numpy(x).cuda() for x in (b.A, b.B, b.C))
        dtab = torch.from_numpy(b.table).cuda()
        small = nbytes < 64e6  # inputs smaller than L2: flush between timed calls
        res = {"workload": b.name, "instances": b.count, "gflop": flops / 1e9,
               "algorithmic_gb": nbytes / 1e9, "intensity_flop_per_byte": inten,
               "l2": "flushed (256 MB write) between timed calls" if small else
                     "inputs larger than L2, no flush"}
        outs = {}
        for mode in ("fp64", "split9"):
            prec = None if mode == "fp64" else bg.precision("split", 9)
            flags = bg.BG_PLAN_CAPTURE_GRAPH | (bg.BG_PLAN_AUTOTUNE | bg.BG_PLAN_USE_CACHE
                                                if mode == "fp64" else 0)
            plan = bg.batched_gemm_plan(b.dtype, b.table, prec, flags, cache)
            C = C0.clone()
            call = lambda: bg.batched_gemm_grouped(plan, A, B, C, b.alpha, b.beta)
            ms = _time_calls(call, steps, warmup, (lambda: flush_buf.zero_()) if small else None)
            C.copy_(C0)
            call()
            torch.cuda.synchronize()
            outs[mode] = C
            tf = flops / (ms * 1e-3) / 1e12
            res[mode] = {"ms_per_call": ms, "value": tf, "unit": UNIT,
                         "frac_of_fp64_roofline": tf / roof,
                         "graph": True, "autotuned": mode == "fp64"}
            if mode == "fp64":
                res["fp64_roofline"] = {"bound": "alu" if fp64_peak <= inten * pk["hbm_gbs"] / 1e3
                                        else "hbm", "peak": roof, "unit": "TFLOP/s",
                                        "fp64_peak": fp64_peak, "hbm_gbs": pk["hbm_gbs"]}
                res["plan"] = json.loads(plan.describe())
            plan.close()
        errbuf = torch.zeros(b.count, dtype=torch.float64, device="cuda")
        bg.rel_err(b.dtype, dtab, A, B, outs["split9"], outs["fp64"], errbuf, b.count)
        res["split9"]["max_err_vs_fp64_path_all"] = float(errbuf.max())
        ids = calibrated_sample(b, cpu_seconds) if b.count > 64 else np.arange(b.count)
        ref, dt, fl, threads = oracle_on(b, ids)
        for mode in ("fp64", "split9"):
            res[mode]["max_err_vs_oracle"] = sample_errors(b, outs[mode].cpu().numpy(), ref)
        res["oracle_sample"] = f"{len(ids)} of {b.count} instances, {threads} cores, {dt:.2f} s"
        if name == "mix-uniform":
            # FP64 rate per size class: one autotuned plan over the class's instances
            per = {}
            for n in synth.SIZE_MIX_SIZES:
                sel = np.flatnonzero(b.table[:, 0] == n)
                if sel.size == 0:
                    continue
                sub = b.table[sel]
                plan = bg.batched_gemm_plan("r64", sub, None, bg.BG_PLAN_AUTOTUNE |
                                            bg.BG_PLAN_USE_CACHE | bg.BG_PLAN_CAPTURE_GRAPH, cache)
                C = C0.clone()
                ms = _time_calls(lambda: bg.batched_gemm_grouped(plan, A, B, C, b.alpha, b.beta),
                                 steps, warmup)
                fl = float(np.sum(2.0 * sub[:, 0] * sub[:, 1] * sub[:, 2]))
                tf = fl / (ms * 1e-3) / 1e12
                per[str(n)] = {"instances": int(sel.size), "ms": ms, "value": tf,
                               "frac_of_fp64_peak": tf / fp64_peak,
                               "program": json.loads(plan.describe())["classes"][0]["program"]}
                plan.close()
            res["fp64_per_class"] = per
        out[name] = res
        del A, B, C0, outs
    return out


def entropy_line(bg, fp64_peak, steps: int = 5, warmup: int = 2, S: int = 17,
                 walkers: int = 128):
    """The entanglement entropy of Alg. 1 ("Calculate Entropy") for `walkers`
    random complex states of S spins (cut after floor(S/2) spins: K = 256,
    M = 512 at S = 17): the Gram matrices through the Hermitian update (FP64 or
    9 slices), then tridiagonalisation and bisection; with 9 slices the
    reduction is blocked, its trailing updates running as 9-slice GEMMs.
    Roofline of the eigenvalue step: the flops of the reduction, (16/3) K^3
    per walker (the LAPACK count of zhetrd), against the live DFMA probe."""
    import torch
    import oracle
    K = 1 << (S // 2)
    gen = torch.Generator(device="cuda").manual_seed(31)
    psi = torch.randn(walkers << S, dtype=torch.complex128, device="cuda", generator=gen)
    ent = torch.zeros(walkers, dtype=torch.float64, device="cuda")
    sample = list(range(0, walkers, max(1, walkers // 4)))[:4]
    host_psi = psi.view(walkers, 1 << S)[sample].cpu().numpy()
    t0 = time.perf_counter()
    want = np.array([oracle.entanglement_entropy(p, S) for p in host_psi])
    cpu_s = (time.perf_counter() - t0) / len(sample)
    res = {"workload": f"{walkers} complex states of {S} spins, cut after {S // 2} spins "
                       f"(Gram matrices {K} x {K} from {K} x {1 << (S - S // 2)} views)",
           "cpu_oracle_s_per_walker": cpu_s}
    tri_flops = walkers * 16.0 / 3.0 * K ** 3
    for mode in ("fp64", "split9"):
        prec = None if mode == "fp64" else bg.precision("split", 9)
        plan = bg.entropy_plan(walkers, S, prec=prec, flags=bg.BG_PLAN_PROFILE)
        for _ in range(warmup):
            bg.batched_entropy(plan, psi, ent)
        plan.kernel_times(reset=True)
        ms = _time_calls(lambda: bg.batched_entropy(plan, psi, ent), steps, 0)
        kt, calls = plan.kernel_times(reset=True)
        got = ent.cpu().numpy()[sample]
        eig_ms = kt[1] / max(calls, 1)
        ach = tri_flops / (eig_ms * 1e-3) / 1e12
        # 9 slices, K > 64: the blocked reduction, whose rank-32 trailing updates
        # (about half the flops) run on the tensor cores
        kernels = ("tridiag_kernel + bisect_kernel" if mode == "fp64" or K <= 64 else
                   "tri_mirror_kernel + (tri_panel_kernel + tri_pack_kernel + split "
                   "GEMM) per 16-column panel + tridiag_kernel (last 64) + bisect_kernel")
        res[mode] = {"ms_per_call": ms, "gram_ms": kt[0] / max(calls, 1), "eig_ms": eig_ms,
                     "value": walkers / (ms * 1e-3), "unit": "walkers/s",
                     "max_abs_err_vs_oracle": float(np.max(np.abs(got - want))),
                     "eig_roofline": {"kernels": kernels, "bound": "alu",
                                      "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                                      "frac": ach / fp64_peak,
                                      "flops": "(16/3) K^3 per walker (Householder reduction)"}}
        plan.close()
    return res


def anneal_line(bg, steps: int = 10, warmup: int = 2, S: int = 17, walkers: int = 128):
    """Whole annealing steps of Alg. 1 for `walkers` states of S spins: per step
    and walker a Haar gate on a random neighbouring pair, the proposal's
    entropy (Gram and trailing updates with 9 slices) and the Metropolis decision
    at a geometric temperature schedule T_t = 0.05 x 0.9^t, minimising the
    entropy. The CPU oracle's step is timed on two walkers for context."""
    import torch
    import oracle
    rng = np.random.default_rng(37)
    gen = torch.Generator(device="cuda").manual_seed(37)
    dim = 1 << S
    psi = torch.randn(walkers * dim, dtype=torch.complex128, device="cuda", generator=gen)
    psi /= psi.view(walkers, dim).abs().pow(2).sum(dim=1).sqrt().repeat_interleave(dim)
    prec = bg.precision("split", 9)
    eplan = bg.entropy_plan(walkers, S, prec=prec)
    energy = torch.zeros(walkers, dtype=torch.float64, device="cuda")
    bg.batched_entropy(eplan, psi, energy)
    e_start = float(energy.mean())
    total = warmup + steps
    z = rng.standard_normal((total, walkers, 4, 4)) + 1j * rng.standard_normal((total, walkers, 4, 4))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    haar = q * (d / np.abs(d))[..., None, :]
    gates = torch.from_numpy(np.ascontiguousarray(haar.transpose(0, 1, 3, 2))).cuda()
    sites_h = rng.integers(0, S - 1, (total, walkers)).astype(np.int32)
    sites = torch.from_numpy(sites_h).cuda()
    u_h = rng.random((total, walkers))
    u = torch.from_numpy(u_h).cuda()
    acc = torch.zeros(walkers, dtype=torch.int32, device="cuda")
    plan = bg.anneal_plan(walkers, S, prec=prec)
    temps = [0.05 * 0.9 ** t for t in range(total)]
    host0 = psi.view(walkers, dim)[:2].cpu().numpy()
    e0_host = energy[:2].cpu().numpy()
    for t in range(warmup):
        bg.anneal_step(plan, psi, energy, sites[t], gates[t], u[t], temps[t], 1, acc)
    torch.cuda.synchronize()
    accepted = 0
    e0, e1 = _events()
    e0.record()
    for t in range(warmup, total):
        bg.anneal_step(plan, psi, energy, sites[t], gates[t], u[t], temps[t], 1, acc)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    accepted = int(acc.sum())  # last step's acceptances
    t0 = time.perf_counter()
    oracle.anneal_step(host0, e0_host, S, sites_h[0, :2], haar[0, :2], u_h[0, :2], temps[0], 1)
    cpu_step = (time.perf_counter() - t0) / 2
    return {"workload": f"{walkers} complex states of {S} spins; gate on a random pair, "
                        f"entropy across the middle cut (Gram with 9 slices), Metropolis "
                        f"minimising it at T_t = 0.05 x 0.9^t",
            "steps": steps, "ms_per_step": ms, "value": walkers / (ms * 1e-3),
            "unit": "walker-steps/s", "mean_entropy_start": e_start,
            "mean_entropy_end": float(energy.mean()),
            "accepted_last_step": accepted,
            "cpu_oracle": {"s_per_walker_step": cpu_step, "walker_steps": 2,
                           "note": "the oracle's gate, entropy (numpy eigvalsh) and decision"}}


def ablation_line(bg, batch, A, B, C0, steps: int, warmup: int, streams=(1, 4, 8, 16)):
    """The paper's taskedGEMM against its batchedGEMM, with this library's kernels
    (Sec. 3, Sec. 4.A): per size class of the log-uniform mix, N concurrent
    streams each submitting its own round-robin share of the class's instances
    as one grouped call (the tasks), against N = 1 (one launch for the whole
    class), and the whole mix as one launch against 16 tasks. FP64 and 9
    slices, default tile programs in both arms."""
    import torch
    cur = torch.cuda.current_stream()
    pool = [torch.cuda.Stream() for _ in range(max(streams))]
    out = {}
    classes = [(str(n), np.flatnonzero(batch.table[:, 0] == n)) for n in
               sorted(set(int(x) for x in batch.table[:, 0]))]
    classes.append(("all", np.arange(batch.count)))
    for mode in ("fp64", "split9"):
        prec = None if mode == "fp64" else bg.precision("split", 9)
        res = {}
        for cname, sel in classes:
            row = {}
            fl = float(np.sum(2.0 * batch.table[sel, 0] * batch.table[sel, 1] *
                              batch.table[sel, 2]))
            for N in (streams if cname != "all" else (1, max(streams))):
                parts = [sel[j::N] for j in range(N) if sel[j::N].size]
                plans = [bg.batched_gemm_plan("r64", batch.table[p], prec) for p in parts]
                C = C0.clone()

                def tasks():
                    for s in pool[:len(plans)]:
                        s.wait_stream(cur)
                    for s, pl in zip(pool, plans):
                        with torch.cuda.stream(s):
                            bg.batched_gemm_grouped(pl, A, B, C, batch.alpha, batch.beta,
                                                    stream=s)
                    for s in pool[:len(plans)]:
                        cur.wait_stream(s)

                ms = _time_calls(tasks, steps, warmup)
                row[f"N={N}"] = {"ms": ms, "value": fl / (ms * 1e-3) / 1e12}
                for pl in plans:
                    pl.close()
                del C
            row["batched_over_tasked16"] = (row[f"N={max(streams)}"]["ms"] /
                                            row["N=1"]["ms"])
            res[cname] = row
        out[mode] = res
    out["unit"] = UNIT
    return out



def run_reference(args, world, rank, pg):
    """--impl reference: the CPU oracle, as it stands, on bounded samples of the workload."""
    if rank != 0:
        return
    batch, desc = make_batch(args.workload, args.count, 0)
    budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    ids = calibrated_sample(batch, budget)
    times, flops, threads = [], 0.0, 1
    for it in range(args.warmup + args.steps):
        _, dt, fl, threads = oracle_on(batch, ids)
        if it >= args.warmup:
            times.append(dt)
            flops = fl
    mean = float(np.mean(times))
    value = flops / mean / 1e12
    sample = (f"{len(ids)} of {batch.count} instances (every "
              f"{max(1, batch.count // max(1, len(ids)))}-th, all size classes), "
              f"{flops / 1e9:.2f} GFLOP per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": desc, "mode": "cpu oracle (plain triple loop, FP64)",
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank, pg)
        return
    import torch
    from paper_2203_09353_gb300 import build as libbuild
    libbuild.build()
    import paper_2203_09353_gb300 as bg

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    log(bind_near_gpu(local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    pk, pk_src = peaks()
    batch, desc = make_batch(args.workload, args.count, rank, world)
    log(f"generated {desc}")
    flops = batch.flops()
    job_flops = sum_over_ranks(pg, flops)  # every rank's shard counts toward the job
    A = torch.from_numpy(batch.A).to(dev)
    B = torch.from_numpy(batch.B).to(dev)
    C0 = torch.from_numpy(batch.C).to(dev)
    dtab = torch.from_numpy(batch.table).to(dev)
    modes = [m for m in args.modes.split(",") if m]
    if args.mode not in modes:
        modes.append(args.mode)

    fp64_peak = bg.probe_fp64_peak()
    log(f"FP64 DFMA probe: {fp64_peak:.3f} TFLOP/s")
    cache = os.path.join(tempfile.gettempdir(), "bgemm_autotune.json")
    plans = {}
    for m in modes:
        if m == "fp64":
            prec, flags = None, bg.BG_PLAN_AUTOTUNE | bg.BG_PLAN_USE_CACHE | bg.BG_PLAN_PROFILE
        else:
            prec, flags = bg.precision("split", int(m[5:])), bg.BG_PLAN_PROFILE
        plans[m] = bg.batched_gemm_plan(batch.dtype, batch.table, prec, flags, cache)

    log("plans built: " + ", ".join(f"{m}: {plans[m].info()['workspace_bytes'] / 2**30:.2f} GiB"
                                    for m in modes))
    # --- correctness of every mode: oracle on a sample (rank 0), FP64 path on all instances
    ref, cpu = None, None
    if rank == 0 and not args.no_cpu:
        ids = calibrated_sample(batch, args.cpu_seconds)
        ref, dt, fl, threads = oracle_on(batch, ids)
        cpu = {"value": fl / dt / 1e12, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": (f"{len(ids)} of {batch.count} instances (every "
                          f"{max(1, batch.count // max(1, len(ids)))}-th, all size classes), "
                          f"{fl / 1e9:.2f} GFLOP in {dt:.2f} s")}
        log(f"oracle sample: {cpu['sample']}")
    outs = {}
    for m in modes:
        Cm = C0.clone()
        bg.batched_gemm_grouped(plans[m], A, B, Cm, batch.alpha, batch.beta)
        outs[m] = Cm
    torch.cuda.synchronize()
    outs_head = outs[args.mode].cpu().numpy() if not args.no_e2e else None
    bg.check_device_errors()
    errs = {}
    errbuf = torch.zeros(batch.count, dtype=torch.float64, device=dev)
    for m in modes:
        e = {}
        if ref is not None:
            e["max_vs_oracle_sample"] = sample_errors(batch, outs[m].cpu().numpy(), ref)
        if "fp64" in outs and m != "fp64":
            bg.rel_err(batch.dtype, dtab, A, B, outs[m], outs["fp64"], errbuf, batch.count)
            e["max_vs_fp64_path_all"] = float(errbuf.max().item())
        errs[m] = e
    # final scalar reduce over ranks, outside the timed region (the ranks share
    # nothing on the data path): the whole job's sum of ||C_i||_F^2 of the
    # headline mode, its instance count and its worst error against the FP64 path
    job_reduce = {
        "sum_c_frobenius_sq": sum_over_ranks(pg, float(outs[args.mode].pow(2).sum())),
        "instances": int(sum_over_ranks(pg, float(batch.count))),
        "max_err_vs_fp64_path": (max_over_ranks(pg, errs[args.mode]["max_vs_fp64_path_all"])
                                 if "max_vs_fp64_path_all" in errs[args.mode] else None)}
    del outs
    log("errors: " + json.dumps(errs))

    # --- timing per mode
    res = {}
    clocks = None
    launches = 0
    for m in modes:
        steps = (args.fp64_steps or args.steps) if m == "fp64" and m != args.mode else args.steps
        Cm = C0.clone()
        for _ in range(args.warmup):
            bg.batched_gemm_grouped(plans[m], A, B, Cm, batch.alpha, batch.beta)
        plans[m].kernel_times(reset=True)
        torch.cuda.synchronize()
        barrier(pg)
        headline = m == args.mode
        if headline:
            sampler = Clocks(local)
            sampler.start()
            bg.launch_count(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            bg.batched_gemm_grouped(plans[m], A, B, Cm, batch.alpha, batch.beta)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(pg)
        if headline:
            launches = bg.launch_count()
            clocks = sampler.stop()
        ms = e0.elapsed_time(e1) / steps
        ms = max_over_ranks(pg, ms)
        kt, calls = plans[m].kernel_times(reset=True)
        log(f"{m}: {ms:.3f} ms/step")
        res[m] = {"ms_per_step": ms, "steps": steps,
                  "value": job_flops / (ms * 1e-3) / 1e12,
                  "kernel_ms": [x / max(calls, 1) for x in kt]}
        del Cm

    # --- split modes with BG_PLAN_AUTOTUNE: each size class on the split path or
    # on the FP64 path, whichever the plan measured faster
    for m in modes:
        if m == "fp64":
            continue
        tp = bg.batched_gemm_plan(batch.dtype, batch.table, bg.precision("split", int(m[5:])),
                                  bg.BG_PLAN_AUTOTUNE | bg.BG_PLAN_USE_CACHE, cache)
        Cm = C0.clone()
        ms = _time_calls(lambda: bg.batched_gemm_grouped(tp, A, B, Cm, batch.alpha, batch.beta),
                         args.steps, args.warmup)
        Cm.copy_(C0)
        bg.batched_gemm_grouped(tp, A, B, Cm, batch.alpha, batch.beta)
        err = sample_errors(batch, Cm.cpu().numpy(), ref) if ref is not None else None
        routes = {str(c["bucket"][0]): c["program"] for c in json.loads(tp.describe())["classes"]}
        ms = max_over_ranks(pg, ms)
        res[m]["autotuned"] = {"ms_per_step": ms, "value": job_flops / (ms * 1e-3) / 1e12,
                               "unit": UNIT, "routes": routes,
                               "default_over_tuned": res[m]["ms_per_step"] / ms,
                               "max_err_vs_oracle_sample": err}
        tp.close()
        del Cm

    # --- roofline of the dominant kernel of each mode
    traffic_ok = args.workload == "mix-loguniform" and split_sources_sha() == NCU_SOURCES_SHA
    t = batch.table.astype(np.float64)
    esz = 16.0 if batch.dtype == "c128" else 8.0
    ab_elems = float(np.sum(t[:, 0] * t[:, 2] + t[:, 2] * t[:, 1]))
    for m in modes:
        r = res[m]
        if m == "fp64":
            k_ms = r["kernel_ms"][0]
            ach = flops / (k_ms * 1e-3) / 1e12
            r["roofline"] = {"kernel": "fp64_persistent", "bound": "alu", "achieved": ach,
                             "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
                             "traffic": None,
                             "peak_source": "DFMA probe measured live (bg_probe_fp64_peak)"}
        else:
            s = int(m[5:])
            pairs = s * (s + 1) // 2
            sp = json.loads(plans[m].describe()).get("split", {})
            # instances on the small-instance kernel (real, m, n, k <= 64) leave
            # the tile GEMM and the slicer; the flops are real-GEMM flops (2 mnk)
            small_fl = 2.0 * sp.get("small_mnk", 0.0)
            small_ab = sp.get("small_ab_elems", 0.0)
            k_ms = r["kernel_ms"][1]
            tf = pairs * (flops - small_fl)
            ach = tf / (k_ms * 1e-3) / 1e12
            pk_bf16 = pk["bf16_tflops"]
            r["roofline"] = {"kernel": "split_gemm_kernel (tcgen05)", "bound": "tensor",
                             "achieved": ach, "peak": pk_bf16, "unit": "TFLOP/s",
                             "frac": ach / pk_bf16,
                             "traffic": (NCU_TRAFFIC_PER_BYTE[m]["gemm"] * batch.bytes_moved()
                                         if traffic_ok and m in NCU_TRAFFIC_PER_BYTE else None),
                             "flops_per_launch": tf,
                             "instances": batch.count - sp.get("small_instances", 0),
                             "peak_source": f"bf16 burst, {pk_src} (MEASURED_PEAKS.json)"}
            if sp.get("small_instances", 0) > 0:
                sm_ms = r["kernel_ms"][2]
                sm_tf = pairs * small_fl / (sm_ms * 1e-3) / 1e12
                # mma.sync BF16 issues 2048 flop/clk/SM, a quarter of tcgen05 (microbenchmark)
                sm_pk = pk_bf16 / 4.0
                r["small"] = {"kernel": "split_small_kernel (mma.sync)", "bound": "tensor",
                              "instances": sp["small_instances"], "ms": sm_ms,
                              "achieved": sm_tf, "peak": sm_pk, "unit": "TFLOP/s",
                              "frac": sm_tf / sm_pk,
                              "peak_source": "bf16 burst / 4 (mma.sync rate, 2048 of 8192 "
                                             "flop/clk/SM)",
                              "flops_per_launch": pairs * small_fl,
                              "traffic": (NCU_TRAFFIC_PER_BYTE[m]["small"] * batch.bytes_moved()
                                          if traffic_ok and m in NCU_TRAFFIC_PER_BYTE else None)}
            sl_ms = r["kernel_ms"][0]
            sl_bytes = (ab_elems - small_ab) * (esz + 2.0 * s * (4.0 if batch.dtype == "c128" else 1.0))
            r["slicer"] = {"kernel": "split_slice_kernel", "bound": "hbm",
                           "achieved": sl_bytes / (sl_ms * 1e-3) / 1e9, "peak": pk["hbm_gbs"],
                           "unit": "GB/s",
                           "frac": sl_bytes / (sl_ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                           "ms": sl_ms, "algorithmic_bytes": sl_bytes,
                           "traffic": (NCU_TRAFFIC_PER_BYTE[m]["slicer"] * batch.bytes_moved()
                                       if traffic_ok and m in NCU_TRAFFIC_PER_BYTE else None)}
            if r["slicer"]["traffic"] is not None:
                r["slicer"]["traffic_over_algorithmic"] = r["slicer"]["traffic"] / sl_bytes
                step_traffic = (r["slicer"]["traffic"] + r["roofline"]["traffic"]
                                + (r["small"]["traffic"] if "small" in r else 0.0))
                r["step_traffic"] = {"bytes": step_traffic, "eq1_bytes": batch.bytes_moved(),
                                     "over_eq1": step_traffic / batch.bytes_moved()}
            r["tensor_tflops_per_step"] = tf / (r["ms_per_step"] * 1e-3) / 1e12
        r["error"] = errs.get(m, {})

    # --- end to end through the public API with host buffers. The batch is cut
    # into instance ranges, each with its own plan; the host->device copies of
    # range i+1, the GEMM of range i and the device->host read of range i-1
    # run on three streams, so that copies in both directions overlap the
    # compute (all within the timed region, every step).
    e2e = None
    head = args.mode
    if not args.no_e2e:
        Ah = torch.from_numpy(batch.A).pin_memory()
        Bh = torch.from_numpy(batch.B).pin_memory()
        Ch = torch.from_numpy(batch.C).pin_memory()
        Co = torch.empty_like(Ch).pin_memory()
        Cd = torch.empty_like(C0)
        nch = max(1, min(args.e2e_chunks, batch.count))
        cuts = [batch.count * j // nch for j in range(nch + 1)]
        prec_h = None if head == "fp64" else bg.precision("split", int(head[5:]))
        flags_h = (bg.BG_PLAN_AUTOTUNE | bg.BG_PLAN_USE_CACHE) if head == "fp64" else 0
        chunks = []
        for j in range(nch):
            i0, i1 = cuts[j], cuts[j + 1]
            if i1 <= i0:
                continue
            rng = []
            for col, n in ((6, batch.A.size), (7, batch.B.size), (8, batch.C.size)):
                lo = int(batch.table[i0, col])
                hi = int(batch.table[i1, col]) if i1 < batch.count else n
                rng.append((lo, hi))
            chunks.append((bg.batched_gemm_plan(batch.dtype, batch.table[i0:i1], prec_h, flags_h,
                                                cache), rng))
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        # two device buffer sets, alternating between steps, so that the copies of
        # step k + 1 need not wait for the GEMMs of step k
        sets = [(A, B, Cd), (torch.empty_like(A), torch.empty_like(B), torch.empty_like(Cd))]
        free_ev = [None, None]  # set k: its last GEMM and read-back of two steps ago
        stepc = [0]

        # phased schedule: a step's read-back waits for its last copy in, and
        # the next step's copies in wait for that read-back, so that the two
        # directions never share the host link
        phased = [False]

        def e2e_step():
            Ad, Bd, Cdd = sets[stepc[0] & 1]
            done_in, done_gemm = [], []
            if free_ev[stepc[0] & 1] is not None:
                s_in.wait_event(free_ev[stepc[0] & 1])
            if phased[0] and free_ev[(stepc[0] - 1) & 1] is not None:
                s_in.wait_event(free_ev[(stepc[0] - 1) & 1])
            for _, ((a0, a1), (b0, b1), (c0, c1)) in chunks:
                with torch.cuda.stream(s_in):
                    Ad[a0:a1].copy_(Ah[a0:a1], non_blocking=True)
                    Bd[b0:b1].copy_(Bh[b0:b1], non_blocking=True)
                    Cdd[c0:c1].copy_(Ch[c0:c1], non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(s_in)
                    done_in.append(ev)
            for (plan_j, _), ev in zip(chunks, done_in):
                stream.wait_event(ev)
                bg.batched_gemm_grouped(plan_j, Ad, Bd, Cdd, batch.alpha, batch.beta, stream=stream)
                evg = torch.cuda.Event()
                evg.record(stream)
                done_gemm.append(evg)
            if phased[0]:
                s_out.wait_event(done_in[-1])
            for (_, (_, _, (c0, c1))), evg in zip(chunks, done_gemm):
                s_out.wait_event(evg)
                with torch.cuda.stream(s_out):
                    Co[c0:c1].copy_(Cdd[c0:c1], non_blocking=True)
            fe = torch.cuda.Event()
            fe.record(s_out)  # after the last read-back, which follows the last GEMM
            free_ev[stepc[0] & 1] = fe
            stepc[0] += 1

        def timed_steps(n):
            for s in (s_in, s_out):
                s.wait_stream(stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for s in (s_in, s_out):
                s.wait_stream(stream)
            for _ in range(n):
                e2e_step()
            stream.wait_stream(s_in)
            stream.wait_stream(s_out)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / n

        def timed_alone(fn, n=3):
            """One resource of the pipeline alone, on the current stream."""
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(n):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / n

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        # packing partners differ between the range plans and the whole-batch
        # plan, so the split mode may differ in the last bits only
        got = Co.numpy()
        assert np.allclose(got, outs_head, rtol=1e-12, atol=1e-12 * float(np.max(np.abs(outs_head)))), \
            "pipelined end-to-end result differs from the whole-batch call"
        barrier(pg)
        n2 = max(2, args.steps // 2)
        # both schedules in this run; concurrent transfers in the two
        # directions have run at very different rates from one process to the
        # next on this machine, so the faster schedule is the one reported
        ms_overlap = max_over_ranks(pg, timed_steps(n2))
        phased[0] = True
        e2e_step()
        torch.cuda.synchronize()
        ms_phased = max_over_ranks(pg, timed_steps(n2))
        phased[0] = False
        ms = min(ms_overlap, ms_phased)
        # the pipeline's three resources, each alone: host-to-device copies of
        # one step, the range GEMMs, the device-to-host read-back
        Ad, Bd, Cdd = sets[0]
        h2d_ms = timed_alone(lambda: (Ad.copy_(Ah, non_blocking=True), Bd.copy_(Bh, non_blocking=True),
                                      Cdd.copy_(Ch, non_blocking=True)))
        gemm_ms = timed_alone(lambda: [bg.batched_gemm_grouped(pl, Ad, Bd, Cdd, batch.alpha,
                                                               batch.beta) for pl, _ in chunks])
        d2h_ms = timed_alone(lambda: Co.copy_(Cdd, non_blocking=True))
        hb, db = Ah.nbytes + Bh.nbytes + Ch.nbytes, Co.nbytes
        del sets  # set 0 is (A, B, Cd): its copies wrote the same values A and B held
        e2e = {"value": job_flops / (ms * 1e-3) / 1e12, "unit": UNIT,
               "h2d_bytes_per_step": int(hb), "d2h_bytes_per_step": int(db), "ms_per_step": ms,
               "pipeline": (f"{len(chunks)} instance ranges on three streams (copies in, range "
                            f"GEMMs, read-back), two device buffer sets alternating between steps"),
               "schedule": "overlapped" if ms_overlap <= ms_phased else "phased",
               "ms_overlapped": ms_overlap, "ms_phased": ms_phased,
               "breakdown": {"h2d_alone_ms": h2d_ms, "h2d_gbs": hb / (h2d_ms * 1e-3) / 1e9,
                             "gemm_alone_ms": gemm_ms, "d2h_alone_ms": d2h_ms,
                             "d2h_gbs": db / (d2h_ms * 1e-3) / 1e9,
                             "bound": "host link" if h2d_ms >= max(gemm_ms, d2h_ms) else
                                      ("GEMM" if gemm_ms >= d2h_ms else "read-back")}}

    # --- the paper's design on this GPU, for context: one cuBLAS GEMM per instance
    lib_base = None
    if not args.no_library_baseline and batch.dtype == "r64":
        ms_l, C_l = cublas_per_instance(batch, A, B, C0, steps=3, warmup=1)
        ms_l = max_over_ranks(pg, ms_l)
        ref64 = C0.clone()
        bg.batched_gemm_grouped(plans[modes[0]], A, B, ref64, batch.alpha, batch.beta)
        diff = float((C_l - ref64).abs().max() / ref64.abs().max())
        lib_base = {"kind": "cuBLAS DGEMM per instance (torch.addmm), 8 concurrent streams, "
                            "replayed as one CUDA graph", "value": job_flops / (ms_l * 1e-3) / 1e12,
                    "unit": UNIT, "ms_per_step": ms_l, "launches_per_step": batch.count,
                    "max_abs_diff_rel_to_max": diff}
        log(f"cuBLAS per instance: {ms_l:.3f} ms/step")
        del C_l, ref64

    chain = None
    if not args.no_chain:
        chain = chain_line(bg)
        log(f"chain: {json.dumps(chain)}")

    gate = None
    if not args.no_gate:
        gate = gate_line(bg, fp64_peak, pk["hbm_gbs"], f"copy bandwidth, {pk_src} (MEASURED_PEAKS.json)")
        log(f"local gate: {json.dumps(gate)}")

    herk = None
    if not args.no_herk:
        herk = herk_line(bg, steps=max(2, args.steps // 2), warmup=1)
        log(f"Hermitian update: {json.dumps(herk)}")

    ablation = None
    if not args.no_ablation and batch.dtype == "r64" and args.workload.startswith("mix-"):
        ablation = ablation_line(bg, batch, A, B, C0, steps=3, warmup=1)
        log(f"ablation: {json.dumps(ablation)}")

    configs = None
    if not args.no_configs:
        configs = configs_line(bg, pk, fp64_peak, steps=max(3, args.steps // 2), warmup=2,
                               cpu_seconds=min(args.cpu_seconds, 4.0), cache=cache)
        log(f"configs: {json.dumps(configs)}")

    entropy = None
    if not args.no_entropy:
        entropy = entropy_line(bg, fp64_peak)
        log(f"entropy: {json.dumps(entropy)}")

    anneal = None
    if not args.no_anneal:
        anneal = anneal_line(bg)
        log(f"anneal: {json.dumps(anneal)}")

    if rank != 0:
        return
    h = res[head]
    roof = dict(h["roofline"])
    line = {
        "metric": METRIC, "value": h["value"], "unit": UNIT, "n_gpus": world,
        "steps": h["steps"], "warmup": args.warmup, "ms_per_step": h["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if head == "fp64" else "bf16 digit planes, fp32 exact sums, int64/f64 "
                                              "recombination",
        "data": "synthetic",
        "config": {"workload": desc, "mode": head, "count": batch.count,
                   "gflop_per_step_fp64_equiv": flops / 1e9,
                   "l2": "inputs (A, B, C) larger than L2, no flush",
                   "parallelism": (f"{world} parts of one batch split longest-first by flops, "
                                   "no collective on the data path" if world > 1 and
                                   args.workload.startswith("mix-") else
                                   f"{world} independent replica(s), no collective")},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "job_reduce": job_reduce,
        "modes": res,
        "fp64_peak_tflops_measured": fp64_peak,
        "library_baseline": lib_base,
        "herk": herk,
        "chain": chain,
        "gate": gate,
        "configs": configs,
        "entropy": entropy,
        "anneal": anneal,
        "ablation": ablation,
        "peaks_source": pk_src,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
