"""GPU parity of the split-BF16 tensor-core mode against the FP64 oracle.

Tolerances (per instance, ||C - C_ref||_F / (||A||_F ||B||_F)): 1e-6 for the
3-slice mode, 1e-12 for the 6- and 9-slice modes. Exactness pins: inputs that
the digit planes represent exactly (small integers times powers of two) must
give the exact product bit for bit, which checks that the FP32 tensor-core
sums and the integer recombination lose nothing.
"""
import numpy as np
import pytest

import oracle
import paper_2203_09353_gb300 as bg
from paper_2203_09353_gb300 import synth

from gpu_util import TOL_FP64, TOL_SPLIT, dev, errors, host, oracle_batch, run_fixed, run_grouped

pytestmark = pytest.mark.gpu


def split(s, beta_bits=0):
    return bg.precision("split", s, beta_bits)


@pytest.mark.parametrize("s", [3, 6, 9])
def test_size_mix_loguniform_reduced(gpu, s):
    """Log-uniform entries (1e-4..1e4, random signs), all six size classes, alpha=1, beta=0.5."""
    b = synth.size_mix_loguniform(count=150)
    C, plan = run_grouped(b, split(s))
    info = plan.info()
    # slicer, small-instance kernel (n <= 64), tile kernel
    assert info["slices"] == s and info["launches_per_call"] == 3
    e = errors(b, host(C), oracle_batch(b))
    assert e.max() <= TOL_SPLIT[s], (s, e.max())


def _small_batch(seed, count, pad=True):
    """Real instances with m, n, k in [1, 64] (k = 0 and the extremes included),
    leading dimensions padded beyond m or k, log-uniform entries."""
    rng = np.random.default_rng(seed)
    shapes = [(int(rng.integers(1, 65)), int(rng.integers(1, 65)), int(rng.integers(1, 65)))
              for _ in range(count)]
    shapes += [(64, 64, 64), (1, 1, 1), (64, 1, 64), (1, 64, 64), (33, 17, 0), (16, 16, 16)]
    rows, ao, bo, co = [], 0, 0, 0
    for (m, n, k) in shapes:
        lda = m + (int(rng.integers(0, 5)) if pad else 0)
        ldb = max(k, 1) + (int(rng.integers(0, 5)) if pad else 0)
        ldc = m + (int(rng.integers(0, 5)) if pad else 0)
        rows.append((m, n, k, lda, ldb, ldc, ao, bo, co))
        ao += lda * max(k, 1) + 8
        bo += ldb * n + 8
        co += ldc * n + 8
    table = np.array(rows, dtype=np.int64)

    def fill(size):
        return rng.choice([-1.0, 1.0], size) * 10.0 ** rng.uniform(-4, 4, size)

    return synth.Batch("small", "r64", table, fill(ao), fill(bo), fill(co), -1.5, 0.75)


@pytest.mark.parametrize("s", [3, 6, 9])
def test_small_instance_kernel(gpu, s):
    """Real instances with m, n, k <= 64 go to the fused small-instance kernel
    (digits cut into shared memory, level sums on mma.sync); the same batch
    planned with BG_PLAN_SPLIT_TILES runs on the digit-plane tile kernels. Both
    meet the mode's tolerance against the oracle."""
    import json
    b = _small_batch(100 + s, 300)
    ref = oracle_batch(b)
    C, plan = run_grouped(b, split(s))
    d = json.loads(plan.describe())["split"]
    # the planner's route: edges <= 32 always; 33..64 above 48 (9 slices), 40 (6), 32 (3)
    edge = b.table[:, :3].max(axis=1)
    small = (edge <= 32) | (edge > {9: 48, 6: 40, 3: 32}[s])
    assert d["small_instances"] == int(small.sum()) > 0
    assert (d["units"] == 0) == bool(small.all())
    assert plan.info()["launches_per_call"] == (1 if small.all() else 3)
    e = errors(b, host(C), ref)
    assert e.max() <= TOL_SPLIT[s], (s, e.max())
    Ct, plan_t = run_grouped(b, split(s), bg.BG_PLAN_SPLIT_TILES)
    dt = json.loads(plan_t.describe())["split"]
    assert dt["small_instances"] == 0 and dt["units"] > 0
    et = errors(b, host(Ct), ref)
    assert et.max() <= TOL_SPLIT[s], (s, et.max())
    bg.check_device_errors()


@pytest.mark.parametrize("s", [3, 6, 9])
def test_small_instance_kernel_extreme_exponents(gpu, s):
    """The small-instance kernel's own line exponents and digit cut at both ends
    of the FP64 range (every edge <= 32, so every instance takes that kernel):
    A or B made only of subnormal values, near-overflow operands, and zero or
    subnormal rows beside normal ones. Errors in exactly rescaled norms, as in
    test_split_extreme_exponents."""
    import json
    rng = np.random.default_rng(33 + s)
    cases = [((24, 20, 30), -1060, 1000), ((17, 31, 32), -1072, 1010),
             ((24, 20, 30), 900, 100), ((20, 24, 30), 1000, -1050), ((32, 32, 32), 0, 0),
             ((16, 16, 16), -1074 + 60, 0), ((9, 5, 3), 0, 0)]
    table, la, lb, lc = synth.pack_table([c[0] for c in cases])
    A, B, C = np.zeros(la), np.zeros(lb), np.zeros(lc)

    def fill(shape, scale):
        x = rng.uniform(-1, 1, shape)
        return x * 2.0 ** scale if abs(scale) < 1000 else x * 2.0 ** (scale // 2) * 2.0 ** (scale - scale // 2)

    for i, ((m, n, k), sa, sb) in enumerate(cases):
        _, _, _, lda, ldb, ldc, ao, bo, co = (int(v) for v in table[i])
        a, b = fill((m, k), sa), fill((k, n), sb)
        if i == 4:
            a[3, :] = 0.0                       # a zero row
            a[5, :] = fill(k, -1074 + 8)        # a row of tiny subnormals among normal ones
            a[7, 2] = 5e-324                    # the smallest subnormal in a normal row
            b[:, 6] = 0.0                       # a zero column
        A[ao:ao + lda * k] = np.asfortranarray(a).ravel(order="F")
        B[bo:bo + ldb * n] = np.asfortranarray(b).ravel(order="F")
    batch = synth.Batch("extreme_small", "r64", table, A, B, C, 1.0, 0.0)
    ref = oracle_batch(batch)
    got, plan = run_grouped(batch, split(s))
    assert json.loads(plan.describe())["split"]["small_instances"] == len(cases)
    got = host(got)
    for i, ((m, n, k), sa, sb) in enumerate(cases):
        _, _, _, lda, ldb, ldc, ao, bo, co = (int(v) for v in table[i])
        g = got[co:co + ldc * n].reshape(n, ldc).T[:m, :]
        r = ref[co:co + ldc * n].reshape(n, ldc).T[:m, :]
        assert np.all(np.isfinite(g)), i
        num = np.linalg.norm(np.ldexp(np.abs(g - r), -(sa + sb)))
        a = np.ldexp(np.abs(batch.instance(i, "A")), -sa)
        b = np.ldexp(np.abs(batch.instance(i, "B")), -sb)
        assert num <= TOL_SPLIT[s] * np.linalg.norm(a) * np.linalg.norm(b), (i, num)


def test_small_instance_kernel_alpha_zero_and_nan_c(gpu):
    """alpha = 0 reads neither A nor B (NaN there); beta = 0 does not read C (NaN there)."""
    b = _small_batch(7, 80)
    plan = bg.batched_gemm_plan("r64", b.table, split(9))
    Cd = dev(b.C)
    bg.batched_gemm_grouped(plan, dev(np.full_like(b.A, np.nan)), dev(np.full_like(b.B, np.nan)),
                            Cd, 0.0, 2.0)
    live = np.zeros(b.C.size, dtype=bool)  # C elements of the instances (not the ldc padding)
    for i in range(b.count):
        m, n, _, _, _, ldc, _, _, co = (int(v) for v in b.table[i])
        for j in range(n):
            live[co + j * ldc: co + j * ldc + m] = True
    assert np.array_equal(host(Cd), np.where(live, 2.0 * b.C, b.C))
    Cn = np.full_like(b.C, np.nan)
    Cd = dev(Cn)
    bg.batched_gemm_grouped(plan, dev(b.A), dev(b.B), Cd, 1.0, 0.0)
    b0 = synth.Batch(b.name, b.dtype, b.table, b.A, b.B, np.zeros_like(b.C), 1.0, 0.0)
    got = host(Cd)
    e = errors(b0, got, oracle_batch(b0))
    assert np.isfinite(e).all() and e.max() <= TOL_SPLIT[9]


@pytest.mark.parametrize("s", [3, 6, 9])
def test_size_mix_uniform_reduced(gpu, s):
    b = synth.size_mix_uniform(count=120)
    C, _ = run_grouped(b, split(s))
    e = errors(b, host(C), oracle_batch(b))
    assert e.max() <= TOL_SPLIT[s], (s, e.max())


@pytest.mark.parametrize("s", [3, 9])
def test_autotuned_plan_routes_and_matches_oracle(gpu, s, tmp_path):
    """BG_PLAN_AUTOTUNE in split mode times each size class on the split path and
    on the FP64 path and gives the class to the faster one; whatever the routes,
    every instance meets the mode's tolerance, and a cached second plan takes
    the same routes without timing."""
    import json
    b = synth.size_mix_loguniform(count=300)
    cache = str(tmp_path / "tune.json")
    flags = bg.BG_PLAN_AUTOTUNE | bg.BG_PLAN_USE_CACHE
    C, plan = run_grouped(b, split(s), flags, cache_path=cache)
    d = json.loads(plan.describe())
    routes = {tuple(c["bucket"]): c["program"] for c in d["classes"]}
    for c in d["classes"]:
        names = [x["program"] for x in c["tried"]]
        assert any(nm.startswith("split") for nm in names) and len(names) >= 2  # both paths timed
        if max(c["bucket"]) <= 64:  # small-instance kernel and tile kernels both timed
            assert {"split_small", "split_tiles"} <= set(names), names
    e = errors(b, host(C), oracle_batch(b))
    assert e.max() <= TOL_SPLIT[s], (s, e.max())
    n_split = sum(1 for v in routes.values() if v.startswith("split"))
    if n_split:
        # the classes given to the small-instance kernel are exactly its instances
        want_small = sum(c["members"] for c in d["classes"] if c["program"] == "split_small")
        assert d["split"]["small_instances"] == want_small
    sp = d.get("split")
    assert (sp is not None) == (n_split > 0)
    # split part: slicer, tile kernel, small-instance kernel (each when it has work); FP64 part
    want = (sum(1 for key in ("slice_jobs", "units", "small_instances") if sp[key] > 0) if sp else 0)
    want += 1 if n_split < len(routes) else 0
    assert plan.info()["launches_per_call"] == want
    C2, plan2 = run_grouped(b, split(s), flags, cache_path=cache)
    d2 = json.loads(plan2.describe())
    assert {tuple(c["bucket"]): c["program"] for c in d2["classes"]} == routes
    assert all(c["tried"] == [] for c in d2["classes"])
    assert np.array_equal(host(C2), host(C))


def test_error_decreases_with_slices(gpu):
    b = synth.size_mix_loguniform(count=100)
    ref = oracle_batch(b)
    prev = np.inf
    for s in (2, 3, 4, 6, 8, 9):
        C, _ = run_grouped(b, split(s))
        e = errors(b, host(C), ref).max()
        assert e <= prev * 1.0001 + 1e-17, (s, e, prev)
        prev = e
    assert prev <= 1e-14


def test_nine_slices_within_fp64_envelope(gpu):
    """9-slice error is of the order of the plain FP64 path's error."""
    b = synth.size_mix_loguniform(count=100)
    ref = oracle_batch(b)
    C64, _ = run_grouped(b)
    C9, _ = run_grouped(b, split(9))
    e64 = errors(b, host(C64), ref)
    e9 = errors(b, host(C9), ref)
    assert e9.max() <= max(8 * e64.max(), 4e-16), (e9.max(), e64.max())


@pytest.mark.parametrize("dtype", ["r64", "c128"])
@pytest.mark.parametrize("n", [16, 48, 64, 130, 256])
@pytest.mark.parametrize("s,beta", [(3, 8), (3, 0), (6, 0), (9, 0)])
def test_exact_on_representable_inputs(gpu, dtype, n, s, beta):
    """Entries d * 2^j with |d| < 2^7 and one power of two per row of A / column of B
    are cut exactly into the digit planes (at least 21 bits per line); every
    product and sum then fits FP64 exactly, so the result must equal the oracle
    bit for bit. beta = 0 takes the library's default width, i.e. the
    compile-time digit cut of the documented modes."""
    rng = np.random.default_rng(n)
    count = 6
    shapes = [(n, n, n)] * count
    table, la, lb, lc = synth.pack_table(shapes)

    def fill(size):
        v = rng.integers(-127, 128, size).astype(np.float64)
        if dtype == "c128":
            v = v + 1j * rng.integers(-127, 128, size)
        return v

    # per row of A a common power of two; per column of B too (exactly representable)
    A, B, C = fill(la), fill(lb), np.zeros(lc, dtype=np.complex128 if dtype == "c128" else np.float64)
    for i in range(count):
        ao, bo = table[i, 6], table[i, 7]
        a = A[ao:ao + n * n].reshape(n, n).T
        a *= (2.0 ** rng.integers(-20, 20, n))[:, None]
        A[ao:ao + n * n] = a.T.ravel()
        bb = B[bo:bo + n * n].reshape(n, n).T
        bb *= (2.0 ** rng.integers(-20, 20, n))[None, :]
        B[bo:bo + n * n] = bb.T.ravel()
    b = synth.Batch("exact", dtype, table, A, B, C, 1.0, 0.0)
    Cg, _ = run_grouped(b, split(s, beta))
    assert np.array_equal(host(Cg), oracle_batch(b))


@pytest.mark.parametrize("dtype", ["r64", "c128"])
def test_fixed_split_modes(gpu, dtype):
    b = synth.fixed_uniform(40, 33, 47, 61, seed=12, dtype=dtype,
                            alpha=(0.5 + 1j) if dtype == "c128" else 0.5,
                            beta=(0.25 - 1j) if dtype == "c128" else 0.25)
    ref = oracle_batch(b)
    for s in (3, 6, 9):
        C = host(run_fixed(b, split(s)))
        e = errors(b, C, ref)
        assert e.max() <= TOL_SPLIT[s], (s, e.max())


def test_hermitian_unitary_split_reduced(gpu):
    b = synth.hermitian_unitary_c128(batch=64)
    ref = oracle_batch(b)
    for s in (3, 6, 9):
        C = host(run_fixed(b, split(s)))
        e = errors(b, C, ref)
        assert e.max() <= TOL_SPLIT[s], (s, e.max())


@pytest.mark.parametrize("dtype", ["r64", "c128"])
def test_split_ragged_shapes_and_zero_k(gpu, dtype):
    rng = np.random.default_rng(8)
    shapes = [(int(rng.integers(1, 150)), int(rng.integers(1, 150)), int(rng.integers(0, 150)))
              for _ in range(30)] + [(5, 5, 0), (64, 64, 64), (20, 20, 20), (20, 20, 20)]
    table, la, lb, lc = synth.pack_table(shapes)
    dt = np.complex128 if dtype == "c128" else np.float64

    def fill(size):
        x = rng.uniform(-1, 1, size)
        return (x + 1j * rng.uniform(-1, 1, size)).astype(dt) if dtype == "c128" else x

    b = synth.Batch("ragged", dtype, table, fill(la), fill(lb), fill(lc),
                    (1 + 1j) if dtype == "c128" else 2.0, (0.5 - 0.5j) if dtype == "c128" else -0.5)
    ref = oracle_batch(b)
    for s in (3, 9):
        C, _ = run_grouped(b, split(s))
        e = errors(b, host(C), ref)
        assert e.max() <= TOL_SPLIT[s], (s, e.max())


def test_split_alpha_zero_and_nan_c(gpu):
    b = synth.size_mix_loguniform(count=40)
    plan = bg.batched_gemm_plan("r64", b.table, split(6))
    An, Bn = dev(np.full_like(b.A, np.nan)), dev(np.full_like(b.B, np.nan))
    Cd = dev(b.C)
    bg.batched_gemm_grouped(plan, An, Bn, Cd, 0.0, 2.0)
    assert np.array_equal(host(Cd), 2.0 * b.C)
    b0 = synth.Batch(b.name, b.dtype, b.table, b.A, b.B, np.full_like(b.C, np.nan), 1.0, 0.0)
    Cd = dev(b0.C)
    bg.batched_gemm_grouped(plan, dev(b.A), dev(b.B), Cd, 1.0, 0.0)
    got = host(Cd)
    live = np.zeros(b.C.size, dtype=bool)
    for i in range(b.count):
        m, n, _, _, _, ldc, _, _, co = b.table[i]
        for j in range(n):
            live[co + j * ldc: co + j * ldc + m] = True
    assert np.all(np.isfinite(got[live]))
    e = errors(b0, got, oracle_batch(b0, C0=np.zeros_like(b.C)))
    assert e.max() <= TOL_SPLIT[6]


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("s,beta", [(3, 8), (6, 7), (9, 7), (4, 5)])
def test_planes_reconstruct_input(gpu, axis, s, beta):
    """sum_p d_p 2^(e - beta p) equals the input to half a unit of the last digit; digits
    are integers within their bounds; the line exponent bounds the line's magnitudes."""
    import torch
    rng = np.random.default_rng(s * 10 + beta + axis)
    m, k = 37, 53
    X = rng.uniform(-1, 1, (m, k)) * 10.0 ** rng.uniform(-6, 6, (m, k))
    X[3, :] = 0.0
    X[:, 5] = 0.0
    Xf = np.asfortranarray(X)
    lines = m if axis == 0 else k
    exps = torch.zeros(lines, dtype=torch.int32, device="cuda")
    digits = torch.zeros(s * m * k, dtype=torch.int16, device="cuda")
    bg.split_planes(m, k, dev(Xf.ravel(order="F")), m, axis, s, beta, exps, digits)
    e = host(exps).astype(np.int64)
    raw = host(digits).view(np.uint16).astype(np.uint32) << 16
    dv = raw.view(np.float32).astype(np.float64).reshape(s, k, m).transpose(0, 2, 1)
    assert np.all(dv == np.round(dv))
    assert np.all(np.abs(dv[0]) <= 2.0 ** beta)
    assert np.all(np.abs(dv[1:]) <= 2.0 ** (beta - 1))
    for l in range(lines):
        line = X[l, :] if axis == 0 else X[:, l]
        if np.all(line == 0):
            assert e[l] == 0
        else:
            assert np.max(np.abs(line)) < 2.0 ** e[l] <= 2 * np.max(np.abs(line))
    E = e[:, None] if axis == 0 else e[None, :]
    recon = np.zeros((m, k))
    for p in range(s):
        recon += dv[p] * np.ldexp(1.0, (E - beta * (p + 1)).astype(np.int64))
    ulp_last = np.ldexp(1.0, (E - beta * s).astype(np.int64))
    assert np.all(np.abs(recon - X) <= 0.5 * ulp_last * (1 + 1e-12))


def test_bounded_wait_reports_timeout(gpu):
    bg.check_device_errors()
    bg.test_bounded_wait(2000)
    with pytest.raises(bg.BgemmError) as ei:
        bg.check_device_errors()
    assert ei.value.status == 6
    bg.check_device_errors()  # cleared


def test_split_runs_leave_no_device_error(gpu):
    b = synth.size_mix_loguniform(count=30)
    run_grouped(b, split(9))
    bg.check_device_errors()


def test_fp64_peak_probe(gpu):
    t = bg.probe_fp64_peak()
    assert 0.1 < t < 100.0


@pytest.mark.parametrize("s", [3, 4, 6, 9])
def test_long_k_multipass_sampled_rows(gpu, s):
    """Two 1024 x 768 instances with k = 2560: every mode then needs several
    exact-sum passes over k (3 slices: 768 per pass, 6 slices: 512, 9 slices:
    1472), each pass added into C. Sampled rows are checked against the oracle
    computing just those rows (m = 1 sub-problems)."""
    rng = np.random.default_rng(40 + s)
    m, n, k = 1024, 768, 2560
    count = 2
    A = rng.uniform(-1, 1, m * k * count)
    B = rng.uniform(-1, 1, k * n * count)
    C = rng.uniform(-1, 1, m * n * count)
    Cd = dev(C)
    bg.batched_gemm_fixed("r64", m, n, k, 1.0, dev(A), m, m * k, dev(B), k, k * n, 0.5, Cd, m,
                          m * n, count, split(s))
    got = host(Cd)
    for i in range(count):
        a, b, c = A[i * m * k:], B[i * k * n:(i + 1) * k * n], C[i * m * n:]
        for r in rng.choice(m, 6, replace=False):
            ref = c[r:].copy()
            oracle.gemm_fixed(1, n, k, 1.0, a[r:], m, 0, b, k, 0, 0.5, ref, m, 0, 1)
            cols = np.arange(n) * m
            row_ref = ref[cols]
            row_got = got[i * m * n + r + cols]
            # normwise for the row: ||c_r - ref_r|| / (||a_r|| ||B||)
            den = np.linalg.norm(a[r::m][:k]) * np.linalg.norm(b)
            assert np.linalg.norm(row_got - row_ref) / den <= TOL_SPLIT.get(s, 1e-6), (s, i, r)


@pytest.mark.parametrize("s", [3, 6, 9])
@pytest.mark.parametrize("dtype", ["r64", "c128"])
def test_split_extreme_exponents(gpu, dtype, s):
    """Operands at both ends of the FP64 range: A (or B) made of subnormal
    values only, which takes the fixed-point cut's left shift and the line
    maximum of a subnormal line; near-overflow operands; rows that are zero or
    subnormal next to normal ones. The product is representable in every case.
    The error is measured in exactly rescaled norms (powers of two), since the
    plain norms of subnormal operands underflow."""
    rng = np.random.default_rng(21)
    # (m, n, k) and the binary scale of A and of B
    cases = [((24, 20, 40), -1060, 1000), ((17, 33, 70), -1072, 1010),
             ((24, 20, 40), 900, 100), ((20, 24, 40), 1000, -1050), ((40, 40, 40), 0, 0)]
    table, la, lb, lc = synth.pack_table([c[0] for c in cases])
    cplx = dtype == "c128"
    dt = np.complex128 if cplx else np.float64
    A, B, C = np.zeros(la, dt), np.zeros(lb, dt), np.zeros(lc, dt)

    def fill(shape, scale):
        x = rng.uniform(-1, 1, shape)
        if cplx:
            x = x + 1j * rng.uniform(-1, 1, shape)
        return x * 2.0 ** scale if abs(scale) < 1000 else x * 2.0 ** (scale // 2) * 2.0 ** (scale - scale // 2)

    for i, ((m, n, k), sa, sb) in enumerate(cases):
        _, _, _, lda, ldb, ldc, ao, bo, co = (int(v) for v in table[i])
        a, b = fill((m, k), sa), fill((k, n), sb)
        if i == 4:
            a[3, :] = 0.0                       # a zero row
            a[5, :] = fill(k, -1074 + 8)        # a row of tiny subnormals among normal ones
            a[7, 2] = 5e-324                    # the smallest subnormal in a normal row
        A[ao:ao + lda * k] = np.asfortranarray(a).ravel(order="F")
        B[bo:bo + ldb * n] = np.asfortranarray(b).ravel(order="F")
    batch = synth.Batch("extreme", dtype, table, A, B, C, 1.0, 0.0)
    ref = oracle_batch(batch)
    got, _ = run_grouped(batch, split(s))
    got = host(got)
    for i, ((m, n, k), sa, sb) in enumerate(cases):
        _, _, _, lda, ldb, ldc, ao, bo, co = (int(v) for v in table[i])
        g = got[co:co + ldc * n].reshape(n, ldc).T[:m, :]
        r = ref[co:co + ldc * n].reshape(n, ldc).T[:m, :]
        assert np.all(np.isfinite(g)), i
        num = np.linalg.norm(np.ldexp(np.abs(g - r), -(sa + sb)))
        a = np.ldexp(np.abs(batch.instance(i, "A")), -sa)
        b = np.ldexp(np.abs(batch.instance(i, "B")), -sb)
        assert num <= TOL_SPLIT[s] * np.linalg.norm(a) * np.linalg.norm(b), (i, num)
