"""Host logic of the N>1 benchmark path, run as two gloo ranks on the CPU.

Every instance of Eq. (1) is independent, so ranks take disjoint seeded shards
of the same size mix (weak scaling) and exchange only their step times: a
barrier around the timed region and a max over ranks. These tests check that
each rank draws a different shard of identical shape statistics, that the
max-reduction returns the slowest rank's time on every rank, and that the
aggregate throughput counts every rank's instances.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist

    import bench

    class Args:
        pass

    w, r, _, pg = bench.dist_setup(Args())
    assert (w, r) == (world, rank) and pg is not None
    assert dist.get_backend() == "gloo"
    batch, desc = bench.make_batch("mix-loguniform", 300, r)
    bench.barrier(pg)
    # rank r pretends its step took (r + 1) ms; every rank must see the slowest
    t_max = bench.max_over_ranks(pg, float(r + 1))
    job_flops = bench.sum_over_ranks(pg, batch.flops())
    np.savez(os.path.join(out_dir, f"rank{r}.npz"), table=batch.table, A=batch.A[:64],
             t_max=t_max, desc=desc, flops=batch.flops(), job_flops=job_flops)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    for p in procs:
        if p.is_alive():
            p.kill()
            pytest.fail("a gloo rank did not finish")
        assert p.exitcode == 0
    r0, r1 = (np.load(tmp_path / f"rank{r}.npz") for r in range(2))
    # the slowest rank's time reaches both ranks
    assert float(r0["t_max"]) == 2.0 and float(r1["t_max"]) == 2.0
    # disjoint seeded shards: different draws, same count and size set
    assert str(r0["desc"]) != str(r1["desc"])
    assert not np.array_equal(r0["A"], r1["A"])
    t0, t1 = r0["table"], r1["table"]
    assert t0.shape == t1.shape == (300, 9)
    assert set(np.unique(t0[:, 0])) <= {16, 32, 64, 128, 256, 512}
    assert set(np.unique(t1[:, 0])) <= {16, 32, 64, 128, 256, 512}
    # the whole-job throughput of the weak-scaled run counts both shards
    fl = [float(np.sum(2.0 * t[:, 0] * t[:, 1] * t[:, 2])) for t in (t0, t1)]
    assert float(r0["flops"]) == fl[0] and float(r1["flops"]) == fl[1]
    assert float(r0["job_flops"]) == float(r1["job_flops"]) == fl[0] + fl[1]


def _lpt_rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist

    import bench
    import oracle

    class Args:
        pass

    _, r, _, pg = bench.dist_setup(Args())
    batch, ids = bench.lpt_shard(5, 150, world, r, "uniform")
    # this rank's per-instance result: ||A_i B_i||_F^2 by the CPU oracle (the
    # GEMM of the path, here on the host), summed, then reduced over ranks
    C = np.zeros_like(batch.C)
    oracle.gemm_grouped(batch.table, 1.0, batch.A, batch.B, 0.0, C)
    local = float(np.sum(C * C))
    total = bench.sum_over_ranks(pg, local)
    n_all = bench.sum_over_ranks(pg, float(batch.count))
    gathered = [None] * world
    dist.all_gather_object(gathered, [int(i) for i in ids])
    np.savez(os.path.join(out_dir, f"lpt{r}.npz"), ids=ids, total=total, n_all=n_all,
             local=local, flops=batch.flops(), everyone=np.concatenate([np.asarray(g) for g in
                                                                      gathered]))
    dist.destroy_process_group()


def test_lpt_partition_of_one_batch_and_scalar_reduce(tmp_path):
    """Two gloo ranks split ONE 300-instance size-mix batch longest-first by flops
    (bg_partition_lpt, computed on each rank), each multiplies its part (CPU
    oracle here) and the job's sum of ||C_i||_F^2 is reduced over the ranks. The
    parts are disjoint and cover every instance once, their flop loads differ by
    at most the largest instance, and the reduced sum equals the one-process sum."""
    import torch.multiprocessing as mp
    import oracle
    import paper_2203_09353_gb300 as bg
    from paper_2203_09353_gb300 import synth
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_lpt_rank_main, args=(r, 2, port, str(tmp_path)))
             for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    for p in procs:
        if p.is_alive():
            p.kill()
            pytest.fail("a gloo rank did not finish")
        assert p.exitcode == 0
    r0, r1 = (np.load(tmp_path / f"lpt{r}.npz") for r in range(2))
    ids0, ids1 = r0["ids"], r1["ids"]
    assert np.intersect1d(ids0, ids1).size == 0
    assert np.array_equal(np.sort(np.concatenate([ids0, ids1])), np.arange(300))
    assert np.array_equal(np.sort(r0["everyone"]), np.arange(300))
    ns = synth.draw_sizes(np.random.default_rng(5), 300)
    cost = 2.0 * ns.astype(np.float64) ** 3
    l0, l1 = cost[ids0].sum(), cost[ids1].sum()
    assert float(r0["flops"]) == l0 and float(r1["flops"]) == l1
    assert abs(l0 - l1) <= cost.max()
    part, load = bg.partition_lpt(cost, 2)
    assert np.array_equal(np.flatnonzero(part == 0), ids0) and np.allclose(load, [l0, l1])
    assert float(r0["total"]) == float(r1["total"]) == float(r0["local"]) + float(r1["local"])
    assert float(r0["n_all"]) == 300.0
    # one process over the same instances (values of each part from its own seed)
    want = 0.0
    for r, ids in ((0, ids0), (1, ids1)):
        b = synth.batch_of_sizes(np.random.default_rng(5 + 1000 * r), ns[ids], "uniform")
        C = np.zeros_like(b.C)
        oracle.gemm_grouped(b.table, 1.0, b.A, b.B, 0.0, C)
        want += float(np.sum(C * C))
    assert abs(float(r0["total"]) - want) <= 1e-12 * want


def test_partition_lpt_rules(bglib):
    """Longest first, ties to the lower index and the lower part; bad input refused."""
    import paper_2203_09353_gb300 as bg
    part, load = bg.partition_lpt([5, 3, 3, 2, 2, 2, 1], 3)
    assert part.tolist() == [0, 1, 2, 1, 2, 0, 1] and load.tolist() == [7, 6, 5]
    part, load = bg.partition_lpt([1.0] * 7, 3)  # equal costs: round robin
    assert part.tolist() == [0, 1, 2, 0, 1, 2, 0]
    part, load = bg.partition_lpt([], 4)
    assert part.size == 0 and load.tolist() == [0, 0, 0, 0]
    rng = np.random.default_rng(9)
    c = rng.random(1000) ** 4
    for parts in (2, 3, 8):
        part, load = bg.partition_lpt(c, parts)
        assert np.allclose(np.bincount(part, weights=c, minlength=parts), load)
        assert load.max() <= c.sum() / parts + c.max()
    for bad, parts in (([1.0, -1.0], 2), ([float("nan")], 2), ([1.0], 0), ([float("inf")], 1)):
        with pytest.raises(bg.BgemmError):
            bg.partition_lpt(bad, parts)
