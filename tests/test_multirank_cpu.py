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
