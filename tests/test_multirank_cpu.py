"""The multi-rank path on CPU: two gloo ranks each simulate their own path
range (with the FP64 oracle standing in for a GPU) and merge the payoff sums
in rank order; the result equals the unsharded simulation."""
import os
import socket
import tempfile

import numpy as np
import pytest

from paper_1006_3340_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    from oracle import oracle as ora
    from oracle import quadrature
    from paper_1006_3340_gb300 import workloads

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = workloads.small_plain(paths=1001)
        x, W = quadrature.rule_for(wl)
        first, count = shard.shard_range(wl.paths, rank, world)
        r = ora.simulate(ora.OracleModel(wl, x, W), ora.PICARD, path0=first, npaths=count, threads=2)
        s1, s2, n = shard.merge_sums(r["sum"], r["sumsq"], count)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), s1=s1, s2=s2, n=n)
    finally:
        dist.destroy_process_group()


def test_shard_ranges_cover_all_paths():
    for total in [1, 7, 1000, 1 << 20]:
        for world in [1, 2, 3, 8]:
            ranges = [shard.shard_range(total, r, world) for r in range(world)]
            assert ranges[0][0] == 0
            for (f0, c0), (f1, _) in zip(ranges, ranges[1:]):
                assert f0 + c0 == f1
            assert sum(c for _, c in ranges) == total


def test_two_gloo_ranks_merge_to_unsharded_result():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    from oracle import oracle as ora
    from oracle import quadrature
    from paper_1006_3340_gb300 import workloads

    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(2, _free_port(), d), nprocs=2, join=True, start_method="spawn")
        res = [np.load(os.path.join(d, f"rank{r}.npz")) for r in range(2)]
        wl = workloads.small_plain(paths=1001)
        x, W = quadrature.rule_for(wl)
        ref = ora.simulate(ora.OracleModel(wl, x, W), ora.PICARD, threads=1)
        for r in res:  # every rank holds the same merged sums
            assert int(r["n"]) == wl.paths
            assert np.allclose(r["s1"], ref["sum"], rtol=1e-12, atol=0)
            assert np.allclose(r["s2"], ref["sumsq"], rtol=1e-12, atol=0)
        assert np.array_equal(res[0]["s1"], res[1]["s1"])
