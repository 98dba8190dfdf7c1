"""Host logic of bench.py and of the workload recipes it times (no GPU):
workload dispatch, the network shape per workload, default schemes, and the
batched configuration's recipe (256 uneven term structures, 2^24 paths)."""
import argparse
import importlib.util
import os

import numpy as np

from paper_1006_3340_gb300 import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)  # imports numpy and the workload recipes only; torch is imported in main()
    return mod


def _args(**kw):
    base = dict(workload="large_single", paths=0, schemes="")
    base.update(kw)
    return argparse.Namespace(**base)


def test_workload_dispatch_and_network_shape():
    b = _bench()
    wl = b._workload(_args())
    assert (wl.N, wl.paths, wl.Q) == (40, 1 << 20, 64)
    assert b._arch(wl) == (128, 3)
    wl = b._workload(_args(workload="long_dated"))
    assert (wl.N, wl.paths, wl.Q) == (120, 1 << 22, 96)
    assert b._arch(wl) == (256, 4)
    assert b._workload(_args(paths=4096)).paths == 4096


def test_default_schemes():
    b = _bench()
    assert b._schemes(_args()) == ["picard", "full", "mlp"]
    assert b._schemes(_args(workload="long_dated")) == ["picard", "full", "mlp_vec"]
    assert b._schemes(_args(schemes="picard,mlp_vec")) == ["picard", "mlp_vec"]
    assert b._code("mlp_vec") == "mlp" and b._code("full") == "full"


def test_batched_recipe():
    wls = workloads.batched_instances()
    assert len(wls) == 256
    assert sum(wl.paths for wl in wls) == 1 << 24
    assert all(8 <= wl.N <= 80 and wl.delta in (0.25, 0.5) and wl.s == 8 and wl.Q == 64 for wl in wls)
    assert all(wl.strikes.shape == (wl.n, 11) for wl in wls)
    assert [wl.inst for wl in wls] == list(range(256))
    # uneven: tenor counts and path budgets both spread
    assert len({wl.N for wl in wls}) > 40
    budgets = np.array([wl.paths for wl in wls])
    assert budgets.max() > 20 * budgets.min()


def test_training_flop_count():
    """6 x params per training row (forward 2, backward 4) over the library's
    Adam steps: per-rate head, pairs = records x (n + 1) / 2 per step."""
    b = _bench()
    wl = workloads.large_single()
    f = b._train_flop(wl, 128, 3, 0, 39432, 4, 8192)
    steps = int((1 << 16) * 8 * 20 // 8192) * 4
    assert f == steps * 8192 * 6.0 * 39432
    fv = b._train_flop(workloads.long_dated(), 256, 4, 1, 263296, 20, 4096)
    assert fv == ((1 << 16) * 8 // 4096) * 20 * 4096 * 6.0 * 263296


def test_traffic_entries_follow_source_hashes(tmp_path):
    """A DRAM-traffic entry counts only while every source it lists still has
    the SHA-1 it was measured with; otherwise, and for unknown keys, the bench
    reports null."""
    import hashlib
    import json

    b = _bench()
    csrc = tmp_path / "paper_1006_3340_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("kernel v1")
    (tmp_path / "profiles").mkdir()
    entry = {"dram_bytes_read": 10.0, "dram_bytes_write": 2.0,
             "sources": {"k.cu": hashlib.sha1(b"kernel v1").hexdigest()}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"x": entry}))
    b.ROOT = str(tmp_path)
    assert b._traffic("x") == 12.0
    assert b._traffic("missing") is None
    (csrc / "k.cu").write_text("kernel v2")
    assert b._traffic("x") is None
