"""Launch-shape autotuner for the path kernels and the batched launch.

For a model context (or a batch) and a scheme it times candidate launch
shapes -- threads per block, lanes per path (1: one lane sweeps all nodes of
its path; 4: four lanes share the node sweep of four paths), table rows per
staged chunk, resident blocks per SM, and the mapping (a sixth value G > 0
selects the tenor-parallel kernel with G lanes per path, each owning a block
of rates) -- with the library's own CUDA-event timing of the path kernel,
keeps the fastest, and caches the choice per GPU, workload shape and scheme
in ``_build/autotune.json`` (a per-machine file).
"""
from __future__ import annotations

import itertools
import json
import os
from typing import Dict, Iterable, Optional, Tuple

from . import build as _build
from . import lll

CACHE = os.path.join(_build.BUILD, "autotune.json")

DEFAULT_CANDIDATES = [
    # (threads, blocks_per_sm, chunk_rows, paths_per_thread, lanes_per_path[, tenor lanes])
    (t, 0, c, 1, l) for t, c, l in itertools.product((64, 128, 256), (0, 16), (1, 2, 4))
] + [(t, 0, c, 2, 1) for t, c in itertools.product((64, 128), (0, 16))] \
  + [(0, 0, 0, 0, 0, g) for g in (4, 8, 16, 32, -1)]


def apply(sim: "lll.LevyLibor", cand) -> None:
    """Set a candidate: the five launch values, then the mapping (sixth value,
    0 or absent: one lane per path; G > 0: tenor-parallel with G lanes per
    path; -1: Picard's step-parallel mapping)."""
    sim.set_launch(*cand[:5])
    g = cand[5] if len(cand) > 5 else 0
    if g < 0:
        sim.set_mapping("step")
    else:
        sim.set_mapping("tenor" if g else "path", g)


def _gpu_name() -> str:
    try:
        import torch

        return torch.cuda.get_device_name(torch.cuda.current_device())
    except Exception:  # pragma: no cover - only without torch/CUDA
        return "unknown"


def cache_key(kind: str, scheme: str, wl, paths: int) -> str:
    return f"{_gpu_name()}|{kind}|{scheme}|N={wl.N}|s={wl.s}|Q={wl.Q}|paths={paths}"


def _load() -> Dict[str, dict]:
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _store(key: str, entry: dict) -> None:
    data = _load()
    data[key] = entry
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".{os.getpid()}.tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def tune(sim: "lll.LevyLibor", scheme: str, paths: Optional[int] = None,
         candidates: Iterable[Tuple[int, int, int, int, int]] = DEFAULT_CANDIDATES,
         repeats: int = 3, use_cache: bool = True) -> dict:
    """Pick the fastest launch shape for ``sim`` and ``scheme`` and apply it."""
    paths = paths or sim.wl.paths
    key = cache_key("single", scheme, sim.wl, paths)
    if use_cache:
        hit = _load().get(key)
        if hit:
            apply(sim, hit["launch"])
            return dict(hit, cached=True)
    results = []
    for cand in candidates:
        try:
            apply(sim, cand)
            sim.simulate(scheme, paths=paths)  # warm-up
            best = min(_timed(sim, scheme, paths) for _ in range(repeats))
            results.append((best, cand))
        except lll.LLLError:
            continue  # shape not supported for this scheme / Q
    if not results:
        raise RuntimeError("no launch shape ran")
    results.sort()
    ms, launch = results[0]
    apply(sim, launch)
    entry = {"launch": list(launch), "ms": ms, "tried": [[m, list(c)] for m, c in results]}
    _store(key, entry)
    return dict(entry, cached=False)


def _timed(sim, scheme, paths) -> float:
    sim.simulate(scheme, paths=paths)
    return sim.kernel_ms()[0]


BATCH_CANDIDATES = [
    # (threads, blocks_per_sm, chunk_rows, paths_per_thread); 64-thread blocks and
    # two blocks per SM measured slowest on the 256-instance batch, and are left out
    (128, 0, 0, 1), (256, 0, 0, 1), (128, 0, 16, 1), (128, 0, 0, 2), (128, 0, 16, 2),
]


def tune_batch(b, instances, scheme: str, candidates: Iterable[Tuple[int, int, int, int]] = BATCH_CANDIDATES,
               repeats: int = 2, seed: int = 42) -> dict:
    """Same for a batch and one scheme (threads, blocks_per_sm, chunk_rows,
    paths_per_thread); applies the best to that scheme only."""
    code = lll.SCHEMES[scheme]
    results = []
    for cand in candidates:
        try:
            lll.lll_batch_set_launch(b, *cand, scheme=code)
            lll.lll_batch_simulate(b, code, seed)
            t = []
            for _ in range(repeats):
                lll.lll_batch_simulate(b, code, seed)
                t.append(lll.lll_batch_kernel_ms(b))
            results.append((min(t), cand))
        except lll.LLLError:
            continue
    if not results:
        raise RuntimeError("no batch launch shape ran")
    results.sort()
    lll.lll_batch_set_launch(b, *results[0][1], scheme=code)
    return {"launch": list(results[0][1]), "ms": results[0][0], "tried": [[m, list(c)] for m, c in results]}
