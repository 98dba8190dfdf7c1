"""Benchmark: path.tenor.steps/s of the Levy LIBOR Monte Carlo on GB300.

One step = one pass of the hot path over one batch: the Picard and the full
Euler schemes (plus the MLP drift when trained weights are available) each
simulate all paths of the workload and accumulate caplet payoffs.  A unit is
one (path, live rate, Euler step); rate i is live for i*s steps, so a path of
the N=40 workload has s*n(n+1)/2 = 6240 units.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (torchrun): rank r simulates its own 2^20 paths (global path indices
r*2^20 ...), weak scaling, no collective on the data path; timing is the max
over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1006_3340_gb300 import workloads  # noqa: E402

METRIC = "path·tenor·steps/s: Picard vs full Euler vs MLP drift, 1 GB300, ≤0.5bp caplet err"
L2_FLUSH_BYTES = 512 << 20


def _workload(args):
    if getattr(args, "workload", "large_single") == "long_dated":
        return workloads.long_dated(paths=args.paths or (1 << 22))
    return workloads.large_single(paths=args.paths or (1 << 20))


def _arch(wl):
    """(hidden width, hidden layers) of the learned compensator for a workload:
    43->128x3->1 on N=40, 123->256x4->1 on N=120."""
    return (256, 4) if wl.N > 61 else (128, 3)


def _schemes(args):
    """Default schemes: the N=40 workload runs the per-rate learned drift of its
    43->128x3->1 network; the N=120 workload runs its learned drift as the
    vector head 121->256x4->119 (one pass per path and step, the network's
    input being t and the 120 log-rates)."""
    if args.schemes:
        return [s for s in args.schemes.split(",") if s]
    return ["picard", "full", "mlp_vec"] if args.workload == "long_dated" else ["picard", "full", "mlp"]


def _train_flop(wl, hid, lay, head, n_params, epochs, batch, train_paths=1 << 16, records=8):
    """Floating-point operations of the GPU training run: Adam steps x rows x
    6 x (multiply-adds of the network) -- forward 2, backward 4 per weight
    (dX and dW); the library takes max(1, pairs / batch) steps per epoch, with
    pairs = records x (n + 1) / 2 per recorded step (per-rate head) or the
    records themselves (vector head)."""
    nrec = train_paths * records
    per_epoch = max(1, int((nrec if head else nrec * (wl.n + 1) / 2.0) // batch))
    return per_epoch * epochs * batch * 6.0 * n_params


def _code(s):
    """Library scheme of a bench scheme name ("mlp_vec": LLL_MLP with the vector-head network)."""
    return "mlp" if s == "mlp_vec" else s


def _describe(wl, schemes):
    return (f"{wl.name}: N={wl.N} (n={wl.n} rates) delta={wl.delta} s={wl.s} Q={wl.Q} "
            f"NIG({wl.alpha},{wl.beta},{wl.dbar}) {wl.paths} paths/GPU, "
            f"{wl.strikes.shape[1]} strikes/maturity, schemes={'+'.join(schemes)}")


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"lll_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for name, val in zip(names[1:], r[5:9]):
                if val.lower() in ("active", "0x1") or val == "1":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def _traffic(key):
    """DRAM bytes per launch from profiles/traffic.json, if the kernel's sources
    are unchanged since the counters were taken (else None)."""
    import hashlib
    try:
        entry = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[key]
        csrc = os.path.join(ROOT, "paper_1006_3340_gb300", "csrc")
        for fn, digest in entry["sources"].items():
            if hashlib.sha1(open(os.path.join(csrc, fn), "rb").read()).hexdigest() != digest:
                return None
        return entry["dram_bytes_read"] + entry["dram_bytes_write"]
    except Exception:
        return None


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def cpu_baseline(wl, schemes, budget_s=12.0, threads=None, mlp=None):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    batches of paths (the same global paths the GPU simulates first)
    alternating the quadrature schemes until the time budget is used, then a
    single-thread figure on a small batch, and (``mlp`` = (params, scales,
    head)) the FP64 oracle of the learned-compensator scheme on a few paths."""
    from oracle import oracle as ora
    from oracle import quadrature

    x, W = quadrature.rule_for(wl)
    model = ora.OracleModel(wl, x, W)
    threads = threads or os.cpu_count() or 1
    codes = {"picard": ora.PICARD, "full": ora.FULL, "frozen": ora.FROZEN}
    batch = 1024 if wl.N <= 61 else 128  # the N=120 oracle costs about 30x more per path
    done = {s: 0 for s in schemes if s in codes}
    secs = {s: 0.0 for s in done}
    t0 = time.perf_counter()
    while done:
        for s in done:
            t1 = time.perf_counter()
            ora.simulate(model, codes[s], path0=done[s], npaths=batch, threads=threads)
            secs[s] += time.perf_counter() - t1
            done[s] += batch
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    units = sum(done.values()) * wl.units_per_path()
    per = {s: done[s] * wl.units_per_path() / secs[s] for s in done}
    sample = ", ".join(f"{s}: paths 0..{done[s] - 1}" for s in done)
    out = {"value": units / dt, "unit": "path·tenor·steps/s", "cores": threads, "kind": "oracle",
           "sample": f"{wl.name} ({sample}); FP64 C oracle, {threads} threads, {dt:.1f} s",
           "per_scheme": per}
    # one thread, the first quadrature scheme, a small batch
    if done:
        s1 = next(iter(done))
        p1 = 64 if wl.N <= 61 else 8
        t1 = time.perf_counter()
        ora.simulate(model, codes[s1], path0=0, npaths=p1, threads=1)
        out["value_1_thread"] = p1 * wl.units_per_path() / (time.perf_counter() - t1)
        out["sample_1_thread"] = f"{s1}, paths 0..{p1 - 1}, 1 thread"
    if mlp is not None:
        from oracle import mlp as omlp
        params, scales, head = mlp
        pm = 64 if wl.N <= 61 else 4
        t1 = time.perf_counter()
        omlp.simulate_scheme(model, params, scales, npaths=pm, head=head)
        out["mlp_fp64"] = {"value": pm * wl.units_per_path() / (time.perf_counter() - t1),
                           "unit": "path·tenor·steps/s",
                           "sample": f"learned-compensator scheme (oracle/mlp.py, numpy FP64 matrix products "
                                     f"on the host's BLAS threads), paths 0..{pm - 1}"}
    return out


def run_reference(args):
    """The oracle as the reference arm: each step simulates a bounded sample of
    the workload per scheme on the host cores -- Picard and full with the C
    oracle, and (where the GPU arm runs it) the learned-compensator scheme with
    the FP64 network oracle on a seeded network of the benchmark's shape (its
    cost does not depend on the weights)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import mlp as omlp
    from oracle import oracle as ora
    from oracle import quadrature

    wl = _workload(args)
    schemes = _schemes(args)
    x, W = quadrature.rule_for(wl)
    model = ora.OracleModel(wl, x, W)
    threads = os.cpu_count() or 1
    codes = {"picard": ora.PICARD, "full": ora.FULL}
    per_step = args.ref_paths
    mlp_paths = max(per_step // 16, 8)
    hid, lay = _arch(wl)
    params = omlp.init_params([wl.N + 3] + [hid] * lay + [1], seed=3)
    scales = np.array([1.0 / (wl.n * wl.delta), 1.0 / wl.n, 5.0, 4.0, 1e-4])

    def step(k, scale=1):
        units = 0
        for s in schemes:
            if s in codes:
                npaths = max(per_step // scale, threads)
                ora.simulate(model, codes[s], path0=k * per_step, npaths=npaths, threads=threads)
            elif s == "mlp":
                npaths = max(mlp_paths // scale, 2)
                omlp.simulate_scheme(model, params, scales, path0=k * mlp_paths, npaths=npaths)
            else:
                continue
            units += npaths * wl.units_per_path()
        return units

    for w in range(args.warmup):
        step(0, scale=8)
    t0 = time.perf_counter()
    units = sum(step(k) for k in range(args.steps))
    dt = time.perf_counter() - t0
    val = units / dt
    unit = "path·tenor·steps/s"
    line = {"metric": METRIC, "value": val, "unit": unit, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": _describe(wl, schemes), "reference_sample_paths_per_scheme": per_step,
                       "reference_sample_paths_mlp": mlp_paths},
            "cpu_baseline": {"value": val, "unit": unit, "cores": threads, "kind": "oracle",
                             "sample": f"per step {per_step} paths per quadrature scheme (C oracle) and "
                                       f"{mlp_paths} paths of the learned scheme (numpy FP64) of {wl.name}"},
            "e2e": {"value": val, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args, steps, warmup, with_cpu=True, with_e2e=True, rates=None):
    """The batched configuration: 256 independent term structures of uneven tenor
    count, strike grid and path budget (2^24 paths in total) in one persistent
    launch per scheme, replayed as a CUDA graph.  One step = the Picard and the
    full scheme over every instance.  Single GPU.  Returns the JSON line."""
    import torch

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_1006_3340_gb300 import autotune, lll

    # --paths: the batch's total path budget (default 2^24; smaller totals are
    # for profiling captures, the instances' budgets scale along)
    wls = workloads.batched_instances(total_paths=(args.paths if args.workload == "batch256" else 0) or (1 << 24))
    schemes = [s for s in args.schemes.split(",") if s in ("picard", "full")] or ["picard", "full"]
    inst = []
    for wl in wls:
        x, W = lll.lll_build_nig_quadrature(wl.alpha, wl.beta, wl.dbar, wl.a, wl.Q)
        inst.append((wl, x, W))
    units = sum(wl.paths * wl.units_per_path() for wl in wls)          # per scheme
    lane_ops = sum(wl.paths * wl.units_per_path() * 3 * wl.Q for wl in wls)
    caplets = sum(wl.n * wl.strikes.shape[1] for wl in wls)
    b, keep = lll.lll_batch_init(inst)  # default stream, the one torch's events record on
    own = args.workload == "batch256"  # not the batch256 block of the default run
    if own and args.launch:  # threads,blocks_per_sm,chunk_rows[,paths_per_thread], both schemes
        shape = [int(v) for v in args.launch.split(",")][:4]
        lll.lll_batch_set_launch(b, *shape)
        tuned = {s: {"launch": shape, "ms": None, "tried": []} for s in schemes}
    elif own and args.no_tune:
        tuned = {s: {"launch": [0, 0, 0, 0], "ms": None, "tried": []} for s in schemes}
    else:  # each scheme its own launch shape
        tuned = {s: autotune.tune_batch(b, inst, s, repeats=1) for s in schemes}
    lll.lll_batch_use_graph(b, True)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def one_step(evs=None):
        for i, s in enumerate(schemes):
            if evs is not None:
                evs[i][0].record()
            lll.lll_batch_simulate(b, lll.SCHEMES[s], 42)
            if evs is not None:
                evs[i][1].record()

    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    per_ms = {s: [] for s in schemes}
    kernel_ms = {s: [] for s in schemes}
    torch.cuda.synchronize()
    for k in range(steps):
        flush.fill_(k & 0xFF)  # L2 flush between timed steps (outside the events)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in schemes]
        for i, s in enumerate(schemes):
            evs[i][0].record()
            lll.lll_batch_simulate(b, lll.SCHEMES[s], 42)
            evs[i][1].record()
            torch.cuda.synchronize()
            kernel_ms[s].append(lll.lll_batch_kernel_ms(b))
        for i, s in enumerate(schemes):
            per_ms[s].append(evs[i][0].elapsed_time(evs[i][1]))
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_ms = sum(sum(v) for v in per_ms.values())
    value = units * len(schemes) * steps / (total_ms * 1e-3)
    per = {}
    for s in schemes:
        ms = statistics.mean(per_ms[s])
        p0, _ = lll.lll_batch_prices(b, 0, wls[0].n, wls[0].strikes.shape[1])
        per[s] = {"units_per_s": units / (ms * 1e-3), "ms": ms, "batch_kernel_ms": statistics.mean(kernel_ms[s]),
                  "caplets_per_s": caplets / (ms * 1e-3), "inst0_atm_first_maturity": float(p0[0, 5])}
    pk = _alu_peaks(lll, torch, dev, rates)
    dom = max(schemes, key=lambda s: statistics.mean(kernel_ms[s]))
    ach = lane_ops / (statistics.mean(kernel_ms[dom]) * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": ach, "peak": pk["fp32"], "unit": "TFP32-lane-op/s",
                "frac": ach / pk["fp32"], "frac_of_nominal_128_lanes": ach / pk["fp32_nominal"], "traffic": None,
                "kernel": f"batch_kernel ({dom}), 3Q FP32 lane-ops per unit, Q=64",
                "peak_basis": pk["fp32_basis"]}

    # end to end through the C ABI from host arrays: batch init (instance inputs
    # host to device, FP64 tables), both schemes, every instance's prices back
    e2e = None
    if with_e2e:
        h2d = sum(wl.L0.nbytes + wl.lam.nbytes + x.nbytes + W.nbytes + wl.strikes.nbytes for wl, x, W in inst)
        d2h = len(schemes) * sum(2 * 8 * wl.n * wl.strikes.shape[1] for wl in wls)
        ts = []
        for _ in range(max(2, steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b2, keep2 = lll.lll_batch_init(inst)
            for s in schemes:
                lll.lll_batch_set_launch(b2, *tuned[s]["launch"], scheme=s)
            for s in schemes:
                lll.lll_batch_simulate(b2, lll.SCHEMES[s], 42)
                for q, wl in enumerate(wls):
                    lll.lll_batch_prices(b2, q, wl.n, wl.strikes.shape[1])
            lll.lll_batch_destroy(b2)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        et = statistics.mean(ts)
        e2e = {"value": units * len(schemes) / et, "unit": "path·tenor·steps/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "caplets_per_s": caplets * len(schemes) / et,
               "note": "lll_batch_init (tables built on the GPU) + lll_batch_simulate per scheme + "
                       "lll_batch_prices of every instance + lll_batch_destroy"}

    cpu = None
    if with_cpu:
        from oracle import oracle as ora
        from oracle import quadrature
        threads = os.cpu_count() or 1
        codes = {"picard": ora.PICARD, "full": ora.FULL}
        done_units, t0, q = 0, time.perf_counter(), 0
        while time.perf_counter() - t0 < 12.0 and q < len(wls):
            wl = wls[q]
            xq, Wq = quadrature.rule_for(wl)
            model = ora.OracleModel(wl, xq, Wq)
            npaths = min(wl.paths, 512)
            for s in schemes:
                ora.simulate(model, codes[s], npaths=npaths, threads=threads, seed=42, inst=q)
                done_units += npaths * wl.units_per_path()
            q += 1
        dt = time.perf_counter() - t0
        cpu = {"value": done_units / dt, "unit": "path·tenor·steps/s", "cores": threads, "kind": "oracle",
               "sample": f"instances 0..{q - 1}, first min(paths, 512) paths each, {'+'.join(schemes)}; "
                         f"FP64 C oracle, {threads} threads, {dt:.1f} s"}

    line = {"metric": METRIC, "value": value, "unit": "path·tenor·steps/s", "n_gpus": 1, "steps": steps,
            "warmup": warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batch256: {len(wls)} uneven term structures (N 8..80, delta 0.25/0.5), "
                                   f"{sum(wl.paths for wl in wls)} paths in total, 11 strikes, "
                                   f"schemes={'+'.join(schemes)}, one persistent launch per scheme (CUDA graph)",
                       "global_paths": sum(wl.paths for wl in wls), "parallelism": "one GPU",
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write outside the events)"},
            "per_scheme": per, "caplets_per_s": caplets * len(schemes) * steps / (total_ms * 1e-3),
            "roofline": roofline, "autotuned": tuned, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": 2 * len(schemes) * steps}
    lll.lll_batch_destroy(b)
    del flush
    torch.cuda.empty_cache()
    return line


def _alu_peaks(lll, torch, dev, rates=None):
    """Roofline denominators of the non-tensor kernels, from the pipe rates the
    library measures on this GPU (lll_measure_pipe_rates: results per SM per
    clock) times the SM count and the maximum SM clock of MEASURED_PEAKS."""
    rates = rates or lll.lll_measure_pipe_rates()
    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    f = sms * sm_max * 1e6 / 1e12
    return {"rates_per_sm_clock": rates, "sms": sms, "sm_max_mhz": sm_max,
            "fp32": rates["ffma2_lane_ops"] * f, "fp32_nominal": 128 * f,
            "fp32_basis": f"{sms} SMs x {rates['ffma2_lane_ops']:.1f} FP32 lane-ops/clk (packed FFMA2, measured "
                          f"in this run by lll_measure_pipe_rates) x {sm_max:.0f} MHz (sm_max_mhz of MEASURED_PEAKS)",
            "tanh": rates["tanh"] * f,
            "tanh_basis": f"{sms} SMs x {rates['tanh']:.1f} tanh.approx/clk (measured in this run by "
                          f"lll_measure_pipe_rates) x {sm_max:.0f} MHz"}


def run_single(args, wl, schemes, steps, warmup, dev, rank, world, local, with_cpu=True, with_e2e=True,
               rates=None, tune=True, tune_candidates=None, tune_repeats=2):
    """One term structure: every scheme simulates all paths of the workload per
    step.  Returns the JSON line (rank 0) or None."""
    import torch
    import torch.distributed as dist

    from paper_1006_3340_gb300 import lll

    hid, lay = _arch(wl)
    n, ns = wl.n, wl.strikes.shape[1]
    first = rank * wl.paths
    stream = torch.cuda.current_stream(dev).cuda_stream
    x, W = lll.lll_build_nig_quadrature(wl.alpha, wl.beta, wl.dbar, wl.a, wl.Q)
    sims = {s: lll.LevyLibor(wl, x, W, stream=stream) for s in schemes}
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    mlp_info = None
    mlp_params = None
    mlp_vec_params = None
    mlp_oracle = None
    if "mlp" in schemes:
        # The learned compensator is trained once, on its own paths (seed 7),
        # with the project's GPU kernels; the timed steps then price with it.
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("train")
        t0 = time.perf_counter()
        loss = lll.lll_mlp_train(sims["mlp"].ctx, hidden=hid, layers=lay, train_paths=1 << 16,
                                 records_per_path=8, epochs=4, batch=8192, lr=2e-3, lr_final=1e-4, seed=7)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        lll.lll_mlp_set_kernel(sims["mlp"].ctx, args.mlp_kernel)
        n_params, in_dim, in_pad, offs = lll.lll_mlp_layout(sims["mlp"].ctx, lay)
        mlp_params = lll.lll_mlp_params(sims["mlp"].ctx, 0, count=n_params)
        train_s = time.perf_counter() - t0
        tflop = _train_flop(wl, hid, lay, 0, n_params, 4, 8192)
        mlp_info = {"train_s": train_s, "final_loss_scaled": loss, "params": int(n_params),
                    "train_tflops": tflop / train_s / 1e12,
                    "train_tflops_frac": tflop / train_s / 1e12 / float(_peaks().get("bf16_tflops_sustained", 1679.9)),
                    "train_flop_basis": "Adam steps x 8192 rows x 6 x params over the whole lll_mlp_train call "
                                        "(data generation by the quadrature full scheme included); GEMMs on tcgen05",
                    "s_y": float(mlp_params[1][4]),
                    "arch": f"{in_dim}->{hid}x{lay}->1 SiLU, BF16 weights, FP32 accumulate",
                    "train_pairs": "2^16 paths x 8 recorded steps x live rates (~1e7)"}
        if with_cpu:
            from oracle import mlp as omlp
            mlp_oracle = (omlp.params_from_flat(mlp_params[0], offs, lay, hid, in_dim, in_pad), mlp_params[1], 0)

    vec_out = None
    if "mlp_vec" in schemes:
        # the vector-head network: one pass per path and step gives every rate's compensator
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("train_vec")
        t0 = time.perf_counter()
        ep_v = 40 if hid == 128 else 20
        lossv = lll.lll_mlp_train(sims["mlp_vec"].ctx, hidden=hid, layers=lay, train_paths=1 << 16,
                                  records_per_path=8, epochs=ep_v, batch=4096, lr=2e-3,
                                  lr_final=1e-4, seed=7, head=1)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        train_s_v = time.perf_counter() - t0
        # the mma.sync kernel has no vector head
        lll.lll_mlp_set_kernel(sims["mlp_vec"].ctx, "auto" if args.mlp_kernel == "warp" else args.mlp_kernel)
        nv, in_dim_v, in_pad_v, offs_v = lll.lll_mlp_layout(sims["mlp_vec"].ctx, lay)
        _, vec_out = lll.lll_mlp_shape(sims["mlp_vec"].ctx)
        mlp_vec_params = lll.lll_mlp_params(sims["mlp_vec"].ctx, 0, count=nv)
        tflop_v = _train_flop(wl, hid, lay, 1, nv, ep_v, 4096)
        mlp_info = dict(mlp_info or {}, vec={"train_s": train_s_v, "final_loss_scaled": lossv,
                                              "train_tflops": tflop_v / train_s_v / 1e12,
                                              "train_tflops_frac": tflop_v / train_s_v / 1e12 /
                                              float(_peaks().get("bf16_tflops_sustained", 1679.9)),
                                              "params": int(nv), "s_y": float(mlp_vec_params[1][4]),
                                              "arch": f"{in_dim_v}->{hid}x{lay}->{vec_out} SiLU (vector head), "
                                                      f"BF16, FP32 acc",
                                              "kernel": "tcgen05 vector-head kernel" if hid == 128 else
                                                        ("layered: tcgen05 GEMMs, layer by layer per Euler step"
                                                         if args.mlp_kernel == "layered" else
                                                         "fused 256-wide vector-head kernel (tcgen05 products, "
                                                         "weights streamed by TMA)")})
        if with_cpu and mlp_oracle is None:
            from oracle import mlp as omlp
            mlp_oracle = (omlp.params_from_flat(mlp_vec_params[0], offs_v, lay, hid, in_dim_v, in_pad_v,
                                                outputs=vec_out), mlp_vec_params[1], 1)

    def one_step(evs=None):
        for i, s in enumerate(schemes):
            if evs is not None:
                evs[i][0].record()
            lll.lll_simulate(sims[s].ctx, lll.SCHEMES[_code(s)], first, wl.paths, wl.seed)
            if evs is not None:
                evs[i][1].record()

    # launch shapes of the quadrature schemes by the project's autotuner
    from paper_1006_3340_gb300 import autotune
    tuned = {}
    if args.launch:
        shape = [int(v) for v in args.launch.split(",")]
        for s in schemes:
            if s in ("picard", "full", "frozen"):
                autotune.apply(sims[s], shape)
                tuned[s] = {"launch(threads,bps,chunk,ppt,lanes[,tenor])": shape, "ms": None}
    elif tune:
        # one lane per path (one or two paths per thread), lane pairs sharing a
        # path pair's nodes, and the tenor- and step-parallel mappings
        cands = tune_candidates or [(128, 0, 0, 1, 1), (256, 0, 0, 1, 1), (128, 0, 16, 1, 1), (128, 0, 0, 2, 1),
                                    (128, 0, 16, 2, 1), (128, 0, 0, 1, 2), (256, 0, 0, 1, 2), (0, 0, 0, 0, 0, 8),
                                    (0, 0, 0, 0, 0, 16), (0, 0, 0, 0, 0, -1)]
        for s in schemes:
            if s in ("picard", "full", "frozen"):
                r = autotune.tune(sims[s], s, candidates=cands, repeats=tune_repeats, use_cache=False)
                tuned[s] = {"launch(threads,bps,chunk,ppt,lanes[,tenor])": r["launch"], "ms": r["ms"]}

    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    per_scheme_ms = {s: [] for s in schemes}
    step_ms = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")  # profilers can select the timed launches
    for k in range(steps):
        flush.fill_(k & 0xFF)  # L2 flush between timed steps (outside the events)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in schemes]
        one_step(evs)
        torch.cuda.synchronize()
        tot = 0.0
        for i, s in enumerate(schemes):
            ms = evs[i][0].elapsed_time(evs[i][1])
            per_scheme_ms[s].append(ms)
            tot += ms
        step_ms.append(tot)
    torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()

    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    units_per_step = len(schemes) * wl.paths * wl.units_per_path() * world
    value = units_per_step * steps / (total_ms * 1e-3)

    # per-scheme throughput and caplet prices of the last step
    per = {}
    for s in schemes:
        ms = statistics.mean(per_scheme_ms[s])
        kms, _ = sims[s].kernel_ms()
        p, se = sims[s].prices()
        per[s] = {"units_per_s": wl.paths * wl.units_per_path() / (ms * 1e-3), "ms": ms,
                  "path_kernel_ms_last": kms, "atm_price_last_maturity": float(p[n - 1, ns // 2]),
                  # one simulation prices every (maturity, strike) caplet of the term structure
                  "caplets_per_s": n * ns / (ms * 1e-3)}
    if "picard" in per and "full" in per:
        pp, _ = sims["picard"].prices()
        pf, _ = sims["full"].prices()
        per["picard_vs_full_max_bp"] = float(np.abs(pp - pf).max() * 1e4)
    if world > 1 and "picard" in sims:
        # one gather of the FP64 payoff sums, added in rank order (outside the timing)
        from paper_1006_3340_gb300 import shard
        s1, s2, cnt = sims["picard"].sums()
        m1, m2, mcnt = shard.merge_sums(s1, s2, cnt)
        per["picard_merged_paths"] = mcnt
        per["picard_merged_atm_last_maturity"] = float(m1[n - 1, ns // 2] / mcnt)
    for s in ("mlp", "mlp_vec"):
        if s in per and "full" in per:
            pv, _ = sims[s].prices()
            pf, _ = sims["full"].prices()
            per[f"{s}_vs_full_max_bp"] = float(np.abs(pv - pf).max() * 1e4)

    # Rooflines.  Quadrature kernels: 3Q FP32 lane-ops per unit (one FMA into
    # A, one multiply w*E, one FMA into P) against the measured packed-FMA
    # rate.  MLP kernels: one tanh.approx per SiLU against the measured MUFU
    # rate (the binding pipe), with the tensor rate (2 x multiply-adds of the
    # network) beside it against the measured sustained BF16 rate.
    pk = _alu_peaks(lll, torch, dev, rates)
    peaks = _peaks()
    units = wl.paths * wl.units_per_path()

    def quad_roofline(s):
        ms = statistics.mean(per_scheme_ms[s])
        ach = units * 3 * wl.Q / (ms * 1e-3) / 1e12
        shape = tuned.get(s, {}).get("launch(threads,bps,chunk,ppt,lanes[,tenor])")
        lanes = shape[4] if shape and shape[4] else 1
        ppt = shape[3] if shape and shape[3] else 1
        tenor = shape[5] if shape and len(shape) > 5 else 0
        key = f"{s}/QP{wl.Q}/lanes{lanes}" + (f"/ppt{ppt}" if ppt > 1 else "")
        traffic = (_traffic(key) if wl.paths == 1 << 20 and not tenor else None)
        r = {"bound": "alu", "achieved": ach, "peak": pk["fp32"], "unit": "TFP32-lane-op/s",
             "frac": ach / pk["fp32"], "frac_of_nominal_128_lanes": ach / pk["fp32_nominal"], "traffic": traffic,
             "kernel": (f"{s} tenor-parallel kernel ({tenor} lanes per path), QP={wl.Q}" if tenor
                        else f"{s} path kernel, QP={wl.Q}"), "peak_basis": pk["fp32_basis"]}
        if clocks and clocks.get("sm_mhz"):
            r["frac_at_sampled_clock"] = r["frac"] * pk["sm_max_mhz"] / clocks["sm_mhz"]
        return r

    def mlp_roofline(s="mlp"):
        """The learned drift: the binding pipe is MUFU (one tanh per SiLU), the
        tensor pipe is reported beside it."""
        ms = statistics.mean(per_scheme_ms[s])
        t = ms * 1e-3
        if s == "mlp":
            in_pad = 16 * ((wl.N + 3 + 15) // 16)
            flop = units * 2 * (in_pad * hid + hid * hid * (lay - 1) + hid)  # per (path, rate, step) row
            silu = units * lay * hid
        else:
            # one pass per (path, step): input (t, u_0 .. u_{N-1}) padded to 16, the hidden
            # layers and the output layer of vec_out columns
            path_steps = wl.paths * wl.steps * world
            in_pad_v = 16 * ((wl.N + 1 + 15) // 16)
            flop = path_steps * 2 * (in_pad_v * hid + hid * hid * (lay - 1) + hid * vec_out)
            silu = path_steps * lay * hid
        tflops = flop / t / 1e12
        bf16 = float(peaks.get("bf16_tflops_sustained", 1679.9))
        ach = silu / t / 1e12
        key = "mlp/L3/KT3" if args.mlp_kernel == "warp" else "mlp_tc/L3/KB1"
        if s == "mlp_vec" and hid != 128 and args.mlp_kernel == "layered":
            # layer by layer: the GEMMs move every activation through HBM; the tensor
            # and MUFU rates are reported beside it
            return {"bound": "tensor", "pipe": "tcgen05 BF16 (layered GEMMs)", "achieved": tflops,
                    "peak": float(peaks.get("bf16_tflops_sustained", 1679.9)), "unit": "TFLOP/s",
                    "frac": tflops / float(peaks.get("bf16_tflops_sustained", 1679.9)),
                    "peak_basis": "bf16_tflops_sustained of MEASURED_PEAKS",
                    "tanh_per_s": ach, "tanh_frac": ach / pk["tanh"], "traffic": None,
                    "kernel": "mlp vector head, layered (tcgen05 GEMMs per Euler step)"}
        if s == "mlp_vec" and hid != 128:
            # one persistent kernel: one tanh per hidden activation on the MUFU pipe,
            # the products on tcgen05 beside it
            return {"bound": "alu", "pipe": "MUFU tanh.approx (SiLU)", "achieved": ach, "peak": pk["tanh"],
                    "unit": "T tanh/s", "frac": ach / pk["tanh"], "peak_basis": pk["tanh_basis"],
                    "tensor_tflops": tflops, "tensor_frac": tflops / bf16,
                    "tensor_peak_basis": "bf16_tflops_sustained of MEASURED_PEAKS",
                    "traffic": _traffic("mlp_wide/L4") if wl.paths == 1 << 22 else None,
                    "kernel": "mlp vector head, fused 256-wide (tcgen05, weights streamed by TMA)"}
        return {"bound": "alu", "pipe": "MUFU tanh.approx (SiLU)", "achieved": ach, "peak": pk["tanh"],
                "unit": "T tanh/s", "frac": ach / pk["tanh"], "peak_basis": pk["tanh_basis"],
                "tensor_tflops": tflops, "tensor_frac": tflops / bf16,
                "tensor_peak_basis": "bf16_tflops_sustained of MEASURED_PEAKS",
                "traffic": _traffic(key) if (s == "mlp" and wl.paths == 1 << 20) else None,
                "kernel": ("mlp layered path (training GEMMs)" if s == "mlp" and hid != 128 else
                           "mlp path kernel (mma.sync bf16)" if s == "mlp" and (args.mlp_kernel == "warp" or wl.N + 3 > 64)
                           else "mlp path kernel (tcgen05 bf16, TMEM accumulators)"
                           + (", vector head" if s == "mlp_vec" else ""))}

    dom = max(schemes, key=lambda s: statistics.mean(per_scheme_ms[s]))
    roofline = mlp_roofline(dom) if dom in ("mlp", "mlp_vec") else (quad_roofline(dom) if dom in ("picard", "full") else None)

    # end to end through the C ABI from host arrays: init (H2D of the model
    # inputs, FP64 tables on the GPU), strikes, each scheme, prices (D2H).
    e2e = None
    if with_e2e:
        h2d = (wl.L0.nbytes + wl.lam.nbytes + x.nbytes + W.nbytes) * len(schemes) + wl.strikes.nbytes * len(schemes)
        if mlp_params is not None:
            h2d += mlp_params[0].nbytes + mlp_params[1].nbytes
        if mlp_vec_params is not None:
            h2d += mlp_vec_params[0].nbytes + mlp_vec_params[1].nbytes
        d2h = len(schemes) * 2 * n * ns * 8
        ts = []
        for k in range(max(2, steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for s in schemes:
                sim = lll.LevyLibor(wl, x, W, stream=stream)
                if s in tuned:
                    autotune.apply(sim, tuned[s]["launch(threads,bps,chunk,ppt,lanes[,tenor])"])
                if s == "mlp":
                    lll.lll_mlp_init(sim.ctx, hid, lay, 0)
                    lll.lll_mlp_params(sim.ctx, 1, mlp_params[0], scales=mlp_params[1])
                    lll.lll_mlp_set_kernel(sim.ctx, args.mlp_kernel)
                if s == "mlp_vec":
                    lll.lll_mlp_init(sim.ctx, hid, lay, 0, head=1)
                    lll.lll_mlp_params(sim.ctx, 1, mlp_vec_params[0], scales=mlp_vec_params[1])
                lll.lll_simulate(sim.ctx, lll.SCHEMES[_code(s)], first, wl.paths, wl.seed)
                sim.prices()
                sim.close()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        et = statistics.mean(ts)
        if world > 1:
            t = torch.tensor([et], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            et = float(t.item())
        e2e = {"value": units_per_step / et, "unit": "path·tenor·steps/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "caplets_per_s": len(schemes) * n * ns * world / et,
               "note": "per scheme: lll_init + lll_set_strikes (+ network parameters for mlp) + lll_simulate + lll_price_caplets + lll_destroy"}

    cpu = None
    if rank == 0 and world == 1 and with_cpu:
        cpu = cpu_baseline(wl, schemes, mlp=mlp_oracle)

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "path·tenor·steps/s", "n_gpus": world,
                "steps": steps, "warmup": warmup, "ms_per_step": total_ms / steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": _describe(wl, schemes), "global_paths": wl.paths * world,
                           "parallelism": f"path shards x{world}", "l2": "flushed between timed steps "
                           f"({L2_FLUSH_BYTES >> 20} MiB write outside the events)"},
                "per_scheme": per, "roofline": roofline,
                "roofline_picard": quad_roofline("picard") if "picard" in schemes else None,
                "roofline_mlp": mlp_roofline("mlp") if "mlp" in schemes else None,
                "roofline_mlp_vec": mlp_roofline("mlp_vec") if "mlp_vec" in schemes else None,
                "measured_pipe_rates_per_sm_clock": pk["rates_per_sm_clock"],
                "mlp": mlp_info, "autotuned": tuned, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clocks, "gpu_launches": 2 * len(schemes) * steps}
    for s in sims.values():
        s.close()
    del flush
    torch.cuda.empty_cache()
    return line


def run_mappings(args, rates=None):
    """Path mapping against the tenor-parallel mapping: device time of one
    simulation of the N=40 term structure (full and Picard) at 2^20 paths and
    at 2^12 paths, for one lane per path (128 and 256 threads per block) and
    for 4, 8, 16 and 32 lanes per path; each with its fraction of the FP32
    roofline (3Q lane-ops per unit against the measured packed-FMA rate).
    --paths and --schemes narrow it to one size and a scheme (for a launch
    list).  Returns the JSON line."""
    import torch

    from paper_1006_3340_gb300 import autotune, lll

    dev = torch.device("cuda", 0)
    pk = _alu_peaks(lll, torch, dev, rates)
    shapes = [("path, 128 threads", (128, 0, 0, 1, 1)), ("path, 256 threads", (256, 0, 0, 1, 1)),
              ("path, 2 paths/thread", (128, 0, 0, 2, 1))] + \
             [(f"tenor, {g} lanes/path", (0, 0, 0, 0, 0, g)) for g in (4, 8, 16, 32)] + \
             [("step-parallel (Picard)", (0, 0, 0, 0, 0, -1))]
    rows = []
    sizes = (args.paths,) if args.paths else (1 << 20, 1 << 12)
    schemes = [s for s in args.schemes.split(",") if s in ("picard", "full")] or ["picard", "full"]
    for paths in sizes:
        wl = workloads.large_single(paths=paths)
        x, W = lll.lll_build_nig_quadrature(wl.alpha, wl.beta, wl.dbar, wl.a, wl.Q)
        sim = lll.LevyLibor(wl, x, W)
        try:
            for scheme in schemes:
                for name, cand in shapes:
                    if scheme == "full" and len(cand) > 5 and cand[5] < 0:
                        continue  # the full scheme's steps are sequential
                    autotune.apply(sim, cand)
                    sim.simulate(scheme)  # warm-up
                    ms = []
                    for _ in range(max(3, args.steps)):
                        sim.simulate(scheme)
                        ms.append(sim.kernel_ms()[0])
                    t = statistics.median(ms)
                    ach = paths * wl.units_per_path() * 3 * wl.Q / (t * 1e-3) / 1e12
                    rows.append({"paths": paths, "scheme": scheme, "mapping": name, "kernel_ms": t,
                                 "units_per_s": paths * wl.units_per_path() / (t * 1e-3),
                                 "fp32_frac": ach / pk["fp32"]})
        finally:
            sim.close()
    return {"metric": "path-kernel device time per mapping", "workload": "large_single (N=40, Q=64)",
            "fp32_peak_basis": pk["fp32_basis"], "rows": rows}


def run_by_length(args, rates=None):
    """Single term structures of the 256-instance recipe, one per tenor count
    N = 8 .. 80 (the first instance of the recipe with that N, or the nearest),
    2^20 paths each, on the batch's launch shape (128 threads, one lane per
    path, 16-row chunks): device time of the path kernel per scheme, the
    throughput in path-rate-steps per second and the fraction of the FP32
    roofline.  Short term structures do less rate work per step, so the work
    every step and every maturity does once weighs more; the batch's cost
    model for work items carries that as a per-step term.  Returns the JSON
    line."""
    import dataclasses

    import torch

    from paper_1006_3340_gb300 import lll

    dev = torch.device("cuda", 0)
    pk = _alu_peaks(lll, torch, dev, rates)
    paths = args.paths or (1 << 20)
    insts = workloads.batched_instances()
    by_n = {}
    for wl in insts:
        by_n.setdefault(wl.N, wl)
    rows = []
    for N in (8, 12, 16, 24, 32, 40, 48, 56, 64, 72, 80):
        wl = dataclasses.replace(by_n[min(by_n, key=lambda v: abs(v - N))], paths=paths)
        x, W = lll.lll_build_nig_quadrature(wl.alpha, wl.beta, wl.dbar, wl.a, wl.Q)
        sim = lll.LevyLibor(wl, x, W)
        try:
            sim.set_launch(128, 0, 16, 1, 1)
            row = {"N": wl.N, "steps": wl.steps, "units_per_path": wl.units_per_path()}
            for scheme in ("picard", "full"):
                sim.simulate(scheme)  # warm-up
                ms = []
                for _ in range(max(3, args.steps)):
                    sim.simulate(scheme)
                    ms.append(sim.kernel_ms()[0])
                t = statistics.median(ms)
                ach = paths * wl.units_per_path() * 3 * wl.Q / (t * 1e-3) / 1e12
                row[scheme] = {"kernel_ms": t, "units_per_s": paths * wl.units_per_path() / (t * 1e-3),
                               "fp32_frac": ach / pk["fp32"]}
            rows.append(row)
        finally:
            sim.close()
    return {"metric": "path-kernel device time per tenor count", "workload": f"batch256 recipe, {paths} paths each",
            "launch": "128 threads, one lane per path, 16-row chunks", "fp32_peak_basis": pk["fp32_basis"],
            "rows": rows}


def _extra_block(line):
    """The figures of another configuration kept in the headline line."""
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "config", "per_scheme", "caplets_per_s",
            "roofline", "roofline_picard", "roofline_mlp", "roofline_mlp_vec", "autotuned", "clocks", "mlp")
    return {k: line[k] for k in keep if k in line}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--paths", type=int, default=0, help="paths per GPU (default 2^20)")
    ap.add_argument("--ref-paths", type=int, default=512, help="oracle paths per scheme per step")
    ap.add_argument("--schemes", default="", help="default picard,full,mlp (large_single), picard,full (long_dated)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="library default launch shapes")
    ap.add_argument("--no-extra", action="store_true",
                    help="default run: leave out the batch256 and long_dated blocks")
    ap.add_argument("--mlp-kernel", default="auto", choices=["auto", "warp", "tc", "layered"],
                    help="LLL_MLP kernel: tcgen05/TMEM (tc), mma.sync (warp), layer by layer (layered) or the library's choice")
    ap.add_argument("--launch", default="", help="fixed launch shape for the quadrature schemes: "
                    "threads,blocks_per_sm,chunk_rows,paths_per_thread,lanes_per_path[,tenor_lanes] (no tuning)")
    ap.add_argument("--workload", default="large_single",
                    choices=["large_single", "long_dated", "batch256", "mappings", "by_length"],
                    help="large_single: the N=40 term structure, 2^20 paths (default); long_dated: N=120, "
                    "Q=96, 2^22 paths; batch256: 256 uneven term structures in one launch per scheme "
                    "(Picard and full only); mappings: path against tenor-parallel mapping, N=40, "
                    "2^20 and 2^12 paths (a table, not a benchmark line); by_length: single term "
                    "structures of the batch256 recipe, N = 8..80, 2^20 paths each (a table)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload == "batch256" and world > 1:
        print(json.dumps({"error": "--workload batch256 runs on one GPU"}), flush=True)
        return 1
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1006_3340_gb300 import build as libbuild
    libbuild.build()
    from paper_1006_3340_gb300 import lll

    rates = lll.lll_measure_pipe_rates()
    if args.workload == "mappings":
        print(json.dumps(run_mappings(args, rates)), flush=True)
        return 0
    if args.workload == "by_length":
        print(json.dumps(run_by_length(args, rates)), flush=True)
        return 0
    if args.workload == "batch256":
        line = run_batch(args, args.steps, args.warmup, not args.no_cpu_baseline, not args.no_e2e, rates)
    else:
        wl = _workload(args)
        line = run_single(args, wl, _schemes(args), args.steps, args.warmup, dev, rank, world, local,
                          with_cpu=not args.no_cpu_baseline, with_e2e=not args.no_e2e, rates=rates,
                          tune=not args.no_tune)
        if (line is not None and world == 1 and args.workload == "large_single" and not args.no_extra
                and not args.paths):
            # the other single-GPU configurations, a few steps each, in the same line
            extra = {"batch256": _extra_block(run_batch(args, 2, 1, False, False, rates))}
            wl5 = workloads.long_dated()
            # two one-lane shapes (a launch of this workload takes about 1.7 s)
            extra["long_dated"] = _extra_block(run_single(
                args, wl5, ["picard", "full", "mlp_vec"], 2, 1, dev, rank, world, local, with_cpu=False,
                with_e2e=False, rates=rates, tune=True, tune_candidates=[(128, 0, 0, 1, 1), (256, 0, 0, 1, 1)],
                tune_repeats=1))
            line["extra_configs"] = extra
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
