#!/usr/bin/env python3
"""Benchmark: effective kernel evaluations per second (M*N*#h / wall time) of
the epsilon-relative Gaussian summation on the D=3 bandwidth-sweep workload
(1e6 monochromatic FP32 points from a 16-component anisotropic mixture plus 5%
uniform background, 16 log-spaced bandwidths from 1e-3 to 1 times the data
diameter, eps = 1e-2).

One step = one pass of the whole path over the workload, inputs resident in
HBM: `--mode lscv` (default) runs gs_lscv -- the dual-tree sums for all 16
bandwidths h and their sqrt(2) h companions (32 Gaussian sums: tree build,
frontier, series, base case, downward pass) and the LSCV reduction;
`--mode sum` runs gs_sum over the 16 bandwidths only; `--eps 0` selects the
exhaustive sums instead of the dual tree; `--mode batch` runs gs_sum_batched
over 256 independent KDE problems (N = M log-uniform in [1e3, 2e5], D in
2..8, 8 bandwidths each, eps = 1e-2).  The L2 cache is flushed before every
timed step (inputs are 12 MB, smaller than L2).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded query sample of the same workload instead.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "effective kernel evals/s (M*N*#h / wall time) at rel. err eps vs GPU exhaustive"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gs", choices=["gs", "reference"])
    ap.add_argument("--mode", default="lscv", choices=["lscv", "sum", "batch", "search"])
    ap.add_argument("--selector", default="rule", choices=["rule", "mlp", "fd_only"],
                    help="pair selector: Fig. 6's rule, the stored learned network, or FD pruning only "
                         "(the paper's DFD/DFDO comparison: no series approximations)")
    ap.add_argument("--best-first", action="store_true",
                    help="ablation: best-first look-ahead of each group's largest bound gaps (GS_FLAG_BEST_FIRST)")
    ap.add_argument("--no-tokens", action="store_true",
                    help="Theorem 2 without the token scheme (each pair within its own W_R share)")
    ap.add_argument("--count", type=int, default=256, help="problems in --mode batch")
    ap.add_argument("--workers", type=int, default=16, help="concurrent problems in --mode batch")
    ap.add_argument("--small-work", type=float, default=0.0,
                    help="--mode batch: problems with M N nh at most this are summed exhaustively "
                         "(0: the library's GS_SMALL_WORK)")
    ap.add_argument("--no-small-exhaustive", action="store_true",
                    help="--mode batch: dual tree even for problems whose exact sum is cheaper")
    ap.add_argument("--eps", type=float, default=None, help="override eps (0 = exhaustive)")
    ap.add_argument("--scale", type=float, default=1.0, help="workload size factor (1 = full)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (library defaults)")
    ap.add_argument("--leaf", type=int, default=0, help="fixed leaf size (skips the autotuner)")
    ap.add_argument("--cost", default="", help="fixed cost weights c_DH,c_DL,c_H2L,c_Direct (skips the autotuner)")
    ap.add_argument("--plimit", type=int, default=0, help="fixed highest series order PLIMIT (with --leaf/--cost; "
                                                           "0: the Section 6 table)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the accuracy check after the timed steps (every result against the GPU "
                         "exhaustive sum)")
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4],
                    help="workload for --mode sum: 1 (D=2, 1e4), 2 (D=3 sweep, 1e6), 3 (D=5, 5e5, eps 1e-3), "
                         "4 (D=16 bichromatic, 2e6 refs x 2e5 queries)")
    return ap.parse_args()


def workload(scale, config=2):
    from workloads import synth
    return {1: synth.config1, 2: synth.config2, 3: synth.config3, 4: synth.config4}[config](scale)


SEARCH_ROUNDS, SEARCH_PER_ROUND = 4, 8   # --mode search: 32 LSCV scores per search
CERTIFY_STEPS = 2                        # re-scorings of the last grid at eps/4, eps/16 to certify h*


def sum_bandwidths(wl, mode):
    """Bandwidths one step sums over: the sweep, plus sqrt(2) h for LSCV;
    for a bandwidth search, the 2 x 32 sums of its scores (their bandwidths
    are chosen as it goes; the sweep's own set stands in for tuning)."""
    from workloads import synth
    if mode == "search":
        return np.resize(synth.lscv_bandwidths(wl.h), 2 * SEARCH_ROUNDS * SEARCH_PER_ROUND)
    return synth.lscv_bandwidths(wl.h) if mode == "lscv" else wl.h


def wl_config(wl, mode, eps):
    name = "kde_sweep_d3_n%d_mono_16h" % wl.N if wl.D == 3 and wl.mono and wl.h.size == 16 else wl.name
    return {"workload": name, "M": wl.M, "N": wl.N, "D": wl.D,
            "nh": int(wl.h.size), "gaussian_sums": int(sum_bandwidths(wl, mode).size), "eps": eps,
            "mode": mode, "leaf_size": wl.leaf_size,
            "h_range_x_diameter": [1e-3, 1.0], "diameter": round(wl.diameter, 6),
            "input_dtype": "f32" if wl.refs.dtype == np.float32 else "f64",
            "l2": "flushed before every timed step (256 MB write)",
            "parallelism": "replicas"}


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id):
        self.bus_id = (bus_id or "").lower()
        self.path = os.path.join(tempfile.gettempdir(), "gs_clocks_%d.csv" % os.getpid())
        self.proc = None

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if self.bus_id:
            mine = [r for r in rows if self.bus_id.endswith(r[1].lower()[-12:]) or r[1].lower().endswith(self.bus_id[-12:])]
            rows = mine or rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[6 + k] and "Not" not in r[6 + k]})
        load = [s for s in sm if mx and s >= 0.5 * max(mx)] or sm
        return {"sm_mhz": float(np.median(load)) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on a bounded sample
# ---------------------------------------------------------------------------
def oracle_sample_rate(wl, nq, hs, seed=0, idx=None):
    """The FP64 oracle timed on nq queries (seeded, or the given indices)
    against every reference and bandwidth; returns (evals/s, seconds,
    threads, the oracle's sums, the query indices)."""
    from oracle import exhaustive as oracle_ex
    if idx is None:
        rng = np.random.default_rng(seed)
        idx = np.sort(rng.choice(wl.M, nq, replace=False))
    t0 = time.perf_counter()
    exact = oracle_ex.gauss_sum(wl.queries[idx], wl.refs, wl.weights, hs)
    dt = time.perf_counter() - t0
    return idx.size * wl.N * hs.size / dt, dt, oracle_ex.num_threads(), exact, idx


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload(args.scale, args.config)
    from oracle import build as ob
    ob.build()
    hs = sum_bandwidths(wl, args.mode)
    nq = max(1, int(100 * min(1.0, 1.0 / args.scale)))   # ~3e9 evals per step at full size
    for _ in range(args.warmup):
        oracle_sample_rate(wl, max(1, nq // 8), hs, seed=99)
    rates, secs = [], []
    for k in range(args.steps):
        r, dt, cores, _, _ = oracle_sample_rate(wl, nq, hs, seed=k)
        rates.append(r)
        secs.append(dt)
    value = float(np.mean(rates))
    sample = "%d seeded queries x all %d refs x %d bandwidths per step" % (nq, wl.N, hs.size)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": wl_config(wl, "oracle_exhaustive", 0.0),
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
# sources of each kernel whose DRAM traffic profiles/traffic.json records
KERNEL_SOURCES = {"k_basecase": ("gs_basemerge.cu", "gs_device.cuh"),
                  "k_basecase_tc": ("gs_basetc.cu", "gs_tc.cuh", "gs_device.cuh"),
                  "k_exhaustive": ("gs_exhaustive.cu", "gs_device.cuh")}


def source_sha(kernel):
    """Hash of the kernel's source files: a recorded traffic figure is used
    only while the kernel is unchanged since its counters were taken."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1206_6857_gb300", "csrc")
    for f in KERNEL_SOURCES.get(kernel, ()):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(kernel, sha, workload, terms):
    """DRAM bytes of one launch of this kernel with `terms` base-case terms:
    the bytes per term recorded on a smaller launch of the same workload
    (records come from L2; the bytes grow with the terms), if the kernel's
    sources are unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    e = d.get(kernel)
    if e and e.get("src_sha") == sha and e.get("workload") == workload and e.get("bytes_per_term"):
        return int(round(e["bytes_per_term"] * terms))
    return None


class Replicas:
    """Process-group plumbing of an N-GPU run.  The path does not shard, so
    every rank runs the whole step on its own copy of the workload (replicas):
    a barrier on both sides of the timed region, the slowest rank's time, and
    the whole job's throughput = the units all ranks processed over that time.
    backend "nccl" (GPU ranks) or "gloo" (the CPU tests)."""

    def __init__(self, backend="nccl", device=None):
        import torch.distributed as dist
        self.dist = dist
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.device = device
        if self.world > 1:
            if backend == "nccl":
                dist.init_process_group("nccl", device_id=device)
            else:
                dist.init_process_group(backend)

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def max_ms(self, ms):
        """The largest of the ranks' step times."""
        if self.world == 1:
            return float(ms)
        import torch
        t = torch.tensor([float(ms)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def throughput(self, units_per_rank, ms):
        """Whole-job units per second: every rank processed units_per_rank."""
        return units_per_rank * self.world / (ms / 1e3)

    def close(self):
        if self.world > 1:
            self.dist.destroy_process_group()


def run_gs(args):
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    reps = Replicas("nccl", torch.device("cuda", local))
    world, rank = reps.world, reps.rank

    from paper_1206_6857_gb300 import build as gbuild
    from paper_1206_6857_gb300 import gs
    if rank == 0:
        gbuild.build()
    reps.barrier()
    gs.load()

    wl = workload(args.scale, args.config)
    if not wl.mono and args.mode == "lscv":
        args.mode = "sum"                 # LSCV needs monochromatic data
    eps = wl.eps if args.eps is None else args.eps
    hs = sum_bandwidths(wl, args.mode)
    dev = torch.device("cuda", local)
    tq = torch.from_numpy(wl.queries).to(dev)
    tr = tq if wl.mono else torch.from_numpy(wl.refs).to(dev)
    tw = torch.from_numpy(wl.weights).to(dev)
    out = torch.empty((wl.M, wl.h.size), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    scores = {}

    # autotuner (setup, not timed): leaf size, PLIMIT and bestMethod cost
    # weights chosen by timing the library on the data with every bandwidth
    # of the step
    tuned, opts = None, None
    if args.leaf or args.cost:
        from paper_1206_6857_gb300 import autotune
        cw = [float(v) for v in args.cost.split(",")] if args.cost else list(gs.GS_COST_DEFAULT)
        tuned = {"leaf_size": args.leaf or 32, "plimit": args.plimit, "cost_weight": cw, "fixed": True}
        opts = autotune.options(tuned)
    elif eps > 0 and not args.no_tune:
        from paper_1206_6857_gb300 import autotune
        t0 = time.perf_counter()
        # every bandwidth of the step: the merged base case handles them in
        # blocks of 8, so a subset would favour the wrong leaf size
        # (a search repeats the sweep's bandwidths: tune on the distinct ones)
        tuned, _table = autotune.tune_staged(tr, tw, np.unique(hs), eps, wl.D, h_subset=0,
                                             queries=None if wl.mono else tq)
        tuned["tuning_seconds"] = time.perf_counter() - t0
        tuned["candidates"] = [[r["leaf_size"], r["plimit"]] + list(r["cost_weight"]) +
                               [round(r["seconds"] * 1e3, 1) if r["seconds"] != float("inf") else "out of memory"]
                               for r in _table]     # leaf, PLIMIT, c_DH, c_DL, c_H2L, c_Direct, ms
        opts = autotune.options(tuned)

    opts, _sel_params = selector_opts(args, opts)
    if tuned is not None:
        tuned["selector"] = args.selector
        tuned["tokens"] = not args.no_tokens
        tuned["best_first"] = bool(args.best_first)

    def step(stats=None):
        if args.mode == "search":
            # the LSCV-optimal bandwidth over the sweep's range: tree built once,
            # SEARCH_ROUNDS calls of SEARCH_PER_ROUND scores each
            from paper_1206_6857_gb300 import lscv_search
            r = lscv_search.minimize(tq, tw, eps, float(wl.h[0]), float(wl.h[-1]), rounds=SEARCH_ROUNDS,
                                     per_round=SEARCH_PER_ROUND, opts=opts, stream=stream, stats=stats,
                                     certify_steps=CERTIFY_STEPS)
            scores["search"] = r[:3] + (r[4],)
        elif args.mode == "lscv":
            scores["lscv"] = gs.gs_lscv(tq, tw, wl.h, eps, opts=opts, stream=stream, stats=stats)
        else:
            gs.gs_sum(tq, tr, tw, wl.h, eps, out=out, opts=opts, stream=stream, stats=stats)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(dev)
    bus = getattr(props, "pci_bus_id", None)
    sampler = ClockSampler(bus)
    sampler.start()
    time.sleep(0.3)
    evs = []
    stats_list = []
    reps.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.fill_(1)
        st = gs.gs_stats()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(st)
        e1.record(stream)
        evs.append((e0, e1))
        stats_list.append(st)
    torch.cuda.synchronize()
    reps.barrier()
    clocks = sampler.stop()
    ms = reps.max_ms(float(sum(a.elapsed_time(b) for a, b in evs)) / args.steps)

    units = float(wl.M) * wl.N * hs.size            # kernel evaluations one step stands for
    value = reps.throughput(units, ms)
    # the dominant kernel: of the base case's kernels (the tensor-core one,
    # the direct one; each timed by CUDA events around its launch on the
    # library's stream) the one that summed more terms; the exhaustive kernel
    # for eps = 0 (its phase holds that one launch)
    all_terms = float(np.mean([s.point_pairs_base for s in stats_list]))
    tc_terms = float(np.mean([s.point_pairs_tc for s in stats_list]))
    use_tc = tc_terms > 0.5 * all_terms
    if eps == 0.0:
        base_ms = float(np.mean([s.ms_phase[gs.GS_PH_BASE] / max(1, s.launches_base) for s in stats_list]))
        evals_base = float(np.mean([s.point_pairs_base / max(1, s.launches_base) for s in stats_list]))
    elif use_tc:
        base_ms = float(np.mean([s.ms_base_kernels[0] for s in stats_list]))
        evals_base = tc_terms
    else:
        base_ms = float(np.mean([s.ms_base_kernels[1] for s in stats_list]))
        evals_base = all_terms - tc_terms
    launches = int(np.mean([s.launches for s in stats_list]))

    # roofline: the base-case / exhaustive kernel is bound by the MUFU ex2 rate
    # (one ex2 per term); peak = measured ex2 lanes/SM/clk x SMs x SM clock
    ex2_rate, ffma_rate = gs.gs_probe_rates()
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    peak = ex2_rate * props.multi_processor_count * sm_mhz * 1e6 / 1e12
    achieved = evals_base / (base_ms / 1e3) / 1e12 if base_ms > 0 else None
    kname = "k_exhaustive" if eps == 0.0 else ("k_basecase_tc" if use_tc else "k_basecase")
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tex2/s",
            "frac": achieved / peak if (peak and achieved) else None,
            "traffic": load_traffic(kname, source_sha(kname), "%s/%s/scale%g/leaf%d" % (
                wl_config(wl, args.mode, eps)["workload"], args.mode, args.scale,
                (tuned or {}).get("leaf_size", wl.leaf_size)), evals_base),
            "kernel": kname, "peak_basis": "measured %.1f ex2 lanes/SM/clk x %d SMs x %.0f MHz (median SM clock under load)"
            % (ex2_rate, props.multi_processor_count, sm_mhz),
            "ffma_lanes_per_sm_clk": ffma_rate, "kernel_ms_per_launch": base_ms}

    # end to end: inputs start in pinned host memory and the step's result
    # comes back to the host, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        hq = torch.from_numpy(wl.queries).pin_memory()
        hw = torch.from_numpy(wl.weights).pin_memory()
        n_e2e = max(1, min(args.steps, 3))
        if args.mode == "search":
            from paper_1206_6857_gb300 import lscv_search

            def e2e_step():
                dq = hq.to(dev, non_blocking=True)
                dw = hw.to(dev, non_blocking=True)
                return lscv_search.minimize(dq, dw, eps, float(wl.h[0]), float(wl.h[-1]), rounds=SEARCH_ROUNDS,
                                            per_round=SEARCH_PER_ROUND, opts=opts, stream=stream,
                                            certify_steps=CERTIFY_STEPS)
            d2h = 2 * 8 * SEARCH_ROUNDS * SEARCH_PER_ROUND
        elif args.mode == "lscv":
            hqn_l, hwn_l = hq.numpy(), hw.numpy()

            def e2e_step():
                # host buffers through the C ABI: the library copies them in
                return gs.gs_lscv_host(hqn_l, hwn_l, wl.h, eps, opts=opts)
            d2h = 2 * 8 * wl.h.size
        else:
            hout = torch.empty((wl.M, wl.h.size), dtype=torch.float64).pin_memory().numpy()

            hqn = hq.numpy()
            hrn = hqn if wl.mono else torch.from_numpy(wl.refs).pin_memory().numpy()   # same object: monochromatic

            def e2e_step():
                gs.gs_sum_host(hqn, hrn, hw.numpy(), wl.h, eps, out=hout, opts=opts)
            d2h = int(hout.nbytes)
        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / n_e2e
        h2d = int(hq.numel() * hq.element_size() + hw.numel() * 4 + (0 if wl.mono else wl.refs.nbytes))
        e2e = {"value": units / dt, "unit": "evals/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3}

    # accuracy of the step's results (after the timed region): every result
    # against the GPU exhaustive sum, and -- in the CPU baseline leg below --
    # a sample that includes the smallest sums against the FP64 oracle
    acc, dt_all, ex_all = None, None, None
    if rank == 0 and args.mode in ("lscv", "sum") and not args.no_accuracy:
        W = float(wl.weights.astype(np.float64).sum())
        floor = 2.0 ** -40 * W
        ex_all = gs.gs_sum(tq, tr, tw, hs, 0.0, stream=stream).cpu().numpy()
        acc = {"floor": "2^-40 W", "results": int(ex_all.size),
               "under_floor": int(np.sum(ex_all < floor))}
        if eps > 0:
            dt_all = gs.gs_sum(tq, tr, tw, hs, eps, opts=opts, stream=stream).cpu().numpy()
            err = np.abs(dt_all - ex_all) / np.maximum(ex_all, floor)
            acc["max_rel_err_vs_gpu_exhaustive"] = float(err.max())
            acc["eps"] = eps
            acc["within_eps"] = bool(err.max() <= eps)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        from oracle import build as ob
        ob.build()
        # a bounded sample: about 4e10 kernel evaluations (10-30 s on the
        # host cores), whatever the workload's N and number of sums; it holds
        # the 64 queries with the smallest sums (a few per bandwidth, chosen
        # from the GPU exhaustive output), where the relative guarantee is
        # hardest, and seeded queries for the rest
        nq = int(min(wl.M, max(80, round(4e10 / (float(wl.N) * hs.size)))))
        pick = np.zeros(0, np.int64)
        if ex_all is not None:
            per_h = max(1, -(-64 // hs.size))
            pick = np.unique(np.concatenate([np.argsort(ex_all[:, j], kind="stable")[:per_h]
                                             for j in range(hs.size)]))[:64]
        rest = np.setdiff1d(np.random.default_rng(0).choice(wl.M, nq, replace=False), pick)[:max(0, nq - pick.size)]
        idx = np.sort(np.concatenate([pick, rest]).astype(np.int64))
        r, secs, cores, exact, idx = oracle_sample_rate(wl, idx.size, hs, idx=idx)
        cpu = {"value": r, "unit": "evals/s", "cores": cores, "kind": "oracle",
               "sample": "%d queries (%d with the smallest GPU-exhaustive sums, %d seeded) x all %d refs x %d "
                         "bandwidths (%.1f s)" % (idx.size, pick.size, idx.size - pick.size, wl.N, hs.size, secs)}
        if acc is not None:
            W = float(wl.weights.astype(np.float64).sum())
            den = np.maximum(exact, 2.0 ** -40 * W)
            acc["oracle_sample"] = "the %d queries of cpu_baseline x %d bandwidths" % (idx.size, hs.size)
            acc["fp32_err_exhaustive_vs_oracle"] = float((np.abs(ex_all[idx] - exact) / den).max())
            if dt_all is not None:
                acc["max_rel_err_vs_oracle"] = float((np.abs(dt_all[idx] - exact) / den).max())
                sel = np.isin(idx, pick)
                acc["max_rel_err_vs_oracle_smallest_sums"] = (
                    float((np.abs(dt_all[idx[sel]] - exact[sel]) / den[sel]).max()) if sel.any() else None)

    if rank == 0:
        s0 = stats_list[-1]
        cfg = wl_config(wl, args.mode, eps)
        if tuned is not None:
            cfg["tuned"] = tuned
        line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": cfg, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clocks, "gpu_launches": launches * args.steps,
                "accuracy": acc,
                "units": "M*N*%d kernel evaluations per step: %s" % (
                    hs.size, "the %d sweep bandwidths and their sqrt(2) h companions, all summed in the step"
                    % wl.h.size if args.mode == "lscv" else "every bandwidth summed in the step"),
                "stats": {k: v for k, v in s0.as_dict().items()}}
        if args.mode == "lscv":
            line["value_per_sweep_bandwidth"] = float(wl.M) * wl.N * wl.h.size / (ms / 1e3) * world
        if "search" in scores:
            hb, sb, eb, cert = scores["search"]
            line["search"] = {"h_best": hb, "score": sb, "err_bound": eb, "rounds": SEARCH_ROUNDS,
                              "per_round": SEARCH_PER_ROUND, "range": [float(wl.h[0]), float(wl.h[-1])],
                              "certified": cert["certified"], "certified_bracket": cert["bracket"],
                              "certifying_eps": cert["eps"], "certified_neighbour_distance": cert["m"],
                              "certified_grid_round": cert.get("grid_round"),
                              "note": "roofline and stats of the search's last call"}
        if "lscv" in scores:
            sc, er = scores["lscv"]
            k = int(np.argmin(sc))
            sep = all(sc[k] + er[k] < sc[i] - er[i] for i in (k - 1, k + 1) if 0 <= i < sc.size)
            line["lscv"] = {"h": [float(v) for v in wl.h], "score": [float(v) for v in sc],
                            "err_bound": [float(v) for v in er], "argmin_h": float(wl.h[k]),
                            "argmin_separated_from_grid_neighbours": bool(sep)}
        print(json.dumps(line), flush=True)
    reps.close()


def selector_opts(args, opts):
    """Options for --selector (the stored learned network for mlp, FD
    pruning only for fd_only) and --no-tokens."""
    from paper_1206_6857_gb300 import gs
    if args.selector == "rule" and not args.no_tokens and not args.best_first:
        return opts, None
    o = opts if opts is not None else gs.gs_opts_default()
    if args.best_first:
        o.flags |= gs.GS_FLAG_BEST_FIRST
    if args.no_tokens:
        o.no_tokens = 1
    if args.selector == "fd_only":
        o.selector = gs.GS_SEL_FD_ONLY
    if args.selector != "mlp":
        return o, None
    from paper_1206_6857_gb300 import selector
    params = selector.load()
    o.selector = gs.GS_SEL_MLP
    o.selector_params = params.data_ptr()
    return o, params


def run_batch(args):
    """Many uneven problems per step through gs_sum_batched (one GPU)."""
    import torch
    from paper_1206_6857_gb300 import build as gbuild
    from paper_1206_6857_gb300 import gs
    from workloads import synth
    gbuild.build()
    gs.load()
    dev = torch.device("cuda", 0)
    wls = synth.config5(scale=args.scale, count=args.count)
    eps = wls[0].eps if args.eps is None else args.eps
    probs = []
    for wl in wls:
        q = torch.from_numpy(wl.queries).to(dev)
        probs.append((q, q, torch.from_numpy(wl.weights).to(dev), wl.h, eps))
    opts = gs.gs_opts_default()
    if not args.no_small_exhaustive:
        opts.flags |= gs.GS_FLAG_SMALL_EXHAUSTIVE     # small problems: the exact sum is cheaper
        opts.small_work = args.small_work
    opts, keep = selector_opts(args, opts)
    units = float(sum(float(wl.M) * wl.N * wl.h.size for wl in wls))
    def small_work(D):
        return args.small_work if args.small_work > 0 else (gs.GS_SMALL_WORK_D2 if D <= 2 else gs.GS_SMALL_WORK)
    n_small = sum(1 for wl in wls if float(wl.M) * wl.N * wl.h.size <= small_work(wl.D))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        gs.gs_sum_batched(probs, opts=opts, nworkers=args.workers, stream=stream)
    torch.cuda.synchronize()
    props = torch.cuda.get_device_properties(dev)
    sampler = ClockSampler(getattr(props, "pci_bus_id", None))
    sampler.start()
    time.sleep(0.3)
    evs, stats_list = [], []
    for _ in range(args.steps):
        flush.fill_(1)
        st = gs.gs_stats()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gs.gs_sum_batched(probs, opts=opts, nworkers=args.workers, stream=stream, stats=st)
        e1.record(stream)
        evs.append((e0, e1))
        stats_list.append(st)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = float(sum(a.elapsed_time(b) for a, b in evs)) / args.steps
    value = units / (ms / 1e3)
    s0 = stats_list[-1]
    ex2_rate, ffma_rate = gs.gs_probe_rates()
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    peak = ex2_rate * props.multi_processor_count * sm_mhz * 1e6 / 1e12
    # problems overlap on concurrent streams, so per-problem kernel times do not
    # add up to device time: the rate is the step's exact-sum terms over its
    # wall time (a lower bound of the kernels' own rate)
    achieved = s0.point_pairs_base / (ms / 1e3) / 1e12 if ms > 0 else None
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tex2/s",
            "frac": achieved / peak if achieved else None, "traffic": None,
            "kernel": "k_basecase" if args.no_small_exhaustive else "k_exhaustive",
            "peak_basis": "measured %.1f ex2 lanes/SM/clk x %d SMs x %.0f MHz; exact-sum terms of all problems "
                          "over the step's wall time" % (ex2_rate, props.multi_processor_count, sm_mhz)}
    e2e = None
    if not args.no_e2e:
        hosts = [(torch.from_numpy(wl.queries).pin_memory(), torch.from_numpy(wl.weights).pin_memory(), wl.h)
                 for wl in wls]
        def e2e_step():
            ps = []
            for hq, hw, h in hosts:
                dq = hq.to(dev, non_blocking=True)
                ps.append((dq, dq, hw.to(dev, non_blocking=True), h, eps))
            outs, _ = gs.gs_sum_batched(ps, opts=opts, nworkers=args.workers, stream=stream)
            return [o.cpu() for o in outs]
        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": units / dt, "unit": "evals/s",
               "h2d_bytes_per_step": int(sum(h[0].numel() * 4 + h[1].numel() * 4 for h in hosts)),
               "d2h_bytes_per_step": int(sum(wl.M * wl.h.size * 8 for wl in wls)), "ms_per_step": dt * 1e3}
    cpu = None
    if not args.no_cpu:
        from oracle import build as ob
        ob.build()
        rates, cores, tot = [], 1, 0.0
        for wl in wls[:16]:
            r, dt, cores, _, _ = oracle_sample_rate(wl, min(wl.M, 20), wl.h)
            rates.append(r)
            tot += dt
        cpu = {"value": float(np.mean(rates)), "unit": "evals/s", "cores": cores, "kind": "oracle",
               "sample": "20 seeded queries x all refs x 8 bandwidths of each of the first 16 problems (%.1f s)" % tot}
    cfg = {"workload": "kde_batch_%d_problems_d2-8_n1e3-2e5_8h" % len(wls), "problems": len(wls),
           "sum_M_N_nh": units, "eps": eps, "mode": "batch", "workers": args.workers, "selector": args.selector,
           "small_exhaustive": (not args.no_small_exhaustive), "problems_summed_exhaustively":
           (0 if args.no_small_exhaustive else n_small),
           "l2": "flushed before every timed step (256 MB write)", "parallelism": "replicas"}
    line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg, "roofline": roof,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": int(s0.launches) * args.steps,
            "stats": s0.as_dict()}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "batch":
        if int(os.environ.get("RANK", "0")) == 0:
            run_batch(args)
    else:
        run_gs(args)


if __name__ == "__main__":
    main()
