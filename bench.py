#!/usr/bin/env python3
"""Benchmark: Wilson-Dirac operator on one GB300 (and N independent replicas).

Headline workload: one full-lattice FP32 Wilson-Dirac application,
D = (m+4) - H/2 with 18-real links, on a 32^4 periodic lattice (1,048,576
sites), smoothed SU(3) links exp(0.2 i H) (seed 1001), Gaussian source
(seed 2001), m = 0.1.  One step = one application.  The metric is achieved
HBM bandwidth in GB/s counted with compulsory bytes (480 B per site:
spinor in 96 B + out 96 B + four 72 B links), reported against the measured
copy bandwidth of the GPU.

Per step the inputs (503 MB) are much larger than the 129 MB L2, so no
explicit flush is needed between steps.

--impl reference times the FP64 CPU oracle (the plain definition of D) on
the host cores, one step = one application on an 8^4 sample lattice of the
same recipe, in the same unit.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DIMS = (32, 32, 32, 32)
MASS = 0.1
LINK_SEED, SRC_SEED = 1001, 2001
BYTES_PER_SITE = {  # compulsory bytes per output site
    ("f32", "full", 18): 480, ("f32", "full", 12): 384, ("f32", "eo", 18): 768, ("f32", "eo", 12): 576,
    ("f64", "full", 18): 960, ("f64", "full", 12): 768, ("f64", "eo", 18): 1536, ("f64", "eo", 12): 1152,
    ("f16", "full", 18): 248, ("f16", "full", 12): 200, ("f16", "eo", 18): 392, ("f16", "eo", 12): 296,
    ("bf16", "full", 18): 248, ("bf16", "full", 12): 200, ("bf16", "eo", 18): 392, ("bf16", "eo", 12): 296,
    ("df", "full", 18): 960, ("df", "full", 12): 768, ("df", "eo", 18): 1536, ("df", "eo", 12): 1152,
}
FLOPS_PER_SITE = 1320
HEADLINE_KERNEL = "hop_kernel<F32, 18, dagger=false, axpy=true>"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic_from_profile():
    """Per-launch DRAM bytes of the headline kernel from the committed ncu summary,
    valid only while the kernel sources are unchanged (source hash recorded there)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "hop_f32_full_r18_32x32x32x32.md")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    h = hashlib.sha256()
    for name in ("dslash_impl.cuh", "wd_device.cuh"):
        with open(os.path.join(ROOT, "paper_1901_07294_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    if vals.get("kernel_source_sha256") != h.hexdigest()[:16]:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """Samples SM clock and throttle reasons with nvidia-smi while active."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


HEADLINE_MAX_BYTES = 4096


def compose_headline(headline: dict, detail: dict, detail_path) -> dict:
    """The one JSON object printed last on stdout: the headline measurement and a
    few key secondary numbers pulled from the detail sections, nothing bulky.

    `headline` holds the measured keys (metric, value, unit, n_gpus, steps, warmup,
    ms_per_step, dtype, config, roofline, e2e, clocks, gpu_launches, cpu_baseline);
    `detail` the full sections, which go to the file `detail_path` instead."""
    line = {"impl": "wdirac"}
    line.update({k: headline[k] for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step")})
    line.update({"higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                 "dtype": headline["dtype"], "data": "synthetic"})
    for k in ("config", "gflops", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        if k in headline:
            line[k] = headline[k]
    cb = line.get("cpu_baseline")
    if cb is not None:
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample") if k in cb}
    sec = {}
    cg = detail.get("cg") or {}
    runs = cg.get("runs", {})
    for m in ("0.1", "0.05"):
        r64, r16, rdf = runs.get(f"m{m}/fp64"), runs.get(f"m{m}/fp16"), runs.get(f"m{m}/fp16_df")
        if r64 and r16:
            sec[f"cg_24x24x24x48_m{m}"] = {"fp64_s": r64["seconds"], "fp16_s": r16["seconds"],
                                            "speedup": round(r64["seconds"] / r16["seconds"], 2),
                                            "fp16_true_rel_resid": r16["true_rel_resid"]}
            if rdf:   # the same with double-word reliable updates
                sec[f"cg_24x24x24x48_m{m}"].update({"fp16_df_s": rdf["seconds"],
                                                    "speedup_df": round(r64["seconds"] / rdf["seconds"], 2),
                                                    "fp16_df_true_rel_resid": rdf["true_rel_resid"]})
    oc = detail.get("cpu_oracle_cg")
    if oc:
        sec["cpu_oracle_cg_24x24x24x48_m0.1_s"] = oc.get("seconds")
    mr = (detail.get("multi_rhs") or {}).get("eo")
    if mr:
        sec["mrhs12_eo_32x32x32x32"] = {"multi_ms": mr["multi_ms"], "singles_ms": mr["singles_ms"],
                                        "frac_hbm": mr["multi_frac_hbm"]}
    srv = (detail.get("serving") or {}).get("rate_200")
    if srv:
        sec["serving_200_per_s"] = {"p50_ms": srv["p50_ms"], "p99_ms": srv["p99_ms"],
                                    "solves_per_s": srv["achieved_per_s"]}
        if "frac_hbm" in srv:
            sec["serving_200_per_s"]["frac_hbm"] = srv["frac_hbm"]
    bt = detail.get("batch") or {}
    if "graph" in bt and "persistent" in bt:
        sec["batch24"] = {"graph_s": bt["graph"]["seconds"], "persistent_s": bt["persistent"]["seconds"],
                          "sequential_s": bt.get("sequential", {}).get("seconds")}
        if "fp16_graph_df" in bt:
            sec["batch24"]["fp16_graph_df_s"] = bt["fp16_graph_df"]["seconds"]
    if sec:
        line["secondary"] = sec
    line["detail"] = detail_path
    return line


def write_detail(detail: dict, path: str):
    """Writes the full detail sections as JSON to `path` (created with its folder);
    returns the path, or None if it could not be written."""
    if not path:
        return None
    try:
        d = os.path.dirname(os.path.abspath(path))
        os.makedirs(d, exist_ok=True)
        with open(path, "w") as f:
            json.dump(detail, f, indent=1, default=float)
        return path
    except OSError as e:
        print(f"[bench] detail not written: {e}", file=sys.stderr, flush=True)
        return None


def _cpu_oracle_cg(dims=(24, 24, 24, 48), mass=0.1, tol=1e-10):
    """One full FP64 oracle CG solve of the even-odd normal equations on 24^3x48 (the mixed-CG
    benchmark's gauge field and source), on all host threads: seconds, iterations and the
    oracle's own true residual."""
    import oracle
    import synth
    U = synth.gauge(dims, seed=1000 + 3)
    b = synth.even_spinor(dims, seed=3001)
    t0 = time.perf_counter()
    _, it, rel = oracle.cg(dims, U, mass, b, tol=tol)
    el = time.perf_counter() - t0
    return {"seconds": round(el, 3), "iters": it, "true_rel_resid": rel, "cores": oracle.max_threads(),
            "cpu_model": _cpu_model(), "lattice": list(dims), "mass": mass, "tol": tol,
            "how": "oracle.cg, textbook FP64 CG from x0 = 0, one full solve"}


_T0 = time.perf_counter()


def _log(section: str) -> None:
    """Progress of the benchmark sections on stderr (the JSON line goes to stdout)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f} s] {section}", file=sys.stderr, flush=True)


def job_time_ms(local_ms: float, ws: int, device) -> float:
    """Whole-job time of the timed region: the slowest rank's (max over ranks)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value_gbs(bytes_per_step: float, steps: int, ws: int, job_ms: float) -> float:
    """Whole-job throughput: all replicas' compulsory bytes over the whole-job time."""
    return bytes_per_step * steps * ws / (job_ms * 1e-3) / 1e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _cpu_baseline(samples_dims=(8, 8, 8, 8), min_seconds=10.0, max_reps=1_000_000):
    """FP64 oracle D on the host cores, in the same GB/s unit (480 B per site)."""
    import oracle
    import synth
    U = synth.gauge(samples_dims, seed=LINK_SEED)
    psi = synth.spinor(samples_dims, seed=SRC_SEED)
    v = synth.volume(samples_dims)
    oracle.dirac(samples_dims, U, psi, MASS)
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.dirac(samples_dims, U, psi, MASS)
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds or reps >= max_reps:
            break
    gbs = BYTES_PER_SITE[("f32", "full", 18)] * v * reps / el / 1e9
    return {"value": gbs, "unit": "GB/s", "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"FP64 oracle D on {'x'.join(map(str, samples_dims))} ({v} sites) x {reps} reps, "
                      f"{el:.1f} s; GB/s = sites/s x 480 B",
            "cpu_model": _cpu_model(), "host_threads": os.cpu_count()}


def _cpu_model():
    """The host CPU's model name (lscpu), or the architecture if lscpu is missing."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def _cpu_sizes(U32, psi32, reps=5):
    """The FP64 oracle D on the operator-benchmark lattices (32^4 with the GPU step's links and
    source, 16^3x32 with its own), `reps` applications each with 1 thread and with all host
    threads: ms per application and GB/s in the 480 B/site unit."""
    import oracle
    import synth
    out = {}
    nmax = oracle.max_threads()
    cases = [((32, 32, 32, 32), U32, psi32),
             ((16, 16, 16, 32), synth.gauge((16, 16, 16, 32), seed=1000 + 2), synth.spinor((16, 16, 16, 32), seed=2002))]
    try:
        for dims, U, psi in cases:
            v = synth.volume(dims)
            row = {}
            for nt in (1, nmax):
                oracle.set_threads(nt)
                oracle.dirac(dims, U, psi, MASS)
                t0 = time.perf_counter()
                for _ in range(reps):
                    oracle.dirac(dims, U, psi, MASS)
                ms = (time.perf_counter() - t0) / reps * 1e3
                row[f"threads_{nt}"] = {"ms_per_D": round(ms, 2),
                                        "gbs": round(BYTES_PER_SITE[("f32", "full", 18)] * v / (ms * 1e-3) / 1e9, 3)}
            out["x".join(map(str, dims))] = row
    finally:
        oracle.set_threads(nmax)
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    import synth
    dims = (8, 8, 8, 8)
    v = synth.volume(dims)
    U = synth.gauge(dims, seed=LINK_SEED)
    psi = synth.spinor(dims, seed=SRC_SEED)
    for _ in range(args.warmup):
        oracle.dirac(dims, U, psi, MASS)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.dirac(dims, U, psi, MASS)
    el = time.perf_counter() - t0
    gbs = BYTES_PER_SITE[("f32", "full", 18)] * v * args.steps / el / 1e9
    line = {
        "impl": "reference", "metric": "dslash_hbm_gbs", "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "wilson_dslash_full_fp32_recon18_32x32x32x32", "lattice": list(DIMS),
                   "sample_lattice": list(dims), "mass": MASS, "link_seed": LINK_SEED, "source_seed": SRC_SEED,
                   "note": "each step is a bounded sample of the workload: one D on an 8^4 lattice of the "
                           "same recipe, timed per site in the same unit"},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": f"one step = FP64 oracle D on 8^4 ({v} sites); GB/s = sites/s x 480 B"},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import numpy as np
    import torch

    import paper_1901_07294_gb300 as wd
    import synth

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    ctx = wd.Context(dev)
    dims = DIMS
    v = synth.volume(dims)
    U = synth.gauge(dims, seed=LINK_SEED)
    psi = synth.spinor(dims, seed=SRC_SEED)
    g = wd.Gauge(ctx, dims, U)
    psi_host = torch.from_numpy(psi.view(np.float64).reshape(-1).copy()).pin_memory()
    aos = psi_host.cuda()
    prec, recon = wd.F32, 18
    g.prepare(prec, recon)
    if args.launch:
        # pinned launch shape (profiling: the tuner's timings are not meaningful under a profiler)
        th, var = (int(t) for t in args.launch.split(","))
        wd.tune_set_dslash(ctx, g, prec, recon, True, True, 1, th, var)
        tune_table = [{"threads": th, "variant": var, "ms": float("nan")}]
    else:
        tune_table = wd.tune_dslash(ctx, g, prec, recon, full=True)   # the autotuner picks the launch shape
    best = min(tune_table, key=lambda t: t["ms"] if t["ms"] == t["ms"] else 0.0)
    fin = wd.alloc_field(dims, wd.SITES_FULL, prec)
    fout = wd.alloc_field(dims, wd.SITES_FULL, prec)
    wd.pack(ctx, dims, wd.SITES_FULL, prec, aos, fin)

    def step():
        wd.dslash_apply(ctx, g, fout, fin, MASS, prec=prec, recon=recon, stream=stream)

    # one event pair around the K back-to-back launches: events between the launches would
    # put their own gaps into the timed region
    events = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    # the sampler starts (and waits for its first samples) before the warm-up, so that the
    # GPU does not sit idle between the warm-up and the timed steps
    with ClockSampler(dev) as clk:
        for _ in range(max(args.warmup, 3)):
            step()
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        events[0].record(stream)
        for k in range(args.steps):
            step()
        events[1].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    local_ms = events[0].elapsed_time(events[1])
    total_ms = job_time_ms(local_ms, ws, "cuda")
    ms_per_step = total_ms / args.steps
    bytes_step = BYTES_PER_SITE[("f32", "full", 18)] * v
    value = job_value_gbs(bytes_step, args.steps, ws, total_ms)
    mean_launch = local_ms / args.steps   # this rank's mean launch duration
    achieved = bytes_step / (mean_launch * 1e-3) / 1e9
    peak, peak_kind = _peaks()

    # end to end through the public API with host buffers.  Three paths, each over the same
    # host-resident spinor, timed the same way (consecutive steps rotate over 2 or 3 streams
    # and buffer sets, so one step's H2D copy overlaps another step's D2H copy and compute):
    #   fp64_copy:   pinned FP64 canonical source -> H2D -> wd.pack -> wd.dslash_apply ->
    #                wd.unpack -> D2H into a pinned FP64 canonical result;
    #   fp64_direct: the pinned FP64 buffers handed to wd.pack / wd.unpack, which read and
    #                write them over the host link (no staging copies);
    #   fp32_copy:   as fp64_copy with FP32 canonical host buffers (wd_pack_f32 /
    #                wd_unpack_f32), half the bytes over the link.
    e2e_steps = max(4, min(args.steps, 20))
    host32 = torch.from_numpy(psi.view(np.float64).reshape(-1).astype(np.float32)).pin_memory()
    NS = 3   # streams (and buffer sets) the end-to-end loops rotate over
    sets = []
    for k in range(NS):
        s_k = torch.cuda.Stream() if k else stream
        sets.append(dict(s=s_k, aos=aos if k == 0 else torch.empty_like(aos), fin=fin if k == 0 else torch.empty_like(fin),
                         fout=fout if k == 0 else torch.empty_like(fout), aos_out=torch.empty_like(aos),
                         out_host=torch.empty_like(psi_host).pin_memory(),
                         aos32=torch.empty(host32.numel(), dtype=torch.float32, device="cuda"),
                         aos32_out=torch.empty(host32.numel(), dtype=torch.float32, device="cuda"),
                         out_host32=torch.empty_like(host32).pin_memory()))

    def fp64_copy(k):
        b = sets[k % nsets[0]]
        with torch.cuda.stream(b["s"]):
            b["aos"].copy_(psi_host, non_blocking=True)
            wd.pack(ctx, dims, wd.SITES_FULL, prec, b["aos"], b["fin"], stream=b["s"])
            wd.dslash_apply(ctx, g, b["fout"], b["fin"], MASS, prec=prec, recon=recon, stream=b["s"])
            wd.unpack(ctx, dims, wd.SITES_FULL, prec, b["fout"], b["aos_out"], stream=b["s"])
            b["out_host"].copy_(b["aos_out"], non_blocking=True)

    def fp64_direct(k):
        b = sets[k % nsets[0]]
        wd.pack(ctx, dims, wd.SITES_FULL, prec, psi_host, b["fin"], stream=b["s"])
        wd.dslash_apply(ctx, g, b["fout"], b["fin"], MASS, prec=prec, recon=recon, stream=b["s"])
        wd.unpack(ctx, dims, wd.SITES_FULL, prec, b["fout"], b["out_host"], stream=b["s"])

    def fp32_copy(k):
        b = sets[k % nsets[0]]
        with torch.cuda.stream(b["s"]):
            b["aos32"].copy_(host32, non_blocking=True)
            wd.pack(ctx, dims, wd.SITES_FULL, prec, b["aos32"], b["fin"], stream=b["s"])
            wd.dslash_apply(ctx, g, b["fout"], b["fin"], MASS, prec=prec, recon=recon, stream=b["s"])
            wd.unpack(ctx, dims, wd.SITES_FULL, prec, b["fout"], b["aos32_out"], stream=b["s"])
            b["out_host32"].copy_(b["aos32_out"], non_blocking=True)

    # the host-link floor of a path: its H2D and D2H copies alone, concurrently
    def copies64(k):
        b = sets[k % nsets[0]]
        with torch.cuda.stream(b["s"]):
            b["aos"].copy_(psi_host, non_blocking=True)
            b["out_host"].copy_(b["aos_out"], non_blocking=True)

    def copies32(k):
        b = sets[k % nsets[0]]
        with torch.cuda.stream(b["s"]):
            b["aos32"].copy_(host32, non_blocking=True)
            b["out_host32"].copy_(b["aos32_out"], non_blocking=True)

    nsets = [NS]   # streams in use by the loops below

    def time_loop(step, n, tries=3):
        """Best of `tries` timed loops of e2e_steps steps over n streams (the host link is
        shared with the machine's other GPUs, so single loops vary)."""
        nsets[0] = n
        for k in range(2 * n):
            step(k)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(tries):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for b in sets[1:n]:
                b["s"].wait_event(e0)
            for k in range(e2e_steps):
                step(k)
            for b in sets[1:n]:
                stream.wait_stream(b["s"])
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / e2e_steps)
        return best

    e2e_paths, e2e_floor = {}, {}
    for n in (2, NS):
        for name, fn in (("fp64_copy", fp64_copy), ("fp64_direct", fp64_direct), ("fp32_copy", fp32_copy)):
            e2e_paths[f"{name}_{n}streams"] = time_loop(fn, n)
        e2e_floor[f"fp64_copy_{n}streams"] = time_loop(copies64, n)
        e2e_floor[f"fp32_copy_{n}streams"] = time_loop(copies32, n)
        e2e_floor[f"fp64_direct_{n}streams"] = e2e_floor[f"fp64_copy_{n}streams"]
    e2e_best = min(e2e_paths, key=e2e_paths.get)
    e2e_ms = e2e_paths[e2e_best]
    e2e_value = bytes_step * ws / (e2e_ms * 1e-3) / 1e9
    e2e_io_bytes = v * 24 * (4 if e2e_best.startswith("fp32") else 8)
    e2e_desc = {"fp64_copy": "pinned FP64 canonical H2D -> wd.pack -> wd.dslash_apply -> wd.unpack -> D2H",
                "fp64_direct": "pinned FP64 canonical source and result passed to wd.pack / wd.unpack, which "
                               "read and write them over the host link; wd.dslash_apply between",
                "fp32_copy": "pinned FP32 canonical H2D -> wd.pack (wd_pack_f32) -> wd.dslash_apply -> "
                             "wd.unpack (wd_unpack_f32) -> D2H"}

    variants = {}
    if not args.no_variants:
        _log("variants")
        device_peaks = {"fp64_tflops": round(wd.probe_fma_tflops(ctx, wd.F64), 3),
                        "fp32_tflops": round(wd.probe_fma_tflops(ctx, wd.F32), 2),
                        "how": "FMA chains on every SM, CUDA events (wd_probe_fma)"}
        variants = _variants(wd, torch, ctx, dims, U, psi, stream, peak, device_peaks["fp64_tflops"])
        variants["device_peaks"] = device_peaks
    mrhs = None
    blas = None
    streams = None
    dd = None
    if not args.no_variants:
        _log("multi_rhs")
        mrhs = _mrhs_section(wd, torch, ctx, U, psi, peak)
        _log("blas")
        blas = _blas_section(wd, torch, ctx, psi, peak, stream,
                             fp64_tflops=variants.get("device_peaks", {}).get("fp64_tflops"))
        _log("dd")
        dd = _dd_section(wd, torch, ctx, U, psi, peak, mean_launch)
        _log("stream")
        streams = _stream_section(wd, torch, ctx, peak, stream,
                                  fp64_tflops=variants.get("device_peaks", {}).get("fp64_tflops"))
    batch = None
    if not args.no_cg:
        _log("batch")
        batch = _batch_section(wd, torch, ctx, peak)
    serving = None
    if not args.no_cg and not args.no_serving:
        _log("serving")
        serving = _serving_section(wd, torch, ctx, peak)
    solve = None
    if not args.no_cg:
        _log("solve")
        solve = _solve_section(wd, torch, ctx, peak)
    cg = None
    if not args.no_cg:
        _log("cg")
        cg = _cg_section(wd, torch, ctx, peak=peak)
    _log("done")

    traffic = _traffic_from_profile()
    props = wd.device_info(ctx)
    headline = {
        "metric": "dslash_hbm_gbs", "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "dtype": "f32",
        "config": {"workload": "wilson_dslash_full_fp32_recon18_32x32x32x32", "lattice": list(dims),
                   "sites": v, "mass": MASS, "links": "exp(0.2 i H) smoothed SU(3), seed 1001",
                   "source": "Gaussian N(0,1), seed 2001", "bytes_per_site": 480,
                   "flops_per_site": FLOPS_PER_SITE, "l2": "inputs 503 MB per step > 129 MB L2, no flush",
                   "parallelism": f"replicas{ws}"},
        "gflops": FLOPS_PER_SITE * v * args.steps * ws / (total_ms * 1e-3) / 1e9,
        "roofline": {"bound": "hbm", "kernel": HEADLINE_KERNEL, "achieved": achieved, "peak": peak,
                     "peak_kind": f"{peak_kind} copy bandwidth (burst)", "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "mean_launch_ms": mean_launch},
        "e2e": {"value": e2e_value, "unit": "GB/s", "h2d_bytes_per_step": e2e_io_bytes,
                "d2h_bytes_per_step": e2e_io_bytes, "ms_per_step": e2e_ms,
                "path": e2e_desc[e2e_best.rsplit("_", 1)[0]] + ", consecutive steps rotating over "
                        + e2e_best.rsplit("_", 1)[1].replace("streams", " streams")},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
    }
    detail = {
        "roofline": {"algorithmic_bytes_per_launch": bytes_step,
                     "traffic_gbs": (traffic / (mean_launch * 1e-3) / 1e9) if traffic else None,
                     "nominal_peak": props["nominal_hbm_gbs"], "frac_of_nominal": achieved / props["nominal_hbm_gbs"],
                     "nominal_from": f"2 x {props['mem_clock_khz'] / 1e3:.0f} MHz x {props['mem_bus_bits']} bit / 8"},
        "e2e": {"copy_floor_ms_per_step": e2e_floor[e2e_best], "frac_of_copy_floor": e2e_floor[e2e_best] / e2e_ms,
                "paths_ms_per_step": e2e_paths, "paths_copy_floor_ms_per_step": e2e_floor},
        "autotune": {"chosen": {"threads": best["threads"], "variant": best["variant"]},
                     "candidates_us": {f"{t['threads']}/v{t['variant']}":
                                       (round(t["ms"] * 1e3, 1) if t["ms"] == t["ms"] else None)
                                       for t in tune_table}},
        "variants": variants,
        "multi_rhs": mrhs,
        "blas": blas,
        "stream": streams,
        "domain_decomposition": dd,
        "cg": cg,
        "solve": solve,
        "batch": batch,
        "serving": serving,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        _log("cpu_baseline")
        headline["cpu_baseline"] = _cpu_baseline()
        _log("cpu_sizes")
        detail["cpu_sizes"] = _cpu_sizes(U, psi)
        if cg is not None and not args.no_oracle_cg:
            _log("cpu_oracle_cg")
            detail["cpu_oracle_cg"] = _cpu_oracle_cg()
    if rank == 0:
        detail_path = write_detail(detail, args.detail_out)
        line = compose_headline(headline, detail, detail_path)
        print(json.dumps(line, separators=(",", ":")), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def _per_launch_ms(torch, fn, stream, reps, flush=None):
    """Mean and median of `reps` launches, each between its own CUDA events on `stream`
    (torch's current stream); with `flush` (a buffer larger than L2) that buffer is
    written before every launch."""
    import statistics
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    # hold the stream for about 100 us per launch so that every launch is queued before the
    # first runs: a launch shorter than the host's submission time is then still timed alone
    torch.cuda._sleep(200_000 * reps)
    for a, b in evs:
        if flush is not None:
            flush.zero_()
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    ts = [a.elapsed_time(b) for a, b in evs]
    return sum(ts) / len(ts), statistics.median(ts)


def _variants(wd, torch, ctx, base_dims, U_base, psi_base, stream, peak, fp64_tflops=None, reps=100):
    """Per-launch times and GB/s of every operator variant of the 32^4 / 16^3x32 configuration:
    mean and median over `reps` launches timed one by one, warm (the inputs of consecutive
    launches may still be in L2: 16^3x32 FP32 is about 63 MB) and with L2 flushed (a buffer of
    twice the L2 size written before each launch)."""
    import numpy as np

    import synth
    l2 = wd.device_info(ctx)["l2_bytes"] or (128 << 20)
    flush = torch.empty(2 * l2 // 4, dtype=torch.float32, device="cuda")
    out = {"timing": f"{reps} launches each, CUDA events per launch; L2 flush: {2 * l2 >> 20} MB written before each"}
    for dims in ((32, 32, 32, 32), (16, 16, 16, 32)):
        if dims == base_dims:
            U, psi = U_base, psi_base
        else:
            U = synth.gauge(dims, seed=1000 + 2)
            psi = synth.spinor(dims, seed=2002)
        v = synth.volume(dims)
        g = wd.Gauge(ctx, dims, U)
        aos = torch.from_numpy(psi.view(np.float64).reshape(-1).copy()).cuda()
        for prec in (wd.F32, wd.F64, wd.F16, wd.BF16, wd.DF):
            pn = wd.PREC_NAMES[prec]
            full_in = wd.alloc_field(dims, wd.SITES_FULL, prec)
            wd.pack(ctx, dims, wd.SITES_FULL, prec, aos, full_in, stream=stream)
            full_out = wd.alloc_field(dims, wd.SITES_FULL, prec)
            half = wd.field_bytes(dims, wd.SITES_EVEN, prec)
            eo_in = full_in[half:]             # odd half
            eo_out = wd.alloc_field(dims, wd.SITES_EVEN, prec)
            for recon in (18, 12):
                g.prepare(prec, recon)
                wd.tune_dslash(ctx, g, prec, recon, full=True)
                wd.tune_dslash(ctx, g, prec, recon, full=False, with_x=False)
                for kind in ("full", "eo"):
                    if kind == "full":
                        fn = lambda: wd.dslash_apply(ctx, g, full_out, full_in, MASS, prec=prec, recon=recon,
                                                     stream=stream)
                        nsite = v
                    else:
                        fn = lambda: wd.dslash_eo_apply(ctx, g, eo_out, eo_in, None, wd.EVEN, 0.0, 1.0,
                                                        prec=prec, recon=recon, stream=stream)
                        nsite = v // 2
                    for _ in range(10):
                        fn()
                    ms, med = _per_launch_ms(torch, fn, stream, reps)
                    ms_fl, med_fl = _per_launch_ms(torch, fn, stream, reps, flush=flush)
                    b = BYTES_PER_SITE[(pn, kind, recon)] * nsite
                    gbs = b / (ms * 1e-3) / 1e9
                    key = f"{'x'.join(map(str, dims))}/{pn}/{kind}/r{recon}"
                    out[key] = {"ms": round(ms, 5), "ms_median": round(med, 5), "gbs": round(gbs, 1),
                                "frac_hbm": round(gbs / peak, 4),
                                "gflops": round(FLOPS_PER_SITE * nsite / (ms * 1e-3) / 1e9, 1),
                                "ms_l2_flushed": round(ms_fl, 5), "ms_l2_flushed_median": round(med_fl, 5),
                                "frac_hbm_l2_flushed": round(b / (ms_fl * 1e-3) / 1e9 / peak, 4)}
                    if pn == "f64" and fp64_tflops:
                        # FP64 is bounded by the FP64 units: the useful 1320 flops/site
                        # against the measured FP64 FMA rate
                        out[key]["frac_fp64_alu"] = round(out[key]["gflops"] / 1e3 / fp64_tflops, 4)
                    if pn == "df":   # double-word FP32 replaces FP64 where 48 bits suffice
                        k64 = key.replace("/df/", "/f64/")
                        if k64 in out:
                            out[key]["speedup_vs_f64"] = round(out[k64]["ms"] / ms, 2)
        g.close()
    return out


def _blas_section(wd, torch, ctx, psi, peak, stream, fp64_tflops=None, reps=30):
    """Per-call GB/s of the field conversions (pack, unpack, convert) and of the
    BLAS-1 kernels with FP64 reductions (norm2, dot, axpby) on 32^4 full-lattice
    fields.  Bytes are the algorithmic ones: each input element read once and each
    output element written once (sizes from wd.field_bytes, so FP16 includes its
    per-site scale).  Consecutive calls rotate over enough buffer sets that more
    than twice the L2 size is touched between two uses of one buffer.

    FP64 arithmetic has its own floor on this part: FP64 instructions per site
    (DFMA, DMUL, DADD; conversions not counted) over the measured FP64 FMA rate.
    `bound` names the larger of the two floors and `frac_bound` = floor / time."""
    import numpy as np

    dims = DIMS
    v = int(np.prod(dims))
    full = wd.SITES_FULL
    aos_bytes = v * 24 * 8
    l2 = 129e6
    aos0 = torch.from_numpy(psi.view(np.float64).reshape(-1).copy()).cuda()
    res = torch.zeros(2, dtype=torch.float64, device="cuda")
    fb = {p: wd.field_bytes(dims, full, p) for p in (wd.F64, wd.F32, wd.F16)}
    out = {"lattice": list(dims), "sites": v}

    def nsets(call_bytes):
        return int(min(16, max(2, int(np.ceil(2 * l2 / call_bytes)) + 1)))

    dp_per_site = {"norm2_f64": 25, "dot_f64": 50, "axpby_f64": 48, "norm2_noalloc_f64": 25,
                   "norm2_f32": 1, "norm2_f16": 1, "dot_f32": 2, "dot_f16": 2}

    def timed(name, call_bytes, make, fn):
        n = nsets(call_bytes)
        sets = [make(k) for k in range(n)]
        for k in range(3):
            fn(sets[k % n])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(reps):
            fn(sets[k % n])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        gbs = call_bytes / (ms * 1e-3) / 1e9
        rec = {"ms": round(ms, 5), "bytes": int(call_bytes), "gbs": round(gbs, 1),
               "frac_hbm": round(gbs / peak, 4), "buffer_sets": n}
        t_hbm = call_bytes / (peak * 1e9)
        dp = dp_per_site.get(name, 0)
        t_alu = v * dp / (fp64_tflops * 1e12 / 2) if (fp64_tflops and dp) else 0.0
        rec["fp64_instr_per_site"] = dp
        rec["bound"] = "fp64_alu" if t_alu > t_hbm else "hbm"
        rec["frac_bound"] = round(max(t_hbm, t_alu) / (ms * 1e-3), 4)
        out[name] = rec

    def packed(p, k):
        f = wd.alloc_field(dims, full, p)
        wd.pack(ctx, dims, full, p, aos0, f, stream=stream)
        return f

    for p in (wd.F64, wd.F32, wd.F16):
        pn = wd.PREC_NAMES[p]
        timed(f"pack_aos_f64_to_{pn}", aos_bytes + fb[p],
              lambda k, p=p: (aos0.clone(), wd.alloc_field(dims, full, p)),
              lambda st, p=p: wd.pack(ctx, dims, full, p, st[0], st[1], stream=stream))
        timed(f"unpack_{pn}_to_aos_f64", aos_bytes + fb[p],
              lambda k, p=p: (packed(p, k), torch.empty_like(aos0)),
              lambda st, p=p: wd.unpack(ctx, dims, full, p, st[0], st[1], stream=stream))
        timed(f"norm2_{pn}", fb[p], lambda k, p=p: packed(p, k),
              lambda f, p=p: wd.norm2(ctx, dims, full, p, f, res, stream=stream))
        timed(f"dot_{pn}", 2 * fb[p], lambda k, p=p: (packed(p, k), packed(p, k)),
              lambda st, p=p: wd.dot(ctx, dims, full, p, st[0], st[1], res, stream=stream))
        timed(f"axpby_{pn}", 3 * fb[p], lambda k, p=p: (packed(p, k), packed(p, k)),
              lambda st, p=p: wd.axpby(ctx, dims, full, p, 0.5, st[0], -0.25, st[1], stream=stream))
    for pi, po in ((wd.F64, wd.F32), (wd.F64, wd.F16), (wd.F16, wd.F64), (wd.F32, wd.F16)):
        ni, no = wd.PREC_NAMES[pi], wd.PREC_NAMES[po]
        timed(f"convert_{ni}_to_{no}", fb[pi] + fb[po],
              lambda k, pi=pi, po=po: (packed(pi, k), wd.alloc_field(dims, full, po)),
              lambda st, pi=pi, po=po: wd.convert(ctx, dims, full, po, st[1], pi, st[0], stream=stream))
    timed("norm2_noalloc_f64", fb[wd.F64], lambda k: packed(wd.F64, k),
          lambda f: wd.norm2_noalloc(dims, full, wd.F64, f, res, stream=stream))
    return out


def _stream_section(wd, torch, ctx, peak, stream, fp64_tflops=None, reps=20):
    """Element-wise products of Sec. IV on 2^26 complex numbers (1 GiB per FP64 array; 2^27 reals
    for the real product), inputs N(0,1) generated on the device: GB/s of the algorithmic bytes
    (inputs read once, output written once) and the binding floor: HBM bytes over the measured
    copy bandwidth or FP64 instructions (1 per real product, 4 per complex one) over the measured
    FP64 FMA rate."""
    n = 1 << 26
    gen = torch.Generator(device="cuda").manual_seed(6001)
    x = torch.randn(2 * n, dtype=torch.float64, device="cuda", generator=gen)
    y = torch.randn(2 * n, dtype=torch.float64, device="cuda", generator=gen)
    z = torch.randn(2 * n, dtype=torch.float64, device="cuda", generator=gen)
    kinds = [("real_mul", wd.STREAM_REAL_MUL, 2 * n, 24, 1), ("cplx_mul", wd.STREAM_CPLX_MUL, n, 48, 4),
             ("cplx_conj_mul", wd.STREAM_CPLX_CONJ_MUL, n, 48, 4), ("cplx_madd", wd.STREAM_CPLX_MADD, n, 64, 4),
             ("cplx_conj_madd", wd.STREAM_CPLX_CONJ_MADD, n, 64, 4)]
    out = {"elements_complex": n, "array_bytes": 16 * n}
    for name, kind, count, bpe, dp in kinds:
        for _ in range(3):
            wd.stream_mul(ctx, kind, count, x, y, z, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            wd.stream_mul(ctx, kind, count, x, y, z, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        nbytes = count * bpe
        gbs = nbytes / (ms * 1e-3) / 1e9
        t_hbm = nbytes / (peak * 1e9)
        t_alu = count * dp / (fp64_tflops * 1e12 / 2) if fp64_tflops else 0.0
        out[name] = {"ms": round(ms, 5), "bytes": nbytes, "gbs": round(gbs, 1), "frac_hbm": round(gbs / peak, 4),
                     "fp64_instr_per_element": dp, "bound": "fp64_alu" if t_alu > t_hbm else "hbm",
                     "frac_bound": round(max(t_hbm, t_alu) / (ms * 1e-3), 4)}
    del x, y, z
    return out


def _dd_section(wd, torch, ctx, U, psi, peak, single_ms, reps=30):
    """The 32^4 FP32 Dslash split along t into nsub slabs with a halo exchange (all slabs on this
    GPU; the exchange is a device copy into each receiver's halo buffer): time per application of
    all slabs, GB/s of the same 480 B/site, and the bytes exchanged, with FP32 and FP16 halos."""
    import numpy as np
    dims = DIMS
    v = int(np.prod(dims))
    aos = torch.from_numpy(psi.view(np.float64).reshape(-1).copy()).cuda()
    out = {"lattice": list(dims), "single_domain_ms": round(single_ms, 5)}
    for nsub in (1, 2, 4, 8):
        dd = wd.DomainDecomposition(ctx, dims, nsub, U)
        ld = dd.local_dims()
        vloc = int(np.prod(ld))
        ins, outs = [], []
        for k in range(nsub):
            f = wd.alloc_field(ld, wd.SITES_FULL, wd.F32)
            wd.pack(ctx, ld, wd.SITES_FULL, wd.F32, aos[k * vloc * 24:(k + 1) * vloc * 24], f)
            ins.append(f)
            outs.append(wd.alloc_field(ld, wd.SITES_FULL, wd.F32))
        for hp in (wd.F32, wd.F16):
            for _ in range(3):
                dd.dslash(outs, ins, MASS, prec=wd.F32, halo_prec=hp)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                dd.dslash(outs, ins, MASS, prec=wd.F32, halo_prec=hp)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            gbs = 480 * v / (ms * 1e-3) / 1e9
            out[f"nsub{nsub}/{wd.PREC_NAMES[hp]}_halo"] = {
                "ms": round(ms, 5), "gbs": round(gbs, 1), "frac_hbm": round(gbs / peak, 4),
                "vs_single_domain": round(single_ms / ms, 3), "halo_bytes": dd.halo_bytes(hp)}
        dd.close()
    return out


def _mrhs_section(wd, torch, ctx, U, psi, peak, reps=20):
    """12 right-hand sides sharing each link load vs 12 single-field launches, FP32, 32^4."""
    import numpy as np

    import synth
    dims = DIMS
    v = synth.volume(dims)
    nrhs = 12
    g = wd.Gauge(ctx, dims, U)
    aos = torch.from_numpy(psi.view(np.float64).reshape(-1).copy()).cuda()
    one = wd.alloc_field(dims, wd.SITES_FULL, wd.F32)
    wd.pack(ctx, dims, wd.SITES_FULL, wd.F32, aos, one)
    out = {"nrhs": nrhs, "lattice": list(dims)}
    for kind, sites_in, sites_out, nsite, bps in (("eo", wd.SITES_ODD, wd.SITES_EVEN, v // 2, (192, 576)),
                                                  ("full", wd.SITES_FULL, wd.SITES_FULL, v, (192, 288))):
        nb_in = wd.field_bytes(dims, sites_in, wd.F32)
        src = one[nb_in:] if kind == "eo" else one
        fin = src.repeat(nrhs)
        fout = wd.alloc_field(dims, sites_out, wd.F32, nrhs)
        full = kind == "full"
        table = wd.tune_dslash(ctx, g, wd.F32, 18, full=full, with_x=False, nrhs=nrhs)
        wd.tune_dslash(ctx, g, wd.F32, 18, full=full, with_x=False, nrhs=1)
        tuned = min(table, key=lambda t: t["ms"])
        by_variant = {}
        for t in table:
            k = str(t["variant"])
            by_variant[k] = round(min(by_variant.get(k, 1e30), t["ms"]), 4)
        nb_out = wd.field_bytes(dims, sites_out, wd.F32)

        def multi():
            if full:
                wd.dslash_apply(ctx, g, fout, fin, MASS, nrhs=nrhs, prec=wd.F32)
            else:
                wd.dslash_eo_apply(ctx, g, fout, fin, None, wd.EVEN, 0.0, 1.0, nrhs=nrhs, prec=wd.F32)

        def singles():
            for k in range(nrhs):
                if full:
                    wd.dslash_apply(ctx, g, fout[k * nb_out:(k + 1) * nb_out], fin[k * nb_in:(k + 1) * nb_in],
                                    MASS, prec=wd.F32)
                else:
                    wd.dslash_eo_apply(ctx, g, fout[k * nb_out:(k + 1) * nb_out], fin[k * nb_in:(k + 1) * nb_in],
                                       None, wd.EVEN, 0.0, 1.0, prec=wd.F32)

        res = {}
        for name, fn in (("multi", multi), ("singles", singles)):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            res[name] = e0.elapsed_time(e1) / reps
        b_multi = (nrhs * bps[0] + bps[1]) * nsite
        out[kind] = {"multi_ms": round(res["multi"], 4), "singles_ms": round(res["singles"], 4),
                     "speedup": round(res["singles"] / res["multi"], 2),
                     "multi_gbs": round(b_multi / (res["multi"] * 1e-3) / 1e9, 1),
                     "multi_frac_hbm": round(b_multi / (res["multi"] * 1e-3) / 1e9 / peak, 4),
                     "bytes_per_site_rhs": round(b_multi / (nsite * nrhs), 1),
                     "tuned": {"threads": tuned["threads"], "variant": tuned["variant"]},
                     "tune_best_ms_by_variant": by_variant}
    g.close()
    return out


def _batch_section(wd, torch, ctx, peak):
    """24 solves of uneven volumes (8 each of 8^4, 16^4, 24^3x48), masses U[0.05, 0.5] (seed 4001),
    tol 1e-10, mixed reliable-update CG with FP32 and with FP16 inner storage: one persistent
    launch vs per-solve CUDA graphs vs 24 sequential cg_solve calls."""
    import numpy as np

    import synth
    rng = np.random.default_rng(4001)
    lattices = [(8, 8, 8, 8), (16, 16, 16, 16), (24, 24, 24, 48)]
    gauges = {}
    probs = []
    for k in range(24):
        dims = lattices[k // 8]
        if dims not in gauges:
            gauges[dims] = wd.Gauge(ctx, dims, synth.gauge(dims, seed=1000 + 10 + k // 8))
        b = synth.even_spinor(dims, seed=3200 + k)
        fb = wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
        wd.pack(ctx, dims, wd.SITES_EVEN, wd.F64, torch.from_numpy(b.view(np.float64).reshape(-1).copy()).cuda(), fb)
        probs.append(dict(gauge=gauges[dims], mass=float(rng.uniform(0.05, 0.5)), tol=1e-10, b=fb,
                          x=wd.alloc_field(dims, wd.SITES_EVEN, wd.F64), inner_prec=wd.F32, delta=0.01))
    t0 = time.perf_counter()
    for p in probs[:1] + probs[8:9] + probs[16:17]:
        for with_x in (False, True):
            for prec in (wd.F32, wd.F16, wd.F64, wd.DF):
                wd.tune_dslash(ctx, p["gauge"], prec, 18, full=False, with_x=with_x)
    tune_s = time.perf_counter() - t0
    out = {"solves": 24, "lattices": [list(d) for d in lattices], "tol": 1e-10, "inner": "fp32 reliable-update, delta 0.01",
           "autotune_seconds": round(tune_s, 3)}
    runs = [(name, mode, wd.F32) for name, mode in (("sequential", wd.BATCH_SEQUENTIAL), ("graph", wd.BATCH_GRAPH),
                                                    ("persistent", wd.BATCH_PERSISTENT))]
    runs += [(name, mode, wd.F16) for name, mode in (("fp16_sequential", wd.BATCH_SEQUENTIAL),
                                                     ("fp16_graph", wd.BATCH_GRAPH),
                                                     ("fp16_persistent", wd.BATCH_PERSISTENT))]
    # double-word reliable updates (the persistent kernel recomputes in FP64 only)
    runs += [("fp16_sequential_df", wd.BATCH_SEQUENTIAL, wd.F16), ("fp16_graph_df", wd.BATCH_GRAPH, wd.F16)]
    for name, mode, inner in runs:
        for p in probs:
            p["inner_prec"] = inner
            p["outer_prec"] = wd.DF if name.endswith("_df") else wd.F64
        wd.cg_solve_batch(ctx, probs, mode=mode)   # warm
        best = None
        for _ in range(2):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st = wd.cg_solve_batch(ctx, probs, mode=mode)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            if best is None or ms < best[0]:
                best = (ms, st)
        ms, st = best
        it_bytes = sum(s_["iters"] * int(np.prod(p["gauge"].dims)) // 2 * _cg_iteration_bytes(inner, 18)
                       for s_, p in zip(st, probs))
        out[name] = {"seconds": round(ms / 1e3, 4), "solves_per_s": round(24 / (ms / 1e3), 1),
                     "iters_total": int(sum(s["iters"] for s in st)),
                     "max_true_rel_resid": max(s["true_rel_resid"] for s in st),
                     "all_converged": all(s["status"] == 0 for s in st),
                     "iter_model_bytes": it_bytes,
                     "iter_frac_hbm_incl_updates": round(it_bytes / (ms / 1e3) / 1e9 / peak, 4)}
    for g in gauges.values():
        g.close()
    return out


def _serving_section(wd, torch, ctx, peak, n_main=2000, n_sweep=150, warm=100):
    """Serving: Poisson arrivals of CG solve requests (volumes uniform over 8^4, 16^4, 24^3x48,
    32^3x64; masses log-uniform in [0.02, 0.5]; tolerances in {1e-8, 1e-10, 1e-12}) on resident
    smoothed-SU(3) configurations, continuous batching with HBM admission.  Headline at 200 req/s
    plus a rate sweep; p50/p99 of submit->result latency."""
    import queue as pyqueue
    import threading as th

    import numpy as np

    import synth
    vols = [(8, 8, 8, 8), (16, 16, 16, 16), (24, 24, 24, 48), (32, 32, 32, 64)]
    gauges, srcs = {}, {}
    for k, dims in enumerate(vols):
        gauges[dims] = wd.Gauge(ctx, dims, synth.gauge(dims, seed=1000 + 20 + k))
        srcs[dims] = []
        for j in range(2):   # a small pool of Gaussian sources per volume
            b = synth.even_spinor(dims, seed=5100 + 10 * k + j)
            fb = wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
            wd.pack(ctx, dims, wd.SITES_EVEN, wd.F64, torch.from_numpy(b.view(np.float64).reshape(-1).copy()).cuda(), fb)
            srcs[dims].append(fb)
        for with_x in (False, True):
            wd.tune_dslash(ctx, gauges[dims], wd.F16, 18, full=False, with_x=with_x)
            wd.tune_dslash(ctx, gauges[dims], wd.F64, 18, full=False, with_x=with_x)
            wd.tune_dslash(ctx, gauges[dims], wd.DF, 18, full=False, with_x=with_x)
    torch.cuda.synchronize()
    pools = {d: [] for d in vols}   # free output buffers per volume

    def run(rate, n, seed, outer):
        rng = np.random.default_rng(seed)
        q = wd.Queue(ctx, hbm_budget_bytes=48 << 30, max_slots=32)
        waits = pyqueue.Queue()
        results = []

        def waiter():
            while True:
                item = waits.get()
                if item is None:
                    return
                t, dims, x, tol = item
                r = q.wait(t)
                pools[dims].append(x)
                results.append((tol, int(np.prod(dims)) // 2, r))

        wt = th.Thread(target=waiter)
        wt.start()
        t_next = time.perf_counter()
        for i in range(n):
            dims = vols[rng.integers(0, 4)]
            mass = float(np.exp(rng.uniform(np.log(0.02), np.log(0.5))))
            tol = float([1e-8, 1e-10, 1e-12][rng.integers(0, 3)])
            t_next += rng.exponential(1.0 / rate)
            while time.perf_counter() < t_next:
                time.sleep(max(0.0, min(0.0005, t_next - time.perf_counter())))
            x = pools[dims].pop() if pools[dims] else wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
            t = q.submit(dict(gauge=gauges[dims], mass=mass, tol=tol, b=srcs[dims][i % 2], x=x,
                              inner_prec=wd.F16, delta=0.01, outer_prec=outer))
            waits.put((t, dims, x, tol))
        waits.put(None)
        wt.join()
        st = q.stats()
        q.close()
        return results, st

    def summarise(results, st, rate, skip):
        tols = [t for t, _, _ in results][skip:]
        vhs = [v for _, v, _ in results][skip:]
        res = [r for _, _, r in results][skip:]
        lat = np.array([r["t_finish"] - r["t_submit"] for r in res])
        span = max(r["t_finish"] for r in res) - min(r["t_submit"] for r in res)
        ok = sum(1 for r in res if r["status"] == 0)
        # iteration bytes as if every request moved its own links (the single-field model);
        # the groups share link loads, so the bytes actually moved are fewer
        it_bytes = sum(r["cg_iters"] * vh * _cg_iteration_bytes(wd.F16, 18) for vh, r in zip(vhs, res))
        return {"offered_per_s": rate, "requests": len(res), "converged": ok,
                "achieved_per_s": round(len(res) / span, 2), "p50_ms": round(1e3 * float(np.percentile(lat, 50)), 2),
                "p99_ms": round(1e3 * float(np.percentile(lat, 99)), 2), "mean_running": round(st["mean_running"], 2),
                "admission_stalls": int(st["admission_stalls"]),
                "group_launches": int(st["group_launches"]), "mean_group_size": round(st["mean_group_size"], 2),
                "iterations": int(sum(r["cg_iters"] for r in res)), "reliable_updates": int(sum(r["cg_reliable_updates"] for r in res)),
                "iter_model_gbs": round(it_bytes / span / 1e9, 1), "frac_hbm": round(it_bytes / span / 1e9 / peak, 4),
                "max_true_resid_over_tol": round(max(r["cg_true_rel_resid"] / t for t, r in zip(tols, res)), 4)}

    out = {"volumes": [list(v) for v in vols],
           "inner": "fp16 storage, fp32 compute; reliable updates recompute the true residual with the "
                    "double-word FP32 operator, convergence confirmed with the FP64 one (rate_200_fp64_updates: "
                    "every update in FP64)",
           "queue": {"hbm_budget_gb": 48, "max_slots": 32, "max_iterations_per_group_launch": 16,
                     "scheduling": "requests grouped by gauge: one shared-link hop launch per hop for a "
                                   "group's ready members; reliable updates on the members' own streams"}}
    results, st = run(200.0, n_main + warm, 5001, wd.DF)
    out["rate_200"] = summarise(results, st, 200.0, warm)
    results, st = run(200.0, n_main + warm, 5001, wd.F64)
    out["rate_200_fp64_updates"] = summarise(results, st, 200.0, warm)
    out["sweep"] = []
    for rate in (10.0, 25.0, 50.0, 100.0):
        results, st = run(rate, n_sweep, 5002 + int(rate), wd.DF)
        out["sweep"].append(summarise(results, st, rate, 10))
    for g in gauges.values():
        g.close()
    return out


def _bicgstab_iteration_bytes(inner_prec, recon):
    """Bytes per even site that one BiCGStab iteration on Mhat moves by design: four
    even-odd hops (two Mhat applications; their second hops read the axpy term),
    p = r + beta (p - omega v) (r, p, v read, p written), <r^, v> (2 fields),
    s = r - alpha v (2 read, 1 written), <t, s> and |t|^2 (2), and the fused update
    (p, s, t, r^ read, r written, x read and written): 26 inner-precision passes, two
    over the x accumulator and four link sets.  Reliable updates come on top."""
    fb = {0: 192, 1: 96, 2: 52, 3: 52}[inner_prec]
    link_b = {0: 8, 1: 4, 2: 2, 3: 2}[inner_prec] * recon * 8
    fx = 192 if inner_prec == 0 else 96
    return 26 * fb + 4 * link_b + 2 * fx


def _cg_iteration_bytes(inner_prec, recon):
    """Bytes per even site that one CG iteration on Mhat^dagger Mhat moves by design
    (every kernel's inputs read once, outputs written once): four even-odd hops
    (spinor in and out, 8 links; the two Mhat hops also read their axpy term),
    Re<p, Ap> with alpha (p, Ap), the fused update (r and x read and written, Ap and
    p read; |r|^2) and p = r + beta p.  That is 19 passes over inner-precision
    fields, two over the x accumulator (FP32 for the reduced precisions, FP64 for
    FP64) and four link sets.  Reliable updates and the final true residual come
    on top."""
    fb = {0: 192, 1: 96, 2: 52, 3: 52}[inner_prec]
    link_b = {0: 8, 1: 4, 2: 2, 3: 2}[inner_prec] * recon * 8
    fx = 192 if inner_prec == 0 else 96
    return 19 * fb + 4 * link_b + 2 * fx


def _solve_section(wd, torch, ctx, peak):
    """Full-system solve D x = b on 24^3x48 (Gaussian source on all sites, seed 3201), tol 1e-10:
    BiCGStab on Mhat vs CG on the normal equations, FP64 and mixed FP16 (reliable updates,
    delta 0.01).  Best of 2 after one warm solve."""
    import numpy as np

    import synth
    dims = (24, 24, 24, 48)
    U = synth.gauge(dims, seed=1000 + 3)
    b = synth.spinor(dims, seed=3201)
    g = wd.Gauge(ctx, dims, U)
    fb = wd.alloc_field(dims, wd.SITES_FULL, wd.F64)
    wd.pack(ctx, dims, wd.SITES_FULL, wd.F64, torch.from_numpy(b.view(np.float64).reshape(-1).copy()).cuda(), fb)
    fx = wd.alloc_field(dims, wd.SITES_FULL, wd.F64)
    vh = int(np.prod(dims)) // 2
    out = {"lattice": list(dims), "tol": 1e-10, "mass": 0.1, "runs": {},
           "iter_model": "per-iteration bytes of the Schur solver's kernels (reliable updates and the "
                         "source and reconstruction hops excluded) over the whole solve time per iteration"}
    runs = [("bicgstab_fp64", wd.SOLVER_BICGSTAB, dict(inner_prec=wd.F64)),
            ("bicgstab_fp16", wd.SOLVER_BICGSTAB, dict(inner_prec=wd.F16, reliable=True, delta=0.01)),
            ("bicgstab_fp32", wd.SOLVER_BICGSTAB, dict(inner_prec=wd.F32, reliable=True, delta=0.01)),
            ("cgne_fp64", wd.SOLVER_CGNE, dict(inner_prec=wd.F64)),
            ("cgne_fp16", wd.SOLVER_CGNE, dict(inner_prec=wd.F16, reliable=True, delta=0.01)),
            ("cgne_fp16_graph", wd.SOLVER_CGNE, dict(inner_prec=wd.F16, reliable=True, delta=0.01, use_graph=True)),
            ("bicgstab_fp16_df", wd.SOLVER_BICGSTAB, dict(inner_prec=wd.F16, reliable=True, delta=0.01,
                                                          outer_prec=wd.DF)),
            ("cgne_fp16_graph_df", wd.SOLVER_CGNE, dict(inner_prec=wd.F16, reliable=True, delta=0.01, use_graph=True,
                                                        outer_prec=wd.DF))]
    for name, solver, kw in runs:
        wd.wilson_solve(ctx, g, 0.1, fx, fb, tol=1e-10, solver=solver, autotune=True, **kw)
        best = None
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st = wd.wilson_solve(ctx, g, 0.1, fx, fb, tol=1e-10, solver=solver, **kw)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            if best is None or ms < best[0]:
                best = (ms, st)
        ms, st = best
        rec = {"seconds": round(ms / 1e3, 5), "iters": st["iters"],
               "reliable_updates": st["reliable_updates"], "true_rel_resid": st["true_rel_resid"]}
        if st["iters"] > 0:
            model = _bicgstab_iteration_bytes if solver == wd.SOLVER_BICGSTAB else _cg_iteration_bytes
            it_bytes = model(kw["inner_prec"], kw.get("inner_recon", 18)) * vh
            per_it = ms / 1e3 / st["iters"]
            rec.update({"ms_per_iter_incl_updates": round(per_it * 1e3, 5), "iter_model_bytes": it_bytes,
                        "iter_frac_hbm_incl_updates": round(it_bytes / per_it / 1e9 / peak, 4)})
        out["runs"][name] = rec
    g.close()
    return out


def _cg_section(wd, torch, ctx, peak: float):
    """Mixed-precision vs FP64 CG on the even-odd normal equations, 24^3x48, tol 1e-10.  Runs named
    *_df recompute the true residual at reliable updates with the double-word FP32 operator
    (outer_prec = DF), confirming convergence with the FP64 one."""
    import numpy as np

    import synth
    dims = (24, 24, 24, 48)
    vh = int(np.prod(dims)) // 2
    U = synth.gauge(dims, seed=1000 + 3)
    b = synth.even_spinor(dims, seed=3001)
    g = wd.Gauge(ctx, dims, U)
    fb = wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
    wd.pack(ctx, dims, wd.SITES_EVEN, wd.F64, torch.from_numpy(b.view(np.float64).reshape(-1).copy()).cuda(), fb)
    fx = wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
    runs = [("fp64", dict(inner_prec=wd.F64)),
            ("fp32", dict(inner_prec=wd.F32, reliable=True, delta=0.01)),
            ("fp16", dict(inner_prec=wd.F16, reliable=True, delta=0.01)),
            ("bf16", dict(inner_prec=wd.BF16, reliable=True, delta=0.01)),
            ("fp16_r12", dict(inner_prec=wd.F16, inner_recon=12, reliable=True, delta=0.01)),
            ("fp16_graph", dict(inner_prec=wd.F16, reliable=True, delta=0.01, use_graph=True)),
            ("fp16_df", dict(inner_prec=wd.F16, reliable=True, delta=0.01, outer_prec=wd.DF)),
            ("fp16_graph_df", dict(inner_prec=wd.F16, reliable=True, delta=0.01, use_graph=True, outer_prec=wd.DF)),
            ("fp32_df", dict(inner_prec=wd.F32, reliable=True, delta=0.01, outer_prec=wd.DF)),
            ("bf16_df", dict(inner_prec=wd.BF16, reliable=True, delta=0.01, outer_prec=wd.DF)),
            ("fp16_delta0.1", dict(inner_prec=wd.F16, reliable=True, delta=0.1)),
            ("fp16_delta0.001", dict(inner_prec=wd.F16, reliable=True, delta=0.001)),
            ("fp16_refine", dict(inner_prec=wd.F16, reliable=False, delta=1e-3))]
    out = {"lattice": list(dims), "tol": 1e-10, "source": "Gaussian on even sites, seed 3001", "runs": {}}
    for mass in (0.1, 0.05):
        for name, kw in runs:
            wd.cg_solve(ctx, g, mass, fx, fb, tol=1e-10, maxiter=20000, autotune=True, **kw)   # warm: layouts, workspace, tuning
            best = None
            for _ in range(3):   # best of 3
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                st = wd.cg_solve(ctx, g, mass, fx, fb, tol=1e-10, maxiter=20000, **kw)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                if best is None or ms < best[0]:
                    best = (ms, st)
            ms, st = best
            rec = {"seconds": round(ms / 1e3, 5), "iters": st["iters"],
                   "reliable_updates": st["reliable_updates"], "true_rel_resid": st["true_rel_resid"]}
            if st["iters"] > 0:
                ps = kw["inner_prec"]
                it_bytes = _cg_iteration_bytes(ps, kw.get("inner_recon", 18)) * vh
                per_it = ms / 1e3 / st["iters"]
                rec.update({"ms_per_iter": round(per_it * 1e3, 5), "iter_model_bytes": it_bytes,
                            "iter_gbs": round(it_bytes / per_it / 1e9, 1),
                            "iter_frac_hbm": round(it_bytes / per_it / 1e9 / peak, 4)})
            out["runs"][f"m{mass}/{name}"] = rec
    for mass in (0.1, 0.05):
        t64 = out["runs"][f"m{mass}/fp64"]["seconds"]
        out[f"speedup_fp16_vs_fp64_m{mass}"] = round(t64 / out["runs"][f"m{mass}/fp16"]["seconds"], 2)
        out[f"speedup_fp16_graph_vs_fp64_m{mass}"] = round(t64 / out["runs"][f"m{mass}/fp16_graph"]["seconds"], 2)
        out[f"speedup_bf16_vs_fp64_m{mass}"] = round(t64 / out["runs"][f"m{mass}/bf16"]["seconds"], 2)
        out[f"speedup_fp16_df_vs_fp64_m{mass}"] = round(t64 / out["runs"][f"m{mass}/fp16_df"]["seconds"], 2)
        out[f"speedup_fp16_graph_df_vs_fp64_m{mass}"] = round(t64 / out["runs"][f"m{mass}/fp16_graph_df"]["seconds"], 2)
    g.close()
    return out


def run_case(argv) -> int:
    """Runs one operator case a few times, for profiling (e.g. under ncu):

        python bench.py --case --op eo --prec f32 --dims 32,32,32,32 --nrhs 12 --launches 4 [--threads 128 --variant 3]
        python bench.py --case --op cg --prec f16 --dims 24,24,24,48 --launches 1
        python bench.py --case --op stream --kind 1 --n 16777216 --launches 3
        python bench.py --case --op dd --nsub 4 --halo f16 --launches 3
        python bench.py --case --op solve --prec f16 --dims 24,24,24,48 --launches 1
        python bench.py --case --op batch --prec f16 --dims 24,24,24,48 --nrhs 8 --launches 1
        python bench.py --case --op eo --prec df --dims 24,24,24,48 --launches 3

    Inputs are the seeded synthetic gauge field and source of the benchmark.  With
    --threads/--variant the launch shape is pinned; otherwise the library default
    is used (no tuning, so few launches precede the profiled ones).  --op cg runs
    `launches` mixed-precision CG solves (inner precision --prec, reliable updates,
    delta 0.01, tol 1e-10, mass 0.1) on an even Gaussian source; --graph drives
    them with CUDA graphs; --outer df recomputes the true residual at the reliable
    updates (cg, solve, batch) with the double-word operator.  --op stream runs `launches` element-wise products of
    kind --kind on --n elements of N(0,1) arrays.  --op dd applies the operator
    `launches` times to the lattice split into --nsub slabs (field precision
    --prec, halos --halo).  --op solve runs `launches` full-system solves
    D x = b by BiCGStab (inner precision --prec, delta 0.01, tol 1e-10, mass 0.1).
    --op batch runs `launches` graph-mode batches of --nrhs solves on one gauge
    (one request group: shared-link hops), masses 0.1, 0.15, ..., tol 1e-10."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["full", "eo", "cg", "stream", "dd", "solve", "batch"], default="full")
    ap.add_argument("--nsub", type=int, default=2)
    ap.add_argument("--halo", choices=["f64", "f32", "f16"], default="f32")
    ap.add_argument("--kind", type=int, default=1)
    ap.add_argument("--n", type=int, default=1 << 24)
    ap.add_argument("--prec", choices=["f64", "f32", "f16", "bf16", "df"], default="f32")
    ap.add_argument("--outer", choices=["f64", "df"], default="f64",
                    help="cg/solve/batch: arithmetic of the reliable updates' operator")
    ap.add_argument("--recon", type=int, default=18)
    ap.add_argument("--dims", default="32,32,32,32")
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--launches", type=int, default=4)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--variant", type=int, default=-1)
    ap.add_argument("--graph", action="store_true")
    a = ap.parse_args(argv)
    import numpy as np
    import torch

    import paper_1901_07294_gb300 as wd
    import synth

    prec = {"f64": wd.F64, "f32": wd.F32, "f16": wd.F16, "bf16": wd.BF16, "df": wd.DF}[a.prec]
    outer = wd.DF if a.outer == "df" else wd.F64
    dims = tuple(int(t) for t in a.dims.split(","))
    ctx = wd.Context(0)
    if a.op == "stream":
        gen = torch.Generator(device="cuda").manual_seed(6001)
        x, y, z = (torch.randn(2 * a.n, dtype=torch.float64, device="cuda", generator=gen) for _ in range(3))
        for _ in range(a.launches):
            wd.stream_mul(ctx, a.kind, a.n, x, y, z)
        torch.cuda.synchronize()
        print(f"case: stream kind={a.kind} n={a.n} launches={a.launches} ok")
        return 0
    if a.op == "dd":
        hp = {"f64": wd.F64, "f32": wd.F32, "f16": wd.F16}[a.halo]
        dd = wd.DomainDecomposition(ctx, dims, a.nsub, synth.gauge(dims, seed=1001))
        ld = dd.local_dims()
        vloc = int(np.prod(ld))
        aos = torch.from_numpy(synth.spinor(dims, seed=2001).view(np.float64).reshape(-1).copy()).cuda()
        ins, outs = [], []
        for k in range(a.nsub):
            f = wd.alloc_field(ld, wd.SITES_FULL, prec)
            wd.pack(ctx, ld, wd.SITES_FULL, prec, aos[k * vloc * 24:(k + 1) * vloc * 24], f)
            ins.append(f)
            outs.append(wd.alloc_field(ld, wd.SITES_FULL, prec))
        for _ in range(a.launches):
            dd.dslash(outs, ins, 0.1, prec=prec, recon=a.recon, halo_prec=hp)
        torch.cuda.synchronize()
        print(f"case: dd {a.prec} halo {a.halo} {a.dims} nsub={a.nsub} launches={a.launches} ok")
        return 0
    g = wd.Gauge(ctx, dims, synth.gauge(dims, seed=1001))
    if a.op == "batch":   # --nrhs solves on this gauge as one request group (graph batch mode)
        probs = []
        for k in range(a.nrhs):
            b = synth.even_spinor(dims, seed=3400 + k)
            fb = wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
            wd.pack(ctx, dims, wd.SITES_EVEN, wd.F64,
                    torch.from_numpy(b.view(np.float64).reshape(-1).copy()).cuda(), fb)
            probs.append(dict(gauge=g, mass=0.1 + 0.05 * k, tol=1e-10, b=fb, x=wd.alloc_field(dims, wd.SITES_EVEN, wd.F64),
                              inner_prec=prec, delta=0.01, outer_prec=outer))
        for _ in range(a.launches):
            st = wd.cg_solve_batch(ctx, probs, mode=wd.BATCH_GRAPH)
        torch.cuda.synchronize()
        print(f"case: batch {a.prec} {a.dims} solves={a.nrhs} iters={[s_['iters'] for s_ in st]} ok")
        return 0
    if a.op == "solve":
        b = synth.spinor(dims, seed=3201)
        fb = wd.alloc_field(dims, wd.SITES_FULL, wd.F64)
        wd.pack(ctx, dims, wd.SITES_FULL, wd.F64, torch.from_numpy(b.view(np.float64).reshape(-1).copy()).cuda(), fb)
        fx = wd.alloc_field(dims, wd.SITES_FULL, wd.F64)
        for _ in range(a.launches):
            st = wd.wilson_solve(ctx, g, 0.1, fx, fb, tol=1e-10, solver=wd.SOLVER_BICGSTAB, inner_prec=prec,
                                 inner_recon=a.recon, reliable=True, delta=0.01, outer_prec=outer)
        torch.cuda.synchronize()
        print(f"case: solve bicgstab {a.prec} {a.dims} solves={a.launches} iters={st['iters']} "
              f"updates={st['reliable_updates']} seconds={st['seconds']:.4f} ok")
        return 0
    if a.op == "cg":
        b = synth.even_spinor(dims, seed=3001)
        fb = wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
        wd.pack(ctx, dims, wd.SITES_EVEN, wd.F64, torch.from_numpy(b.view(np.float64).reshape(-1).copy()).cuda(), fb)
        fx = wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
        for _ in range(a.launches):
            st = wd.cg_solve(ctx, g, 0.1, fx, fb, tol=1e-10, inner_prec=prec, inner_recon=a.recon, reliable=True,
                             delta=0.01, use_graph=a.graph, outer_prec=outer)
        torch.cuda.synchronize()
        print(f"case: cg {a.prec} r{a.recon} {a.dims} solves={a.launches} iters={st['iters']} "
              f"updates={st['reliable_updates']} seconds={st['seconds']:.4f} ok")
        return 0
    g.prepare(prec, a.recon)
    full = a.op == "full"
    if a.threads and a.variant >= 0:
        wd.tune_set_dslash(ctx, g, prec, a.recon, full, False, a.nrhs, a.threads, a.variant)
    aos = torch.from_numpy(synth.spinor(dims, seed=2001).view(np.float64).reshape(-1).copy()).cuda()
    one = wd.alloc_field(dims, wd.SITES_FULL, prec)
    wd.pack(ctx, dims, wd.SITES_FULL, prec, aos, one)
    if full:
        fin = one.repeat(a.nrhs)
        fout = wd.alloc_field(dims, wd.SITES_FULL, prec, a.nrhs)
    else:
        half = wd.field_bytes(dims, wd.SITES_ODD, prec)
        fin = one[half:].repeat(a.nrhs)
        fout = wd.alloc_field(dims, wd.SITES_EVEN, prec, a.nrhs)
    for _ in range(a.launches):
        if full:
            wd.dslash_apply(ctx, g, fout, fin, 0.1, nrhs=a.nrhs, prec=prec, recon=a.recon)
        else:
            wd.dslash_eo_apply(ctx, g, fout, fin, None, wd.EVEN, 0.0, 1.0, nrhs=a.nrhs, prec=prec, recon=a.recon)
    torch.cuda.synchronize()
    print(f"case: {a.op} {a.prec} r{a.recon} {a.dims} nrhs={a.nrhs} launches={a.launches} ok")
    return 0



def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="wdirac", choices=["wdirac", "reference"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cg", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-oracle-cg", action="store_true", help="skip the full FP64 oracle CG solve on the host")
    ap.add_argument("--launch", default="", help="THREADS,VARIANT: pin the headline launch shape instead of tuning")
    ap.add_argument("--detail-out", default=os.path.join("gpurun_out", "bench_detail.json"),
                    help="file for the full detail sections (the stdout line carries the headline only)")
    ap.add_argument("--case", nargs=argparse.REMAINDER, default=None,
                    help="run one operator case for profiling instead of the benchmark (see run_case)")
    args = ap.parse_args()
    if args.case is not None:
        return run_case(args.case)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
