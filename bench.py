#!/usr/bin/env python
"""Benchmark of the gauge-fixing hot path on GB300.

Workload (the configuration the headline metric is quoted on): a 32^3 x 64
SU(3) lattice, links exp(i eps H) with eps = 0.35 (seed 1), gauge fixed to
Landau gauge by overrelaxation (omega = 1.7) until theta < 1e-12, in mixed
precision: FP32 sweeps with 12-real links and FP64 re-unitarisation every
100 sweeps, FP64 theta/functional, and FP64 final sweeps.

One step = one complete gauge fixing of that lattice from a fresh random
point on its gauge orbit (Haar g(x), a different seed per step):
  restore the links from the copy resident in HBM -> random gauge transform
  -> sweeps with theta checks, re-unitarisation and the FP32 -> FP64 switch
  -> theta < 1e-12.
value = site-updates/s over the timed steps; the JSON line also carries
time-to-theta (mixed, and plain FP64 measured once), the roofline of the
dominant kernel, sampled clocks, an end-to-end number through host buffers
and the FP64 CPU oracle timed on a bounded sample.

Multi-GPU (torchrun): every rank fixes its own copies (independent
problems, weak scaling); the only cross-rank traffic is the barrier and the
max over ranks of the elapsed time.

--serving runs the serving workload instead: a Poisson stream of jobs
(lattices 16^4, 24^3 x 48, 32^4, 48^3 x 96; Landau, Coulomb or MAG; mixed
precision; eps = 0.3, seed 4) through the job server, first all at once to
measure the saturated job rate, then at a fraction of that rate; it prints
one JSON line with p50/p99 latency and site-updates/s.

--impl reference times the FP64 CPU oracle (the plain reference this
project checks against) on the host cores, on this same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="landau_or_32c3x64_mixed", dims=(64, 32, 32, 32), gauge="landau", eps=0.35,
                field_seed=1, omega=1.7, theta=1e-12, switch_theta=1e-8, reunit=100, check=20)
METRIC = "site-updates/s & HBM GB/s (mixed vs FP64); time-to-θ<1e-12; job p50/p99"
# 8 links x 12 reals x (load + store); the mixed-precision FP32 sweep also reads and
# writes the site's accumulated gauge transformation (one more 12-real matrix)
BYTES_PER_SU = {"fp32": 768, "fp64": 1536, "fp32_acc": 864}
FLOP_PER_SU = 2274  # App. A: 192 gather + 66 OR + 2016 apply
FP64_PEAK_TFLOPS = 1.25  # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (nominal table)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("gf_device.cuh", "gf_sweep.cuh"):
        with open(os.path.join(ROOT, "paper_1212_5221_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kind):
    """Per-launch DRAM bytes of a sweep kernel from the committed ncu summary
    (profiles/ncu_traffic.txt), if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    try:
        with open(path) as f:
            for line in f:
                p = line.split()
                if len(p) == 3 and not line.startswith("#") and p[0] == kind:
                    return int(p[2]) if p[1] == kernel_source_hash() else None
    except OSError:
        pass
    return None


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"gf_clocks_{os.getpid()}.csv")

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    try:
                        rows.append((float(p[1]), float(p[2]), p[5:9]))
                    except ValueError:
                        pass
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        load = [r[0] for r in rows] or [0]
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return None


def cpu_baseline(dims, omega, seconds_target=20.0, threads=1):
    """Time the FP64 oracle on whole sweeps of the workload's lattice, in a
    fresh process so no GPU state is shared: threads = 1 runs the plain build,
    threads > 1 the same source built with OpenMP (the sites of a parity in
    parallel) on that many host cores."""
    code = f"""
import sys, time, json
sys.path.insert(0, {ROOT!r})
import oracle
if {threads} > 1:
    oracle.use_openmp()
from paper_1212_5221_gb300 import inputs
U = inputs.links({tuple(dims)!r}, "smooth", {WORKLOAD['eps']}, {WORKLOAD['field_seed']})
oracle.random_gauge_transform(U, 1000)
oracle.sweep(U, "landau", "or", {omega}, 1)  # warm-up
n, t0 = 0, time.time()
while True:
    oracle.sweep(U, "landau", "or", {omega}, 1, n + 1)
    n += 1
    if time.time() - t0 > {seconds_target}:
        break
dt = time.time() - t0
print(json.dumps(dict(sweeps=n, seconds=dt)))
"""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        log("cpu baseline failed:", r.stderr[-500:])
        return None
    d = json.loads(r.stdout.strip().splitlines()[-1])
    V = int(np.prod(dims))
    what = "single thread" if threads == 1 else f"OpenMP build, {threads} threads"
    return {"value": d["sweeps"] * V / d["seconds"], "unit": "site-updates/s", "cores": threads, "kind": "oracle",
            "sample": f"{d['sweeps']} FP64 OR sweeps of the {'x'.join(map(str, dims[::-1]))} lattice "
                      f"(after 1 warm-up sweep), {d['seconds']:.1f} s, {what}",
            "cpu": cpu_model()}


def reduce_over_ranks(elapsed, site_updates, device=None):
    """Whole-job numbers for the replicas: the slowest rank's elapsed time and
    the sum of the site-updates of all ranks.  Without an initialised process
    group, the local values."""
    import torch

    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(elapsed), float(site_updates)
    t_max = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    s_sum = torch.tensor([float(site_updates)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t_max, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(s_sum, op=torch.distributed.ReduceOp.SUM)
    return float(t_max.item()), float(s_sum.item())


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle on this workload, on all host cores
    (the OpenMP build of the same source), rank 0 only."""
    if rank != 0:
        return
    import oracle
    from paper_1212_5221_gb300 import inputs

    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    cores = int(os.environ["OMP_NUM_THREADS"])
    if cores > 1:
        oracle.use_openmp()
    oracle.build(openmp=cores > 1)
    dims = WORKLOAD["dims"]
    V = int(np.prod(dims))
    U = inputs.links(dims, "smooth", WORKLOAD["eps"], WORKLOAD["field_seed"])
    oracle.random_gauge_transform(U, 1000)
    # one step = one FP64 OR sweep of the whole lattice (a bounded sample of a fix run)
    for k in range(args.warmup):
        oracle.sweep(U, "landau", "or", WORKLOAD["omega"], 1, k)
    t0 = time.time()
    for k in range(args.steps):
        oracle.sweep(U, "landau", "or", WORKLOAD["omega"], 1, args.warmup + k)
    dt = time.time() - t0
    value = args.steps * V / dt
    sample = (f"{args.steps} FP64 OR sweeps of the 32^3x64 lattice after {args.warmup} warm-up sweeps, "
              f"{cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "lattice": "32^3x64", "gauge": "landau", "omega": 1.7,
                       "step": "one FP64 overrelaxation sweep (oracle)"},
            "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": cores, "kind": "oracle",
                             "sample": sample, "cpu": cpu_model()},
            "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1212_5221_gb300 import build, gf, inputs

    build.build_all()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dims = WORKLOAD["dims"]
    V = int(np.prod(dims))
    W = WORKLOAD

    U = inputs.links(dims, "smooth", W["eps"], W["field_seed"])
    src = torch.from_numpy(U.view(np.float64).reshape(-1)).to(dev)  # resident input (natural order, FP64)
    field = gf.GaugeField(dims, W["gauge"], args.precision, device=dev)
    h = field.h
    fix_kw = dict(algo="or", param=W["omega"], theta_target=W["theta"], max_sweeps=args.max_sweeps,
                  check_interval=W["check"], reunit_interval=W["reunit"], switch_theta=args.switch_theta)

    def step(k):
        gf.gf_load_links_device(h, 0, src.data_ptr())
        gf.gf_random_gauge_transform(h, 1000 + k + 100000 * rank)
        return gf.gf_fix(h, **fix_kw)

    # launch shape: autotune both storage precisions once (setup, untimed)
    gf.gf_load_links_device(h, 0, src.data_ptr())
    gf.gf_random_gauge_transform(h, 999)
    lpt32, _ = gf.gf_autotune(h, "or")
    log(f"[rank {rank}] autotuned links/thread FP32 = {lpt32}")

    for k in range(args.warmup):
        r = step(-1 - k)
        log(f"[rank {rank}] warm-up {k}: {r['sweeps']} sweeps ({r['sweeps_fp32']} FP32), {r['seconds']:.2f} s")

    dist = torch.distributed.is_initialized()
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gf.gf_set_profiling(h, True)
    n0 = gf.gf_launch_count(h)
    results = []
    with Clocks(local_rank) as clocks:
        start.record(field.stream)
        t0 = time.time()
        for k in range(args.steps):
            results.append(step(k))
        stop.record(field.stream)
        torch.cuda.synchronize()
        wall = time.time() - t0
    elapsed = start.elapsed_time(stop) / 1e3
    launches = gf.gf_launch_count(h) - n0
    stats = {kind: gf.gf_kernel_stats(h, kind) for kind in range(5)}
    gf.gf_set_profiling(h, False)
    su = sum(r["site_updates"] for r in results)
    sweeps32 = sum(r["sweeps_fp32"] for r in results)
    sweeps64 = sum(r["sweeps_fp64"] for r in results)
    elapsed_all, su_all = reduce_over_ranks(elapsed, float(su), dev if dist else None)

    # roofline of the dominant kernel (largest total device time)
    peaks, peak_src = measured_peaks()
    kind_names = {0: "sweep_fp32", 1: "sweep_fp64", 2: "observables", 3: "reunitarize", 4: "promote"}
    dom = max(stats, key=lambda k: stats[k][1])
    n_l, ms_l = stats[dom]
    avg_s = ms_l / max(n_l, 1) / 1e3
    sites_per_launch = V // 2  # one sublattice
    if dom == 0:
        b32 = BYTES_PER_SU["fp32_acc" if args.precision == "mixed" else "fp32"]
        roof = {"bound": "hbm", "achieved": b32 * sites_per_launch / avg_s / 1e9,
                "peak": peaks["hbm_gbs"], "unit": "GB/s"}
        roof["traffic"] = ncu_traffic("sweep_fp32_acc" if args.precision == "mixed" else "sweep_fp32")
    elif dom == 1:
        roof = {"bound": "alu", "achieved": FLOP_PER_SU * sites_per_launch / avg_s / 1e12,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s"}
        roof["traffic"] = ncu_traffic("sweep_fp64")
    else:
        roof = {"bound": "hbm", "achieved": None, "peak": peaks["hbm_gbs"], "unit": "GB/s", "traffic": None}
    if roof["achieved"] is not None:
        roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = kind_names[dom]
    roof["avg_launch_ms"] = avg_s * 1e3
    roof["peak_source"] = (f"{peak_src} MEASURED_PEAKS.json hbm_gbs" if dom != 1 else
                           "FP64 ALU: nominal 1.25 TFLOP/s (2 FMA/clk/SM x 152 SMs x 2.07 GHz)")
    kernel_ms = {kind_names[k]: {"launches": stats[k][0], "ms": round(stats[k][1], 3)} for k in stats}
    sweep32_gbs = None
    if stats[0][0]:
        sweep32_gbs = (BYTES_PER_SU["fp32_acc" if args.precision == "mixed" else "fp32"] * sites_per_launch /
                       (stats[0][1] / stats[0][0] / 1e3) / 1e9)
    sweep64_gbs = None
    if stats[1][0]:
        sweep64_gbs = BYTES_PER_SU["fp64"] * sites_per_launch / (stats[1][1] / stats[1][0] / 1e3) / 1e9

    # the FP32 sweep kernel's own roofline (HBM), from the same timed steps
    roof32 = None
    if stats[0][0]:
        b32 = BYTES_PER_SU["fp32_acc" if args.precision == "mixed" else "fp32"]
        a32 = b32 * sites_per_launch / (stats[0][1] / stats[0][0] / 1e3) / 1e9
        roof32 = {"bound": "hbm", "achieved": a32, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                  "frac": a32 / peaks["hbm_gbs"],
                  "traffic": ncu_traffic("sweep_fp32_acc" if args.precision == "mixed" else "sweep_fp32"),
                  "avg_launch_ms": stats[0][1] / stats[0][0]}

    out = {}
    if rank == 0:
        def one_run(prec, switch, orbit_seed):
            fld = gf.GaugeField(dims, W["gauge"], prec, device=dev)
            gf.gf_load_links_device(fld.h, 0, src.data_ptr())
            gf.gf_random_gauge_transform(fld.h, orbit_seed)
            kw = dict(fix_kw, switch_theta=switch)
            r = gf.gf_fix(fld.h, **kw)
            F, T = gf.gf_functional_theta(fld.h)
            fld.close()
            return {"seconds": r["seconds"], "sweeps": r["sweeps"], "sweeps_fp32": r["sweeps_fp32"],
                    "sweeps_fp64": r["sweeps_fp64"], "site_updates_per_s": r["site_updates"] / r["seconds"],
                    "F": float(F[0]), "theta": float(T[0])}

        # plain FP64 on the same problems as the first timed steps (orbit seeds 1000 + k),
        # so that the two arms' time to theta compare like with like; and mixed precision
        # with the switch to FP64 sweeps moved down to the FP32 floor (seed 1000)
        n_match = min(args.fp64_matched, args.steps) if args.fp64_baseline else 0
        fp64_runs = []
        for k in range(n_match):
            r64 = one_run("fp64", args.switch_theta, 1000 + k)
            r64["mixed_seconds"] = results[k]["seconds"]
            r64["mixed_sweeps"] = results[k]["sweeps"]
            r64["rel_dF_mixed_vs_fp64"] = abs(results[k]["F_mean"] - r64["F"]) / abs(r64["F"])
            fp64_runs.append(r64)
            log(f"FP64 arm, orbit seed {1000 + k}: {r64['seconds']:.2f} s ({r64['sweeps']} sweeps); "
                f"mixed {results[k]['seconds']:.2f} s ({results[k]['sweeps']} sweeps)")
        fp64 = fp64_runs[0] if fp64_runs else None
        deep = one_run("mixed", args.deep_switch, 1000) if args.deep_switch > 0 else None
        # end to end through the C ABI with pinned host buffers, on the same orbit seeds as
        # the first timed steps
        e2e = None
        if args.e2e_steps > 0:
            host_in = torch.from_numpy(U.view(np.float64).reshape(-1)).pin_memory()
            host_out = torch.empty_like(host_in).pin_memory()
            hin = host_in.numpy().view(np.complex128).reshape(U.shape)
            hout = host_out.numpy().view(np.complex128).reshape(U.shape)
            n_e2e = min(args.e2e_steps, args.steps)
            torch.cuda.synchronize()
            t0 = time.time()
            su_e = 0
            for k in range(n_e2e):
                gf.gf_load_links(h, 0, hin)
                gf.gf_random_gauge_transform(h, 1000 + k)
                r = gf.gf_fix(h, **fix_kw)
                gf.gf_store_links(h, 0, hout)
                su_e += r["site_updates"]
            te = time.time() - t0
            su_dev = sum(results[k]["site_updates"] for k in range(n_e2e))
            t_dev = sum(results[k]["seconds"] for k in range(n_e2e))
            e2e = {"value": su_e / te, "unit": "site-updates/s", "h2d_bytes_per_step": int(U.nbytes),
                   "d2h_bytes_per_step": int(U.nbytes), "steps": n_e2e,
                   "orbit_seeds": [1000 + k for k in range(n_e2e)],
                   "seconds_per_step": te / n_e2e,
                   "same_steps_resident": {"value": su_dev / t_dev, "seconds_per_step": t_dev / n_e2e}}
        # the oracle on all host cores (OpenMP build), with the single-thread figure beside it
        cpu = None
        if args.cpu_seconds > 0:
            cpu = cpu_baseline(dims, W["omega"], args.cpu_seconds, threads=os.cpu_count() or 1)
            one = cpu_baseline(dims, W["omega"], args.cpu_seconds, threads=1)
            if cpu and one and cpu["cores"] > 1:
                cpu["single_thread"] = {k: one[k] for k in ("value", "cores", "sample")}
            elif one:
                cpu = one
        mixed_tt = elapsed / args.steps
        out = {
            "metric": METRIC,
            "value": su_all / elapsed_all,
            "unit": "site-updates/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": elapsed_all / args.steps * 1e3,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else ("f64" if args.precision == "fp64" else "f32"),
            "data": "synthetic",
            "config": {"workload": W["name"], "lattice": "32^3x64", "gauge": "landau", "algorithm": "OR",
                       "omega": W["omega"], "theta_target": W["theta"], "precision": args.precision,
                       "switch_theta": args.switch_theta, "reunit_interval": W["reunit"],
                       "check_interval": W["check"], "field": f"exp(i 0.35 H), seed {W['field_seed']}, "
                       "then Haar g(x) per step", "l2": "inputs larger than L2 (403 MB FP32 links)",
                       "parallelism": f"replicas x{world}"},
            "time_to_theta_s": {
                "mixed": mixed_tt,
                "matched_orbit_seeds": [1000 + k for k in range(n_match)],
                "mixed_matched": (float(np.mean([r["mixed_seconds"] for r in fp64_runs]))
                                  if fp64_runs else None),
                "fp64_matched": float(np.mean([r["seconds"] for r in fp64_runs])) if fp64_runs else None,
                "speedup_mixed_vs_fp64": (float(np.mean([r["seconds"] for r in fp64_runs]) /
                                                np.mean([r["mixed_seconds"] for r in fp64_runs]))
                                          if fp64_runs else None),
                "mixed_deep_switch": deep["seconds"] if deep else None,
                "speedup_mixed_deep_vs_fp64": (fp64["seconds"] / deep["seconds"]) if (fp64 and deep) else None},
            "same_orbit_runs": {"fp64": fp64_runs, f"mixed_switch_{args.deep_switch:g}": deep,
                                "rel_dF_deep_vs_fp64": abs(deep["F"] - fp64["F"]) / fp64["F"]
                                if (fp64 and deep) else None},
            "sweeps_per_step": {"fp32": sweeps32 / args.steps, "fp64": sweeps64 / args.steps},
            "hbm_gbs": {"sweep_fp32": sweep32_gbs, "sweep_fp64": sweep64_gbs},
            "roofline": roof,
            "roofline_sweep_fp32": roof32,
            "kernel_ms": kernel_ms,
            "gpu_launches": int(launches),
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clocks.summary(),
            "wall_s": wall,
        }
        print(json.dumps(out), flush=True)
    field.close()


SERVING = dict(name="serving_poisson_mixed", seed=4, eps=0.3, field_seed=4, check=20, reunit=100,
               omega={"landau": 1.7, "coulomb": 1.7, "mag": 1.35})


def run_serving(args):
    """Serving workload through gf_server_*: job k of the seeded stream fixes
    the lattice's eps = 0.3 field, moved to a fresh point of its gauge orbit
    by the job's own Haar seed, to theta < --serve-theta (FP32 -> FP64 switch
    a decade below), at most --serve-max-sweeps sweeps; a job that reaches
    the cap counts as finished and unconverged.  MAG jobs run the annealing
    protocol of Sec. 6.5 first (--serve-mag-sa simulated-annealing steps T
    1.45 -> 0.01, then stochastic relaxation until theta < 1e-6, at most
    --serve-mag-sr sweeps), since their overrelaxation alone converges slowly
    from a random gauge.  The saturated rate is measured on the first
    --serve-sat-jobs jobs (all submitted at once); the Poisson stream of all
    --serve-jobs jobs then arrives at each --serve-loads fraction of it."""
    import torch

    from paper_1212_5221_gb300 import build, gf, inputs

    build.build_all()
    S = SERVING
    n = args.serve_jobs
    jobs = inputs.poisson_jobs(n, 1.0, S["seed"])  # unit-rate gaps; scaled per load below
    fields = {}
    for j in jobs:
        if j["dims"] not in fields:
            fields[j["dims"]] = inputs.links(j["dims"], "smooth", S["eps"], S["field_seed"])
    foot = {(d, g): gf.gf_footprint(d, 1, g, "mixed") for d in fields for g in ("landau", "coulomb", "mag")}
    free, _ = torch.cuda.mem_get_info()
    arena = int(min(0.6 * free, args.serve_slots * max(foot.values()) * 1.1))
    log(f"serving: {n} jobs, {args.serve_slots} slots, arena {arena / 1e9:.1f} GB")

    def run(rate, n_jobs):
        srv = gf.gf_server_create(arena, args.serve_slots)
        results, t0 = [], time.time()
        try:
            for k, j in enumerate(jobs[:n_jobs]):
                if rate:
                    wait = j["arrival"] / rate - (time.time() - t0)
                    if wait > 0:
                        results += gf.gf_server_poll(srv, 256, int(wait * 1e3))
                        while time.time() - t0 < j["arrival"] / rate:
                            results += gf.gf_server_poll(srv, 256, 1)
                th = args.serve_theta
                ann = None
                if j["gauge"] == "mag" and (args.serve_mag_sa or args.serve_mag_sr):
                    ann = dict(sa_steps=args.serve_mag_sa, T_start=1.45, T_end=0.01, sr_sweeps=args.serve_mag_sr,
                               sr_p=0.5, sr_theta=1e-6, seed=j["seed"])
                gf.gf_server_submit(srv, j["dims"], j["gauge"], "mixed", host_links=fields[j["dims"]],
                                    orbit_seed=j["seed"], tag=k, param=S["omega"][j["gauge"]], theta_target=th,
                                    max_sweeps=args.serve_max_sweeps, check_interval=S["check"],
                                    reunit_interval=S["reunit"], switch_theta=th / 10, anneal=ann)
            while len(results) < n_jobs:
                results += gf.gf_server_poll(srv, 256, 1000)
        finally:
            gf.gf_server_destroy(srv)
        if args.serve_log:
            with open(args.serve_log, "a") as f:
                for r in sorted(results, key=lambda x: x["tag"]):
                    j = jobs[r["tag"]]
                    f.write(json.dumps({"rate": rate, "tag": r["tag"], "dims": j["dims"], "gauge": j["gauge"],
                                        "status": r["status"], "sweeps": r["sweeps"], "theta": r["theta"],
                                        "latency_s": r["t_done"] - r["t_submit"],
                                        "queue_s": r["t_admit"] - r["t_submit"]}) + "\n")
        bad = [r for r in results if r["status"] not in (0, gf.GF_ENOTCONV)]
        if bad:
            raise RuntimeError(f"{len(bad)} jobs failed, first status {bad[0]['status']}")
        t_first = min(r["t_submit"] for r in results)
        span = max(r["t_done"] for r in results) - t_first
        lat = np.array([r["t_done"] - r["t_submit"] for r in results])
        su = float(sum(r["site_updates"] for r in results))
        by_gauge = {}
        for r in results:
            g = jobs[r["tag"]]["gauge"]
            by_gauge.setdefault(g, []).append(r["t_done"] - r["t_submit"])
        return dict(jobs=n_jobs, seconds=span, jobs_per_s=n_jobs / span, site_updates_per_s=su / span,
                    p50_s_by_gauge={g: float(np.percentile(v, 50)) for g, v in by_gauge.items()},
                    p99_s_by_gauge={g: float(np.percentile(v, 99)) for g, v in by_gauge.items()},
                    p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                    mean_s=float(lat.mean()), max_s=float(lat.max()),
                    queue_p50_s=float(np.percentile([r["t_admit"] - r["t_submit"] for r in results], 50)),
                    unconverged=sum(r["status"] == gf.GF_ENOTCONV for r in results),
                    fp64_sweeps=sum(r["sweeps_fp64"] for r in results),
                    sweeps=sum(r["sweeps"] for r in results))

    with Clocks(0) as clocks:
        if args.serve_rate > 0:  # the saturated rate measured before, given
            sat = {"jobs_per_s": args.serve_rate, "given": True}
        else:
            sat = run(0.0, min(args.serve_sat_jobs, n))
        log("saturated:", json.dumps(sat))
        loads = []
        for f in args.serve_loads:
            rate = f * sat["jobs_per_s"]
            r = run(rate, n)
            r.update(load=f, rate_jobs_per_s=rate)
            loads.append(r)
            log("poisson:", json.dumps(r))
    head = loads[0] if loads else sat
    line = {"metric": "job p50/p99 latency (serving)", "value": head["p99_s"], "unit": "s (p99)", "n_gpus": 1,
            "steps": n, "warmup": 0, "ms_per_step": head["seconds"] / n * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": S["name"], "jobs": n, "stream_seed": S["seed"],
                       "lattices": ["16^4", "24^3x48", "32^4", "48^3x96"], "gauges": ["landau", "coulomb", "mag"],
                       "precision": "mixed", "theta_target": args.serve_theta,
                       "max_sweeps": args.serve_max_sweeps, "slots": args.serve_slots, "arena_bytes": arena,
                       "mag_protocol": {"sa_steps": args.serve_mag_sa, "T": [1.45, 0.01],
                                        "sr_sweeps_max": args.serve_mag_sr, "sr_theta": 1e-6},
                       "saturated_prefix_jobs": min(args.serve_sat_jobs, n)},
            "p50_s": head["p50_s"], "p99_s": head["p99_s"], "site_updates_per_s": head["site_updates_per_s"],
            "saturated": sat, "poisson": loads, "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)


def unitarity(V):
    """max and mean of max|U U^dag - 1| per link, and max|det U - 1|, of
    natural-order links (..., 3, 3)."""
    M = V.reshape(-1, 3, 3)
    dev = np.empty(len(M))
    det = np.empty(len(M))
    for a in range(0, len(M), 1 << 20):
        b = M[a:a + (1 << 20)]
        P = np.einsum("nij,nkj->nik", b, b.conj()) - np.eye(3)
        dev[a:a + len(b)] = np.abs(P).reshape(len(b), -1).max(axis=1)
        det[a:a + len(b)] = np.abs(np.linalg.det(b) - 1)
    return float(dev.max()), float(dev.mean()), float(det.max())


def run_precision_study(args):
    """Unitarity drift and functional deviation over 12000 overrelaxation
    iterations of a 32^4 Landau problem (the shapes of Sec. 4.5's two
    figures, on a synthetic field): FP64 with and without re-unitarisation
    every 100 iterations, FP32 (rows re-projected at every load) with and
    without FP64 re-unitarisation every 100, the paper's MP (Step 1 in FP64
    on FP32 links, Step 2 in FP32) with and without it, and GF_MIXED (FP64
    master moved by exact transformations, synced every 100)."""
    from paper_1212_5221_gb300 import build, gf, inputs

    build.build_all()
    dims, n_iter, every = (32, 32, 32, 32), args.study_iters, args.study_every
    U = inputs.links(dims, "smooth", 0.3, 1)
    variants = [("fp64_reunit100", "fp64", True), ("fp64", "fp64", False), ("fp32_reunit100", "fp32", True),
                ("fp32", "fp32", False), ("mp_reunit100", "mp", True), ("mp", "mp", False),
                ("mixed", "mixed", True)]
    V = np.empty(tuple(dims) + (4, 3, 3), np.complex128)
    rows = {}
    for name, prec, reunit in variants:
        h = gf.gf_create(dims, "landau", prec)
        gf.gf_load_links(h, 0, U)
        gf.gf_random_gauge_transform(h, 1000)
        series, done, t_dev = [], 0, 0.0
        while True:
            F, T = gf.gf_functional_theta(h)
            gf.gf_store_links(h, 0, V)
            umax, umean, dmax = unitarity(V)
            series.append({"iter": done, "F": float(F[0]), "theta": float(T[0]), "unitarity_max": umax,
                           "unitarity_mean": umean, "det_max": dmax})
            log(name, json.dumps(series[-1]))
            if done >= n_iter:
                break
            for _ in range(every // 100):
                t0 = time.time()
                gf.gf_sweep(h, "or", 1.7, 100, observables=False)
                if reunit:
                    gf.gf_reunitarize(h)
                gf.gf_synchronize(h)
                t_dev += time.time() - t0
            done += every
        gf.gf_destroy(h)
        rows[name] = {"series": series, "seconds": t_dev}
    ref = {r["iter"]: r["F"] for r in rows["fp64_reunit100"]["series"]}
    for name in rows:
        for r in rows[name]["series"]:
            r["rel_dF_vs_fp64_reunit100"] = abs(r["F"] - ref[r["iter"]]) / abs(ref[r["iter"]])
    print(json.dumps({"study": "precision", "lattice": "32^4", "gauge": "landau", "omega": 1.7,
                      "field": "exp(i 0.3 H), seed 1, Haar g seed 1000", "iterations": n_iter,
                      "variants": rows}), flush=True)


def run_sa_temperature_study(args):
    """Sec. 6.6's temperature scan: simulated annealing of a hot 32^4 field
    (every link a Haar-random SU(3) matrix), 10000 steps (heat bath + three
    microcanonical sweeps each) with T linear from 8 to 0.01, Landau and MAG,
    mixed precision; F and theta recorded every 100 steps.  gf_anneal over a
    chunk of 100 steps continues the same linear schedule exactly."""
    from paper_1212_5221_gb300 import build, gf, inputs

    build.build_all()
    dims, N, chunk = (32, 32, 32, 32), args.study_iters, 100
    T0, T1 = 8.0, 0.01
    temp = lambda k: T0 + (T1 - T0) * k / (N - 1)
    U = inputs.links(dims, "hot", 0.0, 7)
    out = {}
    for gauge in ("landau", "mag"):
        h = gf.gf_create(dims, gauge, "mixed")
        gf.gf_load_links(h, 0, U)
        F, T = gf.gf_functional_theta(h)
        series = [{"step": 0, "T": T0, "F": float(F[0]), "theta": float(T[0])}]
        t0 = time.time()
        for i in range(N // chunk):
            F, T = gf.gf_anneal(h, temp(i * chunk), temp(i * chunk + chunk - 1), chunk, 17)
            series.append({"step": (i + 1) * chunk, "T": temp(i * chunk + chunk - 1), "F": float(F[0]),
                           "theta": float(T[0])})
        dt = time.time() - t0
        gf.gf_destroy(h)
        Fs = np.array([r["F"] for r in series])
        Ts = np.array([r["T"] for r in series])
        dF = np.abs(np.diff(Fs))
        k = int(np.argmax(dF))
        gain = Fs[-1] - Fs[0]
        t10 = float(Ts[np.argmax(Fs - Fs[0] >= 0.1 * gain)])
        t90 = float(Ts[np.argmax(Fs - Fs[0] >= 0.9 * gain)])
        out[gauge] = {"series": series, "seconds": dt, "sweeps": 4 * N,
                      "site_updates_per_s": 4 * N * float(np.prod(dims)) / dt,
                      "T_steepest": float(0.5 * (Ts[k] + Ts[k + 1])), "T_10pct_gain": t10, "T_90pct_gain": t90}
        log(gauge, json.dumps({k2: v for k2, v in out[gauge].items() if k2 != "series"}))
    print(json.dumps({"study": "sa_temperature", "lattice": "32^4", "field": "hot (Haar links), seed 7",
                      "steps": N, "T": [T0, T1], "precision": "mixed", "gauges": out}), flush=True)


def run_fullsize_study(args):
    """The 64^3 x 256 lattice (67M sites; eps = 0.3, seed 2, Haar g seed 2):
    sweep throughput of Landau and Coulomb (256 time-slices in every launch)
    in FP32, GF_MIXED and FP64, and a mixed-precision Coulomb fix to
    theta < 1e-12 per slice (slices stop individually), at most
    --study-iters sweeps.  The links are generated and loaded in slabs of 16
    time-slices."""
    import torch

    from paper_1212_5221_gb300 import build, gf, inputs

    build.build_all()
    dims = (256, 64, 64, 64)
    V = float(np.prod(dims))

    # the natural-order FP64 field (38.7 GB) generated once, slab by slab, into device memory
    dev = torch.device("cuda", 0)
    per_t = 64 ** 3 * 4 * 18
    src = torch.empty(dims[0] * per_t, dtype=torch.float64, device=dev)
    for t0 in range(0, dims[0], 16):
        slab = inputs.links(dims, "smooth", 0.3, 2, t0=t0, nt=16)
        src[t0 * per_t:(t0 + 16) * per_t].copy_(torch.from_numpy(slab.view(np.float64).reshape(-1)))
    torch.cuda.synchronize()

    def load(h):
        gf.gf_load_links_device(h, 0, src.data_ptr())
        gf.gf_random_gauge_transform(h, 2)

    out = {"lattice": "64^3x256", "throughput": {}}
    for gauge in ("landau", "coulomb"):
        for prec in ("fp32", "mixed", "fp64"):
            need = gf.gf_footprint(dims, 1, gauge, prec)
            if torch.cuda.mem_get_info()[0] < need + (4 << 30):
                out["throughput"][f"{gauge}_{prec}"] = {"skipped": f"needs {need / 1e9:.1f} GB"}
                continue
            h = gf.gf_create(dims, gauge, prec)
            load(h)
            gf.gf_sweep(h, "or", 1.7, 2, observables=False)
            gf.gf_set_profiling(h, True)
            n = 10 if prec != "fp64" else 3
            gf.gf_sweep(h, "or", 1.7, n, observables=False)
            kind = 1 if prec == "fp64" else 0
            nl, ms = gf.gf_kernel_stats(h, kind)
            sweep_ms = ms / nl * 2
            bpsu = {"fp32": 768, "mixed": 864, "fp64": 1536}[prec]
            if gauge == "coulomb":
                bpsu = bpsu * 7 // 8  # six spatial links + the accumulated g
            out["throughput"][f"{gauge}_{prec}"] = {
                "ms_per_sweep": sweep_ms, "site_updates_per_s": V / (sweep_ms / 1e3),
                "hbm_gbs": V * bpsu / (sweep_ms / 1e3) / 1e9, "footprint_gb": need / 1e9}
            log(gauge, prec, json.dumps(out["throughput"][f"{gauge}_{prec}"]))
            gf.gf_destroy(h)
    h = gf.gf_create(dims, "coulomb", "mixed")
    load(h)
    t0 = time.time()
    r = gf.gf_fix(h, "or", 1.7, 1e-12, max_sweeps=args.study_iters, check_interval=20, reunit_interval=100,
                  switch_theta=1e-13, raise_on_notconv=False)
    dt = time.time() - t0
    Ft, Tt = gf.gf_slice_functional_theta(h)
    gf.gf_destroy(h)
    out["coulomb_fix_mixed"] = {"seconds": dt, "sweeps": r["sweeps"], "sweeps_fp32": r["sweeps_fp32"],
                                "sweeps_fp64": r["sweeps_fp64"], "converged": r["converged"],
                                "site_updates_per_s": r["site_updates"] / dt,
                                "slices_below_1e-12": int((Tt[0] < 1e-12).sum()), "theta_max": float(Tt[0].max()),
                                "F_mean": float(Ft[0].mean())}
    log("coulomb fix", json.dumps(out["coulomb_fix_mixed"]))
    print(json.dumps({"study": "fullsize", **out}), flush=True)


def run_config3_study(args):
    """The 64^3 x 256 lattice fixed as stated (eps = 0.3, seed 2, Haar g seed
    2): Coulomb gauge as 256 time-slices in every launch (each slice stops on
    its own) and Landau gauge, both GF_MIXED with the switch to FP64 sweeps at
    theta < 1e-8 and the FP64 sweeps continuing to theta < 1e-12; per-check
    JSON lines go to gpurun_out/ when that folder exists."""
    import torch

    from paper_1212_5221_gb300 import build, gf, inputs

    build.build_all()
    dims = (256, 64, 64, 64)
    per_t = 64 ** 3 * 4 * 18
    dev = torch.device("cuda", 0)
    src = torch.empty(dims[0] * per_t, dtype=torch.float64, device=dev)
    for t0 in range(0, dims[0], 16):
        slab = inputs.links(dims, "smooth", 0.3, 2, t0=t0, nt=16)
        src[t0 * per_t:(t0 + 16) * per_t].copy_(torch.from_numpy(slab.view(np.float64).reshape(-1)))
    torch.cuda.synchronize()
    out = {"lattice": "64^3x256", "switch_theta": 1e-8, "theta_target": 1e-12}
    logdir = os.path.join(ROOT, "gpurun_out")
    runs = [("coulomb", 1.7), ("landau", args.config3_omega)]
    for gauge, omega in [r for r in runs if r[0] in args.config3_gauges.split(",")]:
        cap = args.study_iters
        h = gf.gf_create(dims, gauge, "mixed")
        if os.path.isdir(logdir):
            gf.gf_set_check_log(h, os.path.join(logdir, f"config3_{gauge}_checks.jsonl"))
        gf.gf_load_links_device(h, 0, src.data_ptr())
        gf.gf_random_gauge_transform(h, 2)
        r = gf.gf_fix(h, "or", omega, 1e-12, max_sweeps=cap, check_interval=20, reunit_interval=100,
                      switch_theta=1e-8, raise_on_notconv=False)
        Ft, Tt = gf.gf_slice_functional_theta(h)
        F, T = gf.gf_functional_theta(h)
        gf.gf_destroy(h)
        out[gauge] = {"omega": omega, "seconds": r["seconds"], "sweeps": r["sweeps"],
                      "sweeps_fp32": r["sweeps_fp32"], "sweeps_fp64": r["sweeps_fp64"],
                      "converged": r["converged"], "site_updates_per_s": r["site_updates"] / r["seconds"],
                      "F": float(F[0]), "theta": float(T[0]), "theta_slice_max": float(Tt[0].max()),
                      "slices_below_1e-12": int((Tt[0] < 1e-12).sum())}
        log("config3", gauge, json.dumps(out[gauge]))
    print(json.dumps({"study": "config3", **out}), flush=True)


def run_config4_study(args):
    """Sec. 6.5's protocol on 16 Gribov copies per lattice (MAG, 24^4 and
    32^4, eps = 0.3 field seed 3, copy k on the orbit point of Haar seed
    3000 + k, all copies in one batched context): simulated annealing T 1.45 ->
    0.01 over 3000 steps (heat bath + three microcanonical sweeps each), at
    most 2000 stochastic-relaxation sweeps (p = 0.5, a copy leaves at theta <
    1e-6), then overrelaxation omega = 1.35 to theta < 1e-12 in GF_MIXED
    (FP64 below 1e-8); the best functional is kept."""
    from paper_1212_5221_gb300 import build, gf, inputs

    build.build_all()
    out = {}
    for dims in ((24, 24, 24, 24), (32, 32, 32, 32)):
        U = inputs.links(dims, "smooth", 0.3, 3)
        n = 16
        h = gf.gf_create_batch(dims, n, "mag", "mixed")
        gf.gf_load_links(h, -1, U)
        gf.gf_set_copy_base(h, 3000)
        gf.gf_random_gauge_transform(h, 3000)
        r = gf.gf_protocol(h, args.config4_sa_steps, 1.45, 0.01, sr_sweeps=2000, sr_p=0.5, sr_theta=1e-6,
                           seed=4, omega=1.35, theta_target=1e-12, max_sweeps=args.study_iters,
                           check_interval=20, reunit_interval=100, switch_theta=1e-8, raise_on_notconv=False)
        F, T = gf.gf_functional_theta(h)
        gf.gf_destroy(h)
        key = "x".join(map(str, dims))
        out[key] = {"copies": n, "seconds": r["seconds"], "sweeps": r["sweeps"], "sweeps_fp32": r["sweeps_fp32"],
                    "sweeps_fp64": r["sweeps_fp64"], "converged": r["converged"],
                    "copies_below_1e-12": int((T < 1e-12).sum()), "theta_max": float(T.max()),
                    "F_best": float(F.max()), "F_copies": [float(x) for x in F],
                    "site_updates_per_s": r["site_updates"] / r["seconds"]}
        log("config4", key, json.dumps(out[key]))
    print(json.dumps({"study": "config4", "gauge": "mag", "sa_steps": args.config4_sa_steps, **out}), flush=True)


def run_group_study(args):
    """Small lattices of different extents (32 Landau lattices from 8^4 to
    16^4, FP32 storage, eps = 0.4): overrelaxation sweeps of every lattice
    on its own context and stream (the launches of all contexts overlap on
    the device) against gf_group_sweep, one launch per half-sweep for all of
    them; site-updates/s and launches per sweep of each."""
    import torch

    from paper_1212_5221_gb300 import build, gf, inputs

    build.build_all()
    specs = ([(8, 8, 8, 8)] * 8 + [(12, 12, 12, 12)] * 8 + [(16, 16, 16, 16)] * 8 + [(8, 8, 8, 16)] * 4 +
             [(16, 12, 12, 12)] * 4)
    n = args.study_iters
    hs = [gf.gf_create(d, "landau", "fp32") for d in specs]
    for k, (h, d) in enumerate(zip(hs, specs)):
        gf.gf_load_links(h, 0, inputs.links(d, "smooth", 0.4, k))
    sites = float(sum(np.prod(d) for d in specs))
    out = {"lattices": len(specs), "sites": sites, "sweeps": n}
    for mode in ("alone", "group"):
        for rep in range(2):  # the first pass warms up (graphs, autotuned shapes)
            n0 = sum(gf.gf_launch_count(h) for h in hs)
            torch.cuda.synchronize()
            t0 = time.time()
            if mode == "alone":
                for h in hs:
                    gf.gf_sweep_async(h, "or", 1.7, n)
                for h in hs:
                    gf.gf_synchronize(h)
            else:
                gf.gf_group_sweep(hs, "or", 1.7, n)
            torch.cuda.synchronize()
            dt = time.time() - t0
            launches = sum(gf.gf_launch_count(h) for h in hs) - n0
        out[mode] = {"seconds": dt, "site_updates_per_s": n * sites / dt, "launches_per_sweep": launches / n}
        log("group study", mode, json.dumps(out[mode]))
    for h in hs:
        gf.gf_destroy(h)
    out["speedup_group_vs_alone"] = out["group"]["site_updates_per_s"] / out["alone"]["site_updates_per_s"]
    print(json.dumps({"study": "group", **out}), flush=True)


def run_slab(args, rank, world, local_rank):
    """One lattice split into time slabs over the ranks (Sec. 5; one process
    per GPU under torchrun, NCCL boundary exchange after every half-sweep):
    the 32^3x64 workload's field at the orbit point of seed 1000, --slab-sweeps
    overrelaxation sweeps (omega 1.7) in --slab-precision storage, timed with
    CUDA events between barriers; rank 0 prints one JSON line (strong
    scaling: the lattice is fixed, the ranks share it)."""
    import torch

    from paper_1212_5221_gb300 import build, gf, inputs, slab

    build.build_all()
    W = WORKLOAD
    dims = W["dims"]
    t0, nt = slab.slab_bounds(dims[0], world, rank)
    U = inputs.links(dims, "smooth", W["eps"], W["field_seed"])
    s = slab.GpuSlab(dims, t0, nt, W["gauge"], args.slab_precision)
    h = gf.gf_create(dims, W["gauge"], "fp64")  # the orbit point, made once on this rank's GPU
    gf.gf_load_links(h, 0, U)
    gf.gf_random_gauge_transform(h, 1000)
    gf.gf_store_links(h, 0, U)
    gf.gf_destroy(h)
    s.load(U)
    ts = slab.TimeSlab(s, slab.Ring(), nt, dims[0], W["gauge"])
    ts.sweep("or", W["omega"], 2)  # warm-up
    dist = torch.distributed.is_initialized()
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(s.stream)
    ts.sweep("or", W["omega"], args.slab_sweeps)
    stop.record(s.stream)
    torch.cuda.synchronize()
    elapsed = start.elapsed_time(stop) / 1e3
    F, theta = ts.functional_theta()
    elapsed_all, su_all = reduce_over_ranks(elapsed, float(nt * np.prod(dims[1:]) * args.slab_sweeps),
                                            torch.device("cuda", local_rank) if dist else None)
    s.close()
    if rank == 0:
        print(json.dumps({"metric": "site-updates/s (one lattice in time slabs)", "value": su_all / elapsed_all,
                          "unit": "site-updates/s", "n_gpus": world, "steps": args.slab_sweeps, "warmup": 2,
                          "ms_per_step": elapsed_all / args.slab_sweeps * 1e3, "higher_is_better": True,
                          "scaling": "strong", "dtype": "f64" if args.slab_precision == "fp64" else "f32",
                          "data": "synthetic", "F": F, "theta": theta,
                          "config": {"workload": "landau_or_32c3x64_timeslabs", "slabs": world, "slices_per_slab": nt,
                                     "precision": args.slab_precision, "omega": W["omega"]}}), flush=True)


def run_kernel_target(args):
    """Short, fixed launch sequences on the workload's lattice for ncu captures.
    fp32 / fp64 / mixed: 3 sweeps in that precision (mixed: FP32 sweeps that
    accumulate g); mag64 / mag32: the same in MAG gauge (omega 1.35) in FP64 /
    GF_MIXED storage; check32: 3 mixed FP32 sweeps of which the last sums F
    and theta (the fused check) and the read-only pass over the even sites.
    window: a bounded slice of one bench step -- 100 mixed FP32 sweeps with
    theta checks every 20 and a master sync at 100, the switch to the FP64
    master, and 60 FP64 sweeps with checks."""
    from paper_1212_5221_gb300 import build, gf, inputs

    build.build_all()
    W = WORKLOAD
    dims = W["dims"]
    U = inputs.links(dims, "smooth", W["eps"], W["field_seed"])
    kt = args.kernel_target
    prec = {"window": "mixed", "mag64": "fp64", "mag32": "mixed", "check32": "mixed"}.get(kt, kt)
    gauge = "mag" if kt.startswith("mag") else W["gauge"]
    omega = 1.35 if gauge == "mag" else W["omega"]
    h = gf.gf_create(dims, gauge, prec)
    gf.gf_load_links(h, 0, U)
    gf.gf_random_gauge_transform(h, 1000)
    if args.kernel_target == "window":
        kw = dict(algo="or", param=W["omega"], theta_target=W["theta"], check_interval=W["check"],
                  reunit_interval=W["reunit"], switch_theta=W["switch_theta"], raise_on_notconv=False)
        gf.gf_fix(h, max_sweeps=100, **kw)
        gf.gf_promote(h)
        gf.gf_fix(h, max_sweeps=60, **kw)
    elif kt == "check32":
        gf.gf_fix(h, "or", omega, 1e-30, max_sweeps=3, check_interval=3, reunit_interval=0,
                  switch_theta=1e-40, raise_on_notconv=False)
    else:
        gf.gf_sweep(h, "or", omega, 3, observables=False)
    F, T = gf.gf_functional_theta(h)
    gf.gf_destroy(h)
    print(json.dumps({"kernel_target": args.kernel_target, "F": float(F[0]), "theta": float(T[0])}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64", "fp32"], default="mixed")
    ap.add_argument("--switch-theta", type=float, default=WORKLOAD["switch_theta"])
    ap.add_argument("--max-sweeps", type=int, default=40000)
    ap.add_argument("--deep-switch", type=float, default=1e-13,
                    help="also time one mixed run with the FP32 -> FP64 switch at this theta (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=3,
                    help="end-to-end steps through host buffers, on the orbit seeds of the first timed steps")
    ap.add_argument("--fp64-matched", type=int, default=3,
                    help="plain-FP64 runs on the orbit seeds of the first timed steps (time-to-theta ratio)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-fp64-baseline", dest="fp64_baseline", action="store_false")
    ap.add_argument("--kernel-target", choices=["fp32", "fp64", "mixed", "window", "mag64", "mag32", "check32"],
                    default=None,
                    help="only run a short, fixed launch sequence of the workload (for ncu)")
    ap.add_argument("--serving", action="store_true", help="run the serving workload (job p50/p99)")
    ap.add_argument("--slab", action="store_true",
                    help="one lattice in time slabs over the ranks (strong scaling) instead of replicas")
    ap.add_argument("--slab-sweeps", type=int, default=200)
    ap.add_argument("--slab-precision", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--serve-jobs", type=int, default=2000)
    ap.add_argument("--serve-theta", type=float, default=1e-10)
    ap.add_argument("--serve-max-sweeps", type=int, default=20000)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-sat-jobs", type=int, default=100, help="jobs of the saturated-rate run")
    ap.add_argument("--serve-rate", type=float, default=0.0,
                    help="a saturated rate (jobs/s) measured before: skips the saturated run")
    ap.add_argument("--serve-log", default=None, help="append one JSON line per job to this file")
    ap.add_argument("--serve-mag-sa", type=int, default=300, help="annealing steps of a MAG job")
    ap.add_argument("--serve-mag-sr", type=int, default=1000, help="most stochastic-relaxation sweeps of a MAG job")
    ap.add_argument("--serve-loads", type=lambda v: [float(x) for x in v.split(",") if x], default=[0.7],
                    help="Poisson rates as fractions of the measured saturated job rate")
    ap.add_argument("--study", choices=["precision", "sa-temperature", "fullsize", "config3", "config4", "group"],
                    default=None,
                    help="run a report study instead of the benchmark")
    ap.add_argument("--study-iters", type=int, default=None)
    ap.add_argument("--study-every", type=int, default=2000)
    ap.add_argument("--config3-omega", type=float, default=1.7,
                    help="overrelaxation parameter of the 64^3x256 Landau fix (Coulomb uses 1.7)")
    ap.add_argument("--config3-gauges", default="coulomb,landau", help="which config-3 fixes to run")
    ap.add_argument("--config4-sa-steps", type=int, default=3000)
    args = ap.parse_args()
    if args.study == "precision":
        args.study_iters = args.study_iters or 12000
        run_precision_study(args)
        return
    if args.study == "fullsize":
        args.study_iters = args.study_iters or 8000
        run_fullsize_study(args)
        return
    if args.study == "group":
        args.study_iters = args.study_iters or 200
        run_group_study(args)
        return
    if args.study == "config3":
        args.study_iters = args.study_iters or 30000
        run_config3_study(args)
        return
    if args.study == "config4":
        args.study_iters = args.study_iters or 40000
        run_config4_study(args)
        return
    if args.study == "sa-temperature":
        args.study_iters = args.study_iters or 10000
        run_sa_temperature_study(args)
        return
    if args.kernel_target:
        run_kernel_target(args)
        return
    if args.serving:
        run_serving(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if args.slab:
        run_slab(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
