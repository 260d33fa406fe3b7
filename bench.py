#!/usr/bin/env python
"""Throughput of the lattice path-integral Coulomb sampler on one node.

Workload (one step): one measured compound sweep -- 1 heatbath pass (Eq. (phi))
+ 3 over-relaxation passes, each pass a red and a black half-sweep -- of 64
independent chains of a 128^3 Dirichlet lattice (FP32 field), followed by the
Eq. (nsum2) sample of N = 4096 charges q = +-1 (zero net charge, seeded random
distinct sites) with FP64 sums.  Metric: site-updates/s = 64 * 128^3 * 4 per
step / time.  Under torchrun each rank runs its own 64 chains (own seed): weak
scaling, no collective on the data path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only reference this method
has) on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

L = 128
N_CHARGES = 4096
N_CHAINS = 64
N_HB, N_OR = 1, 3
PASSES = N_HB + N_OR
SITES_PER_STEP = N_CHAINS * L ** 3 * PASSES
METRIC = "site-updates/s"
CONFIG = {
    "workload": "128^3 Dirichlet lattice, N=4096 charges q=+-1 zero net at seeded random distinct "
                "sites, 64 independent chains, FP32 field with FP64 estimator sums, "
                "1 heatbath : 3 over-relaxation, one sample per compound sweep",
    "lattice": [L, L, L], "n_charges": N_CHARGES, "n_chains_per_gpu": N_CHAINS,
    "n_hb": N_HB, "n_or": N_OR,
    "l2": "inputs larger than L2 (512 MiB of fields per GPU vs 126 MB L2); no flush",
}
PROFILE_TRAFFIC = ROOT / "profiles" / "or_halfsweep_128c_64ch.txt"
KERNEL_SOURCES = ["sweep.cu", "device_common.cuh", "internal.h"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--workload", choices=["chains128", "large512", "sweep", "batched"],
                    default="chains128", help="secondary workloads print their own line")
    ap.add_argument("--chains", type=int, default=N_CHAINS,
                    help="chains per GPU (smaller values only for profiler captures)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# --------------------------------------------------------------------------
class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_src_hash():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update((ROOT / "paper_1403_0711_gb300" / "csrc" / name).read_bytes())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per over-relaxation launch from the committed ncu summary,
    or None if the kernel sources changed since it was taken."""
    if not PROFILE_TRAFFIC.exists():
        return None
    kv = {}
    for ln in PROFILE_TRAFFIC.read_text().splitlines():
        if ":" in ln and not ln.startswith("#"):
            k, v = ln.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_src_sha256_16") != kernel_src_hash():
        return None
    try:
        return float(kv["dram_bytes_per_launch_full"])
    except (KeyError, ValueError):
        return None


def golden_e_lat(name):
    """Exact lattice energy of a seeded workload (tests/golden/e_lat.txt, written
    by tests/golden/make_golden.py from the FP64 oracle)."""
    for ln in (ROOT / "tests" / "golden" / "e_lat.txt").read_text().splitlines():
        if ln.startswith(name + " "):
            return float(ln.split()[8])
    return None


def time_to_accuracy(est, seconds, world, eps=1e-3, name="bench_128c_n4096_pm"):
    """Projected wall time to a batch-means error of eps |E_lat|: the timed run
    reached est['stderr'] in `seconds` (all GPUs), and the error falls as
    1/sqrt(time)."""
    e_lat = golden_e_lat(name)
    if not e_lat or not (est.get("stderr") or 0) > 0:
        return None
    t = seconds * (est["stderr"] / (eps * abs(e_lat))) ** 2
    return {"eps": eps, "e_lat": e_lat, "mean": est["mean"], "stderr": est["stderr"],
            "tau_int": est["tau_int"], "samples": est["n"] * world,
            "delta": abs(est["mean"] - e_lat) / abs(e_lat),
            "projected_seconds": t, "projected_hours": t / 3600.0,
            "estimator": "plain, batch means over all chains"}


# --------------------------------------------------------------------------
def cpu_oracle_rate(seconds, Lz=L):
    """Site-updates/s of the FP64 oracle on one chain of a 128 x 128 x Lz box,
    compound sweeps (1 HB + 3 OR) plus the sample, for about `seconds`."""
    from oracle import oracle
    from paper_1403_0711_gb300 import inputs
    oracle.build()
    box = (L, L, Lz)
    sites, q = inputs.plus_minus(box, min(N_CHARGES, (L * L * Lz) // 2 * 2), seed=1)
    ch = oracle.Chain(box, seed=20140303)
    n = 0
    t0 = time.perf_counter()
    while True:
        ch.run(1, N_HB, N_OR, sites, q)
        n += 1
        dt = time.perf_counter() - t0
        if dt >= seconds:
            break
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return L * L * Lz * PASSES * n / dt, cores, n


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle
    from paper_1403_0711_gb300 import inputs
    oracle.build()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    # size the per-step sample so that warm-up + timed steps take ~150 s
    probe = oracle.Chain((L, L, 16), seed=1)
    t0 = time.perf_counter()
    probe.run(1, N_HB, N_OR)
    t_site = (time.perf_counter() - t0) / (L * L * 16)
    budget = 150.0 / max(1, args.steps + args.warmup)
    Lz = int(max(2, min(L, budget / (t_site * L * L))))
    box = (L, L, Lz)
    sites, q = inputs.plus_minus(box, min(N_CHARGES, (L * L * Lz) // 2 * 2), seed=1)
    ch = oracle.Chain(box, seed=20140303)
    for _ in range(args.warmup):
        ch.run(1, N_HB, N_OR, sites, q)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ch.run(1, N_HB, N_OR, sites, q)
    dt = time.perf_counter() - t0
    value = L * L * Lz * PASSES * args.steps / dt
    sample = (f"one chain, one compound sweep (1 HB + 3 OR) + Eq. (nsum2) sample per step on a "
              f"{L}x{L}x{Lz} slab of the workload's lattice, FP64 oracle")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "site-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": CONFIG,
        "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    n_chains = args.chains
    sites_per_step = n_chains * L ** 3 * PASSES

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1403_0711_gb300 import _build, coulps, inputs
    if rank == 0:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    coulps.load()
    coulps.use_torch_allocator()
    stream = torch.cuda.Stream()
    box = (L, L, L)
    sites, q = inputs.plus_minus(box, N_CHARGES, seed=1)
    lat = coulps.Lattice(box, n_chains=n_chains, precision=coulps.F32, seed=20140303 + 7919 * rank,
                         stream=stream)
    ch = coulps.Charges(lat, sites, q)

    def step():
        # one measured compound sweep; the sample is gathered by its last half-sweep
        ch.run(0, 1, N_HB, N_OR)

    lat.set_profiling(True)
    for _ in range(args.warmup):
        step()
    lat.sync()
    lat.kernel_times()  # discard warm-up timings
    ch.reset_stats()  # the timed samples alone feed the time-to-accuracy projection

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)  # let the sampler start
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    ms = ev0.elapsed_time(ev1)
    kt = lat.kernel_times()
    lat.sync()
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * sites_per_step * args.steps / (ms_max / 1e3)
    est_timed = ch.estimate()
    tta = time_to_accuracy(est_timed, ms_max / 1e3, world)

    # roofline of the dominant kernel: the over-relaxation half-sweep
    # (3 of the 4 passes; 12 B per updated site: read other colour, read own, write own)
    or_ms = kt["or_ms"] / max(1, kt["or_n"])
    hb_ms = kt["hb_ms"] / max(1, kt["hb_n"])
    sites_per_launch = n_chains * L ** 3 // 2
    or_bytes = 12 * sites_per_launch
    hb_bytes = 8 * sites_per_launch
    peak, peak_kind = measured_peaks()
    achieved = or_bytes / (or_ms / 1e3) / 1e9
    traffic = profiled_traffic()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "halfsweep_kernel<float, over-relaxation>",
                "algorithmic_bytes_per_launch": or_bytes, "avg_launch_ms": or_ms,
                "peak_kind": f"{peak_kind} (burst copy)",
                "heatbath_halfsweep": {"avg_launch_ms": hb_ms,
                                       "achieved_gbs": hb_bytes / (hb_ms / 1e3) / 1e9,
                                       "algorithmic_bytes_per_launch": hb_bytes}}

    # end to end through the C ABI with host buffers: upload the charge set
    # from host memory, one measured compound sweep (graph replay), read back
    # the per-chain estimator state
    lat.set_profiling(False)
    ch.reset_stats()
    ch.update(sites, q)  # allocate the pinned staging buffers outside the timed region
    ch.run(0, 1, N_HB, N_OR)  # capture the graph outside the timed region
    ch.estimate()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ch.update(sites, q)
        ch.run(0, 1, N_HB, N_OR)
        est = ch.estimate()
    e2e_s = time.perf_counter() - t0
    t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    e2e_s = float(t.item())
    e2e = {"value": world * sites_per_step * args.e2e_steps / e2e_s, "unit": "site-updates/s",
           "h2d_bytes_per_step": N_CHARGES * (4 + 8),
           "d2h_bytes_per_step": n_chains * coulps.STAT_STRIDE * 8 + 4,
           "steps": args.e2e_steps,
           "path": "coulps_charges_update + coulps_run(0, 1, 1, 3) + coulps_estimate"}

    out = None
    if rank == 0:
        launches = args.steps * (2 * PASSES + 1 + 1)  # half-sweeps, pass counter, finalize
        line = {
            "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": dict(CONFIG, parallelism=f"replicas{world}", n_chains_per_gpu=n_chains),
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "time_to_1e-3": tta, "estimate_after_e2e": est,
        }
        if world == 1:
            rate, cores, n = cpu_oracle_rate(args.cpu_seconds)
            line["cpu_baseline"] = {
                "value": rate, "unit": "site-updates/s", "cores": cores, "kind": "oracle",
                "sample": f"{n} compound sweeps (1 HB + 3 OR) + samples of one 128^3 chain, "
                          "FP64 oracle, OpenMP over z planes"}
        out = line
    ch.close()
    lat.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


def run_extra(args):
    """Secondary workloads (single GPU; not the headline line):
    large512  512^3, N = 10^6 charges in 200 Gaussian blobs, 1 chain;
    sweep     128^3 .. 512^3 at the fixed charge density N / L^3 = 0.00745;
    batched   256 systems, edges from {32,48,64,80,96}, N log-uniform in [64, 2048]."""
    import torch

    from paper_1403_0711_gb300 import _build, coulps, inputs
    _build.build()
    coulps.load()
    coulps.use_torch_allocator()
    stream = torch.cuda.Stream()
    results = []

    def timed(step, sites_per_step, steps, warmup):
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        return sites_per_step * steps / (ms / 1e3), ms / steps

    if args.workload in ("large512", "sweep"):
        sizes = [512] if args.workload == "large512" else [128, 256, 384, 512]
        for n in sizes:
            box = (n, n, n)
            nq = 1_000_000 if n == 512 else int(round(0.00745 * n ** 3))
            sites, q = inputs.blobs(box, nq, seed=3)
            lat = coulps.Lattice(box, n_chains=1, precision=coulps.F32, seed=77, stream=stream)
            ch = coulps.Charges(lat, sites, q)
            steps = max(20, min(args.steps, int(2e10 / n ** 3)))
            rate, ms = timed(lambda: ch.run(0, 1, N_HB, N_OR), n ** 3 * PASSES, steps, 5)
            results.append({"L": n, "n_charges": nq, "site_updates_per_s": rate, "ms_per_step": ms,
                            "algorithmic_GBps": rate / PASSES * (8 + 12 * N_OR) / N_HB / 1e9
                            if N_HB == 1 else None})
            ch.close()
            lat.close()
    elif args.workload == "batched":
        systems = inputs.batch_systems(256, seed=7)
        b = coulps.Batch([L_ for L_, _, _ in systems], precision=coulps.F32, seed=77, stream=stream)
        b.set_charges([(s_, q_) for _, s_, q_ in systems])
        info = b.info()
        rate, ms = timed(lambda: b.run(0, 1, N_HB, N_OR), info["sites"] * PASSES, args.steps, 10)
        results.append({"systems": 256, "sites": info["sites"], "tiles": info["tiles"],
                        "persistent_ctas": info["grid"], "site_updates_per_s": rate,
                        "ms_per_step": ms,
                        "algorithmic_GBps": rate / PASSES * (8 + 12 * N_OR) / 1e9})
        b.close()
    print(json.dumps({"workload": args.workload, "metric": METRIC, "results": results}), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload != "chains128":
        run_extra(a)
    else:
        run_ours(a)
