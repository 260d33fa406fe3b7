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
    "l2": "inputs larger than L2 (512 MiB of fields per GPU, and its second copy, vs 126 MB L2); no flush",
}
PROFILE_TRAFFIC = {
    "pass_kernel<float, over-relaxation>": ROOT / "profiles" / "pass_or_128c_64ch.txt",
    "pair_kernel<float, over-relaxation, over-relaxation>":
        ROOT / "profiles" / "pair_or_128c_64ch.txt",
    "halfsweep_kernel<float, heatbath>": ROOT / "profiles" / "heatbath_halfsweep_128c_64ch.txt",
}
KERNEL_SOURCES = ["sweep.cu", "pass_fused.cu", "pass_pair.cu", "tile_march.cuh", "pass_march.cuh",
                  "pair_march.cuh",
                  "device_common.cuh", "internal.h"]
FUSED_MODES = {"off": 0, "on": 1, "all": 2, "pairs": 3, "allpairs": 4}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--schedule", choices=["aligned", "shifted", "phased"], default="aligned",
                    help="shifted: with two streams the odd chains run half a compound sweep "
                         "behind (coulps_set_schedule; measured 0.748 against 0.735 ms per "
                         "step aligned: a pass-pair CTA leaves no room for a heatbath CTA "
                         "on its SM)")
    ap.add_argument("--streams", type=int, choices=[1, 2, 3, 4], default=2,
                    help="chain k on stream k %% n (coulps_set_streams)")
    ap.add_argument("--fused", choices=["pairs", "allpairs", "on", "all", "off"], default="pairs",
                    help="fused passes (ping-pong field copies): over-relaxation passes two per "
                         "kernel (pairs, the default), all passes two per kernel (allpairs), "
                         "over-relaxation passes one per kernel (on), all passes one per kernel "
                         "(all), or none")
    ap.add_argument("--repeats", type=int, default=5,
                    help="timed repetitions of the step loop after the timed region (spread)")
    ap.add_argument("--extras", choices=["on", "off"], default="on",
                    help="secondary configurations in the headline line (256 systems, 512^3, "
                         "learned control variate on the q = 1 cube)")
    ap.add_argument("--cv-steps", type=int, default=800, help="training steps of the learned CV")
    ap.add_argument("--gcv-radius", type=int, default=1,
                    help="local term of P in the global control variate, kernel radius "
                         "(0: Q term only; measured time to 1e-3 on the headline system: "
                         "398 s at R = 0, 187 s at R = 1, 257 s at R = 2)")
    ap.add_argument("--gcv-steps", type=int, default=3000,
                    help="headline run: compound sweeps with the global control variate (0: skip)")
    ap.add_argument("--cv-rounds", type=int, default=64)
    ap.add_argument("--cube-seconds", type=float, default=600.0)
    ap.add_argument("--cv-halo", type=int, default=3,
                    help="the localized control variate's g lives within this many sites of the charges")
    ap.add_argument("--cv-collect", type=int, default=512,
                    help="training rounds (every chain contributes one sample per round)")
    ap.add_argument("--cv-global", action="store_true",
                    help="also run the whole-lattice control variate on the +-1 system")
    ap.add_argument("--batch-fused", type=int, choices=[0, 1, 2, 3], default=None,
                    help="many-system fused mode (coulps_batch_set_fused; default: the library's)")
    ap.add_argument("--workload", choices=["chains128", "large512", "sweep", "batched", "batched_tta",
                                           "cv", "cube",
                                           "cv_eval", "paper", "gcv", "offlattice"],
                    default="chains128", help="secondary workloads print their own line")
    ap.add_argument("--off-seconds", type=float, default=120.0,
                    help="sampling time limit of the off-lattice workload")
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


def profiled_traffic(kernel, key="dram_bytes_per_launch_full"):
    """DRAM bytes per launch of `kernel` (or another per-launch figure, `key`)
    from the committed ncu summary, or None if it holds another kernel or the
    kernel sources changed since it was taken."""
    path = PROFILE_TRAFFIC.get(kernel)
    if path is None or not path.exists():
        return None
    kv = {}
    for ln in path.read_text().splitlines():
        if ":" in ln and not ln.startswith("#"):
            k, v = ln.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_src_sha256_16") != kernel_src_hash() or kv.get("kernel") != kernel:
        return None
    try:
        return float(kv[key])
    except (KeyError, ValueError):
        return None


def golden_e_lat(name, column=8):
    """Exact lattice energy of a seeded workload (tests/golden/e_lat.txt, written
    by tests/golden/make_golden.py from the FP64 oracle); column 9 is the
    continuum Eq. (s1) of the same charges."""
    for ln in (ROOT / "tests" / "golden" / "e_lat.txt").read_text().splitlines():
        if ln.startswith(name + " "):
            return float(ln.split()[column])
    return None


def gcv_time_to_accuracy(args, stream):
    """Time to 1e-3 |E_lat| on the headline system (128^3, 64 chains, N = 4096
    charges +-1, 1 HB : 3 OR) with the global control variate g = Q h (h from
    SOR on A h = -rho, set up on the device), measured directly: sample with
    the control variate recorded every compound sweep until its batch-means
    error reaches 1e-3 |E_lat| (or --cube-seconds).  The plain estimator of the
    same samples gives the variance ratio and its own projected time."""
    import torch

    from paper_1403_0711_gb300 import coulps, inputs
    box = (L, L, L)
    sites, q = inputs.plus_minus(box, N_CHARGES, seed=1)
    e_lat = golden_e_lat("bench_128c_n4096_pm")
    target = 1e-3 * abs(e_lat)
    lat = coulps.Lattice(box, n_chains=N_CHAINS, precision=coulps.F32, seed=20140303, stream=stream)
    ch = coulps.Charges(lat, sites, q)
    lat.sweep(300, N_HB, N_OR)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = coulps.GlobalCV(ch, R=args.gcv_radius)
    t_setup = time.perf_counter() - t0
    info = g.info()
    # cost per compound sweep with and without the control variate
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ch.run(0, 20, N_HB, N_OR)
    ev[0].record(stream)
    ch.run(0, 200, N_HB, N_OR)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms_plain = ev[0].elapsed_time(ev[1]) / 200
    g.run(20, N_HB, N_OR, 1.0)
    ev[0].record(stream)
    g.run(200, N_HB, N_OR, 1.0)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms_cv = ev[0].elapsed_time(ev[1]) / 200
    ch.reset_stats()
    ch.cv_reset()
    t0 = time.perf_counter()
    rounds = 0
    est = None
    while time.perf_counter() - t0 < args.cube_seconds:
        g.run(2000, N_HB, N_OR, 1.0)
        rounds += 2000
        est = ch.cv_estimate()
        if est["stderr"] == est["stderr"] and est["stderr"] <= target:
            break
    wall = time.perf_counter() - t0
    plain = ch.estimate()
    t_plain_proj = rounds * ms_plain / 1e3 * (plain["stderr"] / target) ** 2
    r = {"system": "pm4096_128c_global_cv", "e_lat": e_lat, "sor_iterations": 6 * L + 50,
         "local_p_radius": args.gcv_radius,
         "solve_residual": info["residual"], "setup_s": t_setup,
         "ms_compound_sweep_plain": ms_plain, "ms_compound_sweep_with_cv": ms_cv,
         "rounds": rounds, "samples": est["n"], "wall_s_cv": wall,
         "mean_cv": est["mean"], "stderr_cv": est["stderr"], "tau_int_cv": est["tau_int"],
         "delta_cv": abs(est["mean"] - e_lat) / abs(e_lat),
         "mean_plain": plain["mean"], "stderr_plain": plain["stderr"],
         "tau_int_plain": plain["tau_int"],
         "error_variance_ratio": (est["stderr"] / plain["stderr"]) ** 2,
         "reached_1e-3_cv": bool(est["stderr"] <= target),
         "s_to_1e-3_cv_incl_setup": wall + t_setup,
         "projected_s_to_1e-3_plain": t_plain_proj}
    g.close()
    ch.close()
    lat.close()
    return r


def paper_figures(args, stream):
    """The paper's Fig. 1 and Fig. 2 workloads on one set of samples (every
    charge set is measured on every sample: the samples depend only on the box):
    128^3, 64 chains, 1 HB : 3 OR.  Fig. 2: q = 1 cubes of N = 2^3 .. 32^3 at
    the box centre; Fig. 1: two charges q = 1, one at the centre, the other at
    (n_x, L/2, L/2).  For M = 10^2 .. 10^6 samples (M = 64 x compound sweeps)
    reports delta = |MC - E| / |E| against the exact lattice value and against
    the continuum Coulomb sum Eq. (s1), with the batch-means error."""
    import math

    import torch

    from paper_1403_0711_gb300 import coulps, inputs
    box = (L, L, L)
    lat = coulps.Lattice(box, n_chains=N_CHAINS, precision=coulps.F32, seed=2014, stream=stream)
    sets = [(f"fig2_cube_N{s ** 3}", f"cube_128c_n{s ** 3}_q1", inputs.cube(box, s))
            for s in (2, 4, 8, 16, 32)]
    sets += [(f"fig1_pair_nx{nx}", f"twobody_128c_nx{nx}", inputs.two_body(box, nx))
             for nx in (65, 66, 68, 72, 80, 96, 112, 127)]
    chs = [coulps.Charges(lat, s, q) for _, _, (s, q) in sets]
    lat.sweep(300, N_HB, N_OR)
    torch.cuda.synchronize()
    rows = {name: {"set": name, "n_charges": len(q), "e_lat": golden_e_lat(gold),
                   "e_continuum": golden_e_lat(gold, 9), "by_M": []}
            for name, gold, (_, q) in sets}
    done = 0
    t0 = time.perf_counter()
    for M in (10 ** 2, 10 ** 3, 10 ** 4, 10 ** 5, 10 ** 6):
        k = math.ceil(M / N_CHAINS) - done
        if k > 0:
            coulps.run_sets(lat, chs, 0, k, N_HB, N_OR)
            done += k
        lat.sync()
        wall = time.perf_counter() - t0
        for (name, _, _), ch in zip(sets, chs):
            est = ch.estimate()
            r = rows[name]
            r["by_M"].append({
                "M": est["n"], "wall_s": wall, "mean": est["mean"], "stderr": est["stderr"],
                "delta_lat": abs(est["mean"] - r["e_lat"]) / abs(r["e_lat"]),
                "delta_continuum": abs(est["mean"] - r["e_continuum"]) / abs(r["e_continuum"]),
                "rel_stderr": est["stderr"] / abs(r["e_lat"])})
    for ch in chs:
        ch.close()
    lat.close()
    return list(rows.values())


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
    lat.set_fused(FUSED_MODES[args.fused])
    ch = coulps.Charges(lat, sites, q)

    # Measured compound sweeps (the sample is gathered by the last half-sweep of
    # each).  A step is one measured compound sweep of every chain; all K timed
    # steps are one call.  --schedule phased runs chain k mod 4 passes behind
    # (launches mix heatbath and over-relaxation tiles; measured no faster).
    lat.set_schedule({"phased": coulps.SCHEDULE_PHASED, "aligned": coulps.SCHEDULE_ALIGNED,
                      "shifted": coulps.SCHEDULE_SHIFTED}[args.schedule])
    # The timed steps run as the library runs them: the measured compound
    # sweep captured once as a CUDA graph and replayed, with the odd chains on
    # a second stream (--streams 2).  Per-kernel CUDA-event timing (which
    # launches kernel by kernel) is taken separately below.
    lat.set_streams(args.streams)
    ch.run(0, max(3, args.warmup), N_HB, N_OR)
    lat.sync()
    ch.reset_stats()  # the timed samples alone feed the time-to-accuracy projection

    # the K timed steps in one call, or from K = 100 on in five calls with an
    # event at each boundary: the whole region gives the value, the chunks its
    # spread (each call of the shifted schedule has its own prologue and
    # epilogue, so short chunks would time them more often than a run does)
    n_chunks = 5 if args.steps >= 100 else 1
    bounds = [round(args.steps * i / n_chunks) for i in range(n_chunks + 1)]
    evs = [torch.cuda.Event(enable_timing=True) for _ in bounds]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)  # let the sampler start
    evs[0].record(stream)
    for i in range(n_chunks):
        ch.run(0, bounds[i + 1] - bounds[i], N_HB, N_OR)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    ms = evs[0].elapsed_time(evs[-1])
    chunk_ms = [evs[i].elapsed_time(evs[i + 1]) / (bounds[i + 1] - bounds[i])
                for i in range(n_chunks) if bounds[i + 1] > bounds[i]]
    lat.sync()
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * sites_per_step * args.steps / (ms_max / 1e3)
    est_timed = ch.estimate()

    # Per-kernel durations: CUDA events around every launch, on one stream
    # (with two streams the halves' kernels overlap, so a launch's duration
    # would not isolate one kernel), over n_rf compound sweeps right after the
    # timed region, same lattice and charges
    n_rf = min(args.steps, 300)
    lat.set_streams(1)
    lat.set_profiling(True)
    ch.run(0, 3, N_HB, N_OR)
    lat.kernel_times()  # discard
    ch.run(0, n_rf, N_HB, N_OR)
    kt = lat.kernel_times()
    lat.set_profiling(False)
    lat.set_streams(args.streams)

    # roofline of the dominant kernel (largest share of the device time of a
    # step).  Algorithmic bytes per launch: a half-sweep reads the other
    # colour and writes its own (heatbath, 8 B per updated site) and also
    # reads its old value (over-relaxation, 12 B); a fused pass and a pass pair
    # read every site once and write it once (8 B per site, for one pass or
    # for two); the mixed half-sweep of the phased schedule is counted as its
    # share of 8 / 12 B per updated site.
    peak, peak_kind = measured_peaks()
    n_sites = n_chains * L ** 3
    kinds = {
        "hb": ("halfsweep_kernel<float, heatbath>", 8 * n_sites // 2),
        "or": ("halfsweep_kernel<float, over-relaxation>", 12 * n_sites // 2),
        "pass_hb": ("pass_kernel<float, heatbath>", 8 * n_sites),
        "pass_or": ("pass_kernel<float, over-relaxation>", 8 * n_sites),
        "pair_hb": ("pair_kernel<float, heatbath pass in the pair>", 8 * n_sites),
        "pair_or": ("pair_kernel<float, over-relaxation, over-relaxation>", 8 * n_sites),
        "mixed": ("halfsweep_mixed_kernel<float> (phase-shifted heatbath + over-relaxation)",
                  n_sites // 2 * (8 * N_HB + 12 * N_OR) // PASSES),
    }
    total_ms = sum(kt[k + "_ms"] for k in kinds)
    dom_kind = max(kinds, key=lambda k: kt[k + "_ms"])
    name, bytes_per_launch = kinds[dom_kind]
    avg_ms = kt[dom_kind + "_ms"] / max(1, kt[dom_kind + "_n"])
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    dom = {"kernel": name, "algorithmic_bytes_per_launch": bytes_per_launch,
           "avg_launch_ms": avg_ms,
           "share_of_sweep_kernel_time": kt[dom_kind + "_ms"] / total_ms if total_ms else None,
           "launches_per_compound_sweep": {k: kt[k + "_n"] / n_rf for k in kinds if kt[k + "_n"]},
           "avg_launch_ms_by_kind": {k: kt[k + "_ms"] / kt[k + "_n"] for k in kinds
                                     if kt[k + "_n"]},
           "sweep_kernel_ms_per_compound_sweep": total_ms / n_rf}
    traffic = profiled_traffic(name)
    roofline = dict({"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": f"{peak_kind} (burst copy)",
                     "timing": f"CUDA events around every launch, one stream, {n_rf} compound "
                               "sweeps after the timed region"}, **dom)
    # every sweep kernel of the step against both of its limits: HBM (algorithmic
    # bytes / launch time, of the measured copy bandwidth) and instruction issue
    # (warp instructions of the committed ncu capture / launch time, of the
    # GPU's issue capacity at the clock sampled during the timed region: SMs x 4
    # schedulers x 1 warp instruction per cycle)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = clk.get("sm_mhz") if isinstance(clk, dict) and clk.get("sm_mhz") else 2070.0
    by_kernel = {}
    for k, (kname, kbytes) in kinds.items():
        if not kt[k + "_n"]:
            continue
        kms = kt[k + "_ms"] / kt[k + "_n"]
        kach = kbytes / (kms / 1e3) / 1e9
        e = {"kernel": kname, "avg_launch_ms": kms, "algorithmic_bytes_per_launch": kbytes,
             "achieved_GBps": kach, "hbm_frac": kach / peak,
             "share_of_sweep_kernel_time": kt[k + "_ms"] / total_ms if total_ms else None,
             "traffic": profiled_traffic(kname)}
        winst = profiled_traffic(kname, "warp_instructions_per_launch_full")
        if winst:
            e["warp_instructions_per_launch"] = winst
            e["issue_frac"] = winst / (kms / 1e3) / (sms * 4 * mhz * 1e6)
        by_kernel[k] = e
    roofline["by_kernel"] = by_kernel
    roofline["issue_peak"] = {"warp_instructions_per_s": sms * 4 * mhz * 1e6, "sms": sms,
                              "sm_mhz": mhz}
    sweep_launches = sum(kt[k + "_n"] for k in kinds) / n_rf  # all chains, one stream

    # spread: the step loop timed again, --repeats times, right after the
    # timed region (same graph, same streams)
    rep_ms = []
    n_rep_steps = max(args.steps, 100)
    for _ in range(max(0, args.repeats)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ch.run(0, n_rep_steps, N_HB, N_OR)
        e1.record(stream)
        torch.cuda.synchronize()
        rep_ms.append(e0.elapsed_time(e1) / n_rep_steps)
    repeats = None
    if rep_ms:
        repeats = {"steps_each": n_rep_steps, "ms_per_step": rep_ms,
                   "median_ms_per_step": statistics.median(rep_ms),
                   "min_ms_per_step": min(rep_ms), "max_ms_per_step": max(rep_ms),
                   "median_site_updates_per_s": world * sites_per_step /
                   (statistics.median(rep_ms) / 1e3)}

    # end to end through the C ABI with host buffers: every step uploads the
    # charge set from host memory, runs one measured compound sweep (graph
    # replay) and reads the estimate back to the host.  The read is
    # pipelined: step k's state is posted (a queued copy into pinned memory)
    # and the estimate of step k - 1 taken while step k runs, so the GPU
    # never waits for the host's pooling
    lat.set_profiling(False)
    ch.reset_stats()
    ch.update(sites, q)  # allocate the pinned staging buffers outside the timed region
    ch.run(0, 1, N_HB, N_OR)  # capture the graph outside the timed region
    ch.estimate_post()  # and the pinned estimate slots
    ch.estimate_take()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for k in range(args.e2e_steps):
        ch.update(sites, q)
        ch.run(0, 1, N_HB, N_OR)
        ch.estimate_post()
        if k > 0:
            est = ch.estimate_take()
    est = ch.estimate_take()
    e2e_s = time.perf_counter() - t0
    t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    e2e_s = float(t.item())
    e2e = {"value": world * sites_per_step * args.e2e_steps / e2e_s, "unit": "site-updates/s",
           "h2d_bytes_per_step": N_CHARGES * (4 + 8),
           "d2h_bytes_per_step": n_chains * coulps.STAT_STRIDE * 8 + 4,
           "steps": args.e2e_steps,
           "path": "per step coulps_charges_update + coulps_run(0, 1, 1, 3) + coulps_estimate_post, "
                   "and coulps_estimate_take of the previous step's state"}

    # time to 1e-3, plain and with the global control variate g = Q h, both
    # projected from the same args.gcv_steps compound sweeps of every chain
    # (bench.py --workload gcv measures the latter directly): the plain
    # estimator of those samples at the plain cost per sweep of the timed
    # region, the control variate at its own measured cost
    tta, tta_cv = None, None
    if args.gcv_steps <= 0:
        tta = time_to_accuracy(est_timed, ms_max / 1e3, world)
    if args.gcv_steps > 0:
        ch.reset_stats()
        ch.cv_reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gcv = coulps.GlobalCV(ch, R=args.gcv_radius)
        setup = time.perf_counter() - t0
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        gcv.run(args.gcv_steps, N_HB, N_OR, 1.0)
        ev1.record(stream)
        torch.cuda.synchronize()
        cv_s = ev0.elapsed_time(ev1) / 1e3
        est_cv, est_pl = ch.cv_estimate(), ch.estimate()
        e_lat = golden_e_lat("bench_128c_n4096_pm")
        tta = time_to_accuracy(est_pl, args.gcv_steps * (ms_max / args.steps) / 1e3, world)
        if tta:
            tta["estimator"] = ("plain Eq. (nsum2), batch means over all chains, on the "
                                f"{est_pl['n'] * world} samples of the control-variate run, "
                                "timed at the plain cost per compound sweep")
        if est_cv["stderr"] > 0 and est_pl["stderr"] > 0:
            t_cv = cv_s * (est_cv["stderr"] / (1e-3 * abs(e_lat))) ** 2
            tta_cv = {"eps": 1e-3,
                      "estimator": "control variates g = Q h (h by SOR) + local P term "
                                   f"(R = {args.gcv_radius}), c = 1",
                      "setup_s": setup, "samples": est_cv["n"] * world,
                      "ms_per_step_with_cv": 1e3 * cv_s / args.gcv_steps,
                      "mean": est_cv["mean"], "stderr": est_cv["stderr"],
                      "tau_int": est_cv["tau_int"],
                      "delta": abs(est_cv["mean"] - e_lat) / abs(e_lat),
                      "error_variance_ratio_vs_plain_same_samples":
                          (est_cv["stderr"] / est_pl["stderr"]) ** 2,
                      "projected_seconds": t_cv + setup, "projected_hours": (t_cv + setup) / 3600}
            if tta:
                tta_cv["plain_over_cv_time"] = tta["projected_seconds"] / tta_cv["projected_seconds"]
        gcv.close()

    extras = None
    if rank == 0 and world == 1 and args.extras == "on":
        ch.close()
        lat.close()
        ch = lat = None
        torch.cuda.empty_cache()
        extras = {"batched_256_systems": batched_throughput(args, stream, steps=50),
                  "batched_256_time_to_1e-3": batched_time_to_accuracy(args, stream, steps=2000),
                  "large_512_1e6_charges": large_throughput(args, stream, 512, steps=20),
                  "learned_cv_q1_cube": cv_local_cube(args, stream, seconds=60.0)}

    out = None
    if rank == 0:
        # per step and half of the chains (two streams: each half has its own
        # sweep kernels and finalize): the sweep kernels counted by the
        # profiled sweeps above, one finalize; one pass-counter advance per step
        launches = int(round(args.steps * (args.streams * (sweep_launches + 1) + 1)))
        line = {
            "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": dict(CONFIG, parallelism=f"replicas{world}", n_chains_per_gpu=n_chains,
                                           fused_passes=args.fused, streams=args.streams),
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "timed_chunks": {"ms_per_step": chunk_ms, "median": statistics.median(chunk_ms),
                             "min": min(chunk_ms), "max": max(chunk_ms)},
            "repeats": repeats,
            "time_to_1e-3": tta, "time_to_1e-3_cv": tta_cv, "estimate_after_e2e": est,
            "secondary_configs": extras,
        }
        if world == 1:
            rate, cores, n = cpu_oracle_rate(args.cpu_seconds)
            line["cpu_baseline"] = {
                "value": rate, "unit": "site-updates/s", "cores": cores, "kind": "oracle",
                "sample": f"{n} compound sweeps (1 HB + 3 OR) + samples of one 128^3 chain, "
                          "FP64 oracle, OpenMP over z planes"}
        out = line
    if ch is not None:
        ch.close()
        lat.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


def batched_throughput(args, stream, steps):
    """256 independent systems in one persistent launch per half-sweep (one
    CUDA graph per measured compound sweep): edges from {32,48,64,80,96}, N
    log-uniform in [64, 2048], q in [-1, 1] shifted to zero net, FP32,
    1 HB : 3 OR, the sample of every system each compound sweep."""
    import torch

    from paper_1403_0711_gb300 import coulps, inputs
    systems = inputs.batch_systems(256, seed=7)
    b = coulps.Batch([L_ for L_, _, _ in systems], precision=coulps.F32, seed=77, stream=stream)
    if getattr(args, "batch_fused", None) is not None:
        b.set_fused(args.batch_fused)
    b.set_charges([(s_, q_) for _, s_, q_ in systems])
    info = b.info()
    rate, ms = _timed(stream, lambda: b.run(0, 1, N_HB, N_OR), info["sites"] * PASSES, steps, 10)
    r = {"systems": 256, "sites": info["sites"], "tiles": info["tiles"], "fused_mode": b.fused(),
         "persistent_ctas": info["grid"], "site_updates_per_s": rate, "ms_per_step": ms,
         "steps": steps,
         "algorithmic_GBps_halfsweep_bytes": rate / PASSES * (8 + 12 * N_OR) / 1e9}
    b.close()
    torch.cuda.empty_cache()
    return r


def batched_time_to_accuracy(args, stream, steps, eps=1e-3):
    """Time until every one of the 256 systems of the batched workload has its
    E_N to a batch-means standard error of eps: plain Eq. (nsum2) samples
    against the global control variate of every system (coulps_batch_gcv,
    h by SOR, local P term R = 1, c = 1).  Each arm samples `steps` measured
    compound sweeps (1 HB : 3 OR) of all systems after 100 unmeasured ones,
    timed with CUDA events; a system needing n_s = n (se_s / eps)^2 samples,
    all systems advance together, so the projected time is max_s n_s times the
    measured time per compound sweep (CV setup added to the CV arm)."""
    import numpy as np
    import torch

    from paper_1403_0711_gb300 import coulps, inputs
    systems = inputs.batch_systems(256, seed=7)
    b = coulps.Batch([L_ for L_, _, _ in systems], precision=coulps.F32, seed=77, stream=stream)
    b.set_charges([(s_, q_) for _, s_, q_ in systems])
    b.sweep(100, N_HB, N_OR)

    def project(est, ms):
        need = est["n"] * (est["stderr"] / eps) ** 2
        worst = float(np.max(need))
        return {"ms_per_step": ms, "samples": int(est["n"][0]),
                "max_stderr": float(np.max(est["stderr"])),
                "median_stderr": float(np.median(est["stderr"])),
                "median_tau_int": float(np.median(est["tau_int"])),
                "steps_needed_worst_system": worst,
                "steps_needed_median_system": float(np.median(need)),
                "projected_seconds": worst * ms / 1e3}

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b.reset_stats()
    torch.cuda.synchronize()
    e0.record(stream)
    b.run(0, steps, N_HB, N_OR)
    e1.record(stream)
    torch.cuda.synchronize()
    plain = project(b.estimate(), e0.elapsed_time(e1) / steps)
    t0 = time.perf_counter()
    g = coulps.BatchGlobalCV(b, R=1)
    b.sync()
    setup = time.perf_counter() - t0
    g.run(10, N_HB, N_OR, 1.0)  # graph capture and warm-up
    g.reset()
    torch.cuda.synchronize()
    e0.record(stream)
    g.run(steps, N_HB, N_OR, 1.0)
    e1.record(stream)
    torch.cuda.synchronize()
    cv = project(g.estimate(), e0.elapsed_time(e1) / steps)
    cv["setup_s"] = setup
    cv["projected_seconds"] += setup
    g.close()
    b.close()
    torch.cuda.empty_cache()
    return {"systems": 256, "eps": eps, "estimator_cv": "global CV per system, R = 1, c = 1",
            "plain": plain, "cv": cv,
            "plain_over_cv_time": plain["projected_seconds"] / cv["projected_seconds"]}


def large_throughput(args, stream, n, steps):
    """One n^3 chain (FP32 field, FP64 sums), charges in 200 Gaussian blobs
    (sigma = 6 sites), q in [-0.8, 0.8] shifted to zero net: 10^6 charges at
    512^3, else the same density N / L^3 = 0.00745; 1 HB : 3 OR measured
    compound sweeps on the default schedule."""
    import torch

    from paper_1403_0711_gb300 import coulps, inputs
    box = (n, n, n)
    nq = 1_000_000 if n == 512 else int(round(0.00745 * n ** 3))
    sites, q = inputs.blobs(box, nq, seed=3)
    lat = coulps.Lattice(box, n_chains=1, precision=coulps.F32, seed=77, stream=stream)
    ch = coulps.Charges(lat, sites, q)
    rate, ms = _timed(stream, lambda: ch.run(0, 1, N_HB, N_OR), n ** 3 * PASSES, steps, 5)
    r = {"L": n, "n_charges": nq, "site_updates_per_s": rate, "ms_per_step": ms, "steps": steps,
         "fused_mode": lat.info()["fused"]}
    ch.close()
    lat.close()
    torch.cuda.empty_cache()
    return r


def _timed(stream, step, sites_per_step, steps, warmup):
    import torch
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
    if args.workload in ("large512", "sweep"):
        sizes = [512] if args.workload == "large512" else [128, 256, 384, 512]
        for n in sizes:
            results.append(large_throughput(args, stream, n,
                                            max(20, min(args.steps, int(2e10 / n ** 3)))))
    elif args.workload == "batched":
        results.append(batched_throughput(args, stream, args.steps))
    elif args.workload == "batched_tta":
        results.append(batched_time_to_accuracy(args, stream, max(args.steps, 500)))
    elif args.workload == "gcv":
        results.append(gcv_time_to_accuracy(args, stream))
    elif args.workload == "paper":
        results.extend(paper_figures(args, stream))
    elif args.workload == "cv_eval":
        results.append(cv_eval_cost(args, stream))
    elif args.workload == "cv":
        results.extend(cv_experiment(args, stream))
    elif args.workload == "cube":
        results.append(cube_time_to_accuracy(args, stream))
    elif args.workload == "offlattice":
        results.append(offlattice_cube(args, stream))
    print(json.dumps({"workload": args.workload, "metric": METRIC, "results": results}), flush=True)


def cv_experiment(args, stream):
    out = [cv_local_cube(args, stream)]
    if args.cv_global:
        out.extend(cv_global(args, stream))
    return out


def cv_local_cube(args, stream, seconds=None):
    """Localized learned Stein control variate on the paper's Fig. 2 geometry
    (N = 8 charges q = 1 in a cube at the centre of a 128^3 box): g is the net
    within --cv-halo sites of the charges, evaluated on that sub-box only.
    Train on the chains' own samples, then sample with the CV recorded on the
    device every compound sweep until its batch-means error reaches
    1e-3 |E_lat| (or --cube-seconds), and compare with the plain estimator of
    the same samples (its time to 1e-3 projected from its error and its own
    cost per sweep)."""
    import numpy as np
    import torch

    from paper_1403_0711_gb300 import coulps, inputs, stein
    box = (L, L, L)
    sites, q = inputs.cube(box, 2)
    e_lat = golden_e_lat("cube_128c_n8_q1")
    target = 1e-3 * abs(e_lat)
    lat = coulps.Lattice(box, n_chains=N_CHAINS, precision=coulps.F32, seed=4243, stream=stream)
    ch = coulps.Charges(lat, sites, q)
    rho = stein.charge_density(box, sites, q)
    lo = sites.min(axis=0) - args.cv_halo
    hi = sites.max(axis=0) + 1 + args.cv_halo
    cv = stein.LocalSteinCV(box, lo, hi, seed=0, scale=0.3)
    lat.sweep(300, N_HB, N_OR)
    lat.sync()
    t0 = time.perf_counter()
    phis, Aphis, es = stein.collect_region(cv, lat, ch, rho, n_rounds=args.cv_collect, every=1,
                                           n_hb=N_HB, n_or=N_OR)
    t_collect = time.perf_counter() - t0
    log = []
    t0 = time.perf_counter()
    tg_fit = stein.fit_region(cv, phis, Aphis, es, rho, steps=args.cv_steps, batch=256, lr=3e-3,
                              log=log)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    n_tr = int(len(es) * 0.75)
    e_ho, t_ho = es[n_tr:].numpy(), tg_fit[n_tr:].cpu().numpy()
    ratio_holdout = float(np.var(e_ho - cv.c * t_ho) / np.var(e_ho))
    del phis, Aphis
    # the CV evaluation and recording as one CUDA graph of library kernels
    graph, tg = cv.record_graph(lat, ch, rho)

    def cv_step():
        with torch.cuda.stream(stream):
            graph.replay()

    # cost of one compound sweep with and without the CV, on the device
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ms_plain = ms_cv = 0.0
    for r in range(20):
        ev[0].record(stream)
        ch.run(0, 1, N_HB, N_OR)
        ev[1].record(stream)
        cv_step()
        ev[2].record(stream)
        stream.synchronize()
        if r >= 5:
            ms_plain += ev[0].elapsed_time(ev[1]) / 15
            ms_cv += ev[1].elapsed_time(ev[2]) / 15
    ch.reset_stats()
    ch.cv_reset()
    lat.sync()
    t0 = time.perf_counter()
    rounds = 0
    cvest = None
    limit = args.cube_seconds if seconds is None else seconds
    while time.perf_counter() - t0 < limit:
        for _ in range(250):
            ch.run(0, 1, N_HB, N_OR)
            cv_step()
        rounds += 250
        cvest = ch.cv_estimate()
        if cvest["stderr"] == cvest["stderr"] and cvest["stderr"] <= target and rounds >= 2000:
            break
    wall = time.perf_counter() - t0
    plain = ch.estimate()
    # the plain estimator alone: same samples at its own (lower) cost per sweep
    plain_wall_same = rounds * ms_plain / 1e3
    t_plain_proj = plain_wall_same * (plain["stderr"] / target) ** 2
    r = {"system": "cube8_q1_local_cv", "e_lat": e_lat, "halo": args.cv_halo,
         "region_lo": [int(v) for v in lo], "region_hi": [int(v) for v in hi],
         "eval_box": list(cv.edims), "training_samples": int(len(es)), "collect_s": t_collect,
         "train_s": t_train, "train_steps": args.cv_steps,
         "loss_first20": float(np.mean(log[:20])), "loss_last20": float(np.mean(log[-20:])),
         "c": cv.c, "variance_ratio_holdout": ratio_holdout,
         "ms_compound_sweep": ms_plain, "ms_cv_eval": ms_cv,
         "rounds": rounds, "samples": cvest["n"], "wall_s_cv": wall,
         "mean_cv": cvest["mean"], "stderr_cv": cvest["stderr"], "tau_int_cv": cvest["tau_int"],
         "mean_plain": plain["mean"], "stderr_plain": plain["stderr"],
         "tau_int_plain": plain["tau_int"],
         "variance_ratio": (cvest["stderr"] / plain["stderr"]) ** 2,
         "delta_cv": abs(cvest["mean"] - e_lat) / abs(e_lat),
         "reached_1e-3_cv": bool(cvest["stderr"] <= target),
         "s_to_1e-3_cv_incl_training": wall + t_collect + t_train,
         "projected_s_to_1e-3_plain": t_plain_proj}
    ch.close()
    lat.close()
    torch.cuda.empty_cache()
    return r


def cv_eval_cost(args, stream):
    """Device time of one localized-CV evaluation + recording (the CUDA graph
    the cv workload replays after every sweep) for 64 chains on the 128^3 q = 1
    cube, sub-box 14^3: pack, three tensor-core convs, region divergence,
    charge-site term, record.  Untrained weights (the cost does not depend on
    them)."""
    import torch

    from paper_1403_0711_gb300 import coulps, inputs, stein
    box = (L, L, L)
    sites, q = inputs.cube(box, 2)
    lat = coulps.Lattice(box, n_chains=N_CHAINS, precision=coulps.F32, seed=5, stream=stream)
    ch = coulps.Charges(lat, sites, q)
    lat.sweep(20, N_HB, N_OR)
    rho = stein.charge_density(box, sites, q)
    cv = stein.LocalSteinCV(box, sites.min(axis=0) - args.cv_halo,
                            sites.max(axis=0) + 1 + args.cv_halo, seed=0, scale=0.3, w3_scale=0.1)
    cv.c = 1.0
    graph, tg = cv.record_graph(lat, ch, rho)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with torch.cuda.stream(stream):
        for _ in range(5):
            graph.replay()
        ev[0].record(stream)
        for _ in range(args.steps):
            graph.replay()
        ev[1].record(stream)
    stream.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    ex, ey, ez = cv.edims
    conv_sites = N_CHAINS * (ex + 1) * ey * ez  # interleaved boxes with gutters
    conv_flops = 3 * conv_sites * 16 * 16 * 27 * 2
    r = {"system": "cube8_q1_local_cv_eval", "eval_box": list(cv.edims), "chains": N_CHAINS,
         "ms_per_eval": ms, "evals": args.steps, "conv_flops_per_eval": conv_flops,
         "conv_tflops_if_all_time": conv_flops / (ms / 1e3) / 1e12}
    ch.close()
    lat.close()
    return r


def cv_global(args, stream):
    """Whole-lattice learned Stein control variate on the 128^3 lattice: train on
    2048 of the chains' own samples, then compare plain and CV estimators on
    fresh samples.  Runs on the +-1 zero-net N=4096 system."""
    import numpy as np
    import torch

    from paper_1403_0711_gb300 import coulps, inputs, stein
    out = []
    box = (L, L, L)
    for name, (sites, q), gold in (
            ("pm4096", inputs.plus_minus(box, N_CHARGES, seed=1), "bench_128c_n4096_pm"),):
        lat = coulps.Lattice(box, n_chains=N_CHAINS, precision=coulps.F32, seed=4242, stream=stream)
        ch = coulps.Charges(lat, sites, q, log_capacity=4096)
        rho = stein.charge_density(box, sites, q)
        lat.sweep(300, N_HB, N_OR)
        t0 = time.perf_counter()
        phis, Aphis, es = stein.collect(lat, ch, rho, n_rounds=32, every=4, n_hb=N_HB, n_or=N_OR)
        t_collect = time.perf_counter() - t0
        cv = stein.SteinCV(seed=0, scale=0.3)
        log = []
        t0 = time.perf_counter()
        stein.fit(cv, phis, Aphis, es, rho, steps=args.cv_steps, batch=16, lr=2e-3, log=log)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        del phis, Aphis
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e_list, tg_list, ms_sweep, ms_cv = [], [], 0.0, 0.0
        rounds = args.cv_rounds
        for r in range(rounds):
            ev[0].record(stream)
            ch.run(0, 1, N_HB, N_OR)
            ev[1].record(stream)
            tg = cv.evaluate(lat, rho)
            ev[2].record(stream)
            torch.cuda.synchronize()
            ms_sweep += ev[0].elapsed_time(ev[1])
            ms_cv += ev[1].elapsed_time(ev[2])
            e_list.append(ch.samples()[-1, :, 2].copy())
            tg_list.append(tg.cpu().numpy())
        e = np.stack(e_list)  # (rounds, chains)
        tgv = np.stack(tg_list)
        ecv = e - cv.c * tgv
        e_lat = golden_e_lat(gold)
        ms_sweep /= rounds
        ms_cv /= rounds
        # per-chain means are independent; the time to eps|E| scales with the
        # variance of one chain's mean per unit time
        def proj(x, ms):
            var_chain_mean = x.mean(axis=0).var(ddof=1)  # over chains, `rounds` samples each
            se_now = (var_chain_mean / x.shape[1]) ** 0.5
            t_now = rounds * ms / 1e3
            return t_now * (se_now / (1e-3 * abs(e_lat))) ** 2, float(x.mean()), se_now
        t_plain, m_plain, se_plain = proj(e, ms_sweep)
        t_cv, m_cv, se_cv = proj(ecv, ms_sweep + ms_cv)
        k = 4  # CV on every 4th sample: the other samples stay plain
        mix = np.concatenate([e[i::k] if i else ecv[0::k] for i in range(k)], axis=0)
        t_cv4, m_cv4, se_cv4 = proj(mix, ms_sweep + ms_cv / k)
        out.append({
            "system": name, "e_lat": e_lat, "training_samples": int(len(es)),
            "collect_s": t_collect, "train_s": t_train, "train_steps": args.cv_steps,
            "loss_first10": float(np.mean(log[:10])), "loss_last10": float(np.mean(log[-10:])),
            "c": cv.c, "var_plain": float(e.var()), "var_cv": float(ecv.var()),
            "variance_ratio": float(ecv.var() / e.var()),
            "mean_plain": m_plain, "se_plain": se_plain, "mean_cv": m_cv, "se_cv": se_cv,
            "ms_compound_sweep": ms_sweep, "ms_cv_eval": ms_cv,
            "projected_s_to_1e-3_plain": t_plain, "projected_s_to_1e-3_cv": t_cv,
            "projected_s_to_1e-3_cv_every4": t_cv4, "eval_rounds": rounds})
        ch.close()
        lat.close()
        torch.cuda.empty_cache()
    return out


def cube_time_to_accuracy(args, stream):
    """The paper's Fig. 2 geometry (N=8 charges q=1 in a cube at the centre of a
    128^3 box): run until the batch-means error is 1e-3 |E_lat| (or a time
    limit) and report the wall time and the error against E_lat."""
    import torch

    from paper_1403_0711_gb300 import coulps, inputs
    box = (L, L, L)
    sites, q = inputs.cube(box, 2)
    e_lat = golden_e_lat("cube_128c_n8_q1")
    lat = coulps.Lattice(box, n_chains=N_CHAINS, precision=coulps.F32, seed=99, stream=stream)
    ch = coulps.Charges(lat, sites, q)
    lat.sweep(300, N_HB, N_OR)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    est = None
    while time.perf_counter() - t0 < args.cube_seconds:
        ch.run(0, 500, N_HB, N_OR)
        est = ch.estimate()
        if est["stderr"] == est["stderr"] and est["stderr"] <= 1e-3 * abs(e_lat) and \
                est["n"] > 64 * 2000:
            break
    wall = time.perf_counter() - t0
    r = {"system": "cube8_q1", "e_lat": e_lat, "wall_s": wall, "samples": est["n"],
         "mean": est["mean"], "stderr": est["stderr"], "tau_int": est["tau_int"],
         "rel_stderr": est["stderr"] / abs(e_lat),
         "delta": abs(est["mean"] - e_lat) / abs(e_lat),
         "reached_1e-3": bool(est["stderr"] <= 1e-3 * abs(e_lat))}
    ch.close()
    lat.close()
    return r


def golden_offlattice(name):
    """Exact energies of the off-lattice cube (tests/golden/offlattice.txt,
    written by tests/golden/make_golden.py from the FP64 oracle)."""
    keys = ["n_pairs", "e_far", "e_direct", "e_plain", "continuum"]
    for ln in (ROOT / "tests" / "golden" / "offlattice.txt").read_text().splitlines():
        if ln.startswith(name + " "):
            v = ln.split()
            return dict(zip(keys, [int(v[8])] + [float(x) for x in v[9:13]]))
    return None


def offlattice_cube(args, stream):
    """The paper's closing remarks on the Fig. 2 cube: the 8 charges q = 1
    moved off their sites (uniform offsets in [-0.3, 0.3] per axis) and read
    through trilinear weights, with forces, and with the pairs closer than
    r_c = 1.5 computed directly (continuum Eq. (s1) terms).  Both estimators
    (near pairs left out, and plain interpolated lattice) are measured on the
    same samples, with forces, until the near-field estimate's error reaches
    1e-3 of the total or --off-seconds; reported against the oracle's exact
    values."""
    import numpy as np
    import torch

    from paper_1403_0711_gb300 import coulps, inputs
    box = (L, L, L)
    pos, q = inputs.off_lattice_cube(box, 2, 0, 0.3)
    gold = golden_offlattice("offcube_128c_n8_q1")
    rc = 1.5
    lat = coulps.Lattice(box, n_chains=N_CHAINS, precision=coulps.F32, seed=123, stream=stream)
    near = coulps.Charges.off_lattice(lat, pos, q, forces=True)
    plain = coulps.Charges.off_lattice(lat, pos, q, forces=True)
    info = near.near(rc)
    lat.sweep(300, N_HB, N_OR)
    # cost of a measured compound sweep with both sets against the sweep alone
    coulps.run_sets(lat, [near, plain], 0, 50, N_HB, N_OR)
    lat.sweep(50, N_HB, N_OR)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    lat.sweep(200, N_HB, N_OR)
    ev[1].record(stream)
    coulps.run_sets(lat, [near, plain], 0, 200, N_HB, N_OR)
    ev[2].record(stream)
    torch.cuda.synchronize()
    ms_sweep = ev[0].elapsed_time(ev[1]) / 200
    ms_meas = ev[1].elapsed_time(ev[2]) / 200
    near.reset_stats()
    plain.reset_stats()
    e_total = gold["e_far"] + info["e_direct"]
    t0 = time.perf_counter()
    est = None
    while time.perf_counter() - t0 < args.off_seconds:
        coulps.run_sets(lat, [near, plain], 0, 500, N_HB, N_OR)
        est = near.estimate()
        if est["stderr"] == est["stderr"] and est["stderr"] <= 1e-3 * abs(e_total) and \
                est["n"] > N_CHAINS * 2000:
            break
    wall = time.perf_counter() - t0
    est_p = plain.estimate()
    f_near, f_err = near.forces()
    f_tot = f_near + info["f_direct"]
    r = {"system": "off-lattice cube, 8 charges q=1 (jitter 0.3), 128^3, 64 chains",
         "r_c": rc, "near_pairs": info["n_pairs"], "golden_pairs": gold["n_pairs"],
         "ms_per_compound_sweep": ms_sweep,
         "ms_per_compound_sweep_with_two_offlattice_sets_and_forces": ms_meas,
         "wall_s": wall, "samples": est["n"], "tau_int": est["tau_int"],
         "near": {"mean_far": est["mean"], "stderr": est["stderr"], "exact_far": gold["e_far"],
                  "e_direct": info["e_direct"], "total": est["mean"] + info["e_direct"],
                  "delta_vs_exact_total": abs(est["mean"] - gold["e_far"]) / abs(e_total),
                  "rel_stderr": est["stderr"] / abs(e_total)},
         "plain": {"mean": est_p["mean"], "stderr": est_p["stderr"], "exact": gold["e_plain"],
                   "delta": abs(est_p["mean"] - gold["e_plain"]) / abs(gold["e_plain"])},
         "continuum_Eq_s1": gold["continuum"],
         "gap_to_continuum": {"plain_lattice": abs(gold["e_plain"] - gold["continuum"])
                              / gold["continuum"],
                              "near_field_corrected": abs(e_total - gold["continuum"])
                              / gold["continuum"]},
         "forces": {"max_abs": float(np.abs(f_tot).max()),
                    "max_stderr": float(np.abs(f_err).max()),
                    "net_force_norm": float(np.linalg.norm(f_tot.sum(axis=0)))}}
    for c in (near, plain):
        c.close()
    lat.close()
    return r


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload != "chains128":
        run_extra(a)
    else:
        run_ours(a)
