"""Autotuner for the tile shapes (ty rows x dz planes per CTA) of the
half-sweep kernel and of the fused-pass kernel.

The shape changes only the work decomposition, never the results (the tests
check fields bitwise across shapes), so the tuner may pick freely.  For a box
shape it times every candidate with the library's own per-kernel CUDA-event
timing (coulps_set_profiling / coulps_kernel_times) over a few compound
sweeps and keeps the fastest.  Results are cached in a JSON file keyed by box,
chain count, precision, compound-sweep mix and GPU name
($COULPS_TUNE_CACHE, default ~/.cache/coulps_tune.json).

tune_lattice(lat)  tunes and applies both shapes of a Lattice (the half-sweep
                   shape serves passes that are not fused).
tune_batch(batch)  tunes each distinct system shape of a Batch (with as many
                   chains as the batch has systems of that shape, so the tuned
                   lattice carries the same load) and applies them.
"""
from __future__ import annotations

import json
import os
from pathlib import Path

from . import coulps


def _cache_path() -> Path:
    return Path(os.environ.get("COULPS_TUNE_CACHE", Path.home() / ".cache" / "coulps_tune.json"))


def _load_cache() -> dict:
    p = _cache_path()
    try:
        return json.loads(p.read_text())
    except (OSError, ValueError):
        return {}


def _save_cache(c: dict) -> None:
    p = _cache_path()
    try:
        p.parent.mkdir(parents=True, exist_ok=True)
        tmp = p.with_suffix(f".{os.getpid()}.tmp")
        tmp.write_text(json.dumps(c, indent=1, sort_keys=True))
        os.replace(tmp, p)
    except OSError:
        pass


def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:
        return "gpu"


def row_stride(Lx: int, precision: int) -> int:
    es = 4 if precision == coulps.F32 else 8
    a = 32 // es
    return (4 * ((Lx + 7) // 8) + a - 1) // a * a


def candidates(L, precision):
    """Tile shapes with at most 256 threads, box rows <= 256."""
    Lx, Ly, Lz = L
    qw = row_stride(Lx, precision) // 4
    tys = sorted({t for t in (1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128)
                  if t <= Ly and qw * t <= 256 and t + 2 <= 256} |
                 {min(Ly, 254, max(1, 256 // qw))})  # the default shape; halo box <= 256 rows
    dzs = sorted({d for d in (2, 4, 8, 16, 32, 64) if d <= Lz} | {Lz if Lz < 2 else min(Lz, 16)})
    return [(t, d) for t in tys for d in dzs]


def pass_candidates(L, precision):
    """Fused-pass tile shapes: (ty + 2) rows of quads within 512 threads."""
    Lx, Ly, Lz = L
    qw = row_stride(Lx, precision) // 4
    # odd row counts too: at 128^3 x 64 chains 13 rows was the fastest of 44
    # shapes measured (ty + 2 rows of quads per CTA, two rows per warp)
    tys = sorted({t for t in (1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 13, 14, 15, 22, 29, 30, 46, 62,
                              126)
                  if t <= Ly and qw * (t + 2) <= 512 and t + 4 <= 256} | {1})
    dzs = sorted({d for d in (8, 16, 32, 64) if d <= Lz} | {Lz})
    return [(t, d) for t in tys for d in dzs]


def _time_shapes(L, n_chains, precision, shapes, n_hb, n_or, reps, stream, fused=False):
    lat = coulps.Lattice(L, n_chains=n_chains, precision=precision, seed=1, stream=stream)
    lat.set_fused(fused)
    lat.set_profiling(True)
    out = {}
    try:
        lat.sweep(2, n_hb, n_or)
        for ty, dz in shapes:
            try:
                if fused:
                    lat.set_pass_tile(ty, dz)
                else:
                    lat.set_tile(ty, dz)
            except coulps.CoulpsError:
                continue  # a shape the library refuses (e.g. its shared memory would not fit)
            lat.sweep(1, n_hb, n_or)
            lat.kernel_times()
            lat.sweep(reps, n_hb, n_or)
            kt = lat.kernel_times()
            out[(ty, dz)] = kt["hb_ms"] + kt["or_ms"] + kt["pass_hb_ms"] + kt["pass_or_ms"]
    finally:
        lat.close()
    return out


def tune_shape(L, n_chains=1, precision=coulps.F32, n_hb=1, n_or=3, reps=3, stream=None,
               use_cache=True):
    """Best (ty, dz) for a box shape; cached."""
    L = tuple(int(v) for v in L)
    key = f"{L[0]}x{L[1]}x{L[2]}|{n_chains}|{precision}|{n_hb}:{n_or}|{_gpu_name()}"
    cache = _load_cache() if use_cache else {}
    if key in cache:
        return tuple(cache[key]["tile"])
    times = _time_shapes(L, n_chains, precision, candidates(L, precision), n_hb, n_or, reps, stream)
    best = min(times, key=times.get)
    if use_cache:
        cache = _load_cache()
        cache[key] = {"tile": list(best), "ms": times[best]}
        _save_cache(cache)
    return best


def tune_pass_shape(L, n_chains=1, precision=coulps.F32, n_hb=1, n_or=3, reps=3, stream=None,
                    use_cache=True):
    """Best fused-pass (ty, dz) for a box shape; cached.  Times an even number
    of passes per compound sweep (all of them fused)."""
    L = tuple(int(v) for v in L)
    if (n_hb + n_or) % 2:
        n_or += 1
    key = f"pass|{L[0]}x{L[1]}x{L[2]}|{n_chains}|{precision}|{n_hb}:{n_or}|{_gpu_name()}"
    cache = _load_cache() if use_cache else {}
    if key in cache:
        return tuple(cache[key]["tile"])
    times = _time_shapes(L, n_chains, precision, pass_candidates(L, precision), n_hb, n_or, reps,
                         stream, fused=True)
    best = min(times, key=times.get)
    if use_cache:
        cache = _load_cache()
        cache[key] = {"tile": list(best), "ms": times[best]}
        _save_cache(cache)
    return best


def tune_lattice(lat: "coulps.Lattice", n_hb=1, n_or=3, reps=3, stream=None):
    """Tunes both shapes; returns the half-sweep shape (the pass shape is
    applied too and readable from lat.info())."""
    s = stream or lat._stream
    best = tune_shape(lat.L, lat.n_chains, lat.precision, n_hb, n_or, reps, s)
    lat.set_tile(*best)
    pbest = tune_pass_shape(lat.L, lat.n_chains, lat.precision, n_hb, n_or, reps, s)
    lat.set_pass_tile(*pbest)
    return best


def tune_batch(batch: "coulps.Batch", n_hb=1, n_or=3, reps=3, stream=None):
    shapes = {}
    for L in batch.dims:
        shapes[L] = shapes.get(L, 0) + 1
    best = {L: tune_shape(L, cnt, batch.precision, n_hb, n_or, reps, stream)
            for L, cnt in shapes.items()}
    batch.set_tiles([best[L] for L in batch.dims])
    return best
