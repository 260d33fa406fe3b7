"""Autotuner for the tile shapes (ty rows x dz planes per CTA) of the
half-sweep kernel, the fused-pass kernel and the pass-pair kernel.

The shape changes only the work decomposition, never the results (the tests
check fields bitwise across shapes), so the tuner may pick freely.  For a box
shape it times every candidate with the library's own per-kernel CUDA-event
timing (coulps_set_profiling / coulps_kernel_times) over a few compound
sweeps and keeps the fastest.  Results are cached in a JSON file keyed by box,
chain count, precision, compound-sweep mix and GPU name
($COULPS_TUNE_CACHE, default ~/.cache/coulps_tune.json).

tune_lattice(lat)  tunes and applies the three shapes of a Lattice (the
                   half-sweep shape serves passes that are not fused).
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


def pair_candidates(L, precision):
    """Pass-pair tile shapes: (ty + 6) rows of quads within 512 threads (FP32)
    or 256 (FP64), colour-1 boxes of ty + 8 <= 256 rows."""
    Lx, Ly, Lz = L
    qw = row_stride(Lx, precision) // 4
    max_threads = 512 if precision == coulps.F32 else 256
    tys = sorted({t for t in (4, 6, 8, 10, 14, 18, 22, 26, 42, 58, 122)
                  if t <= Ly and qw * (t + 6) <= max_threads and t + 8 <= 256} |
                 ({min(Ly, max_threads // qw - 6, 248)} if max_threads // qw - 6 >= 1 else set()))
    dzs = sorted({d for d in (16, 32, 64, 128) if d <= Lz} | {Lz})
    return [(t, d) for t in tys for d in dzs]


def _time_shapes(L, n_chains, precision, shapes, n_hb, n_or, reps, stream, fused=False,
                 pair=False):
    """Device time of the sweep kernels per `reps` compound sweeps for each
    shape: half-sweep tiles (default), fused-pass tiles (fused=True, all
    passes fused) or pass-pair tiles (pair=True, over-relaxation pairs)."""
    lat = coulps.Lattice(L, n_chains=n_chains, precision=precision, seed=1, stream=stream)
    lat.set_fused(3 if pair else (2 if fused else 0))
    lat.set_profiling(True)
    out = {}
    try:
        lat.sweep(2, n_hb, n_or)
        for ty, dz in shapes:
            try:
                if pair:
                    lat.set_pair_tile(ty, dz)
                elif fused:
                    lat.set_pass_tile(ty, dz)
                else:
                    lat.set_tile(ty, dz)
            except coulps.CoulpsError:
                continue  # a shape the library refuses (e.g. its shared memory would not fit)
            lat.sweep(1, n_hb, n_or)
            lat.kernel_times()
            lat.sweep(reps, n_hb, n_or)
            kt = lat.kernel_times()
            out[(ty, dz)] = sum(v for k, v in kt.items() if k.endswith("_ms"))
    finally:
        lat.close()
    return out


def _best(times, L, what):
    """The fastest shape; an error naming the box when the library refused
    every candidate."""
    if not times:
        raise coulps.CoulpsError(
            coulps.EINVAL, f"autotune: the library refused every {what} tile shape for box {L}")
    return min(times, key=times.get)


def tune_shape(L, n_chains=1, precision=coulps.F32, n_hb=1, n_or=3, reps=3, stream=None,
               use_cache=True):
    """Best (ty, dz) for a box shape; cached."""
    L = tuple(int(v) for v in L)
    key = f"{L[0]}x{L[1]}x{L[2]}|{n_chains}|{precision}|{n_hb}:{n_or}|{_gpu_name()}"
    cache = _load_cache() if use_cache else {}
    if key in cache:
        return tuple(cache[key]["tile"])
    times = _time_shapes(L, n_chains, precision, candidates(L, precision), n_hb, n_or, reps, stream)
    best = _best(times, L, "half-sweep")
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
    best = _best(times, L, "fused-pass")
    if use_cache:
        cache = _load_cache()
        cache[key] = {"tile": list(best), "ms": times[best]}
        _save_cache(cache)
    return best


def tune_pair_shape(L, n_chains=1, precision=coulps.F32, n_hb=1, n_or=3, reps=3, stream=None,
                    use_cache=True):
    """Best pass-pair (ty, dz) for a box shape (the schedule of fused mode 3:
    heatbath half-sweeps, over-relaxation pairs); cached.  None when the row
    is too wide for a pair CTA."""
    L = tuple(int(v) for v in L)
    cands = pair_candidates(L, precision)
    if not cands:
        return None
    key = f"pair|{L[0]}x{L[1]}x{L[2]}|{n_chains}|{precision}|{n_hb}:{n_or}|{_gpu_name()}"
    cache = _load_cache() if use_cache else {}
    if key in cache:
        return tuple(cache[key]["tile"])
    times = _time_shapes(L, n_chains, precision, cands, n_hb, n_or, reps, stream, pair=True)
    best = _best(times, L, "pass-pair")
    if use_cache:
        cache = _load_cache()
        cache[key] = {"tile": list(best), "ms": times[best]}
        _save_cache(cache)
    return best


def tune_lattice(lat: "coulps.Lattice", n_hb=1, n_or=3, reps=3, stream=None):
    """Tunes the half-sweep, fused-pass and pass-pair shapes; returns the
    half-sweep shape (the others are applied too: lat.info(), lat.pair_tile())."""
    s = stream or lat._stream
    best = tune_shape(lat.L, lat.n_chains, lat.precision, n_hb, n_or, reps, s)
    lat.set_tile(*best)
    pbest = tune_pass_shape(lat.L, lat.n_chains, lat.precision, n_hb, n_or, reps, s)
    lat.set_pass_tile(*pbest)
    qbest = tune_pair_shape(lat.L, lat.n_chains, lat.precision, n_hb, n_or, reps, s)
    if qbest is not None and lat.pair_tile()[0] > 0:
        lat.set_pair_tile(*qbest)
    return best


def tune_batch(batch: "coulps.Batch", n_hb=1, n_or=3, reps=3, stream=None):
    shapes = {}
    for L in batch.dims:
        shapes[L] = shapes.get(L, 0) + 1
    best = {L: tune_shape(L, cnt, batch.precision, n_hb, n_or, reps, stream)
            for L, cnt in shapes.items()}
    batch.set_tiles([best[L] for L in batch.dims])
    return best
