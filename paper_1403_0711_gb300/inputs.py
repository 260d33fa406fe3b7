"""Seeded synthetic charge sets.

This module only places charges; it holds none of the sampler's or the
estimator's arithmetic, so both the CUDA path and the oracle can take their
inputs from it.  Sites are int32 rows (x, y, z), 0-based, x fastest in the
field; charges are float64.  All generators draw from numpy's PCG64 seeded by
the caller and produce distinct sites.

Workloads (the paper's own experiments and the throughput workloads):
  two_body       Fig. 1: q=1 at (L/2, L/2, L/2) and q=1 at (n_x, L/2, L/2).
  cube           Fig. 2: N = n^3 charges q=1 filling the cube
                 L/2 - n/2 .. L/2 + n/2 - 1 on each axis (the paper's 1-based
                 range L/2 - n/2 + 1 .. L/2 + n/2, shifted to 0-based).
  plus_minus     N charges, exactly N/2 of +1 and N/2 of -1, uniformly random
                 distinct sites (zero net charge).
  uniform_q      N charges with q uniform in [-qmax, qmax], shifted by their
                 mean so the net charge is zero.
  blobs          N charges in n_blob Gaussian blobs (centres uniform in the
                 box, per-axis offsets round(N(0, sigma^2))), q uniform in
                 [-qmax, qmax] shifted to zero net charge.
  batch_systems  the many-system workload: edges drawn from a list, N
                 log-uniform, uniform_q charges per system.
"""
from __future__ import annotations

import math

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def _distinct_uniform_sites(rng, L, n):
    """n distinct sites uniform over the box, by rejection of repeats."""
    Lx, Ly, Lz = L
    vol = Lx * Ly * Lz
    if n > vol:
        raise ValueError("more charges than sites")
    chosen = np.empty(0, dtype=np.int64)
    seen = set()
    out = []
    while len(out) < n:
        draw = rng.integers(0, vol, size=max(16, 2 * (n - len(out))), dtype=np.int64)
        for v in draw.tolist():
            if v not in seen:
                seen.add(v)
                out.append(v)
                if len(out) == n:
                    break
    chosen = np.asarray(out, dtype=np.int64)
    x = chosen % Lx
    y = (chosen // Lx) % Ly
    z = chosen // (Lx * Ly)
    return np.stack([x, y, z], axis=1).astype(np.int32)


def two_body(L, nx):
    Lx, Ly, Lz = L
    sites = np.array([[Lx // 2, Ly // 2, Lz // 2], [nx, Ly // 2, Lz // 2]], dtype=np.int32)
    return sites, np.ones(2)


def cube(L, n_side, q=1.0):
    Lx, Ly, Lz = L
    rng_x = np.arange(Lx // 2 - n_side // 2, Lx // 2 - n_side // 2 + n_side)
    rng_y = np.arange(Ly // 2 - n_side // 2, Ly // 2 - n_side // 2 + n_side)
    rng_z = np.arange(Lz // 2 - n_side // 2, Lz // 2 - n_side // 2 + n_side)
    z, y, x = np.meshgrid(rng_z, rng_y, rng_x, indexing="ij")
    sites = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.int32)
    return sites, np.full(len(sites), float(q))


def plus_minus(L, n, seed):
    if n % 2:
        raise ValueError("plus_minus needs an even N")
    rng = _rng(seed)
    sites = _distinct_uniform_sites(rng, L, n)
    q = np.concatenate([np.ones(n // 2), -np.ones(n // 2)])
    rng.shuffle(q)
    return sites, q


def uniform_q(L, n, seed, qmax=1.0):
    rng = _rng(seed)
    sites = _distinct_uniform_sites(rng, L, n)
    q = rng.uniform(-qmax, qmax, size=n)
    if n > 0:
        q -= q.mean()
    return sites, q


def gaussian_fields(L, n, seed, scale=0.5):
    """n seeded test fields (Lz, Ly, Lx) of independent normal values times
    scale (about the size of a sampled field's fluctuations), for comparing
    field functions of the library and the oracle on the same inputs."""
    Lx, Ly, Lz = L
    rng = _rng(seed)
    return [scale * rng.standard_normal((Lz, Ly, Lx)) for _ in range(n)]


def off_lattice(L, n, seed, qmax=1.0):
    """n particles at real positions uniform in [0, L - 1] per axis (x, y, z),
    charges uniform in [-qmax, qmax]; a few are put on exact lattice points,
    box faces and the far corner (the edge cases of the corner choice)."""
    rng = _rng(seed)
    hi = np.asarray(L, dtype=np.float64) - 1.0
    pos = rng.uniform(0.0, 1.0, size=(n, 3)) * hi
    special = [hi, np.zeros(3), np.floor(hi / 2), np.array([hi[0], 0.0, hi[2] / 3])]
    for k in range(min(n // 2, len(special))):
        pos[k] = special[k]
    q = rng.uniform(-qmax, qmax, size=n)
    return pos, q


def off_lattice_cube(L, n_side, seed, jitter=0.3, q=1.0):
    """The paper's Fig. 2 cube of n_side^3 charges q at the centre of the box,
    each moved off its site by a uniform offset in [-jitter, jitter] per axis
    (real positions (x, y, z))."""
    sites, qq = cube(L, n_side, q)
    rng = _rng(seed)
    pos = sites.astype(np.float64) + rng.uniform(-jitter, jitter, size=sites.shape)
    return pos, qq


def blobs(L, n, seed, n_blob=200, sigma=6.0, qmax=0.8):
    Lx, Ly, Lz = L
    rng = _rng(seed)
    centres = np.stack([rng.integers(0, Lx, n_blob), rng.integers(0, Ly, n_blob),
                        rng.integers(0, Lz, n_blob)], axis=1)
    seen = set()
    out = []
    while len(out) < n:
        m = max(1024, 2 * (n - len(out)))
        b = rng.integers(0, n_blob, m)
        off = np.rint(rng.normal(0.0, sigma, size=(m, 3))).astype(np.int64)
        p = centres[b] + off
        ok = ((p[:, 0] >= 0) & (p[:, 0] < Lx) & (p[:, 1] >= 0) & (p[:, 1] < Ly)
              & (p[:, 2] >= 0) & (p[:, 2] < Lz))
        lin = (p[:, 0] + Lx * (p[:, 1] + Ly * p[:, 2]))[ok]
        for v in lin.tolist():
            if v not in seen:
                seen.add(v)
                out.append(v)
                if len(out) == n:
                    break
    lin = np.asarray(out, dtype=np.int64)
    sites = np.stack([lin % Lx, (lin // Lx) % Ly, lin // (Lx * Ly)], axis=1).astype(np.int32)
    q = rng.uniform(-qmax, qmax, size=n)
    q -= q.mean()
    return sites, q


def batch_systems(n_systems, seed, edges=(32, 48, 64, 80, 96), n_min=64, n_max=2048):
    """List of (L, sites, q) for the many-system workload."""
    rng = _rng(seed)
    out = []
    for s in range(n_systems):
        e = int(edges[rng.integers(0, len(edges))])
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        L = (e, e, e)
        sub_seed = int(rng.integers(0, 2**62))
        sites, q = uniform_q(L, n, sub_seed)
        out.append((L, sites, q))
    return out
