"""FP64 oracle of off-lattice charges and forces.

TEST INFRASTRUCTURE ONLY (same rules as oracle.py): loaded by tests/ and the
CPU legs of bench.py, never by the library.

The paper's closing remarks suggest that a particle need not sit on a lattice
site: its coordinate can be modelled through the eight lattice sites around
it, and forces evaluated by interpolation in the same way.  Here a particle at
r = (x, y, z) (0 <= x <= Lx - 1 etc.) takes the trilinear weights
    w_c(r) = prod_mu (c_mu ? f_mu : 1 - f_mu),   f = r - b,  b = floor(r)
(b clipped to L - 2 so that all eight corners b + c, c in {0,1}^3, are in the
box), so phi~(r) = sum_c w_c phi(b + c) and, per sample,
    Q = sum_i q_i phi~(r_i),  P = sum_i (q_i phi~(r_i))^2,  e = Q^2 - P
as in Eq. (nsum2).  Its mean is
    E = sum_{i != j} q_i q_j G~(r_i, r_j),  G~(r, s) = sum_{c,d} w_c(r) w_d(s) G(b_r + c, b_s + d).
The measure does not depend on the positions, so the force on particle i is
the mean of the derivative of e:
    F_i = -<de/dr_i> = -< 2 q_i (Q - q_i phi~_i) grad phi~_i >,
    grad phi~(r) = sum_c grad w_c(r) phi(b + c),
and its exact value is F_i = -2 q_i sum_{j != i} q_j grad_r G~(r_i, r_j).
"""
from __future__ import annotations

import itertools

import numpy as np

CORNERS = np.array(list(itertools.product((0, 1), repeat=3)))  # (c_x, c_y, c_z), x slowest


def corners(L, pos):
    """Corner sites (n, 8, 3) as (x, y, z), weights (n, 8) and weight
    gradients (n, 8, 3) of the trilinear interpolation."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    Lv = np.asarray(L, dtype=np.int64)
    base = np.clip(np.floor(pos).astype(np.int64), 0, np.maximum(Lv - 2, 0))
    f = pos - base
    sites = base[:, None, :] + CORNERS[None, :, :]
    fac = np.where(CORNERS[None, :, :] == 1, f[:, None, :], 1.0 - f[:, None, :])  # (n, 8, 3)
    dfac = np.where(CORNERS[None, :, :] == 1, 1.0, -1.0) * np.ones_like(fac)
    w = fac.prod(axis=2)
    grad = np.empty_like(fac)
    for mu in range(3):
        others = [m for m in range(3) if m != mu]
        grad[:, :, mu] = dfac[:, :, mu] * fac[:, :, others[0]] * fac[:, :, others[1]]
    return sites, w, grad


def interpolate(phi, L, pos):
    """phi~(r_i) and grad phi~(r_i) for one field (Lz, Ly, Lx)."""
    s, w, g = corners(L, pos)
    vals = phi[s[..., 2], s[..., 1], s[..., 0]]  # (n, 8)
    return (w * vals).sum(axis=1), (g * vals[..., None]).sum(axis=1)


def sample(phi, L, pos, q):
    """(Q, P, e) of one field."""
    t = np.asarray(q, dtype=np.float64) * interpolate(phi, L, pos)[0]
    Q, P = float(t.sum()), float((t * t).sum())
    return Q, P, Q * Q - P


def force_sample(phi, L, pos, q):
    """-de/dr_i = -2 q_i (Q - q_i phi~_i) grad phi~_i, shape (n, 3)."""
    q = np.asarray(q, dtype=np.float64)
    pt, gr = interpolate(phi, L, pos)
    Q = float((q * pt).sum())
    return -2.0 * (q * (Q - q * pt))[:, None] * gr


def _green_tilde(G, L, pos):
    """G~ (n, n) and its gradient in the first argument (n, n, 3), dense G."""
    Lx, Ly, Lz = L
    s, w, g = corners(L, pos)
    flat = s[..., 0] + Lx * (s[..., 1] + Ly * s[..., 2])  # (n, 8)
    Gc = G[flat[:, :, None, None], flat[None, None, :, :]]  # (n, 8, n, 8)
    Gt = np.einsum("ic,icjd,jd->ij", w, Gc, w)
    dGt = np.einsum("icm,icjd,jd->ijm", g, Gc, w)
    return Gt, dGt


def energy_exact(G, L, pos, q):
    """E = sum_{i != j} q_i q_j G~(r_i, r_j) with the dense lattice G."""
    q = np.asarray(q, dtype=np.float64)
    Gt, _ = _green_tilde(G, L, pos)
    return float(q @ Gt @ q - np.sum(q * q * np.diag(Gt)))


def force_exact(G, L, pos, q):
    """F_i = -2 q_i sum_{j != i} q_j grad_r G~(r_i, r_j), shape (n, 3)."""
    q = np.asarray(q, dtype=np.float64)
    _, dGt = _green_tilde(G, L, pos)
    n = len(q)
    mask = 1.0 - np.eye(n)
    return -2.0 * q[:, None] * np.einsum("ijm,j,ij->im", dGt, q, mask)
