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


# --------------------------------------------------------------------------
# Near-field direct correction
# --------------------------------------------------------------------------
# The paper's closing remarks propose computing close particles directly,
# because the lattice Green function misrepresents the steep core of the
# Coulomb potential.  Reading used here: the near set N = {(i, j): i < j,
# |r_i - r_j| < r_c} is fixed when the set is built; its pairs are removed
# from every sample,
#     e_far = Q^2 - P - s_N,   s_N = 2 sum_{(i,j) in N} q_i q_j phi~_i phi~_j,
# (the mean of e_far is the lattice energy of the far pairs) and added back
# with the continuum kernel of Eq. (s1),
#     E_N^direct = 2 sum_{(i,j) in N} q_i q_j / (4 pi |r_i - r_j|),
# so that E ~ <e_far> + E_N^direct.  Forces follow in the same way.


def near_pairs(pos, rc):
    """All pairs i < j with |r_i - r_j| < rc, shape (m, 2), by brute force."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    out = []
    for i in range(len(pos)):
        for j in range(i + 1, len(pos)):
            if np.sqrt(np.sum((pos[i] - pos[j]) ** 2)) < rc:
                out.append((i, j))
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def near_sample(phi, L, pos, q, pairs):
    """(Q, P + s_N, e_far) of one field: s_N moves into the subtracted part
    so that e_far = Q^2 - (P + s_N)."""
    q = np.asarray(q, dtype=np.float64)
    t = q * interpolate(phi, L, pos)[0]
    Q, P = float(t.sum()), float((t * t).sum())
    s = 0.0
    for i, j in pairs:
        s += 2.0 * t[i] * t[j]
    return Q, P + s, Q * Q - P - s


def near_force_sample(phi, L, pos, q, pairs):
    """-de_far/dr_i = -2 q_i (Q - q_i phi~_i - sum_{j near i} q_j phi~_j) grad phi~_i."""
    q = np.asarray(q, dtype=np.float64)
    pt, gr = interpolate(phi, L, pos)
    t = q * pt
    u = np.zeros(len(q))
    for i, j in pairs:
        u[i] += t[j]
        u[j] += t[i]
    Q = float(t.sum())
    return -2.0 * (q * (Q - t - u))[:, None] * gr


def near_direct_energy(pos, q, pairs):
    """E_N^direct = 2 sum_{(i,j) in N} q_i q_j / (4 pi r_ij)."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    tot = 0.0
    for i, j in pairs:
        tot += 2.0 * q[i] * q[j] / np.sqrt(np.sum((pos[i] - pos[j]) ** 2))
    return tot / (4.0 * np.pi)


def near_direct_forces(pos, q, pairs):
    """-dE_N^direct/dr_i = 2 q_i sum_{j near i} q_j (r_i - r_j) / (4 pi r_ij^3)."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    F = np.zeros_like(pos)
    for i, j in pairs:
        d = pos[i] - pos[j]
        r = np.sqrt(np.sum(d * d))
        f = 2.0 * q[i] * q[j] * d / (4.0 * np.pi * r ** 3)
        F[i] += f
        F[j] -= f
    return F


def far_energy_exact(G, L, pos, q, pairs):
    """Mean of e_far: the exact interpolated-lattice energy without the pairs of N."""
    q = np.asarray(q, dtype=np.float64)
    Gt, _ = _green_tilde(G, L, pos)
    E = float(q @ Gt @ q - np.sum(q * q * np.diag(Gt)))
    for i, j in pairs:
        E -= 2.0 * q[i] * q[j] * Gt[i, j]
    return E


def far_force_exact(G, L, pos, q, pairs):
    """Mean of -de_far/dr_i: -2 q_i sum_{j != i, (i,j) not in N} q_j grad_r G~(r_i, r_j)."""
    q = np.asarray(q, dtype=np.float64)
    _, dGt = _green_tilde(G, L, pos)
    n = len(q)
    mask = 1.0 - np.eye(n)
    for i, j in pairs:
        mask[i, j] = mask[j, i] = 0.0
    return -2.0 * q[:, None] * np.einsum("ijm,j,ij->im", dGt, q, mask)


def _corner_pairs(L, pos_a, pos_b):
    """Flattened corner-site pairs and weight products of particle pairs
    (a_k, b_k): returns sites_a (m*64, 3), sites_b (m*64, 3), weights (m*64,)."""
    sa, wa, _ = corners(L, pos_a)
    sb, wb, _ = corners(L, pos_b)
    m = len(sa)
    A = np.repeat(sa, 8, axis=1).reshape(m * 64, 3)
    B = np.tile(sb, (1, 8, 1)).reshape(m * 64, 3)
    W = (wa[:, :, None] * wb[:, None, :]).reshape(m * 64)
    return A, B, W


def far_energy_solve(L, pos, q, pairs, chunk=2048):
    """far_energy_exact for large boxes without a dense G:
        rho~^T G rho~ - sum_i q_i^2 G~(r_i, r_i) - 2 sum_{(i,j) in N} q_i q_j G~(r_i, r_j),
    rho~ = sum_i q_i w_i (the particles' weights spread on the lattice), G rho~
    by the oracle's DST-I solve, G~ of particle pairs as weighted sums of
    lattice G entries by heat-kernel quadrature."""
    from . import oracle
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64)
    Lx, Ly, Lz = L
    s, w, _ = corners(L, pos)
    rho = np.zeros((Lz, Ly, Lx))
    np.add.at(rho, (s[..., 2].ravel(), s[..., 1].ravel(), s[..., 0].ravel()),
              (q[:, None] * w).ravel())
    E = float(np.vdot(rho, oracle.solve_dst(rho)))

    def gtilde(ia, ib):
        out = np.empty(len(ia))
        for k0 in range(0, len(ia), chunk):
            a, b = ia[k0:k0 + chunk], ib[k0:k0 + chunk]
            A, B, W = _corner_pairs(L, pos[a], pos[b])
            out[k0:k0 + chunk] = (oracle.green_pairs(L, A, B) * W).reshape(len(a), 64).sum(axis=1)
        return out

    idx = np.arange(len(q))
    E -= float(np.sum(q * q * gtilde(idx, idx)))
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    if len(pairs):
        E -= 2.0 * float(np.sum(q[pairs[:, 0]] * q[pairs[:, 1]] * gtilde(pairs[:, 0], pairs[:, 1])))
    return E
