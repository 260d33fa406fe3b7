"""FP64 oracle of the learned Stein control variate.

TEST INFRASTRUCTURE ONLY (same rules as oracle.py).

The control variate is not part of the paper; it rests on the integration-by-
parts (Stein) identity for the lattice measure exp(-H_L) of Eq. (proplat):
for any smooth vector field g(phi) with one component per site,
    E[ sum_x ( dg_x/dphi_x - g_x dH_L/dphi_x ) ] = 0,   dH_L/dphi = A phi,
so  e - T g,  T g = sum_x (dg_x/dphi_x - g_x (A phi)_x),  has the same mean
as the Eq. (nsum2) sample e and, for a good g, a smaller variance.

g is a 3-layer 3x3x3 convolutional net with zero padding:
    psi = (phi, rho, rho phi)              (rho = charge density per site)
    h1 = b1 + conv(psi, W1),  a1 = tanh(h1)       16 channels
    h2 = b2 + conv(a1,  W2),  a2 = tanh(h2)       16 channels
    g  = b3 + conv(a2,  W3)                        1 channel
conv(a, W)[co, x] = sum_{ci, d in {-1,0,1}^3} W[co, ci, d] a[ci, x + d]
(PyTorch conv3d's cross-correlation convention, W[co, ci, kz, ky, kx] with
d = (kz-1, ky-1, kx-1) acting on (z, y, x)).

The divergence is computed here by the plain chain rule, site by site:
    dg_x/dphi_x = sum_{c2, f} W3[c2, f] s2[c2, x+f]
                  sum_{c1, e} W2[c2, c1, e] s1[c1, x+f+e] w1_x[c1, -(f+e)],
    w1_x[c1, u] = W1[c1, 0, u] + rho_x W1[c1, 2, u]
(phi_x enters h1 through the phi channel and through the rho phi channel),
with s = tanh'(h) = 1 - a^2, every position inside the box and -(f+e) a
valid kernel offset.  Arrays are (C, Lz, Ly, Lx).
"""
from __future__ import annotations

import itertools

import numpy as np

OFFS = list(itertools.product((-1, 0, 1), repeat=3))  # (dz, dy, dx), index 9kz+3ky+kx


def _shift(a, d):
    """b[..., z, y, x] = a[..., z+dz, y+dy, x+dx] with zeros outside."""
    dz, dy, dx = d
    out = np.zeros_like(a)
    Z, Y, X = a.shape[-3:]
    zs, ys, xs = slice(max(0, -dz), Z - max(0, dz)), slice(max(0, -dy), Y - max(0, dy)), \
        slice(max(0, -dx), X - max(0, dx))
    zt, yt, xt = slice(max(0, dz), Z - max(0, -dz)), slice(max(0, dy), Y - max(0, -dy)), \
        slice(max(0, dx), X - max(0, -dx))
    out[..., zs, ys, xs] = a[..., zt, yt, xt]
    return out


def conv(a, W, b=None):
    """conv(a, W)[co] = sum_{ci, d} W[co, ci, d] a[ci, x + d]; a (Ci, Z, Y, X)."""
    co = W.shape[0]
    out = np.zeros((co,) + a.shape[1:])
    for k, d in enumerate(OFFS):
        kz, ky, kx = d[0] + 1, d[1] + 1, d[2] + 1
        out += np.tensordot(W[:, :, kz, ky, kx], _shift(a, d), axes=(1, 0))
    if b is not None:
        out += b.reshape(-1, 1, 1, 1)
    return out


def forward(phi, rho, p):
    psi = np.stack([phi, rho, rho * phi])
    h1 = conv(psi, p["W1"], p["b1"])
    a1 = np.tanh(h1)
    h2 = conv(a1, p["W2"], p["b2"])
    a2 = np.tanh(h2)
    g = conv(a2, p["W3"], p["b3"])[0]
    return {"h1": h1, "a1": a1, "h2": h2, "a2": a2, "g": g}


def region_mask(shape, region):
    """1 inside region = ((z0, z1), (y0, y1), (x0, x1)) (half-open), else 0."""
    m = np.zeros(shape)
    if region is None:
        m[...] = 1.0
        return m
    (z0, z1), (y0, y1), (x0, x1) = region
    m[z0:z1, y0:y1, x0:x1] = 1.0
    return m


def divergence(phi, rho, p, region=None):
    """sum_x dg_x/dphi_x by the chain rule (positions outside the box absent);
    with a region, only x inside it (g is taken as 0 elsewhere)."""
    f = forward(phi, rho, p)
    s1, s2 = 1.0 - f["a1"] ** 2, 1.0 - f["a2"] ** 2
    W1, W2, W3 = p["W1"], p["W2"], p["W3"]
    mask = region_mask(phi.shape, region)[None]
    total = 0.0
    for fo in OFFS:
        s2f = _shift(s2, fo)  # s2[c2, x+f] (0 outside)
        w3 = W3[0, :, fo[0] + 1, fo[1] + 1, fo[2] + 1]  # (c2,)
        for eo in OFFS:
            u = (-(fo[0] + eo[0]), -(fo[1] + eo[1]), -(fo[2] + eo[2]))
            if max(abs(v) for v in u) > 1:
                continue
            w1 = W1[:, 0, u[0] + 1, u[1] + 1, u[2] + 1]  # (c1,)
            w1r = W1[:, 2, u[0] + 1, u[1] + 1, u[2] + 1]  # (c1,), times rho_x
            w2 = W2[:, :, eo[0] + 1, eo[1] + 1, eo[2] + 1]  # (c2, c1)
            # s1 at x+f+e, defined only where x+f is inside (s2f carries that)
            s1fe = _shift(_shift(s1, eo), fo)
            inner = np.tensordot(w2 * w1[None, :], s1fe, axes=(1, 0))  # (c2, Z, Y, X)
            inner += rho[None] * np.tensordot(w2 * w1r[None, :], s1fe, axes=(1, 0))
            total += float(np.sum(w3[:, None, None, None] * s2f * inner * mask))
    return total


def apply_A(phi):
    out = 6.0 * phi
    out[1:] -= phi[:-1]
    out[:-1] -= phi[1:]
    out[:, 1:] -= phi[:, :-1]
    out[:, :-1] -= phi[:, 1:]
    out[:, :, 1:] -= phi[:, :, :-1]
    out[:, :, :-1] -= phi[:, :, 1:]
    return out


def stein_term(phi, rho, p, region=None):
    """T g = sum_x (dg_x/dphi_x - g_x (A phi)_x); with a region, g is the net
    inside it and 0 outside (still a smooth field, so E[T g] = 0)."""
    g = forward(phi, rho, p)["g"] * region_mask(phi.shape, region)
    return divergence(phi, rho, p, region) - float(np.sum(g * apply_A(phi)))


def random_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((16, 3, 3, 3, 3)) * scale,
        "b1": rng.standard_normal(16) * 0.1,
        "W2": rng.standard_normal((16, 16, 3, 3, 3)) * scale / 4,
        "b2": rng.standard_normal(16) * 0.1,
        "W3": rng.standard_normal((1, 16, 3, 3, 3)) * scale / 4,
        "b3": rng.standard_normal(1) * 0.1,
    }


def global_stein_term(phi, rho, h):
    """T g for the global control variate g_x = Q(phi) h_x, Q = sum_x rho_x phi_x
    and h a fixed field: dg_x/dphi_x = rho_x h_x, so
        T g = sum_x rho_x h_x - Q sum_x h_x (A phi)_x = h . rho - Q (A h) . phi
    (A symmetric).  Mean 0 under exp(-H_L) for any h; with h = -G rho it equals
    Q^2 - rho . G rho for every phi."""
    Q = float(np.sum(rho * phi))
    return float(np.sum(h * rho) - Q * np.sum(apply_A(h) * phi))


def cube_green(R):
    """Dirichlet Green function of the (2R+1)^3 cube at its centre, (dz, dy, dx)
    from -R to R: the column of the dense inverse of the cube's A."""
    from oracle import oracle
    m = 2 * R + 1
    G = oracle.green_dense((m, m, m))
    return G[:, (R * m + R) * m + R].reshape(m, m, m)


def local_p_stein_term(phi, sites, q, k):
    """T g for g_x = sum_i q_i^2 phi(r_i) k(x - r_i) (x in the box, k of radius
    R = (len(k) - 1) / 2 indexed [dz + R, dy + R, dx + R]):
        T g = k(0) sum_i q_i^2 - sum_i q_i^2 phi(r_i) w_i,
        w_i = sum_d k(d) (A phi)(r_i + d)   over r_i + d in the box.
    Mean 0 under exp(-H_L) for any k; sites are (x, y, z)."""
    R = (k.shape[0] - 1) // 2
    Lz, Ly, Lx = phi.shape
    Ap = apply_A(phi)
    q = np.asarray(q, dtype=np.float64)
    t = float(k[R, R, R] * np.sum(q * q))
    for (x, y, z), qi in zip(np.asarray(sites).reshape(-1, 3), q):
        z0, z1 = max(z - R, 0), min(z + R + 1, Lz)
        y0, y1 = max(y - R, 0), min(y + R + 1, Ly)
        x0, x1 = max(x - R, 0), min(x + R + 1, Lx)
        kk = k[z0 - (z - R):z1 - (z - R), y0 - (y - R):y1 - (y - R), x0 - (x - R):x1 - (x - R)]
        t -= qi * qi * phi[z, y, x] * float(np.sum(kk * Ap[z0:z1, y0:y1, x0:x1]))
    return t
