"""Pins of the control-variate oracle (oracle/stein.py).

- The chain-rule divergence equals central finite differences of g_x in phi_x.
- Under exact Gaussian samples phi = L^-T z (A = L L^T, so phi ~ exp(-H_L)),
  the Stein term has mean zero within 4 sigma, while each of its two parts
  alone does not (the test has power).
"""
import math

import numpy as np


import pytest


@pytest.mark.parametrize("only_rho_phi", [False, True])
def test_divergence_matches_finite_differences(only_rho_phi):
    """With only_rho_phi, phi reaches the net through the rho phi channel
    alone, so the divergence is entirely the rho_x W1[:, 2] term."""
    from oracle import stein
    rng = np.random.default_rng(0)
    Z, Y, X = 3, 4, 5
    phi = rng.standard_normal((Z, Y, X))
    rho = np.zeros((Z, Y, X))
    rho[1, 2, 3], rho[0, 1, 1] = 1.0, -1.0
    p = stein.random_params(1)
    if only_rho_phi:
        p["W1"][:, 0] = 0.0
    div = stein.divergence(phi, rho, p)
    h = 1e-5
    fd = 0.0
    for z in range(Z):
        for y in range(Y):
            for x in range(X):
                a, b = phi.copy(), phi.copy()
                a[z, y, x] += h
                b[z, y, x] -= h
                fd += (stein.forward(a, rho, p)["g"][z, y, x] - stein.forward(b, rho, p)["g"][z, y, x]) / (2 * h)
    assert abs(div - fd) < 1e-7 * max(1.0, abs(div)), (div, fd)


def test_stein_term_has_zero_mean_under_exact_samples(orc):
    from oracle import stein
    L = (3, 3, 3)
    A = orc.laplacian_dense(L)
    C = np.linalg.cholesky(A)
    rng = np.random.default_rng(5)
    rho = np.zeros((3, 3, 3))
    rho[1, 1, 1], rho[0, 2, 1] = 1.0, -1.0
    p = stein.random_params(3, scale=0.6)
    n = 3000
    tg, div_only, gA_only = [], [], []
    for _ in range(n):
        z = rng.standard_normal(27)
        phi = np.linalg.solve(C.T, z).reshape(3, 3, 3)
        d = stein.divergence(phi, rho, p)
        g = stein.forward(phi, rho, p)["g"]
        ga = float(np.sum(g * stein.apply_A(phi)))
        tg.append(d - ga)
        div_only.append(d)
        gA_only.append(ga)
    tg = np.array(tg)
    se = tg.std(ddof=1) / math.sqrt(n)
    assert abs(tg.mean()) < 4 * se, (tg.mean(), se)
    # each part alone has a clearly non-zero mean
    d = np.array(div_only)
    assert abs(d.mean()) > 8 * d.std(ddof=1) / math.sqrt(n)


def test_region_divergence_matches_finite_differences():
    """g restricted to a region (zero outside): the divergence sums over the
    region only and still equals finite differences of the masked g."""
    from oracle import stein
    rng = np.random.default_rng(2)
    Z, Y, X = 5, 6, 7
    phi = rng.standard_normal((Z, Y, X))
    rho = np.zeros((Z, Y, X))
    rho[2, 3, 3], rho[2, 3, 1] = 1.0, 0.7  # one charge outside the region, one inside
    p = stein.random_params(4)
    region = ((1, 4), (2, 5), (0, 3))
    m = stein.region_mask(phi.shape, region)
    div = stein.divergence(phi, rho, p, region)
    h = 1e-5
    fd = 0.0
    for z, y, x in zip(*np.nonzero(m)):
        a, b = phi.copy(), phi.copy()
        a[z, y, x] += h
        b[z, y, x] -= h
        fd += (stein.forward(a, rho, p)["g"][z, y, x] - stein.forward(b, rho, p)["g"][z, y, x]) / (2 * h)
    assert abs(div - fd) < 1e-7 * max(1.0, abs(div))


def test_global_stein_term_matches_finite_differences_and_closed_form(orc):
    """Global control variate g = Q h: the divergence by finite differences of g,
    and with h = -G rho (dense inverse) the closed form T g = Q^2 - rho.G.rho
    for an arbitrary phi."""
    from oracle import stein
    L = (4, 3, 5)
    rng = np.random.default_rng(11)
    phi = rng.standard_normal((L[2], L[1], L[0]))
    rho = np.zeros_like(phi)
    rho[1, 1, 2], rho[3, 0, 0], rho[4, 2, 3] = 1.0, -1.0, 0.5
    h = rng.standard_normal(phi.shape)
    # T g from its definition: divergence by central differences of g_x = Q h_x
    eps = 1e-6
    div = 0.0
    for idx in np.ndindex(phi.shape):
        a, b = phi.copy(), phi.copy()
        a[idx] += eps
        b[idx] -= eps
        div += (np.sum(rho * a) * h[idx] - np.sum(rho * b) * h[idx]) / (2 * eps)
    g = np.sum(rho * phi) * h
    tg_def = div - float(np.sum(g * stein.apply_A(phi)))
    tg = stein.global_stein_term(phi, rho, h)
    assert abs(tg - tg_def) < 1e-7 * max(1.0, abs(tg)), (tg, tg_def)
    # closed form with h = -G rho
    G = orc.green_dense(L)
    r = rho.reshape(-1)
    hG = -(G @ r).reshape(phi.shape)
    Q = float(np.sum(rho * phi))
    assert abs(stein.global_stein_term(phi, rho, hG) - (Q * Q - r @ G @ r)) < 1e-12 * (1 + Q * Q)


def test_global_stein_term_has_zero_mean_under_exact_samples(orc):
    from oracle import stein
    L = (3, 4, 3)
    A = orc.laplacian_dense(L)
    C = np.linalg.cholesky(A)
    rng = np.random.default_rng(12)
    rho = np.zeros((L[2], L[1], L[0]))
    rho[1, 1, 1], rho[0, 3, 2], rho[2, 0, 0] = 1.0, -1.0, 0.7
    h = rng.standard_normal(rho.shape) + 2.0 * rho  # h . rho clearly non-zero
    n = 20000
    z = rng.standard_normal((n, A.shape[0]))
    phis = np.linalg.solve(C.T, z.T).T.reshape(n, L[2], L[1], L[0])
    tg = np.array([stein.global_stein_term(p, rho, h) for p in phis])
    se = tg.std(ddof=1) / math.sqrt(n)
    assert abs(tg.mean()) < 4 * se, (tg.mean(), se)
    # the second part alone averages to h . rho, not 0 (the test has power)
    qa = np.array([np.sum(rho * p) * np.sum(stein.apply_A(h) * p) for p in phis])
    assert abs(qa.mean()) > 8 * qa.std(ddof=1) / math.sqrt(n)
    assert abs(qa.mean() - np.sum(h * rho)) < 4 * qa.std(ddof=1) / math.sqrt(n)


def test_local_p_term_matches_definition_and_has_zero_mean(orc):
    """Local term of P: g_x = sum_i q_i^2 phi(r_i) k(x - r_i).  Its Stein term
    equals the definition (divergence by central differences, g . A phi by
    hand) with charges at the box faces, and averages to 0 under exact
    samples; with k the cube Green function A k = e_centre inside the cube."""
    from oracle import stein
    k = stein.cube_green(1)
    # A k = delta inside the cube (k = 0 outside it)
    Ak = stein.apply_A(k)
    assert abs(Ak[1, 1, 1] - 1.0) < 1e-12 and np.abs(np.delete(Ak.reshape(-1), 13)).max() < 1e-12
    L = (5, 4, 3)
    rng = np.random.default_rng(3)
    phi = rng.standard_normal((L[2], L[1], L[0]))
    sites = np.array([[0, 0, 0], [2, 1, 1], [4, 3, 2], [3, 1, 1]])
    q = np.array([1.0, -0.5, 0.8, 1.0])

    def g_of(p):
        g = np.zeros_like(p)
        for (x, y, z), qi in zip(sites, q):
            for dz in range(-1, 2):
                for dy in range(-1, 2):
                    for dx in range(-1, 2):
                        xx, yy, zz = x + dx, y + dy, z + dz
                        if 0 <= xx < L[0] and 0 <= yy < L[1] and 0 <= zz < L[2]:
                            g[zz, yy, xx] += qi * qi * p[z, y, x] * k[dz + 1, dy + 1, dx + 1]
        return g

    eps = 1e-6
    div = 0.0
    for idx in np.ndindex(phi.shape):
        a, b = phi.copy(), phi.copy()
        a[idx] += eps
        b[idx] -= eps
        div += (g_of(a)[idx] - g_of(b)[idx]) / (2 * eps)
    tg_def = div - float(np.sum(g_of(phi) * stein.apply_A(phi)))
    tg = stein.local_p_stein_term(phi, sites, q, k)
    assert abs(tg - tg_def) < 1e-7 * max(1.0, abs(tg)), (tg, tg_def)
    # zero mean under exact samples
    A = orc.laplacian_dense(L)
    C = np.linalg.cholesky(A)
    n = 20000
    z = rng.standard_normal((n, A.shape[0]))
    phis = np.linalg.solve(C.T, z.T).T.reshape(n, L[2], L[1], L[0])
    t = np.array([stein.local_p_stein_term(p, sites, q, k) for p in phis])
    assert abs(t.mean()) < 4 * t.std(ddof=1) / math.sqrt(n), (t.mean(), t.std())
