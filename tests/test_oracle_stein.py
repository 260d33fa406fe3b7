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
