"""Pins of the oracle's exact lattice energy.

The exact value the sampler converges to is E_lat = sum_{i!=j} q_i q_j G_ij with
G = A^{-1}, A the matrix of H_L = 1/2 phi^T A phi (Eq. (proplat), phi = 0 outside
the box).  The pins are independent of each other:
  - A built site by site from H_L vs the stencil apply_A and vs 2*H_L itself;
  - three independent solvers (Cholesky, sine transform, CG) agree and satisfy
    A G = I through the stencil;
  - the heat-kernel quadrature of G_ii / G_ij agrees with the dense inverse;
  - the infinite-lattice G(0) equals Watson's closed form (golden fixture),
    G(1,0,0) = G(0) - 1/6 exactly (a row of A G = I plus cubic symmetry), and
    4 pi r G(r) -> 1 (the paper's continuum limit 1/(4 pi r));
  - deep inside a finite box, G(c, c+r) - G(c, c+2r) matches the
    infinite-lattice difference, which times 8 pi r approaches 1;
  - box symmetries and E_lat of two charges = 2 q1 q2 G_12 (Fig. 1's setup).
"""
import math
from pathlib import Path

import numpy as np
import pytest
import scipy.special as ss

GOLDEN = Path(__file__).resolve().parent / "golden"


def _watson():
    for line in (GOLDEN / "watson.txt").read_text().splitlines():
        if line.startswith("W_s"):
            return float(line.split()[1])


def test_dense_A_matches_action(orc):
    L = (3, 4, 2)
    A = orc.laplacian_dense(L)
    rng = np.random.default_rng(1)
    phi = rng.standard_normal((L[2], L[1], L[0]))
    v = phi.reshape(-1)
    assert abs(0.5 * v @ A @ v - orc.action(phi)) < 1e-12 * abs(orc.action(phi))
    assert np.allclose((A @ v).reshape(phi.shape), orc.apply_A(phi), atol=1e-13)
    assert np.allclose(A, A.T)
    assert np.all(np.diag(A) == 6.0)


@pytest.mark.parametrize("L", [(1, 1, 1), (2, 2, 2), (3, 4, 5), (6, 6, 6), (7, 2, 3)])
def test_three_solvers_agree(orc, L):
    G = orc.green_dense(L)
    rng = np.random.default_rng(sum(L))
    rho = rng.standard_normal((L[2], L[1], L[0]))
    u_dense = (G @ rho.reshape(-1)).reshape(rho.shape)
    u_dst = orc.solve_dst(rho)
    u_cg, _ = orc.solve_cg(rho, rtol=1e-14)
    scale = np.abs(u_dense).max()
    assert np.abs(u_dst - u_dense).max() < 1e-13 * scale
    assert np.abs(u_cg - u_dense).max() < 1e-11 * scale
    # A G = I through the stencil (not through the dense A)
    assert np.abs(orc.apply_A(u_dst) - rho).max() < 1e-12 * np.abs(rho).max()


def test_single_site_green(orc):
    # one site, all six neighbours are ghosts: A = 6, G = 1/6
    assert abs(orc.green_dense((1, 1, 1))[0, 0] - 1.0 / 6.0) < 1e-15


def test_heat_kernel_diag_and_pairs(orc):
    L = (6, 5, 7)
    G = orc.green_dense(L)
    rng = np.random.default_rng(3)
    sites = np.stack([rng.integers(0, L[0], 20), rng.integers(0, L[1], 20),
                      rng.integers(0, L[2], 20)], axis=1)
    idx = orc.site_index(L, sites)
    assert np.abs(orc.green_diag(L, sites) - np.diag(G)[idx]).max() < 1e-12
    a, b = sites[:10], sites[10:]
    gp = orc.green_pairs(L, a, b)
    assert np.abs(gp - G[orc.site_index(L, a), orc.site_index(L, b)]).max() < 1e-12


def test_green_box_symmetries(orc):
    L = (4, 4, 4)
    G = orc.green_dense(L)
    Gr = G.reshape(4, 4, 4, 4, 4, 4)  # (z,y,x, z',y',x')
    assert np.allclose(G, G.T, atol=1e-15)
    # reflection x -> 3 - x, and the x<->z axis swap of the cube
    assert np.allclose(Gr, Gr[:, :, ::-1, :, :, ::-1], atol=1e-15)
    assert np.allclose(Gr, Gr.transpose(2, 1, 0, 5, 4, 3), atol=1e-15)


def test_watson_closed_form_and_golden():
    w_closed = (math.sqrt(6) / (32 * math.pi ** 3) * ss.gamma(1 / 24) * ss.gamma(5 / 24)
                * ss.gamma(7 / 24) * ss.gamma(11 / 24))
    assert abs(w_closed - _watson()) < 1e-14


def test_infinite_lattice_green(orc):
    g0 = orc.green_infinite((0, 0, 0))
    assert abs(g0 - _watson() / 6.0) < 1e-12
    g1 = orc.green_infinite((1, 0, 0))
    assert abs(g1 - (g0 - 1.0 / 6.0)) < 1e-12
    assert abs(orc.green_infinite((0, 1, 0)) - g1) < 1e-13
    # continuum limit of Eq. (proplat): 4 pi r G(r) -> 1
    prev = None
    for r in (2, 4, 8, 16, 32):
        v = 4 * math.pi * r * orc.green_infinite((r, 0, 0))
        assert v > 1.0
        if prev is not None:
            assert v - 1.0 < 0.3 * (prev - 1.0)  # O(1/r^2) approach
        prev = v
    assert abs(prev - 1.0) < 3e-4


def test_box_green_differences_continuum(orc):
    # Deep inside a box, G(c, c+r) - G(c, c+2r) approaches the infinite-lattice
    # difference (the box's regular part cancels to leading order), and that
    # difference times 8 pi r approaches 1 = the continuum 1/(4 pi r) - 1/(8 pi r).
    L = (48, 48, 48)
    c = np.array([24, 24, 24])
    prev = None
    for r, tol in ((2, 1e-3), (4, 5e-3)):
        g = orc.green_pairs(L, np.array([c, c]), np.array([c + [r, 0, 0], c + [2 * r, 0, 0]]))
        d_inf = orc.green_infinite((r, 0, 0)) - orc.green_infinite((2 * r, 0, 0))
        assert abs((g[0] - g[1]) / d_inf - 1.0) < tol, r
    for r in (2, 4, 8, 16):
        d = (orc.green_infinite((r, 0, 0)) - orc.green_infinite((2 * r, 0, 0))) * 8 * math.pi * r
        assert d > 1.0
        if prev is not None:
            assert d - 1.0 < 0.4 * (prev - 1.0)
        prev = d
    assert prev - 1.0 < 2e-3


def test_e_lat_methods_agree(orc):
    from paper_1403_0711_gb300 import inputs
    L = (8, 7, 9)
    sites, q = inputs.uniform_q(L, 30, seed=5)
    e_dense = orc.e_lat(L, sites, q, "dense")
    assert abs(orc.e_lat(L, sites, q, "dst") - e_dense) < 1e-11 * max(1, abs(e_dense))
    assert abs(orc.e_lat(L, sites, q, "cg") - e_dense) < 1e-9 * max(1, abs(e_dense))


def test_two_body_energy(orc):
    # Fig. 1's setup: E_2 = 2 q1 q2 G_12 (Eq. (s1) counts ordered pairs)
    L = (10, 10, 10)
    G = orc.green_dense(L)
    sites = np.array([[5, 5, 5], [8, 5, 5]])
    idx = orc.site_index(L, sites)
    assert abs(orc.e_lat(L, sites, [1.0, -2.0], "dst") - 2 * (1.0) * (-2.0) * G[idx[0], idx[1]]) < 1e-12
    # continuum Eq. (s1) for the same pair
    assert abs(orc.coulomb_direct(sites, [1.0, -2.0]) - 2 * (-2.0) / (4 * math.pi * 3)) < 1e-15


def test_e_lat_single_and_coincident(orc):
    L = (5, 5, 5)
    # heat-kernel quadrature of G_ii agrees with the spectral solve to ~1e-13
    assert orc.e_lat(L, np.array([[2, 2, 2]]), [3.0], "dst") == pytest.approx(0.0, abs=2e-12)
    G = orc.green_dense(L)
    i = orc.site_index(L, [[1, 2, 3]])[0]
    # two unit charges on the same site: 2 G_ii
    assert orc.e_lat(L, np.array([[1, 2, 3], [1, 2, 3]]), [1.0, 1.0], "dst") == pytest.approx(
        2 * G[i, i], rel=1e-12)
