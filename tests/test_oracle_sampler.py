"""Pins of the oracle's sampler (heatbath Eq. (phi), over-relaxation, Eq. (nsum2)).

- Over-relaxation reflects phi_n about its conditional mean S/6, so it leaves
  H_L unchanged: catches a wrong neighbour set or coefficient.
- With the random term switched off, a heatbath pass is one red/black
  Gauss-Seidel sweep for A phi = 0, whose asymptotic contraction per pass is
  rho_J^2 with rho_J = (1/3) sum_mu cos(pi/(L_mu+1)) (Young's theorem for the
  2-cyclic red/black ordering).  Any error in the stencil, the 1/6, or the
  colouring changes the rate.
- On a 2x2x2 box the sampled covariance <phi_m phi_n> equals the dense A^{-1}
  (Eq. (proplat) on the lattice) within its batch-means error.
- The estimator's mean matches E_lat within 4 sigma (Eq. (nsum) with
  Eq. (nsum2)), and its per-sample variance matches the Wick value
  Var(e) = 2 tr(M G M G).
- Special cases: one charge gives e = 0 in every sample; doubling every
  charge multiplies e by exactly 4.
"""
import math

import numpy as np
import pytest


def test_overrelaxation_conserves_action(orc):
    rng = np.random.default_rng(7)
    for L in [(5, 4, 3), (8, 8, 8), (1, 6, 2), (7, 7, 1)]:
        phi = rng.standard_normal((L[2], L[1], L[0]))
        h0 = orc.action(phi)
        orc.halfsweep(phi, 0, heatbath=False)
        assert abs(orc.action(phi) - h0) < 1e-12 * h0
        orc.halfsweep(phi, 1, heatbath=False)
        assert abs(orc.action(phi) - h0) < 1e-12 * h0


def test_overrelaxation_is_reflection_about_heatbath_mean(orc):
    # OR then a zero-noise heatbath give S/6 - (S/3 - phi) ... the mean of the
    # two equals the heatbath mean S/6
    L = (6, 5, 4)
    rng = np.random.default_rng(8)
    phi = rng.standard_normal((L[2], L[1], L[0]))
    a = phi.copy()
    orc.halfsweep(a, 0, heatbath=False)
    b = phi.copy()
    orc.halfsweep(b, 0, heatbath=True, noise_scale=0.0)
    red = (np.add.outer(np.add.outer(np.arange(L[2]), np.arange(L[1])), np.arange(L[0])) % 2) == 0
    assert np.allclose(((a + phi) / 2)[red], b[red], atol=1e-14)
    assert np.array_equal(a[~red], phi[~red])


@pytest.mark.parametrize("L", [(6, 5, 7), (9, 9, 9), (4, 11, 3)])
def test_zero_noise_heatbath_is_red_black_gauss_seidel(orc, L):
    rng = np.random.default_rng(1)
    phi = rng.standard_normal((L[2], L[1], L[0]))
    rho_j = sum(math.cos(math.pi / (n + 1)) for n in L) / 3.0
    norms = []
    for p in range(160):
        orc.one_pass(phi, heatbath=True, noise_scale=0.0)
        norms.append(np.sqrt(orc.action(phi)))
    ratio = norms[-1] / norms[-2]
    assert abs(ratio - rho_j ** 2) < 1e-6, (ratio, rho_j ** 2)


def test_heatbath_covariance_matches_dense_green(orc):
    L = (2, 2, 2)
    G = orc.green_dense(L)
    ch = orc.Chain(L, seed=2024)
    ch.run(20)
    M, nb = 40000, 40
    acc = np.zeros((nb, 8, 8))
    per = M // nb
    for b in range(nb):
        for _ in range(per):
            ch.run(1)
            v = ch.phi.reshape(-1)
            acc[b] += np.outer(v, v)
    bm = acc / per
    mean = bm.mean(axis=0)
    se = bm.std(axis=0, ddof=1) / math.sqrt(nb)
    z = np.abs(mean - G) / se
    assert z.max() < 5.0, z.max()
    assert np.abs(mean - G).max() < 0.05 * G.max()


def test_estimator_mean_matches_e_lat_cube(orc):
    # the paper's Fig. 2 geometry in a small box: N = 8 charges q=1 in a cube
    from paper_1403_0711_gb300 import inputs
    L = (8, 8, 8)
    sites, q = inputs.cube(L, 2)
    exact = orc.e_lat(L, sites, q, "dense")
    ch = orc.Chain(L, seed=77)
    ch.run(50)
    out = ch.run(12000, 1, 1, sites, q)
    mean, se = orc.batch_means(out[:, 2], 32)
    assert abs(mean - exact) < 4 * se, (mean, exact, se)
    assert se < 0.05 * abs(exact)


def test_estimator_variance_matches_wick(orc):
    from paper_1403_0711_gb300 import inputs
    L = (4, 4, 4)
    sites, q = inputs.plus_minus(L, 4, seed=1)
    var_exact = orc.wick_variance(L, sites, q)
    ch = orc.Chain(L, seed=5)
    ch.run(50)
    out = ch.run(30000, 1, 1, sites, q)
    v = out[:, 2].var()
    assert abs(v / var_exact - 1.0) < 0.1, (v, var_exact)


def test_single_charge_gives_zero(orc):
    L = (5, 6, 7)
    ch = orc.Chain(L, seed=3)
    out = ch.run(20, 1, 2, np.array([[2, 3, 4]]), [1.7])
    assert np.all(out[:, 2] == 0.0)
    assert np.all(out[:, 1] > 0.0)


def test_scaling_charges(orc):
    from paper_1403_0711_gb300 import inputs
    L = (6, 6, 6)
    sites, q = inputs.uniform_q(L, 10, seed=4)
    a = orc.Chain(L, seed=9).run(15, 1, 1, sites, q)
    b = orc.Chain(L, seed=9).run(15, 1, 1, sites, 2 * q)
    assert np.array_equal(b[:, 2], 4 * a[:, 2])
    assert np.array_equal(b[:, 0], 2 * a[:, 0])


def test_chains_resume_and_differ(orc):
    L = (5, 4, 6)
    a = orc.Chain(L, seed=1, chain=0)
    a.run(10, 1, 3)
    b = orc.Chain(L, seed=1, chain=0)
    b.run(4, 1, 3)
    b.run(6, 1, 3)
    assert np.array_equal(a.phi, b.phi) and a.pass_ == b.pass_ == 40
    c = orc.Chain(L, seed=1, chain=1)
    c.run(10, 1, 3)
    assert not np.array_equal(a.phi, c.phi)
