"""Pins of the off-lattice oracle (oracle/offlattice.py): trilinear weights,
the on-lattice special case, exact forces against finite differences of the
exact energy, and the Monte Carlo estimators against the exact values."""
import math

import numpy as np


def _pos(L, n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, (n, 3)) * (np.asarray(L) - 1)


def test_weights_partition_unity_and_interpolate_linear_fields():
    from oracle import offlattice as off
    L = (6, 5, 7)
    pos = _pos(L, 20, 1)
    s, w, g = off.corners(L, pos)
    assert np.allclose(w.sum(axis=1), 1.0, atol=1e-14)
    assert np.allclose(g.sum(axis=1), 0.0, atol=1e-14)
    assert s.min() >= 0 and (s < np.asarray(L)).all()
    z, y, x = np.meshgrid(np.arange(L[2]), np.arange(L[1]), np.arange(L[0]), indexing="ij")
    a = np.array([0.3, -1.1, 0.7])
    phi = a[0] * x + a[1] * y + a[2] * z + 2.0
    val, grad = off.interpolate(phi, L, pos)
    assert np.allclose(val, pos @ a + 2.0, atol=1e-12)
    assert np.allclose(grad, a[None, :], atol=1e-12)


def test_on_lattice_positions_reduce_to_the_lattice_estimator(orc):
    from oracle import offlattice as off
    from paper_1403_0711_gb300 import inputs
    L = (6, 5, 4)
    sites, q = inputs.plus_minus(L, 8, seed=2)
    G = orc.green_dense(L)
    assert abs(off.energy_exact(G, L, sites.astype(float), q) - orc.e_lat(L, sites, q, "dense")) < 1e-13
    rng = np.random.default_rng(3)
    phi = rng.standard_normal((L[2], L[1], L[0]))
    assert np.allclose(off.sample(phi, L, sites.astype(float), q), orc.measure(phi, sites, q),
                       rtol=1e-13, atol=1e-13)


def test_exact_force_is_minus_the_gradient_of_the_exact_energy(orc):
    from oracle import offlattice as off
    L = (5, 6, 4)
    pos = _pos(L, 5, 4)
    pos = np.floor(pos) + np.clip(pos - np.floor(pos), 0.1, 0.9)  # away from cell faces
    q = np.array([1.0, -1.0, 0.5, 0.8, -1.3])
    G = orc.green_dense(L)
    F = off.force_exact(G, L, pos, q)
    h = 1e-6
    for i in range(len(q)):
        for mu in range(3):
            a, b = pos.copy(), pos.copy()
            a[i, mu] += h
            b[i, mu] -= h
            fd = -(off.energy_exact(G, L, a, q) - off.energy_exact(G, L, b, q)) / (2 * h)
            assert abs(F[i, mu] - fd) < 1e-7 * max(1.0, abs(fd)), (i, mu, F[i, mu], fd)


def test_estimators_average_to_the_exact_energy_and_forces(orc):
    from oracle import offlattice as off
    L = (4, 4, 3)
    pos = _pos(L, 4, 5)
    q = np.array([1.0, -1.0, 1.0, -1.0])
    G = orc.green_dense(L)
    A = orc.laplacian_dense(L)
    C = np.linalg.cholesky(A)
    rng = np.random.default_rng(6)
    n = 20000
    z = rng.standard_normal((n, A.shape[0]))
    phis = np.linalg.solve(C.T, z.T).T.reshape(n, L[2], L[1], L[0])
    e = np.array([off.sample(p, L, pos, q)[2] for p in phis])
    f = np.array([off.force_sample(p, L, pos, q) for p in phis])  # (n, 4, 3)
    E = off.energy_exact(G, L, pos, q)
    F = off.force_exact(G, L, pos, q)
    assert abs(e.mean() - E) < 4 * e.std(ddof=1) / math.sqrt(n), (e.mean(), E)
    se = f.std(axis=0, ddof=1) / math.sqrt(n)
    assert (np.abs(f.mean(axis=0) - F) < 4 * se + 1e-12).all(), (f.mean(axis=0), F, se)
