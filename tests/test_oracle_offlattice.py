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


def test_near_pairs_against_cell_free_enumeration():
    from oracle import offlattice as off
    pos = _pos((9, 8, 7), 60, 7)
    rc = 2.2
    pairs = off.near_pairs(pos, rc)
    d = np.linalg.norm(pos[:, None, :] - pos[None, :, :], axis=2)
    want = {(i, j) for i in range(60) for j in range(i + 1, 60) if d[i, j] < rc}
    assert {tuple(p) for p in pairs} == want and len(pairs) == len(want) > 0


def test_near_correction_limits(orc):
    """No pairs: the plain estimator.  All pairs near: e_far == 0 for every
    field (Q^2 = P + s_N identically) and the direct part is Eq. (s1)."""
    from oracle import offlattice as off
    L = (7, 6, 5)
    pos = _pos(L, 6, 8)
    q = np.array([1.0, -0.5, 0.8, -1.2, 0.3, 1.0])
    rng = np.random.default_rng(9)
    phi = rng.standard_normal((L[2], L[1], L[0]))
    none = off.near_pairs(pos, 0.0)
    assert len(none) == 0
    assert np.allclose(off.near_sample(phi, L, pos, q, none), off.sample(phi, L, pos, q), rtol=0, atol=0)
    assert np.array_equal(off.near_force_sample(phi, L, pos, q, none), off.force_sample(phi, L, pos, q))
    allp = off.near_pairs(pos, 1e9)
    assert len(allp) == 15
    Q, Pn, e = off.near_sample(phi, L, pos, q, allp)
    assert abs(e) < 1e-12 * Q * Q + 1e-14
    assert np.abs(off.near_force_sample(phi, L, pos, q, allp)).max() < 1e-12
    assert abs(off.near_direct_energy(pos, q, allp) - orc.coulomb_direct(pos, q)) < 1e-13
    G = orc.green_dense(L)
    assert abs(off.far_energy_exact(G, L, pos, q, allp)) < 1e-13


def test_near_forces_are_minus_gradients():
    """Per-sample far force = -d e_far/dr_i at a fixed field and direct force
    = -dE_direct/dr_i, both against central differences."""
    from oracle import offlattice as off
    L = (6, 7, 5)
    pos = _pos(L, 5, 10)
    pos = np.floor(pos) + np.clip(pos - np.floor(pos), 0.1, 0.9)
    q = np.array([1.0, -1.0, 0.6, 0.9, -0.7])
    pairs = off.near_pairs(pos, 3.0)
    assert 0 < len(pairs) < 10
    rng = np.random.default_rng(11)
    phi = rng.standard_normal((L[2], L[1], L[0]))
    f = off.near_force_sample(phi, L, pos, q, pairs)
    fd_ = off.near_direct_forces(pos, q, pairs)
    h = 1e-6
    for i in range(len(q)):
        for mu in range(3):
            a, b = pos.copy(), pos.copy()
            a[i, mu] += h
            b[i, mu] -= h
            fd = -(off.near_sample(phi, L, a, q, pairs)[2] - off.near_sample(phi, L, b, q, pairs)[2]) / (2 * h)
            assert abs(f[i, mu] - fd) < 1e-6 * max(1.0, abs(fd)), (i, mu)
            fd = -(off.near_direct_energy(a, q, pairs) - off.near_direct_energy(b, q, pairs)) / (2 * h)
            assert abs(fd_[i, mu] - fd) < 1e-7 * max(1.0, abs(fd)), (i, mu)


def test_far_estimators_average_to_exact_far_values(orc):
    from oracle import offlattice as off
    L = (5, 4, 4)
    pos = _pos(L, 5, 12)
    q = np.array([1.0, -1.0, 1.0, -0.5, 0.5])
    pairs = off.near_pairs(pos, 1.8)
    assert 0 < len(pairs) < 10
    G = orc.green_dense(L)
    C = np.linalg.cholesky(orc.laplacian_dense(L))
    rng = np.random.default_rng(13)
    n = 20000
    z = rng.standard_normal((n, C.shape[0]))
    phis = np.linalg.solve(C.T, z.T).T.reshape(n, L[2], L[1], L[0])
    e = np.array([off.near_sample(p, L, pos, q, pairs)[2] for p in phis])
    f = np.array([off.near_force_sample(p, L, pos, q, pairs) for p in phis])
    E = off.far_energy_exact(G, L, pos, q, pairs)
    F = off.far_force_exact(G, L, pos, q, pairs)
    assert abs(e.mean() - E) < 4 * e.std(ddof=1) / math.sqrt(n), (e.mean(), E)
    se = f.std(axis=0, ddof=1) / math.sqrt(n)
    assert (np.abs(f.mean(axis=0) - F) < 4 * se + 1e-12).all()
    # the far force is the gradient of the far energy
    h = 1e-6
    for i, mu in ((0, 0), (2, 1), (4, 2)):
        a, b = pos.copy(), pos.copy()
        a[i, mu] += h
        b[i, mu] -= h
        fd = -(off.far_energy_exact(G, L, a, q, pairs) - off.far_energy_exact(G, L, b, q, pairs)) / (2 * h)
        assert abs(F[i, mu] - fd) < 1e-6 * max(1.0, abs(fd))


def test_far_energy_by_solve_equals_dense(orc):
    """The large-box route (DST solve + heat-kernel quadrature) against the
    dense-G definition on small boxes, with and without near pairs."""
    from oracle import offlattice as off
    for L, n, rc, seed in (((7, 6, 5), 6, 2.0, 14), ((9, 4, 6), 9, 0.0, 15)):
        pos = _pos(L, n, seed)
        q = np.random.default_rng(seed).uniform(-1, 1, n)
        pairs = off.near_pairs(pos, rc)
        G = orc.green_dense(L)
        want = off.far_energy_exact(G, L, pos, q, pairs)
        got = off.far_energy_solve(L, pos, q, pairs)
        assert abs(got - want) < 1e-10 * max(1.0, abs(want)), (got, want)
