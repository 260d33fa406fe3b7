"""Off-lattice charges (coulps_charges_create_off) against the FP64 oracle.

Per sample: the CUDA path's (Q, P, e) of trilinearly interpolated charges and
its force sums -de/dr_i equal the oracle's (oracle/offlattice.py) on the
oracle chain's own fields (same seed, chain ids and Philox counters, FP64),
to 1e-12 relative.  In distribution: the pooled mean of e and the mean forces
over many chains match the exact interpolated-Green-function values on a
small box within a few standard errors."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def cl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_0711_gb300 import _build, coulps
    _build.build()
    coulps.load()
    coulps.use_torch_allocator()
    return coulps


@pytest.fixture(scope="module")
def stream():
    import torch
    return torch.cuda.Stream()


def _oracle_steps(orc, L, seed, chain, n_therm, n_meas, n_hb, n_or, pos, q):
    from oracle import offlattice as off
    c = orc.Chain(L, seed=seed, chain=chain)
    c.run(n_therm, n_hb, n_or)
    qpe, forces = [], []
    for _ in range(n_meas):
        c.run(1, n_hb, n_or)
        qpe.append(off.sample(c.phi, L, pos, q))
        forces.append(off.force_sample(c.phi, L, pos, q))
    return np.array(qpe), np.array(forces)


def _rel(got, ref):
    Q, P = ref[:, 0], ref[:, 1]
    den = np.maximum(Q * Q + P, 1e-300)
    eq = np.abs(got[:, 0] - Q) / np.sqrt(np.maximum(P, 1e-300))
    return max(eq.max(), (np.abs(got[:, 1] - P) / den).max(), (np.abs(got[:, 2] - ref[:, 2]) / den).max())


@pytest.mark.parametrize("L,n,path", [((13, 7, 5), 9, "run"), ((9, 2, 17), 5, "measure"),
                                      ((2, 2, 2), 3, "run"), ((33, 17, 9), 40, "sets")])
def test_off_lattice_samples_and_forces_match_oracle(cl, stream, orc, L, n, path):
    from paper_1403_0711_gb300 import inputs
    pos, q = inputs.off_lattice(L, n, seed=sum(L))
    n_chains, n_therm, n_meas, n_hb, n_or, seed = 2, 2, 5, 1, 2, 11
    lat = cl.Lattice(L, n_chains=n_chains, precision=cl.F64, seed=seed, stream=stream)
    ch = cl.Charges.off_lattice(lat, pos, q, log_capacity=n_meas, forces=True)
    if path == "run":
        ch.run(n_therm, n_meas, n_hb, n_or)
    elif path == "measure":
        lat.sweep(n_therm, n_hb, n_or)
        for _ in range(n_meas):
            lat.sweep(1, n_hb, n_or)
            ch.measure()
    else:  # beside an on-lattice set, through the multi-set path
        sites, qq = inputs.uniform_q(L, 7, seed=3)
        on = cl.Charges(lat, sites, qq, log_capacity=n_meas)
        cl.run_sets(lat, [on, ch], n_therm, n_meas, n_hb, n_or)
        ref_on = orc.Chain(L, seed=seed, chain=1)
        ref_on.run(n_therm, n_hb, n_or)
        want = ref_on.run(n_meas, n_hb, n_or, sites, qq)
        assert _rel(on.samples()[:, 1], want) < TOL64
        on.close()
    s = ch.samples()
    assert s.shape == (n_meas, n_chains, 3)
    fsum = np.zeros((n, 3))
    for k in range(n_chains):
        ref, f = _oracle_steps(orc, L, seed, k, n_therm, n_meas, n_hb, n_or, pos, q)
        assert _rel(s[:, k], ref) < TOL64, k
        fsum += f.sum(axis=0)
    mean, err = ch.forces()
    want = fsum / (n_chains * n_meas)
    scale = np.abs(want).max() + 1e-300
    assert np.abs(mean - want).max() < 1e-11 * scale
    assert np.all(np.isfinite(err))
    # reset clears the samples and the force sums
    ch.reset_stats()
    ch.measure()
    m1, _ = ch.forces()
    assert ch.estimate()["n"] == n_chains
    assert np.all(np.isfinite(m1))
    ch.close()
    lat.close()


def test_off_lattice_mean_and_forces_match_exact(cl, stream, orc):
    """8 x 7 x 6 box, 4 particles: pooled mean of e against E = sum_{i!=j}
    q_i q_j G~(r_i, r_j) and mean forces against -2 q_i sum_j q_j grad G~,
    both from the dense lattice Green function, within 5 standard errors."""
    from oracle import offlattice as off
    L = (8, 7, 6)
    pos = np.array([[2.3, 3.1, 2.7], [4.6, 3.4, 2.2], [3.5, 1.2, 3.9], [5.2, 5.5, 1.4]])
    q = np.array([1.0, -1.0, 0.7, -0.4])
    G = orc.green_dense(L)
    E = off.energy_exact(G, L, pos, q)
    F = off.force_exact(G, L, pos, q)
    lat = cl.Lattice(L, n_chains=256, precision=cl.F32, seed=77, stream=stream)
    ch = cl.Charges.off_lattice(lat, pos, q, forces=True)
    ch.run(100, 2000, 1, 1)
    est = ch.estimate()
    mean, err = ch.forces()
    ch.close()
    lat.close()
    assert abs(est["mean"] - E) < 5 * est["stderr"], (est, E)
    z = np.abs(mean - F) / err
    assert z.max() < 5, (mean, F, err)
    assert np.abs(mean - F).max() < 0.15 * np.abs(F).max()


def test_off_lattice_rejects_bad_input(cl, stream):
    L = (6, 5, 4)
    lat = cl.Lattice(L, n_chains=1, precision=cl.F32, seed=1, stream=stream)
    for pos in ([[5.01, 1, 1]], [[-0.01, 1, 1]], [[1, 1, np.nan]]):
        with pytest.raises(cl.CoulpsError):
            cl.Charges.off_lattice(lat, pos, [1.0])
    flat = cl.Lattice((6, 1, 4), n_chains=1, precision=cl.F32, seed=1, stream=stream)
    with pytest.raises(cl.CoulpsError):
        cl.Charges.off_lattice(flat, [[1, 0, 1]], [1.0])
    ch = cl.Charges.off_lattice(lat, [[1.5, 2.5, 0.5]], [1.0])
    with pytest.raises(cl.CoulpsError):
        ch.forces()  # created without forces
    with pytest.raises(cl.CoulpsError):
        ch.update([[1, 1, 1]], [1.0])
    with pytest.raises(cl.CoulpsError):
        cl.GlobalCV(ch)
    ch.close()
    # an empty set samples zeros
    e = cl.Charges.off_lattice(lat, np.zeros((0, 3)), np.zeros(0), log_capacity=2, forces=True)
    e.run(1, 2, 1, 1)
    assert np.all(e.samples() == 0)
    e.close()
    flat.close()
    lat.close()


@pytest.mark.parametrize("L,n,rc,path", [((13, 7, 5), 30, 2.5, "run"), ((9, 8, 17), 60, 1.7, "measure"),
                                         ((5, 4, 3), 6, 1e9, "run")])
def test_near_correction_matches_oracle(cl, stream, orc, L, n, rc, path):
    """Near pairs found on the host (cell grid) = the oracle's brute-force
    set; direct energy and forces; per-sample (Q, P + s_N, e_far) and far
    force sums equal to the oracle's on the oracle chain's fields."""
    from oracle import offlattice as off
    from paper_1403_0711_gb300 import inputs
    pos, q = inputs.off_lattice(L, n, seed=n)
    pairs = off.near_pairs(pos, rc)
    n_chains, n_therm, n_meas, n_hb, n_or, seed = 2, 2, 4, 1, 1, 21
    lat = cl.Lattice(L, n_chains=n_chains, precision=cl.F64, seed=seed, stream=stream)
    ch = cl.Charges.off_lattice(lat, pos, q, log_capacity=n_meas, forces=True)
    info = ch.near(rc)
    assert info["n_pairs"] == len(pairs) > 0
    ed = off.near_direct_energy(pos, q, pairs)
    assert abs(info["e_direct"] - ed) < 1e-12 * max(1.0, abs(ed))
    fd = off.near_direct_forces(pos, q, pairs)
    assert np.abs(info["f_direct"] - fd).max() < 1e-12 * max(1.0, np.abs(fd).max())
    if path == "run":
        ch.run(n_therm, n_meas, n_hb, n_or)
    else:
        lat.sweep(n_therm, n_hb, n_or)
        for _ in range(n_meas):
            lat.sweep(1, n_hb, n_or)
            ch.measure()
    s = ch.samples()
    fsum = np.zeros((n, 3))
    for k in range(n_chains):
        c = orc.Chain(L, seed=seed, chain=k)
        c.run(n_therm, n_hb, n_or)
        ref = []
        for _ in range(n_meas):
            c.run(1, n_hb, n_or)
            ref.append(off.near_sample(c.phi, L, pos, q, pairs))
            fsum += off.near_force_sample(c.phi, L, pos, q, pairs)
        ref = np.array(ref)
        den = ref[:, 0] ** 2 + np.abs(ref[:, 1]) + 1e-300
        assert np.abs(s[:, k, 0] - ref[:, 0]).max() < TOL64 * np.sqrt(den).max()
        assert (np.abs(s[:, k, 1:] - ref[:, 1:]) / den[:, None]).max() < TOL64
    mean, _ = ch.forces()
    want = fsum / (n_chains * n_meas)
    # (all pairs near: the force is 0 up to rounding of O(1) terms)
    assert np.abs(mean - want).max() < 1e-11 * (np.abs(want).max() + 1e-3)
    if rc > 100:  # every pair near: e_far vanishes identically
        assert np.abs(s[:, :, 2]).max() < 1e-12 * (s[:, :, 0] ** 2).max()
    ch.close()
    lat.close()


def test_near_correction_off_again_is_bitwise_plain(cl, stream):
    from paper_1403_0711_gb300 import inputs
    L = (12, 10, 9)
    pos, q = inputs.off_lattice(L, 50, seed=4)
    out = []
    for near in (False, True):
        lat = cl.Lattice(L, n_chains=3, precision=cl.F32, seed=8, stream=stream)
        ch = cl.Charges.off_lattice(lat, pos, q, log_capacity=6, forces=True)
        if near:
            assert ch.near(2.0)["n_pairs"] > 0
            ch.run(1, 3, 1, 1)
            assert ch.near(0.0)["n_pairs"] == 0
            assert ch.estimate()["n"] == 0
            ch.close()
            lat.close()
            lat = cl.Lattice(L, n_chains=3, precision=cl.F32, seed=8, stream=stream)
            ch = cl.Charges.off_lattice(lat, pos, q, log_capacity=6, forces=True)
            ch.near(2.0)
            ch.near(0.0)
        ch.run(2, 6, 1, 2)
        out.append((ch.samples(), ch.forces()[0]))
        ch.close()
        lat.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_near_far_mean_matches_exact(cl, stream, orc):
    """8 x 7 x 6 box, 6 particles, near pairs within 2.2: pooled mean of e_far
    against the exact far lattice energy and far forces against their exact
    values, within 5 standard errors."""
    from oracle import offlattice as off
    L = (8, 7, 6)
    pos = np.array([[2.3, 3.1, 2.7], [4.6, 3.4, 2.2], [3.5, 1.2, 3.9], [5.2, 5.5, 1.4],
                    [3.1, 3.9, 3.3], [6.0, 2.5, 4.1]])
    q = np.array([1.0, -1.0, 0.7, -0.4, 0.9, -0.6])
    pairs = off.near_pairs(pos, 2.2)
    assert 0 < len(pairs) < 15
    G = orc.green_dense(L)
    E = off.far_energy_exact(G, L, pos, q, pairs)
    F = off.far_force_exact(G, L, pos, q, pairs)
    lat = cl.Lattice(L, n_chains=256, precision=cl.F32, seed=78, stream=stream)
    ch = cl.Charges.off_lattice(lat, pos, q, forces=True)
    info = ch.near(2.2)
    assert info["n_pairs"] == len(pairs)
    ch.run(100, 2000, 1, 1)
    est = ch.estimate()
    mean, err = ch.forces()
    ch.close()
    lat.close()
    assert abs(est["mean"] - E) < 5 * est["stderr"], (est, E)
    assert (np.abs(mean - F) / err).max() < 5, (mean, F, err)


def test_off_lattice_checkpoint_resume_bitwise(cl, stream, tmp_path):
    """Save and restore an off-lattice set with forces and near pairs: samples,
    estimate and mean forces after the resume equal the uninterrupted run's
    bit for bit; a set without force sums refuses a file that has them."""
    from paper_1403_0711_gb300 import inputs
    L = (20, 14, 12)
    pos, q = inputs.off_lattice(L, 25, seed=9)

    def make():
        lat = cl.Lattice(L, n_chains=3, precision=cl.F32, seed=31, stream=stream)
        ch = cl.Charges.off_lattice(lat, pos, q, log_capacity=10, forces=True)
        ch.near(2.5)
        return lat, ch

    lat, ch = make()
    ch.run(2, 10, 1, 3)
    full = (ch.samples(), ch.estimate(), ch.forces())
    ch.close()
    lat.close()

    lat, ch = make()
    ch.run(2, 4, 1, 3)
    path = tmp_path / "off.ckpt"
    lat.checkpoint_save(path, ch)
    ch.close()
    lat.close()

    lat, ch = make()
    lat.checkpoint_load(path, ch)
    ch.run(0, 6, 1, 3)
    assert np.array_equal(ch.samples(), full[0])
    assert ch.estimate() == full[1]
    m, e = ch.forces()
    assert np.array_equal(m, full[2][0]) and np.array_equal(e, full[2][1])
    plain = cl.Charges.off_lattice(lat, pos, q, log_capacity=10)
    with pytest.raises(cl.CoulpsError) as ei:
        lat.checkpoint_load(path, plain)
    assert ei.value.status == cl.ECORRUPT
    for o in (plain, ch, lat):
        o.close()
