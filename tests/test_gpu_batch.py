"""Many-system batched sweeps (one launch per half-sweep over all systems)
against the FP64 oracle, through the C ABI.

System s of a batch is a one-chain lattice whose Philox chain id is s, so the
oracle's Chain(L_s, seed, chain=s) runs the same Markov chain.
"""
import numpy as np
import pytest

from test_gpu_parity import TOL32, TOL64, field_err, orc_run, sample_err

pytestmark = pytest.mark.gpu


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


DIMS = [(13, 7, 5), (16, 16, 16), (9, 1, 17), (24, 5, 3), (33, 17, 9), (1, 1, 1), (40, 23, 19)]


def _charges(dims, seed):
    from paper_1403_0711_gb300 import inputs
    out = []
    for i, L in enumerate(dims):
        n = min(7, L[0] * L[1] * L[2])
        out.append(inputs.uniform_q(L, n, seed=seed + i))
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_matches_oracle(cl, stream, orc, prec):
    systems = _charges(DIMS, 5)
    b = cl.Batch(DIMS, precision=prec, seed=17, stream=stream)
    b.set_charges(systems, log_capacity=6)
    b.run(2, 6, 1, 2)
    s = b.samples()
    tol = TOL32 if prec == 0 else TOL64
    for k, L in enumerate(DIMS):
        ref, phi = orc_run(orc, L, 17, k, systems[k][0], systems[k][1], 2, 6, 1, 2)
        assert sample_err(s[:, k], ref) < tol, (k, L)
        assert field_err(b.field(k), phi) < tol, (k, L)
    est = b.estimate()
    assert np.all(est["n"] == 6)
    b.close()


def test_batch_tiles_do_not_change_fields(cl, stream):
    systems = _charges(DIMS, 9)
    a = cl.Batch(DIMS, precision=0, seed=3, stream=stream)
    a.set_charges(systems, log_capacity=4)
    a.run(1, 4, 1, 1)
    b = cl.Batch(DIMS, precision=0, seed=3, stream=stream)
    b.set_tiles([(max(1, min(3, L[1])), 2) for L in DIMS])
    b.set_charges(systems, log_capacity=4)
    b.run(1, 4, 1, 1)
    sa, sb = a.samples(), b.samples()
    for k in range(len(DIMS)):
        assert np.array_equal(a.field(k), b.field(k)), k
        assert sample_err(sb[:, k], sa[:, k]) < 1e-13, k
    a.close()
    b.close()


@pytest.mark.parametrize("prec,n_hb,n_or", [(0, 1, 3), (0, 1, 2), (1, 2, 2), (0, 0, 3), (0, 0, 2),
                                           (1, 1, 1), (0, 2, 3), (0, 1, 0)])
def test_batch_fused_passes_equal_half_sweeps(cl, stream, prec, n_hb, n_or):
    """Fused over-relaxation passes and pass pairs (the default) against
    half-sweeps only: the fields bitwise, the samples to FP64 summation order
    (the last kernel gathers over other tiles), for odd and even
    over-relaxation counts with and without heatbath passes, uneven boxes
    down to one site."""
    systems = _charges(DIMS, 21)
    out = []
    for fused in (0, 1, 2, 3):
        b = cl.Batch(DIMS, precision=prec, seed=29, stream=stream)
        if fused != 2:
            b.set_fused(fused)
        assert b.fused() == fused
        b.set_charges(systems, log_capacity=5)
        b.sweep(3, 1, 1)  # a non-zero field for over-relaxation-only mixes
        b.run(1, 5, n_hb, n_or)
        out.append((b.samples(), [b.field(k) for k in range(len(DIMS))], b.info()["pass"]))
        b.close()
    sa, fa, pa = out[0]
    for sb, fb, pb in out[1:]:
        assert pa == pb
        for k in range(len(DIMS)):
            assert np.array_equal(fa[k], fb[k]), k
            if n_hb + n_or > 0:
                assert sample_err(sb[:, k], sa[:, k]) < 1e-13, k


PAIR_DIMS = [(8, 6, 130), (64, 40, 20), (13, 7, 5), (1, 1, 1), (40, 23, 19), (96, 9, 11)]


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("n_hb,n_or", [(1, 3), (1, 4), (0, 5), (0, 4), (2, 2), (3, 2), (1, 0),
                                       (2, 0)])
def test_batch_pair_tiles_equal_half_sweeps(cl, stream, mode, n_hb, n_or):
    """Pass pairs (over-relaxation only, or with heatbath passes: mode 3) on
    small tiles (several y tiles and z slabs per system, a slab split at
    Lz >= 128 by default) against half-sweeps only: fields bitwise, samples
    to summation order; many pair launches in a row (the tile counter resets
    itself)."""
    systems = _charges(PAIR_DIMS, 41)
    a = cl.Batch(PAIR_DIMS, precision=0, seed=5, stream=stream)
    a.set_fused(0)
    b = cl.Batch(PAIR_DIMS, precision=0, seed=5, stream=stream)
    b.set_fused(mode)
    assert b.pair_tiles()[0] == (6, 64)  # whole y (2 quads a row), z split at 64
    c = cl.Batch(PAIR_DIMS, precision=0, seed=5, stream=stream)
    c.set_fused(mode)
    c.set_pair_tiles([(max(1, min(2, L[1])), 3) for L in PAIR_DIMS])
    assert c.pair_tiles()[1] == (2, 3)
    for x in (a, b, c):
        x.set_charges(systems, log_capacity=6)
        x.sweep(2, 1, 1)
        x.run(2, 6, n_hb, n_or)
    for x in (b, c):
        assert x.fused() == mode
        for k in range(len(PAIR_DIMS)):
            assert np.array_equal(a.field(k), x.field(k)), k
            assert sample_err(x.samples()[:, k], a.samples()[:, k]) < 1e-13, k
    with pytest.raises(cl.CoulpsError):
        c.set_pair_tiles([(300, 0)] * len(PAIR_DIMS))
    for x in (a, b, c):
        x.close()


def test_batch_without_pair_tile_uses_fused_passes(cl, stream):
    """A system whose rows are too wide for a pair tile (FP64, Lx = 512: 64
    quads a row, 7 rows > 256 threads) keeps fused passes; pairs are refused."""
    b = cl.Batch([(512, 3, 4), (8, 8, 8)], precision=1, seed=1, stream=stream)
    assert b.fused() == 1 and b.pair_tiles()[0][0] == 0
    for mode in (2, 3):
        with pytest.raises(cl.CoulpsError):
            b.set_fused(mode)
    b.close()


def test_batch_pass_tiles_do_not_change_fields(cl, stream):
    systems = _charges(DIMS, 23)
    a = cl.Batch(DIMS, precision=0, seed=31, stream=stream)
    a.set_charges(systems, log_capacity=4)
    a.run(1, 4, 1, 3)
    b = cl.Batch(DIMS, precision=0, seed=31, stream=stream)
    b.set_pass_tiles([(max(1, min(3, L[1])), 2) for L in DIMS])
    assert b.pass_tiles()[0] == (3, 2)
    b.set_charges(systems, log_capacity=4)
    b.run(1, 4, 1, 3)
    sa, sb = a.samples(), b.samples()
    for k in range(len(DIMS)):
        assert np.array_equal(a.field(k), b.field(k)), k
        assert sample_err(sb[:, k], sa[:, k]) < 1e-13, k
    with pytest.raises(cl.CoulpsError):
        b.set_pass_tiles([(300, 0)] * len(DIMS))
    a.close()
    b.close()


def test_batch_system0_equals_single_lattice(cl, stream):
    from paper_1403_0711_gb300 import inputs
    L = (20, 18, 16)
    sites, q = inputs.uniform_q(L, 30, seed=2)
    b = cl.Batch([L, (8, 8, 8)], precision=0, seed=44, stream=stream)
    b.set_charges([(sites, q), inputs.uniform_q((8, 8, 8), 5, seed=1)], log_capacity=5)
    b.run(2, 5, 1, 3)
    lat = cl.Lattice(L, n_chains=1, precision=0, seed=44, stream=stream)
    ch = cl.Charges(lat, sites, q, log_capacity=5)
    ch.run(2, 5, 1, 3)
    assert np.array_equal(b.field(0), lat.field(0))
    assert sample_err(b.samples()[:, 0], ch.samples()[:, 0]) < 1e-13
    ch.close()
    lat.close()
    b.close()


def test_many_uneven_systems_sampled(cl, stream, orc):
    """256 systems, edges from {32, 48, 64, 80, 96}, N log-uniform in [64, 2048]
    (the many-system workload); systems 0, 101 and 255 against the oracle."""
    from paper_1403_0711_gb300 import inputs
    sysl = inputs.batch_systems(256, seed=7)
    b = cl.Batch([L for L, _, _ in sysl], precision=0, seed=5, stream=stream)
    b.set_charges([(s, q) for _, s, q in sysl], log_capacity=3)
    b.run(1, 3, 1, 3)
    s = b.samples()
    for k in (0, 101, 255):
        L, sites, q = sysl[k]
        ref, phi = orc_run(orc, L, 5, k, sites, q, 1, 3, 1, 3)
        assert sample_err(s[:, k], ref) < TOL32, k
        assert field_err(b.field(k), phi) < TOL32, k
    info = b.info()
    assert info["n_systems"] == 256 and info["tiles"] >= 256
    b.close()


def test_batch_means_match_e_lat(cl, stream, orc):
    """Eight small boxes with the paper's q=1 cube: each system's mean within
    4.5 batch-means sigma of its own E_lat."""
    from paper_1403_0711_gb300 import inputs
    dims = [(8, 8, 8), (10, 10, 10), (12, 12, 12), (9, 11, 10), (8, 8, 8), (12, 10, 8),
            (10, 10, 10), (11, 9, 12)]
    systems = [inputs.cube(L, 2) for L in dims]
    b = cl.Batch(dims, precision=0, seed=99, stream=stream)
    b.set_charges(systems)
    b.run(200, 20000, 1, 1)
    est = b.estimate()
    for k, L in enumerate(dims):
        exact = orc.e_lat(L, systems[k][0], systems[k][1], "dense")
        assert abs(est["mean"][k] - exact) < 4.5 * est["stderr"][k], (k, est["mean"][k], exact)
        assert est["stderr"][k] < 0.05 * abs(exact)
    b.close()
