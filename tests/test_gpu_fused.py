"""Fused passes (one kernel per pass, field copied back and forth between two
buffers) against the half-sweep path: the fields must be bitwise identical
(same arithmetic per site, same Philox counters), over heatbath and
over-relaxation passes, odd and even pass counts, FP32 and FP64, ragged
boxes, and any fused tile shape.  Samples agree to rounding (the fused path
gathers with the separate gather kernel, in another summation order)."""
import numpy as np
import pytest

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


def _run(cl, stream, L, prec, n_chains, seed, sites, q, n_therm, n_meas, n_hb, n_or, fused,
         pass_tile=None, pair_tile=None):
    from paper_1403_0711_gb300 import inputs
    lat = cl.Lattice(L, n_chains=n_chains, precision=prec, seed=seed, stream=stream)
    lat.set_fused(fused)
    if pass_tile:
        lat.set_pass_tile(*pass_tile)
    if pair_tile:
        lat.set_pair_tile(*pair_tile)
    # seeded Gaussian start (an over-relaxation-only run from phi = 0 stays 0)
    for k, f in enumerate(inputs.gaussian_fields(L, n_chains, seed=seed)):
        lat.set_field(k, f)
    ch = cl.Charges(lat, sites, q, log_capacity=max(1, n_meas))
    ch.run(n_therm, n_meas, n_hb, n_or)
    s = ch.samples()
    f = [lat.field(k) for k in range(n_chains)]
    info = lat.info()
    ch.close()
    lat.close()
    return s, f, info


def _rel(a, b):
    den = np.abs(b[..., 0]) ** 2 + np.abs(b[..., 1]) + 1e-300
    return float(np.max(np.abs(a - b) / den[..., None]))


@pytest.mark.parametrize("L,prec,n_hb,n_or,tile,mode", [
    ((37, 29, 23), "F32", 1, 3, None, 1),   # three OR passes fused, the HB pass out of place
    ((21, 18, 12), "F64", 2, 3, None, 1),   # two HB passes (the second in place on the copy)
    ((12, 7, 9), "F32", 1, 1, (2, 3), 1),   # one fused OR pass after one HB pass
    ((37, 29, 23), "F32", 1, 3, (3, 5), 2),  # all four passes fused
    ((16, 16, 16), "F64", 2, 2, None, 1),
    ((16, 16, 16), "F64", 2, 2, None, 2),
    ((10, 9, 8), "F32", 1, 2, None, 2),      # odd pass count: last pass as half-sweeps
    ((130, 5, 70), "F32", 0, 4, (1, 64), 1),
    ((64, 64, 64), "F32", 1, 3, (30, 16), 2),
    ((9, 1, 1), "F64", 1, 1, None, 2),
    ((25, 40, 3), "F32", 3, 1, (6, 1), 2),
    ((25, 40, 3), "F32", 1, 5, (6, 1), 1),
    ((512, 12, 6), "F32", 1, 3, None, 1),   # 64-quad rows: the default 5-row, 512-thread tile
    ((384, 9, 5), "F64", 1, 3, None, 1),    # 48-quad rows, FP64
])
def test_fused_passes_equal_half_sweeps(cl, stream, L, prec, n_hb, n_or, tile, mode):
    from paper_1403_0711_gb300 import inputs
    p = getattr(cl, prec)
    n = min(12, L[0] * L[1] * L[2] // 2) // 2 * 2
    sites, q = inputs.plus_minus(L, n, seed=3)
    ref = _run(cl, stream, L, p, 3, 17, sites, q, 2, 4, n_hb, n_or, 0)
    got = _run(cl, stream, L, p, 3, 17, sites, q, 2, 4, n_hb, n_or, mode, tile)
    assert got[2]["fused"] == mode and ref[2]["fused"] == 0
    assert got[2]["pass"] == ref[2]["pass"]
    for a, b in zip(got[1], ref[1]):
        assert np.array_equal(a, b)
    assert _rel(got[0], ref[0]) < 1e-13


# Pass pairs: mode 3 (heatbath passes as half-sweeps, over-relaxation passes
# as pairs + one single for an odd count, the heatbath pass out of place when
# the count of these kernels is odd) and mode 4 (all passes as pairs + single
# fused passes: n = 4: two pairs; 5: one pair + three singles; 6: two pairs +
# two singles; 3: one pair + one single; 2: two singles, pairs of every kind),
# pair tiles from one row to the default, slabs of one plane to the whole box,
# rows narrower than a tile and boxes thinner than the pipeline (Lz < 4).
@pytest.mark.parametrize("mode", [3, 4])
@pytest.mark.parametrize("L,prec,n_hb,n_or,pair_tile", [
    ((37, 29, 23), "F32", 1, 3, None),
    ((37, 29, 23), "F32", 1, 3, (3, 5)),
    ((21, 18, 12), "F64", 2, 3, None),
    ((16, 16, 16), "F64", 2, 2, None),
    ((16, 16, 16), "F32", 2, 2, (4, 3)),
    ((10, 9, 8), "F32", 1, 2, None),
    ((12, 7, 9), "F32", 1, 1, None),
    ((130, 5, 70), "F32", 0, 4, (1, 64)),
    ((64, 64, 64), "F32", 1, 3, (26, 16)),
    ((128, 64, 40), "F32", 1, 3, None),
    ((9, 1, 1), "F64", 1, 1, None),
    ((25, 40, 3), "F32", 3, 1, (6, 1)),
    ((25, 40, 3), "F32", 1, 5, (6, 1)),
    ((8, 8, 200), "F32", 1, 3, (8, 7)),
    ((100, 3, 50), "F64", 1, 3, (2, 9)),
    ((2, 3, 4), "F32", 1, 3, None),
    ((1, 1, 1), "F32", 1, 3, None),
])
def test_pass_pairs_equal_half_sweeps(cl, stream, L, prec, n_hb, n_or, pair_tile, mode):
    from paper_1403_0711_gb300 import inputs
    p = getattr(cl, prec)
    n = max(2, min(12, L[0] * L[1] * L[2] // 2) // 2 * 2)
    if L == (1, 1, 1):
        n = 1
    sites, q = (inputs.plus_minus(L, n, seed=3) if n > 1 else
                (np.zeros((1, 3), np.int32), np.ones(1)))
    ref = _run(cl, stream, L, p, 3, 17, sites, q, 2, 4, n_hb, n_or, 0)
    got = _run(cl, stream, L, p, 3, 17, sites, q, 2, 4, n_hb, n_or, mode, pair_tile=pair_tile)
    assert got[2]["fused"] == mode
    assert got[2]["pass"] == ref[2]["pass"]
    for a, b in zip(got[1], ref[1]):
        assert np.array_equal(a, b)
    assert _rel(got[0], ref[0]) < 1e-13


def test_pair_tile_limits(cl, stream):
    lat = cl.Lattice((128, 128, 128), n_chains=1, precision=cl.F32, seed=1, stream=stream)
    lat.set_fused(3)
    ty, dz = lat.pair_tile()
    assert (ty + 6) * 16 <= 512 and ty >= 4 and dz >= 1
    with pytest.raises(cl.CoulpsError):
        lat.set_pair_tile(27, 8)  # 33 rows x 16 quads > 512 threads
    lat.set_pair_tile(26, 128)
    assert lat.pair_tile() == (26, 128)
    lat.close()
    # rows of 512 sites: no pair tile, the pair modes run single fused passes
    wide = cl.Lattice((512, 4, 4), n_chains=1, precision=cl.F32, seed=1, stream=stream)
    wide.set_fused(4)
    assert wide.pair_tile() == (0, 0)
    wide.close()


def test_fused_is_default_and_costs_a_second_copy(cl, stream):
    L = (32, 32, 32)
    lat = cl.Lattice(L, n_chains=2, precision=cl.F32, seed=1, stream=stream)
    info = lat.info()
    assert info["fused"] == 3 and info["pass_ty"] >= 1 and info["pass_dz"] >= 1
    assert lat.pair_tile()[0] >= 4
    b_on = info["bytes"]
    lat.set_fused(False)
    b_off = lat.info()["bytes"]
    field = 2 * 2 * 32 * 32 * 16 * 4  # chains x colours x Lz x Ly x W x 4 B
    assert b_on - b_off == field
    with pytest.raises(cl.CoulpsError):
        lat.set_pass_tile(0, 4)
    lat.close()


def test_default_tile_shapes(cl, stream):
    """Default shapes: fused-pass rows of more than 42 quads take up to 512
    threads (a 512-site row gets 5 rows, not 1); the z slabs of a lattice too
    small to fill the GPU are halved (not below 4 planes for a half-sweep or a
    fused pass, 8 for a pair) until one launch has 2 CTAs per SM (1 for a pair),
    and a lattice that fills it keeps 16 / 32 / 64 planes."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    wide = cl.Lattice((512, 12, 6), n_chains=1, precision=cl.F32, seed=1, stream=stream)
    assert wide.info()["pass_ty"] == 5
    wide.close()
    small = cl.Lattice((64, 64, 64), n_chains=1, precision=cl.F32, seed=1, stream=stream)
    info = small.info()
    ty, dz = small.pair_tile()
    # half-sweep 32 rows x 16 planes -> 2 x 4 CTAs per chain, halved to 4 planes
    assert (info["ty"], info["dz"]) == (32, 4)
    # fused pass 29 rows x 32 planes -> 3 x 2 CTAs, halved to 4 planes
    assert (info["pass_ty"], info["pass_dz"]) == (29, 4)
    # pair 58 rows x 32 planes -> 2 x 2 CTAs, halved to 8 planes
    assert (ty, dz) == (58, 8)
    small.close()
    chains = 2 * sms  # 2 row tiles x 4 slabs x chains >= 2 x SMs: slabs kept
    full = cl.Lattice((64, 64, 64), n_chains=chains, precision=cl.F32, seed=1, stream=stream)
    info = full.info()
    assert info["dz"] == 16 and info["pass_dz"] == 32
    full.close()
