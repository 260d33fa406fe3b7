"""Several streams per compound sweep (coulps_set_streams): chain k runs on
stream k % n, the extra streams forked from and joined into the lattice's
stream.  Fields,
samples and estimates must be bitwise those of the one-stream path, with
graph replay and direct launches, every fused mode, multi-set measurement
and the global control variate."""
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


@pytest.mark.parametrize("L,prec,chains,fused,n_hb,n_or,profiling", [
    ((24, 13, 11), "F32", 5, 1, 1, 3, False),
    ((24, 13, 11), "F32", 5, 1, 1, 3, True),
    ((17, 9, 12), "F64", 4, 0, 1, 2, False),
    ((20, 16, 8), "F32", 3, 2, 1, 3, False),
    ((16, 16, 16), "F32", 1, 1, 1, 3, False),
    ((33, 10, 6), "F32", 6, 1, 2, 2, False),
    ((24, 13, 11), "F32", 5, 3, 1, 3, False),
    ((24, 13, 11), "F32", 5, 3, 1, 3, True),
    ((17, 9, 12), "F64", 4, 4, 1, 3, False),
    ((33, 10, 6), "F32", 6, 3, 2, 2, False),
    ((33, 10, 6), "F32", 6, 4, 2, 3, False),
])
def test_two_streams_bitwise(cl, stream, L, prec, chains, fused, n_hb, n_or, profiling):
    from paper_1403_0711_gb300 import inputs
    sites, q = inputs.uniform_q(L, 30, seed=5)
    out = []
    for n in (1, 2, 3, 4):
        lat = cl.Lattice(L, n_chains=chains, precision=getattr(cl, prec), seed=41, stream=stream)
        lat.set_fused(fused)
        lat.set_streams(n)
        lat.set_profiling(profiling)
        ch = cl.Charges(lat, sites, q, log_capacity=8)
        ch.run(2, 5, n_hb, n_or)
        ch.run(0, 3, n_hb, n_or)
        lat.sweep(2, n_hb, n_or)
        out.append((ch.samples(), [lat.field(k) for k in range(chains)], ch.estimate(),
                    lat.info()["pass"]))
        ch.close()
        lat.close()
    a = out[0]
    for b in out[1:]:
        assert np.array_equal(a[0], b[0])
        for fa, fb in zip(a[1], b[1]):
            assert np.array_equal(fa, fb)
        assert a[2] == b[2] and a[3] == b[3]


def test_two_streams_sets_and_global_cv_bitwise(cl, stream):
    from paper_1403_0711_gb300 import inputs
    L = (20, 18, 16)
    sets = [inputs.plus_minus(L, 20, seed=1), inputs.uniform_q(L, 33, seed=2)]
    out = []
    for n in (1, 2, 4):
        lat = cl.Lattice(L, n_chains=4, precision=cl.F32, seed=43, stream=stream)
        lat.set_streams(n)
        cs = [cl.Charges(lat, s, q, log_capacity=6) for s, q in sets]
        cl.run_sets(lat, cs, 2, 6, 1, 3)
        g = cl.GlobalCV(cs[0], R=0)
        g.run(8, 1, 3, 1.0)
        out.append(([c.samples() for c in cs], cs[0].cv_chain_stats(), lat.field(3)))
        g.close()
        for c in cs:
            c.close()
        lat.close()
    a = out[0]
    for b in out[1:]:
        for x, y in zip(a[0], b[0]):
            assert np.array_equal(x, y)
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("L,prec,chains,fused,n_hb,n_or,n_meas,profiling", [
    ((24, 13, 11), "F32", 5, 3, 1, 3, 6, False),   # pair + single, no flip
    ((24, 13, 11), "F32", 5, 3, 1, 3, 6, True),    # direct launches
    ((24, 13, 11), "F32", 4, 3, 1, 2, 2, False),   # one pair after an out-of-place heatbath pass
    ((17, 9, 12), "F64", 3, 3, 2, 3, 5, False),
    ((20, 16, 8), "F32", 2, 1, 1, 3, 4, False),    # fused mode 1
    ((20, 16, 8), "F32", 6, 1, 1, 1, 3, False),
    ((33, 10, 6), "F32", 7, 3, 1, 1, 4, False),    # one single after an out-of-place heatbath pass
])
def test_shifted_schedule_bitwise(cl, stream, L, prec, chains, fused, n_hb, n_or, n_meas,
                                  profiling):
    """The shifted schedule (odd chains half a compound sweep behind, two
    streams) gives bitwise the samples, estimates, fields and pass counter of
    the aligned one-stream schedule, over repeated runs, with thermalisation
    and plain sweeps between them."""
    from paper_1403_0711_gb300 import inputs
    sites, q = inputs.uniform_q(L, 30, seed=8)
    out = []
    for schedule, n in ((cl.SCHEDULE_ALIGNED, 1), (cl.SCHEDULE_SHIFTED, 2)):
        lat = cl.Lattice(L, n_chains=chains, precision=getattr(cl, prec), seed=43, stream=stream)
        lat.set_fused(fused)
        lat.set_streams(n)
        lat.set_schedule(schedule)
        lat.set_profiling(profiling)
        ch = cl.Charges(lat, sites, q, log_capacity=3 * n_meas)
        ch.run(2, n_meas, n_hb, n_or)
        lat.sweep(1, n_hb, n_or)
        ch.run(0, n_meas, n_hb, n_or)
        ch.run(0, n_meas, n_hb, n_or)
        out.append((ch.samples(), [lat.field(k) for k in range(chains)], ch.estimate(),
                    lat.info()["pass"]))
        ch.close()
        lat.close()
    a, b = out
    assert np.array_equal(a[0], b[0])
    for fa, fb in zip(a[1], b[1]):
        assert np.array_equal(fa, fb)
    assert a[2] == b[2] and a[3] == b[3]
