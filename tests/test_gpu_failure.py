"""Failure detection without a GPU fault: a bounded device wait that runs out
(coulps_selftest_wait: a flag nothing sets, given up after a few ms) records
COULPS_ETIMEOUT; the host sees it at the next synchronisation, the context
stays usable, and after coulps_clear_error the sampler continues with the
same chain as an uninterrupted run (the wait touches no field)."""
import time

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


def test_bounded_wait_times_out_and_recovers(cl):
    import torch
    from paper_1403_0711_gb300 import inputs
    stream = torch.cuda.Stream()
    L = (20, 16, 12)
    sites, q = inputs.plus_minus(L, 16, seed=2)
    out = []
    for inject in (False, True):
        lat = cl.Lattice(L, n_chains=3, precision=cl.F32, seed=12, stream=stream)
        ch = cl.Charges(lat, sites, q, log_capacity=8)
        ch.run(1, 4, 1, 3)
        if inject:
            t0 = time.perf_counter()
            lat.selftest_wait(20_000_000)  # 20 ms
            with pytest.raises(cl.CoulpsError) as ei:
                lat.sync()
            assert ei.value.status == cl.ETIMEOUT
            assert time.perf_counter() - t0 >= 0.015
            with pytest.raises(cl.CoulpsError) as ei:  # sticky until cleared
                ch.estimate()
            assert ei.value.status == cl.ETIMEOUT
            lat.clear_error()
            lat.sync()
        ch.run(0, 4, 1, 3)
        out.append((ch.samples(), lat.field(1), ch.estimate()))
        ch.close()
        lat.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


def test_selftest_rejects_bad_limits(cl):
    lat = cl.Lattice((8, 8, 8), n_chains=1, precision=cl.F32, seed=1)
    for bad in (0, 999, 2_000_000_000):
        with pytest.raises(cl.CoulpsError):
            lat.selftest_wait(bad)
    lat.close()
