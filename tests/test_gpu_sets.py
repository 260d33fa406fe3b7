"""Several charge sets measured on the same samples (coulps_run_sets /
coulps_measure_sets) equal the one-set path bit for bit: same fields, and per
set the same (Q, P, e) as coulps_measure takes (same per-CTA arithmetic, same
fixed-order finalize), also past the 32 sets of one gather launch."""
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


def _sets(L, n_sets):
    from paper_1403_0711_gb300 import inputs
    out = [inputs.cube(L, 2), inputs.plus_minus(L, 40, seed=1), inputs.uniform_q(L, 333, seed=2),
           (np.zeros((0, 3), np.int32), np.zeros(0))]
    k = 0
    while len(out) < n_sets:
        out.append(inputs.two_body(L, 1 + k % 5))
        k += 1
    return out[:n_sets]


@pytest.mark.parametrize("n_sets,prec,fused", [(4, "F32", 1), (40, "F32", 0), (5, "F64", 1)])
def test_sets_equal_single_set_measurements(cl, stream, n_sets, prec, fused):
    L = (21, 18, 16)
    p = getattr(cl, prec)
    charge_sets = _sets(L, n_sets)
    n_meas = 6
    a = cl.Lattice(L, n_chains=3, precision=p, seed=5, stream=stream)
    a.set_fused(fused)
    sa = [cl.Charges(a, s, q, log_capacity=n_meas) for s, q in charge_sets]
    cl.run_sets(a, sa, 2, n_meas, 1, 3)
    b = cl.Lattice(L, n_chains=3, precision=p, seed=5, stream=stream)
    b.set_fused(fused)
    sb = [cl.Charges(b, s, q, log_capacity=n_meas) for s, q in charge_sets]
    b.sweep(2, 1, 3)
    for _ in range(n_meas):
        b.sweep(1, 1, 3)
        for c in sb:
            c.measure()
    for k in range(3):
        assert np.array_equal(a.field(k), b.field(k))
    for ca, cb in zip(sa, sb):
        assert np.array_equal(ca.samples(), cb.samples())
        assert np.array_equal(ca.chain_stats(), cb.chain_stats())
    # one more sample of every set from the current fields
    cl.measure_sets(a, sa)
    for c in sb:
        c.measure()
    for ca, cb in zip(sa, sb):
        assert np.array_equal(ca.samples(), cb.samples())
    for o in sa + sb + [a, b]:
        o.close()


def test_sets_reject_bad_arguments(cl, stream):
    L = (8, 8, 8)
    a = cl.Lattice(L, n_chains=1, precision=cl.F32, seed=1, stream=stream)
    b = cl.Lattice(L, n_chains=1, precision=cl.F32, seed=1, stream=stream)
    ca = cl.Charges(a, *_sets(L, 1)[0])
    cb = cl.Charges(b, *_sets(L, 1)[0])
    with pytest.raises(cl.CoulpsError):
        cl.run_sets(a, [ca, cb], 0, 1, 1, 1)
    with pytest.raises(cl.CoulpsError):
        cl.measure_sets(a, [])
    for o in (ca, cb, a, b):
        o.close()
