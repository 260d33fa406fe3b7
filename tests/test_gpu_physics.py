"""Properties of the CUDA sweeps that hold at any size, checked on seeded
fields set into the lattice:
  * over-relaxation (phi -> S/3 - phi, a reflection about the conditional
    mean) leaves H_L = 1/2 sum over unordered neighbour pairs, box-ghost links
    included, of (phi_x - phi_y)^2 unchanged, for the half-sweep and the fused
    paths alike (to the rounding of the field's precision);
  * setting and reading a field round-trips exactly on ragged shapes."""
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


def _h_l(phi):
    """1/2 sum over unordered nearest-neighbour pairs of (difference)^2, with
    phi = 0 on the ghost layer around the box (each box-ghost link once)."""
    p = np.pad(phi, 1)
    h = 0.0
    for ax in range(3):
        d = np.diff(p, axis=ax)
        h += 0.5 * float(np.sum(d * d))
    return h


@pytest.mark.parametrize("L,prec,fused,n_or", [((13, 7, 5), "F64", 0, 3), ((13, 7, 5), "F64", 1, 4),
                                               ((24, 17, 9), "F32", 1, 2), ((31, 8, 12), "F32", 0, 1),
                                               ((16, 16, 16), "F64", 2, 2),
                                               ((24, 17, 9), "F32", 3, 2), ((13, 7, 5), "F64", 3, 4),
                                               ((24, 17, 9), "F32", 4, 3)])
def test_over_relaxation_conserves_action(cl, stream, L, prec, fused, n_or):
    from paper_1403_0711_gb300 import inputs
    fields = inputs.gaussian_fields(L, 2, seed=sum(L))
    lat = cl.Lattice(L, n_chains=2, precision=getattr(cl, prec), seed=1, stream=stream)
    lat.set_fused(fused)
    for k, f in enumerate(fields):
        lat.set_field(k, f)
    before = [_h_l(lat.field(k)) for k in range(2)]
    lat.sweep(3, 0, n_or)
    tol = 1e-12 if prec == "F64" else 2e-5
    for k in range(2):
        after = _h_l(lat.field(k))
        assert abs(after - before[k]) < tol * before[k], (k, before[k], after)
        assert not np.array_equal(lat.field(k), fields[k])  # the field did move
    lat.close()


@pytest.mark.parametrize("L,prec", [((13, 7, 5), "F64"), ((9, 1, 17), "F32"), ((2, 3, 4), "F64"),
                                    ((128, 5, 3), "F32")])
def test_field_round_trip(cl, stream, L, prec):
    from paper_1403_0711_gb300 import inputs
    lat = cl.Lattice(L, n_chains=3, precision=getattr(cl, prec), seed=2, stream=stream)
    fields = inputs.gaussian_fields(L, 3, seed=7)
    if prec == "F32":
        fields = [f.astype(np.float32).astype(np.float64) for f in fields]
    for k, f in enumerate(fields):
        lat.set_field(k, f)
    for k, f in enumerate(fields):
        assert np.array_equal(lat.field(k), f)
    lat.close()
