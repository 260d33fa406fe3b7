"""The autotuner's candidate tile shapes respect the kernels' launch limits
(host logic only): half-sweep CTAs of at most 256 threads with halo boxes of
at most 256 rows, fused-pass CTAs of at most 512 threads with colour-1 boxes
of at most 256 rows, slabs no thicker than the box."""
import pytest


@pytest.mark.parametrize("L", [(128, 128, 128), (13, 7, 5), (512, 3, 40), (2, 300, 2), (96, 96, 96)])
@pytest.mark.parametrize("prec", [0, 1])
def test_candidates_within_limits(L, prec):
    from paper_1403_0711_gb300 import autotune
    Lx, Ly, Lz = L
    qw = autotune.row_stride(Lx, prec) // 4
    c = autotune.candidates(L, prec)
    assert c
    for ty, dz in c:
        assert 1 <= ty <= Ly and qw * ty <= 256 and ty + 2 <= 256 and 1 <= dz <= max(Lz, 1)
    p = autotune.pass_candidates(L, prec)
    assert p
    for ty, dz in p:
        assert 1 <= ty <= max(Ly, 1) and qw * (ty + 2) <= 512 and ty + 4 <= 256 and 1 <= dz <= Lz
    if L == (128, 128, 128) and prec == 0:
        assert (13, 32) in p and (16, 16) in c  # the defaults are candidates
    maxt = 512 if prec == 0 else 256
    for ty, dz in autotune.pair_candidates(L, prec):
        assert 1 <= ty <= Ly and qw * (ty + 6) <= maxt and ty + 8 <= 256 and 1 <= dz <= Lz
    if L == (128, 128, 128) and prec == 0:
        assert (26, 64) in autotune.pair_candidates(L, prec)  # the default pair tile


def test_row_stride_matches_layout():
    from paper_1403_0711_gb300 import autotune
    # 32-byte rows of ceil(Lx / 2) same-colour sites, quads of 4
    assert autotune.row_stride(128, 0) == 64 and autotune.row_stride(13, 0) == 8
    assert autotune.row_stride(13, 1) == 8 and autotune.row_stride(1, 1) == 4
    assert autotune.row_stride(100, 0) == 56


def test_every_shape_refused_is_an_error(monkeypatch):
    """When the library refuses every candidate the tuner says so for the box
    (a CoulpsError), instead of failing on an empty timing table."""
    from paper_1403_0711_gb300 import autotune, coulps
    monkeypatch.setattr(autotune, "_time_shapes", lambda *a, **k: {})
    for fn in (autotune.tune_shape, autotune.tune_pass_shape, autotune.tune_pair_shape):
        with pytest.raises(coulps.CoulpsError, match="refused every"):
            fn((16, 16, 16), use_cache=False)
