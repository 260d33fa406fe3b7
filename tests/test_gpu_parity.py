"""Parity of the CUDA sampler with the FP64 oracle, through the C ABI.

Both sides run the same chain: same seed, chain ids, Philox counters, red/black
order and cold start, so each sample (Q, P, e) and each field can be compared
one to one.  Metrics (relative, so they are meaningful when e ~ 0):
  field:  max |phi_gpu - phi_orc| / rms(phi_orc)
  Q:      |Q_gpu - Q_orc| / sqrt(P_orc)
  P, e:   |.| / (Q_orc^2 + P_orc)
Tolerances: FP64 mode 1e-12 over full runs; FP32 mode 1e-5 (the field is
FP32, every update adds an FP32 rounding of S/6 and of the erfc^-1 deviate,
and the Gaussian chain contracts such errors, so they stay at a few times
the single-update rounding).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


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


def gpu_run(cl, stream, L, n_chains, prec, seed, sites, q, n_therm, n_meas, n_hb, n_or,
            tile=None, fields=(), fused=None):
    lat = cl.Lattice(L, n_chains=n_chains, precision=prec, seed=seed, stream=stream)
    if tile:
        lat.set_tile(*tile)
    if fused is not None:
        lat.set_fused(fused)
    ch = cl.Charges(lat, sites, q, log_capacity=max(1, n_meas))
    ch.run(n_therm, n_meas, n_hb, n_or)
    s = ch.samples()
    f = {k: lat.field(k) for k in fields}
    est = ch.estimate()
    ch.close()
    lat.close()
    return s, f, est


def orc_run(orc, L, seed, chain, sites, q, n_therm, n_meas, n_hb, n_or):
    c = orc.Chain(L, seed=seed, chain=chain)
    c.run(n_therm, n_hb, n_or)
    out = c.run(n_meas, n_hb, n_or, sites, q) if n_meas else np.zeros((0, 3))
    return out, c.phi


def sample_err(got, ref):
    Q, P = ref[:, 0], ref[:, 1]
    den = Q * Q + P
    den = np.where(den > 0, den, 1.0)
    eq = np.abs(got[:, 0] - Q) / np.sqrt(np.where(P > 0, P, 1.0))
    ep = np.abs(got[:, 1] - P) / den
    ee = np.abs(got[:, 2] - ref[:, 2]) / den
    return max(eq.max(initial=0), ep.max(initial=0), ee.max(initial=0))


def field_err(got, ref):
    rms = np.sqrt(np.mean(ref * ref))
    return float(np.abs(got - ref).max() / (rms if rms > 0 else 1.0))


def test_fp64_plain_method_16cubed(cl, stream, orc):
    """16^3, 8 charges +-1, one chain, FP64, heatbath only, 200 + 2000 sweeps."""
    from paper_1403_0711_gb300 import inputs
    L = (16, 16, 16)
    sites, q = inputs.plus_minus(L, 8, seed=1)
    s, f, est = gpu_run(cl, stream, L, 1, cl.F64, 1, sites, q, 200, 2000, 1, 0, fields=(0,))
    ref, phi = orc_run(orc, L, 1, 0, sites, q, 200, 2000, 1, 0)
    assert s.shape == (2000, 1, 3)
    assert sample_err(s[:, 0], ref) < TOL64
    assert field_err(f[0], phi) < TOL64
    # the estimate is the mean of exactly these samples
    assert est["n"] == 2000
    assert abs(est["mean"] - ref[:, 2].mean()) < 1e-9 * max(1.0, np.abs(ref[:, 2]).mean())


RAGGED = [(1, 1, 1), (2, 3, 4), (13, 7, 5), (9, 1, 17), (33, 17, 9), (24, 5, 3), (17, 40, 2)]


@pytest.mark.parametrize("L", RAGGED)
def test_fp64_ragged_shapes(cl, stream, orc, L):
    from paper_1403_0711_gb300 import inputs
    n = min(6, L[0] * L[1] * L[2])
    sites, q = inputs.uniform_q(L, n, seed=sum(L))
    s, f, _ = gpu_run(cl, stream, L, 3, cl.F64, 5, sites, q, 3, 6, 1, 2, fields=(0, 2))
    for k in (0, 2):
        ref, phi = orc_run(orc, L, 5, k, sites, q, 3, 6, 1, 2)
        assert sample_err(s[:, k], ref) < TOL64, k
        assert field_err(f[k], phi) < TOL64, k


@pytest.mark.parametrize("L", RAGGED)
def test_fp32_ragged_shapes(cl, stream, orc, L):
    from paper_1403_0711_gb300 import inputs
    n = min(6, L[0] * L[1] * L[2])
    sites, q = inputs.uniform_q(L, n, seed=sum(L))
    s, f, _ = gpu_run(cl, stream, L, 2, cl.F32, 7, sites, q, 3, 6, 1, 3, fields=(1,))
    ref, phi = orc_run(orc, L, 7, 1, sites, q, 3, 6, 1, 3)
    assert sample_err(s[:, 1], ref) < TOL32
    assert field_err(f[1], phi) < TOL32


def test_fp32_window_64cubed(cl, stream, orc):
    """A 200-compound-sweep comparison window (1 heatbath : 3 over-relaxation)."""
    from paper_1403_0711_gb300 import inputs
    L = (64, 64, 64)
    sites, q = inputs.plus_minus(L, 512, seed=2)
    s, f, _ = gpu_run(cl, stream, L, 1, cl.F32, 3, sites, q, 0, 200, 1, 3, fields=(0,))
    ref, phi = orc_run(orc, L, 3, 0, sites, q, 0, 200, 1, 3)
    assert sample_err(s[:, 0], ref) < TOL32
    assert field_err(f[0], phi) < TOL32


@pytest.mark.parametrize("fused", [1, 3, 4])
def test_fp32_full_size_sampled_chains(cl, stream, orc, fused):
    """128^3, 4096 charges +-1, 64 chains, 1 HB : 3 OR, default tiles, on the
    fused-pass (1), the over-relaxation pass-pair (3, the benchmark launch
    configuration) and the all-pairs (4) schedules, the sample gathered by the
    sweep's last kernel; chains 0, 37 and 63 checked against the oracle."""
    from paper_1403_0711_gb300 import inputs
    L = (128, 128, 128)
    sites, q = inputs.plus_minus(L, 4096, seed=1)
    s, f, _ = gpu_run(cl, stream, L, 64, cl.F32, 1, sites, q, 1, 3, 1, 3, fields=(0, 37, 63),
                      fused=fused)
    for k in (0, 37, 63):
        ref, phi = orc_run(orc, L, 1, k, sites, q, 1, 3, 1, 3)
        assert sample_err(s[:, k], ref) < TOL32, k
        assert field_err(f[k], phi) < TOL32, k


@pytest.mark.parametrize("tile", [(1, 1), (3, 5), (7, 128), (16, 2)])
def test_tile_shape_does_not_change_results(cl, stream, tile):
    from paper_1403_0711_gb300 import inputs
    L = (40, 23, 19)
    sites, q = inputs.uniform_q(L, 50, seed=3)
    base, fb, _ = gpu_run(cl, stream, L, 2, cl.F32, 9, sites, q, 2, 4, 1, 2, fields=(1,))
    got, fg, _ = gpu_run(cl, stream, L, 2, cl.F32, 9, sites, q, 2, 4, 1, 2, tile=tile, fields=(1,))
    # the field is bitwise the same; the fused gather's CTA partials follow the
    # tile decomposition, so Q and P differ only in FP64 summation order
    assert np.array_equal(fb[1], fg[1])
    for k in range(2):
        assert sample_err(got[:, k], base[:, k]) < 1e-13


@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4])
def test_fused_and_separate_gather_agree(cl, stream, mode):
    """coulps_run gathers inside the sweep's last kernel (a half-sweep with
    mode 0, a fused pass with modes 1, 2 and 3, a pass pair with mode 4);
    coulps_measure runs the separate gather kernel on the same fields: same
    samples."""
    from paper_1403_0711_gb300 import inputs
    L = (48, 33, 29)
    sites, q = inputs.uniform_q(L, 700, seed=12)
    fused, _, _ = gpu_run(cl, stream, L, 3, cl.F32, 13, sites, q, 1, 5, 1, 3, fused=mode)
    lat = cl.Lattice(L, n_chains=3, precision=cl.F32, seed=13, stream=stream)
    lat.set_fused(mode)
    ch = cl.Charges(lat, sites, q, log_capacity=5)
    lat.sweep(1, 1, 3)
    for _ in range(5):
        lat.sweep(1, 1, 3)
        ch.measure()
    sep = ch.samples()
    ch.close()
    lat.close()
    for k in range(3):
        assert sample_err(sep[:, k], fused[:, k]) < 1e-13


def test_bitwise_reproducible(cl, stream):
    from paper_1403_0711_gb300 import inputs
    L = (32, 32, 32)
    sites, q = inputs.plus_minus(L, 100, seed=4)
    a, _, ea = gpu_run(cl, stream, L, 8, cl.F32, 11, sites, q, 5, 20, 1, 3)
    b, _, eb = gpu_run(cl, stream, L, 8, cl.F32, 11, sites, q, 5, 20, 1, 3)
    assert np.array_equal(a, b)
    assert ea == eb


def test_single_and_no_charges(cl, stream):
    L = (10, 9, 8)
    s, _, est = gpu_run(cl, stream, L, 4, cl.F32, 2, np.array([[3, 4, 5]]), [1.5], 2, 10, 1, 1)
    assert np.all(s[:, :, 2] == 0.0)
    assert np.all(s[:, :, 1] > 0.0)
    assert est["mean"] == 0.0
    s, _, est = gpu_run(cl, stream, L, 2, cl.F32, 2, np.zeros((0, 3), np.int32), [], 2, 5, 1, 1)
    assert np.all(s == 0.0)


def test_invalid_arguments_raise(cl, stream):
    lat = cl.Lattice((8, 8, 8), n_chains=1, precision=cl.F32, seed=0, stream=stream)
    with pytest.raises(cl.CoulpsError) as ei:
        cl.Charges(lat, np.array([[8, 0, 0]]), [1.0])
    assert ei.value.status == cl.EINVAL
    with pytest.raises(cl.CoulpsError):
        cl.Charges(lat, np.array([[0, 0, 0]]), [float("nan")])
    with pytest.raises(cl.CoulpsError):
        lat.sweep(-1, 1, 0)
    with pytest.raises(cl.CoulpsError):
        lat.set_tile(300, 1)
    lat.close()


def test_checkpoint_resume_bitwise(cl, stream, tmp_path):
    from paper_1403_0711_gb300 import inputs
    L = (20, 18, 16)
    sites, q = inputs.uniform_q(L, 30, seed=6)
    full, ff, efull = gpu_run(cl, stream, L, 3, cl.F32, 21, sites, q, 2, 12, 1, 2, fields=(2,))

    lat = cl.Lattice(L, n_chains=3, precision=cl.F32, seed=21, stream=stream)
    ch = cl.Charges(lat, sites, q, log_capacity=12)
    ch.run(2, 5, 1, 2)
    path = tmp_path / "state.ckpt"
    lat.checkpoint_save(path, ch)
    ch.close()
    lat.close()

    lat = cl.Lattice(L, n_chains=3, precision=cl.F32, seed=21, stream=stream)
    ch = cl.Charges(lat, sites, q, log_capacity=12)
    lat.checkpoint_load(path, ch)
    ch.run(0, 7, 1, 2)
    s = ch.samples()
    assert np.array_equal(s, full)
    assert np.array_equal(lat.field(2), ff[2])
    assert ch.estimate() == efull
    # a corrupted file is rejected
    raw = bytearray(path.read_bytes())
    raw[200] ^= 0xFF
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(bytes(raw))
    with pytest.raises(cl.CoulpsError) as ei:
        lat.checkpoint_load(bad, ch)
    assert ei.value.status == cl.ECORRUPT
    ch.close()
    lat.close()


def test_mc_mean_matches_e_lat(cl, stream, orc):
    """The paper's Fig. 2 geometry (8 charges q=1 in a cube) in a 16^3 box:
    pooled mean over 64 chains within 4 batch-means sigma of E_lat."""
    from paper_1403_0711_gb300 import inputs
    L = (16, 16, 16)
    sites, q = inputs.cube(L, 2)
    exact = orc.e_lat(L, sites, q, "dense")
    lat = cl.Lattice(L, n_chains=64, precision=cl.F32, seed=1234, stream=stream)
    ch = cl.Charges(lat, sites, q)
    ch.run(200, 3000, 1, 1)
    est = ch.estimate()
    ch.close()
    lat.close()
    assert abs(est["mean"] - exact) < 4 * est["stderr"], (est, exact)
    assert est["stderr"] < 0.01 * abs(exact)


def test_fp32_large_system_blobs_512(cl, stream, orc):
    """512^3 lattice (0.5 GB FP32 per field), N = 10^6 charges in 200 Gaussian
    blobs (sigma = 6), q uniform in [-0.8, 0.8] shifted to zero net, 1 chain,
    default tile: one thermalisation and one measured compound sweep against
    the oracle (sample and field)."""
    from paper_1403_0711_gb300 import inputs
    L = (512, 512, 512)
    sites, q = inputs.blobs(L, 1_000_000, seed=3)
    assert len(np.unique(sites[:, 0] + 512 * (sites[:, 1] + 512 * sites[:, 2]))) == 1_000_000
    assert abs(q.sum()) < 1e-6
    s, f, _ = gpu_run(cl, stream, L, 1, cl.F32, 8, sites, q, 1, 1, 1, 3, fields=(0,))
    ref, phi = orc_run(orc, L, 8, 0, sites, q, 1, 1, 1, 3)
    assert sample_err(s[:, 0], ref) < TOL32
    assert field_err(f[0], phi) < TOL32


@pytest.mark.parametrize("n_hb,n_or,chains,profiling", [(1, 3, 8, False), (1, 3, 8, True),
                                                         (2, 1, 5, False), (1, 1, 3, False)])
def test_phased_schedule_is_bitwise_identical(cl, stream, n_hb, n_or, chains, profiling):
    """The phase-shifted schedule does every chain's passes and samples exactly
    as the aligned one (graph replay and direct launches alike)."""
    from paper_1403_0711_gb300 import inputs
    L = (24, 13, 11)
    sites, q = inputs.uniform_q(L, 40, seed=21)
    out = {}
    for sched in (cl.SCHEDULE_ALIGNED, cl.SCHEDULE_PHASED):
        lat = cl.Lattice(L, n_chains=chains, precision=cl.F32, seed=31, stream=stream)
        lat.set_fused(False)  # the half-sweep path on both sides (fusion has its own tests)
        lat.set_schedule(sched)
        lat.set_profiling(profiling)
        ch = cl.Charges(lat, sites, q, log_capacity=9)
        ch.run(2, 6, n_hb, n_or)
        ch.run(0, 3, n_hb, n_or)
        out[sched] = (ch.samples(), [lat.field(k) for k in range(chains)], ch.estimate(),
                      lat.info()["pass"], lat.kernel_times())
        ch.close()
        lat.close()
    a, b = out[cl.SCHEDULE_ALIGNED], out[cl.SCHEDULE_PHASED]
    assert np.array_equal(a[0], b[0])
    for fa, fb in zip(a[1], b[1]):
        assert np.array_equal(fa, fb)
    assert a[2] == b[2] and a[3] == b[3]
    if profiling:
        assert b[4]["mixed_n"] > 0 and a[4]["mixed_n"] == 0


def test_pipelined_estimates_equal_synchronous(cl, stream):
    """coulps_estimate_post / _take, one step behind, return for every step
    exactly what coulps_estimate returns on an identical chain read
    synchronously; the posting rules are enforced."""
    from paper_1403_0711_gb300 import inputs
    L = (24, 20, 18)
    sites, q = inputs.plus_minus(L, 16, seed=5)

    def chain():
        lat = cl.Lattice(L, n_chains=6, precision=cl.F32, seed=41, stream=stream)
        ch = cl.Charges(lat, sites, q)
        ch.run(3, 0, 1, 3)
        return lat, ch

    lat, ch = chain()
    sync = []
    for _ in range(7):
        ch.update(sites, q)
        ch.run(0, 1, 1, 3)
        sync.append(ch.estimate())
    ch.close()
    lat.close()

    lat, ch = chain()
    with pytest.raises(cl.CoulpsError):
        ch.estimate_take()  # nothing posted
    piped = []
    for k in range(7):
        ch.update(sites, q)
        ch.run(0, 1, 1, 3)
        ch.estimate_post()
        if k > 0:
            piped.append(ch.estimate_take())
    piped.append(ch.estimate_take())
    ch.estimate_post()
    ch.estimate_post()
    with pytest.raises(cl.CoulpsError):
        ch.estimate_post()  # two states not taken yet
    a, b = ch.estimate_take(), ch.estimate_take()
    assert a == b == ch.estimate()
    ch.close()
    lat.close()
    assert [e["n"] for e in piped] == [6 * (k + 1) for k in range(7)]
    assert piped == sync
