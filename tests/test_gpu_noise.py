"""The heatbath's random term -erfc^-1(2r)/sqrt(3) as the sweep kernels form
it (coulps_heatbath_noise), against the FP64 oracle's value for the same
32-bit word.  FP64: CUDA's erfcinv, 1e-14 relative.  FP32: the library's own
erfc^-1 (polynomial in Giles' variable, both u and 1 - u formed from the
integer word) within 5e-7 relative everywhere (about 8 FP32 ulps; the fit
itself is 2e-8, the rest is FP32 rounding of u, x, w, the Horner steps and
the fast logarithm), including the tails where r -> 0 or 1 and the words
around the branch at w = 5."""
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
    return coulps


def _words():
    rng = np.random.default_rng(2024)
    w = [rng.integers(0, 2**32, 150000, dtype=np.uint64)]
    edges = np.array([0, 1, 2, 3, 2**31 - 3, 2**31 - 2, 2**31 - 1, 2**31, 2**31 + 1, 2**31 + 2,
                      2**32 - 3, 2**32 - 2, 2**32 - 1], dtype=np.uint64)
    w.append(edges)
    # around the FP32 deviate's switch between its two polynomials:
    # v = -log2(u (2 - u)) = 9, u = 1 - sqrt(1 - 2^-9)
    s9 = int((1.0 - np.sqrt(1.0 - 2.0**-9)) * 2**31)
    near = np.arange(s9 - 2000, s9 + 2000, dtype=np.uint64)
    w += [near, (2**32 - 1) - near]
    # the first and last 20000 words of each side (r -> 0, r -> 1/2, r -> 1)
    k = np.arange(20000, dtype=np.uint64)
    w += [k, 2**31 - 1 - k, 2**31 + k, 2**32 - 1 - k]
    return np.concatenate(w).astype(np.uint32)


def test_heatbath_noise_matches_oracle(cl, orc):
    import torch
    w = _words()
    ref = np.array([orc.heatbath_noise(int(v)) for v in w])
    t = torch.from_numpy(w.view(np.int32)).cuda()
    got64 = cl.heatbath_noise(t, cl.F64).cpu().numpy()
    got32 = cl.heatbath_noise(t, cl.F32).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    den = np.abs(ref)
    assert np.all(den > 0)
    # (FP64: relative to |ref| + 1e-3, as erfc^-1 near u = 1 is ~1e-10 and
    # the two FP64 routines differ there by ~1e-19 absolute)
    r64 = np.abs(got64 - ref) / (den + 1e-3)
    r32 = np.abs(got32 - ref) / den
    print(f"max relative error FP32 {r32.max():.3e}, FP64 {r64.max():.3e}")
    assert r64.max() < 1e-13, r64.max()
    assert r32.max() < 5e-7, (r32.max(), w[r32.argmax()])
    # the sign convention: w < 2^31 is 2r < 1, a negative term
    assert np.all((got32 < 0) == (w < 2**31))
