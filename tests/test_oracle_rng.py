"""Pins of the oracle's random draws.

- Philox4x32-10 against cuRAND's host Philox4_32_10 generator (an independent,
  installed implementation): key = seed; the counter layout of its output is
  described at the test.
- The heatbath deviate of Eq. (phi), -erfc^-1(2r)/sqrt(3) with
  r = (w + 1/2) 2^-32, against scipy's inverse normal CDF:
  Phi^-1(r) = -sqrt(2) erfc^-1(2r), so the deviate is Phi^-1(r)/sqrt(6).
"""
import ctypes
import math
from pathlib import Path

import numpy as np
import pytest
import scipy.special as ss


def _curand():
    for p in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(p)
        except OSError:
            continue
    pytest.skip("libcurand not available")


def _curand_philox(seed, offset, n):
    lib = _curand()
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = (ctypes.c_uint32 * n)()
        assert lib.curandGenerate(gen, out, ctypes.c_size_t(n)) == 0
        return list(out)
    finally:
        lib.curandDestroyGenerator(gen)


# cuRAND's host Philox generator interleaves 65536 subsequences: output group j
# (four words) of a run started at offset 4 * 65536 * pos is Philox of counter
# (pos mod 2^32, pos div 2^32, j, 0).  This pins the key schedule and counter
# words 0, 1 and 2; word 3 is pinned on the GPU against cuRAND's device API.
@pytest.mark.parametrize("seed,pos", [(0, 0), (0x123456789ABCDEF0, 7),
                                      (0xFFFFFFFFFFFFFFFF, (1 << 32) + 5), (42, (1 << 40) + 3)])
def test_philox_matches_curand(orc, seed, pos):
    got = _curand_philox(seed, 4 * 65536 * pos, 4 * 24)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in range(24):
        ref = orc.philox4x32_10([pos & 0xFFFFFFFF, pos >> 32, j, 0], key)
        assert ref == got[4 * j:4 * j + 4], j


def test_philox_curand_subsequence_wrap(orc):
    # group 65536 + j continues subsequence j at the next counter
    seed = 0xC0FFEE
    got = _curand_philox(seed, 0, 4 * (65536 + 3))
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in range(3):
        assert orc.philox4x32_10([1, 0, j, 0], key) == got[4 * (65536 + j):4 * (65536 + j) + 4]


def test_philox_high_counter_words_matter(orc):
    # counter words 2 and 3 (chain, colour in the sampler) must change the output
    base = orc.philox4x32_10([5, 6, 0, 0], [1, 2])
    assert orc.philox4x32_10([5, 6, 1, 0], [1, 2]) != base
    assert orc.philox4x32_10([5, 6, 0, 1], [1, 2]) != base
    assert orc.philox4x32_10([5, 6, 1, 0], [1, 2]) != orc.philox4x32_10([5, 6, 0, 1], [1, 2])


def test_philox_bytes_uniform(orc):
    # chi^2 on the byte histogram over counters (w, pass, chain, colour)
    counts = np.zeros(256)
    for i in range(2000):
        w = orc.philox4x32_10([i, 3, i % 7, i & 1], [0xDEADBEEF, 0x12345678])
        for v in w:
            for b in range(4):
                counts[(v >> (8 * b)) & 0xFF] += 1
    exp = counts.sum() / 256
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    # 255 dof: mean 255, sd ~22.6; 5 sd bounds
    assert 140 < chi2 < 370


def test_erfcinv_against_scipy(orc):
    v = np.concatenate([np.logspace(-15, 0, 200), 2 - np.logspace(-15, -0.01, 100)])
    for x in v:
        ref = ss.erfcinv(x)
        got = orc.erfcinv(x)
        assert abs(got - ref) <= 4e-15 * max(1.0, abs(ref)), (x, got, ref)


@pytest.mark.parametrize("w", [0, 1, 2, 1000, 0x3FFFFFFF, 0x7FFFFFFE, 0x7FFFFFFF, 0x80000000,
                               0x80000001, 0xC0000000, 0xFFFFFFFE, 0xFFFFFFFF])
def test_noise_is_normal_quantile(orc, w):
    r = (w + 0.5) * 2.0 ** -32
    ref = ss.ndtri(r) / math.sqrt(6.0)
    got = orc.heatbath_noise(w)
    assert abs(got - ref) <= 1e-14 * max(1.0, abs(ref)) + 1e-17, (w, got, ref)


def test_noise_antisymmetric(orc):
    rng = np.random.default_rng(0)
    for w in rng.integers(0, 2**32, 500).tolist():
        assert orc.heatbath_noise(w) == -orc.heatbath_noise(0xFFFFFFFF - w)


def test_noise_moments(orc):
    # a stratified grid of words: the deviate is N(0, 1/6) (variance of Eq. (phi))
    ws = (np.arange(20000, dtype=np.uint64) * 214748 + 107374) % (1 << 32)
    z = np.array([orc.heatbath_noise(int(w)) for w in ws])
    assert abs(z.mean()) < 1e-3
    assert abs(z.var() - 1.0 / 6.0) < 2e-3


def test_site_word_uses_quad_numbering(orc):
    # four consecutive same-colour sites of a row share one Philox call
    L = (20, 3, 2)
    seed, chain, pass_ = 99, 5, 17
    y, z = 1, 1
    colour = 0
    key = [seed & 0xFFFFFFFF, seed >> 32]
    xs = [x for x in range(L[0]) if (x + y + z) % 2 == colour]
    Wq = (L[0] + 7) // 8
    for x in xs:
        quad = (z * L[1] + y) * Wq + (x >> 3)
        words = orc.philox4x32_10([quad, pass_, chain, colour], key)
        assert orc.site_word(L, x, y, z, colour, seed, chain, pass_) == words[(x >> 1) & 3]
