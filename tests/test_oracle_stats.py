"""Pins of the oracle's error bars on processes with known answers.

An AR(1) series x_t = a x_{t-1} + sqrt(1 - a^2) eps_t has unit variance and
integrated autocorrelation time tau_int = (1 + a) / (2 (1 - a)), so the
standard error of its mean over n samples is sqrt(2 tau_int / n).
"""
import math

import numpy as np


def _ar1(a, n, seed):
    rng = np.random.default_rng(seed)
    eps = rng.standard_normal(n)
    x = np.empty(n)
    x[0] = eps[0]
    c = math.sqrt(1 - a * a)
    for t in range(1, n):
        x[t] = a * x[t - 1] + c * eps[t]
    return x


def test_tau_int_ar1(orc):
    for a in (0.0, 0.5, 0.9):
        x = _ar1(a, 200000, seed=int(a * 10))
        tau = orc.tau_int(x)
        exact = (1 + a) / (2 * (1 - a))
        assert abs(tau / exact - 1) < 0.1, (a, tau, exact)


def test_batch_means_error_ar1(orc):
    a, n = 0.8, 320000
    exact = math.sqrt(2 * (1 + a) / (2 * (1 - a)) / n)
    ses = [orc.batch_means(_ar1(a, n, seed=s), 32)[1] for s in range(4)]
    assert abs(np.mean(ses) / exact - 1) < 0.15, (np.mean(ses), exact)


def test_batch_means_iid(orc):
    rng = np.random.default_rng(3)
    x = rng.standard_normal(64000) * 3 + 1
    m, se = orc.batch_means(x, 32)
    assert abs(m - x.mean()) < 1e-12
    assert abs(se / (3 / math.sqrt(64000)) - 1) < 0.35
