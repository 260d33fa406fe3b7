"""Writes the polynomial coefficients of the FP32 heatbath deviate
(device_common.cuh, hb_noise_f32).

The deviate needs erfc^-1(u) / sqrt(3) for u in (0, 1].  It is written as
x q(v) with x = 1 - u and v = -log2(u (2 - u)) = -log2(u (1 + x)), the change
of variable of M. Giles ("Approximating the erfinv function", GPU Computing
Gems Jade Edition, 2011) taken in base 2 so that the device's log2 is used
as is: q is smooth in v, so two polynomials cover the range, one of degree
10 in v - 4.5 for v < 9 and one of degree 9 in sqrt(v) - 3.6 for
9 <= v <= 33 (u >= 2^-32 keeps v < 32).  The factor 1/sqrt(3) of Eq. (phi) is folded into q.  The
coefficients are fitted here from scratch: least squares on Chebyshev nodes,
weighted by 1/q (relative error), reweighted a few times towards the
equal-ripple (minimax) solution, against scipy's erfcinv in FP64.

Run: python fit_erfcinv.py   (prints the two coefficient lists, lowest order
first, with their fit errors and the emulated error of the FP32 evaluation)
"""
import numpy as np
from scipy.special import erfcinv

N_NODES = 4000
SPLIT = 9.0
CENTRAL = (0.0, SPLIT, False, 4.5, 10)  # v range, in sqrt(v)?, centre, degree
TAIL = (SPLIT, 33.0, True, 3.6, 9)


def target(v):
    """q(v) = erfc^-1(u) / (sqrt(3) x) where u (2 - u) = 2^-v."""
    x = np.sqrt(-np.expm1(-v * np.log(2.0)))  # x^2 = 1 - 2^-v
    return erfcinv(1.0 - x) / (np.sqrt(3.0) * x)


def fit(v_lo, v_hi, use_sqrt, centre, degree, iters=30):
    a, b = (np.sqrt(v_lo), np.sqrt(v_hi)) if use_sqrt else (v_lo, v_hi)
    a, b = a - centre, b - centre
    k = np.arange(N_NODES)
    z = 0.5 * (a + b) + 0.5 * (b - a) * np.cos(np.pi * (k + 0.5) / N_NODES)
    v = (z + centre) ** 2 if use_sqrt else z + centre
    v = np.maximum(v, 1e-12)
    q = target(v)
    V = np.vander(z, degree + 1, increasing=True)
    wt = np.ones(N_NODES)
    for _ in range(iters):
        s = wt / np.abs(q)
        c, *_ = np.linalg.lstsq(V * s[:, None], q * s, rcond=None)
        r = (V @ c - q) / q
        wt = wt * np.sqrt(np.abs(r)) + 1e-300
        wt /= wt.max()
    return c, float(np.abs(r).max())


def emulate_fp32(central, tail, n=2_000_000, seed=0):
    """Max relative error of the device's FP32 steps (one rounding per
    operation, fused multiply-adds rounded once) against FP64, over random
    and extreme words."""
    f32 = np.float32
    rng = np.random.default_rng(seed)
    s = np.concatenate([rng.integers(0, 2**31, n), np.arange(100000),
                        2**31 - 1 - np.arange(100000)]).astype(np.int64)
    u = (s.astype(f32) * f32(2.0**-31) + f32(2.0**-32)).astype(f32)
    x = ((2**31 - 1 - s).astype(f32) * f32(2.0**-31) + f32(2.0**-32)).astype(f32)
    t = (u.astype(np.float64) * x + u).astype(f32)
    v = (-np.log2(t.astype(np.float64))).astype(f32)
    out = np.empty(len(s))
    m = v < f32(SPLIT)
    for mask, c, spec in ((m, central, CENTRAL), (~m, tail, TAIL)):
        vv = v[mask]
        z = (np.sqrt(vv).astype(f32) if spec[2] else vv) - f32(spec[3])
        z = z.astype(f32)
        cf = c.astype(f32)
        p = np.full(z.shape, cf[-1], dtype=f32)
        for ck in cf[-2::-1]:
            p = (p.astype(np.float64) * z + ck).astype(f32)
        out[mask] = (p * x[mask]).astype(f32)
    ref = erfcinv((s + 0.5) * 2.0**-31) / np.sqrt(3.0)
    return float(np.max(np.abs(out - ref) / ref))


def main():
    central, e1 = fit(*CENTRAL)
    tail, e2 = fit(*TAIL)
    for name, c, e in (("central (v - 4.5)", central, e1), ("tail (sqrt(v) - 3.6)", tail, e2)):
        print(f"{name}: max relative fit error {e:.2e}")
        print("  " + ", ".join(f"{float(np.float32(v)):.8g}f" for v in c))
    print(f"emulated FP32 evaluation: max relative error {emulate_fp32(central, tail):.2e}")


if __name__ == "__main__":
    main()
