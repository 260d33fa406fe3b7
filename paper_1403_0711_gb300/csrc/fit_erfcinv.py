"""Writes the polynomial coefficients of the FP32 heatbath deviate
(device_common.cuh, hb_erfcinv_f32).

erfc^-1(u) for u in (0, 1] is written as x p(w) with x = 1 - u and
w = -ln(u (2 - u)) (the change of variable of M. Giles, "Approximating the
erfinv function", GPU Computing Gems Jade Edition, 2011): p is smooth in w, so
two polynomials cover the whole range, one in w - 2.5 for w < 5 and one in
sqrt(w) - 3 for 5 <= w <= 22.5 (u >= 2^-32 gives w < 21.5).  The
coefficients here are fitted from scratch: least squares on Chebyshev nodes,
weighted by 1/p (relative error), reweighted a few times towards the
equal-ripple (minimax) solution, against scipy's erfcinv in FP64.

Run: python fit_erfcinv.py   (prints the two arrays and the fit errors)
"""
import numpy as np
from scipy.special import erfcinv

N_NODES = 4000


def fit(w_lo, w_hi, use_sqrt, centre, degree, iters=30):
    a, b = (np.sqrt(w_lo), np.sqrt(w_hi)) if use_sqrt else (w_lo, w_hi)
    a, b = a - centre, b - centre
    k = np.arange(N_NODES)
    z = 0.5 * (a + b) + 0.5 * (b - a) * np.cos(np.pi * (k + 0.5) / N_NODES)
    w = (z + centre) ** 2 if use_sqrt else z + centre
    x = np.sqrt(-np.expm1(-w))          # u (2 - u) = e^-w  <=>  x^2 = 1 - e^-w
    u = 1.0 - x
    p = erfcinv(u) / x
    V = np.vander(z, degree + 1, increasing=True)
    wt = np.ones(N_NODES)
    for _ in range(iters):
        s = wt / np.abs(p)
        c, *_ = np.linalg.lstsq(V * s[:, None], p * s, rcond=None)
        r = (V @ c - p) / p
        wt = wt * np.sqrt(np.abs(r)) + 1e-300
        wt /= wt.max()
    return c, float(np.abs(r).max())


def main():
    central, e1 = fit(1e-12, 5.0, False, 2.5, 9)
    tail, e2 = fit(5.0, 22.5, True, 3.0, 10)
    for name, c, e in (("kErfcinvCentral", central, e1), ("kErfcinvTail", tail, e2)):
        vals = ", ".join(f"{np.float32(v)!r:}f".replace("np.float32(", "").replace(")", "")
                         for v in c)
        print(f"// max relative fit error {e:.2e}")
        print(f"__constant__ ... {name}[{len(c)}] = {{{vals}}};")


if __name__ == "__main__":
    main()
