"""FP64 oracle for the lattice path-integral Coulomb method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The product library
never imports, links or executes anything under ``oracle/``.  Nothing here is
shared with the CUDA path.

Two independent halves (Sugihara, Higo & Nakamura, JPSJ 2014):

1. The exact value the Monte Carlo converges to.  Eq. (nsum) with the lattice
   two-point function of Eq. (proplat) gives
       E_lat = sum_{i != j} q_i q_j G(r_i, r_j),   G = A^{-1},
   where A = -Delta_lat is the matrix of H_L = 1/2 phi^T A phi with phi = 0
   outside the box (6 on the diagonal, -1 per nearest-neighbour pair).  G is
   obtained here by dense inversion (tiny boxes), by the sine-transform
   (DST-I) spectral solve (A's eigenvectors are products of sines), by plain
   conjugate gradients, and -- for the diagonal G(r, r) at many sites -- by
   quadrature of the heat-kernel integral G = int_0^inf exp(-tA) dt, which
   factorises over the three axes.
   The continuum Eq. (s1) and the infinite-lattice G of Eq. (proplat) are here
   too, for the 1/(4 pi r) limit.

2. The same-chain sampler (``orc.c``): heatbath Eq. (phi) / over-relaxation
   half-sweeps and the estimator Eq. (nsum2), one site at a time in FP64.
   Error bars follow the usual batch-means rule.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import sys
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "orc.c"
_LIB = _HERE / "liborc.so"


# --------------------------------------------------------------------------
# Build and load the C half
# --------------------------------------------------------------------------
def build(force: bool = False) -> Path:
    """Compile orc.c into liborc.so with gcc (OpenMP within a colour)."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".{os.getpid()}.tmp.so")
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               str(_SRC), "-o", str(tmp), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB))
        u32, u64, i32, i64, f64 = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                                   ctypes.c_int64, ctypes.c_double)
        P = ctypes.POINTER
        L.orc_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
        L.orc_philox4x32_10.restype = None
        L.orc_erfcinv.argtypes = [f64]
        L.orc_erfcinv.restype = f64
        L.orc_heatbath_noise.argtypes = [u32]
        L.orc_heatbath_noise.restype = f64
        L.orc_site_word.argtypes = [i32, i32, i32, i32, i32, i32, u64, u32, u32]
        L.orc_site_word.restype = u32
        L.orc_halfsweep.argtypes = [P(f64), i32, i32, i32, i32, i32, u64, u32, u32, f64]
        L.orc_halfsweep.restype = None
        L.orc_pass.argtypes = [P(f64), i32, i32, i32, i32, u64, u32, u32, f64]
        L.orc_pass.restype = None
        L.orc_measure.argtypes = [P(f64), P(i64), P(f64), i64, P(f64)]
        L.orc_measure.restype = None
        L.orc_action.argtypes = [P(f64), i32, i32, i32]
        L.orc_action.restype = f64
        L.orc_run.argtypes = [P(f64), i32, i32, i32, u64, u32, P(u32), i32, i32, i32,
                              P(i64), P(f64), i64, P(f64)]
        L.orc_run.restype = None
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(shape):
    """shape is (Lz, Ly, Lx) of a natural-order field array."""
    Lz, Ly, Lx = shape
    return int(Lx), int(Ly), int(Lz)


# --------------------------------------------------------------------------
# Sampler wrappers (field arrays are float64, shape (Lz, Ly, Lx), C order)
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def erfcinv(v: float) -> float:
    return lib().orc_erfcinv(float(v))


def heatbath_noise(w: int) -> float:
    """-erfc^-1(2r)/sqrt(3) for r = (w + 1/2) 2^-32 (the random term of Eq. (phi))."""
    return lib().orc_heatbath_noise(int(w) & 0xffffffff)


def site_word(L, x, y, z, colour, seed, chain, pass_):
    Lx, Ly, _ = L
    return lib().orc_site_word(Lx, Ly, x, y, z, colour, seed, chain, pass_)


def halfsweep(phi, colour, heatbath, seed=0, chain=0, pass_=0, noise_scale=1.0):
    assert phi.dtype == np.float64 and phi.flags.c_contiguous
    Lx, Ly, Lz = _dims(phi.shape)
    lib().orc_halfsweep(_dp(phi), Lx, Ly, Lz, int(colour), int(bool(heatbath)),
                        int(seed), int(chain), int(pass_), float(noise_scale))


def one_pass(phi, heatbath, seed=0, chain=0, pass_=0, noise_scale=1.0):
    Lx, Ly, Lz = _dims(phi.shape)
    lib().orc_pass(_dp(phi), Lx, Ly, Lz, int(bool(heatbath)), int(seed), int(chain),
                   int(pass_), float(noise_scale))


def action(phi) -> float:
    """H_L of the paper (each nearest-neighbour pair once, ghosts = 0)."""
    Lx, Ly, Lz = _dims(phi.shape)
    return lib().orc_action(_dp(phi), Lx, Ly, Lz)


def site_index(L, sites):
    """Natural x-fastest index of (x, y, z) rows."""
    Lx, Ly, _ = L
    s = np.asarray(sites, dtype=np.int64).reshape(-1, 3)
    return s[:, 0] + Lx * (s[:, 1] + Ly * s[:, 2])


def measure(phi, sites, q):
    """(Q, P, e) of Eq. (nsum2) for one field."""
    L = _dims(phi.shape)
    idx = np.ascontiguousarray(site_index(L, sites))
    qq = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_measure(_dp(phi), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                      _dp(qq), len(qq), _dp(out))
    return out


class Chain:
    """One Markov chain of the oracle sampler (cold start phi = 0)."""

    def __init__(self, L, seed, chain=0):
        self.L = tuple(int(v) for v in L)
        Lx, Ly, Lz = self.L
        self.phi = np.zeros((Lz, Ly, Lx), dtype=np.float64)
        self.seed = int(seed)
        self.chain = int(chain)
        self.pass_ = 0

    def run(self, n_compound, n_hb=1, n_or=0, sites=None, q=None):
        """n_compound compound sweeps; returns the (n_compound, 3) array of
        (Q, P, e) after each one if charges are given, else None."""
        Lx, Ly, Lz = self.L
        pc = ctypes.c_uint32(self.pass_)
        if sites is not None:
            idx = np.ascontiguousarray(site_index(self.L, sites))
            qq = np.ascontiguousarray(q, dtype=np.float64)
            out = np.zeros((n_compound, 3))
            lib().orc_run(_dp(self.phi), Lx, Ly, Lz, self.seed, self.chain, ctypes.byref(pc),
                          int(n_compound), int(n_hb), int(n_or),
                          idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(qq),
                          len(qq), _dp(out))
        else:
            out = None
            lib().orc_run(_dp(self.phi), Lx, Ly, Lz, self.seed, self.chain, ctypes.byref(pc),
                          int(n_compound), int(n_hb), int(n_or), None, None, 0, None)
        self.pass_ = int(pc.value)
        return out


# --------------------------------------------------------------------------
# The lattice operator A = -Delta_lat (Dirichlet) and its inverse G
# --------------------------------------------------------------------------
def apply_A(phi):
    """(A phi) for a (Lz, Ly, Lx) field, phi = 0 outside the box."""
    out = 6.0 * phi
    out[1:, :, :] -= phi[:-1, :, :]
    out[:-1, :, :] -= phi[1:, :, :]
    out[:, 1:, :] -= phi[:, :-1, :]
    out[:, :-1, :] -= phi[:, 1:, :]
    out[:, :, 1:] -= phi[:, :, :-1]
    out[:, :, :-1] -= phi[:, :, 1:]
    return out


def laplacian_dense(L):
    """Dense A in natural x-fastest order, built site by site from H_L."""
    Lx, Ly, Lz = L
    n = Lx * Ly * Lz
    A = np.zeros((n, n))
    for z in range(Lz):
        for y in range(Ly):
            for x in range(Lx):
                i = x + Lx * (y + Ly * z)
                A[i, i] = 6.0
                for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    xx, yy, zz = x + dx, y + dy, z + dz
                    if 0 <= xx < Lx and 0 <= yy < Ly and 0 <= zz < Lz:
                        A[i, xx + Lx * (yy + Ly * zz)] = -1.0
    return A


def green_dense(L):
    """G = A^{-1} by Cholesky (library routine); for boxes up to ~16^3."""
    import scipy.linalg as sl
    A = laplacian_dense(L)
    c = sl.cho_factor(A)
    return sl.cho_solve(c, np.eye(A.shape[0]))


def axis_eigenvalues(n):
    """Eigenvalues 2 - 2 cos(pi k/(n+1)), k = 1..n, of the 1D Dirichlet -Delta."""
    k = np.arange(1, n + 1)
    return 2.0 - 2.0 * np.cos(np.pi * k / (n + 1))


def solve_dst(rho):
    """u = A^{-1} rho by the DST-I spectral solve (rho shape (Lz, Ly, Lx))."""
    import scipy.fft as sf
    Lz, Ly, Lx = rho.shape
    lam = (axis_eigenvalues(Lz)[:, None, None] + axis_eigenvalues(Ly)[None, :, None]
           + axis_eigenvalues(Lx)[None, None, :])
    R = sf.dstn(rho, type=1, workers=-1)
    return sf.idstn(R / lam, type=1, workers=-1)


def solve_cg(rho, rtol=1e-13, maxiter=100000):
    """u = A^{-1} rho by plain conjugate gradients (A is SPD)."""
    x = np.zeros_like(rho)
    r = rho.copy()
    p = r.copy()
    rr = float(np.vdot(r, r))
    stop = rtol * rtol * float(np.vdot(rho, rho))
    it = 0
    while rr > stop and it < maxiter:
        Ap = apply_A(p)
        alpha = rr / float(np.vdot(p, Ap))
        x += alpha * p
        r -= alpha * Ap
        rr_new = float(np.vdot(r, r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


# heat-kernel quadrature --------------------------------------------------
def _heat_nodes(L, h=0.02):
    """Nodes t_j = exp(s_j) and trapezoid weights for int_0^inf f(t) dt with
    f decaying like exp(-t * lambda_min); substitution t = e^s."""
    lam_min = sum(axis_eigenvalues(n)[0] for n in L)
    s_hi = math.log(60.0 / lam_min)
    s_lo = -36.0
    s = np.arange(s_lo, s_hi + h, h)
    t = np.exp(s)
    return t, h * t


def heat_kernel_table(n, t):
    """K(a, a; t_j) = sum_k s_k(a)^2 exp(-t_j lambda_k), shape (n, len(t))."""
    lam = axis_eigenvalues(n)
    a = np.arange(n)
    k = np.arange(1, n + 1)
    S2 = (2.0 / (n + 1)) * np.sin(np.pi * np.outer(a + 1, k) / (n + 1)) ** 2  # (a, k)
    return S2 @ np.exp(-np.outer(lam, t))


def heat_kernel_pair(n, a, b, t):
    """K(a, b; t_j) for index arrays a, b: shape (len(a), len(t))."""
    lam = axis_eigenvalues(n)
    k = np.arange(1, n + 1)
    sa = math.sqrt(2.0 / (n + 1)) * np.sin(np.pi * np.outer(np.asarray(a) + 1, k) / (n + 1))
    sb = math.sqrt(2.0 / (n + 1)) * np.sin(np.pi * np.outer(np.asarray(b) + 1, k) / (n + 1))
    return (sa * sb) @ np.exp(-np.outer(lam, t))


def green_diag(L, sites, chunk=4096):
    """G(r_i, r_i) for many sites by heat-kernel quadrature."""
    Lx, Ly, Lz = L
    s = np.asarray(sites, dtype=np.int64).reshape(-1, 3)
    t, w = _heat_nodes(L)
    Tx, Ty, Tz = heat_kernel_table(Lx, t), heat_kernel_table(Ly, t), heat_kernel_table(Lz, t)
    out = np.empty(len(s))
    for i0 in range(0, len(s), chunk):
        ss = s[i0:i0 + chunk]
        out[i0:i0 + chunk] = (Tx[ss[:, 0]] * Ty[ss[:, 1]] * Tz[ss[:, 2]]) @ w
    return out


def green_pairs(L, sa, sb):
    """G(a_i, b_i) for paired site arrays by heat-kernel quadrature."""
    Lx, Ly, Lz = L
    sa = np.asarray(sa, dtype=np.int64).reshape(-1, 3)
    sb = np.asarray(sb, dtype=np.int64).reshape(-1, 3)
    t, w = _heat_nodes(L)
    K = (heat_kernel_pair(Lx, sa[:, 0], sb[:, 0], t) * heat_kernel_pair(Ly, sa[:, 1], sb[:, 1], t)
         * heat_kernel_pair(Lz, sa[:, 2], sb[:, 2], t))
    return K @ w


def charge_density(L, sites, q):
    Lx, Ly, Lz = L
    rho = np.zeros((Lz, Ly, Lx))
    s = np.asarray(sites, dtype=np.int64).reshape(-1, 3)
    np.add.at(rho, (s[:, 2], s[:, 1], s[:, 0]), np.asarray(q, dtype=np.float64))
    return rho


def e_lat(L, sites, q, method="dst"):
    """E_lat = sum_{i != j} q_i q_j G(r_i, r_j) = rho^T G rho - sum_i q_i^2 G_ii.

    method: "dense" (G by Cholesky; small boxes), "dst" (spectral solve for
    G rho, heat-kernel quadrature for G_ii) or "cg" (CG for G rho, heat-kernel
    quadrature for G_ii)."""
    q = np.asarray(q, dtype=np.float64)
    s = np.asarray(sites, dtype=np.int64).reshape(-1, 3)
    if len(q) == 0:
        return 0.0
    if method == "dense":
        G = green_dense(L)
        idx = site_index(L, s)
        Gc = G[np.ix_(idx, idx)]
        return float(q @ Gc @ q - np.sum(q * q * np.diag(Gc)))
    rho = charge_density(L, s, q)
    if method == "dst":
        u = solve_dst(rho)
    elif method == "cg":
        u, _ = solve_cg(rho)
    else:
        raise ValueError(method)
    return float(np.vdot(rho, u) - np.sum(q * q * green_diag(L, s)))


def wick_variance(L, sites, q):
    """Var(e) = 2 tr(M G M G), M = q q^T - diag(q^2), over the charge sites
    (e = phi^T M phi with phi ~ N(0, G)).  Dense G; small boxes only."""
    G = green_dense(L)
    idx = site_index(L, sites)
    Gc = G[np.ix_(idx, idx)]
    q = np.asarray(q, dtype=np.float64)
    M = np.outer(q, q) - np.diag(q * q)
    MG = M @ Gc
    return float(2.0 * np.trace(MG @ MG))


# --------------------------------------------------------------------------
# Continuum and infinite-lattice references
# --------------------------------------------------------------------------
def coulomb_direct(sites, q):
    """Eq. (s1): (1/4 pi) sum over ordered pairs i != j of q_i q_j / |r_i - r_j|."""
    s = np.asarray(sites, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64)
    tot = 0.0
    for i in range(len(q)):
        d = np.sqrt(np.sum((s - s[i]) ** 2, axis=1))
        d[i] = np.inf
        tot += q[i] * np.sum(q / d)
    return tot / (4.0 * np.pi)


def green_infinite(r):
    """Infinite-lattice G(r) = int_0^inf prod_mu exp(-2t) I_{r_mu}(2t) dt."""
    from scipy.integrate import quad
    from scipy.special import ive
    r = [abs(int(v)) for v in r]

    def f(t):
        return ive(r[0], 2 * t) * ive(r[1], 2 * t) * ive(r[2], 2 * t)

    # finite part plus the tail, where prod ive ~ (4 pi t)^(-3/2) (1 + O(1/t))
    T = 2.0e4
    a, _ = quad(f, 0.0, T, limit=2000, epsabs=1e-15, epsrel=1e-13, points=[1, 10, 100, 1000])
    # tail: large-argument expansion ive(n, x) = (2 pi x)^(-1/2) (1 - (4n^2 - 1)/(8x) + ...)
    c = sum((4 * n * n - 1) / 16.0 for n in r)  # coefficient of 1/t in prod ive * (4 pi t)^{3/2}
    tail = (4 * np.pi) ** -1.5 * (2.0 / math.sqrt(T) - c * (2.0 / 3.0) * T ** -1.5)
    return a + tail


# --------------------------------------------------------------------------
# Error bars
# --------------------------------------------------------------------------
def batch_means(e, n_batches=32):
    """Mean and batch-means standard error of one chain's series e (the tail
    that does not fill a batch is dropped from the error, not from the mean)."""
    e = np.asarray(e, dtype=np.float64)
    n = len(e)
    b = n // n_batches
    mean = float(np.mean(e))
    if b == 0:
        return mean, float("nan")
    bm = e[: b * n_batches].reshape(n_batches, b).mean(axis=1)
    return mean, float(np.std(bm, ddof=1) / math.sqrt(n_batches))


def tau_int(e, c=6.0):
    """Integrated autocorrelation time with Sokal's automatic window
    (smallest W with W >= c * tau(W))."""
    e = np.asarray(e, dtype=np.float64)
    n = len(e)
    x = e - e.mean()
    f = np.fft.rfft(x, 2 * n)
    acf = np.fft.irfft(f * np.conj(f))[:n]
    acf /= acf[0]
    tau = 0.5
    for W in range(1, n):
        tau += acf[W]
        if W >= c * tau:
            break
    return float(tau)
