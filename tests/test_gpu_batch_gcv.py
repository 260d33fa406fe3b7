"""Global control variate of every system of a batch (coulps_batch_gcv_*):
each system's SOR solution h against the oracle's spectral solve of
A h = -rho, each system's Stein term against oracle/stein.py's
global_stein_term (+ local_p_stein_term) with the same h, h bitwise that of
the single-lattice control variate for the same box, and zero mean plus the
variance removed under the batched sampler."""
import math

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


def _p_scale(phi, sites, q, k):
    """Magnitude against which FP32 evaluation of the local P term rounds:
    sum_i q_i^2 |phi_i| sum_d |k(d)| (6 |phi| + sum of |phi| at the six
    neighbours)(r_i + d)."""
    R = (k.shape[0] - 1) // 2
    a = np.abs(phi)
    pad = np.pad(a, 1)
    Aabs = (6 * a + pad[1:-1, 1:-1, :-2] + pad[1:-1, 1:-1, 2:] + pad[1:-1, :-2, 1:-1] +
            pad[1:-1, 2:, 1:-1] + pad[:-2, 1:-1, 1:-1] + pad[2:, 1:-1, 1:-1])
    Lz, Ly, Lx = phi.shape
    tot = 0.0
    for (x, y, z), qi in zip(np.asarray(sites).reshape(-1, 3), np.asarray(q, dtype=np.float64)):
        z0, z1 = max(z - R, 0), min(z + R + 1, Lz)
        y0, y1 = max(y - R, 0), min(y + R + 1, Ly)
        x0, x1 = max(x - R, 0), min(x + R + 1, Lx)
        kk = np.abs(k[z0 - z + R:z1 - z + R, y0 - y + R:y1 - y + R, x0 - x + R:x1 - x + R])
        tot += qi * qi * a[z, y, x] * float(np.sum(kk * Aabs[z0:z1, y0:y1, x0:x1]))
    return tot


DIMS = [(23, 18, 15), (13, 7, 5), (16, 16, 16), (9, 11, 17), (1, 1, 1), (30, 4, 6)]


@pytest.mark.parametrize("prec,R", [(0, 0), (0, 1), (0, 2), (1, 1)])
def test_h_and_stein_terms_match_oracle(cl, stream, prec, R):
    import torch
    from oracle import oracle as O
    from oracle import stein as ost
    from paper_1403_0711_gb300 import inputs
    systems = [inputs.uniform_q(L, min(30, L[0] * L[1] * L[2]), seed=4 + k)
               for k, L in enumerate(DIMS)]
    b = cl.Batch(DIMS, precision=prec, seed=8, stream=stream)
    b.set_charges(systems)
    fields = [inputs.gaussian_fields(L, 1, seed=9 + k)[0] for k, L in enumerate(DIMS)]
    for k, f in enumerate(fields):
        b.set_field(k, f)
    g = cl.BatchGlobalCV(b, n_iter=400, R=R)
    info = g.info()
    tg = torch.zeros(len(DIMS), dtype=torch.float64, device="cuda")
    g.eval(tg.data_ptr())
    b.sync()
    tg = tg.cpu().numpy()
    # the library keeps the local term's kernel in FP32 (any kernel gives a
    # mean-zero term): compare with the oracle's kernel rounded the same way
    kc = ost.cube_green(R).astype(np.float32).astype(np.float64) if R > 0 else None
    for k, L in enumerate(DIMS):
        sites, q = systems[k]
        rho = O.charge_density(L, sites, q)
        h = g.h(k).astype(np.float64)
        assert info["residual"][k] < 1e-9, (k, info["residual"][k])
        u = O.solve_dst(rho)  # A^-1 rho
        assert np.abs(h + u).max() <= 1e-6 * np.abs(u).max(), k
        assert abs(info["h_dot_rho"][k] - float(np.sum(h * rho))) <= 1e-12 * abs(info["h_dot_rho"][k])
        phi = fields[k].astype(np.float32).astype(np.float64) if prec == 0 else fields[k]
        ref = ost.global_stein_term(phi, rho, h)
        if R > 0:
            ref += ost.local_p_stein_term(phi, sites, q, kc)
        Q = float(np.sum(rho * phi))
        scale = abs(info["h_dot_rho"][k]) + abs(Q) * float(np.abs(ost.apply_A(h) * phi).sum())
        if R > 0:
            scale += _p_scale(phi, sites, q, kc)
        # FP32: v . phi sums 16 FP32 products in FP32 (as the lattice's) and the
        # local term is evaluated in FP32; FP64 fields: FP64 throughout
        tol = 1e-6 if prec == 0 else 1e-12
        assert abs(tg[k] - ref) <= tol * scale + 1e-300, (k, tg[k], ref)
    g.close()
    b.close()


def test_h_is_the_single_lattice_one(cl, stream):
    from paper_1403_0711_gb300 import inputs
    L = (20, 14, 11)
    sites, q = inputs.uniform_q(L, 25, seed=12)
    b = cl.Batch([(8, 8, 8), L], precision=0, seed=1, stream=stream)
    b.set_charges([inputs.uniform_q((8, 8, 8), 5, seed=13), (sites, q)])
    gb = cl.BatchGlobalCV(b, n_iter=137, R=1)
    lat = cl.Lattice(L, n_chains=1, precision=0, seed=1, stream=stream)
    ch = cl.Charges(lat, sites, q)
    gl = cl.GlobalCV(ch, n_iter=137, R=1)
    assert np.array_equal(gb.h(1), gl.h())
    # h . rho: the same terms, added in another order
    a, c = gb.info()["h_dot_rho"][1], gl.info()["h_dot_rho"]
    assert abs(a - c) <= 1e-14 * abs(c), (a, c)
    for x in (gl, ch, lat, gb, b):
        x.close()


def _pooled(st):
    """mean over systems of the per-system sample means, and the variance of
    all samples pooled (every system has the same number of samples)."""
    n = st[:, 0].sum()
    mean = st[:, 1].sum() / n
    return mean, st[:, 2].sum() / n - mean ** 2


def test_batch_gcv_unbiased_and_removes_variance(cl, stream):
    from oracle import oracle as O
    from paper_1403_0711_gb300 import inputs
    L = (16, 16, 16)
    n_sys = 32
    sites, q = inputs.plus_minus(L, 32, seed=6)
    e_lat = O.e_lat(L, sites, q, "dst")
    b = cl.Batch([L] * n_sys, precision=0, seed=10, stream=stream)
    b.set_charges([(sites, q)] * n_sys)
    b.sweep(200, 1, 3)
    out = {}
    for R in (0, 2):
        g = cl.BatchGlobalCV(b, R=R)
        b.reset_stats()
        g.reset()
        g.run(1500, 1, 3, 1.0)
        plain, cvst = b.stats(), g.stats()
        assert np.all(plain[:, 0] == 1500) and np.all(cvst[:, 0] == 1500)
        _, var_p = _pooled(plain)
        _, var_c = _pooled(cvst)
        out[R] = (var_p, var_c)
        est = g.estimate()
        m = est["mean"].mean()
        se = math.sqrt(float(np.sum(est["stderr"] ** 2))) / n_sys
        assert abs(m - e_lat) < 4 * se, (R, m, se, e_lat)
        pe = b.estimate()
        mp = pe["mean"].mean()
        sep = math.sqrt(float(np.sum(pe["stderr"] ** 2))) / n_sys
        assert abs(mp - e_lat) < 4 * sep, (R, mp, sep, e_lat)
        # per-system means of T g (c = 1): e - y, zero within errors
        tg_sys = (plain[:, 1] - cvst[:, 1]) / plain[:, 0]
        assert abs(tg_sys.mean()) < 4 * tg_sys.std(ddof=1) / math.sqrt(n_sys)
        g.close()
    assert out[0][1] < 0.05 * out[0][0], out
    assert out[2][1] < 0.2 * out[0][1] and out[2][1] < 0.005 * out[2][0], out
    b.close()
