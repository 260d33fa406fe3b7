"""Global control variate g = Q h (coulps_gcv_*): the SOR solution h against
the oracle's spectral solve of A h = -rho, the per-chain Stein term against
the oracle's formula with the same h, zero mean under the sampler, and the
variance it removes from the +-1 estimator."""
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


@pytest.mark.parametrize("R", [0, 1, 2])
def test_h_and_stein_term_match_oracle(cl, stream, R):
    import torch
    from oracle import oracle as O
    from oracle import stein as ost
    from paper_1403_0711_gb300 import inputs
    L = (23, 18, 15)
    sites, q = inputs.uniform_q(L, 30, seed=4)
    lat = cl.Lattice(L, n_chains=3, precision=cl.F32, seed=8, stream=stream)
    ch = cl.Charges(lat, sites, q, log_capacity=4)
    fields = inputs.gaussian_fields(L, 3, seed=9)
    for k, f in enumerate(fields):
        lat.set_field(k, f)
    g = cl.GlobalCV(ch, n_iter=400, R=R)
    info = g.info()
    assert info["residual"] < 1e-9
    rho = O.charge_density(L, sites, q)
    u = O.solve_dst(rho)  # A^-1 rho
    h = g.h().astype(np.float64)
    assert np.abs(h + u).max() < 1e-6 * np.abs(u).max()
    assert abs(info["h_dot_rho"] - float(np.sum(h * rho))) < 1e-12 * abs(info["h_dot_rho"])
    tg = torch.zeros(3, dtype=torch.float64, device="cuda")
    g.eval(tg.data_ptr())
    lat.sync()
    tg = tg.cpu().numpy()
    # the library keeps the local term's kernel in FP32 (any kernel gives a
    # mean-zero term): compare with the oracle's kernel rounded the same way
    kc = ost.cube_green(R).astype(np.float32).astype(np.float64) if R > 0 else None
    for k in range(3):
        phi = fields[k].astype(np.float32).astype(np.float64)  # as stored (FP32 lattice)
        ref = ost.global_stein_term(phi, rho, h)
        if R > 0:
            ref += ost.local_p_stein_term(phi, sites, q, kc)
        Q = float(np.sum(rho * phi))
        scale = abs(info["h_dot_rho"]) + abs(Q) * float(np.abs(ost.apply_A(h) * phi).sum())
        if R > 0:
            scale += _p_scale(phi, sites, q, kc)
        # v . phi: FP32 partial sums of 16 products, FP64 across them; the local
        # term of P evaluated in FP32 with k in FP32
        assert abs(tg[k] - ref) < 1e-6 * scale, (k, tg[k], ref)
    g.close()
    ch.close()
    lat.close()


def test_gcv_unbiased_and_removes_the_far_pair_variance(cl, stream):
    from oracle import oracle as O
    from paper_1403_0711_gb300 import inputs
    L = (32, 32, 32)
    sites, q = inputs.plus_minus(L, 64, seed=6)
    e_lat = O.e_lat(L, sites, q, "dst")
    lat = cl.Lattice(L, n_chains=64, precision=cl.F32, seed=10, stream=stream)
    ch = cl.Charges(lat, sites, q)
    lat.sweep(200, 1, 3)
    g = cl.GlobalCV(ch, R=0)  # the Q term alone first
    ch.reset_stats()
    ch.cv_reset()
    g.run(1500, 1, 3, 1.0)
    plain, cvst = ch.chain_stats(), ch.cv_chain_stats()
    n = plain[:, 0].sum()
    var_p = plain[:, 2].sum() / n - (plain[:, 1].sum() / n) ** 2
    var_c = cvst[:, 2].sum() / n - (cvst[:, 1].sum() / n) ** 2
    assert var_c < 0.05 * var_p, (var_c, var_p)
    a, b = ch.estimate(), ch.cv_estimate()
    assert abs(b["mean"] - e_lat) < 4 * b["stderr"], (b, e_lat)
    assert abs(a["mean"] - e_lat) < 4 * a["stderr"], (a, e_lat)
    # per-chain means of T g (c = 1): e - y, zero within errors
    tg_chain = (plain[:, 1] - cvst[:, 1]) / plain[:, 0]
    assert abs(tg_chain.mean()) < 4 * tg_chain.std(ddof=1) / math.sqrt(len(tg_chain))
    g.close()
    # with the local term of P the variance drops much further, still unbiased
    g = cl.GlobalCV(ch, R=2)
    ch.reset_stats()
    ch.cv_reset()
    g.run(1500, 1, 3, 1.0)
    plain, cvst = ch.chain_stats(), ch.cv_chain_stats()
    n = plain[:, 0].sum()
    var_p = plain[:, 2].sum() / n - (plain[:, 1].sum() / n) ** 2
    var_c2 = cvst[:, 2].sum() / n - (cvst[:, 1].sum() / n) ** 2
    assert var_c2 < 0.2 * var_c and var_c2 < 0.005 * var_p, (var_c2, var_c, var_p)
    b = ch.cv_estimate()
    assert abs(b["mean"] - e_lat) < 4 * b["stderr"], (b, e_lat)
    tg_chain = (plain[:, 1] - cvst[:, 1]) / plain[:, 0]
    assert abs(tg_chain.mean()) < 4 * tg_chain.std(ddof=1) / math.sqrt(len(tg_chain))
    g.close()
    ch.close()
    lat.close()
