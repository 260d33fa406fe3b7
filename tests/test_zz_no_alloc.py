"""coulps_measure_static, the allocation-free measurement, against coulps_measure.

Callers that cannot allocate device memory when they measure (code running
during a CUDA stream capture, real-time controllers that forbid allocation
after start-up, plugins whose host application reserved all device memory)
pass their own field, charge and output buffers to coulps_measure_static; its
only working memory is a fixed device array inside the library.  This file
checks through the C ABI, on two calls in a row, that it returns the same
(Q, P, e) per chain as the allocating coulps_measure path, and that requests
beyond the fixed array are refused.  It is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64-mode tolerance of the parity tests; both paths sum in FP64


def _row_stride(Lx, precision):
    es = 4 if precision == 0 else 8
    w = 4 * ((Lx + 7) // 8)
    a = 32 // es
    return (w + a - 1) // a * a


def _storage(fields, L, precision):
    """Natural-order fields -> the library's [chain][colour][z][y][h] layout."""
    Lx, Ly, Lz = L
    W = _row_stride(Lx, precision)
    out = np.zeros((len(fields), 2, Lz, Ly, W), dtype=np.float32 if precision == 0 else np.float64)
    z, y, x = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    c = (x + y + z) & 1
    for k, f in enumerate(fields):
        out[k][c, z, y, x >> 1] = f
    return out.reshape(-1)


def _site_index(sites, L, precision):
    Lx, Ly, Lz = L
    W = _row_stride(Lx, precision)
    s = np.asarray(sites, dtype=np.int64)
    c = (s[:, 0] + s[:, 1] + s[:, 2]) & 1
    return (c * (Lz * Ly * W) + (s[:, 2] * Ly + s[:, 1]) * W + (s[:, 0] >> 1)).astype(np.uint32)


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_0711_gb300 import _build, coulps
    _build.build()
    lib = coulps.load()
    coulps.use_torch_allocator()
    return torch, coulps, lib, torch.cuda.Stream()


def _rel_err(got, ref):
    Q, P = ref[:, 0], ref[:, 1]
    den = np.where(Q * Q + P > 0, Q * Q + P, 1.0)
    return max(float((np.abs(got[:, 0] - Q) / np.sqrt(np.where(P > 0, P, 1.0))).max()),
               float((np.abs(got[:, 1:] - ref[:, 1:]) / den[:, None]).max()))


@pytest.mark.parametrize("precision,L,nc,n", [(0, (24, 19, 17), 5, 300), (1, (23, 16, 11), 3, 2500)])
def test_static_scratch_matches_measure(env, precision, L, nc, n):
    torch, coulps, lib, stream = env
    from paper_1403_0711_gb300 import inputs
    sites, q = inputs.uniform_q(L, n, seed=8)
    lat = coulps.Lattice(L, n_chains=nc, precision=precision, seed=4, stream=stream)
    ch = coulps.Charges(lat, sites, q, log_capacity=2)
    d_idx = torch.from_numpy(_site_index(sites, L, precision).view(np.int32)).cuda()
    d_q = torch.from_numpy(np.asarray(q, dtype=np.float64)).cuda()
    d_out = torch.empty(3 * nc, dtype=torch.float64, device="cuda")
    for call in range(2):
        lat.sweep(2, 1, 2)
        ch.measure()
        ref = ch.samples()[call]  # (nc, 3) from the allocating path
        d_field = torch.from_numpy(_storage([lat.field(k) for k in range(nc)], L, precision)).cuda()
        d_out.fill_(float("nan"))
        torch.cuda.synchronize()
        st = lib.coulps_measure_static(
            ctypes.c_void_p(d_field.data_ptr()), L[0], L[1], L[2], nc, precision,
            ctypes.c_void_p(d_idx.data_ptr()), ctypes.c_void_p(d_q.data_ptr()), n,
            ctypes.c_void_p(d_out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == coulps.OK, coulps.error_string(st)
        stream.synchronize()
        got = d_out.cpu().numpy().reshape(nc, 3)
        assert np.all(np.isfinite(got))
        assert _rel_err(got, ref) < TOL, call
    ch.close()
    lat.close()


def test_static_scratch_rejects_oversized_requests(env):
    torch, coulps, lib, stream = env
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    # 600 chains x 64 CTAs x 2 doubles > 65536: refused before any launch
    st = lib.coulps_measure_static(p, 8, 8, 8, 600, 0, p, p, 100000, p, None)
    assert st == coulps.EINVAL
    # a bad precision or a null output is refused
    assert lib.coulps_measure_static(p, 8, 8, 8, 4, 3, p, p, 10, p, None) == coulps.EINVAL
    assert lib.coulps_measure_static(p, 8, 8, 8, 4, 0, p, p, 10, None, None) == coulps.EINVAL
