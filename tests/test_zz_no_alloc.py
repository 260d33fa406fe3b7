"""coulps_measure_static, the allocation-free measurement, against coulps_measure
and the FP64 oracle.

Callers that cannot allocate device memory when they measure (code running
during a CUDA stream capture, real-time controllers that forbid allocation
after start-up, plugins whose host application reserved all device memory)
pass their own field, charge and output buffers to coulps_measure_static; its
only working memory is a fixed device array inside the library.  This file
checks through the C ABI, on two calls in a row, that it returns bitwise the
(Q, P, e) per chain of the allocating coulps_measure path and, to 1e-12, that
of the oracle's Eq. (nsum2) on the same fields; that a call captured into a
CUDA graph after a first call replays correctly; that the fixed array's limit
is exact; and that out-of-range offsets are not read.  It is collected last
on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64-mode tolerance of the parity tests; both sides sum in FP64


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


def _call(lib, d_field, L, nc, precision, d_idx, d_q, n, d_out, stream):
    return lib.coulps_measure_static(
        ctypes.c_void_p(d_field.data_ptr()), L[0], L[1], L[2], nc, precision,
        ctypes.c_void_p(d_idx.data_ptr()), ctypes.c_void_p(d_q.data_ptr()), n,
        ctypes.c_void_p(d_out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


def _rel_err(got, ref):
    Q, P = ref[:, 0], ref[:, 1]
    den = np.where(Q * Q + P > 0, Q * Q + P, 1.0)
    return max(float((np.abs(got[:, 0] - Q) / np.sqrt(np.where(P > 0, P, 1.0))).max()),
               float((np.abs(got[:, 1:] - ref[:, 1:]) / den[:, None]).max()))


@pytest.mark.parametrize("precision,L,nc,n", [(0, (24, 19, 17), 5, 300), (1, (23, 16, 11), 3, 2500),
                                              (0, (9, 8, 7), 4, 70000)])
def test_static_scratch_matches_measure_and_oracle(env, orc, precision, L, nc, n):
    torch, coulps, lib, stream = env
    from paper_1403_0711_gb300 import inputs
    if n > L[0] * L[1] * L[2]:  # more charges than sites: repeated sites (the math allows them)
        rng = np.random.default_rng(5)
        sites = np.stack([rng.integers(0, L[i], n) for i in range(3)], axis=1).astype(np.int32)
        q = rng.uniform(-1, 1, n)
    else:
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
        fields = [lat.field(k) for k in range(nc)]
        d_field = torch.from_numpy(_storage(fields, L, precision)).cuda()
        d_out.fill_(float("nan"))
        torch.cuda.synchronize()
        st = _call(lib, d_field, L, nc, precision, d_idx, d_q, n, d_out, stream)
        assert st == coulps.OK, coulps.error_string(st)
        stream.synchronize()
        got = d_out.cpu().numpy().reshape(nc, 3)
        assert np.all(np.isfinite(got))
        # the same CTA partials added in the same order as coulps_measure
        assert np.array_equal(got, ref), call
        # the oracle's Eq. (nsum2) on the same fields (FP64, another order)
        orc_ref = np.stack([orc.measure(fields[k], sites, q) for k in range(nc)])
        assert _rel_err(got, orc_ref) < TOL, call
    ch.close()
    lat.close()


def test_static_scratch_in_a_captured_graph(env):
    """The call such callers make: a first call on the device (it looks up the
    array's address), then the call captured into a CUDA graph on a side
    stream and replayed twice on new fields."""
    torch, coulps, lib, stream = env
    from paper_1403_0711_gb300 import inputs
    L, nc, precision = (20, 17, 13), 4, 0
    sites, q = inputs.uniform_q(L, 500, seed=9)
    lat = coulps.Lattice(L, n_chains=nc, precision=precision, seed=6, stream=stream)
    ch = coulps.Charges(lat, sites, q, log_capacity=3)
    d_idx = torch.from_numpy(_site_index(sites, L, precision).view(np.int32)).cuda()
    d_q = torch.from_numpy(np.asarray(q, dtype=np.float64)).cuda()
    d_out = torch.empty(3 * nc, dtype=torch.float64, device="cuda")
    lat.sweep(1, 1, 1)
    d_field = torch.from_numpy(_storage([lat.field(k) for k in range(nc)], L, precision)).cuda()
    torch.cuda.synchronize()
    assert _call(lib, d_field, L, nc, precision, d_idx, d_q, 500, d_out, stream) == coulps.OK
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        st = _call(lib, d_field, L, nc, precision, d_idx, d_q, 500, d_out, side)
    assert st == coulps.OK
    for r in range(2):
        lat.sweep(2, 1, 2)
        ch.measure()
        ref = ch.samples()[r]
        d_field.copy_(torch.from_numpy(_storage([lat.field(k) for k in range(nc)], L, precision)))
        d_out.fill_(float("nan"))
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(d_out.cpu().numpy().reshape(nc, 3), ref), r
    ch.close()
    lat.close()


def test_static_scratch_limit_is_exact(env):
    """n > 65536 charges: 64 CTAs per chain; 512 chains fill the 65536-double
    array exactly and are accepted, 513 are refused before any launch."""
    torch, coulps, lib, stream = env
    L, precision, n = (2, 2, 2), 0, 65537
    chain_elems = 2 * 2 * 2 * _row_stride(2, precision)
    field = torch.zeros(513 * chain_elems, dtype=torch.float32, device="cuda")
    idx = torch.zeros(n, dtype=torch.int32, device="cuda")
    q = torch.ones(n, dtype=torch.float64, device="cuda")
    out = torch.full((3 * 513,), float("nan"), dtype=torch.float64, device="cuda")
    assert _call(lib, field, L, 512, precision, idx, q, n, out, stream) == coulps.OK
    stream.synchronize()
    assert np.all(out.cpu().numpy()[:3 * 512] == 0.0)
    assert _call(lib, field, L, 513, precision, idx, q, n, out, stream) == coulps.EINVAL


def test_static_scratch_skips_out_of_range_offsets(env):
    torch, coulps, lib, stream = env
    L, precision, nc = (8, 8, 8), 0, 3
    chain_elems = 2 * 8 * 8 * _row_stride(8, precision)
    field = torch.ones(nc * chain_elems, dtype=torch.float32, device="cuda")
    q = torch.ones(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(3 * nc, dtype=torch.float64, device="cuda")
    good = torch.tensor([0, 1, 2, chain_elems - 1], dtype=torch.int32, device="cuda")
    assert _call(lib, field, L, nc, precision, good, q, 4, out, stream) == coulps.OK
    stream.synchronize()
    assert np.allclose(out.cpu().numpy().reshape(nc, 3)[:, :2], [[4.0, 4.0]] * nc)
    bad = torch.tensor([0, 1, chain_elems, 2], dtype=torch.int32, device="cuda")
    assert _call(lib, field, L, nc, precision, bad, q, 4, out, stream) == coulps.OK
    stream.synchronize()
    assert np.all(np.isnan(out.cpu().numpy()))
    # the next valid call is not affected (the counter is cleared per call)
    assert _call(lib, field, L, nc, precision, good, q, 4, out, stream) == coulps.OK
    stream.synchronize()
    assert np.all(np.isfinite(out.cpu().numpy()))


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
