"""The tcgen05 BF16 3x3x3 convolution (16 -> 16 channels, FP32 accumulate)
against a plain PyTorch FP32 conv3d of the same BF16-rounded operands."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_0711_gb300 import _build, coulps
    _build.build()
    lib = coulps.load()
    return torch, coulps, lib


def _pack(lib, w):
    w = np.ascontiguousarray(w, dtype=np.float32)
    out = np.zeros(27 * 256, dtype=np.uint16)
    assert lib.coulps_cv_pack_weights(w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16))) == 0
    return out


@pytest.mark.parametrize("shape", [(2, 5, 4, 128), (1, 3, 7, 37), (2, 4, 3, 130), (1, 1, 1, 1),
                                   (1, 6, 5, 300)])
def test_conv3d_matches_torch(env, shape):
    torch, coulps, lib = env
    nb, Lz, Ly, Lx = shape
    g = torch.Generator().manual_seed(sum(shape))
    a = torch.randn(nb, Lz, Ly, Lx, 16, generator=g).to(torch.bfloat16)
    w = (torch.randn(16, 16, 3, 3, 3, generator=g) * 0.2).to(torch.bfloat16).float()
    bias = torch.randn(16, generator=g)
    ref = torch.nn.functional.conv3d(a.float().permute(0, 4, 1, 2, 3), w, bias, padding=1)
    ref = ref.permute(0, 2, 3, 4, 1).contiguous()
    wp = torch.from_numpy(_pack(lib, w.numpy()).view(np.int16)).cuda()
    d_a = a.cuda().contiguous()
    d_b = bias.cuda()
    out = torch.full((nb, Lz, Ly, Lx, 16), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = lib.coulps_cv_conv3d(ctypes.c_void_p(d_a.data_ptr()), ctypes.c_void_p(wp.data_ptr()),
                              ctypes.c_void_p(d_b.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                              nb, Lx, Ly, Lz, 0, ctypes.c_void_p(err.data_ptr()), None)
    assert st == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    got = out.cpu()
    scale = (a.float().abs().max() * w.abs().sum(dim=(1, 2, 3, 4)).max()).item()
    assert torch.isfinite(got).all()
    assert (got - ref).abs().max().item() < 2e-6 * scale + 1e-6


def test_conv3d_tanh_epilogue(env):
    torch, coulps, lib = env
    nb, Lz, Ly, Lx = 2, 6, 5, 130
    g = torch.Generator().manual_seed(11)
    a = torch.randn(nb, Lz, Ly, Lx, 16, generator=g).to(torch.bfloat16)
    w = (torch.randn(16, 16, 3, 3, 3, generator=g) * 0.1).to(torch.bfloat16).float()
    bias = torch.randn(16, generator=g) * 0.2
    h = torch.nn.functional.conv3d(a.float().permute(0, 4, 1, 2, 3), w, bias, padding=1)
    t = torch.tanh(h.permute(0, 2, 3, 4, 1))
    wp = torch.from_numpy(_pack(lib, w.numpy()).view(np.int16)).cuda()
    d_a, d_b = a.cuda().contiguous(), bias.cuda()
    act = torch.empty(nb, Lz, Ly, Lx, 16, dtype=torch.bfloat16, device="cuda")
    der = torch.empty_like(act)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = lib.coulps_cv_conv3d_tanh(ctypes.c_void_p(d_a.data_ptr()), ctypes.c_void_p(wp.data_ptr()),
                                   ctypes.c_void_p(d_b.data_ptr()), ctypes.c_void_p(act.data_ptr()),
                                   ctypes.c_void_p(der.data_ptr()), nb, Lx, Ly, Lz, 0,
                                   ctypes.c_void_p(err.data_ptr()), None)
    assert st == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    # BF16 outputs: 2^-8 relative
    assert (act.float().cpu() - t).abs().max().item() < 8e-3
    assert (der.float().cpu() - (1 - t * t)).abs().max().item() < 8e-3


def test_interleaved_boxes_equal_separate_boxes(env):
    """Boxes side by side along x with one zero column after each, convolved
    as one lattice with x_period = box width + 1 (gutters re-zeroed in the
    epilogue), give each box's own zero-padded convolution; two layers in a
    row keep the gutters at 0."""
    torch, coulps, lib = env
    nb, Lz, Ly, ex = 11, 7, 9, 14
    P = ex + 1
    g = torch.Generator().manual_seed(5)
    a = torch.randn(nb, Lz, Ly, ex, 16, generator=g).to(torch.bfloat16)
    w = (torch.randn(16, 16, 3, 3, 3, generator=g) * 0.1).to(torch.bfloat16).float()
    bias = torch.randn(16, generator=g) * 0.2
    F = torch.nn.functional
    h = F.conv3d(a.float().permute(0, 4, 1, 2, 3), w, bias, padding=1)
    t1 = torch.tanh(h).to(torch.bfloat16).float()
    h2 = F.conv3d(t1, w, bias, padding=1).permute(0, 2, 3, 4, 1)  # (nb, Lz, Ly, ex, 16)
    # interleave: [z][y][b][x + gutter]
    inter = torch.zeros(Lz, Ly, nb, P, 16, dtype=torch.bfloat16)
    inter[:, :, :, :ex] = a.permute(1, 2, 0, 3, 4)
    d_in = inter.reshape(1, Lz, Ly, nb * P, 16).cuda().contiguous()
    wp = torch.from_numpy(_pack(lib, w.numpy()).view(np.int16)).cuda()
    d_b = bias.cuda()
    act = torch.full_like(d_in, float("nan"))
    der = torch.empty_like(d_in)
    out = torch.full((1, Lz, Ly, nb * P, 16), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    assert lib.coulps_cv_conv3d_tanh(vp(d_in), vp(wp), vp(d_b), vp(act), vp(der), 1, nb * P, Ly, Lz,
                                     P, vp(err), None) == 0
    assert lib.coulps_cv_conv3d(vp(act), vp(wp), vp(d_b), vp(out), 1, nb * P, Ly, Lz, P, vp(err),
                                None) == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    A = act.cpu().reshape(Lz, Ly, nb, P, 16)
    assert not A[:, :, :, ex].float().abs().any()  # gutters stay 0
    got = out.cpu().reshape(Lz, Ly, nb, P, 16)[:, :, :, :ex].permute(2, 0, 1, 3, 4)
    assert not out.cpu().reshape(Lz, Ly, nb, P, 16)[:, :, :, ex].abs().any()
    # the second layer saw BF16 tanh values equal to t1 up to tanh rounding
    assert (A[:, :, :, :ex].permute(2, 0, 1, 3, 4).float() - t1.permute(0, 2, 3, 4, 1)).abs().max() < 8e-3
    scale = float(w.abs().sum(dim=(1, 2, 3, 4)).max())
    assert (got - h2).abs().max().item() < 1e-2 * scale
