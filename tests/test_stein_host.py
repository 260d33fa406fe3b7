"""The control variate's divergence formulation (host logic of stein.py):
one extra conv with K = W2 * (W3 x W1) plus the face-site corrections plus the
charge-site term of the rho phi channel equals the oracle's plain chain-rule
divergence.  Convolutions here are PyTorch FP64
conv3d on the CPU; the GPU tests run the same formulation on the tensor cores."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _bf16(p):
    """Weights rounded to BF16 values (the net's divergence uses the rounded
    weights the tensor-core convs see, so the oracle gets the same ones)."""
    p = dict(p)
    for k in ("W1", "W2", "W3"):
        p[k] = torch.from_numpy(p[k]).to(torch.bfloat16).double().numpy()
    return p


def _load(cv, p):
    with torch.no_grad():
        for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
            getattr(cv, k).data = torch.from_numpy(p[k]).double()


@pytest.mark.parametrize("shape", [(5, 4, 3), (1, 3, 4), (2, 2, 2), (6, 1, 5)])
def test_k_trick_with_face_corrections_equals_chain_rule(shape):
    from oracle import stein as ost
    from paper_1403_0711_gb300 import stein
    Z, Y, X = shape
    rng = np.random.default_rng(sum(shape))
    phi = rng.standard_normal((Z, Y, X))
    rho = np.zeros((Z, Y, X))
    rho.flat[rng.integers(0, Z * Y * X, 3)] = [1.0, -1.0, 0.5]
    p = _bf16(ost.random_params(7, scale=0.5))
    exact = ost.divergence(phi, rho, p)

    cv = stein.SteinCV(device="cpu")
    _load(cv, p)
    cv.set_density(torch.from_numpy(rho))
    F = torch.nn.functional
    psi = torch.from_numpy(np.stack([phi, rho, rho * phi]))[None]
    h1 = F.conv3d(psi, cv.W1, cv.b1, padding=1)
    s1 = 1 - torch.tanh(h1) ** 2
    h2 = F.conv3d(torch.tanh(h1), cv.W2, cv.b2, padding=1)
    s2 = 1 - torch.tanh(h2) ** 2
    K = stein.divergence_kernel(cv.W1, cv.W2, cv.W3)
    D = F.conv3d(s1, K, padding=1)
    main = (s2 * D).sum()
    s1c, s2c = s1.permute(0, 2, 3, 4, 1), s2.permute(0, 2, 3, 4, 1)
    face = cv._face_term(s1c, s2c)[0]
    charge = stein.charge_term(stein.charge_matrix(cv.W1, cv.W2, cv.W3), s1c, s2c, cv._cq,
                               cv._crho.double())[0]
    got = float(main + face + charge)
    assert abs(got - exact) < 1e-10 * max(1.0, abs(exact)), (got, exact)
    # the g path agrees too
    g = F.conv3d(torch.tanh(h2), cv.W3, cv.b3, padding=1)[0, 0].detach().numpy()
    assert np.abs(g - ost.forward(phi, rho, p)["g"]).max() < 1e-12


@pytest.mark.parametrize("L,lo,hi", [
    ((10, 8, 9), (3, 2, 3), (6, 5, 5)),     # interior region, E clipped on y and z
    ((12, 11, 10), (4, 4, 4), (8, 7, 6)),   # E strictly inside the lattice
    ((7, 6, 5), (0, 0, 2), (3, 6, 3)),      # region on the lattice faces, one-site-thick in z
])
def test_region_divergence_on_sub_box_equals_oracle(L, lo, hi):
    """LocalSteinCV's per-class kernels on the sub-box E = R + 3 give the
    oracle's region-restricted Stein term of the net on the whole lattice."""
    from oracle import stein as ost
    from paper_1403_0711_gb300 import stein
    X, Y, Z = L
    rng = np.random.default_rng(X * Y * Z)
    phi = rng.standard_normal((Z, Y, X))
    rho = np.zeros((Z, Y, X))
    rho.flat[rng.integers(0, Z * Y * X, 4)] = [1.0, -1.0, 0.5, 1.0]
    rho[lo[2], lo[1], lo[0]] = 0.75  # a charge inside R on its corner
    p = _bf16(ost.random_params(3, scale=0.5))
    region = ((lo[2], hi[2]), (lo[1], hi[1]), (lo[0], hi[0]))
    exact = ost.stein_term(phi, rho, p, region)

    cv = stein.LocalSteinCV(L, lo, hi, device="cpu")
    _load(cv, p)
    cv.set_density(torch.from_numpy(rho))
    (x0, y0, z0), (x1, y1, z1) = cv.e_lo, cv.e_hi
    F = torch.nn.functional
    psi = torch.from_numpy(np.stack([phi, rho, rho * phi])[:, z0:z1, y0:y1, x0:x1])[None]
    h1 = F.conv3d(psi, cv.W1, cv.b1, padding=1)
    s1 = 1 - torch.tanh(h1) ** 2
    h2 = F.conv3d(torch.tanh(h1), cv.W2, cv.b2, padding=1)
    s2 = 1 - torch.tanh(h2) ** 2
    g = F.conv3d(torch.tanh(h2), cv.W3, cv.b3, padding=1)[0, 0]
    s1c, s2c = s1.permute(0, 2, 3, 4, 1), s2.permute(0, 2, 3, 4, 1)
    div = cv.region_divergence(s1c, s2c)[0] + stein.charge_term(
        stein.charge_matrix(cv.W1, cv.W2, cv.W3), s1c, s2c, cv._cq, cv._crho.double())[0]
    Aphi = torch.from_numpy(ost.apply_A(phi)[z0:z1, y0:y1, x0:x1])
    got = float(div - (g * Aphi * cv._rmask.double()).sum())
    assert abs(got - exact) < 1e-10 * max(1.0, abs(exact)), (got, exact)
    assert cv._cq.shape[0] >= 1
    # every q next to R is covered exactly once, none beyond R + 1
    m = cv._q.shape[0]
    nr = [min(b + 1, e) - max(a - 1, 0) for a, b, e in zip(cv.r_lo, cv.r_hi, cv.edims)]
    assert m == nr[0] * nr[1] * nr[2]
