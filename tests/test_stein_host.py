"""The control variate's divergence formulation (host logic of stein.py):
one extra conv with K = W2 * (W3 x W1) plus the face-site corrections equals the
oracle's plain chain-rule divergence.  Convolutions here are PyTorch FP64
conv3d on the CPU; the GPU tests run the same formulation on the tensor cores."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


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
    p = ost.random_params(7, scale=0.5)
    exact = ost.divergence(phi, rho, p)

    cv = stein.SteinCV(device="cpu")
    _load(cv, p)
    F = torch.nn.functional
    psi = torch.from_numpy(np.stack([phi, rho]))[None]
    h1 = F.conv3d(psi, cv.W1, cv.b1, padding=1)
    s1 = 1 - torch.tanh(h1) ** 2
    h2 = F.conv3d(torch.tanh(h1), cv.W2, cv.b2, padding=1)
    s2 = 1 - torch.tanh(h2) ** 2
    K = stein.divergence_kernel(cv.W1, cv.W2, cv.W3)
    D = F.conv3d(s1, K, padding=1)
    main = (s2 * D).sum()
    face = cv._face_term(s1.permute(0, 2, 3, 4, 1), s2.permute(0, 2, 3, 4, 1))[0]
    got = float(main + face)
    assert abs(got - exact) < 1e-10 * max(1.0, abs(exact)), (got, exact)
    # the g path agrees too
    g = F.conv3d(torch.tanh(h2), cv.W3, cv.b3, padding=1)[0, 0].detach().numpy()
    assert np.abs(g - ost.forward(phi, rho, p)["g"]).max() < 1e-12
