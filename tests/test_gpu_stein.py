"""The learned Stein control variate on the GPU.

- Library-kernel evaluation = autograd path = FP64 oracle (BF16 tolerance).
- The tensor-core conv's autograd gradients = PyTorch FP32 conv3d gradients
  of the same BF16 operands.
- The Stein term has zero mean under the library's own sampler.
- Training lowers the loss and the fitted estimator keeps the plain mean.
"""
import math

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
    coulps.load()
    coulps.use_torch_allocator()
    return torch, coulps, torch.cuda.Stream()


def test_evaluate_matches_autograd_path_and_oracle(env):
    torch, coulps, stream = env
    from oracle import stein as ost
    from paper_1403_0711_gb300 import inputs, stein
    L = (20, 12, 9)
    sites, q = inputs.uniform_q(L, 12, seed=3)
    lat = coulps.Lattice(L, n_chains=3, precision=coulps.F32, seed=5, stream=stream)
    lat.sweep(20, 1, 1)
    rho = stein.charge_density(L, sites, q)
    cv = stein.SteinCV(seed=2, scale=0.6, w3_scale=0.1)
    tg_eval = cv.evaluate(lat, rho).cpu().numpy()
    phis, Aphis = stein.pack_inputs(lat, rho)
    with torch.no_grad():
        tg_grad = cv.stein_term(stein.inputs_from(phis, rho), Aphis).double().cpu().numpy()
    p = {k: getattr(cv, k).detach().double().cpu().numpy() for k in ("W1", "b1", "W2", "b2", "W3", "b3")}
    r = rho.cpu().numpy().astype(np.float64)
    for k in range(3):
        phi = lat.field(k)
        div = ost.divergence(phi, r, p)
        gA = float(np.sum(ost.forward(phi, r, p)["g"] * ost.apply_A(phi)))
        scale = abs(div) + abs(gA)
        assert abs(tg_eval[k] - (div - gA)) < 3e-2 * scale, (k, tg_eval[k], div - gA, scale)
        assert abs(tg_grad[k] - tg_eval[k]) < 1e-2 * scale, (k, tg_grad[k], tg_eval[k])
    lat.close()


def test_conv_autograd_matches_torch(env):
    torch, coulps, stream = env
    from paper_1403_0711_gb300 import stein
    g = torch.Generator().manual_seed(0)
    a = torch.randn(2, 5, 6, 37, 16, generator=g).to(torch.bfloat16).cuda()
    W = (torch.randn(16, 16, 3, 3, 3, generator=g) * 0.2).to(torch.bfloat16).float().cuda()
    b = torch.randn(16, generator=g).cuda()
    R = torch.randn(2, 5, 6, 37, 16, generator=g).cuda()
    a1, W1, b1 = a.clone().requires_grad_(), W.clone().requires_grad_(), b.clone().requires_grad_()
    (stein.Conv3dTC.apply(a1, W1, b1) * R).sum().backward()
    a2 = a.float().clone().requires_grad_()
    W2, b2 = W.clone().requires_grad_(), b.clone().requires_grad_()
    h = torch.nn.functional.conv3d(a2.permute(0, 4, 1, 2, 3), W2, b2, padding=1).permute(0, 2, 3, 4, 1)
    (h * R).sum().backward()

    def rel(x, y):
        return float((x.float() - y.float()).abs().max() / y.float().abs().max())

    assert rel(b1.grad, b2.grad) < 1e-5
    assert rel(W1.grad, W2.grad) < 1e-2  # dh rounded to BF16 in the backward
    assert rel(a1.grad, a2.grad) < 1e-2


def test_stein_term_has_zero_mean_under_sampler(env):
    torch, coulps, stream = env
    from paper_1403_0711_gb300 import inputs, stein
    L = (6, 6, 6)
    sites, q = inputs.cube(L, 2)
    lat = coulps.Lattice(L, n_chains=512, precision=coulps.F32, seed=77, stream=stream)
    lat.sweep(200, 1, 0)
    rho = stein.charge_density(L, sites, q)
    cv = stein.SteinCV(seed=4, scale=0.6, w3_scale=0.1)
    vals = []
    for _ in range(40):
        lat.sweep(8, 1, 0)
        vals.append(cv.evaluate(lat, rho).cpu().numpy())
    v = np.stack(vals)  # (rounds, chains): chains independent
    per_chain = v.mean(axis=0)
    se = per_chain.std(ddof=1) / math.sqrt(len(per_chain))
    assert abs(per_chain.mean()) < 4 * se, (per_chain.mean(), se)
    assert v.std() > 0.0
    lat.close()


def test_training_lowers_loss_and_keeps_mean(env):
    torch, coulps, stream = env
    from paper_1403_0711_gb300 import inputs, stein
    L = (16, 16, 16)
    sites, q = inputs.cube(L, 2)
    lat = coulps.Lattice(L, n_chains=32, precision=coulps.F32, seed=9, stream=stream)
    ch = coulps.Charges(lat, sites, q, log_capacity=400)
    lat.sweep(100, 1, 1)
    rho = stein.charge_density(L, sites, q)
    phis, Aphis, es = stein.collect(lat, ch, rho, n_rounds=8, every=4, n_hb=1, n_or=1)
    cv = stein.SteinCV(seed=1, scale=0.3)
    log = []
    stein.fit(cv, phis, Aphis, es, rho, steps=60, batch=16, lr=3e-3, log=log)
    assert np.mean(log[-10:]) < np.mean(log[:10])
    # held-out samples: the CV estimator's mean agrees with the plain one
    ph2, A2, e2 = stein.collect(lat, ch, rho, n_rounds=8, every=4, n_hb=1, n_or=1)
    tg = stein.stein_terms(cv, ph2, A2, rho).cpu()
    e_cv = e2 - cv.c * tg
    se = float(np.sqrt(float(e2.var()) / len(e2) + float(e_cv.var()) / len(e_cv)))
    assert abs(float(e_cv.mean() - e2.mean())) < 4 * se
    ch.close()
    lat.close()
