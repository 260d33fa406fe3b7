"""Learned Stein control variate for the Eq. (nsum2) estimator.

For the lattice measure exp(-H_L) (Eq. (proplat), phi = 0 outside the box)
and any smooth vector field g(phi) with one component per site,
    E[ T g ] = 0,   T g = sum_x ( dg_x/dphi_x - g_x (A phi)_x ),   A phi = dH_L/dphi,
so e_CV = e - c T g has the mean of the plain sample e for any fixed c.
g is a 3-layer 3x3x3 conv net on the input channels (phi, rho, rho phi), 16
hidden channels, tanh, zero padding; c and the weights are fitted to minimise
Var(e - c T g) on stored samples of the chain.

All convolutions run in libcoulps.so's tcgen05 kernel (BF16 operands, FP32
accumulate), wrapped in a torch.autograd.Function whose backward uses the same
kernel for the input gradient (flipped, transposed weights) and the library's
weight-gradient kernel.  The divergence uses the identity
    sum_x dg_x/dphi_x = sum_q sum_c2 s2[c2,q] (conv(s1, K) + face corrections)[c2,q],
    K[c2,c1,e] = W2[c2,c1,e] sum_f W3[c2,f] W1[c1,phi,-(e+f)],
with s = tanh' of the pre-activations: one extra 16 -> 16 conv plus a
correction on the box's face sites (where some x = q - f fall outside), plus
the charge-site term of the rho phi channel (phi_x reaches h1 through it with
weight rho_x W1[c1, 2]), a 343-pair sum at each charge.

Training runs through autograd (the convs are the library's kernels; the
elementwise glue is PyTorch).  Evaluation inside the sampler (``evaluate``)
calls only library kernels.
"""
from __future__ import annotations

import ctypes
import itertools

import numpy as np
import torch

from . import coulps

OFFS = list(itertools.product((-1, 0, 1), repeat=3))  # index 9 (dz+1) + 3 (dy+1) + (dx+1)


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def pack_weights(W: torch.Tensor) -> torch.Tensor:
    """(16,16,3,3,3) float -> packed BF16 bits on the device (coulps_cv_pack_weights)."""
    w = np.ascontiguousarray(W.detach().float().cpu().numpy())
    out = np.zeros(27 * 256, dtype=np.uint16)
    st = coulps.load().coulps_cv_pack_weights(w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)))
    coulps._check(st, "coulps_cv_pack_weights")
    return torch.from_numpy(out.view(np.int16)).to(W.device)


def conv3d_tc(a: torch.Tensor, W: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """h = conv3d(a, W) + b with the library's tensor-core kernel.
    a: (n, Z, Y, X, 16) BF16 contiguous; W (16, 16, 3, 3, 3); b (16,)."""
    n, Z, Y, X, C = a.shape
    assert C == 16 and a.dtype == torch.bfloat16 and a.is_contiguous()
    out = torch.empty((n, Z, Y, X, 16), dtype=torch.float32, device=a.device)
    err = torch.zeros(1, dtype=torch.int32, device=a.device)
    wp = pack_weights(W)
    bias = b.detach().float().contiguous()
    st = coulps.load().coulps_cv_conv3d(_vp(a), _vp(wp), _vp(bias), _vp(out), n, X, Y, Z, 0, _vp(err),
                                        _stream())
    coulps._check(st, "coulps_cv_conv3d")
    return out


def conv3d_tanh_tc(a: torch.Tensor, W: torch.Tensor, b: torch.Tensor):
    """(tanh(h), 1 - tanh(h)^2) as BF16 for h = conv3d(a, W) + b (fused epilogue)."""
    n, Z, Y, X, C = a.shape
    assert C == 16 and a.dtype == torch.bfloat16 and a.is_contiguous()
    act = torch.empty((n, Z, Y, X, 16), dtype=torch.bfloat16, device=a.device)
    der = torch.empty_like(act)
    err = torch.zeros(1, dtype=torch.int32, device=a.device)
    wp = pack_weights(W)
    bias = b.detach().float().contiguous()
    st = coulps.load().coulps_cv_conv3d_tanh(_vp(a), _vp(wp), _vp(bias), _vp(act), _vp(der), n, X,
                                             Y, Z, 0, _vp(err), _stream())
    coulps._check(st, "coulps_cv_conv3d_tanh")
    return act, der


def conv3d_wgrad(a: torch.Tensor, dh: torch.Tensor) -> torch.Tensor:
    n, Z, Y, X, _ = a.shape
    ntiles = n * Z * Y * ((X + 63) // 64)
    nblk = min(1024, (ntiles + 31) // 32)
    scratch = torch.empty(nblk * 27 * 256, dtype=torch.float32, device=a.device)
    dW = torch.empty(16 * 16 * 27, dtype=torch.float32, device=a.device)
    st = coulps.load().coulps_cv_conv3d_wgrad(_vp(a), _vp(dh), _vp(dW), n, X, Y, Z, _vp(scratch),
                                              scratch.numel(), _stream())
    coulps._check(st, "coulps_cv_conv3d_wgrad")
    return dW.view(16, 16, 3, 3, 3)


class Conv3dTC(torch.autograd.Function):
    """conv3d 3x3x3, 16 -> 16 channels, channels last, on the tensor cores."""

    @staticmethod
    def forward(ctx, a, W, b):
        ctx.save_for_backward(a, W)
        return conv3d_tc(a, W, b)

    @staticmethod
    def backward(ctx, dh):
        a, W = ctx.saved_tensors
        dh16 = dh.contiguous().to(torch.bfloat16)
        da = dW = db = None
        if ctx.needs_input_grad[0]:
            Wt = W.detach().transpose(0, 1).flip(2, 3, 4).contiguous()
            da = conv3d_tc(dh16, Wt, torch.zeros(16, device=dh.device)).to(a.dtype)
        if ctx.needs_input_grad[1]:
            dW = conv3d_wgrad(a, dh16)
        if ctx.needs_input_grad[2]:
            db = dh.sum(dim=(0, 1, 2, 3))
        return da, dW, db


def _face_masks():
    """Allowed f (x = q - f inside) per face class c: 0 low, 1 inside, 2 high, 3 both."""
    allowed = {0: (-1, 0), 1: (-1, 0, 1), 2: (0, 1), 3: (0,)}
    masks = {}
    for cz, cy, cx in itertools.product(range(4), repeat=3):
        m = torch.tensor([1.0 if (f[0] in allowed[cz] and f[1] in allowed[cy]
                                  and f[2] in allowed[cx]) else 0.0 for f in OFFS])
        masks[cx + 4 * cy + 16 * cz] = m
    return masks


_FACE_MASKS = _face_masks()
_FACE_CLASSES = sorted(_FACE_MASKS)
_INSIDE = 1 + 4 + 16


def _pair_tensor():
    """P[e, f, u] = 1 where u = -(e + f) is a kernel offset."""
    P = torch.zeros(27, 27, 27)
    for ei, e in enumerate(OFFS):
        for fi, f in enumerate(OFFS):
            u = (-(e[0] + f[0]), -(e[1] + f[1]), -(e[2] + f[2]))
            if max(abs(v) for v in u) <= 1:
                P[ei, fi, OFFS.index(u)] = 1.0
    return P


_P = _pair_tensor()


def _charge_pairs():
    """The 343 (f, e) with f + e a kernel offset, in the library's order
    p = 49 az + 7 ay + ax, per axis a -> (f, e) as listed in _AXIS_PAIRS."""
    fi, ei, ui, fo, feo = [], [], [], [], []
    for az, ay, ax in itertools.product(range(7), repeat=3):
        (fz, ez), (fy, ey), (fx, ex) = _AXIS_PAIRS[az], _AXIS_PAIRS[ay], _AXIS_PAIRS[ax]
        f, e = (fz, fy, fx), (ez, ey, ex)
        u = (-(fz + ez), -(fy + ey), -(fx + ex))
        fi.append(OFFS.index(f))
        ei.append(OFFS.index(e))
        ui.append(OFFS.index(u))
        fo.append(f)
        feo.append((fz + ez, fy + ey, fx + ex))
    return (torch.tensor(fi), torch.tensor(ei), torch.tensor(ui), torch.tensor(fo),
            torch.tensor(feo))


_AXIS_PAIRS = ((-1, 0), (-1, 1), (0, -1), (0, 0), (0, 1), (1, -1), (1, 0))
_CP_F, _CP_E, _CP_U, _CP_FO, _CP_FEO = _charge_pairs()


def charge_matrix(W1, W2, W3):
    """M[p, c2, c1] = W3[0, c2, f_p] W2[c2, c1, e_p] W1[c1, 2, -(f_p + e_p)]."""
    dev = W1.device
    w3 = W3[0].reshape(16, 27)[:, _CP_F.to(dev)].T  # (p, c2)
    w2 = W2.reshape(16, 16, 27)[:, :, _CP_E.to(dev)].permute(2, 0, 1)  # (p, c2, c1)
    w1 = W1[:, 2].reshape(16, 27)[:, _CP_U.to(dev)].T  # (p, c1)
    return w3[:, :, None] * w2 * w1[:, None, :]


def charge_term(M, s1, s2, cq, crho):
    """sum_k crho[k] sum_p s2[x_k + f_p] . M[p] s1[x_k + f_p + e_p] per sample;
    s1, s2 (n, Z, Y, X, 16), cq (k, 3) sites as (z, y, x), zero outside."""
    if cq.shape[0] == 0:
        return torch.zeros(s1.shape[0], dtype=s1.dtype, device=s1.device)
    dev = s1.device
    s1p = torch.nn.functional.pad(s1, (0, 0, 2, 2, 2, 2, 2, 2))
    s2p = torch.nn.functional.pad(s2, (0, 0, 1, 1, 1, 1, 1, 1))
    fo, feo = _CP_FO.to(dev), _CP_FEO.to(dev)
    z, y, x = cq[:, 0:1], cq[:, 1:2], cq[:, 2:3]
    S2 = s2p[:, z + fo[None, :, 0] + 1, y + fo[None, :, 1] + 1, x + fo[None, :, 2] + 1]
    S1 = s1p[:, z + feo[None, :, 0] + 2, y + feo[None, :, 1] + 2, x + feo[None, :, 2] + 2]
    return torch.einsum("nkpa,pab,nkpb,k->n", S2, M.to(s1.dtype), S1, crho.to(s1.dtype))


def divergence_kernel(W1, W2, W3, fmask=None):
    """K[c2, c1, e] = W2[c2, c1, e] sum_f fmask[f] W3[0, c2, f] W1[c1, 0, -(e+f)];
    with fmask of shape (k, 27) returns (k, 16, 16, 3, 3, 3)."""
    w1 = W1[:, 0].reshape(16, 27)
    w2 = W2.reshape(16, 16, 27)
    w3 = W3[0].reshape(16, 27)
    P = _P.to(W1.device, W1.dtype)
    if fmask is None:
        M = torch.einsum("efu,af,bu->abe", P, w3, w1)
        return (w2 * M).reshape(16, 16, 3, 3, 3)
    M = torch.einsum("efu,kf,af,bu->kabe", P, fmask.to(W1.device, W1.dtype), w3, w1)
    return (w2[None] * M).reshape(-1, 16, 16, 3, 3, 3)


class SteinCV(torch.nn.Module):
    def __init__(self, seed=0, scale=0.3, device="cuda", w3_scale=0.0):
        super().__init__()
        g = torch.Generator().manual_seed(seed)

        def rnd(*s, sc):
            return torch.nn.Parameter((torch.randn(*s, generator=g) * sc).to(device))

        self.W1 = rnd(16, 3, 3, 3, 3, sc=scale)  # inputs phi, rho, rho phi
        self.b1 = rnd(16, sc=0.1)
        self.W2 = rnd(16, 16, 3, 3, 3, sc=scale / 4)
        self.b2 = rnd(16, sc=0.1)
        # the output layer starts at zero: T g = 0, i.e. the plain estimator
        self.W3 = rnd(1, 16, 3, 3, 3, sc=w3_scale)
        self.b3 = rnd(1, sc=0.0)
        self.c = 1.0  # coefficient of T g, set by fit()

    def weights(self):
        """(W1, W2, W3) rounded to BF16 as the tensor-core convs use them
        (straight-through for training).  The divergence must be that of the
        function actually evaluated: with unrounded weights in the divergence
        the Stein term picks up a bias."""
        return tuple(w + (w.to(torch.bfloat16).to(w.dtype) - w).detach()
                     for w in (self.W1, self.W2, self.W3))

    # -- parameters in the 16-channel form the kernel takes
    def _w1p(self):
        return torch.cat([self.W1, torch.zeros(16, 13, 3, 3, 3, device=self.W1.device)], dim=1)

    def set_density(self, rho: torch.Tensor):
        """The charge density the net sees (Lz, Ly, Lx); its non-zero sites are
        where the rho phi channel adds to the divergence."""
        self._rho = rho
        cq = torch.nonzero(rho)  # (k, 3) as (z, y, x), row-major order
        self._cq = cq
        self._crho = rho[cq[:, 0], cq[:, 1], cq[:, 2]].float()
        self._cq_xyz = cq.flip(1).to(torch.int32).contiguous()

    def _charges_for(self, rho):
        if getattr(self, "_rho", None) is not rho:
            self.set_density(rho)
        return self._cq, self._crho

    def _w3p(self):
        return torch.cat([self.W3, torch.zeros(15, 16, 3, 3, 3, device=self.W3.device)], dim=0)

    def _b3p(self):
        return torch.cat([self.b3, torch.zeros(15, device=self.b3.device)])

    def face_corrections(self):
        """(64, 16, 16, 27) K_b - K for every face class (zero for class 'inside')."""
        masks = torch.stack([_FACE_MASKS[b] for b in range(64)])
        Kb = divergence_kernel(*self.weights(), masks).reshape(64, 16, 16, 27)
        return Kb - Kb[_INSIDE][None]

    # -- differentiable T g: x0 (n, Z, Y, X, 16) BF16 input, Aphi (n, Z, Y, X).
    # faces=False drops the face-site divergence correction (used to train:
    # the coefficient c and every evaluation use the exact term, so the
    # estimator stays unbiased whatever the training objective).
    def stein_term(self, x0, Aphi, faces=True):
        """x0 from inputs_from(phi, rho) with the rho of set_density."""
        h1 = Conv3dTC.apply(x0, self._w1p(), self.b1)
        a1 = torch.tanh(h1)
        s1 = 1.0 - a1 * a1
        h2 = Conv3dTC.apply(a1.to(torch.bfloat16), self.W2, self.b2)
        a2 = torch.tanh(h2)
        s2 = 1.0 - a2 * a2
        g = Conv3dTC.apply(a2.to(torch.bfloat16), self._w3p(), self._b3p())[..., 0]
        K = divergence_kernel(*self.weights())
        D = Conv3dTC.apply(s1.to(torch.bfloat16), K, torch.zeros(16, device=x0.device))
        div = (s2 * D).sum(dim=(1, 2, 3, 4))
        if faces:
            div = div + self._face_term(s1, s2)
        div = div + charge_term(charge_matrix(*self.weights()), s1, s2, self._cq,
                                self._crho)
        return div - (g * Aphi).sum(dim=(1, 2, 3))

    def _face_term(self, s1, s2):
        n, Z, Y, X, _ = s1.shape
        s1p = torch.nn.functional.pad(s1, (0, 0, 1, 1, 1, 1, 1, 1))  # zero ring
        total = torch.zeros(n, device=s1.device)
        dK = self.face_corrections()
        zz, yy, xx = torch.meshgrid(torch.arange(Z), torch.arange(Y), torch.arange(X), indexing="ij")

        def cls(v, L):
            c = torch.ones_like(v)
            c[v == 0] = 0
            c[v == L - 1] = 2
            if L == 1:
                c[:] = 3
            return c

        cl = cls(xx, X) + 4 * cls(yy, Y) + 16 * cls(zz, Z)
        for b in torch.unique(cl).tolist():
            if b == _INSIDE:
                continue
            sel = (cl == b).nonzero()  # (m, 3) z, y, x
            patches = torch.stack([s1p[:, sel[:, 0] + 1 + o[0], sel[:, 1] + 1 + o[1],
                                       sel[:, 2] + 1 + o[2]] for o in OFFS], dim=2)  # (n, m, 27, 16)
            dD = torch.einsum("nmec,dce->nmd", patches, dK[b])
            total = total + (s2[:, sel[:, 0], sel[:, 1], sel[:, 2]] * dD).sum(dim=(1, 2))
        return total

    # -- evaluation with library kernels only
    @torch.no_grad()
    def evaluate(self, lat: "coulps.Lattice", rho: torch.Tensor) -> torch.Tensor:
        """T g for every chain of an FP32 lattice (float64 tensor of n_chains),
        computed on the lattice's stream."""
        lib = coulps.load()
        Lx, Ly, Lz = lat.L
        n = lat.n_chains
        dev = rho.device
        stream = lat._stream if isinstance(lat._stream, torch.cuda.Stream) else \
            torch.cuda.current_stream()
        K = divergence_kernel(*self.weights())
        dK = self.face_corrections().contiguous()
        M = charge_matrix(*self.weights()).float().contiguous()
        self._charges_for(rho)
        torch.cuda.current_stream().synchronize()
        with torch.cuda.stream(stream):
            x0 = torch.empty((n, Lz, Ly, Lx, 16), dtype=torch.bfloat16, device=dev)
            Aphi = torch.empty((n, Lz, Ly, Lx), dtype=torch.float32, device=dev)
            coulps._check(lib.coulps_cv_pack_field(lat.handle, _vp(rho), _vp(x0), _vp(Aphi)),
                          "coulps_cv_pack_field")
            a1, s1 = conv3d_tanh_tc(x0, self._w1p(), self.b1)
            a2, s2 = conv3d_tanh_tc(a1, self.W2, self.b2)
            g16 = conv3d_tc(a2, self._w3p(), self._b3p())
            D = conv3d_tc(s1, K, torch.zeros(16, device=dev))
            out = torch.empty(n, dtype=torch.float64, device=dev)
            scratch = torch.empty(128 * n, dtype=torch.float64, device=dev)
            coulps._check(lib.coulps_cv_stein_sum(
                _vp(g16), _vp(D), _vp(s2), _vp(Aphi), _vp(s1), _vp(dK), n, Lx, Ly, Lz,
                _vp(scratch), scratch.numel(), _vp(out), _stream()), "coulps_cv_stein_sum")
            nq = self._cq_xyz.shape[0]
            if nq:
                cscr = torch.empty(49 * nq * n, dtype=torch.float64, device=dev)
                coulps._check(lib.coulps_cv_charge_term(
                    _vp(s1), _vp(s2), _vp(M), _vp(self._cq_xyz), _vp(self._crho), nq, n,
                    (ctypes.c_int32 * 3)(Lx, Ly, Lz), 0, _vp(cscr), cscr.numel(), _vp(out),
                    _stream()),
                    "coulps_cv_charge_term")
        stream.synchronize()
        return out


def charge_density(L, sites, q, device="cuda") -> torch.Tensor:
    Lx, Ly, Lz = L
    rho = np.zeros((Lz, Ly, Lx), dtype=np.float32)
    s = np.asarray(sites, dtype=np.int64).reshape(-1, 3)
    np.add.at(rho, (s[:, 2], s[:, 1], s[:, 0]), np.asarray(q, dtype=np.float32))
    return torch.from_numpy(rho).to(device)


# --------------------------------------------------------------------------
# Training data and fitting
# --------------------------------------------------------------------------
@torch.no_grad()
def pack_inputs(lat: "coulps.Lattice", rho: torch.Tensor):
    """(phi BF16 (n, Z, Y, X), A phi FP32 (n, Z, Y, X)) of every chain, by the
    library's packing kernel."""
    Lx, Ly, Lz = lat.L
    n = lat.n_chains
    x0 = torch.empty((n, Lz, Ly, Lx, 16), dtype=torch.bfloat16, device=rho.device)
    Aphi = torch.empty((n, Lz, Ly, Lx), dtype=torch.float32, device=rho.device)
    coulps._check(coulps.load().coulps_cv_pack_field(lat.handle, _vp(rho), _vp(x0), _vp(Aphi)),
                  "coulps_cv_pack_field")
    lat.sync()
    return x0[..., 0].clone(), Aphi


def inputs_from(phi16: torch.Tensor, rho: torch.Tensor) -> torch.Tensor:
    """Rebuild the net input (phi, rho, rho phi, 0, ...) from stored BF16 phi."""
    x0 = torch.zeros(phi16.shape + (16,), dtype=torch.bfloat16, device=phi16.device)
    x0[..., 0] = phi16
    x0[..., 1] = rho.to(torch.bfloat16)
    x0[..., 2] = (rho.float() * phi16.float()).to(torch.bfloat16)
    return x0


def collect(lat, ch, rho, n_rounds, every=1, n_hb=1, n_or=3):
    """Run the sampler and keep, after every `every`-th measured compound
    sweep, each chain's (BF16 phi, A phi, e).  The charge set must log at
    least n_rounds * every samples."""
    phis, Aphis, es = [], [], []
    for r in range(n_rounds):
        ch.run(0, every, n_hb, n_or)
        p, a = pack_inputs(lat, rho)
        phis.append(p)
        Aphis.append(a)
        es.append(torch.from_numpy(ch.samples()[-1, :, 2].copy()))
    return torch.cat(phis), torch.cat(Aphis), torch.cat(es).double()


def fit(cv: SteinCV, phis, Aphis, es, rho, steps=200, batch=16, lr=2e-3, seed=0, log=None):
    """Minimise Var(e - T g) over the stored samples (Adam on all weights),
    then set cv.c = Cov(e, T g) / Var(T g) on the same samples."""
    g = torch.Generator().manual_seed(seed)
    opt = torch.optim.Adam([cv.W1, cv.b1, cv.W2, cv.b2, cv.W3, cv.b3], lr=lr)
    n = len(es)
    dev = phis.device
    es_d = es.to(dev)
    cv._charges_for(rho)
    for step in range(steps):
        idx = torch.randperm(n, generator=g)[:batch].to(dev)
        tg = cv.stein_term(inputs_from(phis[idx], rho), Aphis[idx], faces=False)
        r = es_d[idx].float() - tg
        loss = ((r - r.mean()) ** 2).mean() / (es_d.float().var() + 1e-30)
        opt.zero_grad()
        loss.backward()
        opt.step()
        if log is not None:
            log.append(float(loss.detach()))
    tgs = stein_terms(cv, phis, Aphis, rho)
    e = es.to(tgs.device)
    cv.c = float(((e - e.mean()) * (tgs - tgs.mean())).sum() / ((tgs - tgs.mean()) ** 2).sum())
    return tgs


@torch.no_grad()
def stein_terms(cv: SteinCV, phis, Aphis, rho, batch=16):
    cv._charges_for(rho)
    out = []
    for i in range(0, len(phis), batch):
        out.append(cv.stein_term(inputs_from(phis[i:i + batch], rho), Aphis[i:i + batch]).double())
    return torch.cat(out)


# --------------------------------------------------------------------------
# Localized control variate
# --------------------------------------------------------------------------
# T is linear in g, and g = (net inside a box R, 0 elsewhere) is still a smooth
# field of phi, so its Stein term keeps mean 0.  Around a compact cluster of
# charges (the q = 1 cube) most of the variance of e comes from the field near
# the charges, and a g supported there can cancel it.  The net only has to be
# evaluated on the sub-box E = R + 3 (its receptive field), which costs almost
# nothing next to a sweep of the whole lattice.

# per-axis allowed sets of the last layer's offset f for q within one site of
# R, indexed as the library's region kernel expects (f = -1 is bit 0)
_AXIS_SETS = ((-1,), (0,), (-1, 0), (1,), (0, 1), (-1, 0, 1))
_MASK_INDEX = {1: 0, 2: 1, 3: 2, 4: 3, 6: 4, 7: 5}


def _region_fmasks():
    """(216, 27) f masks, class ix + 6 iy + 36 iz."""
    m = torch.zeros(216, 27)
    for iz, iy, ix in itertools.product(range(6), repeat=3):
        for fi, f in enumerate(OFFS):  # f = (dz, dy, dx)
            if f[0] in _AXIS_SETS[iz] and f[1] in _AXIS_SETS[iy] and f[2] in _AXIS_SETS[ix]:
                m[ix + 6 * iy + 36 * iz, fi] = 1.0
    return m


_REGION_FMASKS = _region_fmasks()


def _axis_index(n, lo, hi):
    """Per coordinate 0..n-1 the allowed-set index, -1 when not next to [lo, hi)."""
    out = []
    for q in range(n):
        m = sum(1 << (f + 1) for f in (-1, 0, 1) if lo <= q - f < hi)
        out.append(_MASK_INDEX.get(m, -1))
    return out


class LocalSteinCV(SteinCV):
    """SteinCV whose g is the net inside the box R = [lo, hi) (lattice x, y, z
    coordinates, half-open) and 0 elsewhere."""

    def __init__(self, L, lo, hi, seed=0, scale=0.3, device="cuda", w3_scale=0.0):
        super().__init__(seed=seed, scale=scale, device=device, w3_scale=w3_scale)
        self.L = tuple(int(v) for v in L)
        lo = tuple(int(v) for v in lo)
        hi = tuple(int(v) for v in hi)
        if any(not (0 <= a < b <= n) for a, b, n in zip(lo, hi, self.L)):
            raise ValueError("region must be a non-empty box inside the lattice")
        self.e_lo = tuple(max(a - 3, 0) for a in lo)
        self.e_hi = tuple(min(b + 3, n) for b, n in zip(hi, self.L))
        self.edims = tuple(b - a for a, b in zip(self.e_lo, self.e_hi))
        self.r_lo = tuple(a - e for a, e in zip(lo, self.e_lo))  # R in E coordinates
        self.r_hi = tuple(b - e for b, e in zip(hi, self.e_lo))
        ex, ey, ez = self.edims
        ix = _axis_index(ex, self.r_lo[0], self.r_hi[0])
        iy = _axis_index(ey, self.r_lo[1], self.r_hi[1])
        iz = _axis_index(ez, self.r_lo[2], self.r_hi[2])
        # sites q of E next to R and their classes, for the differentiable term
        qs, cls = [], []
        for z in range(ez):
            for y in range(ey):
                for x in range(ex):
                    if ix[x] >= 0 and iy[y] >= 0 and iz[z] >= 0:
                        qs.append((z, y, x))
                        cls.append(ix[x] + 6 * iy[y] + 36 * iz[z])
        self._q = torch.tensor(qs, device=device)
        self._qcls = torch.tensor(cls, device=device)
        rmask = torch.zeros(ez, ey, ex, device=device)
        rmask[self.r_lo[2]:self.r_hi[2], self.r_lo[1]:self.r_hi[1], self.r_lo[0]:self.r_hi[0]] = 1
        self._rmask = rmask

    def set_density(self, rho: torch.Tensor):
        """rho of the whole box; the charge-site term keeps the charges inside R
        (in E coordinates)."""
        self._rho = rho
        (x0, y0, z0), (x1, y1, z1) = self.e_lo, self.e_hi
        re = rho[z0:z1, y0:y1, x0:x1] * self._rmask.to(rho.device, rho.dtype)
        cq = torch.nonzero(re)
        self._cq = cq
        self._crho = re[cq[:, 0], cq[:, 1], cq[:, 2]].float()
        self._cq_xyz = cq.flip(1).to(torch.int32).contiguous()

    def region_kernels(self):
        """(216, 16, 16, 27) divergence kernel per allowed-offset class."""
        return divergence_kernel(*self.weights(), _REGION_FMASKS).reshape(216, 16, 16, 27)

    def rho_region(self, rho):
        """The density restricted to E, (ez, ey, ex)."""
        (x0, y0, z0), (x1, y1, z1) = self.e_lo, self.e_hi
        return rho[z0:z1, y0:y1, x0:x1]

    # -- differentiable T g on E-sized inputs: x0 (n, ez, ey, ex, 16) BF16
    def stein_term(self, x0, Aphi, faces=True):
        h1 = Conv3dTC.apply(x0, self._w1p(), self.b1)
        a1 = torch.tanh(h1)
        s1 = 1.0 - a1 * a1
        h2 = Conv3dTC.apply(a1.to(torch.bfloat16), self.W2, self.b2)
        a2 = torch.tanh(h2)
        s2 = 1.0 - a2 * a2
        g = Conv3dTC.apply(a2.to(torch.bfloat16), self._w3p(), self._b3p())[..., 0]
        # s rounded like the library kernel's BF16 copies (straight-through)
        s1 = s1 + (s1.to(torch.bfloat16).float() - s1).detach()
        s2 = s2 + (s2.to(torch.bfloat16).float() - s2).detach()
        div = self.region_divergence(s1, s2) + charge_term(
            charge_matrix(*self.weights()), s1, s2, self._cq, self._crho)
        return div - (g * Aphi * self._rmask).sum(dim=(1, 2, 3))

    def region_divergence(self, s1, s2):
        """sum_{x in R} dg_x/dphi_x from s1, s2 (n, ez, ey, ex, 16): for each q
        next to R, s2[q] . (K_class(q) applied to the 27 neighbours of s1)."""
        s1p = torch.nn.functional.pad(s1, (0, 0, 1, 1, 1, 1, 1, 1))
        qz, qy, qx = self._q[:, 0], self._q[:, 1], self._q[:, 2]
        patches = torch.stack([s1p[:, qz + 1 + o[0], qy + 1 + o[1], qx + 1 + o[2]] for o in OFFS],
                              dim=2)  # (n, m, 27, 16)
        Kq = self.region_kernels()[self._qcls]  # (m, 16 c2, 16 c1, 27)
        d = torch.einsum("nmec,mdce->nmd", patches, Kq)
        return (s2[:, qz, qy, qx] * d).sum(dim=(1, 2))

    @torch.no_grad()
    def pack(self, lat: "coulps.Lattice", rho: torch.Tensor, interleave=False):
        """(net input on E BF16, A phi on E FP32) of every chain, by the
        library's packing kernel on the lattice's stream: (n, ez, ey, ex, 16)
        and (n, ez, ey, ex), or with interleave the boxes side by side along x
        with a zero gutter column each, (1, ez, ey, n (ex + 1), 16) and
        (1, ez, ey, n (ex + 1))."""
        n = lat.n_chains
        ex, ey, ez = self.edims
        shape = (1, ez, ey, n * (ex + 1)) if interleave else (n, ez, ey, ex)
        x0 = torch.empty(shape + (16,), dtype=torch.bfloat16, device=rho.device)
        Aphi = torch.empty(shape, dtype=torch.float32, device=rho.device)
        o = (ctypes.c_int32 * 3)(*self.e_lo)
        d = (ctypes.c_int32 * 3)(*self.edims)
        coulps._check(coulps.load().coulps_cv_pack_region(lat.handle, _vp(rho), o, d,
                                                          1 if interleave else 0, _vp(x0),
                                                          _vp(Aphi)), "coulps_cv_pack_region")
        return x0, Aphi

    def prepare(self):
        """Pack the weights and class kernels for evaluate (call after fitting)."""
        with torch.no_grad():
            dev = self.W1.device
            self._ev = {
                "w1": pack_weights(self._w1p()), "w2": pack_weights(self.W2),
                "b1": self.b1.detach().float().contiguous(), "b2": self.b2.detach().float().contiguous(),
                # per class [e][c2][c1], packed below for the region kernel
                "K": self.region_kernels().detach().float().permute(0, 3, 1, 2).contiguous(),
                "M": charge_matrix(*self.weights()).detach().float().contiguous(),
                # the last layer for the sites of R: [o][ci], o = 9 kz + 3 ky + kx
                "w3g": self.weights()[2][0].detach().float().permute(1, 2, 3, 0)
                       .reshape(27, 16).contiguous(),
                "b3g": float(self.b3.detach()[0]),
                "err": torch.zeros(1, dtype=torch.int32, device=dev),
            }
            # the class kernels as the region kernel's tensor-core operand
            # (three BF16 parts each), formed once per set of weights
            self._ev["Kpack"] = torch.empty(216 * 41472, dtype=torch.uint8, device=dev)
            coulps._check(coulps.load().coulps_cv_region_pack(
                _vp(self._ev["K"]), _vp(self._ev["Kpack"]),
                ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)),
                "coulps_cv_region_pack")
            # evaluate runs on the lattice's stream, which may be another one
            torch.cuda.current_stream(dev).synchronize()

    # -- evaluation with library kernels only, on the lattice's stream
    @torch.no_grad()
    def evaluate(self, lat: "coulps.Lattice", rho: torch.Tensor, out=None) -> torch.Tensor:
        """T g for every chain (float64 tensor of n_chains, on the device), all
        in library kernels queued on the lattice's stream; not synchronised."""
        if not hasattr(self, "_ev"):
            self.prepare()
        ev = self._ev
        self._charges_for(rho)
        lib = coulps.load()
        n = lat.n_chains
        ex, ey, ez = self.edims
        dev = rho.device
        stream = lat._stream if isinstance(lat._stream, torch.cuda.Stream) else \
            torch.cuda.current_stream()
        sp = ctypes.c_void_p(stream.cuda_stream)
        # the chains' boxes side by side along x (zero gutters between them), so
        # the tensor-core tiles (128 sites of x) are filled
        P = ex + 1
        X = n * P
        with torch.cuda.stream(stream):
            x0, Aphi = self.pack(lat, rho, interleave=True)
            a1 = torch.empty_like(x0)
            s1 = torch.empty_like(x0)
            a2 = torch.empty_like(x0)
            s2 = torch.empty_like(x0)
            # rows and planes the region terms read: the first layer's outputs
            # within 2 sites of R (s1 around R + 1, a1 for the second layer),
            # the second layer's within 1 (s2 and a2 on R + 1)
            for src, w, b, dst, m in ((x0, "w1", "b1", (a1, s1), 2), (a1, "w2", "b2", (a2, s2), 1)):
                y0, y1 = max(self.r_lo[1] - m, 0), min(self.r_hi[1] + m, ey)
                z0, z1 = max(self.r_lo[2] - m, 0), min(self.r_hi[2] + m, ez)
                coulps._check(lib.coulps_cv_conv3d_tanh_rows(
                    _vp(src), _vp(ev[w]), _vp(ev[b]), _vp(dst[0]), _vp(dst[1]), 1, X, ey, ez, P,
                    y0, y1, z0, z1, _vp(ev["err"]), sp), "coulps_cv_conv3d_tanh_rows")
            # the last layer is formed at the sites of R inside the region kernel
            if out is None:
                out = torch.empty(n, dtype=torch.float64, device=dev)
            nr = ((self.r_hi[0] - self.r_lo[0]) * (self.r_hi[1] - self.r_lo[1]) *
                  (self.r_hi[2] - self.r_lo[2]))
            scratch = torch.empty((self._q.shape[0] + nr) * n, dtype=torch.float64, device=dev)
            ed = (ctypes.c_int32 * 3)(*self.edims)
            rl = (ctypes.c_int32 * 3)(*self.r_lo)
            rh = (ctypes.c_int32 * 3)(*self.r_hi)
            coulps._check(lib.coulps_cv_stein_region(
                _vp(a2), _vp(ev["w3g"]), ev["b3g"], _vp(s1), _vp(s2), _vp(Aphi), _vp(ev["Kpack"]),
                n, ed, 1, rl, rh,
                _vp(scratch), scratch.numel(), _vp(out), _vp(ev["err"]), sp),
                "coulps_cv_stein_region")
            nq = self._cq_xyz.shape[0]
            if nq:
                cscr = torch.empty(49 * nq * n, dtype=torch.float64, device=dev)
                coulps._check(lib.coulps_cv_charge_term(
                    _vp(s1), _vp(s2), _vp(ev["M"]), _vp(self._cq_xyz), _vp(self._crho), nq, n, ed,
                    1, _vp(cscr), cscr.numel(), _vp(out), sp), "coulps_cv_charge_term")
        return out

    @torch.no_grad()
    def record_graph(self, lat: "coulps.Lattice", ch: "coulps.Charges", rho: torch.Tensor):
        """A CUDA graph of evaluate + coulps_cv_record (y = e - c T g for every
        chain), to replay on the lattice's stream after each measured sweep:
        library kernels only, no host work per sample.  Returns (graph, tg)."""
        if not hasattr(self, "_ev"):
            self.prepare()
        stream = lat._stream if isinstance(lat._stream, torch.cuda.Stream) else \
            torch.cuda.current_stream()
        tg = torch.zeros(lat.n_chains, dtype=torch.float64, device=rho.device)
        self.evaluate(lat, rho, out=tg)  # first launches (kernel attributes) outside capture
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            self.evaluate(lat, rho, out=tg)
            ch.cv_record(tg.data_ptr(), self.c)
        return graph, tg


def collect_region(cv: LocalSteinCV, lat, ch, rho, n_rounds, every=1, n_hb=1, n_or=3):
    """Like collect, on E only: (BF16 phi (k, ez, ey, ex), A phi, e)."""
    phis, Aphis, es = [], [], []
    for r in range(n_rounds):
        ch.run(0, every, n_hb, n_or)
        x0, a = cv.pack(lat, rho)
        lat.sync()
        phis.append(x0[..., 0].clone())
        Aphis.append(a)
        es.append(torch.from_numpy(ch.chain_stats()[:, 7].copy()))  # latest sample e
    return torch.cat(phis), torch.cat(Aphis), torch.cat(es).double()


def fit_region(cv: LocalSteinCV, phis, Aphis, es, rho, steps=400, batch=64, lr=3e-3, seed=0,
               log=None, holdout=0.25):
    """Minimise Var(e - T g) (Adam with a cosine learning-rate decay, exact
    region term), then set
    cv.c = Cov(e, T g) / Var(T g) on held-out samples (the last `holdout`
    fraction), which keeps the coefficient independent of the weights' fit."""
    g = torch.Generator().manual_seed(seed)
    opt = torch.optim.Adam([cv.W1, cv.b1, cv.W2, cv.b2, cv.W3, cv.b3], lr=lr)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, T_max=max(1, steps), eta_min=lr / 30)
    n = len(es)
    n_tr = max(2, int(n * (1.0 - holdout)))
    dev = phis.device
    es_d = es.to(dev)
    rho_e = cv.rho_region(rho)
    cv._charges_for(rho)
    var_e = es_d[:n_tr].float().var() + 1e-30
    for step in range(steps):
        idx = torch.randint(0, n_tr, (batch,), generator=g).to(dev)
        tg = cv.stein_term(inputs_from(phis[idx], rho_e), Aphis[idx])
        r = es_d[idx].float() - tg
        loss = ((r - r.mean()) ** 2).mean() / var_e
        opt.zero_grad()
        loss.backward()
        opt.step()
        sched.step()
        if log is not None:
            log.append(float(loss.detach()))
    with torch.no_grad():
        tgs = torch.cat([cv.stein_term(inputs_from(phis[i:i + 256], rho_e), Aphis[i:i + 256]).double()
                         for i in range(0, n, 256)])
    e, t = es.to(tgs.device)[n_tr:], tgs[n_tr:]
    if len(e) < 2:
        e, t = es.to(tgs.device), tgs
    cv.c = float(((e - e.mean()) * (t - t.mean())).sum() / ((t - t.mean()) ** 2).sum())
    cv.prepare()
    return tgs
