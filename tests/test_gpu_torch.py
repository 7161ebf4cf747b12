"""torch.autograd functions over the C ABI, checked by finite differences.

* nnp_energy: dE/dpos = -F against a central difference of the library
  energy along a random unit direction (h = 5e-3 A; FP32 energy noise
  ~2e-6 eV gives ~4e-4 eV/A of FD noise) -> 1 % agreement;
* force_match_loss: dL/dparams (nnp_force_match_grad) against a central
  difference of the library loss along the normalised gradient of one
  layer (h = 3e-4), and against the FP64 oracle's exact gradient;
* nnp_forces: d(sum W*F)/dparams through the dL/dF entry point against the
  oracle.
"""
import numpy as np
import pytest

import synth
from common import weights32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_2604_21441_b300 import build
    build.build()
    import paper_2604_21441_b300 as P
    from paper_2604_21441_b300 import torch_nnp
    return P, torch_nnp


def _setup(P, w):
    pot = P.NNP(atomic_numbers=(1, 8))
    pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in x] for x in w])
    return pot


def test_energy_grad_fd(T):
    import torch
    P, tn = T
    s = synth.water_box(64, 1001)
    w = weights32(2, 128, 41, 42)
    pot = _setup(P, w)
    Z = torch.tensor(s.Z, device="cuda")
    pos = torch.tensor(s.pos, device="cuda", requires_grad=True)
    E = tn.nnp_energy(pot, pos, Z, s.box)
    E.backward()
    g = pos.grad.detach()
    d = torch.randn(pos.shape, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    d /= d.norm()
    h = 5e-3
    with torch.no_grad():
        Ep = tn.nnp_energy(pot, pos + h * d, Z, s.box)
        Em = tn.nnp_energy(pot, pos - h * d, Z, s.box)
    fd = float((Ep - Em) / (2 * h))
    an = float((g * d).sum())
    assert abs(fd - an) <= 1e-2 * abs(an) + 1e-3, (fd, an)


def _pack(dW, db):
    return np.concatenate([np.r_[np.asarray(W).ravel(), np.asarray(b).ravel()]
                           for sW, sb in zip(dW, db) for W, b in zip(sW, sb)])


def test_force_match_loss_fd_and_oracle(T, oracle_mod):
    import torch
    P, tn = T
    s = synth.water_box(27, 5)
    w = weights32(2, 128, 43, 44)
    wt = weights32(2, 128, 45, 46)
    p = oracle_mod.Params()
    sp = p.species_of(s.Z)
    Fref = oracle_mod.energy_forces(oracle_mod.Model(p, wt), s.pos, sp, s.box)[2]
    pot = _setup(P, w)
    Z = torch.tensor(s.Z, device="cuda")
    pos = torch.tensor(s.pos, device="cuda")
    params = tn.pack_params(w).requires_grad_(True)
    L = tn.force_match_loss(pot, params, pos, Z, s.box, Fref)
    L.backward()
    g = params.grad.detach().numpy()
    _, dW, db, _ = oracle_mod.force_match(oracle_mod.Model(p, w), s.pos, sp, s.box, Fref)
    gref = _pack(dW, db)
    assert np.abs(g - gref).max() <= 2e-3 * np.abs(gref).max()
    # finite difference along the (normalised) gradient restricted to W2 of species 0
    D = 128
    off = D * 160 + 160
    n2 = 160 * 128
    d = np.zeros_like(g)
    d[off:off + n2] = g[off:off + n2]
    d /= np.linalg.norm(d)
    h = 3e-4
    with torch.no_grad():
        base = params.detach()
        Lp = float(tn.force_match_loss(pot, base + h * torch.tensor(d), pos, Z, s.box, Fref))
        Lm = float(tn.force_match_loss(pot, base - h * torch.tensor(d), pos, Z, s.box, Fref))
    fd = (Lp - Lm) / (2 * h)
    an = float(g @ d)
    assert abs(fd - an) <= 3e-2 * abs(an), (fd, an)


def test_forces_function_vjp(T, oracle_mod):
    import torch
    P, tn = T
    s = synth.water_box(27, 6)
    w = weights32(2, 128, 47, 48)
    pot = _setup(P, w)
    Z = torch.tensor(s.Z, device="cuda")
    pos = torch.tensor(s.pos, device="cuda")
    params = tn.pack_params(w).requires_grad_(True)
    Wgt = torch.tensor(np.random.default_rng(1).normal(size=(s.n, 3)), device="cuda")
    E, F = tn.nnp_forces(pot, params, pos, Z, s.box)
    (F * Wgt).sum().backward()
    g = params.grad.detach().numpy()
    # oracle: v = Wgt  <=>  Fref = F - 3n Wgt / 2 in the force-matching loss
    p = oracle_mod.Params()
    sp = p.species_of(s.Z)
    m = oracle_mod.Model(p, w)
    Fo = oracle_mod.energy_forces(m, s.pos, sp, s.box)[2]
    Fref = Fo - 1.5 * s.n * Wgt.cpu().numpy()
    _, dW, db, _ = oracle_mod.force_match(m, s.pos, sp, s.box, Fref)
    gref = _pack(dW, db)
    assert np.abs(g - gref).max() <= 2e-3 * np.abs(gref).max()
