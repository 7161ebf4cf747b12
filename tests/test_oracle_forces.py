"""Pins of the oracle's network, energy, forces and force-matching gradient.

* MLP forward and input-gradient equal torch.nn.functional (linear, celu)
  and torch.autograd in float64 (library routines, not this project's code);
* forces equal central finite differences of the energy (Eq. 2), also for
  boxes shorter than the cutoff (self-images) and isolated clusters;
* sum F = 0, zero torque for isolated clusters;
* E is invariant under translation, the 24 rotations of the cube (periodic),
  any rotation (isolated) and permutation of same-species atoms;
* W1 = 0 gives F = 0; a lone atom has G = 0 and E = MLP(0);
* the directional derivative of the AEV equals finite differences;
* dL/dtheta of the force-matching loss equals finite differences in the
  weights; b4 has no effect on forces (its gradient is exactly 0).
"""
import itertools

import numpy as np
import pytest
import torch

import synth


def _setup(oracle_mod, Zs=(1, 8), seed=4, bias=True):
    p = oracle_mod.Params(atomic_numbers=Zs)
    w = synth.xavier_weights(p.n_species, p.aev_length, seed)
    if bias:
        w = synth.random_biases(w, seed + 1)
    return p, w, oracle_mod.Model(p, w)


def test_mlp_matches_torch(oracle_mod):
    p, w, m = _setup(oracle_mod)
    rng = np.random.default_rng(0)
    for s in range(2):
        x = rng.uniform(0, 1.5, size=p.aev_length)
        e, dx = oracle_mod.mlp(m, s, x)
        xt = torch.tensor(x, dtype=torch.float64, requires_grad=True)
        h = xt
        for l, (W, b) in enumerate(w[s]):
            h = torch.nn.functional.linear(h, torch.tensor(W.T), torch.tensor(b))
            if l < 3:
                h = torch.nn.functional.celu(h, alpha=0.1)
        (g,) = torch.autograd.grad(h.sum(), xt)
        assert e == pytest.approx(float(h.detach()), rel=1e-13, abs=1e-13)
        # torch's float64 CELU backward rounds alpha through single precision
        # (relative error ~3e-9 on this input); the mpmath check below is tight.
        assert np.abs(dx - g.numpy()).max() < 1e-7 * np.abs(dx).max()


def test_mlp_gradient_mpmath(oracle_mod):
    """40-digit evaluation of one input-gradient entry by central difference."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    p, w, m = _setup(oracle_mod)
    x = np.random.default_rng(0).uniform(0, 1.5, size=p.aev_length)
    _, dx = oracle_mod.mlp(m, 0, x)
    al = mpmath.mpf(1) / 10

    def f(xv):
        h = [mpmath.mpf(v) for v in xv]
        for l, (W, b) in enumerate(w[0]):
            out = []
            for j in range(W.shape[1]):
                acc = mpmath.mpf(b[j]) + mpmath.fsum(h[k] * mpmath.mpf(W[k, j]) for k in range(W.shape[0]))
                if l < 3 and acc <= 0:
                    acc = al * (mpmath.exp(acc / al) - 1)
                out.append(acc)
            h = out
        return h[0]

    for k in (3, 81):
        xp = [mpmath.mpf(v) for v in x]
        xm = list(xp)
        eps = mpmath.mpf("1e-15")
        xp[k] += eps
        xm[k] -= eps
        fd = (f(xp) - f(xm)) / (2 * eps)
        assert abs(dx[k] - float(fd)) < 1e-14 * max(1.0, abs(float(fd)))


def _fd_forces(oracle_mod, m, pos, sp, box, h=1e-5, atoms=None):
    atoms = range(pos.shape[0]) if atoms is None else atoms
    F = {}
    for i in atoms:
        for c in range(3):
            xp = pos.copy(); xp[i, c] += h
            xm = pos.copy(); xm[i, c] -= h
            ep = oracle_mod.energy_forces(m, xp, sp, box)[0]
            em = oracle_mod.energy_forces(m, xm, sp, box)[0]
            F[(i, c)] = -(ep - em) / (2 * h)
    return F


@pytest.mark.parametrize("case", ["small_pbc", "tiny_pbc", "isolated"])
def test_forces_finite_difference(oracle_mod, case):
    p, w, m = _setup(oracle_mod)
    if case == "isolated":
        s = synth.water_box(27, 3)
        pos, Z, box = s.pos[:12], s.Z[:12], None
    elif case == "tiny_pbc":                     # L = 6.2 A < Rc: self-images
        s = synth.water_box(8, 4)
        pos, Z, box = s.pos, s.Z, s.box
    else:
        s = synth.water_box(27, 5)
        pos, Z, box = s.pos, s.Z, s.box
    sp = p.species_of(Z)
    E, Ei, F, G = oracle_mod.energy_forces(m, pos, sp, box)
    assert E == pytest.approx(Ei.sum(), rel=1e-14)
    atoms = list(range(0, pos.shape[0], max(1, pos.shape[0] // 8)))
    fd = _fd_forces(oracle_mod, m, pos, sp, box, atoms=atoms)
    scale = np.abs(F).max()
    for (i, c), v in fd.items():
        assert abs(F[i, c] - v) < 2e-7 * max(1.0, scale), (i, c, F[i, c], v)


def test_force_sums_and_torque(oracle_mod):
    p, w, m = _setup(oracle_mod)
    s = synth.water_box(64, 1001)
    sp = p.species_of(s.Z)
    _, _, F, _ = oracle_mod.energy_forces(m, s.pos, sp, s.box)
    assert np.abs(F.sum(0)).max() < 1e-11 * max(1, np.abs(F).max()) * s.n
    x = s.pos[:30]
    _, _, F, _ = oracle_mod.energy_forces(m, x, sp[:30], None)
    assert np.abs(F.sum(0)).max() < 1e-12 * 30
    torque = np.cross(x - x.mean(0), F).sum(0)
    assert np.abs(torque).max() < 1e-11 * 30


def test_invariances(oracle_mod):
    p, w, m = _setup(oracle_mod)
    s = synth.water_box(27, 6)
    sp = p.species_of(s.Z)
    L = s.box[0]
    E0, _, F0, _ = oracle_mod.energy_forces(m, s.pos, sp, s.box)
    # translation
    E1, _, F1, _ = oracle_mod.energy_forces(m, s.pos + np.array([1.7, -40.2, 9.9]), sp, s.box)
    assert E1 == pytest.approx(E0, rel=1e-12) and np.allclose(F1, F0, atol=1e-10)
    # 24 rotations of the cube: signed axis permutations with det +1, then wrap
    rots = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3))
            for r, (c, sg) in enumerate(zip(perm, signs)):
                R[r, c] = sg
            if np.linalg.det(R) > 0:
                rots.append(R)
    assert len(rots) == 24
    for R in rots[::3]:
        x = np.mod((s.pos - L / 2) @ R.T + L / 2, L)
        E2, _, F2, _ = oracle_mod.energy_forces(m, x, sp, s.box)
        assert E2 == pytest.approx(E0, rel=1e-12)
        assert np.allclose(F2, F0 @ R.T, atol=1e-10)
    # arbitrary rotation of an isolated cluster
    x = s.pos[:24]
    q = np.linalg.qr(np.random.default_rng(2).normal(size=(3, 3)))[0]
    Ea, _, Fa, _ = oracle_mod.energy_forces(m, x, sp[:24], None)
    Eb, _, Fb, _ = oracle_mod.energy_forces(m, x @ q.T, sp[:24], None)
    assert Eb == pytest.approx(Ea, rel=1e-12) and np.allclose(Fb, Fa @ q.T, atol=1e-10)
    # permutation of atoms (species travel with them)
    perm = np.random.default_rng(3).permutation(s.n)
    E3, _, F3, _ = oracle_mod.energy_forces(m, s.pos[perm], sp[perm], s.box)
    assert E3 == pytest.approx(E0, rel=1e-12) and np.allclose(F3, F0[perm], atol=1e-10)


def test_zero_first_layer_and_lone_atom(oracle_mod):
    p, w, m = _setup(oracle_mod)
    w0 = [[(np.zeros_like(W) if l == 0 else W, b) for l, (W, b) in enumerate(sp_)] for sp_ in w]
    m0 = oracle_mod.Model(p, w0)
    s = synth.water_box(27, 7)
    sp = p.species_of(s.Z)
    E, Ei, F, _ = oracle_mod.energy_forces(m0, s.pos, sp, s.box)
    assert np.all(F == 0)
    e_h = oracle_mod.mlp(m0, 0, np.zeros(128))[0]
    e_o = oracle_mod.mlp(m0, 1, np.zeros(128))[0]
    assert E == pytest.approx((sp == 0).sum() * e_h + (sp == 1).sum() * e_o, rel=1e-13)
    # lone O in a 20 A box: G = 0, E = MLP_O(0), F = 0
    E, Ei, F, G = oracle_mod.energy_forces(m, np.array([[3.0, 4.0, 5.0]]), np.array([1]),
                                           np.array([20.0, 20.0, 20.0]))
    assert np.all(G == 0) and np.all(F == 0)
    assert E == pytest.approx(oracle_mod.mlp(m, 1, np.zeros(128))[0], rel=1e-15)


def test_aev_jvp_finite_difference(oracle_mod):
    p, w, m = _setup(oracle_mod)
    s = synth.water_box(8, 8)
    sp = p.species_of(s.Z)
    v = np.random.default_rng(5).normal(size=s.pos.shape)
    T = oracle_mod.aev_jvp(m, s.pos, sp, s.box, v)
    h = 1e-6
    Gp = oracle_mod.energy_forces(m, s.pos + h * v, sp, s.box)[3]
    Gm = oracle_mod.energy_forces(m, s.pos - h * v, sp, s.box)[3]
    assert np.allclose(T, (Gp - Gm) / (2 * h), atol=2e-7 * max(1, np.abs(T).max()))


def _loss(oracle_mod, p, w, pos, sp, box, Fref):
    m = oracle_mod.Model(p, w)
    _, _, F, _ = oracle_mod.energy_forces(m, pos, sp, box)
    return ((F - Fref) ** 2).sum() / (3 * pos.shape[0])


@pytest.mark.parametrize("Zs,kind", [((1, 8), "water"), ((1, 6, 7, 8), "hcno")])
def test_force_match_gradient(oracle_mod, Zs, kind):
    p, w, m = _setup(oracle_mod, Zs)
    if kind == "water":
        s = synth.water_box(8, 9)
        pos, Z, box = s.pos, s.Z, s.box
    else:
        rng = np.random.default_rng(1)
        pos = np.cumsum(rng.normal(size=(14, 3)) * 0.8, 0)
        pos = pos - pos.min(0) + 1.0
        Z = np.array([1, 6, 7, 8, 1, 1, 6, 6, 8, 1, 7, 1, 6, 1])
        box = None
    sp = p.species_of(Z)
    # teacher network of the same architecture gives the reference forces
    wt = synth.random_biases(synth.xavier_weights(p.n_species, p.aev_length, 99), 98)
    Fref = oracle_mod.energy_forces(oracle_mod.Model(p, wt), pos, sp, box)[2]
    L, dW, db, F = oracle_mod.force_match(m, pos, sp, box, Fref)
    assert L == pytest.approx(_loss(oracle_mod, p, w, pos, sp, box, Fref), rel=1e-13)
    rng = np.random.default_rng(11)
    for s_ in range(p.n_species):
        for l in range(4):
            for which in ("W", "b"):
                if which == "b" and l == 3:
                    assert np.all(db[s_][3] == 0)
                    continue
                D = [[(np.zeros_like(W), np.zeros_like(b)) for W, b in sp_] for sp_ in w]
                ref = w[s_][l][0] if which == "W" else w[s_][l][1]
                # unit direction: CELU'' jumps at z = 0, so a long step would
                # cross kinks of dL/dtheta and spoil the central difference
                dirn = rng.normal(size=ref.shape)
                dirn /= np.linalg.norm(dirn)
                if which == "W":
                    D[s_][l] = (dirn, np.zeros_like(w[s_][l][1]))
                    analytic = float((dW[s_][l] * dirn).sum())
                else:
                    D[s_][l] = (np.zeros_like(w[s_][l][0]), dirn)
                    analytic = float((db[s_][l] * dirn).sum())
                errs = []
                for h in (1e-5, 1e-6):
                    wp = [[(W + h * dw, b + h * dbb) for (W, b), (dw, dbb) in zip(a, d)] for a, d in zip(w, D)]
                    wm = [[(W - h * dw, b - h * dbb) for (W, b), (dw, dbb) in zip(a, d)] for a, d in zip(w, D)]
                    fd = (_loss(oracle_mod, p, wp, pos, sp, box, Fref) -
                          _loss(oracle_mod, p, wm, pos, sp, box, Fref)) / (2 * h)
                    errs.append(abs(analytic - fd) / max(abs(fd), 1e-6))
                # a neuron within ~h of z = 0 spoils one step size, never both
                assert min(errs) < 1e-6, (s_, l, which, errs)


def test_force_match_zero_at_target(oracle_mod):
    p, w, m = _setup(oracle_mod)
    s = synth.water_box(8, 10)
    sp = p.species_of(s.Z)
    F = oracle_mod.energy_forces(m, s.pos, sp, s.box)[2]
    L, dW, db, _ = oracle_mod.force_match(m, s.pos, sp, s.box, F)
    assert L == 0.0
    assert all(np.all(x == 0) for sp_ in dW for x in sp_)
