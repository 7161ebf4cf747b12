"""Pins of the oracle's network ensemble (mean of M networks over one
descriptor).

* M members equal ONE wider network: the first layers side by side, the
  hidden layers block-diagonal, the output layer stacked and divided by M
  and the output bias the mean (CELU acts element by element, so the blocks
  never mix).  That single network runs through the oracle's plain network
  and force path, not through the mean.
* M copies of one network give that network's energy, per-atom energies and
  forces.
* The ensemble forces equal central finite differences of the ensemble
  energy.
* The force-matching gradient of the ensemble (the loss of the members'
  mean force) equals central finite differences of that loss along unit
  directions in each member's layers, and equals the gradient of the
  equivalent wider network, mapped back to the members' blocks (output
  weights: the wide network stores w4 / M, so its gradient there is M times
  the member's).
"""
import numpy as np

import synth
from common import weights32


def _members(M, seed):
    return [weights32(2, 128, seed + 7 * m, seed + 7 * m + 1) for m in range(M)]


def _wide(members):
    """One network equal to the mean of the members (per species)."""
    M = len(members)
    out = []
    for s in range(len(members[0])):
        L = [mem[s] for mem in members]
        W1 = np.concatenate([l[0][0] for l in L], axis=1)
        b1 = np.concatenate([l[0][1] for l in L])
        layers = [(W1, b1)]
        for k in (1, 2):
            blocks = [l[k][0] for l in L]
            fi, fo = blocks[0].shape
            W = np.zeros((M * fi, M * fo))
            for m, B in enumerate(blocks):
                W[m * fi:(m + 1) * fi, m * fo:(m + 1) * fo] = B
            layers.append((W, np.concatenate([l[k][1] for l in L])))
        W4 = np.concatenate([l[3][0] for l in L], axis=0) / M
        b4 = np.array([np.mean([l[3][1][0] for l in L])])
        layers.append((W4, b4))
        out.append(layers)
    return out


def test_ensemble_is_one_block_network(oracle_mod):
    M = 3
    mem = _members(M, 501)
    p = oracle_mod.Params()
    models = [oracle_mod.Model(p, w) for w in mem]
    wide = oracle_mod.Model(oracle_mod.Params(hidden=(160 * M, 128 * M, 96 * M)), _wide(mem))
    s = synth.water_box(27, 502)
    sp = p.species_of(s.Z)
    E, Ei, F = oracle_mod.ensemble_energy_forces(models, s.pos, sp, s.box)
    Ew, Eiw, Fw, _ = oracle_mod.energy_forces(wide, s.pos, sp, s.box)
    assert abs(E - Ew) <= 1e-11 * np.abs(Eiw).sum()
    assert np.abs(Ei - Eiw).max() <= 1e-12 * max(1.0, np.abs(Eiw).max())
    assert np.abs(F - Fw).max() <= 1e-11
    # and the members really differ, so the mean is not a copy of one of them
    E0 = oracle_mod.energy_forces(models[0], s.pos, sp, s.box)[0]
    assert abs(E0 - E) > 1e-3 * np.abs(Ei).sum() / len(Ei)


def test_copies_equal_the_single_network(oracle_mod):
    w = weights32(2, 128, 511, 512)
    p = oracle_mod.Params()
    m = oracle_mod.Model(p, w)
    s = synth.water_box(8, 513)
    sp = p.species_of(s.Z)
    E1, Ei1, F1, _ = oracle_mod.energy_forces(m, s.pos, sp, s.box)
    E, Ei, F = oracle_mod.ensemble_energy_forces([m] * 4, s.pos, sp, s.box)
    assert abs(E - E1) <= 1e-12 * np.abs(Ei1).sum()
    assert np.abs(F - F1).max() <= 1e-12


def test_ensemble_forces_are_finite_differences(oracle_mod):
    p = oracle_mod.Params()
    models = [oracle_mod.Model(p, w) for w in _members(2, 521)]
    s = synth.water_box(8, 522)
    sp = p.species_of(s.Z)
    _, _, F = oracle_mod.ensemble_energy_forces(models, s.pos, sp, s.box)
    h = 1e-5
    for a in (0, 7, 19):
        for c in range(3):
            pp, pm = s.pos.copy(), s.pos.copy()
            pp[a, c] += h
            pm[a, c] -= h
            fd = -(oracle_mod.ensemble_energy_forces(models, pp, sp, s.box)[0]
                   - oracle_mod.ensemble_energy_forces(models, pm, sp, s.box)[0]) / (2 * h)
            assert abs(F[a, c] - fd) <= 1e-6 * max(1.0, abs(fd))


def _ens_loss(oracle_mod, p, members, pos, sp, box, Fref):
    models = [oracle_mod.Model(p, w) for w in members]
    F = oracle_mod.ensemble_energy_forces(models, pos, sp, box)[2]
    return ((F - Fref) ** 2).sum() / (3 * pos.shape[0])


def test_ensemble_force_match_finite_differences(oracle_mod):
    M = 2
    mem = _members(M, 531)
    p = oracle_mod.Params()
    s = synth.water_box(8, 532)
    sp = p.species_of(s.Z)
    Fref = 0.3 * np.random.default_rng(533).standard_normal((s.n, 3))
    models = [oracle_mod.Model(p, w) for w in mem]
    L, dW, db, F = oracle_mod.ensemble_force_match(models, s.pos, sp, s.box, Fref)
    assert L == _ens_loss(oracle_mod, p, mem, s.pos, sp, s.box, Fref) or \
        abs(L - _ens_loss(oracle_mod, p, mem, s.pos, sp, s.box, Fref)) <= 1e-13 * L
    rng = np.random.default_rng(534)
    for m in range(M):
        for s_ in range(2):
            for l in range(4):
                ref = mem[m][s_][l][0]
                dirn = rng.normal(size=ref.shape)
                dirn /= np.linalg.norm(dirn)
                analytic = float((dW[m][s_][l] * dirn).sum())
                errs = []
                for h in (1e-5, 1e-6):
                    def shifted(sign):
                        out = [[list(x) for x in wm] for wm in mem]
                        W, b = mem[m][s_][l]
                        out[m][s_][l] = (W + sign * h * dirn, b)
                        return [[tuple(x) for x in wm] for wm in out]
                    fd = (_ens_loss(oracle_mod, p, shifted(1), s.pos, sp, s.box, Fref) -
                          _ens_loss(oracle_mod, p, shifted(-1), s.pos, sp, s.box, Fref)) / (2 * h)
                    errs.append(abs(analytic - fd) / max(abs(fd), 1e-6))
                assert min(errs) < 1e-6, (m, s_, l, errs)
        assert all(np.all(db[m][s_][3] == 0) for s_ in range(2))


def test_ensemble_force_match_is_the_wide_networks(oracle_mod):
    M = 3
    mem = _members(M, 541)
    p = oracle_mod.Params()
    s = synth.water_box(8, 542)
    sp = p.species_of(s.Z)
    Fref = 0.3 * np.random.default_rng(543).standard_normal((s.n, 3))
    L, dW, db, _ = oracle_mod.ensemble_force_match([oracle_mod.Model(p, w) for w in mem],
                                                    s.pos, sp, s.box, Fref)
    wide = oracle_mod.Model(oracle_mod.Params(hidden=(160 * M, 128 * M, 96 * M)), _wide(mem))
    Lw, dWw, dbw, _ = oracle_mod.force_match(wide, s.pos, sp, s.box, Fref)
    assert abs(L - Lw) <= 1e-12 * Lw
    scale = np.abs(np.concatenate([x.ravel() for x in dWw[0]])).max()
    tol = 1e-10 * scale
    for m in range(M):
        for s_ in range(2):
            c1, c2, c3 = slice(160 * m, 160 * (m + 1)), slice(128 * m, 128 * (m + 1)), slice(96 * m, 96 * (m + 1))
            assert np.abs(dW[m][s_][0] - dWw[s_][0][:, c1]).max() <= tol
            assert np.abs(dW[m][s_][1] - dWw[s_][1][c1, c2]).max() <= tol
            assert np.abs(dW[m][s_][2] - dWw[s_][2][c2, c3]).max() <= tol
            assert np.abs(dW[m][s_][3] - dWw[s_][3][c3] / M).max() <= tol
            assert np.abs(db[m][s_][0] - dbw[s_][0][c1]).max() <= tol
            assert np.abs(db[m][s_][1] - dbw[s_][1][c2]).max() <= tol
            assert np.abs(db[m][s_][2] - dbw[s_][2][c3]).max() <= tol
