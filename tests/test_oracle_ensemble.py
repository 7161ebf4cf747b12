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
