"""Pins of the oracle at seven species (H, C, N, O, F, S, Cl: the element set
of the ANI-2x model, D = 16 * 7 + 32 * 28 = 1008).

* The radial terms of an F-Cl dimer sit in the blocks of the partner's
  species and equal the closed form 1/4 exp(-eta (r - R_m)^2) fc(r); every
  other entry is zero.
* Water seen by a seven-species model equals water seen by a two-species
  (H, O) model whose first-layer rows are the seven-species rows of the H
  and O blocks (radial blocks 0 and 3, angular blocks p(0,0) = 0,
  p(0,3) = 3, p(3,3) = 18 of the row-major upper triangle), whatever the
  rows of the absent species hold: energies and forces agree to rounding.
* Forces in a seven-element box equal central finite differences.
"""
import math

import numpy as np

import synth
from common import weights32

Z7 = (1, 6, 7, 8, 9, 16, 17)
SHF_R = [0.9 + 0.26875 * m for m in range(16)]


def test_dimer_blocks_closed_form(oracle_mod):
    p = oracle_mod.Params(atomic_numbers=Z7)
    assert p.aev_length == 1008
    m = oracle_mod.Model(p, weights32(7, 1008, 601))
    r = 2.6  # fc(5.2 / 2) = 1/2; beyond the angular cutoff's pairs (one neighbour only)
    pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    Z = np.array([9, 17])
    _, _, _, G = oracle_mod.energy_forces(m, pos, p.species_of(Z), None)
    ref = np.array([0.25 * math.exp(-16.0 * (r - R) ** 2) * 0.5 for R in SHF_R])
    # F (species 4) sees Cl (species 6): radial block 6; Cl sees F: block 4
    for atom, block in ((0, 6), (1, 4)):
        g = G[atom]
        assert np.allclose(g[16 * block:16 * block + 16], ref, rtol=1e-13, atol=0.0)
        rest = np.delete(g, np.arange(16 * block, 16 * block + 16))
        assert np.all(rest == 0.0)


def _pair7(a, b):
    S = 7
    return a * S - a * (a - 1) // 2 + (b - a)


def test_water_in_seven_species_model(oracle_mod):
    w7 = weights32(7, 1008, 611, 612)
    rows = np.concatenate([np.arange(0, 16), np.arange(48, 64)] +
                          [112 + 32 * _pair7(a, b) + np.arange(32) for a, b in ((0, 0), (0, 3), (3, 3))])
    assert [_pair7(a, b) for a, b in ((0, 0), (0, 3), (3, 3))] == [0, 3, 18]
    w2 = []
    for s7 in (0, 3):  # H and O networks
        layers = [(w7[s7][0][0][rows].copy(), w7[s7][0][1])] + list(w7[s7][1:])
        w2.append(layers)
    m7 = oracle_mod.Model(oracle_mod.Params(atomic_numbers=Z7), w7)
    p2 = oracle_mod.Params(atomic_numbers=(1, 8))
    m2 = oracle_mod.Model(p2, w2)
    s = synth.water_box(27, 613)
    E7, Ei7, F7, _ = oracle_mod.energy_forces(m7, s.pos, m7.p.species_of(s.Z), s.box)
    E2, Ei2, F2, _ = oracle_mod.energy_forces(m2, s.pos, p2.species_of(s.Z), s.box)
    assert abs(E7 - E2) <= 1e-12 * np.abs(Ei2).sum()
    assert np.abs(F7 - F2).max() <= 1e-12


def test_seven_element_forces_finite_differences(oracle_mod):
    s = synth.hcno_box(621, L=12.0, n_cluster_atoms=60, max_waters=20,
                       elements=synth.ANI2X_Z, probs=synth.ANI2X_P)
    p = oracle_mod.Params(atomic_numbers=Z7)
    m = oracle_mod.Model(p, weights32(7, 1008, 622, 623))
    sp = p.species_of(s.Z)
    assert len(set(sp.tolist())) >= 6
    E, Ei, F, _ = oracle_mod.energy_forces(m, s.pos, sp, s.box)
    h = 1e-5
    for a in np.random.default_rng(1).choice(s.n, 6, replace=False):
        for c in range(3):
            pp, pm = s.pos.copy(), s.pos.copy()
            pp[a, c] += h
            pm[a, c] -= h
            fd = -(oracle_mod.energy_forces(m, pp, sp, s.box)[0] - oracle_mod.energy_forces(m, pm, sp, s.box)[0]) / (2 * h)
            assert abs(F[a, c] - fd) <= 2e-7 * max(1.0, np.abs(F).max()), (a, c, F[a, c], fd)
    assert np.abs(F.sum(axis=0)).max() <= 1e-9
