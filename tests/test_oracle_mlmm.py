"""Pins of the oracle's ML/MM mechanical embedding (Sec. Methods: ML group
plus link atoms r_L = r_ML + d (r_MM - r_ML) / |r_MM - r_ML|, link forces
passed on by the chain rule).

* a bond stored across the periodic boundary gives the same energy and
  forces as the same bond stored without the image (minimum image);
* the forces on every atom of the whole system equal central finite
  differences of the embedded energy taken in the whole system's coordinates
  (this checks the link placement and the chain rule together, including a
  bond that crosses the periodic boundary and a link distance other than 1 A);
* atoms neither in the group nor bonded to a link get exactly zero force;
* the net force is zero (the embedded energy is translation invariant);
* a link atom placed exactly on its MM atom (d = |R|) gives the energy of the
  plain subsystem that contains that atom with the link's species.
"""
import numpy as np

import synth


def _system(oracle_mod):
    p = oracle_mod.Params(atomic_numbers=(1, 8))
    w = synth.random_biases(synth.xavier_weights(p.n_species, p.aev_length, 21), 22)
    m = oracle_mod.Model(p, w)
    s = synth.water_box(8, 23)
    sp = p.species_of(s.Z)
    # group: waters 0-3 without the first H of waters 1 and 2 (MM, bonded to ML O atoms)
    ml = np.array([0, 1, 2, 3, 5, 6, 8, 9, 10, 11], dtype=np.int64)
    link_ml = np.array([3, 6], dtype=np.int64)
    link_mm = np.array([4, 7], dtype=np.int64)
    return p, m, s, sp, ml, link_ml, link_mm


def test_mlmm_forces_are_finite_differences(oracle_mod):
    p, m, s, sp, ml, lml, lmm = _system(oracle_mod)
    pos = s.pos.copy()
    # MM atom 7 stored one box length away from its O: the bond needs the minimum image
    pos[7] = pos[6] + np.array([0.3, -0.8, 0.5]) + np.array([s.box[0], 0.0, 0.0])
    d = np.array([1.0, 0.93])
    E, F, _ = oracle_mod.mlmm_energy_forces(m, pos, sp, s.box, ml, lml, lmm, d, 0)
    near = pos.copy()
    near[7] -= np.array([s.box[0], 0.0, 0.0])  # the same bond without the image
    E_near, F_near, _ = oracle_mod.mlmm_energy_forces(m, near, sp, s.box, ml, lml, lmm, d, 0)
    assert abs(E - E_near) <= 1e-12 * max(1.0, abs(E)) and np.abs(F - F_near).max() <= 1e-10
    h = 1e-5
    movable = sorted(set(ml.tolist()) | set(lmm.tolist()))
    for a in movable:
        for c in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[a, c] += h
            pm[a, c] -= h
            Ep, _, _ = oracle_mod.mlmm_energy_forces(m, pp, sp, s.box, ml, lml, lmm, d, 0)
            Em, _, _ = oracle_mod.mlmm_energy_forces(m, pm, sp, s.box, ml, lml, lmm, d, 0)
            fd = -(Ep - Em) / (2 * h)
            assert abs(F[a, c] - fd) <= 1e-6 * max(1.0, abs(fd)), (a, c, F[a, c], fd)
    others = [a for a in range(s.n) if a not in movable]
    assert np.all(F[others] == 0.0)
    assert np.abs(F.sum(axis=0)).max() <= 1e-9


def test_mlmm_link_on_its_mm_atom(oracle_mod):
    p, m, s, sp, ml, lml, lmm = _system(oracle_mod)
    R = np.linalg.norm(s.pos[lmm] - s.pos[lml], axis=1)  # no bond crosses the box here
    E, _, _ = oracle_mod.mlmm_energy_forces(m, s.pos, sp, s.box, ml, lml, lmm, R, 0)
    sub = np.concatenate([s.pos[ml], s.pos[lmm]])
    sub_sp = np.concatenate([sp[ml], np.zeros(len(lmm), dtype=sp.dtype)])
    Eref, _, _, _ = oracle_mod.energy_forces(m, sub, sub_sp, s.box)
    assert abs(E - Eref) <= 1e-12 * max(1.0, abs(Eref))
