"""Pins of the oracle's general periodic cell (triclinic boxes; rows of the
3 x 3 cell are the cell vectors).

* a rectangular cell given as a 3 x 3 matrix gives the same pairs, energy
  and forces as the edge-length form;
* the same lattice described by a sheared cell (a unimodular change of cell
  vectors) gives the same energy and forces: the wrap and the image range
  are right whatever the cell's shape;
* one atom in a primitive FCC cell has the textbook shells within the cutoff
  (12 at a/sqrt2, 6 at a, 24 at a sqrt(3/2), 12 at a sqrt2, 24 at a sqrt(5/2));
* forces in a skewed box equal central finite differences of the energy.
"""
import numpy as np

import synth


def _model(oracle_mod, seed=71):
    p = oracle_mod.Params(atomic_numbers=(1, 8))
    w = synth.random_biases(synth.xavier_weights(p.n_species, p.aev_length, seed), seed + 1)
    return p, oracle_mod.Model(p, w)


def _pair_set(pi, pj, pd):
    return sorted(zip(pi.tolist(), pj.tolist(), np.round(pd, 9).tolist()))


def test_rectangular_cell_equals_edges(oracle_mod):
    p, m = _model(oracle_mod)
    s = synth.water_box(8, 72)
    cell = np.diag(s.box)
    a = oracle_mod.pairs_brute(s.pos, s.box, 5.2)
    b = oracle_mod.pairs_brute_cell(s.pos, cell, 5.2)
    assert _pair_set(*a) == _pair_set(*b)
    sp = p.species_of(s.Z)
    E1, _, F1, _ = oracle_mod.energy_forces(m, s.pos, sp, s.box)
    E2, _, F2, _ = oracle_mod.energy_forces(m, s.pos, sp, cell)
    assert abs(E1 - E2) <= 1e-12 * max(1.0, abs(E1)) and np.abs(F1 - F2).max() <= 1e-10


def test_sheared_cell_of_the_same_lattice(oracle_mod):
    p, m = _model(oracle_mod)
    s = synth.water_box(27, 73)
    a, b, c = np.diag(s.box)
    sheared = np.array([a, b + a, c + a - b])  # determinant 1 change of cell vectors
    sp = p.species_of(s.Z)
    E1, _, F1, _ = oracle_mod.energy_forces(m, s.pos, sp, np.diag(s.box))
    E2, _, F2, _ = oracle_mod.energy_forces(m, s.pos, sp, sheared)
    assert abs(E1 - E2) <= 1e-10 * max(1.0, abs(E1))
    assert np.abs(F1 - F2).max() <= 1e-9


def test_fcc_shells(oracle_mod):
    A = 3.0
    cell = 0.5 * A * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    pi, pj, pd = oracle_mod.pairs_brute_cell(np.zeros((1, 3)), cell, 5.0)
    r = np.sort(np.linalg.norm(pd, axis=1))
    radii = A * np.sqrt(np.array([0.5, 1.0, 1.5, 2.0, 2.5]))
    counts = [int(np.sum(np.abs(r - x) < 1e-9)) for x in radii]
    assert counts == [12, 6, 24, 12, 24]
    assert len(r) == sum(counts)


def test_skewed_box_forces_are_finite_differences(oracle_mod):
    p, m = _model(oracle_mod, 74)
    s = synth.water_box(8, 75)
    L = s.box[0]
    cell = np.array([[L, 0.0, 0.0], [0.23 * L, 0.97 * L, 0.0], [-0.15 * L, 0.31 * L, 1.02 * L]])
    sp = p.species_of(s.Z)
    E, _, F, _ = oracle_mod.energy_forces(m, s.pos, sp, cell)
    h = 1e-5
    rng = np.random.default_rng(0)
    for a in rng.choice(s.n, 6, replace=False):
        for c in range(3):
            pp, pm = s.pos.copy(), s.pos.copy()
            pp[a, c] += h
            pm[a, c] -= h
            fd = -(oracle_mod.energy_forces(m, pp, sp, cell)[0] - oracle_mod.energy_forces(m, pm, sp, cell)[0]) / (2 * h)
            assert abs(F[a, c] - fd) <= 1e-6 * max(1.0, abs(fd)), (a, c, F[a, c], fd)
    assert np.abs(F.sum(axis=0)).max() <= 1e-9
