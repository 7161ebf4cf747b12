"""GPU parity for triclinic boxes (rows of the 3 x 3 box are the cell
vectors): the cell grid is sized by the cell's heights, atoms are wrapped
through fractional coordinates, and image shifts are sums of cell steps.

* the same lattice in a sheared cell gives the orthorhombic evaluation's
  energy and forces (FP32 form, up to FP32 rounding of the cell-local
  offsets and the order of sums), at 192 and 12,288 atoms;
* a skewed box (a different periodic system) matches the FP64 oracle's
  general-cell evaluation within the FP32 bounds;
* a caller's pair list in a skewed box gives the cell search's result.
"""
import numpy as np
import pytest

import synth
from common import E_REL_TOL, F_ABS_TOL, energy_error, weights32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2604_21441_b300 import build
    build.build()
    import paper_2604_21441_b300 as P
    return P


def _pot(P, w, prec="fp32", **kw):
    pot = P.NNP(atomic_numbers=(1, 8), precision=prec, **kw)
    pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in sp] for sp in w])
    return pot


def _sheared(L):
    a, b, c = np.diag(L)
    return np.array([a, b + a, c + b])


def _skewed(L):
    return np.array([[L[0], 0.0, 0.0], [0.2 * L[1], 0.98 * L[1], 0.0], [-0.1 * L[2], 0.25 * L[2], 1.0 * L[2]]])


@pytest.mark.parametrize("waters,seed", [(64, 81), (4096, None)])
def test_sheared_cell_equals_orthorhombic(P, waters, seed):
    if seed is None:
        wl = synth.workload(2)
        s = wl["systems"][0]
        w = weights32(2, 128, wl["weight_seed"])
    else:
        s = synth.water_box(waters, seed)
        w = weights32(2, 128, seed + 1, seed + 2)
    pot = _pot(P, w, max_atoms=s.n)
    E0, F0 = pot.eval(s.pos, s.Z, np.diag(s.box))
    Ei = pot.atom_energies(s.n)
    E1, F1 = pot.eval(s.pos, s.Z, _sheared(s.box))
    print(f"sheared cell, {s.n} atoms: |dE|/sum|Ei| {abs(E1 - E0) / np.abs(Ei).sum():.1e}, "
          f"max|dF| {np.abs(F1 - F0).max():.1e}")
    # the two cell grids store different FP32 offsets of each atom from its
    # cell's corner (a few A, rounded to ~5e-7 A), so the displacements differ
    # in the last bits as well as the order of the sums; both evaluations stay
    # within the FP32 form's 1e-4 eV/A of the exact forces
    assert abs(E1 - E0) <= 1e-6 * np.abs(Ei).sum()
    assert np.abs(F1 - F0).max() <= 5e-5


def test_skewed_box_vs_oracle(P, oracle_mod):
    s = synth.water_box(64, 83)
    w = weights32(2, 128, 84, 85)
    cell = _skewed(s.box)
    pot = _pot(P, w)
    E, F = pot.eval(s.pos, s.Z, cell)
    p = oracle_mod.Params()
    m = oracle_mod.Model(p, w)
    Er, Eir, Fr, _ = oracle_mod.energy_forces(m, s.pos, p.species_of(s.Z), cell)
    print(f"skewed box: rel E err {energy_error(E, Er, Eir):.2e}, max|dF| {np.abs(F - Fr).max():.2e}")
    assert energy_error(E, Er, Eir) <= E_REL_TOL
    assert np.abs(F - Fr).max() <= F_ABS_TOL
    # BF16 form on the same box, within its own bounds
    b = _pot(P, w, "bf16")
    Eb, Fb = b.eval(s.pos, s.Z, cell)
    assert energy_error(Eb, Er, Eir) <= 1e-2 and np.abs(Fb - Fr).max() <= 0.1


def test_skewed_box_pair_list(P, oracle_mod):
    s = synth.water_box(64, 86)
    w = weights32(2, 128, 87, 88)
    cell = _skewed(s.box)
    pi, pj, pd = oracle_mod.pairs_brute_cell(s.pos, cell, 6.0)
    keep = pi < pj
    pairs = np.stack([pi[keep], pj[keep]], axis=1).astype(np.int32)
    shifts = pd[keep] - (s.pos[pj[keep]] - s.pos[pi[keep]])
    pot = _pot(P, w)
    E, F = pot.eval_pairs(s.pos, s.Z, pairs, shifts, cell)
    Es, Fs = pot.eval(s.pos, s.Z, cell)
    Ei = pot.atom_energies(s.n)
    assert abs(E - Es) <= 1e-6 * np.abs(Ei).sum() and np.abs(F - Fs).max() <= 1e-5


def test_triclinic_batch(P):
    """Two skewed systems and one orthorhombic one in one batched launch equal
    their separate evaluations."""
    w = weights32(2, 128, 89, 90)
    systems = [synth.water_box(64, 91), synth.water_box(27, 92), synth.water_box(125, 93)]
    cells = [_skewed(systems[0].box), np.diag(systems[1].box), _sheared(systems[2].box)]
    pot = _pot(P, w)
    off = np.concatenate([[0], np.cumsum([s.n for s in systems])])
    pos = np.concatenate([s.pos for s in systems])
    Z = np.concatenate([s.Z for s in systems])
    Eb, Fb = pot.eval_batch(off, pos, Z, np.stack(cells))
    for k, (s, c) in enumerate(zip(systems, cells)):
        E, F = pot.eval(s.pos, s.Z, c)
        assert abs(Eb[k] - E) <= 1e-6 * max(1.0, abs(E))
        assert np.abs(Fb[off[k]:off[k + 1]] - F).max() <= 1e-5
