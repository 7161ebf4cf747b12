"""GPU tests of nnp_eval_pairs: neighbour lists from a caller's pair list
(Methods: the 2026 nnpot interface passes the MD engine's pair list) instead
of the library's cell search.

* a buffered half list (every pair within 6 A once, with its periodic shift)
  gives the FP64 oracle's energy and forces within the FP32 bounds, and the
  same result as the cell search up to the order of FP32 sums (|dE| <= 1e-9
  relative would be bitwise; the list order follows atomics, so 1e-6 relative
  and 1e-5 eV/A);
* the order of the pairs and the direction of each pair ((j, i, -s) for
  (i, j, s)) do not matter;
* an isolated cluster takes a list without shifts;
* the 12,288-atom box with a k-d-tree list matches the cell search;
* an index out of range or a shift that is not a whole image is rejected,
  and the context keeps working.
"""
import numpy as np
import pytest

import synth
from common import E_REL_TOL, F_ABS_TOL, box9, energy_error, weights32

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


def _half_list(oracle_mod, pos, box, rc=6.0):
    """Every pair within rc once (i < j), with its shift s: d = r_j - r_i + s."""
    pi, pj, pd = oracle_mod.pairs_brute(pos, box, rc)
    keep = pi < pj
    pairs = np.stack([pi[keep], pj[keep]], axis=1).astype(np.int32)
    shifts = pd[keep] - (pos[pj[keep]] - pos[pi[keep]])
    return pairs, shifts


def test_pairs_water64_vs_oracle_and_search(P, oracle_mod):
    s = synth.water_box(64, synth.GEOM_SEED[1])
    w = weights32(2, 128, synth.WEIGHT_SEED[1], 7)
    pot = _pot(P, w)
    pairs, shifts = _half_list(oracle_mod, s.pos, s.box)
    E, F = pot.eval_pairs(s.pos, s.Z, pairs, shifts, box9(s.box))
    p = oracle_mod.Params()
    m = oracle_mod.Model(p, w)
    Er, Eir, Fr, _ = oracle_mod.energy_forces(m, s.pos, p.species_of(s.Z), s.box)
    print(f"pair list water-64: rel E err {energy_error(E, Er, Eir):.2e}, max|dF| {np.abs(F - Fr).max():.2e},"
          f" {len(pairs)} pairs")
    assert energy_error(E, Er, Eir) <= E_REL_TOL
    assert np.abs(F - Fr).max() <= F_ABS_TOL
    Es, Fs = pot.eval(s.pos, s.Z, box9(s.box))
    assert abs(E - Es) <= 1e-6 * np.abs(Eir).sum() and np.abs(F - Fs).max() <= 1e-5
    # order and direction of the pairs do not matter
    rng = np.random.default_rng(3)
    perm = rng.permutation(len(pairs))
    flip = rng.random(len(pairs)) < 0.5
    pairs2 = pairs[perm].copy()
    shifts2 = shifts[perm].copy()
    pairs2[flip] = pairs2[flip][:, ::-1]
    shifts2[flip] = -shifts2[flip]
    E2, F2 = pot.eval_pairs(s.pos, s.Z, pairs2, shifts2, box9(s.box))
    assert abs(E2 - E) <= 1e-6 * np.abs(Eir).sum() and np.abs(F2 - F).max() <= 1e-5


def test_pairs_device_pointers(P, oracle_mod):
    import torch
    s = synth.water_box(216, 61)
    w = weights32(2, 128, 62, 63)
    pairs, shifts = _half_list(oracle_mod, s.pos, s.box)
    a = _pot(P, w)
    t = lambda x: torch.tensor(x, device="cuda")
    E, F = a.eval_pairs(t(s.pos), t(s.Z), t(pairs), t(shifts), box9(s.box))
    Es, Fs = a.eval(t(s.pos), t(s.Z), box9(s.box))
    Ei = a.atom_energies(s.n)
    assert abs(float(E) - float(Es)) <= 1e-6 * np.abs(Ei).sum()
    assert (F - Fs).abs().max().item() <= 1e-5


def test_pairs_isolated_cluster(P, oracle_mod):
    s = synth.water_box(64, 64)
    centre = 0.5 * s.box
    order = np.argsort(np.linalg.norm(s.pos[0::3] - centre, axis=1))[:16]
    atoms = np.sort(np.concatenate([3 * order, 3 * order + 1, 3 * order + 2]))
    pos, Z = s.pos[atoms] - centre, s.Z[atoms]
    w = weights32(2, 128, 65, 66)
    pot = _pot(P, w)
    pi, pj, _ = oracle_mod.pairs_brute(pos, None, 6.0)
    keep = pi < pj
    pairs = np.stack([pi[keep], pj[keep]], axis=1).astype(np.int32)
    E, F = pot.eval_pairs(pos, Z, pairs, None, None)
    p = oracle_mod.Params()
    m = oracle_mod.Model(p, w)
    Er, Eir, Fr, _ = oracle_mod.energy_forces(m, pos, p.species_of(Z), None)
    assert energy_error(E, Er, Eir) <= E_REL_TOL
    assert np.abs(F - Fr).max() <= F_ABS_TOL


def test_pairs_water4096_matches_search(P):
    """12,288 atoms: a k-d-tree half list with minimum-image shifts."""
    from scipy.spatial import cKDTree
    wl = synth.workload(2)
    s = wl["systems"][0]
    w = weights32(2, 128, wl["weight_seed"])
    L = s.box
    wrapped = np.mod(s.pos, L)
    ij = cKDTree(wrapped, boxsize=L).query_pairs(5.6, output_type="ndarray")
    d = s.pos[ij[:, 1]] - s.pos[ij[:, 0]]
    shifts = -L * np.round(d / L)
    # FP32 form: the BF16 form rounds G, so a different sum order can move a
    # value across a BF16 rounding boundary and compare no better than its own error
    pot = _pot(P, w, max_atoms=s.n)
    E, F = pot.eval_pairs(s.pos, s.Z, ij.astype(np.int32), shifts, box9(L))
    Es, Fs = pot.eval(s.pos, s.Z, box9(L))
    Ei = pot.atom_energies(s.n)
    print(f"pair list water-4096: {len(ij)} pairs, |dE|/sum|Ei| {abs(E - Es) / np.abs(Ei).sum():.1e},"
          f" max|dF| {np.abs(F - Fs).max():.1e}")
    assert abs(E - Es) <= 1e-6 * np.abs(Ei).sum()
    assert np.abs(F - Fs).max() <= 1e-5


def test_pairs_rejects_bad_lists(P, oracle_mod):
    s = synth.water_box(64, 67)
    w = weights32(2, 128, 68)
    pot = _pot(P, w)
    pairs, shifts = _half_list(oracle_mod, s.pos, s.box)
    bad = pairs.copy()
    bad[5, 1] = s.n  # out of range
    with pytest.raises(P.NNPError):
        pot.eval_pairs(s.pos, s.Z, bad, shifts, box9(s.box))
    off = shifts.copy()
    k = int(np.argmin(np.linalg.norm(s.pos[pairs[:, 1]] - s.pos[pairs[:, 0]] + shifts, axis=1)))
    off[k] += np.array([0.3 * s.box[0], 0.0, 0.0])  # not a whole image, still within the cutoff
    with pytest.raises(P.NNPError):
        pot.eval_pairs(s.pos, s.Z, pairs, off, box9(s.box))
    E, F = pot.eval_pairs(s.pos, s.Z, pairs, shifts, box9(s.box))
    Es, _ = pot.eval(s.pos, s.Z, box9(s.box))
    assert np.isfinite(E) and abs(E - Es) <= 1e-5 * max(1.0, abs(Es))


def test_pairs_empty_list_is_isolated_atoms(P, oracle_mod):
    """No pairs: every atom alone, G = 0, so E = sum over atoms of its
    species' network at zero input, and all forces vanish."""
    s = synth.water_box(27, 69)
    w = weights32(2, 128, 70, 71)
    pot = _pot(P, w)
    E, F = pot.eval_pairs(s.pos, s.Z, np.zeros((0, 2), dtype=np.int32), None, box9(s.box))
    p = oracle_mod.Params()
    m = oracle_mod.Model(p, w)
    e0 = [oracle_mod.mlp(m, sp, np.zeros(p.aev_length))[0] for sp in range(2)]
    ref = sum(e0[sp] for sp in p.species_of(s.Z))
    assert abs(E - ref) <= 1e-6 * max(1.0, abs(ref))
    assert np.all(F == 0.0)


def test_pairs_fp8_form(P, oracle_mod):
    """The FP8 form calibrates through the same path (the caller's list)."""
    s = synth.water_box(64, 72)
    w = weights32(2, 128, 73, 74)
    pairs, shifts = _half_list(oracle_mod, s.pos, s.box)
    a = _pot(P, w, "fp8")
    E, F = a.eval_pairs(s.pos, s.Z, pairs, shifts, box9(s.box))
    b = _pot(P, w, "fp8")
    Es, Fs = b.eval(s.pos, s.Z, box9(s.box))
    Ei = b.atom_energies(s.n)
    # same neighbour sets, so the same calibration and (up to sum order) the same result
    assert abs(E - Es) <= 1e-3 * np.abs(Ei).sum() and np.abs(F - Fs).max() <= 0.05
