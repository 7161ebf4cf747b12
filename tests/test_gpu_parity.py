"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

FP32 form bounds: |dE| / max(|E|, sum_i |E_i|) <= 1e-6 and max |dF| <= 1e-4
eV/A.  Small systems are compared atom by atom in full; the full-size water
boxes (12,288 and 98,304 atoms, in the configuration the benchmark times)
on sampled atoms that the oracle evaluates one by one, plus properties that
hold at any size (sum F = 0, E = sum E_i).
"""
import numpy as np
import pytest

import synth
from common import E_REL_TOL, F_ABS_TOL, box9, energy_error, oracle_subset, targeted_atoms, weights32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2604_21441_b300 import build
    build.build()
    import paper_2604_21441_b300 as P
    return P


def _pot(P, weights, Zs=(1, 8), **kw):
    pot = P.NNP(atomic_numbers=Zs, **kw)
    pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in sp]
                         for sp in weights])
    return pot


def _oracle(oracle_mod, weights, Zs=(1, 8)):
    p = oracle_mod.Params(atomic_numbers=Zs)
    return p, oracle_mod.Model(p, weights)


def _compare(pot, oracle_mod, weights, pos, Z, box, Zs=(1, 8), device=False):
    p, m = _oracle(oracle_mod, weights, Zs)
    Er, Eir, Fr, _ = oracle_mod.energy_forces(m, pos, p.species_of(Z), box)
    if device:
        import torch
        E, F = pot.eval(torch.tensor(pos, device="cuda"), torch.tensor(Z, device="cuda"), box9(box))
        E, F = float(E), F.cpu().numpy()
    else:
        E, F = pot.eval(pos, Z, box9(box))
    Ei = pot.atom_energies(len(Z))
    err_e = energy_error(E, Er, Eir)
    err_f = np.abs(F - Fr).max()
    assert err_e <= E_REL_TOL, (err_e, E, Er)
    assert err_f <= F_ABS_TOL, (err_f, np.sqrt((Fr ** 2).mean()))
    assert np.abs(Ei - Eir).max() <= 1e-5 * max(1.0, np.abs(Eir).max())
    return err_e, err_f


@pytest.mark.parametrize("bias", [False, True])
@pytest.mark.parametrize("device", [False, True])
def test_water64(P, oracle_mod, bias, device):
    s = synth.water_box(64, synth.GEOM_SEED[1])
    w = weights32(2, 128, synth.WEIGHT_SEED[1], 7 if bias else None)
    pot = _pot(P, w)
    _compare(pot, oracle_mod, w, s.pos, s.Z, s.box, device=device)


@pytest.mark.parametrize("n_waters", [8, 16, 27, 125])
def test_small_boxes_multi_image(P, oracle_mod, n_waters):
    """Boxes of 6.2 to 15.5 A: one or two cells per edge, several images of
    the same neighbour within the cutoff."""
    s = synth.water_box(n_waters, 300 + n_waters)
    w = weights32(2, 128, 11, 12)
    _compare(_pot(P, w), oracle_mod, w, s.pos, s.Z, s.box)


def test_orthorhombic_unwrapped(P, oracle_mod):
    rng = np.random.default_rng(5)
    box = np.array([7.3, 11.9, 16.4])
    n = 150
    pos = rng.uniform(0, 1, size=(n, 3)) * box
    keep = [0]
    for i in range(1, n):  # drop atoms closer than 0.8 A (min image)
        d = pos[keep] - pos[i]
        d -= box * np.round(d / box)
        if np.min(np.einsum("ij,ij->i", d, d)) > 0.64:
            keep.append(i)
    pos = pos[keep]
    Z = rng.choice([1, 8], size=len(keep)).astype(np.int32)
    pos_unwrapped = pos + rng.integers(-2, 3, size=pos.shape) * box
    w = weights32(2, 128, 13, 14)
    _compare(_pot(P, w), oracle_mod, w, pos_unwrapped, Z, box)


def test_isolated_cluster(P, oracle_mod):
    s = synth.water_box(64, 21)
    pos, Z = s.pos[:90] + 40.0, s.Z[:90]
    w = weights32(2, 128, 15, 16)
    _compare(_pot(P, w), oracle_mod, w, pos, Z, None)


def test_four_species(P, oracle_mod):
    s = synth.hcno_box(77, L=16.0, n_cluster_atoms=120, max_waters=60)
    w = weights32(4, 384, 17, 18)
    _compare(_pot(P, w, Zs=(1, 6, 7, 8)), oracle_mod, w, s.pos, s.Z, s.box, Zs=(1, 6, 7, 8))


def test_batch(P, oracle_mod):
    systems = [synth.water_box(n, 40 + n) for n in (16, 9, 40, 27, 64)]
    w = weights32(2, 128, 19, 20)
    pot = _pot(P, w, max_systems=8)
    off = np.cumsum([0] + [s.n for s in systems])
    pos = np.concatenate([s.pos for s in systems])
    Z = np.concatenate([s.Z for s in systems])
    E, F = pot.eval_batch(off, pos, Z, np.stack([s.box for s in systems]))
    p, m = _oracle(oracle_mod, w)
    for b, s in enumerate(systems):
        Er, Eir, Fr, _ = oracle_mod.energy_forces(m, s.pos, p.species_of(s.Z), s.box)
        assert energy_error(E[b], Er, Eir) <= E_REL_TOL
        assert np.abs(F[off[b]:off[b + 1]] - Fr).max() <= F_ABS_TOL


def test_capacity_regrowth(P, oracle_mod):
    s = synth.water_box(64, synth.GEOM_SEED[1])
    w = weights32(2, 128, 23, 24)
    pot = _pot(P, w, nbr_capacity=16, ang_capacity=4)
    _compare(pot, oracle_mod, w, s.pos, s.Z, s.box)
    assert pot.query("nbr_capacity") > 16 and pot.query("ang_capacity") > 4
    assert pot.query("max_nbr") <= pot.query("nbr_capacity")


def test_graph_and_direct_launches_agree(P):
    s = synth.water_box(64, 3)
    w = weights32(2, 128, 25, 26)
    a = _pot(P, w)
    b = _pot(P, w, flags=P.FLAG_NO_GRAPH)
    c = _pot(P, w, flags=P.FLAG_NONDETERMINISTIC_BINS)
    Ea, Fa = a.eval(s.pos, s.Z, s.box)
    for _ in range(3):
        Eb, Fb = b.eval(s.pos, s.Z, s.box)
        Ea2, Fa2 = a.eval(s.pos, s.Z, s.box)
        # energies: FP64 sums of per-warp partials; forces: FP64 reductions
        # of FP32 terms, whose order (and last bits) vary from launch to launch
        assert abs(Ea2 - Ea) <= 1e-12 * abs(Ea) and np.abs(Fa2 - Fa).max() < 1e-11
        assert abs(Eb - Ea) <= 1e-12 * abs(Ea) and np.abs(Fb - Fa).max() < 1e-11
    Ec, Fc = c.eval(s.pos, s.Z, s.box)
    # another row order changes the FP32 sums inside each descriptor
    assert abs(Ec - Ea) <= 1e-7 * abs(Ea) and np.abs(Fc - Fa).max() < 1e-5
    assert a.query("graph_captures") == 1
    # cells (one block for a system this small), neighbours, descriptor,
    # network, descriptor backward
    assert a.query("launches_per_eval") == 5


def test_error_codes(P):
    s = synth.water_box(27, 4)
    w = weights32(2, 128, 27, None)
    pot = _pot(P, w)
    bad = s.Z.copy()
    bad[5] = 6
    with pytest.raises(P.NNPError) as e:
        pot.eval(s.pos, bad, s.box)
    assert e.value.code == 2
    nanpos = s.pos.copy()
    nanpos[3, 1] = np.nan
    with pytest.raises(P.NNPError) as e:
        pot.eval(nanpos, s.Z, s.box)
    assert e.value.code == 1
    L = s.box[0]
    thin = np.array([[L, 0.0, 0.0], [0.95 * L, 0.3 * L, 0.0], [0.0, 0.0, L]])  # a height of 0.3 L < rc
    with pytest.raises(P.NNPError) as e:
        pot.eval(s.pos, s.Z, thin)
    assert e.value.code == 3
    left = np.diag(s.box)[[1, 0, 2]]  # left-handed cell
    with pytest.raises(P.NNPError) as e:
        pot.eval(s.pos, s.Z, left)
    assert e.value.code == 1
    with pytest.raises(P.NNPError) as e:
        pot.eval(s.pos, s.Z, [5.0, 9.3, 9.3])
    assert e.value.code == 3
    empty = P.NNP(atomic_numbers=(1, 8))
    with pytest.raises(P.NNPError) as e:
        empty.eval(s.pos, s.Z, s.box)
    assert e.value.code == 7
    # the context still works after errors
    E, F = pot.eval(s.pos, s.Z, s.box)
    assert np.isfinite(E) and np.all(np.isfinite(F))


@pytest.mark.parametrize("k", [2, 3])
def test_full_size_sampled(P, oracle_mod, k):
    """12,288 / 98,304 atoms, device-resident inputs, graph replay (the
    benchmark's configuration): E_i and F_j against the oracle on 128 random
    atoms plus the atoms at the box faces and corners (neighbours through
    periodic images, edge cells) and the 32 atoms with the most angular
    neighbours."""
    import torch
    wl = synth.workload(k)
    s = wl["systems"][0]
    w = weights32(2, 128, wl["weight_seed"])
    pot = _pot(P, w, max_atoms=s.n)
    pos = torch.tensor(s.pos, device="cuda")
    Z = torch.tensor(s.Z, device="cuda")
    for _ in range(2):
        E, F = pot.eval(pos, Z, box9(s.box))
    E = float(E)
    F = F.cpu().numpy()
    Ei = pot.atom_energies(s.n)
    rng = np.random.default_rng(k)
    sel = targeted_atoms(s.pos, s.box, rng)
    assert len(sel) >= 160
    Eir, Fr = oracle_subset((1, 8), w, s.pos, s.Z, s.box, sel, sel)
    err_ei = np.abs(Ei[sel] - Eir).max()
    err_f = np.abs(F[sel] - Fr).max()
    print(f"water k={k}: {len(sel)} atoms, max|dEi| {err_ei:.2e} eV, max|dF| {err_f:.2e} eV/A")
    assert err_ei <= 1e-5 * max(1.0, np.abs(Eir).max())
    assert err_f <= F_ABS_TOL
    assert abs(E - Ei.sum()) <= 1e-6 * np.abs(Ei).sum()
    assert np.abs(F.sum(0)).max() <= 1e-6 * np.abs(F).sum()


def test_dense_water_rows_beyond_the_pair_matrix(P, oracle_mod):
    """Water compressed to about twice its density: rows have more angular
    neighbours than the backward's shared-memory pair matrix holds (32), so
    those rows take the path that adds pair forces with shared-memory
    atomics.  Checked atom by atom against the oracle, FP32 bounds."""
    s = synth.water_box(64, 95)
    scale = 0.8
    pos, box = s.pos * scale, s.box * scale
    w = weights32(2, 128, 96, 97)
    pot = _pot(P, w)
    E, F = pot.eval(pos, s.Z, box9(box))
    assert pot.query("max_ang") > 32  # the path under test is taken
    p = oracle_mod.Params()
    m = oracle_mod.Model(p, w)
    Er, Eir, Fr, _ = oracle_mod.energy_forces(m, pos, p.species_of(s.Z), box)
    print(f"dense water: max angular {pot.query('max_ang')}, rel E err {energy_error(E, Er, Eir):.2e}, "
          f"max|dF| {np.abs(F - Fr).max():.2e}")
    assert energy_error(E, Er, Eir) <= E_REL_TOL
    assert np.abs(F - Fr).max() <= F_ABS_TOL


def test_page_locked_host_buffers(P, oracle_mod):
    """Page-locked host inputs are read in place by the binning kernel (no
    staging copy); pageable host and device inputs go through their own
    paths.  All three against the oracle, and against each other to the FP64
    reduction order, on a box with unwrapped coordinates."""
    import torch
    s = synth.water_box(125, 35)
    pos = s.pos + np.array([1.5, -2.0, 0.5]) * s.box  # outside the primary cell
    w = weights32(2, 128, 36, 37)
    pot = _pot(P, w, max_atoms=s.n)
    p, m = _oracle(oracle_mod, w)
    Er, Eir, Fr, _ = oracle_mod.energy_forces(m, pos, p.species_of(s.Z), s.box)
    pos_p = torch.from_numpy(np.ascontiguousarray(pos)).pin_memory()
    Z_p = torch.from_numpy(s.Z.astype(np.int32)).pin_memory()
    E_p = torch.zeros(1, dtype=torch.float64).pin_memory()
    F_p = torch.zeros((s.n, 3), dtype=torch.float64).pin_memory()
    pot.eval_into(pos_p, Z_p, box9(s.box), E_p, F_p)
    Ep, Fp = float(E_p[0]), F_p.numpy().copy()
    Eh, Fh = pot.eval(pos, s.Z, box9(s.box))  # pageable host buffers
    Ed, Fd = pot.eval(torch.tensor(pos, device="cuda"), torch.tensor(s.Z.astype(np.int32), device="cuda"),
                      box9(s.box))
    Ed, Fd = float(Ed), Fd.cpu().numpy()
    for E, F in ((Ep, Fp), (Eh, Fh), (Ed, Fd)):
        assert energy_error(E, Er, Eir) <= E_REL_TOL
        assert np.abs(F - Fr).max() <= F_ABS_TOL
    assert abs(Ep - Eh) <= 1e-9 * np.abs(Eir).sum() and np.abs(Fp - Fh).max() <= 1e-9
    assert abs(Ep - Ed) <= 1e-9 * np.abs(Eir).sum() and np.abs(Fp - Fd).max() <= 1e-9
