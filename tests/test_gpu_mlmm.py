"""GPU parity of the ML/MM mechanical embedding (nnp_eval_mlmm) against the
FP64 oracle: the ML group of a periodic water box plus link atoms on cut
O-H bonds, one of them stored across the box boundary.

FP32 form: the same bounds as the plain evaluation (|dE| / max(|E|, sum
|E_i|) <= 1e-6, max |dF| <= 1e-4 eV/A), on every atom of the whole system;
atoms outside the group and not bonded to a link must get exactly zero.
Host and device pointers give the same result; invalid index sets are
rejected on the host with NNP_ERR_INVALID_ARG.
"""
import numpy as np
import pytest

import synth
from common import E_REL_TOL, F_ABS_TOL, box9, weights32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2604_21441_b300 import build
    build.build()
    import paper_2604_21441_b300 as P
    return P


def _pot(P, w, prec="fp32"):
    pot = P.NNP(atomic_numbers=(1, 8), precision=prec)
    pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in sp] for sp in w])
    return pot


def _embedding(n_waters=64, seed=41, group_waters=24):
    s = synth.water_box(n_waters, seed)
    pos = s.pos.copy()
    # cut O-H bonds: waters 3, 8 and 17 keep their O in the group, their first H is MM
    cut = [3, 8, 17]
    ml = [a for a in range(3 * group_waters) if not (a % 3 == 1 and a // 3 in cut)]
    link_ml = [3 * w for w in cut]
    link_mm = [3 * w + 1 for w in cut]
    pos[link_mm[1]] += np.array([s.box[0], 0.0, 0.0])  # one bond stored across the boundary
    link_d = [1.0, 0.95, 1.05]
    return s, pos, np.array(ml, dtype=np.int64), np.array(link_ml, dtype=np.int64), \
        np.array(link_mm, dtype=np.int64), np.array(link_d)


def _oracle(oracle_mod, w, s, pos, ml, lml, lmm, ld):
    p = oracle_mod.Params(atomic_numbers=(1, 8))
    m = oracle_mod.Model(p, w)
    sp = p.species_of(s.Z)
    return oracle_mod.mlmm_energy_forces(m, pos, sp, s.box, ml, lml, lmm, ld, 0)


def test_mlmm_fp32_vs_oracle(P, oracle_mod):
    w = weights32(2, 128, 42, 43)
    s, pos, ml, lml, lmm, ld = _embedding()
    pot = _pot(P, w)
    E, F = pot.eval_mlmm(pos, s.Z, ml, lml, lmm, ld, 1, box=box9(s.box))
    Er, Fr, Eir = _oracle(oracle_mod, w, s, pos, ml, lml, lmm, ld)
    err_e = abs(E - Er) / max(abs(Er), float(np.abs(Eir).sum()))
    err_f = np.abs(F - Fr).max()
    print(f"ML/MM fp32: rel E err {err_e:.2e}, max|dF| {err_f:.2e} ({len(ml)} group atoms, {len(lml)} links)")
    assert err_e <= E_REL_TOL
    assert err_f <= F_ABS_TOL
    outside = np.setdiff1d(np.arange(s.n), np.concatenate([ml, lmm]))
    assert np.all(F[outside] == 0.0)
    assert np.all(F[lmm] != 0.0)  # the MM atoms of the links receive their share
    assert np.abs(F.sum(axis=0)).max() <= 1e-4


def test_mlmm_device_pointers_and_repeat(P):
    import torch
    w = weights32(2, 128, 44, 45)
    s, pos, ml, lml, lmm, ld = _embedding(seed=46)
    pot = _pot(P, w)
    E1, F1 = pot.eval_mlmm(pos, s.Z, ml, lml, lmm, ld, 1, box=box9(s.box))
    t = lambda a: torch.tensor(a, device="cuda")
    E2, F2 = pot.eval_mlmm(t(pos), t(s.Z), t(ml), t(lml), t(lmm), t(ld), 1, box=box9(s.box))
    F2 = F2.cpu().numpy()
    # FP32 force sums by atomic reductions inside the NNP: the last bits vary
    assert abs(float(E2) - E1) <= 1e-9 * abs(E1)
    assert np.abs(F2 - F1).max() <= 1e-5


def test_mlmm_bf16(P, oracle_mod):
    w = weights32(2, 128, 47, 48)
    s, pos, ml, lml, lmm, ld = _embedding(seed=49)
    pot = _pot(P, w, "bf16")
    E, F = pot.eval_mlmm(pos, s.Z, ml, lml, lmm, ld, 1, box=box9(s.box))
    Er, Fr, Eir = _oracle(oracle_mod, w, s, pos, ml, lml, lmm, ld)
    # the BF16 form's own bounds (relative energy 1e-2, forces max 0.1 eV/A)
    assert abs(E - Er) / max(abs(Er), float(np.abs(Eir).sum())) <= 1e-2
    assert np.abs(F - Fr).max() <= 0.1


def test_mlmm_rejects_bad_index_sets(P):
    w = weights32(2, 128, 50)
    s, pos, ml, lml, lmm, ld = _embedding(seed=51)
    pot = _pot(P, w)
    with pytest.raises(P.NNPError):  # repeated group index
        pot.eval_mlmm(pos, s.Z, np.concatenate([ml, ml[:1]]), lml, lmm, ld, 1, box=box9(s.box))
    with pytest.raises(P.NNPError):  # link whose MM atom is in the group
        pot.eval_mlmm(pos, s.Z, ml, lml, np.array([0, 4, 7]), ld, 1, box=box9(s.box))
    with pytest.raises(P.NNPError):  # index out of range
        pot.eval_mlmm(pos, s.Z, np.append(ml, s.n), lml, lmm, ld, 1, box=box9(s.box))
    with pytest.raises(P.NNPError):  # non-positive link distance
        pot.eval_mlmm(pos, s.Z, ml, lml, lmm, np.array([1.0, 0.0, 1.0]), 1, box=box9(s.box))
    # device-resident index sets are checked by kernels and rejected the same way
    import torch
    t = lambda a: torch.tensor(a, device="cuda")
    with pytest.raises(P.NNPError):
        pot.eval_mlmm(t(pos), t(s.Z), t(np.concatenate([ml, ml[:1]])), t(lml), t(lmm), t(ld), 1,
                      box=box9(s.box))
    with pytest.raises(P.NNPError):
        pot.eval_mlmm(t(pos), t(s.Z), t(ml), t(lml), t(np.array([0, 4, 7])), t(ld), 1, box=box9(s.box))
    with pytest.raises(P.NNPError):
        pot.eval_mlmm(t(pos), t(s.Z), t(np.append(ml, s.n)), t(lml), t(lmm), t(ld), 1, box=box9(s.box))
    # the context still evaluates after the rejections
    E, F = pot.eval_mlmm(pos, s.Z, ml, lml, lmm, ld, 1, box=box9(s.box))
    assert np.isfinite(E) and np.isfinite(F).all()


def test_mlmm_open_cluster(P, oracle_mod):
    """No box: an isolated cluster of 12 waters with two cut bonds."""
    w = weights32(2, 128, 52, 53)
    s = synth.water_box(64, 54)
    centre = 0.5 * s.box
    order = np.argsort(np.linalg.norm(s.pos[0::3] - centre, axis=1))[:12]  # the 12 central waters
    atoms = np.sort(np.concatenate([3 * order, 3 * order + 1, 3 * order + 2]))
    pos = s.pos[atoms] - centre
    assert np.all(np.linalg.norm(pos[1::3] - pos[0::3], axis=1) < 1.1)  # whole molecules
    Z = s.Z[atoms]
    ml = np.array([a for a in range(len(atoms)) if a not in (1, 4)], dtype=np.int64)
    lml, lmm = np.array([0, 3], dtype=np.int64), np.array([1, 4], dtype=np.int64)
    pot = _pot(P, w)
    E, F = pot.eval_mlmm(pos, Z, ml, lml, lmm, None, 1, box=None)
    p = oracle_mod.Params(atomic_numbers=(1, 8))
    m = oracle_mod.Model(p, w)
    Er, Fr, Eir = oracle_mod.mlmm_energy_forces(m, pos, p.species_of(Z), None, ml, lml, lmm, None, 0)
    assert abs(E - Er) / max(abs(Er), float(np.abs(Eir).sum())) <= E_REL_TOL
    assert np.abs(F - Fr).max() <= F_ABS_TOL


def test_mlmm_without_links_is_the_group(P):
    """No cut bonds: the embedding is the plain evaluation of the group."""
    w = weights32(2, 128, 55, 56)
    s = synth.water_box(64, 57)
    ml = np.arange(3 * 20, dtype=np.int64)  # 20 whole waters
    pot = _pot(P, w)
    E, F = pot.eval_mlmm(s.pos, s.Z, ml, (), (), None, 1, box=box9(s.box))
    Eg, Fg = pot.eval(s.pos[ml], s.Z[ml], box9(s.box))
    assert abs(E - Eg) <= 1e-9 * max(1.0, abs(Eg))
    assert np.abs(F[ml] - Fg).max() <= 1e-5 and np.all(F[3 * 20:] == 0.0)
