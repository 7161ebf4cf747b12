"""GPU tests of the electrostatic embedding (nnp_eval_ee): ML charges from a
second per-element network, shifted to the total charge, in Coulomb
interaction with MM point charges (TIP3P-like waters: O -0.834 e, H
+0.417 e).

Bounds (FP32 form): the Coulomb sums cancel strongly over neutral waters,
so their FP32 rounding scales with the sum of the terms' magnitudes, not
with the result.  The energy error is normalised by
max(|E|, sum_i |E_i| + k_e sum_i sum_J |q'_i Q_J| / r_iJ) and held to 1e-6;
forces on ML and MM atoms to 1e-4 eV/A; charges to 1e-6 e.  BF16 form: the
network bounds of the BF16 tests (1e-2 relative energy, 0.1 eV/A).

* a periodic 27-water box (6 ML waters) and the same as an isolated
  cluster, against the FP64 oracle, host and device buffers;
* a four-species box (H/C/N/O clusters as ML, waters as MM), FP32 and BF16;
* no MM charges reproduces nnp_eval and conserves the total charge;
* an ensemble of two energy networks with the charge network, FP32 and BF16;
* refusals: no FLAG_CHARGES, missing charge weights, FP8.
"""
import numpy as np
import pytest

import synth
from common import F_ABS_TOL, box9, weights32

pytestmark = pytest.mark.gpu
K_E = 14.3996454784
TIP3P = np.array([-0.834, 0.417, 0.417])


@pytest.fixture(scope="module")
def P():
    from paper_2604_21441_b300 import build
    build.build()
    import paper_2604_21441_b300 as P
    return P


def _f32(w):
    return [[(W.astype(np.float32), b.astype(np.float32)) for W, b in sp] for sp in w]


def _charge_weights(S, D, seed):
    wq = weights32(S, D, seed, seed + 1)
    return [[(W if l < 3 else 0.2 * W, b if l < 3 else 0.2 * b) for l, (W, b) in enumerate(sp)] for sp in wq]


def _pot(P, w, wq, Zs=(1, 8), prec="fp32", **kw):
    pot = P.NNP(atomic_numbers=Zs, precision=prec, flags=P.FLAG_CHARGES, **kw)
    pot.set_all_weights(_f32(w))
    pot.set_charge_weights(_f32(wq))
    return pot


def _oracle(oracle_mod, w, wq, Zs, pos, Z, box, mm_pos, mm_q, Q):
    p = oracle_mod.Params(atomic_numbers=Zs)
    m, mq = oracle_mod.Model(p, w), oracle_mod.Model(p, wq)
    sp = p.species_of(Z)
    E, F, Fmm, q = oracle_mod.ee_energy_forces(m, mq, pos, sp, box, mm_pos, mm_q, total_charge=Q)
    _, Ei, _, _ = oracle_mod.energy_forces(m, pos, sp, box)
    return E, F, Fmm, q, max(abs(E), np.abs(Ei).sum() + _coulomb_scale(pos, q, mm_pos, mm_q, box))


def _coulomb_scale(pos, q, mm_pos, mm_q, box):
    """k_e sum_i sum_J |q_i Q_J| / r_iJ: the magnitude of the Coulomb sum's terms."""
    total = 0.0
    for i in range(len(pos)):
        d = mm_pos - pos[i]
        if box is not None:
            d -= box * np.round(d / box)
        total += K_E * np.sum(np.abs(q[i] * mm_q) / np.sqrt((d * d).sum(axis=1)))
    return total


def _water_split(seed, n_ml=6, n=27):
    s = synth.water_box(n, seed)
    k = 3 * n_ml
    return s, s.pos[:k], s.Z[:k], s.pos[k:], np.tile(TIP3P, n - n_ml)


@pytest.mark.parametrize("periodic", [True, False])
def test_ee_water_vs_oracle(P, oracle_mod, periodic):
    s, pos, Z, mm_pos, mm_q = _water_split(901)
    box = s.box if periodic else None
    w, wq = weights32(2, 128, 902, 903), _charge_weights(2, 128, 904)
    pot = _pot(P, w, wq)
    E, F, Fmm, q = pot.eval_ee(pos, Z, mm_pos, mm_q, box=None if box is None else box9(box), total_charge=0.25)
    Er, Fr, Fmr, qr, scale = _oracle(oracle_mod, w, wq, (1, 8), pos, Z, box, mm_pos, mm_q, 0.25)
    print(f"ee water (periodic={periodic}): rel E {abs(E - Er) / scale:.2e}, max|dF| {np.abs(F - Fr).max():.2e},"
          f" max|dFmm| {np.abs(Fmm - Fmr).max():.2e}, max|dq| {np.abs(q - qr).max():.2e}")
    assert abs(E - Er) <= 1e-6 * scale
    assert np.abs(F - Fr).max() <= F_ABS_TOL
    assert np.abs(Fmm - Fmr).max() <= F_ABS_TOL
    assert np.abs(q - qr).max() <= 1e-6
    assert abs(q.sum() - 0.25) <= 1e-9
    # device buffers give the same result
    import torch
    t = lambda a: torch.tensor(a, device="cuda")
    E2, F2, Fm2, q2 = pot.eval_ee(t(pos), t(Z), t(mm_pos), t(mm_q), box=None if box is None else box9(box),
                                  total_charge=0.25)
    assert abs(float(E2) - E) <= 1e-6 * scale
    assert np.abs(F2.cpu().numpy() - F).max() <= 1e-5 and np.abs(Fm2.cpu().numpy() - Fmm).max() <= 1e-5


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_ee_four_species(P, oracle_mod, prec):
    Zs = (1, 6, 7, 8)
    s = synth.hcno_box(911, L=16.0, n_cluster_atoms=120, max_waters=60)
    ncl = s.meta["n_cluster_atoms"]
    pos, Z = s.pos[:ncl], s.Z[:ncl]
    mm_pos = s.pos[ncl:]
    mm_q = np.tile(TIP3P, len(mm_pos) // 3)
    w, wq = weights32(4, 384, 912, 913), _charge_weights(4, 384, 914)
    pot = _pot(P, w, wq, Zs=Zs, prec=prec)
    E, F, Fmm, q = pot.eval_ee(pos, Z, mm_pos, mm_q, box=box9(s.box), total_charge=-1.0)
    Er, Fr, Fmr, qr, scale = _oracle(oracle_mod, w, wq, Zs, pos, Z, s.box, mm_pos, mm_q, -1.0)
    print(f"ee 4 species {prec} ({ncl} ML, {len(mm_pos)} MM): rel E {abs(E - Er) / scale:.2e},"
          f" max|dF| {np.abs(F - Fr).max():.2e}, max|dFmm| {np.abs(Fmm - Fmr).max():.2e},"
          f" max|dq| {np.abs(q - qr).max():.2e}")
    if prec == "fp32":
        assert abs(E - Er) <= 1e-6 * scale
        assert np.abs(F - Fr).max() <= F_ABS_TOL and np.abs(Fmm - Fmr).max() <= F_ABS_TOL
        assert np.abs(q - qr).max() <= 1e-6
    else:
        assert abs(E - Er) <= 1e-2 * scale
        assert np.abs(F - Fr).max() <= 0.1 and np.abs(Fmm - Fmr).max() <= 0.1
        assert np.abs(q - qr).max() <= 1e-2
    assert abs(q.sum() + 1.0) <= 1e-9


def test_ee_without_mm_is_plain_eval(P):
    s = synth.water_box(64, 921)
    w, wq = weights32(2, 128, 922, 923), _charge_weights(2, 128, 924)
    pot = _pot(P, w, wq)
    E, F, Fmm, q = pot.eval_ee(s.pos, s.Z, np.zeros((0, 3)), np.zeros(0), box=box9(s.box), total_charge=1.5)
    E0, F0 = pot.eval(s.pos, s.Z, box9(s.box))
    Ei = pot.atom_energies(s.n)
    assert abs(E - E0) <= 1e-7 * np.abs(Ei).sum() and np.abs(F - F0).max() <= 1e-5
    assert Fmm.shape == (0, 3) and abs(q.sum() - 1.5) <= 1e-9


def test_ee_refusals(P):
    s, pos, Z, mm_pos, mm_q = _water_split(931)
    w, wq = weights32(2, 128, 932), _charge_weights(2, 128, 933)
    plain = P.NNP(atomic_numbers=(1, 8))
    plain.set_all_weights(_f32(w))
    with pytest.raises(P.NNPError) as e:
        plain.eval_ee(pos, Z, mm_pos, mm_q)
    assert e.value.code == 3
    pot = P.NNP(atomic_numbers=(1, 8), flags=P.FLAG_CHARGES)
    pot.set_all_weights(_f32(w))
    with pytest.raises(P.NNPError) as e:
        pot.eval_ee(pos, Z, mm_pos, mm_q)
    assert e.value.code == 7
    pot.set_charge_weights(_f32(wq))
    E, F, Fmm, q = pot.eval_ee(pos, Z, mm_pos, mm_q)
    assert np.isfinite(E)
    with pytest.raises(P.NNPError) as e:
        P.NNP(atomic_numbers=(1, 8), precision="fp8", flags=P.FLAG_CHARGES)
    assert e.value.code == 3


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_ee_with_ensemble(P, oracle_mod, prec):
    """Two energy networks (their mean) plus the charge network: the charge
    network is the weight set after the ensemble's and stays out of the
    members' launch.  Oracle: the embedding terms with member 0, its NNP part
    replaced by the ensemble's."""
    s, pos, Z, mm_pos, mm_q = _water_split(941)
    mem = [weights32(2, 128, 942 + 5 * m, 943 + 5 * m) for m in range(2)]
    wq = _charge_weights(2, 128, 951)
    pot = P.NNP(atomic_numbers=(1, 8), precision=prec, flags=P.FLAG_CHARGES, n_members=2)
    pot.set_member_weights([_f32(w) for w in mem])
    pot.set_charge_weights(_f32(wq))
    E, F, Fmm, q = pot.eval_ee(pos, Z, mm_pos, mm_q, box=box9(s.box), total_charge=0.0)
    p = oracle_mod.Params()
    sp = p.species_of(Z)
    models = [oracle_mod.Model(p, w) for w in mem]
    Ee, Fe, Fmr, qr = oracle_mod.ee_energy_forces(models[0], oracle_mod.Model(p, wq), pos, sp, s.box, mm_pos, mm_q)
    E0, _, F0, _ = oracle_mod.energy_forces(models[0], pos, sp, s.box)
    Em, Eim, Fm = oracle_mod.ensemble_energy_forces(models, pos, sp, s.box)
    Er, Fr = Ee - E0 + Em, Fe - F0 + Fm
    scale = max(abs(Er), np.abs(Eim).sum() + _coulomb_scale(pos, qr, mm_pos, mm_q, s.box))
    tolE, tolF = (1e-6, F_ABS_TOL) if prec == "fp32" else (1e-2, 0.1)
    print(f"ee + ensemble {prec}: rel E {abs(E - Er) / scale:.2e}, max|dF| {np.abs(F - Fr).max():.2e},"
          f" max|dFmm| {np.abs(Fmm - Fmr).max():.2e}")
    assert abs(E - Er) <= tolE * scale
    assert np.abs(F - Fr).max() <= tolF and np.abs(Fmm - Fmr).max() <= tolF
    assert np.abs(q - qr).max() <= (1e-6 if prec == "fp32" else 1e-2)
