"""Pins of the oracle's electrostatic embedding (ML charges from a second
per-element network, shifted to the total charge, in Coulomb interaction
with MM point charges).

* One ML atom and one MM charge: the neutrality shift makes the ML charge
  the total charge Q whatever the network says, so E_es = k Q q / r exactly,
  the MM force is k Q q / r^2 along the axis, and the ML force is its
  opposite (a lone atom has no NNP force).
* MM charges all zero: the plain NNP's energy and forces, no MM forces, and
  the charges still sum to Q.
* The total force on ML and MM atoms vanishes (translation invariance of
  E_NNP + E_es), isolated and in a box with minimum images.
* Forces on ML and on MM atoms equal central finite differences of the
  energy.
"""
import numpy as np
import pytest

import synth
from common import weights32

K_E = 14.3996454784


def _models(oracle_mod, seed=801):
    p = oracle_mod.Params()
    w = weights32(2, 128, seed, seed + 1)
    wq = weights32(2, 128, seed + 2, seed + 3)
    wq = [[(W if l < 3 else 0.2 * W, b if l < 3 else 0.2 * b) for l, (W, b) in enumerate(sp)] for sp in wq]
    return p, oracle_mod.Model(p, w), oracle_mod.Model(p, wq)


def _split(seed, n_ml_waters=6, n_waters=27):
    """ML: the first waters of a box; MM: the other waters as TIP3P charges."""
    s = synth.water_box(n_waters, seed)
    k = 3 * n_ml_waters
    mm_q = np.tile([-0.834, 0.417, 0.417], n_waters - n_ml_waters)
    return s, s.pos[:k], s.Z[:k], s.pos[k:], mm_q


def test_single_pair_closed_form(oracle_mod):
    p, m, mq = _models(oracle_mod)
    r = 3.7
    pos = np.array([[0.3, -0.2, 0.5]])
    mm = pos + np.array([[r, 0.0, 0.0]])
    E, F, Fmm, q = oracle_mod.ee_energy_forces(m, mq, pos, p.species_of([8]), None, mm, [0.6], total_charge=-0.8)
    e0 = oracle_mod.mlp(m, 1, np.zeros(p.aev_length))[0]
    assert q[0] == pytest.approx(-0.8, abs=1e-15)
    assert E == pytest.approx(e0 + K_E * (-0.8) * 0.6 / r, rel=1e-14)
    fmag = K_E * (-0.8) * 0.6 / r ** 2
    assert np.allclose(Fmm[0], [fmag, 0.0, 0.0], rtol=1e-13, atol=1e-15)
    assert np.allclose(F[0], -Fmm[0], rtol=1e-13, atol=1e-15)


def test_zero_mm_charges_is_plain_nnp(oracle_mod):
    p, m, mq = _models(oracle_mod)
    s, pos, Z, mm_pos, mm_q = _split(811)
    sp = p.species_of(Z)
    E, F, Fmm, q = oracle_mod.ee_energy_forces(m, mq, pos, sp, None, mm_pos, 0.0 * mm_q, total_charge=0.5)
    E0, _, F0, _ = oracle_mod.energy_forces(m, pos, sp, None)
    assert E == pytest.approx(E0, rel=1e-14) and np.abs(F - F0).max() <= 1e-12
    assert np.all(Fmm == 0.0)
    assert q.sum() == pytest.approx(0.5, abs=1e-12)


@pytest.mark.parametrize("periodic", [False, True])
def test_total_force_vanishes(oracle_mod, periodic):
    p, m, mq = _models(oracle_mod, 821)
    s, pos, Z, mm_pos, mm_q = _split(822)
    box = s.box if periodic else None
    E, F, Fmm, q = oracle_mod.ee_energy_forces(m, mq, pos, p.species_of(Z), box, mm_pos, mm_q)
    tot = F.sum(axis=0) + Fmm.sum(axis=0)
    assert np.abs(tot).max() <= 1e-10 * max(1.0, np.abs(F).max())
    assert abs(q.sum()) <= 1e-12
    assert np.abs(Fmm).max() > 1e-3  # the embedding does act


@pytest.mark.parametrize("periodic", [False, True])
def test_forces_are_finite_differences(oracle_mod, periodic):
    p, m, mq = _models(oracle_mod, 831)
    s, pos, Z, mm_pos, mm_q = _split(832)
    box = s.box if periodic else None
    sp = p.species_of(Z)
    E, F, Fmm, _ = oracle_mod.ee_energy_forces(m, mq, pos, sp, box, mm_pos, mm_q, total_charge=0.3)
    h = 1e-5
    energy = lambda x, y: oracle_mod.ee_energy_forces(m, mq, x, sp, box, y, mm_q, total_charge=0.3)[0]
    for a in (0, 4, 11):
        for c in range(3):
            xp, xm = pos.copy(), pos.copy()
            xp[a, c] += h
            xm[a, c] -= h
            fd = -(energy(xp, mm_pos) - energy(xm, mm_pos)) / (2 * h)
            assert abs(F[a, c] - fd) <= 1e-6 * max(1.0, abs(fd)), (a, c, F[a, c], fd)
    for j in (0, 7, 20):
        for c in range(3):
            yp, ym = mm_pos.copy(), mm_pos.copy()
            yp[j, c] += h
            ym[j, c] -= h
            fd = -(energy(pos, yp) - energy(pos, ym)) / (2 * h)
            assert abs(Fmm[j, c] - fd) <= 1e-6 * max(1.0, abs(fd)), (j, c, Fmm[j, c], fd)
