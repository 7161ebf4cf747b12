"""GPU force-matching weight gradients against the FP64 oracle.

L = |F - Fref|^2 / (3N) with Fref from an independently seeded teacher
network (oracle), or seeded random reference forces on the full-size box.
The GPU computes F and dL/dtheta in FP32 (FP32 sums over 256-row segments,
added into the FP64 gradient).  Bounds, about three times the measured errors:
relative loss error <= 2e-6; gradient max-abs error, relative to the largest
gradient entry, <= 2e-5 on the small systems (measured <= 7e-6) and <= 2e-4
on the 6,134-atom workload (measured 5.8e-5); relative L2 error <= 1.5e-5
(small, measured <= 4.5e-6) and <= 1e-4 (full size, measured 2.4e-5).
"""
GRAD_MAX, GRAD_L2 = 2e-5, 1.5e-5          # small systems
GRAD_MAX_FULL, GRAD_L2_FULL = 2e-4, 1e-4  # the 6,134-atom workload
LOSS_REL = 2e-6
import numpy as np
import pytest

import synth
from common import (E_REL_TOL, F_ABS_TOL, box9, energy_error, oracle_energy_forces_job,
                    oracle_force_match_job, weights32)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2604_21441_b300 import build
    build.build()
    import paper_2604_21441_b300 as P
    return P


def _pack(dW, db):
    parts = []
    for sW, sb in zip(dW, db):
        for W, b in zip(sW, sb):
            parts += [np.asarray(W).reshape(-1), np.asarray(b).reshape(-1)]
    return np.concatenate(parts)


@pytest.mark.parametrize("kind", ["hcno", "water"])
def test_force_match_gradient(P, oracle_mod, kind):
    if kind == "hcno":
        s = synth.hcno_box(55, L=16.0, n_cluster_atoms=120, max_waters=60)
        Zs = (1, 6, 7, 8)
    else:
        s = synth.water_box(64, 1001)
        Zs = (1, 8)
    p = oracle_mod.Params(atomic_numbers=Zs)
    w = weights32(len(Zs), p.aev_length, 31, 32)
    wt = weights32(len(Zs), p.aev_length, 33, 34)
    sp = p.species_of(s.Z)
    Fref = oracle_mod.energy_forces(oracle_mod.Model(p, wt), s.pos, sp, s.box)[2]
    Lr, dW, db, Fo = oracle_mod.force_match(oracle_mod.Model(p, w), s.pos, sp, s.box, Fref)
    gref = _pack(dW, db)
    pot = P.NNP(atomic_numbers=Zs)
    pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in x] for x in w])
    assert pot.param_count() == gref.size
    pot.eval(s.pos, s.Z, box9(s.box))
    L, g = pot.force_match_grad(Fref=Fref, want_loss=True)
    err_max = np.abs(g - gref).max() / np.abs(gref).max()
    err_l2 = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    print(f"{kind}: L {L:.6e} ref {Lr:.6e} (rel {abs(L - Lr) / Lr:.2e}); grad max err {err_max:.2e}, "
          f"rel L2 {err_l2:.2e}")
    assert abs(L - Lr) <= LOSS_REL * Lr
    assert err_max <= GRAD_MAX and err_l2 <= GRAD_L2
    # the v = dL/dF entry point gives the same gradient
    n = s.n
    F, _ = Fo, None
    v = 2.0 * (Fo - Fref) / (3 * n)
    g2 = pot.force_match_grad(v=v)
    assert np.abs(g2 - g).max() <= 1e-4 * np.abs(g).max()
    # b4 has no effect on forces: its gradient is exactly 0
    per = g.size // len(Zs)
    assert all(g[(k + 1) * per - 1] == 0.0 for k in range(len(Zs)))


def test_force_match_workload5_full_size(P, oracle_mod):
    """The four-species workload at full size: H/C/N/O clusters of 2,000 atoms
    in water, 40 A box, 6,134 atoms, D = 384.  H has 3,651 rows, so each of
    its weight-gradient tiles adds the sums of fifteen 256-row segments.
    Reference forces: seeded random, RMS 0.3 eV/A (the loss and its gradient
    are defined for any reference).  Energy and every force in FP32 bounds,
    then L and dL/dtheta against the oracle."""
    import concurrent.futures as cf
    import multiprocessing as mp
    wl = synth.workload(5)
    s = wl["systems"][0]
    Zs = tuple(int(z) for z in wl["atomic_numbers"])
    p = oracle_mod.Params(atomic_numbers=Zs)
    sp = p.species_of(s.Z)
    assert np.bincount(sp)[0] > 2048
    w = weights32(len(Zs), p.aev_length, wl["weight_seed"], 51)
    Fref = 0.3 * np.random.default_rng(52).standard_normal((s.n, 3))
    with cf.ProcessPoolExecutor(2, mp_context=mp.get_context("spawn")) as ex:
        f_ef = ex.submit(oracle_energy_forces_job, Zs, w, s.pos, s.Z, s.box)
        f_fm = ex.submit(oracle_force_match_job, Zs, w, s.pos, s.Z, s.box, Fref)
        Er, Eir, Fr = f_ef.result()
        Lr, dW, db, Fo = f_fm.result()
        gref = _pack(dW, db)
    pot = P.NNP(atomic_numbers=Zs, max_atoms=s.n)
    pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in x] for x in w])
    E, F = pot.eval(s.pos, s.Z, box9(s.box))
    err_e, err_f = energy_error(E, Er, Eir), np.abs(F - Fr).max()
    L, g = pot.force_match_grad(Fref=Fref, want_loss=True)
    err_l = abs(L - Lr) / Lr
    err_max = np.abs(g - gref).max() / np.abs(gref).max()
    err_l2 = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    print(f"workload 5 ({s.n} atoms): rel E {err_e:.2e}, max|dF| {err_f:.2e}; L rel {err_l:.2e}, "
          f"grad max err {err_max:.2e} of max entry, rel L2 {err_l2:.2e}")
    assert err_e <= E_REL_TOL and err_f <= F_ABS_TOL
    assert np.abs(Fo - Fr).max() <= 1e-10
    assert err_l <= LOSS_REL
    assert err_max <= GRAD_MAX_FULL and err_l2 <= GRAD_L2_FULL



def test_force_match_ensemble(P, oracle_mod):
    """Three networks averaged (the ANI-2x form): the loss of the mean force,
    member by member gradients (member-major in the packed vector) against
    the oracle's ensemble gradient; FP32 form and a BF16 context (whose
    gradient path is FP32 too)."""
    s = synth.water_box(64, 1001)
    Zs = (1, 8)
    M = 3
    p = oracle_mod.Params(atomic_numbers=Zs)
    members = [weights32(2, p.aev_length, 61 + 2 * m, 62 + 2 * m) for m in range(M)]
    sp = p.species_of(s.Z)
    Fref = 0.3 * np.random.default_rng(63).standard_normal((s.n, 3))
    Lr, dW, db, Fr = oracle_mod.ensemble_force_match([oracle_mod.Model(p, w) for w in members],
                                                      s.pos, sp, s.box, Fref)
    gref = np.concatenate([_pack(dW[m], db[m]) for m in range(M)])
    for prec in ("fp32", "bf16"):
        pot = P.NNP(atomic_numbers=Zs, precision=prec, n_members=M)
        for m in range(M):
            pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in x]
                                 for x in members[m]], m)
        assert pot.param_count() == gref.size
        pot.eval(s.pos, s.Z, box9(s.box))
        L, g = pot.force_match_grad(Fref=Fref, want_loss=True)
        err_max = np.abs(g - gref).max() / np.abs(gref).max()
        err_l2 = np.linalg.norm(g - gref) / np.linalg.norm(gref)
        print(f"ensemble M={M} ({prec} context): L rel {abs(L - Lr) / Lr:.2e}, grad max err {err_max:.2e}, "
              f"rel L2 {err_l2:.2e}")
        assert abs(L - Lr) <= LOSS_REL * Lr
        assert err_max <= GRAD_MAX and err_l2 <= GRAD_L2
        pot.close()


def test_force_match_seven_species(P, oracle_mod):
    """The seven elements of ANI-2x (D = 1,008): H, C, N, O, F, S, Cl clusters
    in water, 16 A box."""
    s = synth.hcno_box(757, L=16.0, n_cluster_atoms=160, max_waters=60,
                       elements=synth.ANI2X_Z, probs=synth.ANI2X_P)
    Zs = tuple(int(z) for z in sorted(synth.ANI2X_Z))
    p = oracle_mod.Params(atomic_numbers=Zs)
    sp = p.species_of(s.Z)
    assert len(np.unique(sp)) == 7
    w = weights32(7, p.aev_length, 71, 72)
    Fref = 0.3 * np.random.default_rng(73).standard_normal((s.n, 3))
    Lr, dW, db, Fo = oracle_mod.force_match(oracle_mod.Model(p, w), s.pos, sp, s.box, Fref)
    gref = _pack(dW, db)
    pot = P.NNP(atomic_numbers=Zs)
    pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in x] for x in w])
    assert pot.param_count() == gref.size
    pot.eval(s.pos, s.Z, box9(s.box))
    L, g = pot.force_match_grad(Fref=Fref, want_loss=True)
    err_max = np.abs(g - gref).max() / np.abs(gref).max()
    err_l2 = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    print(f"seven species ({s.n} atoms): L rel {abs(L - Lr) / Lr:.2e}, grad max err {err_max:.2e}, "
          f"rel L2 {err_l2:.2e}")
    assert abs(L - Lr) <= LOSS_REL * Lr
    assert err_max <= GRAD_MAX and err_l2 <= GRAD_L2


def test_force_match_stage_profile(P):
    """nnp_profile_force_match reports four positive stage durations; the
    gradient written into a caller's device buffer equals the host one."""
    s = synth.water_box(64, 1001)
    w = weights32(2, 128, 81, 82)
    pot = P.NNP(atomic_numbers=(1, 8), flags=P.FLAG_STAGE_EVENTS)
    pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in x] for x in w])
    pot.eval(s.pos, s.Z, box9(s.box))
    with pytest.raises(P.NNPError):
        pot.profile_force_match()
    g_host = pot.force_match_grad(Fref=np.zeros((s.n, 3)))
    t = pot.profile_force_match()
    assert len(t) == 4 and all(x > 0 for x in t), t
    # into a caller's device buffer, twice (the job list is reused): the same gradient
    import torch
    out = torch.zeros(pot.param_count(), dtype=torch.float64, device="cuda")
    for _ in range(2):
        g_dev = pot.force_match_grad(Fref=np.zeros((s.n, 3)), out=out)
        assert g_dev is out
        assert np.abs(out.cpu().numpy() - g_host).max() <= 1e-12 * np.abs(g_host).max()
