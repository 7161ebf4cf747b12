"""GPU tests of the BF16 tensor-core form (tcgen05 network).

The BF16 form rounds descriptors, weights and activations to BF16 (8-bit
mantissa) and accumulates in FP32, so it is not held to the FP32 bounds.
Its measured error against the FP64 oracle is reported and must stay within
bounds derived from that rounding: relative energy error <= 1e-2 (same
normalisation as the FP32 form) and force errors max <= 0.1 eV/A, RMS <=
0.02 eV/A for forces of RMS ~0.3 eV/A.
"""
import numpy as np
import pytest

import synth
from common import box9, energy_error, weights32

pytestmark = pytest.mark.gpu

E_BF16 = 1e-2
F_MAX_BF16 = 0.1
F_RMS_BF16 = 0.02


@pytest.fixture(scope="module")
def P():
    from paper_2604_21441_b300 import build
    build.build()
    import paper_2604_21441_b300 as P
    return P


def _pot(P, w, prec, **kw):
    pot = P.NNP(atomic_numbers=(1, 8), precision=prec, **kw)
    pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in sp] for sp in w])
    return pot


def test_bf16_water64_vs_oracle(P, oracle_mod):
    s = synth.water_box(64, synth.GEOM_SEED[1])
    w = weights32(2, 128, synth.WEIGHT_SEED[1], 7)
    pot = _pot(P, w, "bf16")
    E, F = pot.eval(s.pos, s.Z, box9(s.box))
    p = oracle_mod.Params()
    m = oracle_mod.Model(p, w)
    Er, Eir, Fr, _ = oracle_mod.energy_forces(m, s.pos, p.species_of(s.Z), s.box)
    ee = energy_error(E, Er, Eir)
    dF = F - Fr
    print(f"bf16 water-64: rel E err {ee:.2e}, max|dF| {np.abs(dF).max():.3e}, "
          f"rms dF {np.sqrt((dF ** 2).mean()):.3e}, rms F {np.sqrt((Fr ** 2).mean()):.3f}")
    assert ee <= E_BF16
    assert np.abs(dF).max() <= F_MAX_BF16
    assert np.sqrt((dF ** 2).mean()) <= F_RMS_BF16
    Ei = pot.atom_energies(s.n)
    assert abs(Ei.sum() - E) <= 1e-6 * np.abs(Ei).sum()


def test_bf16_matches_fp32_form(P):
    """Same inputs through both forms: differences are BF16 rounding only,
    and repeated BF16 evaluations are stable."""
    s = synth.water_box(512, 77)
    w = weights32(2, 128, 78, 79)
    a = _pot(P, w, "fp32")
    b = _pot(P, w, "bf16")
    Ea, Fa = a.eval(s.pos, s.Z, box9(s.box))
    Eb, Fb = b.eval(s.pos, s.Z, box9(s.box))
    Eb2, Fb2 = b.eval(s.pos, s.Z, box9(s.box))
    Ei = a.atom_energies(s.n)
    assert abs(Eb - Ea) <= E_BF16 * np.abs(Ei).sum()
    assert np.abs(Fb - Fa).max() <= F_MAX_BF16
    # FP32 force sums by atomic reductions: the order, and the last bits, vary
    assert abs(Eb2 - Eb) <= 1e-9 * abs(Eb) and np.abs(Fb2 - Fb).max() <= 1e-5


def test_bf16_full_size_sampled(P, oracle_mod):
    """98,304 atoms: every SM runs several tiles (persistent loop)."""
    import torch
    wl = synth.workload(3)
    s = wl["systems"][0]
    w = weights32(2, 128, wl["weight_seed"])
    pot = _pot(P, w, "bf16", max_atoms=s.n)
    pos = torch.tensor(s.pos, device="cuda")
    Z = torch.tensor(s.Z, device="cuda")
    E, F = pot.eval(pos, Z, box9(s.box))
    F = F.cpu().numpy()
    Ei = pot.atom_energies(s.n)
    rng = np.random.default_rng(5)
    sel_e = np.sort(rng.choice(s.n, 64, replace=False))
    sel_f = np.sort(rng.choice(s.n, 12, replace=False))
    p = oracle_mod.Params()
    m = oracle_mod.Model(p, w)
    Eir, Fr = oracle_mod.energy_forces_subset(m, s.pos, p.species_of(s.Z), s.box, sel_e, sel_f)
    print(f"bf16 water-32768 sampled: max|dEi| {np.abs(Ei[sel_e] - Eir).max():.2e}, "
          f"max|dF| {np.abs(F[sel_f] - Fr).max():.3e}")
    assert np.abs(Ei[sel_e] - Eir).max() <= E_BF16 * max(1.0, np.abs(Eir).max()) * 5
    assert np.abs(F[sel_f] - Fr).max() <= F_MAX_BF16
    assert abs(float(E) - Ei.sum()) <= 1e-6 * np.abs(Ei).sum()
