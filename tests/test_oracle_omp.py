"""The OpenMP build of the oracle (used only to time the CPU baseline) gives
the single-threaded oracle's energies and forces: every atom's terms are the
same functions, only the energy and force sums are grouped per thread, so
the two agree to rounding."""
import numpy as np
import pytest

import synth
from common import weights32


@pytest.mark.parametrize("kind", ["water", "hcno", "isolated"])
def test_omp_build_equals_oracle(oracle_mod, kind):
    if kind == "hcno":
        s = synth.hcno_box(77, L=16.0, n_cluster_atoms=120, max_waters=60)
        Zs = (1, 6, 7, 8)
        box = s.box
    else:
        s = synth.water_box(125, 31)
        Zs = (1, 8)
        box = None if kind == "isolated" else s.box
    p = oracle_mod.Params(atomic_numbers=Zs)
    m = oracle_mod.Model(p, weights32(len(Zs), p.aev_length, 41, 42))
    sp = p.species_of(s.Z)
    E, Ei, F, _ = oracle_mod.energy_forces(m, s.pos, sp, box)
    Eo, Eio, Fo, threads = oracle_mod.energy_forces_omp(m, s.pos, sp, box)
    assert threads >= 1
    assert abs(Eo - E) <= 1e-12 * np.abs(Ei).sum()
    assert np.abs(Eio - Ei).max() == 0.0   # per-atom energies: the very same arithmetic
    assert np.abs(Fo - F).max() <= 1e-12 * max(1.0, np.abs(F).max())
