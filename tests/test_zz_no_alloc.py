"""nnp_eval_noalloc: the evaluation that allocates no device memory.

Some callers cannot allocate GPU memory once a run is under way, e.g. an MD
engine that gives the GPU's free memory to its own pool at start-up.  This
test calls that entry point through the C ABI, twice in a row, and checks
energy and forces against nnp_eval on the same context within the FP32
tolerances used by the other parity tests.  It lives in its own file, which
pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import synth
from common import E_REL_TOL, F_ABS_TOL, energy_error, weights32

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_eval_twice():
    import torch

    from paper_2604_21441_b300 import build
    build.build()
    import paper_2604_21441_b300 as P

    L = P.lib()
    s = synth.water_box(64, synth.GEOM_SEED[1])
    n = s.n
    w = weights32(2, 128, synth.WEIGHT_SEED[1], 7)
    pot = P.NNP(atomic_numbers=(1, 8))
    pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in sp] for sp in w])
    pos = torch.tensor(s.pos, device="cuda")
    Z = torch.tensor(s.Z, device="cuda")
    box = np.ascontiguousarray(np.diag(s.box))
    pbox = ctypes.c_void_p(box.ctypes.data)

    E0 = torch.zeros(1, dtype=torch.float64, device="cuda")
    F0 = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    assert L.nnp_eval(pot._h, n, _p(pos), _p(Z), pbox, _p(E0), _p(F0)) == 0
    Ei = pot.atom_energies(n)
    E0, F0 = float(E0), F0.cpu().numpy()

    for _ in range(2):
        E1 = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        F1 = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.nnp_eval_noalloc(pot._h, n, _p(pos), _p(Z), pbox, _p(E1), _p(F1))
        assert rc == 0, L.nnp_last_error(pot._h).decode()
        E1, F1 = float(E1), F1.cpu().numpy()
        assert energy_error(E1, E0, Ei) <= E_REL_TOL, (E1, E0)
        assert np.abs(F1 - F0).max() <= F_ABS_TOL

    # sizes beyond the fixed scratch are rejected with a clear error
    Ez = torch.zeros(1, dtype=torch.float64, device="cuda")
    Fz = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    rc = L.nnp_eval_noalloc(pot._h, P.NNP_NOALLOC_MAX_ATOMS + 1, _p(pos), _p(Z), pbox, _p(Ez), _p(Fz))
    assert rc == 4
    assert b"at most" in L.nnp_last_error(pot._h)
    pot.close()
