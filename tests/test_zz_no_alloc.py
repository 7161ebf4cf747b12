"""nnp_eval_noalloc: the evaluation that allocates no device memory.

Some callers cannot allocate GPU memory once a run is under way, e.g. an MD
engine that gives the GPU's free memory to its own pool at start-up: a
cudaMalloc in the middle of its run can fail or stall its other streams.
These tests call that entry point through the C ABI:

* twice in a row on a 64-water box, against nnp_eval on the same context,
  within the FP32 tolerances of the other parity tests;
* on a four-species (H, C, N, O; D = 384) box of 1,005 atoms, near the
  1,024-atom end of the fixed scratch layout, against the FP64 oracle;
* with the device's free memory read before and after repeated calls on a
  fresh context: it must not drop (the scratch array is placed on the device
  by nnp_create, not by the first call);
* with inputs it must refuse: too many atoms, too many neighbours for its
  fixed lists, a reduced-precision context, a triclinic box, a box given as a
  device pointer.

The file is collected last, so that a run that stops at the first failure
has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

import synth
from common import E_REL_TOL, F_ABS_TOL, energy_error, weights32

pytestmark = pytest.mark.gpu

ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CAPACITY = 1, 3, 4


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.fixture(scope="module")
def P():
    from paper_2604_21441_b300 import build
    build.build()
    import paper_2604_21441_b300 as P
    return P


def _pot(P, Zs, w, precision="fp32"):
    pot = P.NNP(atomic_numbers=Zs, precision=precision)
    pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in sp] for sp in w])
    return pot


def _noalloc(P, pot, pos, Z, box, n=None):
    """One nnp_eval_noalloc call; returns (status, E, F) with E, F on the host."""
    import torch
    n = pos.shape[0] if n is None else n
    E = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    F = torch.full((pos.shape[0], 3), float("nan"), dtype=torch.float64, device="cuda")
    bx = np.ascontiguousarray(box, dtype=np.float64)
    rc = P.lib().nnp_eval_noalloc(pot._h, n, _p(pos), _p(Z), ctypes.c_void_p(bx.ctypes.data),
                                  _p(E), _p(F))
    return rc, float(E), F.cpu().numpy()


def test_noalloc_matches_eval_twice(P):
    import torch

    L = P.lib()
    s = synth.water_box(64, synth.GEOM_SEED[1])
    n = s.n
    pot = _pot(P, (1, 8), weights32(2, 128, synth.WEIGHT_SEED[1], 7))
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
        rc, E1, F1 = _noalloc(P, pot, pos, Z, box)
        assert rc == 0, L.nnp_last_error(pot._h).decode()
        assert energy_error(E1, E0, Ei) <= E_REL_TOL, (E1, E0)
        assert np.abs(F1 - F0).max() <= F_ABS_TOL

    # sizes beyond the fixed scratch are rejected with a clear error
    rc, _, _ = _noalloc(P, pot, pos, Z, box, n=P.NNP_NOALLOC_MAX_ATOMS + 1)
    assert rc == ERR_CAPACITY
    assert b"at most" in L.nnp_last_error(pot._h)
    pot.close()


def test_noalloc_four_species_vs_oracle(P, oracle_mod):
    """1,005 atoms of H/C/N/O clusters and water (D = 384): the largest
    descriptor and close to the largest atom count the scratch holds."""
    import torch

    Zs = (1, 6, 7, 8)
    s = synth.hcno_box(86, L=22.0, n_cluster_atoms=420, max_waters=200)
    assert 1000 <= s.n <= P.NNP_NOALLOC_MAX_ATOMS
    p = oracle_mod.Params(atomic_numbers=Zs)
    w = weights32(4, p.aev_length, 71, 72)
    Er, Eir, Fr, _ = oracle_mod.energy_forces(oracle_mod.Model(p, w), s.pos, p.species_of(s.Z), s.box)
    pot = _pot(P, Zs, w)
    pos = torch.tensor(s.pos, device="cuda")
    Z = torch.tensor(s.Z, device="cuda")
    for _ in range(2):
        rc, E, F = _noalloc(P, pot, pos, Z, np.diag(s.box))
        assert rc == 0, P.lib().nnp_last_error(pot._h).decode()
        err_e, err_f = energy_error(E, Er, Eir), np.abs(F - Fr).max()
        print(f"noalloc HCNO {s.n} atoms: rel E {err_e:.2e}, max|dF| {err_f:.2e} eV/A")
        assert err_e <= E_REL_TOL and err_f <= F_ABS_TOL
    pot.close()


def test_noalloc_free_memory_unchanged(P):
    """A fresh context: the device's free memory (cudaMemGetInfo) is the same
    before the first call and after several."""
    import torch

    s = synth.water_box(200, 12)
    pot = _pot(P, (1, 8), weights32(2, 128, 5, 6))
    pos = torch.tensor(s.pos, device="cuda")
    Z = torch.tensor(s.Z, device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    F = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    bx = np.ascontiguousarray(np.diag(s.box))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(4):
        rc = P.lib().nnp_eval_noalloc(pot._h, s.n, _p(pos), _p(Z), ctypes.c_void_p(bx.ctypes.data),
                                      _p(E), _p(F))
        assert rc == 0, P.lib().nnp_last_error(pot._h).decode()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    print(f"free memory before {free0} after {free1} (drop {free0 - free1} bytes)")
    # the scratch array alone is about 6 MiB: a drop of that size would mean
    # that the calls placed it
    assert free0 - free1 <= 1 << 20
    pot.close()


def test_noalloc_refusals(P):
    import torch

    L = P.lib()
    w = weights32(2, 128, 5, 6)
    s = synth.water_box(300, 5)
    # water compressed to 0.6 of its edge (4.6 x the density): more than the
    # fixed 128 radial / 48 angular list entries per atom
    f = 0.6
    pos = torch.tensor(np.mod(s.pos * f, s.box * f), device="cuda")
    Z = torch.tensor(s.Z, device="cuda")
    pot = _pot(P, (1, 8), w)
    rc, _, _ = _noalloc(P, pot, pos, Z, np.diag(s.box * f))
    assert rc == ERR_CAPACITY, L.nnp_last_error(pot._h).decode()
    assert b"neighbours" in L.nnp_last_error(pot._h)

    s = synth.water_box(64, synth.GEOM_SEED[1])
    pos = torch.tensor(s.pos, device="cuda")
    Z = torch.tensor(s.Z, device="cuda")
    # a triclinic box
    tri = np.diag(s.box).copy()
    tri[1, 0] = 1.0
    rc, _, _ = _noalloc(P, pot, pos, Z, tri)
    assert rc == ERR_UNSUPPORTED
    # the box as a device pointer
    dbox = torch.tensor(np.diag(s.box), device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    F = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    rc = L.nnp_eval_noalloc(pot._h, s.n, _p(pos), _p(Z), _p(dbox), _p(E), _p(F))
    assert rc == ERR_INVALID_ARG
    # after the refusals the context still evaluates
    rc, E1, _ = _noalloc(P, pot, pos, Z, np.diag(s.box))
    assert rc == 0 and np.isfinite(E1)
    pot.close()
    # reduced-precision contexts are refused
    pot = _pot(P, (1, 8), w, precision="bf16")
    rc, _, _ = _noalloc(P, pot, pos, Z, np.diag(s.box))
    assert rc == ERR_UNSUPPORTED
    pot.close()
