"""Checkpoint and resume on the GPU.

* Weights: a context's weights written with save_weights and read into a new
  context (NNP.from_weights, and load_weights into one made by hand) give the
  same energy and forces (the same kernels on the same inputs; the FP64
  force sums may add in another order: 1e-11 eV/A), for an ensemble of two
  members over three species;
* load_weights refuses a file of other species;
* NVE: 40 steps of 0.5 fs in one run against 20 steps, a checkpoint
  (NVE.save), a restore into a new integrator on a new context and 20 more
  steps.  The restore recomputes the forces from the saved positions, so the
  two runs differ only by the order of FP64 force sums (1e-12 relative):
  positions within 1e-8 A, velocities within 1e-8 A/fs.
"""
import numpy as np
import pytest

import synth
from common import box9, weights32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2604_21441_b300 import build
    build.build()
    import paper_2604_21441_b300 as P
    return P


def _f32(w):
    return [[(W.astype(np.float32), b.astype(np.float32)) for W, b in sp] for sp in w]


def test_weights_round_trip(P, tmp_path):
    zs = (1, 6, 8)
    s = synth.hcno_box(801, L=16.0, n_cluster_atoms=120, max_waters=60,
                       elements=np.array(zs, dtype=np.int32), probs=np.full(3, 1.0 / 3))
    mem = [_f32(weights32(3, 240, 802 + 3 * m, 803 + 3 * m)) for m in range(2)]
    a = P.NNP(atomic_numbers=zs, n_members=2, max_atoms=s.n)
    a.set_member_weights(mem)
    E0, F0 = a.eval(s.pos, s.Z, box9(s.box))
    path = str(tmp_path / "model.npz")
    a.save_weights(path)
    b = P.NNP.from_weights(path, max_atoms=s.n)
    assert b.atomic_numbers == zs and b.n_members == 2
    E1, F1 = b.eval(s.pos, s.Z, box9(s.box))
    c = P.NNP(atomic_numbers=zs, n_members=2, max_atoms=s.n)
    c.load_weights(path)
    E2, F2 = c.eval(s.pos, s.Z, box9(s.box))
    for E, F in ((E1, F1), (E2, F2)):
        assert abs(E - E0) <= 1e-12 * abs(E0)
        assert np.abs(F - F0).max() <= 1e-11
    other = P.NNP(atomic_numbers=(1, 8), n_members=2)
    with pytest.raises(ValueError):
        other.load_weights(path)
    for pot in (a, b, c, other):
        pot.close()


def test_nve_checkpoint_resume(P, tmp_path):
    import torch
    from paper_2604_21441_b300 import torch_nnp as tn
    s = synth.water_box(512, 811)
    w = _f32(synth.xavier_weights(2, 128, 812, final_scale=0.03))
    vel = synth.maxwell_boltzmann(s.Z, 300.0, 813)

    def pot():
        p = P.NNP(atomic_numbers=(1, 8), max_atoms=s.n, stream=torch.cuda.Stream())
        p.set_all_weights(w)
        return p

    md = tn.NVE(pot(), s.pos, s.Z, s.box, vel, dt_fs=0.5)
    md.step(20)
    path = str(tmp_path / "nve.npz")
    md.save(path)
    md.step(20)
    md2 = tn.NVE.restore(path, pot())
    assert md2.steps_done == 20 and md2.dt == 0.5
    md2.step(20)
    assert md.steps_done == md2.steps_done == 40
    dr = (md.r - md2.r).abs().max().item()
    dv = (md.v - md2.v).abs().max().item()
    print(f"NVE resume after 20 steps: max |dr| {dr:.2e} A, max |dv| {dv:.2e} A/fs")
    assert dr <= 1e-8 and dv <= 1e-8
