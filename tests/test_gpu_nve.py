"""Velocity-Verlet NVE on the 12,288-atom water box (4,096 waters, 49.7 A):
1,000 steps of 0.5 fs with FP32 library forces, Maxwell-Boltzmann start at
300 K.  Energy conservation checks that forces are the exact negative
gradient of the energy the library reports.  There is no reference value
for the drift (parity unpinned); the bounds are max |E_tot(t) - E_tot(0)| / N
<= 1e-4 eV/atom over the run and <= 1e-5 eV/atom over the first 250 fs.

A random-weight network has no repulsive core and its descriptors grow with
local density, so unscaled Xavier weights let the box collapse within ~100
fs (neighbour counts double, the integrator then fails).  The output layer
is scaled by NVE_FINAL_SCALE so that the 500 fs stay before any collapse."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

# Output-layer scale of the random network for the dynamics (see the module doc).
NVE_FINAL_SCALE = 0.03


def test_nve_drift():
    import torch
    from paper_2604_21441_b300 import build
    build.build()
    import paper_2604_21441_b300 as P
    from paper_2604_21441_b300 import torch_nnp as tn

    wl = synth.workload(2)
    s = wl["systems"][0]
    w = synth.xavier_weights(2, 128, wl["weight_seed"], final_scale=NVE_FINAL_SCALE)
    stream = torch.cuda.Stream()
    pot = P.NNP(atomic_numbers=(1, 8), max_atoms=s.n, stream=stream,
                nbr_capacity=128, ang_capacity=48)
    pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in x] for x in w])
    vel = synth.maxwell_boltzmann(s.Z, 300.0, 7)
    md = tn.NVE(pot, s.pos, s.Z, s.box, vel, dt_fs=0.5)
    e0 = md.total_energy()
    es = [e0]
    for _ in range(20):
        md.step(50)
        es.append(md.total_energy())
    es = np.array(es)
    dev = np.abs(es - e0).max() / s.n
    slope = np.polyfit(np.arange(len(es)) * 25.0, es / s.n, 1)[0] * 1000.0  # eV/atom/ps
    print(f"NVE 1000 x 0.5 fs, {s.n} atoms: max |dE_tot|/N = {dev:.2e} eV/atom, "
          f"drift {slope * 1e3:.3f} meV/atom/ps, E_tot(0)/N {es[0] / s.n:.4f}, "
          f"rollbacks {md.retries}, max neighbours {pot.query('max_nbr')} / {pot.query('max_ang')}")
    print("E_tot/N every 25 fs:", np.array2string(es / s.n, precision=6))
    early = np.abs(es[:11] - e0).max() / s.n
    print(f"first 250 fs: max |dE_tot|/N = {early:.2e} eV/atom")
    assert early <= 1e-5
    assert dev <= 1e-4
