"""The batched form on the full 256-box workload (16-2,048 waters per box,
338,622 atoms): one graph launch over all systems, whose persistent kernels
draw (system, cell) and (system, row-tile) work items from their queues, with
autotuned grid caps and tiles.  Sampled systems (the two smallest, the
median, the largest) against the oracle (FP32 bounds), every system against
a separate single-system evaluation."""
import numpy as np
import pytest

import synth
from common import E_REL_TOL, F_ABS_TOL, energy_error, weights32

pytestmark = pytest.mark.gpu


def test_batch_256(oracle_mod):
    import torch
    from paper_2604_21441_b300 import build
    build.build()
    import paper_2604_21441_b300 as P

    wl = synth.workload(4)
    systems = wl["systems"]
    w = weights32(2, 128, wl["weight_seed"], 3)
    w32 = [[(W.astype(np.float32), b.astype(np.float32)) for W, b in x] for x in w]
    off = np.cumsum([0] + [s.n for s in systems]).astype(np.int64)
    pos = torch.tensor(np.concatenate([s.pos for s in systems]), device="cuda")
    Z = torch.tensor(np.concatenate([s.Z for s in systems]), device="cuda")
    boxes = np.stack([s.box for s in systems])
    pot = P.NNP(atomic_numbers=(1, 8), max_atoms=int(off[-1]), max_systems=len(systems),
                flags=P.FLAG_AUTOTUNE)
    pot.set_all_weights(w32)
    E, F = pot.eval_batch(off, pos, Z, boxes)
    E, F = E.cpu().numpy(), F.cpu().numpy()
    tuned = {k: pot.query("tune_" + k) for k in ("neighbours", "descriptor", "backward",
                                                  "descriptor_tile", "backward_tile", "neighbours_form")}
    print("batch-256 tuned shapes:", tuned)
    # one of the autotuner's candidates (tile < 0: static order, > 0: queue;
    # neighbour form: bit 0 queue, bit 1 row groups over two warps)
    assert (tuned["neighbours"], tuned["neighbours_form"]) in {
        (4, 0), (8, 0), (16, 0), (16, 2), (8, 1), (16, 1), (32, 1), (16, 3)}
    assert (tuned["descriptor"], tuned["descriptor_tile"]) in {
        (2, -1), (4, -1), (8, -1), (16, -1), (8, 1), (8, 2), (8, 4), (16, 2)}
    assert tuned["backward"] in (4, 8, 12, 16, 24, 32, 48, 64) and tuned["backward_tile"] == -1
    # every system against its own single-system evaluation: the same kernels
    # on the same neighbour lists; only the order of the sums differs (energy
    # partial sums per warp start at other row offsets; the FP64 force
    # reductions add FP32 terms in launch order, and a system's row order
    # inside its cells is the same).  1e-5 eV/A bounds that with margin (the
    # parity bound against the oracle is 1e-4).
    single = P.NNP(atomic_numbers=(1, 8), max_atoms=int(max(s.n for s in systems)))
    single.set_all_weights(w32)
    for b, s in enumerate(systems):
        e1, f1 = single.eval(s.pos, s.Z, s.box)
        assert abs(E[b] - e1) <= 1e-7 * (abs(e1) + s.n), b
        assert np.abs(F[off[b]:off[b + 1]] - f1).max() <= 1e-5, b
    # sampled systems against the oracle
    p = oracle_mod.Params()
    m = oracle_mod.Model(p, w)
    order = np.argsort([s.n for s in systems])
    for b in (order[0], order[1], order[len(order) // 2], order[-1]):
        s = systems[b]
        Er, Eir, Fr, _ = oracle_mod.energy_forces(m, s.pos, p.species_of(s.Z), s.box)
        assert energy_error(E[b], Er, Eir) <= E_REL_TOL
        assert np.abs(F[off[b]:off[b + 1]] - Fr).max() <= F_ABS_TOL
