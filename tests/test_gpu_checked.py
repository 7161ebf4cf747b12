"""The bounds-checked build (libnnp_checked.so, compiled with -DNNP_CHECKED).

Indices read from device data -- neighbour-list entries and their image
codes, list and window positions, bins and slots, tile species, force slots
-- are checked before they address memory; a bad one is recorded in the
device flags and the call returns NNP_ERR_BOUNDS.  In a fresh process on the
checked library:

* its self-test index is caught (status 9) and the context keeps working;
* small cases of every path run clean (status 0) and agree with the FP64
  oracle within the usual bounds: FP32 and BF16 water-64, four species (FP32),
  a batch of three boxes (one small enough for the lane-per-row path), a
  two-member BF16 ensemble over three species (the ensemble dE/dG product),
  a caller's pair list, the allocation-free call and a force-matching loss.

The ordinary library reports that it was built without the checks.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import ctypes, json, os, sys
import numpy as np
sys.path.insert(0, __ROOT_DIR__)
sys.path.insert(0, os.path.join(__ROOT_DIR__, "tests"))
import synth, oracle
import paper_2604_21441_b300 as P
from paper_2604_21441_b300 import build
P.LIB_PATH = build.build(checked=True)
from common import box9, energy_error, weights32
out = {}
f32 = lambda w: [[(W.astype(np.float32), b.astype(np.float32)) for W, b in sp] for sp in w]

def check(name, zs, members, s, prec="fp32", tolE=1e-6, tolF=1e-4, batch=None):
    p = oracle.Params(atomic_numbers=zs)
    models = [oracle.Model(p, w) for w in members]
    pot = P.NNP(atomic_numbers=zs, precision=prec, n_members=len(members), max_atoms=4096, max_systems=4)
    pot.set_member_weights([f32(w) for w in members])
    assert pot.query("checked_build") == 1
    if batch is None:
        E, F = pot.eval(s.pos, s.Z, box9(s.box))
        Er, Eir, Fr = oracle.ensemble_energy_forces(models, s.pos, p.species_of(s.Z), s.box)
        errs = [(energy_error(E, Er, Eir), float(np.abs(F - Fr).max()))]
    else:
        off = np.cumsum([0] + [x.n for x in batch]).astype(np.int64)
        E, F = pot.eval_batch(off, np.concatenate([x.pos for x in batch]), np.concatenate([x.Z for x in batch]),
                              np.stack([x.box for x in batch]))
        errs = []
        for b, x in enumerate(batch):
            Er, Eir, Fr = oracle.ensemble_energy_forces(models, x.pos, p.species_of(x.Z), x.box)
            errs.append((energy_error(E[b], Er, Eir), float(np.abs(F[off[b]:off[b + 1]] - Fr).max())))
    out[name] = [max(e for e, _ in errs), max(f for _, f in errs)]
    assert out[name][0] <= tolE and out[name][1] <= tolF, (name, out[name])
    return pot

w2 = weights32(2, 128, 5, 6)
s64 = synth.water_box(64, synth.GEOM_SEED[1])
pot = check("water64_fp32", (1, 8), [w2], s64)
out["selftest"] = pot.selftest_bounds()
E, F = pot.eval(s64.pos, s64.Z, box9(s64.box))  # still usable
check("water64_bf16", (1, 8), [w2], s64, "bf16", 3e-3, 2e-2)
zs4 = (1, 6, 7, 8)
h4 = synth.hcno_box(86, L=16.0, n_cluster_atoms=120, max_waters=60)
check("hcno_fp32", zs4, [weights32(4, 384, 7, 8)], h4)
batch = [synth.water_box(n, 90 + n) for n in (8, 64, 300)]
check("batch_fp32", (1, 8), [w2], None, batch=batch)
zs3 = (1, 6, 8)
h3 = synth.hcno_box(93, L=16.0, n_cluster_atoms=120, max_waters=60, elements=np.array(zs3, dtype=np.int32),
                    probs=np.full(3, 1.0 / 3))
# the wide-descriptor BF16 bounds of tests/test_gpu_seven_species.py
check("ensemble_bf16", zs3, [weights32(3, 240, 11 + m, 12 + m) for m in range(2)], h3, "bf16", 5e-3, 6e-2)
# the caller's pair list
p2 = oracle.Params()
pi, pj, pd = oracle.pairs_brute(s64.pos, s64.box, 6.0)
keep = pi < pj
pairs = np.stack([pi[keep], pj[keep]], axis=1).astype(np.int32)
Ep, Fp = pot.eval_pairs(s64.pos, s64.Z, pairs, pd[keep] - (s64.pos[pj[keep]] - s64.pos[pi[keep]]), box9(s64.box))
Er, Eir, Fr, _ = oracle.energy_forces(oracle.Model(p2, w2), s64.pos, p2.species_of(s64.Z), s64.box)
out["pairs"] = [energy_error(Ep, Er, Eir), float(np.abs(Fp - Fr).max())]
assert out["pairs"][0] <= 1e-6 and out["pairs"][1] <= 1e-4
# the allocation-free call (device buffers)
import torch
pos, Z = torch.tensor(s64.pos, device="cuda"), torch.tensor(s64.Z, device="cuda")
En = torch.zeros(1, dtype=torch.float64, device="cuda")
Fn = torch.zeros((s64.n, 3), dtype=torch.float64, device="cuda")
bx = np.ascontiguousarray(np.diag(s64.box))
pp = lambda t: ctypes.c_void_p(t.data_ptr())
out["noalloc_rc"] = P.lib().nnp_eval_noalloc(pot._h, s64.n, pp(pos), pp(Z), ctypes.c_void_p(bx.ctypes.data), pp(En), pp(Fn))
assert out["noalloc_rc"] == 0 and abs(float(En) - Er) <= 1e-6 * np.abs(Eir).sum()
# force matching: the loss against a teacher network's forces
teacher = oracle.Model(p2, weights32(2, 128, 31, 32))
_, _, Ft, _ = oracle.energy_forces(teacher, s64.pos, p2.species_of(s64.Z), s64.box)
pot.eval(s64.pos, s64.Z, box9(s64.box))
L, _ = pot.force_match_grad(Fref=Ft, want_loss=True)
Lr, _, _, _ = oracle.force_match(oracle.Model(p2, w2), s64.pos, p2.species_of(s64.Z), s64.box, Ft)
out["fm_loss_rel"] = abs(L - Lr) / Lr
assert out["fm_loss_rel"] <= 2e-6
print("RESULT", json.dumps(out))
'''


def test_checked_build():
    code = SCRIPT.replace("__ROOT_DIR__", repr(ROOT))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    res = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1][len("RESULT "):])
    print(res)
    assert res["selftest"] == 9


def test_ordinary_build_has_no_checks():
    from paper_2604_21441_b300 import build
    build.build()
    import paper_2604_21441_b300 as P
    pot = P.NNP(atomic_numbers=(1, 8))
    assert pot.query("checked_build") == 0
    assert pot.selftest_bounds() == 3
    pot.close()
