"""Other launch forms of the persistent kernels give the static order's results.

The neighbour kernel can take its cells, and the descriptor kernel its tiles
of row pairs, from a per-stage work queue instead of in static order, and the
neighbour kernel can split each cell's row groups over two warps; the autotuner
keeps such a shape only where it measures faster, so an ordinary run may
never take those paths.  Here the autotuner's cache file
(NNP_AUTOTUNE_CACHE, read once per process) presets the shapes for a single
box and for a batch, in a fresh process, and the results are compared with a
context that keeps the default static shapes: the neighbour lists are the
same and every row's arithmetic is the same; only the order of the FP64
force reductions differs.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import json, math, os, sys
import numpy as np
sys.path.insert(0, __ROOT_DIR__)
import synth
import paper_2604_21441_b300 as P
from paper_2604_21441_b300 import build
build.build()
w = synth.xavier_weights(2, 128, 7)
w32 = [[(W.astype(np.float32), b.astype(np.float32)) for W, b in x] for x in w]
out = {}

def key(rows, B):  # the autotuner's cache key (species, precision, row bucket, batch)
    bucket = int(math.ceil(math.log2(max(rows, 2))))
    return ((2 * 4 + 1) * 64 + bucket) + (1000000 if B > 1 else 0)

single = synth.water_box(4096, 11)
systems = [synth.water_box(n, 20 + n) for n in (40, 300, 1000, 77, 2000)]
off = np.cumsum([0] + [s.n for s in systems]).astype(np.int64)
bpos = np.concatenate([s.pos for s in systems]); bZ = np.concatenate([s.Z for s in systems])
boxes = np.stack([s.box for s in systems])

ref = P.NNP(atomic_numbers=(1, 8), precision="bf16", max_atoms=int(off[-1]), max_systems=8)
ref.set_all_weights(w32)
E0, F0 = ref.eval(single.pos, single.Z, single.box)
rows_single = ref.query("rows")
Eb0, Fb0 = ref.eval_batch(off, bpos, bZ, boxes)
rows_batch = ref.query("rows")
# the preset shapes: "nbr fwd bwd fwd_tile bwd_tile nbr_form"
with open(__CACHE_FILE__, "w") as f:
    for k in (key(rows_single, 1), key(rows_batch, len(systems))):
        f.write(f"{k} __SHAPE__\n")
os.environ["NNP_AUTOTUNE_CACHE"] = __CACHE_FILE__
q = P.NNP(atomic_numbers=(1, 8), precision="bf16", max_atoms=int(off[-1]), max_systems=8,
          flags=P.FLAG_AUTOTUNE)
q.set_all_weights(w32)
E1, F1 = q.eval(single.pos, single.Z, single.box)
out["single_shapes"] = [q.query("tune_neighbours_form"), q.query("tune_descriptor_tile")]
for _ in range(2):
    E1, F1 = q.eval(single.pos, single.Z, single.box)
Eb1, Fb1 = q.eval_batch(off, bpos, bZ, boxes)
out["batch_shapes"] = [q.query("tune_neighbours_form"), q.query("tune_descriptor_tile")]
out["dE"] = abs(E1 - E0) / abs(E0)
out["dF"] = float(np.abs(F1 - F0).max())
out["dEb"] = float(np.max(np.abs(Eb1 - Eb0) / np.abs(Eb0)))
out["dFb"] = float(np.abs(Fb1 - Fb0).max())
print("RESULT", json.dumps(out))
'''


# (cache shape, expected (neighbour form, descriptor tile)): neighbour cells
# and descriptor tiles of 2 row pairs from the queues; each cell's row groups
# over two warps, static and from the queue, with static descriptor tiles
FORMS = {"queue": ("8 8 16 2 -1 1", [1, 2]), "split_cells": ("8 8 16 -1 -1 2", [2, -1]),
         "split_cells_queue": ("16 8 16 -1 -1 3", [3, -1])}


@pytest.mark.parametrize("form", sorted(FORMS))
def test_launch_form_matches_static_order(tmp_path, form):
    shape, expect = FORMS[form]
    cache = str(tmp_path / "tune_cache.txt")
    code = SCRIPT.replace("__ROOT_DIR__", repr(ROOT)).replace("__CACHE_FILE__", repr(cache))
    code = code.replace("__SHAPE__", shape)
    env = dict(os.environ)
    env.pop("NNP_AUTOTUNE_CACHE", None)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    print(res)
    assert res["single_shapes"] == expect and res["batch_shapes"] == expect
    # same per-row arithmetic; the FP64 force sums add FP32 terms in another order
    assert res["dE"] <= 1e-12 and res["dEb"] <= 1e-12
    assert res["dF"] <= 1e-11 and res["dFb"] <= 1e-11
