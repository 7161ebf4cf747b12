"""Benchmark: NNP energy+force atom-steps/s on one B300 (BF16 vs FP32 forms).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32|fp8]
                    [--impl ours|reference] [--workload 1..5]

One step = one full evaluation of the hot path (wrap + cell lists,
neighbour lists, descriptors, per-element networks with energy sum, network
backward, descriptor backward to forces) for the 98,304-atom water box
(32,768 rigid waters at 1 g/cm^3, 99.4 A, seeded synthetic input) unless
--workload says otherwise.  `value` times the device-resident path
(graph replay through nnp_eval_async on device pointers) with CUDA events on
the library's stream; L2 is flushed (a 256 MB write) between timed steps,
outside the event pair.  `e2e` times nnp_eval with pinned host buffers
(H2D of positions and atomic numbers, D2H of energy and forces inside the
timed region).  Multi-GPU: one independent replica per rank (the path
needs no exchange), value = all ranks' atom-steps / max rank time.

--impl reference times the FP64 CPU oracle (the reference arm) on bounded
samples of the same workload.

Output: auxiliary measurements (MD throughput, ML/MM, pair lists,
ensembles, seven species, electrostatic embedding, the size scan) come first,
one per line, each starting with "# aux"; the benchmark's JSON line comes
last, with the two forms' numbers ("forms") and the force-matching gradient
("force_match") at its end.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NNP energy+force atom-steps/s: BF16 vs FP32 form on one B300 at stated force error"
UNIT = "atom-steps/s"
FP32_LANES_PER_SM = 128


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
                "sm_max_mhz": 2032.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic work per stage (FP32 operations, FMA = 2)

# Per-atom work of the water model (two species, D = 128, 1 g/cm^3) as the
# scope table of the hot path states it: descriptor forward 35 kFLOP per
# atom; descriptor backward 8 GFLOP on the 98,304-atom box (about 2.3 times
# the forward); network forward and backward 106,688 + 106,496 FLOP.
SCOPE_FLOP_PER_ATOM = {"descriptor": 35.0e3, "descriptor_backward": 8.0e9 / 98304,
                        "network": 106688.0 + 106496.0}


def algorithmic_flops(n_pairs_r, n_triplets, n_rows, D, S):
    """FP32 work of the descriptor forward / backward and the network,
    counted per radial pair and angular triplet from the arithmetic the
    kernels' formulas need (the instruction-level count)."""
    rad_fwd = n_pairs_r * 16 * 6          # x, x^2*eta, exp, fma per term
    ang_fwd = n_triplets * (32 * 2 + 8 * 9 + 4 * 6)
    rad_bwd = n_pairs_r * 16 * 9
    ang_bwd = n_triplets * (8 * 27 + 4 * 8 + 40)
    mlp = n_rows * 2 * (2 * (D * 160 + 160 * 128 + 128 * 96) + 96)
    return rad_fwd + ang_fwd, mlp, rad_bwd + ang_bwd


# ---------------------------------------------------------------------------

def build_workload(k, waters=0):
    """Workload k of synth.workload, or (waters > 0) one seeded water box of
    that many molecules with the water workloads' weights (other sizes, e.g.
    for a profiler capture of a box between the named ones)."""
    import synth
    if waters > 0:
        s = synth.water_box(waters, 1000 + waters)
        wl = dict(name=f"water-{waters} ({3 * waters:,} atoms, {s.box[0]:.1f} A)", systems=[s],
                  atomic_numbers=(1, 8), weight_seed=synth.WEIGHT_SEED[3])
    else:
        wl = synth.workload(k)
    S = len(wl["atomic_numbers"])
    D = synth.aev_length(S)
    w = synth.xavier_weights(S, D, wl["weight_seed"])
    return wl, w, S, D


def concat(systems):
    off = np.cumsum([0] + [s.n for s in systems]).astype(np.int64)
    pos = np.concatenate([s.pos for s in systems])
    Z = np.concatenate([s.Z for s in systems]).astype(np.int32)
    boxes = np.stack([np.diag(s.box) for s in systems])
    return off, pos, Z, boxes


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2604_21441_b300 as P

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    wl, w, S, D = build_workload(args.workload, args.waters)
    off, pos_h, Z_h, boxes = concat(wl["systems"])
    B = len(wl["systems"])
    n = int(off[-1])
    stream = torch.cuda.Stream(device=dev)
    w32 = [[(W.astype(np.float32), b.astype(np.float32)) for W, b in sp] for sp in w]

    import synth
    f32 = lambda wm: [[(W.astype(np.float32), b.astype(np.float32)) for W, b in sp] for sp in wm]
    members = [w32] + [f32(synth.xavier_weights(S, D, wl["weight_seed"] + m)) for m in range(1, args.members)]

    def make(prec, flags=0):
        pot = P.NNP(atomic_numbers=wl["atomic_numbers"], precision=prec, max_atoms=n,
                    max_systems=B, stream=stream, flags=flags | P.FLAG_AUTOTUNE, n_members=args.members)
        pot.set_member_weights(members)
        return pot

    pos = torch.tensor(pos_h, device=dev)
    Z = torch.tensor(Z_h, device=dev)
    E = torch.zeros(B, dtype=torch.float64, device=dev)
    F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def step_async(pot):
        if B == 1:
            pot.eval_into(pos, Z, boxes[0], E, F, sync=False)
        else:
            pot.eval_batch_into(off, pos, Z, boxes, E, F, sync=False)

    def step_sync(pot):
        if B == 1:
            pot.eval_into(pos, Z, boxes[0], E, F, sync=True)
        else:
            pot.eval_batch_into(off, pos, Z, boxes, E, F, sync=True)

    def timed(pot, K, W, stage=False):
        step_sync(pot)  # settles list capacities (synchronous calls regrow them)
        for _ in range(W):
            step_async(pot)
            pot.sync()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        stages = []
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for k in range(K):
                flush.zero_()
                starts[k].record(stream)
                step_async(pot)
                ends[k].record(stream)
                if stage:
                    stages.append(pot.profile_stages())
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        pot.sync()
        ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        return ms, stages

    forms = {}
    results = {}
    prec_list = [args.precision] + [p for p in ("fp32", "bf16", "fp8")
                                    if p != args.precision and p in args.compare]
    clocks = ClockSampler(local_rank)
    clocks.start()
    main = None
    for prec in prec_list:
        try:
            pot = make(prec)
        except P.NNPError as e:
            forms[prec] = {"unavailable": str(e)}
            if prec == args.precision:
                raise
            continue
        ms, _ = timed(pot, args.steps, args.warmup)
        t = float(np.sum(ms)) / 1e3
        forms[prec] = {"value": n * args.steps / t, "ms_per_step": float(np.mean(ms)),
                       "ms_p10": float(np.percentile(ms, 10)), "ms_p90": float(np.percentile(ms, 90))}
        results[prec] = (E.cpu().numpy().copy(), F.cpu().numpy().copy())
        if prec == "fp32":
            ei_abs = float(np.abs(pot.atom_energies(n)).sum())
            if prec != args.precision:  # the FP32 network's stage time (its roofline, in the line)
                spot32 = make(prec, flags=P.FLAG_STAGE_EVENTS)
                _, st32 = timed(spot32, 5, 2, stage=True)
                forms[prec]["network_ms"] = float(np.mean(np.array(st32), axis=0)[3])
                spot32.close()
        if prec == args.precision:
            main = (pot, ms)
        else:
            pot.close()
    clk = clocks.stop()
    # error of the reduced-precision forms against the FP32 form (which the
    # parity tests hold to 1e-6 relative energy and 1e-4 eV/A of the FP64 oracle)
    if "fp32" in results:
        E32, F32 = results["fp32"]
        for prec, (Eq, Fq) in results.items():
            if prec != "fp32":
                dF = Fq - F32
                forms[prec]["vs_fp32"] = {
                    "max_abs_dF_eV_per_A": float(np.abs(dF).max()),
                    "rms_dF_eV_per_A": float(np.sqrt((dF ** 2).mean())),
                    "rms_F_eV_per_A": float(np.sqrt((F32 ** 2).mean())),
                    # |sum dE| / max(|E|, sum_i |E_i|), the normalisation of the FP32 parity bound
                    "rel_dE": float(abs(Eq.sum() - E32.sum()) / max(abs(E32.sum()), ei_abs))}
    pot, ms = main
    # per-stage durations (instrumented graph, same protocol)
    spot = make(args.precision, flags=P.FLAG_STAGE_EVENTS)
    _, stages = timed(spot, max(3, min(args.steps, 20)), 2, stage=True)
    stage_ms = np.mean(np.array(stages), axis=0)
    nbr_r = spot.query("max_nbr")
    spot.close()
    # e2e through host buffers: pinned inputs and outputs (one system: the
    # library copies them with plain asynchronous DMA), pageable for the batch
    if B == 1:
        pos_p = torch.from_numpy(np.ascontiguousarray(pos_h, dtype=np.float64)).pin_memory()
        Z_p = torch.from_numpy(np.ascontiguousarray(Z_h, dtype=np.int32)).pin_memory()
        E_p = torch.zeros(1, dtype=torch.float64).pin_memory()
        F_p = torch.zeros((n, 3), dtype=torch.float64).pin_memory()
    for _ in range(2):
        if B == 1:
            pot.eval_into(pos_p, Z_p, boxes[0], E_p, F_p)
        else:
            pot.eval_batch(off, pos_h, Z_h, boxes)
    t0 = time.perf_counter()
    K_e2e = max(3, args.steps // 2)
    for _ in range(K_e2e):
        if B == 1:
            pot.eval_into(pos_p, Z_p, boxes[0], E_p, F_p)
        else:
            e_, f_ = pot.eval_batch(off, pos_h, Z_h, boxes)
    t_e2e = time.perf_counter() - t0
    launches = pot.query("launches_per_eval")
    tuned = {k: pot.query("tune_" + k) for k in ("neighbours", "descriptor", "backward",
                                                  "descriptor_tile", "backward_tile", "neighbours_form")}
    per_system = None
    if B > 1:  # the same batch as one graph launch per system (one context each)
        pots = [P.NNP(atomic_numbers=wl["atomic_numbers"], precision=args.precision,
                      max_atoms=int(off[b + 1] - off[b]), stream=stream) for b in range(B)]
        for q in pots:
            q.set_all_weights(w32)

        def per_sys_step():
            for b, q in enumerate(pots):
                q.eval_into(pos[off[b]:off[b + 1]], Z[off[b]:off[b + 1]], boxes[b],
                            E[b:b + 1], F[off[b]:off[b + 1]], sync=False)
        for b, q in enumerate(pots):
            q.eval_into(pos[off[b]:off[b + 1]], Z[off[b]:off[b + 1]], boxes[b],
                        E[b:b + 1], F[off[b]:off[b + 1]], sync=True)
        for _ in range(2):
            per_sys_step()
            for q in pots:
                q.sync()
        ts = []
        with torch.cuda.stream(stream):
            for _ in range(max(3, args.steps // 3)):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                per_sys_step()
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
        for q in pots:
            q.sync()
            q.close()
        per_system = float(np.mean(ts))
    return dict(tuned=tuned, per_system_ms=per_system, n=n, B=B, S=S, D=D, ms=ms, forms=forms, clocks=clk, stage_ms=stage_ms.tolist(),
                e2e=n * K_e2e / t_e2e, e2e_ms=t_e2e / K_e2e * 1e3, launches=launches,
                wl=wl, pot=pot, pos_h=pos_h, Z_h=Z_h, boxes=boxes, w=w)


def nve_rate(precision, steps=400):
    """Velocity-Verlet throughput on the 4,096-water box (12,288 atoms,
    0.5 fs): library forces plus the four elementwise updates per step, all
    on the library's stream, device-resident state; timed with CUDA events.
    The network's output layer is scaled by 0.03 (as in the NVE test) so that
    random weights give stable dynamics."""
    import torch
    import synth
    import paper_2604_21441_b300 as P
    from paper_2604_21441_b300 import torch_nnp as tn
    wl = synth.workload(2)
    s = wl["systems"][0]
    w = synth.xavier_weights(2, 128, wl["weight_seed"], final_scale=0.03)
    stream = torch.cuda.Stream()
    pot = P.NNP(atomic_numbers=(1, 8), precision=precision, max_atoms=s.n, stream=stream,
                nbr_capacity=128, ang_capacity=48)
    pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in x] for x in w])
    md = tn.NVE(pot, s.pos, s.Z, s.box, synth.maxwell_boltzmann(s.Z, 300.0, 7), dt_fs=0.5)
    md.step(50, check_every=50)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    md.step(steps, check_every=steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    pot.close()
    return {"workload": "water-4096 (12,288 atoms, 49.7 A)", "precision": precision, "dt_fs": 0.5,
            "steps": steps, "ms_per_step": ms, "ns_per_day": 0.5e-6 * 86400e3 / ms,
            "rollbacks": md.retries}


def mlmm_rate(precision, steps=50):
    """ML/MM mechanical embedding through nnp_eval_mlmm (device buffers) on
    the 4,096-water box: the first 2,048 waters form the ML group, and 64 of
    them have one O-H bond cut (the H is MM, a link atom at 1 A replaces it).
    Each call validates the index sets, gathers the subsystem, evaluates it
    and scatters the forces to all 12,288 atoms; it is synchronous, so it is
    timed by wall clock.  The plain evaluation of a subsystem of the same size
    is timed beside it."""
    import torch
    import synth
    import paper_2604_21441_b300 as P
    wl = synth.workload(2)
    s = wl["systems"][0]
    w = synth.xavier_weights(2, 128, wl["weight_seed"])
    pot = P.NNP(atomic_numbers=(1, 8), precision=precision, max_atoms=s.n)
    pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in x] for x in w])
    cut = np.arange(0, 2048, 32)
    group = np.setdiff1d(np.arange(3 * 2048), 3 * cut + 1)
    dev = lambda a: torch.tensor(a, device="cuda")
    pos, Z = dev(s.pos), dev(s.Z.astype(np.int32))
    ml, lml, lmm = dev(group.astype(np.int64)), dev((3 * cut).astype(np.int64)), dev((3 * cut + 1).astype(np.int64))
    box = np.diag(s.box)
    for _ in range(5):
        pot.eval_mlmm(pos, Z, ml, lml, lmm, None, 1, box=box)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        pot.eval_mlmm(pos, Z, ml, lml, lmm, None, 1, box=box)
    ms = (time.perf_counter() - t0) * 1e3 / steps
    n_sub = len(group) + len(cut)
    sub_pos, sub_Z = pos[:n_sub].contiguous(), Z[:n_sub].contiguous()
    for _ in range(5):
        pot.eval(sub_pos, sub_Z, box)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        pot.eval(sub_pos, sub_Z, box)
    ms_plain = (time.perf_counter() - t0) * 1e3 / steps
    pot.close()
    return {"workload": "water-4096 (12,288 atoms): 2,048-water ML group, 64 link atoms",
            "precision": precision, "subsystem_atoms": n_sub, "links": len(cut), "steps": steps,
            "ms_per_step": ms, "subsystem_atom_steps_per_s": n_sub / (ms * 1e-3),
            "plain_eval_ms_same_size": ms_plain}


def pairs_rate(precision, steps=20):
    """The pair-list path (nnp_eval_pairs) on the 32,768-water box: a buffered
    half list (every pair within 5.6 A once, minimum-image shifts; built once
    on the host with a k-d tree, resident on the device) replaces the cell
    search.  Both paths are synchronous calls with device buffers, timed by
    wall clock over the same number of calls."""
    import torch
    import synth
    import paper_2604_21441_b300 as P
    from scipy.spatial import cKDTree
    wl = synth.workload(3)
    s = wl["systems"][0]
    w = synth.xavier_weights(2, 128, wl["weight_seed"])
    L = s.box
    ij = cKDTree(np.mod(s.pos, L), boxsize=L).query_pairs(5.6, output_type="ndarray")
    shifts = -L * np.round((s.pos[ij[:, 1]] - s.pos[ij[:, 0]]) / L)
    pot = P.NNP(atomic_numbers=(1, 8), precision=precision, max_atoms=s.n)
    pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in x] for x in w])
    dev = lambda a: torch.tensor(a, device="cuda")
    pos, Z, pr, sh = dev(s.pos), dev(s.Z.astype(np.int32)), dev(ij.astype(np.int32)), dev(shifts)
    box = np.diag(L)
    out = {}
    for name, fn in (("pair_list", lambda: pot.eval_pairs(pos, Z, pr, sh, box)),
                     ("cell_search", lambda: pot.eval(pos, Z, box))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            fn()
        out[name] = (time.perf_counter() - t0) * 1e3 / steps
    pot.close()
    return {"workload": "water-32768 (98,304 atoms), half list within 5.6 A", "precision": precision,
            "pairs": int(len(ij)), "steps": steps, "ms_per_step_pair_list": out["pair_list"],
            "ms_per_step_cell_search": out["cell_search"],
            "atom_steps_per_s_pair_list": s.n / (out["pair_list"] * 1e-3)}


def ensemble_rate(precision, members=8, steps=20):
    """An ensemble of M networks (the ANI-2x model is eight networks over one
    descriptor) on the 32,768-water box: synchronous calls with device
    buffers, timed by wall clock beside the single network.  The descriptor,
    its backward and the neighbour search run once; only the network stage
    runs M times."""
    import torch
    import synth
    import paper_2604_21441_b300 as P
    wl = synth.workload(3)
    s = wl["systems"][0]
    dev = lambda a: torch.tensor(a, device="cuda")
    pos, Z = dev(s.pos), dev(s.Z.astype(np.int32))
    box = np.diag(s.box)
    out = {}
    for M in (1, members):
        pot = P.NNP(atomic_numbers=(1, 8), precision=precision, max_atoms=s.n, n_members=M)
        for m in range(M):
            w = synth.xavier_weights(2, 128, wl["weight_seed"] + m)
            pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in x] for x in w], m)
        for _ in range(3):
            pot.eval(pos, Z, box)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            pot.eval(pos, Z, box)
        out[M] = (time.perf_counter() - t0) * 1e3 / steps
        pot.close()
    return {"workload": "water-32768 (98,304 atoms)", "precision": precision, "members": members,
            "steps": steps, "ms_per_step_single": out[1], "ms_per_step_ensemble": out[members],
            "atom_steps_per_s_ensemble": s.n / (out[members] * 1e-3)}


def seven_species_rate(members=8, steps=20):
    """The seven-element model (H, C, N, O, F, S, Cl; D = 1008, the ANI-2x
    element set) on HCNOFSCl-40A (2,000 cluster atoms + 1,349 waters), FP32
    and BF16 forms: one network and an ensemble of M, synchronous calls with
    device buffers, timed by wall clock."""
    import torch
    import synth
    import paper_2604_21441_b300 as P
    wl = synth.workload(6)
    s = wl["systems"][0]
    dev = lambda a: torch.tensor(a, device="cuda")
    pos, Z = dev(s.pos), dev(s.Z.astype(np.int32))
    box = np.diag(s.box)
    S = len(wl["atomic_numbers"])
    out = {}
    for prec, M in (("fp32", 1), ("fp32", members), ("bf16", 1), ("bf16", members)):
        pot = P.NNP(atomic_numbers=wl["atomic_numbers"], precision=prec, max_atoms=s.n, n_members=M)
        for m in range(M):
            w = synth.xavier_weights(S, synth.aev_length(S), wl["weight_seed"] + m)
            pot.set_all_weights([[(W.astype(np.float32), b.astype(np.float32)) for W, b in x] for x in w], m)
        for _ in range(3):
            pot.eval(pos, Z, box)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            pot.eval(pos, Z, box)
        out[prec, M] = (time.perf_counter() - t0) * 1e3 / steps
        pot.close()
    res = {"workload": wl["name"], "atoms": s.n, "species": S, "aev_length": synth.aev_length(S),
           "members": members, "steps": steps}
    for prec in ("fp32", "bf16"):
        res[prec] = {"ms_per_step_single": out[prec, 1], "ms_per_step_ensemble": out[prec, members],
                     "atom_steps_per_s_single": s.n / (out[prec, 1] * 1e-3),
                     "atom_steps_per_s_ensemble": s.n / (out[prec, members] * 1e-3)}
    return res


def ee_rate(precision, steps=50, n_ml_waters=64):
    """Electrostatic embedding (nnp_eval_ee) on the 32,768-water box: the
    first 64 waters (192 atoms) are the ML region, the other 98,112 atoms are
    MM point charges (O -0.834 e, H +0.417 e).  Synchronous calls with device
    buffers, timed by wall clock beside the plain evaluation of the ML atoms."""
    import torch
    import synth
    import paper_2604_21441_b300 as P
    wl = synth.workload(3)
    s = wl["systems"][0]
    k = 3 * n_ml_waters
    dev = lambda a: torch.tensor(a, device="cuda")
    pos, Z = dev(s.pos[:k]), dev(s.Z[:k].astype(np.int32))
    mm_pos = dev(s.pos[k:])
    mm_q = dev(np.tile([-0.834, 0.417, 0.417], (s.n - k) // 3))
    box = np.diag(s.box)
    w = synth.xavier_weights(2, 128, wl["weight_seed"])
    wq = synth.xavier_weights(2, 128, wl["weight_seed"] + 100, final_scale=0.2)
    f32 = lambda ws: [[(W.astype(np.float32), b.astype(np.float32)) for W, b in x] for x in ws]
    pot = P.NNP(atomic_numbers=(1, 8), precision=precision, max_atoms=k, flags=P.FLAG_CHARGES)
    pot.set_all_weights(f32(w))
    pot.set_charge_weights(f32(wq))
    out = {}
    for name, fn in (("ee", lambda: pot.eval_ee(pos, Z, mm_pos, mm_q, box=box)),
                     ("plain", lambda: pot.eval(pos, Z, box))):
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            fn()
        out[name] = (time.perf_counter() - t0) * 1e3 / steps
    pot.close()
    return {"workload": "water-32768: 64 ML waters (192 atoms), 98,112 MM point charges", "precision": precision,
            "steps": steps, "ms_per_step_ee": out["ee"], "ms_per_step_plain_ml": out["plain"],
            "ml_mm_pairs": k * (s.n - k)}


PAPER_SIZES = (3, 9, 21, 30, 90, 210, 300, 900, 2100, 3000, 9000, 21000, 30000)  # atoms (Table S3)


def size_scan(steps=30, sizes=PAPER_SIZES):
    """ms per synchronous evaluation (device buffers, wall clock, as one MD
    step would call it) of water boxes at the sizes of the paper's
    performance table, for (a) the two-species water model, one network,
    BF16, and (b) the ANI-2x-scale model: seven species (D = 1008) and an
    ensemble of eight networks, BF16.  Boxes shorter than the 5.2 A radial
    cutoff (1 and 3 waters) are run as isolated clusters."""
    import torch
    import synth
    import paper_2604_21441_b300 as P
    Z7 = tuple(int(z) for z in synth.ANI2X_Z)
    f32 = lambda ws: [[(W.astype(np.float32), b.astype(np.float32)) for W, b in x] for x in ws]
    models = {"water_bf16": ((1, 8), 1), "ani2x_scale_bf16": (Z7, 8)}
    pots = {}
    for name, (zs, M) in models.items():
        S = len(zs)
        pot = P.NNP(atomic_numbers=zs, precision="bf16", max_atoms=max(sizes), n_members=M)
        for m in range(M):
            pot.set_all_weights(f32(synth.xavier_weights(S, synth.aev_length(S), 3000 + 17 * m + S)), m)
        pots[name] = pot
    rows = []
    for n_atoms in sizes:
        s = synth.water_box(n_atoms // 3, 4000 + n_atoms)
        periodic = s.box[0] >= 5.2
        box = np.diag(s.box) if periodic else None
        pos = torch.tensor(s.pos if periodic else s.pos - s.pos.mean(axis=0), device="cuda")
        Z = torch.tensor(s.Z.astype(np.int32), device="cuda")
        row = {"atoms": n_atoms, "periodic": bool(periodic)}
        for name, pot in pots.items():
            for _ in range(5):
                pot.eval(pos, Z, box)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(steps):
                pot.eval(pos, Z, box)
            row[name + "_ms"] = (time.perf_counter() - t0) * 1e3 / steps
        rows.append(row)
    for pot in pots.values():
        pot.close()
    return rows


def oracle_sample(wl, w, seconds=20.0, seed=0):
    """Time the FP64 oracle on bounded samples of the workload: sampled atoms
    get E_i and F_i, which evaluates them and every atom within the radial
    cutoff of them.  Returns (atoms evaluated per second, description)."""
    import oracle
    S = len(wl["atomic_numbers"])
    p = oracle.Params(atomic_numbers=tuple(wl["atomic_numbers"]))
    m = oracle.Model(p, w)
    s = wl["systems"][0]
    sp = p.species_of(s.Z)
    rng = np.random.default_rng(seed)
    evaluated, t_tot, calls = 0, 0.0, 0
    from scipy.spatial import cKDTree
    tree = cKDTree(np.mod(s.pos, s.box[0]), boxsize=s.box[0])
    while t_tot < seconds:
        sel = np.sort(rng.choice(s.n, 4, replace=False))
        need = set(sel.tolist())
        for i in sel:
            need.update(tree.query_ball_point(np.mod(s.pos[i], s.box[0]), p.rc_r))
        t0 = time.perf_counter()
        oracle.energy_forces_subset(m, s.pos, sp, s.box, sel, sel)
        t_tot += time.perf_counter() - t0
        evaluated += len(need)
        calls += 1
    desc = (f"{calls} oracle calls on the {s.n}-atom box, each E_i and F_i of 4 random atoms "
            f"(fully evaluates them and their radial neighbours: {evaluated} atom evaluations, "
            f"plus the O(N) pair search per call), {t_tot:.1f} s single-threaded FP64")
    return evaluated / t_tot, desc, calls, t_tot


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_full_omp(wl, w):
    """One full evaluation of the workload (E and F of every atom of every
    system) by the OpenMP build of the oracle.  Returns (seconds, threads)."""
    import oracle
    p = oracle.Params(atomic_numbers=tuple(wl["atomic_numbers"]))
    m = oracle.Model(p, w)
    t0 = time.perf_counter()
    threads = 1
    for s in wl["systems"]:
        threads = oracle.energy_forces_omp(m, s.pos, p.species_of(s.Z), s.box)[3]
    return time.perf_counter() - t0, threads


def oracle_full_serial(wl, w):
    """One full evaluation of the workload by the single-threaded oracle."""
    import oracle
    p = oracle.Params(atomic_numbers=tuple(wl["atomic_numbers"]))
    m = oracle.Model(p, w)
    t0 = time.perf_counter()
    for s in wl["systems"]:
        oracle.energy_forces(m, s.pos, p.species_of(s.Z), s.box)
    return time.perf_counter() - t0


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, same workload,
    metric and config as the GPU arm.  Each timed step is one full
    evaluation of the workload by the OpenMP build of the oracle.  The first
    warm-up step is one such evaluation (it also sizes the run); the oracle
    keeps no state, so the other warm-up steps are short sampled calls.  If K
    full evaluations would take more than --ref-budget seconds, each step is
    instead a bounded sample (--ref-seconds of sampled atoms, single-threaded).
    --serial-full 1 also times one full single-threaded evaluation."""
    wl, w, S, D = build_workload(args.workload, args.waters)
    n = sum(s.n for s in wl["systems"])
    t_probe, threads = oracle_full_omp(wl, w)
    full = t_probe * args.steps <= args.ref_budget
    times, evaluated = [], 0
    if full:
        for k in range(args.warmup - 1):
            oracle_sample(wl, w, seconds=0.2, seed=1000 + k)
        for _ in range(args.steps):
            t, _ = oracle_full_omp(wl, w)
            times.append(t)
        evaluated = n * args.steps
        sample = (f"each step one full evaluation (E, F of all {n} atoms) by the OpenMP build of the "
                  f"oracle over {threads} threads")
    else:
        for k in range(args.warmup):
            oracle_sample(wl, w, seconds=0.5, seed=1000 + k)
        per_step = min(args.ref_seconds, max(1.5, 120.0 / max(1, args.steps)))
        for k in range(args.steps):
            v, d, calls, t = oracle_sample(wl, w, seconds=per_step, seed=k)
            times.append(t)
            evaluated += v * t
        threads = 1
        sample = (f"each step {per_step:.1f} s of sampled atoms, single-threaded (a full OpenMP "
                  f"evaluation took {t_probe:.1f} s)")
    t_all = float(np.sum(times)) * args.members  # an ensemble: every member evaluated in full
    value = evaluated / t_all
    if args.members > 1:
        sample += f"; one member's time times {args.members} members"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_all / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded water boxes, random Xavier weights)",
            "config": workload_config(wl, args.precision, args.gpus, args.members),
            "cpu_baseline": {"value": r4(value), "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample, "cpu": cpu_model(), "nproc": os.cpu_count()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if args.serial_full:
        ts = oracle_full_serial(wl, w)
        line["serial_full_eval"] = {"seconds": r4(ts), "atom_steps_per_s": r4(n / ts), "threads": 1}
    print(json.dumps(line), flush=True)


def aggregate_ranks(t_rank, units, world, device):
    """Whole-job timing of independent replicas: the slowest rank's timed
    seconds and the units (atom-steps) summed over ranks.  Any process group
    backend (NCCL on GPUs, gloo on CPU)."""
    if world <= 1:
        return t_rank, float(units)
    import torch
    import torch.distributed as dist
    tmax = torch.tensor([t_rank], dtype=torch.float64, device=device)
    tsum = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax.item()), float(tsum.item())


def r4(x):
    """A float rounded to 4 significant digits (keeps the JSON line short)."""
    return None if x is None else float(f"{x:.4g}")


def force_match_rate(steps=20):
    """Force-matching weight gradient (nnp_force_match_grad, FP32 with FP64
    sums) on the HCNO workload: 2,000 cluster atoms of H, C, N, O in water,
    40 A box, 6,134 atoms, D = 384.  The reference forces come from a second,
    independently seeded network of the same architecture (the teacher),
    evaluated by the library.  Each call recomputes the forces of the last
    evaluation, the tangent descriptors, the networks' tangent and adjoint
    passes and the weight-gradient reductions, and leaves the gradient in a
    device buffer (as an optimiser on the GPU would use it): synchronous
    calls timed by wall clock, stage durations by CUDA events (separate
    calls).  Work per stage (FP32, FMA = 2; the roofline is the FP32 ALU
    peak): the descriptor kernels' per-pair/per-triplet counts; the networks'
    primal and tangent forward, 2 x 2 (D*160 + 160*128 + 128*96) per atom, and
    the two adjoints, 2 x 2 (96*128 + 128*160); the weight gradients,
    4 (D*160 + 160*128 + 128*96 + 96) per atom."""
    import torch
    import synth
    import paper_2604_21441_b300 as P
    wl = synth.workload(5)
    s = wl["systems"][0]
    Zs = tuple(int(z) for z in wl["atomic_numbers"])
    S, D = len(Zs), synth.aev_length(len(Zs))
    f32 = lambda ws: [[(W.astype(np.float32), b.astype(np.float32)) for W, b in x] for x in ws]
    dev = lambda a: torch.tensor(a, device="cuda")
    pos, Z = dev(s.pos), dev(s.Z.astype(np.int32))
    box = np.diag(s.box)
    teacher = P.NNP(atomic_numbers=Zs, precision="fp32", max_atoms=s.n)
    teacher.set_all_weights(f32(synth.xavier_weights(S, D, wl["weight_seed"] + 1000)))
    _, Fref = teacher.eval(pos, Z, box)
    teacher.close()
    pot = P.NNP(atomic_numbers=Zs, precision="fp32", max_atoms=s.n, flags=P.FLAG_STAGE_EVENTS)
    pot.set_all_weights(f32(synth.xavier_weights(S, D, wl["weight_seed"])))
    pot.eval(pos, Z, box)
    grad = torch.zeros(pot.param_count(), dtype=torch.float64, device="cuda")  # stays on the device
    for _ in range(3):
        pot.force_match_grad(Fref=Fref, out=grad)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        L, _ = pot.force_match_grad(Fref=Fref, want_loss=True, out=grad)
    ms = (time.perf_counter() - t0) * 1e3 / steps
    stages = []
    for _ in range(5):
        pot.force_match_grad(Fref=Fref, out=grad)
        stages.append(pot.profile_force_match())
    pot.close()
    st = np.mean(np.array(stages), axis=0)
    names = ("forces", "tangent_descriptors", "networks", "weight_gradients")
    n_pairs, n_trip = neighbour_stats({"wl": wl})
    fl_desc, fl_mlp, fl_bwd = algorithmic_flops(n_pairs, n_trip, s.n, D, S)
    net_fwd = 2 * (D * 160 + 160 * 128 + 128 * 96)
    work = {"forces": fl_desc + fl_mlp + fl_bwd, "tangent_descriptors": fl_bwd,
            "networks": s.n * (2 * net_fwd + 2 * 2 * (96 * 128 + 128 * 160)),
            "weight_gradients": s.n * 4 * (D * 160 + 160 * 128 + 128 * 96 + 96)}
    stage = dict(zip(names, st.tolist()))
    dom = max(stage, key=stage.get)
    peak = alu_peak_tflops()
    ach = work[dom] / (stage[dom] * 1e-3) / 1e12
    return {"workload": wl["name"], "atoms": s.n, "species": S, "aev_length": D, "precision": "fp32",
            "loss": r4(L), "ms_per_gradient": r4(ms), "stage_ms": {k: r4(v) for k, v in stage.items()},
            "dominant": dom, "achieved_tflops": r4(ach), "peak_tflops": r4(peak), "frac": r4(ach / peak),
            "bound": "alu"}


def alu_peak_tflops(dev=0):
    """FP32 ALU peak of the device: SMs (read from the device) x 128 FP32
    lanes x 2 FLOP x the maximum SM clock (MEASURED_PEAKS.json, else the
    device's own figure)."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    pk, _ = peaks()
    mhz = pk.get("sm_max_mhz") or props.clock_rate / 1e3
    return props.multi_processor_count * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp8"])
    ap.add_argument("--compare", default="fp32,bf16,fp8")
    ap.add_argument("--workload", type=int, default=3)
    ap.add_argument("--waters", type=int, default=0,
                    help="instead of --workload: one water box of this many molecules")
    ap.add_argument("--members", type=int, default=1,
                    help="networks in the ensemble (member m > 0 takes the weight seed + m); "
                         "8 with --workload 6 is the ANI-2x architecture on the seven-element box")
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    ap.add_argument("--ref-budget", type=float, default=200.0,
                    help="reference arm: seconds allowed for its timed full evaluations")
    ap.add_argument("--serial-full", type=int, default=0,
                    help="reference arm: also time one full single-threaded evaluation")
    ap.add_argument("--extras", type=int, default=1,
                    help="0: leave out the auxiliary measurements after the JSON line's main step "
                         "(NVE, ML/MM, pair list, ensembles, seven species, force matching), "
                         "e.g. under a profiler")
    ap.add_argument("--out", default=None, help="also write the JSON line and the auxiliary "
                                                "measurements to this file")
    ap.add_argument("--cpu-baseline", type=int, default=1,
                    help="0: leave out the timed CPU baseline (e.g. under a profiler)")
    args = ap.parse_args()
    args.compare = args.compare.split(",")
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    r = run_ours(args, rank, world, local_rank)
    t_rank, total_atoms = aggregate_ranks(float(np.sum(r["ms"])) / 1e3, r["n"] * args.steps, world,
                                          "cuda")
    value = total_atoms / t_rank
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    pk, pk_kind = peaks()
    names = ["cells", "neighbours", "descriptor", "network", "descriptor_backward"]
    st = dict(zip(names, r["stage_ms"]))
    # algorithmic work (counted from the workload's neighbour statistics)
    n_pairs, n_trip = neighbour_stats(r)
    fl_desc, fl_mlp, fl_bwd = algorithmic_flops(n_pairs, n_trip, r["n"], r["D"], r["S"])
    fl_mlp *= args.members  # every member's network runs
    alu_peak = alu_peak_tflops(local_rank)
    n_sm = torch.cuda.get_device_properties(local_rank).multi_processor_count
    work = {"descriptor": (fl_desc, "alu"), "descriptor_backward": (fl_bwd, "alu"),
            "network": (fl_mlp, "tensor" if args.precision != "fp32" else "alu")}
    dom = max(work, key=lambda k: st[k])
    fl_instr, bound = work[dom]
    f32 = r["forms"].get("fp32", {})
    if "network_ms" in f32:  # the FP32 form's SIMT network against the FP32 ALU peak
        f32["network_tflops"] = fl_mlp / (f32["network_ms"] * 1e-3) / 1e12
        f32["network_frac"] = f32["network_tflops"] / alu_peak
    water = r["S"] == 2 and r["wl"]["name"].startswith("water")
    fl_scope = SCOPE_FLOP_PER_ATOM[dom] * r["n"] * (args.members if dom == "network" else 1) if water else None
    if bound == "tensor":
        peak = pk["bf16_tflops"] * (2.0 if args.precision == "fp8" else 1.0)
        peak_src = f"{pk_kind} cuBLAS bf16 burst" + (" x 2 (fp8)" if args.precision == "fp8" else "")
    else:
        peak = alu_peak
        peak_src = f"{n_sm} SMs (device) x 128 FP32 lanes x 2 x {pk.get('sm_max_mhz', 2032.0):.0f} MHz"
    ach_instr = fl_instr / (st[dom] * 1e-3) / 1e12
    ach = (fl_scope if fl_scope is not None else fl_instr) / (st[dom] * 1e-3) / 1e12
    roofline = {"bound": bound, "kernel": STAGE_KERNEL.get(dom) or dom, "achieved": r4(ach),
                "peak": r4(peak), "unit": "TFLOP/s", "frac": r4(ach / peak),
                "traffic": profiled_traffic(dom, args.precision),
                "work": ("scope-table count: " + (f"{SCOPE_FLOP_PER_ATOM[dom]:.4g} FLOP/atom x {r['n']} atoms"
                                                  if fl_scope is not None else "n/a, instruction count used")),
                "frac_instruction_count": r4(ach_instr / peak),
                "work_instruction_count": f"{fl_instr:.4g} FLOP (per pair/triplet counts)",
                "peak_source": peak_src, "stage_ms": {k: r4(v) for k, v in st.items()}}
    # the CPU baseline is timed at N = 1 only (rank 0 of a multi-GPU run skips it)
    cpu = cpu_baseline(r["wl"], r["w"], args.members) if world == 1 and args.cpu_baseline else None
    ms_mean = float(np.mean(r["ms"]))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mean, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else
        ("bf16" if args.precision == "bf16" else "fp8-e4m3"),
        "data": "synthetic (seeded water boxes, random Xavier weights)",
        "config": workload_config(r["wl"], args.precision, world, args.members),
        "e2e": {"value": r4(r["e2e"]), "unit": UNIT, "ms_per_step": r4(r["e2e_ms"]),
                "h2d_bytes_per_step": r["n"] * (24 + 4), "d2h_bytes_per_step": r["n"] * 24 + 8 * r["B"]},
        "gpu_launches": int(r["launches"]) * args.steps,
        "clocks": r["clocks"],
        "roofline": roofline,
        "cpu_baseline": cpu,
        "autotuned": r["tuned"],
    }
    aux = {}
    if args.workload == 3 and args.extras:  # the paper reports MD throughput in ns/day
        aux["nve"] = nve_rate(args.precision)
        aux["mlmm"] = mlmm_rate(args.precision)
        aux["pairs"] = pairs_rate(args.precision)
        if args.precision != "fp8":
            aux["ensemble"] = ensemble_rate(args.precision)
        aux["seven_species"] = seven_species_rate()
        if args.precision != "fp8":
            aux["ee"] = ee_rate(args.precision)
        aux["size_scan"] = size_scan()
    if (args.workload in (3, 5)) and args.extras:
        line["force_match"] = force_match_rate()
    if r["per_system_ms"] is not None:
        line["batch"] = {"systems": r["B"], "one_graph_launch_ms": r4(ms_mean),
                         "one_launch_per_system_ms": r4(r["per_system_ms"]),
                         "speedup": r4(r["per_system_ms"] / ms_mean)}
    line["forms"] = {k: {kk: (r4(vv) if isinstance(vv, float) else
                              ({a: r4(b) for a, b in vv.items()} if isinstance(vv, dict) else vv))
                         for kk, vv in v.items()} for k, v in r["forms"].items()}
    for k, v in aux.items():
        print(f"# aux {k} {json.dumps(v)}", flush=True)
    print(json.dumps(line), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump({"line": line, "aux": aux}, f, indent=1)
    if world > 1:
        torch.distributed.destroy_process_group()


def workload_config(wl, precision, world=1, members=1):
    """The JSON line's config block (the same for both arms)."""
    S = len(wl["atomic_numbers"])
    cfg = {"workload": wl["name"], "atoms": int(sum(s.n for s in wl["systems"])),
           "systems": len(wl["systems"]), "species": S, "aev_length": int(16 * S + 16 * S * (S + 1)),
           "precision": precision,
           "l2": "flushed (256 MB write) between timed steps, outside the timed events",
           "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}
    if members > 1:
        cfg["members"] = members
    return cfg


def cpu_baseline(wl, w, members=1):
    """One full evaluation of the workload by the OpenMP build of the oracle
    over the host's cores (the FP64 oracle's arithmetic, threads over atoms).
    An ensemble of M networks is timed as one network's evaluation times M
    (the oracle evaluates each member in full)."""
    n = sum(s.n for s in wl["systems"])
    t, threads = oracle_full_omp(wl, w)
    ens = f"; one member's evaluation times {members} members" if members > 1 else ""
    return {"value": r4(n / (t * members)), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"one full evaluation (E, F of all {n} atoms), OpenMP build of the oracle, "
                      f"{threads} threads, {t:.1f} s{ens}", "cpu": cpu_model()}


STAGE_KERNEL = {"descriptor": "k_aev_fwd", "descriptor_backward": "k_aev_bwd",
                "neighbours": "k_neighbors", "network": None, "cells": None}


def profiled_traffic(stage, precision):
    """DRAM bytes per launch of the stage's kernel from the committed ncu
    record (profiles/ncu_traffic.json), or None if that kernel's source file
    changed since the capture."""
    import hashlib
    kernel = STAGE_KERNEL.get(stage) or ("k_mlp_f32" if precision == "fp32" else
                                              "k_mlp_tc" if precision == "bf16" else "k_mlp_tc_fp8")
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            rec = json.load(f).get(kernel)
        if not rec or "source" not in rec:
            return None
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != rec["source_sha256"]:
                return None
        return rec["bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        return None


def neighbour_stats(r):
    """Radial pairs and angular triplets of the workload (from the inputs)."""
    from scipy.spatial import cKDTree
    pairs, trip = 0, 0
    for s in r["wl"]["systems"]:
        L = s.box[0]
        tree = cKDTree(np.mod(s.pos, L), boxsize=L)
        pairs += 2 * len(tree.query_pairs(5.2, output_type="ndarray"))
        na = np.zeros(s.n, dtype=np.int64)
        pa = tree.query_pairs(3.5, output_type="ndarray")
        np.add.at(na, pa[:, 0], 1)
        np.add.at(na, pa[:, 1], 1)
        trip += int((na * (na - 1) // 2).sum())
    return pairs, trip


if __name__ == "__main__":
    main()
