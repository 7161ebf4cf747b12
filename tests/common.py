"""Shared helpers of the test-suite (inputs and comparison only)."""
import numpy as np

import synth

# FP32 form bounds (stated by the target): relative energy error 1e-6 with
# the normalisation max(|E|, sum_i |E_i|), max |dF| 1e-4 eV/A.
E_REL_TOL = 1e-6
F_ABS_TOL = 1e-4


def weights32(n_species, d_in, seed, bias_seed=None):
    """Weights rounded to FP32 (what the library stores), as float64 arrays
    so that the oracle evaluates exactly the same function."""
    w = synth.xavier_weights(n_species, d_in, seed)
    if bias_seed is not None:
        w = synth.random_biases(w, bias_seed)
    return [[(W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64))
             for W, b in sp] for sp in w]


def energy_error(E, E_ref, Ei_ref):
    return abs(E - E_ref) / max(abs(E_ref), float(np.abs(Ei_ref).sum()))


def box9(box):
    return None if box is None else np.diag(np.asarray(box, dtype=np.float64))


def targeted_atoms(pos, box, rng, n_random=128, face_depth=0.5, per_face=4, per_corner=2,
                   n_crowded=32, rc_a=3.5):
    """Atoms that a sampled full-size check must include (cubic or
    orthorhombic box, edges `box`):
      * n_random atoms drawn at random;
      * per_face atoms within face_depth of each of the six faces (after
        wrapping), whose neighbours lie across the periodic boundary;
      * per_corner atoms nearest each of the eight corners, whose
        neighbours are images through up to three faces at once;
      * the n_crowded atoms with the most neighbours within rc_a (the
        longest angular pair loops).
    Returns a sorted array of distinct indices."""
    from scipy.spatial import cKDTree
    L = np.asarray(box, dtype=np.float64)
    x = np.mod(pos, L)
    n = len(x)
    picks = [rng.choice(n, min(n_random, n), replace=False)]
    for d in range(3):
        for near in (x[:, d] < face_depth, x[:, d] > L[d] - face_depth):
            idx = np.flatnonzero(near)
            if idx.size:
                picks.append(rng.choice(idx, min(per_face, idx.size), replace=False))
    for c in range(8):
        corner = L * np.array([(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1])
        d = x - corner
        d -= L * np.round(d / L)
        picks.append(np.argsort(np.einsum("ij,ij->i", d, d))[:per_corner])
    tree = cKDTree(x, boxsize=L)
    cnt = np.zeros(n, dtype=np.int64)
    pa = tree.query_pairs(rc_a, output_type="ndarray")
    np.add.at(cnt, pa[:, 0], 1)
    np.add.at(cnt, pa[:, 1], 1)
    picks.append(np.argsort(-cnt, kind="stable")[:n_crowded])
    return np.unique(np.concatenate(picks)).astype(np.int64)


def _subset_job(job):
    import oracle
    Zs, weights, pos, Z, box, sel_e, sel_f = job
    p = oracle.Params(atomic_numbers=Zs)
    m = oracle.Model(p, weights)
    return oracle.energy_forces_subset(m, pos, p.species_of(Z), box, sel_e, sel_f)


def oracle_subset(Zs, weights, pos, Z, box, sel_e, sel_f, chunk=24, workers=None):
    """The oracle's E_i (atoms sel_e) and F_j (atoms sel_f) of a large system,
    the force atoms split into chunks evaluated by worker processes (spawned,
    so that none inherits a CUDA context).  Same values as one
    oracle.energy_forces_subset call."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    sel_f = np.asarray(sel_f, dtype=np.int64)
    parts = [sel_f[k:k + chunk] for k in range(0, len(sel_f), chunk)] or [sel_f]
    jobs = [(tuple(Zs), weights, pos, Z, box, np.asarray(sel_e) if k == 0 else np.zeros(0, np.int64), f)
            for k, f in enumerate(parts)]
    nw = workers or max(1, min(len(jobs), (os.cpu_count() or 2) - 1, 32))
    with cf.ProcessPoolExecutor(nw, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_subset_job, jobs))
    Ei = res[0][0]
    F = np.concatenate([r[1] for r in res]) if len(sel_f) else np.zeros((0, 3))
    return Ei, F


def oracle_energy_forces_job(Zs, weights, pos, Z, box):
    """oracle.energy_forces as a job for a spawned worker: (E, E_i, F)."""
    import oracle
    p = oracle.Params(atomic_numbers=tuple(Zs))
    E, Ei, F, _ = oracle.energy_forces(oracle.Model(p, weights), pos, p.species_of(Z), box)
    return E, Ei, F


def oracle_force_match_job(Zs, weights, pos, Z, box, Fref):
    """oracle.force_match as a job for a spawned worker: (L, dW, db, F)."""
    import oracle
    p = oracle.Params(atomic_numbers=tuple(Zs))
    return oracle.force_match(oracle.Model(p, weights), pos, p.species_of(Z), box, Fref)
