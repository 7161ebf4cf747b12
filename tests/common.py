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
