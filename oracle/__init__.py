"""FP64 CPU oracle of the NNP energy/force path (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may import this package.  The product library never loads it and
shares no code with it.

The arithmetic lives in ``nnp_oracle.c`` (plain C, double precision,
single-threaded); this module compiles it with gcc on first use and wraps it
with ctypes.  Descriptor constants are this module's own copy of the readings
of the ANI descriptor (radial: 16 shifts 0.9 + 0.26875 m, eta 16, cutoff
5.2 A; angular: 4 shifts 0.9 + 0.65 a, eta 8, zeta 32, sectors
(2z + 1) pi / 16, cutoff 3.5 A; CELU alpha 0.1).

Parity status per function
--------------------------
pairs_brute / pairs_cells : pinned (lattice shell counts, brute force = cells)
pairs_brute_cell           : pinned (shell counts of a triclinic lattice, equal
                             to pairs_brute for a rectangular cell)
aev                        : pinned (closed forms of special geometries,
                             invariances, block placement)
mlp                        : pinned (torch.nn.functional library routines)
energy_forces              : pinned (finite differences, sum F = 0,
                             translation / rotation / permutation invariance;
                             general cells: the same lattice in a sheared cell
                             gives the same result)
aev_jvp, force_match       : pinned (finite differences in positions and in
                             weights)
ensemble_energy_forces     : pinned (equals one wider network with
                             block-diagonal hidden layers and the output layer
                             divided by M; M copies of one network equal it)
ensemble_force_match       : pinned (finite differences of the ensemble loss
                             in each member's weights; the gradient of the
                             equivalent wider network, mapped back to the
                             members' blocks)
ee_energy_forces           : pinned (one ML atom and one MM charge: the
                             closed-form Coulomb pair; zero MM charges give
                             the plain NNP; total charge conserved; the total
                             force on ML and MM atoms vanishes; finite
                             differences in ML and MM coordinates)
mlmm_energy_forces         : pinned (finite differences of the embedded energy
                             in the whole system's coordinates, zero net
                             force, a link placed on its MM atom)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nnp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MAX_SPECIES = 8
MAX_SHF = 32
MAX_LAYERS = 8


_SRC_OMP = os.path.join(_HERE, "nnp_oracle_omp.c")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")


def build(force: bool = False) -> str:
    """Compile nnp_oracle.c into liboracle.so (no fast-math: FP64 as written),
    and the OpenMP build of the same source (liboracle_omp.so, used only to
    time the CPU baseline)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-shared",
                               "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_OMP))
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < newest:
        tmp = _LIB_OMP + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-shared",
                               "-fPIC", "-o", tmp, _SRC_OMP, "-lm"])
        os.replace(tmp, _LIB_OMP)
    return _LIB


class _Model(ctypes.Structure):
    _fields_ = [
        ("n_species", ctypes.c_int),
        ("n_rad", ctypes.c_int),
        ("n_ang_r", ctypes.c_int),
        ("n_ang_z", ctypes.c_int),
        ("rc_r", ctypes.c_double), ("eta_r", ctypes.c_double),
        ("rc_a", ctypes.c_double), ("eta_a", ctypes.c_double),
        ("zeta", ctypes.c_double),
        ("shf_r", ctypes.c_double * MAX_SHF),
        ("shf_a", ctypes.c_double * MAX_SHF),
        ("shf_z", ctypes.c_double * MAX_SHF),
        ("n_layers", ctypes.c_int),
        ("width", ctypes.c_int * (MAX_LAYERS + 1)),
        ("celu_alpha", ctypes.c_double),
        ("W", ctypes.POINTER(ctypes.c_double) * (MAX_SPECIES * MAX_LAYERS)),
        ("b", ctypes.POINTER(ctypes.c_double) * (MAX_SPECIES * MAX_LAYERS)),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.or_pairs_brute.restype = ctypes.c_long
        L.or_pairs_brute.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_long, ip, ip, dp]
        L.or_pairs_cells.restype = ctypes.c_long
        L.or_pairs_cells.argtypes = L.or_pairs_brute.argtypes
        L.or_pairs_brute_cell.restype = ctypes.c_long
        L.or_pairs_brute_cell.argtypes = L.or_pairs_brute.argtypes
        L.or_energy_forces_cell.argtypes = [ctypes.POINTER(_Model), ctypes.c_int, dp, ip, dp, dp, dp, dp, dp]
        L.or_aev_length.restype = ctypes.c_int
        L.or_aev.argtypes = [ctypes.POINTER(_Model), ctypes.c_int, ip, ctypes.c_long, ip, ip, dp, dp]
        L.or_mlp.restype = ctypes.c_double
        L.or_mlp.argtypes = [ctypes.POINTER(_Model), ctypes.c_int, dp, dp]
        L.or_energy_forces.argtypes = [ctypes.POINTER(_Model), ctypes.c_int, dp, ip, dp, dp, dp, dp, dp]
        L.or_energy_forces_subset.argtypes = [ctypes.POINTER(_Model), ctypes.c_int, dp, ip, dp,
                                              ctypes.c_int, ip, dp, ctypes.c_int, ip, dp]
        L.or_aev_jvp.argtypes = [ctypes.POINTER(_Model), ctypes.c_int, dp, ip, dp, dp, dp]
        L.or_force_match.argtypes = [ctypes.POINTER(_Model), ctypes.c_int, dp, ip, dp, dp, dp,
                                     ctypes.POINTER(dp), ctypes.POINTER(dp), dp]
        L.or_weighted_energy_forces.argtypes = [ctypes.POINTER(_Model), ctypes.c_int, dp, ip, dp, dp, dp, dp, dp]
        L.or_pair_index.restype = ctypes.c_int
        L.or_pair_index.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


@dataclass
class Params:
    """Descriptor and network hyper-parameters (the oracle's own copy)."""
    atomic_numbers: tuple = (1, 8)
    rc_r: float = 5.2
    eta_r: float = 16.0
    shf_r: tuple = tuple(0.9 + 0.26875 * m for m in range(16))
    rc_a: float = 3.5
    eta_a: float = 8.0
    zeta: float = 32.0
    shf_a: tuple = tuple(0.9 + 0.65 * a for a in range(4))
    shf_z: tuple = tuple((2 * z + 1) * math.pi / 16 for z in range(8))
    hidden: tuple = (160, 128, 96)
    celu_alpha: float = 0.1

    @property
    def n_species(self) -> int:
        return len(self.atomic_numbers)

    @property
    def aev_length(self) -> int:
        S = self.n_species
        return len(self.shf_r) * S + len(self.shf_a) * len(self.shf_z) * S * (S + 1) // 2

    def species_of(self, Z) -> np.ndarray:
        """Z -> species index in ascending-Z order; unknown Z raises."""
        order = sorted(self.atomic_numbers)
        lut = {z: k for k, z in enumerate(order)}
        try:
            return np.array([lut[int(z)] for z in np.asarray(Z)], dtype=np.int32)
        except KeyError as e:
            raise ValueError(f"unknown atomic number {e}") from None


class Model:
    """Parameters plus per-species weights [(W1,b1),...,(W4,b4)] (W: in x out)."""

    def __init__(self, params: Params, weights):
        self.p = params
        S = params.n_species
        if len(weights) != S:
            raise ValueError("need one weight set per species")
        self._keep = []
        m = _Model()
        m.n_species = S
        m.n_rad = len(params.shf_r)
        m.n_ang_r = len(params.shf_a)
        m.n_ang_z = len(params.shf_z)
        m.rc_r, m.eta_r = params.rc_r, params.eta_r
        m.rc_a, m.eta_a, m.zeta = params.rc_a, params.eta_a, params.zeta
        for k, v in enumerate(params.shf_r):
            m.shf_r[k] = v
        for k, v in enumerate(params.shf_a):
            m.shf_a[k] = v
        for k, v in enumerate(params.shf_z):
            m.shf_z[k] = v
        widths = (params.aev_length,) + tuple(params.hidden) + (1,)
        m.n_layers = len(widths) - 1
        for k, w in enumerate(widths):
            m.width[k] = w
        m.celu_alpha = params.celu_alpha
        for s in range(S):
            if len(weights[s]) != m.n_layers:
                raise ValueError("wrong number of layers")
            for l, (W, b) in enumerate(weights[s]):
                W = np.ascontiguousarray(W, dtype=np.float64)
                b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
                if W.shape != (widths[l], widths[l + 1]) or b.shape != (widths[l + 1],):
                    raise ValueError(f"layer {l} of species {s} has shape {W.shape}")
                self._keep += [W, b]
                m.W[s * MAX_LAYERS + l] = _dp(W)
                m.b[s * MAX_LAYERS + l] = _dp(b)
        self.widths = widths
        self.weights = weights
        self._m = m

    @property
    def ref(self):
        return ctypes.byref(self._m)


def _pairs(fn, pos, box, rc):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = pos.shape[0]
    bx = None if box is None else np.ascontiguousarray(box, dtype=np.float64)
    cap = max(16, n * 128)
    while True:
        pi = np.empty(cap, np.int32)
        pj = np.empty(cap, np.int32)
        pd = np.empty((cap, 3), np.float64)
        cnt = fn(n, _dp(pos), None if bx is None else _dp(bx), rc, cap, _ip(pi), _ip(pj), _dp(pd))
        if cnt <= cap:
            return pi[:cnt].copy(), pj[:cnt].copy(), pd[:cnt].copy()
        cap = int(cnt)


def pairs_brute(pos, box, rc):
    """(i, j, d) of every pair/image within rc, brute force over images."""
    return _pairs(lib().or_pairs_brute, pos, box, rc)


def pairs_brute_cell(pos, cell, rc):
    """(i, j, d) of every pair/image within rc in a general periodic cell
    (3 x 3, rows = cell vectors), brute force over images."""
    return _pairs(lib().or_pairs_brute_cell, pos, np.asarray(cell, dtype=np.float64).reshape(9), rc)


def pairs_cells(pos, box, rc):
    """Same set as pairs_brute, through a cell list."""
    return _pairs(lib().or_pairs_cells, pos, box, rc)


def pair_index(S, s1, s2) -> int:
    return lib().or_pair_index(S, s1, s2)


def aev(model: Model, species, pairs) -> np.ndarray:
    pi, pj, pd = pairs
    species = np.ascontiguousarray(species, dtype=np.int32)
    n = species.shape[0]
    G = np.zeros((n, model.p.aev_length))
    lib().or_aev(model.ref, n, _ip(species), len(pi), _ip(np.ascontiguousarray(pi)),
                 _ip(np.ascontiguousarray(pj)), _dp(np.ascontiguousarray(pd)), _dp(G))
    return G


def mlp(model: Model, s: int, x) -> tuple[float, np.ndarray]:
    x = np.ascontiguousarray(x, dtype=np.float64)
    dx = np.zeros_like(x)
    e = lib().or_mlp(model.ref, int(s), _dp(x), _dp(dx))
    return e, dx


def energy_forces(model: Model, pos, species, box):
    """E (float), Ei (n,), F (n,3), G (n,D).  box: None (isolated), 3 edge
    lengths (orthorhombic) or a 3 x 3 cell whose rows are the cell vectors
    (general periodic cell, pairs by brute force over images)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    species = np.ascontiguousarray(species, dtype=np.int32)
    n = pos.shape[0]
    bx = None if box is None else np.ascontiguousarray(box, dtype=np.float64)
    E = np.zeros(1)
    Ei = np.zeros(n)
    F = np.zeros((n, 3))
    G = np.zeros((n, model.p.aev_length))
    if bx is not None and bx.size == 9:
        lib().or_energy_forces_cell(model.ref, n, _dp(pos), _ip(species), _dp(bx.reshape(9)),
                                    _dp(E), _dp(Ei), _dp(F), _dp(G))
    else:
        lib().or_energy_forces(model.ref, n, _dp(pos), _ip(species),
                               None if bx is None else _dp(bx), _dp(E), _dp(Ei), _dp(F), _dp(G))
    return float(E[0]), Ei, F, G


def energy_forces_subset(model: Model, pos, species, box, sel_e, sel_f):
    """E_i for atoms sel_e and F_j for atoms sel_f of a (large) system, each
    by the same definition as energy_forces."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    species = np.ascontiguousarray(species, dtype=np.int32)
    sel_e = np.ascontiguousarray(sel_e, dtype=np.int32)
    sel_f = np.ascontiguousarray(sel_f, dtype=np.int32)
    n = pos.shape[0]
    bx = None if box is None else np.ascontiguousarray(box, dtype=np.float64)
    Ei = np.zeros(len(sel_e))
    F = np.zeros((len(sel_f), 3))
    lib().or_energy_forces_subset(model.ref, n, _dp(pos), _ip(species),
                                  None if bx is None else _dp(bx), len(sel_e), _ip(sel_e),
                                  _dp(Ei), len(sel_f), _ip(sel_f), _dp(F))
    return Ei, F


def aev_jvp(model: Model, pos, species, box, v) -> np.ndarray:
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    species = np.ascontiguousarray(species, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.float64)
    n = pos.shape[0]
    bx = None if box is None else np.ascontiguousarray(box, dtype=np.float64)
    T = np.zeros((n, model.p.aev_length))
    lib().or_aev_jvp(model.ref, n, _dp(pos), _ip(species),
                     None if bx is None else _dp(bx), _dp(v), _dp(T))
    return T


def force_match(model: Model, pos, species, box, Fref):
    """L, dW (list per species of per-layer arrays), db (same), F."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    species = np.ascontiguousarray(species, dtype=np.int32)
    Fref = np.ascontiguousarray(Fref, dtype=np.float64)
    n = pos.shape[0]
    bx = None if box is None else np.ascontiguousarray(box, dtype=np.float64)
    S = model.p.n_species
    dW = [[np.zeros_like(np.asarray(W, dtype=np.float64)) for W, _ in model.weights[s]]
          for s in range(S)]
    db = [[np.zeros(np.asarray(b).reshape(-1).shape[0]) for _, b in model.weights[s]]
          for s in range(S)]
    PW = (ctypes.POINTER(ctypes.c_double) * (MAX_SPECIES * MAX_LAYERS))()
    PB = (ctypes.POINTER(ctypes.c_double) * (MAX_SPECIES * MAX_LAYERS))()
    for s in range(S):
        for l in range(len(dW[s])):
            PW[s * MAX_LAYERS + l] = _dp(dW[s][l])
            PB[s * MAX_LAYERS + l] = _dp(db[s][l])
    L = np.zeros(1)
    F = np.zeros((n, 3))
    lib().or_force_match(model.ref, n, _dp(pos), _ip(species), None if bx is None else _dp(bx),
                         _dp(Fref), _dp(L), PW, PB, _dp(F))
    return float(L[0]), dW, db, F


def ensemble_energy_forces(models, pos, species, box):
    """Ensemble of M networks of one architecture over one descriptor (the
    ANI-2x model of the performance-scaling study in the Results is an
    ensemble of eight): energy, per-atom energies and forces are the means of
    the members' values.  Returns E, Ei (n,), F (n, 3)."""
    M = len(models)
    E, Ei, F = 0.0, 0.0, 0.0
    for m in models:
        e, ei, f, _ = energy_forces(m, pos, species, box)
        E, Ei, F = E + e, Ei + ei, F + f
    return E / M, Ei / M, F / M


_lib_omp = None


def energy_forces_omp(model: Model, pos, species, box):
    """energy_forces computed by the OpenMP build of the same source (all
    host cores unless OMP_NUM_THREADS says otherwise): the per-atom work is
    the oracle's own, only the energy and force sums are grouped per thread.
    For timing the CPU baseline.  Returns E, Ei, F, threads."""
    global _lib_omp
    if _lib_omp is None:
        build()
        L = ctypes.CDLL(_LIB_OMP)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.or_energy_forces_omp.argtypes = [ctypes.POINTER(_Model), ctypes.c_int, dp, ip, dp, dp, dp, dp]
        L.or_omp_threads.restype = ctypes.c_int
        _lib_omp = L
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    species = np.ascontiguousarray(species, dtype=np.int32)
    n = pos.shape[0]
    bx = None if box is None else np.ascontiguousarray(box, dtype=np.float64)
    E, Ei, F = np.zeros(1), np.zeros(n), np.zeros((n, 3))
    _lib_omp.or_energy_forces_omp(model.ref, n, _dp(pos), _ip(species), None if bx is None else _dp(bx),
                                  _dp(E), _dp(Ei), _dp(F))
    return float(E[0]), Ei, F, int(_lib_omp.or_omp_threads())


def ensemble_force_match(models, pos, species, box, Fref):
    """Force matching of an ensemble of M networks (mean energy, Results on
    ANI-2x's eight networks; Eq. 2's forces): L = |F - Fref|^2 / (3N) with F
    the members' mean force, and dL/dtheta for every member's weights.

    The ensemble energy is (1/M) sum_m E_m, so member m's gradient is 1/M
    times the single-network gradient of E_m taken along the ensemble's
    v = 2 (F - Fref) / (3N).  force_match of member m with the reference
    F_m - F + Fref has exactly that v.  Returns L, dW, db (lists over
    members of per-species per-layer arrays), F."""
    M = len(models)
    Fm = [energy_forces(m, pos, species, box)[2] for m in models]
    F = sum(Fm) / M
    Fref = np.asarray(Fref, dtype=np.float64)
    L = float(((F - Fref) ** 2).sum() / (3 * F.shape[0]))
    dWs, dbs = [], []
    for m, Fmm in zip(models, Fm):
        _, dW, db, _ = force_match(m, pos, species, box, Fmm - F + Fref)
        dWs.append([[x / M for x in sp] for sp in dW])
        dbs.append([[x / M for x in sp] for sp in db])
    return L, dWs, dbs, F


def weighted_energy_forces(model: Model, pos, species, box, wt):
    """E = sum_i wt_i E_i and F = -dE/dr with the weights held fixed
    (orthorhombic box or None).  Returns E, Ei (unweighted), F."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    species = np.ascontiguousarray(species, dtype=np.int32)
    wt = np.ascontiguousarray(wt, dtype=np.float64)
    n = pos.shape[0]
    bx = None if box is None else np.ascontiguousarray(box, dtype=np.float64)
    E, Ei, F = np.zeros(1), np.zeros(n), np.zeros((n, 3))
    lib().or_weighted_energy_forces(model.ref, n, _dp(pos), _ip(species), None if bx is None else _dp(bx),
                                    _dp(wt), _dp(E), _dp(Ei), _dp(F))
    return float(E[0]), Ei, F


COULOMB_EV_A = 14.3996454784  # e^2 / (4 pi eps0) in eV A


def ee_energy_forces(model: Model, charge_model: Model, pos, species, box, mm_pos, mm_q,
                     total_charge: float = 0.0):
    """Electrostatic embedding (Methods, the nnpot interface: the model
    predicts in vacuo charges of the ML atoms, which interact with the MM
    point charges; the MM atoms receive forces).  Readings:

    * charges: q_i = charge_model's per-element network on the same
      descriptor, shifted so that they sum to total_charge,
      q'_i = q_i - (sum_k q_k - Q) / n;
    * E = E_NNP + E_es, E_es = k_e sum_i sum_J q'_i Q_J / |r_iJ|, over every
      MM charge J; with a box (edge lengths) r_iJ is the minimum image;
    * no polarisation term.

    Returns E, F (ML atoms, n x 3), F_mm (MM atoms, m x 3), q' (n)."""
    pos = np.asarray(pos, dtype=np.float64)
    mm_pos = np.asarray(mm_pos, dtype=np.float64).reshape(-1, 3)
    mm_q = np.asarray(mm_q, dtype=np.float64).reshape(-1)
    n = pos.shape[0]
    E_nnp, _, F_nnp, _ = energy_forces(model, pos, species, box)
    _, q_raw, _, _ = energy_forces(charge_model, pos, species, box)
    q = q_raw - (q_raw.sum() - total_charge) / n
    V = np.zeros(n)
    field = np.zeros((n, 3))  # -grad V at the ML atom
    F_mm = np.zeros_like(mm_pos)
    for i in range(n):
        d = mm_pos - pos[i]  # r_J - r_i
        if box is not None:
            L = np.asarray(box, dtype=np.float64)
            d -= L * np.round(d / L)
        r = np.sqrt((d * d).sum(axis=1))
        V[i] = COULOMB_EV_A * np.sum(mm_q / r)
        pair = COULOMB_EV_A * (mm_q / r ** 3)[:, None] * d  # k Q_J (r_J - r_i) / r^3
        field[i] = -pair.sum(axis=0)
        F_mm += q[i] * pair
    E_es = float(np.sum(q * V))
    # charge dependence: dE_es/dq_raw_i = V_i - mean(V) (neutrality shift)
    _, _, F_q = weighted_energy_forces(charge_model, pos, species, box, V - V.mean())
    F = F_nnp + q[:, None] * field + F_q
    return E_nnp + E_es, F, F_mm, q


def mlmm_energy_forces(model: Model, pos, species, box, ml_index, link_ml, link_mm, link_d,
                       link_species):
    """ML/MM mechanical embedding (Sec. Methods, the nnpot interface and its
    link-atom equation): the NNP on the ML group (pos[ml_index], in that
    order) followed by one link atom per cut bond at
        r_L = r_ML + d (r_MM - r_ML) / |r_MM - r_ML|
    (minimum image in the orthorhombic box), of species link_species.
    Returns E, the forces on all atoms (group atoms their own, link forces
    passed to the bonded pair by the chain rule of that equation, all other
    atoms zero) and the subsystem's atom energies (group, then links)."""
    pos = np.asarray(pos, dtype=np.float64)
    species = np.asarray(species)
    ml_index = np.asarray(ml_index, dtype=np.int64)
    link_ml = np.asarray(link_ml, dtype=np.int64)
    link_mm = np.asarray(link_mm, dtype=np.int64)
    nl = len(link_ml)
    d = np.ones(nl) if link_d is None else np.asarray(link_d, dtype=np.float64)
    L = None if box is None else np.asarray(box, dtype=np.float64)

    def bond(i, j):
        R = pos[j] - pos[i]
        if L is not None:
            R = R - L * np.round(R / L)
        return R

    sub = [pos[a] for a in ml_index]
    for l in range(nl):
        R = bond(link_ml[l], link_mm[l])
        sub.append(pos[link_ml[l]] + d[l] * R / np.linalg.norm(R))
    sub = np.array(sub)
    sub_species = np.concatenate([species[ml_index], np.full(nl, link_species)]).astype(np.int32)
    E, Ei, Fs, _ = energy_forces(model, sub, sub_species, box)
    F = np.zeros_like(pos)
    F[ml_index] = Fs[:len(ml_index)]
    for l in range(nl):
        i, j = link_ml[l], link_mm[l]
        R = bond(i, j)
        r = np.linalg.norm(R)
        u = R / r
        FL = Fs[len(ml_index) + l]
        # dr_L/dr_MM = (d/r)(I - u u^T) (symmetric); dr_L/dr_ML = I - dr_L/dr_MM
        J = (d[l] / r) * (np.eye(3) - np.outer(u, u))
        F[j] += J @ FL
        F[i] += FL - J @ FL
    return E, F, Ei
