"""libnnp Python binding: ANI-style neural-network-potential energy and forces
on one B300 GPU.

Thin ctypes layer over the C ABI declared in include/nnp.h.  Every step of
an evaluation runs in the library's CUDA kernels; this module only marshals
arguments (NumPy arrays or torch tensors, host or device) and raises on
error codes.  There is no CPU fallback: if libnnp.so is missing the import
fails.

    from paper_2604_21441_b300 import NNP
    pot = NNP(atomic_numbers=(1, 8), precision="fp32")
    for s, layers in enumerate(weights):          # [(W1,b1),...,(W4,b4)]
        pot.set_weights(s, layers)
    E, F = pot.eval(pos, Z, box)                  # eV, eV/A
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["NNP", "NNPError", "lib", "LIB_PATH", "PRECISIONS", "ABI_FUNCTIONS", "write_weights",
           "read_weights"]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnnp.so")

NNP_MAX_SPECIES = 8
NNP_MAX_SHIFTS = 32
NNP_NOALLOC_MAX_ATOMS = 1024
PRECISIONS = {"fp32": 0, "bf16": 1, "fp8": 2}
FLAG_NO_GRAPH = 0x1
FLAG_NONDETERMINISTIC_BINS = 0x2
FLAG_STAGE_EVENTS = 0x4
FLAG_AUTOTUNE = 0x8
FLAG_CHARGES = 0x10
STAGES = ("cells", "neighbours", "descriptor", "network", "descriptor_backward")

# Every entry point declared in include/nnp.h.
ABI_FUNCTIONS = ("nnp_config_init", "nnp_create", "nnp_destroy", "nnp_last_error",
                 "nnp_set_weights", "nnp_eval", "nnp_eval_async", "nnp_sync",
                 "nnp_eval_batch", "nnp_param_count", "nnp_force_match_grad", "nnp_query",
                 "nnp_profile_stages", "nnp_atom_energies", "nnp_eval_noalloc", "nnp_eval_mlmm", "nnp_eval_pairs", "nnp_selftest",
                 "nnp_eval_batch_async", "nnp_set_member_weights", "nnp_set_charge_weights", "nnp_eval_ee",
                 "nnp_profile_force_match")

QUERY = {"launches_per_eval": 0, "nbr_capacity": 1, "ang_capacity": 2, "max_nbr": 3,
         "max_ang": 4, "rows": 5, "graph_captures": 6,
         "tune_neighbours": 7, "tune_descriptor": 8, "tune_backward": 9,
         "fp8_calibrated": 10, "tune_descriptor_tile": 11, "tune_backward_tile": 12,
         "tune_neighbours_form": 13, "tune_neighbours_queue": 13, "checked_build": 14, "fp8_passes": 15}

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNKNOWN_SPECIES", 3: "UNSUPPORTED", 4: "CAPACITY",
          5: "CUDA", 6: "TIMEOUT", 7: "NO_WEIGHTS", 8: "NO_STATE", 9: "BOUNDS"}


class NNPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libnnp {STATUS.get(code, code)}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [
        ("n_species", ctypes.c_int32),
        ("atomic_numbers", ctypes.c_int32 * NNP_MAX_SPECIES),
        ("rc_r", ctypes.c_double), ("eta_r", ctypes.c_double),
        ("n_rad", ctypes.c_int32),
        ("shf_r", ctypes.c_double * NNP_MAX_SHIFTS),
        ("rc_a", ctypes.c_double), ("eta_a", ctypes.c_double), ("zeta", ctypes.c_double),
        ("n_ang_r", ctypes.c_int32), ("n_ang_z", ctypes.c_int32),
        ("shf_a", ctypes.c_double * NNP_MAX_SHIFTS),
        ("shf_z", ctypes.c_double * NNP_MAX_SHIFTS),
        ("hidden", ctypes.c_int32 * 3),
        ("celu_alpha", ctypes.c_double),
        ("precision", ctypes.c_int32),
        ("max_atoms", ctypes.c_int64),
        ("max_systems", ctypes.c_int32),
        ("nbr_capacity", ctypes.c_int32),
        ("ang_capacity", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("flags", ctypes.c_uint32),
        ("n_members", ctypes.c_int32),
    ]


_lib = None

# Weight files (checkpoints of a model): one .npz with the species list, the
# member count and, per member m, species s and layer l, the arrays
# m{m}_s{s}_W{l} (fan_in x fan_out, float32) and m{m}_s{s}_b{l}.
WEIGHTS_FORMAT = 1


def write_weights(path, atomic_numbers, members):
    """members[m][s] = [(W1, b1), ..., (W4, b4)] of member m, species s."""
    arrays = {"format": np.int64(WEIGHTS_FORMAT),
              "atomic_numbers": np.asarray(atomic_numbers, dtype=np.int32),
              "n_members": np.int64(len(members))}
    for m, species in enumerate(members):
        if len(species) != len(atomic_numbers):
            raise ValueError(f"member {m}: {len(species)} species, expected {len(atomic_numbers)}")
        for sp, layers in enumerate(species):
            for l, (W, b) in enumerate(layers):
                arrays[f"m{m}_s{sp}_W{l}"] = np.ascontiguousarray(W, dtype=np.float32)
                arrays[f"m{m}_s{sp}_b{l}"] = np.ascontiguousarray(b, dtype=np.float32).reshape(-1)
    np.savez(path, **arrays)


def read_weights(path):
    """(atomic_numbers, members) from a file of write_weights."""
    with np.load(path) as f:
        if int(f["format"]) != WEIGHTS_FORMAT:
            raise ValueError(f"{path}: weight file format {int(f['format'])}, expected {WEIGHTS_FORMAT}")
        zs = tuple(int(z) for z in f["atomic_numbers"])
        members = []
        for m in range(int(f["n_members"])):
            species = []
            for sp in range(len(zs)):
                layers = []
                l = 0
                while f"m{m}_s{sp}_W{l}" in f.files:
                    layers.append((f[f"m{m}_s{sp}_W{l}"], f[f"m{m}_s{sp}_b{l}"]))
                    l += 1
                if not layers:
                    raise ValueError(f"{path}: no layers for member {m}, species {sp}")
                species.append(layers)
            members.append(species)
    return zs, members


def lib() -> ctypes.CDLL:
    """Load libnnp.so (built in-tree by paper_2604_21441_b300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2604_21441_b300.build` (no CPU fallback exists)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    L.nnp_config_init.argtypes = [ctypes.POINTER(Config), i32, ctypes.POINTER(i32)]
    L.nnp_config_init.restype = ctypes.c_int
    L.nnp_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(vp)]
    L.nnp_create.restype = ctypes.c_int
    L.nnp_destroy.argtypes = [vp]
    L.nnp_destroy.restype = None
    L.nnp_last_error.argtypes = [vp]
    L.nnp_last_error.restype = ctypes.c_char_p
    L.nnp_set_weights.argtypes = [vp, i32, ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.nnp_set_weights.restype = ctypes.c_int
    L.nnp_set_member_weights.argtypes = [vp, i32, i32, ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.nnp_set_member_weights.restype = ctypes.c_int
    L.nnp_eval.argtypes = [vp, i64, dp, dp, dp, dp, dp]
    L.nnp_eval.restype = ctypes.c_int
    L.nnp_eval_async.argtypes = [vp, i64, dp, dp, dp, dp, dp]
    L.nnp_eval_async.restype = ctypes.c_int
    L.nnp_sync.argtypes = [vp]
    L.nnp_sync.restype = ctypes.c_int
    L.nnp_eval_batch.argtypes = [vp, i32, dp, dp, dp, dp, dp, dp]
    L.nnp_eval_batch.restype = ctypes.c_int
    L.nnp_eval_batch_async.argtypes = [vp, i32, dp, dp, dp, dp, dp, dp]
    L.nnp_eval_batch_async.restype = ctypes.c_int
    L.nnp_param_count.argtypes = [vp]
    L.nnp_param_count.restype = i64
    L.nnp_force_match_grad.argtypes = [vp, dp, dp, dp, dp]
    L.nnp_force_match_grad.restype = ctypes.c_int
    L.nnp_query.argtypes = [vp, i32, ctypes.POINTER(i64)]
    L.nnp_query.restype = ctypes.c_int
    L.nnp_profile_stages.argtypes = [vp, ctypes.POINTER(ctypes.c_double), i32]
    L.nnp_profile_stages.restype = ctypes.c_int
    L.nnp_profile_force_match.argtypes = [vp, ctypes.POINTER(ctypes.c_double), i32]
    L.nnp_profile_force_match.restype = ctypes.c_int
    L.nnp_atom_energies.argtypes = [vp, dp]
    L.nnp_atom_energies.restype = ctypes.c_int
    L.nnp_eval_noalloc.argtypes = [vp, i64, dp, dp, dp, dp, dp]
    L.nnp_eval_noalloc.restype = ctypes.c_int
    L.nnp_eval_mlmm.argtypes = [vp, i64, dp, dp, dp, i64, dp, i32, dp, dp, dp, i32, dp, dp]
    L.nnp_eval_mlmm.restype = ctypes.c_int
    L.nnp_eval_pairs.argtypes = [vp, i64, dp, dp, dp, i64, dp, dp, dp, dp]
    L.nnp_set_charge_weights.argtypes = [vp, i32, ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.nnp_set_charge_weights.restype = ctypes.c_int
    L.nnp_eval_ee.argtypes = [vp, i64, dp, dp, dp, i64, dp, dp, ctypes.c_double, dp, dp, dp, dp]
    L.nnp_eval_ee.restype = ctypes.c_int
    L.nnp_eval_pairs.restype = ctypes.c_int
    L.nnp_selftest.argtypes = [vp, i32]
    L.nnp_selftest.restype = ctypes.c_int
    _lib = L
    return L


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, keepalive) of a contiguous array of the given numpy dtype."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch
        tdt = {np.float64: torch.float64, np.int32: torch.int32, np.float32: torch.float32,
               np.int64: torch.int64}[dtype]
        if x.dtype != tdt or not x.is_contiguous():
            x = x.to(tdt).contiguous()
        return ctypes.c_void_p(x.data_ptr()), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return ctypes.c_void_p(a.ctypes.data), a


def _box9(box):
    """None, 3 edge lengths or a 3x3 cell -> host float64[9] (or None)."""
    if box is None:
        return None
    b = box.detach().cpu().numpy() if _is_torch(box) else np.asarray(box)
    b = np.asarray(b, dtype=np.float64)
    if b.shape == (3,):
        b = np.diag(b)
    return np.ascontiguousarray(b.reshape(-1), dtype=np.float64)


class NNP:
    """One libnnp context (one CUDA stream)."""

    def __init__(self, atomic_numbers=(1, 8), precision: str = "fp32", max_atoms: int = 4096,
                 max_systems: int = 1, stream=None, flags: int = 0, n_members: int = 1, **overrides):
        L = lib()
        self._L = L
        zs = (ctypes.c_int32 * NNP_MAX_SPECIES)(*atomic_numbers)
        cfg = Config()
        rc = L.nnp_config_init(ctypes.byref(cfg), len(atomic_numbers), zs)
        if rc:
            raise NNPError(rc, "nnp_config_init rejected the species list")
        cfg.precision = PRECISIONS[precision]
        cfg.max_atoms = int(max_atoms)
        cfg.max_systems = int(max_systems)
        cfg.flags = int(flags)
        cfg.n_members = int(n_members)
        self.n_members = int(n_members)
        self.torch_stream = None
        if stream is not None:
            handle = stream if isinstance(stream, int) else stream.cuda_stream
            if not handle:
                raise ValueError("pass a non-default CUDA stream (the legacy default stream "
                                 "does not order against the library's own stream)")
            cfg.stream = ctypes.c_void_p(handle)
            if not isinstance(stream, int):
                self.torch_stream = stream
        for k, v in overrides.items():
            if k in ("shf_r", "shf_a", "shf_z"):
                arr = getattr(cfg, k)
                for i, x in enumerate(v):
                    arr[i] = x
            else:
                setattr(cfg, k, v)
        self.cfg = cfg
        self.atomic_numbers = tuple(atomic_numbers)
        self.n_species = len(atomic_numbers)
        self.precision = precision
        self._host_weights = {}  # (member, species) -> layers as set, for save_weights
        h = ctypes.c_void_p()
        rc = L.nnp_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc:
            raise NNPError(rc, L.nnp_last_error(None).decode())
        self._h = h

    # -- helpers
    def _check(self, rc):
        if rc:
            raise NNPError(rc, self._L.nnp_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.nnp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def aev_length(self) -> int:
        S = self.n_species
        return 16 * S + 32 * S * (S + 1) // 2

    def param_count(self) -> int:
        return int(self._L.nnp_param_count(self._h))

    def query(self, key: str) -> int:
        v = ctypes.c_int64()
        self._check(self._L.nnp_query(self._h, QUERY[key], ctypes.byref(v)))
        return int(v.value)

    # -- weights
    def set_weights(self, species: int, layers, member: int = 0):
        """layers = [(W1, b1), ..., (W4, b4)], W_l (fan_in x fan_out)."""
        keep, Wp, bp = [], (ctypes.c_void_p * 4)(), (ctypes.c_void_p * 4)()
        for l, (W, b) in enumerate(layers):
            pw, kw = _ptr(W, np.float32)
            pb, kb = _ptr(b, np.float32)
            keep += [kw, kb]
            Wp[l], bp[l] = pw.value, pb.value
        if member == 0:
            self._check(self._L.nnp_set_weights(self._h, int(species), Wp, bp))
        else:
            self._check(self._L.nnp_set_member_weights(self._h, int(member), int(species), Wp, bp))
        self._host_weights[int(member), int(species)] = [
            (np.array(W, dtype=np.float32, copy=True), np.array(b, dtype=np.float32, copy=True)) for W, b in layers]

    def save_weights(self, path):
        """Write every member's weights, as set, to a weight file (write_weights)."""
        members = []
        for m in range(self.n_members):
            species = []
            for sp in range(self.n_species):
                if (m, sp) not in self._host_weights:
                    raise ValueError(f"weights of member {m}, species {sp} were never set")
                species.append(self._host_weights[m, sp])
            members.append(species)
        write_weights(path, self.atomic_numbers, members)

    def load_weights(self, path):
        """Set every member's weights from a weight file; its species list and
        member count must be this context's."""
        zs, members = read_weights(path)
        if zs != self.atomic_numbers:
            raise ValueError(f"{path}: species {zs}, this context has {self.atomic_numbers}")
        self.set_member_weights(members)

    @classmethod
    def from_weights(cls, path, **kw):
        """A context for the species and member count of a weight file, with its weights."""
        zs, members = read_weights(path)
        pot = cls(atomic_numbers=zs, n_members=len(members), **kw)
        pot.set_member_weights(members)
        return pot

    def set_all_weights(self, weights, member: int = 0):
        for s, layers in enumerate(weights):
            self.set_weights(s, layers, member)

    def set_charge_weights(self, weights):
        """Charge network (context created with FLAG_CHARGES): per-species layers."""
        for s_, layers in enumerate(weights):
            keep, Wp, bp = [], (ctypes.c_void_p * 4)(), (ctypes.c_void_p * 4)()
            for l, (W, b) in enumerate(layers):
                pw, kw = _ptr(W, np.float32)
                pb, kb = _ptr(b, np.float32)
                keep += [kw, kb]
                Wp[l], bp[l] = pw.value, pb.value
            self._check(self._L.nnp_set_charge_weights(self._h, int(s_), Wp, bp))

    def eval_ee(self, pos, Z, mm_pos, mm_q, box=None, total_charge=0.0):
        """Electrostatic embedding: (E, F of the ML atoms, F of the MM charges,
        ML charges), on the library/device of pos."""
        n = int(pos.shape[0])
        m = int(mm_pos.shape[0])
        pp, kp = _ptr(pos, np.float64)
        pz, kz = _ptr(Z, np.int32)
        px, kx = _ptr(mm_pos, np.float64) if m else (None, None)
        pq, kq = _ptr(mm_q, np.float64) if m else (None, None)
        b9 = _box9(box)
        pbox = None if b9 is None else ctypes.c_void_p(b9.ctypes.data)
        if _is_torch(pos):
            import torch
            mk = lambda *shape: torch.zeros(shape, dtype=torch.float64, device=pos.device)
            E, F, Fm, q = mk(1), mk(n, 3), mk(max(m, 1), 3), mk(n)
            ptr = lambda t: ctypes.c_void_p(t.data_ptr())
        else:
            E, F, Fm, q = np.zeros(1), np.zeros((n, 3)), np.zeros((max(m, 1), 3)), np.zeros(n)
            ptr = lambda a: ctypes.c_void_p(a.ctypes.data)
        self._check(self._L.nnp_eval_ee(self._h, n, pp, pz, pbox, m, px, pq, float(total_charge),
                                        ptr(E), ptr(F), ptr(Fm), ptr(q)))
        return (float(E[0]) if not _is_torch(pos) else E[0]), F, Fm[:m], q

    def set_member_weights(self, members):
        """members[m] = per-species layers of ensemble member m (len = n_members)."""
        if len(members) != self.n_members:
            raise ValueError(f"expected {self.n_members} members, got {len(members)}")
        for m, weights in enumerate(members):
            self.set_all_weights(weights, m)

    # -- evaluation
    def eval(self, pos, Z, box=None, forces=True):
        """Energy (float) and forces (n x 3, same library/device as pos)."""
        n = int(pos.shape[0])
        pp, kp = _ptr(pos, np.float64)
        pz, kz = _ptr(Z, np.int32)
        b9 = _box9(box)
        pbox = None if b9 is None else ctypes.c_void_p(b9.ctypes.data)
        if _is_torch(pos):
            import torch
            E = torch.zeros(1, dtype=torch.float64, device=pos.device)
            F = torch.empty((n, 3), dtype=torch.float64, device=pos.device) if forces else None
            pE = ctypes.c_void_p(E.data_ptr())
            pF = ctypes.c_void_p(F.data_ptr()) if forces else None
        else:
            E = np.zeros(1)
            F = np.empty((n, 3)) if forces else None
            pE = ctypes.c_void_p(E.ctypes.data)
            pF = ctypes.c_void_p(F.ctypes.data) if forces else None
        self._check(self._L.nnp_eval(self._h, n, pp, pz, pbox, pE, pF))
        return (float(E[0]) if not _is_torch(pos) else E[0]), F

    def eval_into(self, pos, Z, box, E_out, F_out, sync: bool = True):
        """Device-pointer evaluation into caller buffers (torch CUDA tensors)."""
        b9 = _box9(box)
        pbox = None if b9 is None else ctypes.c_void_p(b9.ctypes.data)
        fn = self._L.nnp_eval if sync else self._L.nnp_eval_async
        self._check(fn(self._h, int(pos.shape[0]), ctypes.c_void_p(pos.data_ptr()),
                       ctypes.c_void_p(Z.data_ptr()), pbox,
                       ctypes.c_void_p(E_out.data_ptr()), ctypes.c_void_p(F_out.data_ptr())))

    def eval_mlmm(self, pos, Z, ml_index, link_ml=(), link_mm=(), link_d=None, link_Z=1, box=None):
        """ML/MM mechanical embedding: energy of the ML group plus link atoms,
        and forces on all atoms of the system (same library/device as pos)."""
        n = int(pos.shape[0])
        pp, kp = _ptr(pos, np.float64)
        pz, kz = _ptr(Z, np.int32)
        mi, kmi = _ptr(ml_index, np.int64)
        n_ml = int(ml_index.shape[0]) if hasattr(ml_index, "shape") else len(ml_index)
        n_link = len(link_ml)
        if n_link:
            pl, kl = _ptr(link_ml, np.int64)
            pm, km = _ptr(link_mm, np.int64)
        else:
            pl = pm = None
        pd, kd = _ptr(link_d, np.float64) if link_d is not None else (None, None)
        b9 = _box9(box)
        pbox = None if b9 is None else ctypes.c_void_p(b9.ctypes.data)
        if _is_torch(pos):
            import torch
            E = torch.zeros(1, dtype=torch.float64, device=pos.device)
            F = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
            pE, pF = ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(F.data_ptr())
        else:
            E, F = np.zeros(1), np.empty((n, 3))
            pE, pF = ctypes.c_void_p(E.ctypes.data), ctypes.c_void_p(F.ctypes.data)
        self._check(self._L.nnp_eval_mlmm(self._h, n, pp, pz, pbox, n_ml, mi, n_link, pl, pm, pd,
                                          int(link_Z), pE, pF))
        return (float(E[0]) if not _is_torch(pos) else E[0]), F

    def eval_pairs(self, pos, Z, pairs, shifts=None, box=None):
        """Energy and forces with the caller's pair list (n_pairs x 2 atom
        indices, each unordered pair once; optional n_pairs x 3 shifts)."""
        n = int(pos.shape[0])
        pp, kp = _ptr(pos, np.float64)
        pz, kz = _ptr(Z, np.int32)
        npairs = int(pairs.shape[0])
        pq, kq = _ptr(pairs, np.int32)
        ps, ks = _ptr(shifts, np.float64) if shifts is not None else (None, None)
        b9 = _box9(box)
        pbox = None if b9 is None else ctypes.c_void_p(b9.ctypes.data)
        if _is_torch(pos):
            import torch
            E = torch.zeros(1, dtype=torch.float64, device=pos.device)
            F = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
            pE, pF = ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(F.data_ptr())
        else:
            E, F = np.zeros(1), np.empty((n, 3))
            pE, pF = ctypes.c_void_p(E.ctypes.data), ctypes.c_void_p(F.ctypes.data)
        self._check(self._L.nnp_eval_pairs(self._h, n, pp, pz, pbox, npairs, pq, ps, pE, pF))
        return (float(E[0]) if not _is_torch(pos) else E[0]), F

    def selftest_wait_timeout(self):
        """Run the bounded-wait self-test; raises NNPError (code 6, timeout),
        which is the expected outcome."""
        self._check(self._L.nnp_selftest(self._h, 1))

    def selftest_bounds(self) -> int:
        """Run the bounds-check self-test; returns its status: 9 (BOUNDS) from
        the bounds-checked library, 3 (UNSUPPORTED) from the ordinary one."""
        return int(self._L.nnp_selftest(self._h, 2))

    def sync(self):
        self._check(self._L.nnp_sync(self._h))

    def eval_batch(self, offsets, pos, Z, boxes):
        """B systems: offsets (B+1), boxes (B x 3 edges or B x 3 x 3, or None)."""
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        B = off.shape[0] - 1
        n = int(off[-1])
        pp, kp = _ptr(pos, np.float64)
        pz, kz = _ptr(Z, np.int32)
        if boxes is None:
            pbx, bx = None, None
        else:
            bx = np.asarray(boxes, dtype=np.float64)
            if bx.ndim == 2 and bx.shape[1] == 3:
                bx = np.stack([np.diag(r) for r in bx])
            bx = np.ascontiguousarray(bx.reshape(B, 9))
            pbx = ctypes.c_void_p(bx.ctypes.data)
        if _is_torch(pos):
            import torch
            E = torch.zeros(B, dtype=torch.float64, device=pos.device)
            F = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
            pE, pF = ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(F.data_ptr())
        else:
            E = np.zeros(B)
            F = np.empty((n, 3))
            pE, pF = ctypes.c_void_p(E.ctypes.data), ctypes.c_void_p(F.ctypes.data)
        self._check(self._L.nnp_eval_batch(self._h, B, ctypes.c_void_p(off.ctypes.data), pp, pz,
                                           pbx, pE, pF))
        return E, F

    def eval_batch_into(self, offsets, pos, Z, boxes, E_out, F_out, sync: bool = True):
        """Batch evaluation on device tensors into caller buffers."""
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        bx = np.asarray(boxes, dtype=np.float64)
        if bx.ndim == 2 and bx.shape[1] == 3:
            bx = np.stack([np.diag(r) for r in bx])
        bx = np.ascontiguousarray(bx.reshape(-1, 9))
        fn = self._L.nnp_eval_batch if sync else self._L.nnp_eval_batch_async
        self._check(fn(self._h, int(off.shape[0] - 1), ctypes.c_void_p(off.ctypes.data),
                       ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(Z.data_ptr()),
                       ctypes.c_void_p(bx.ctypes.data), ctypes.c_void_p(E_out.data_ptr()),
                       ctypes.c_void_p(F_out.data_ptr())))

    def force_match_grad(self, v=None, Fref=None, want_loss: bool = False, out=None):
        """dL/dtheta (packed, nnp_param_count doubles) for the last eval.
        out: optional contiguous float64 buffer of that size (NumPy array or
        torch tensor, host or device) to write into; by default a new NumPy
        array."""
        npar = self.param_count()
        if out is None:
            out = np.zeros(npar)
        if _is_torch(out):
            if str(out.dtype) != "torch.float64" or not out.is_contiguous() or out.numel() != npar:
                raise ValueError("out must be a contiguous float64 tensor of param_count() entries")
            pg = ctypes.c_void_p(out.data_ptr())
        else:
            if out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"] or out.size != npar:
                raise ValueError("out must be a contiguous float64 array of param_count() entries")
            pg = ctypes.c_void_p(out.ctypes.data)
        pv, kv = _ptr(v, np.float64)
        pr, kr = _ptr(Fref, np.float64)
        loss = np.zeros(1)
        self._check(self._L.nnp_force_match_grad(
            self._h, pv, pr, ctypes.c_void_p(loss.ctypes.data) if want_loss else None, pg))
        return (float(loss[0]), out) if want_loss else out

    def atom_energies(self, n: int) -> np.ndarray:
        """Per-atom energies of the last evaluation (input order)."""
        out = np.zeros(n)
        self._check(self._L.nnp_atom_energies(self._h, ctypes.c_void_p(out.ctypes.data)))
        return out

    def profile_stages(self):
        out = (ctypes.c_double * 5)()
        self._check(self._L.nnp_profile_stages(self._h, out, 5))
        return list(out)

    def profile_force_match(self):
        """ms of the last force_match_grad's stages: forces, tangent
        descriptors, network passes, weight gradients."""
        out = (ctypes.c_double * 4)()
        self._check(self._L.nnp_profile_force_match(self._h, out, 4))
        return list(out)


def pack_weights(weights) -> np.ndarray:
    """Per-species [(W,b)...] -> the packed parameter layout of nnp_param_count."""
    parts = []
    for layers in weights:
        for W, b in layers:
            parts += [np.asarray(W, np.float64).reshape(-1), np.asarray(b, np.float64).reshape(-1)]
    return np.concatenate(parts)
