"""PyTorch autograd functions and a velocity-Verlet NVE driver over libnnp.

Argument marshalling only: every energy, force and gradient comes from the
library's CUDA kernels (through the C ABI).

    E = nnp_energy(pot, pos, Z, box)          # d E / d pos = -F (library forces)
    L = force_match_loss(pot, params, pos, Z, box, Fref)
                                              # d L / d params from nnp_force_match_grad
    E, F = nnp_forces(pot, params, pos, Z, box)
                                              # d(any loss of F) / d params via dL/dF

params is a flat float64 tensor in the packed layout of nnp_param_count
(per species W1 b1 W2 b2 W3 b3 W4 b4, each W row-major fan_in x fan_out).
"""
from __future__ import annotations

import numpy as np
import torch

from . import NNP

# 1 eV / (A amu) in A / fs^2
ACC_UNIT = 9.64853321e-3
MASS = {1: 1.008, 6: 12.011, 7: 14.007, 8: 15.999, 16: 32.06, 9: 18.998, 17: 35.45}


def layer_shapes(pot: NNP):
    D = pot.aev_length
    w = (D, 160, 128, 96, 1)
    return [(w[l], w[l + 1]) for l in range(4)]


def unpack_params(pot: NNP, params) -> list:
    """Flat packed parameters -> per-species [(W1,b1),...,(W4,b4)] (float32, host)."""
    p = params.detach().cpu().numpy() if torch.is_tensor(params) else np.asarray(params)
    out, k = [], 0
    for _ in range(pot.n_species):
        layers = []
        for fi, fo in layer_shapes(pot):
            W = p[k:k + fi * fo].reshape(fi, fo)
            k += fi * fo
            b = p[k:k + fo]
            k += fo
            layers.append((W.astype(np.float32), b.astype(np.float32)))
        out.append(layers)
    assert k == p.size, "parameter vector has the wrong length"
    return out


def pack_params(weights) -> torch.Tensor:
    parts = []
    for layers in weights:
        for W, b in layers:
            parts += [np.asarray(W, np.float64).reshape(-1), np.asarray(b, np.float64).reshape(-1)]
    return torch.tensor(np.concatenate(parts))


def _box9(box):
    b = box.detach().cpu().numpy() if torch.is_tensor(box) else np.asarray(box, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.diag(b) if b.shape == (3,) else b.reshape(3, 3)


class _Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, pot, Z, box):
        E, F = pot.eval(pos.detach().contiguous(), Z, _box9(box))
        F = torch.as_tensor(F, device=pos.device, dtype=pos.dtype)
        ctx.save_for_backward(F)
        return torch.as_tensor(E, device=pos.device, dtype=pos.dtype).reshape(())

    @staticmethod
    def backward(ctx, gE):
        (F,) = ctx.saved_tensors
        return -F * gE, None, None, None


def nnp_energy(pot: NNP, pos: torch.Tensor, Z, box) -> torch.Tensor:
    """Energy (eV) differentiable in positions: dE/dpos = -F (Eq. 2)."""
    return _Energy.apply(pos, pot, Z, box)


class _Forces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, pot, pos, Z, box):
        pot.set_all_weights(unpack_params(pot, params))
        E, F = pot.eval(pos.detach().contiguous(), Z, _box9(box))
        ctx.pot = pot
        F = torch.as_tensor(F, dtype=torch.float64, device=pos.device)
        return torch.as_tensor(E, dtype=torch.float64, device=pos.device).reshape(()), F

    @staticmethod
    def backward(ctx, gE, gF):
        if gF is None:
            return None, None, None, None, None
        v = gF.detach().to(torch.float64).contiguous()
        g = ctx.pot.force_match_grad(v=v)
        return torch.as_tensor(g, dtype=torch.float64), None, None, None, None


def nnp_forces(pot: NNP, params: torch.Tensor, pos, Z, box):
    """(E, F) with F differentiable in the packed parameters (energy is not)."""
    return _Forces.apply(params, pot, pos, Z, box)


class _ForceMatch(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, pot, pos, Z, box, Fref):
        pot.set_all_weights(unpack_params(pot, params))
        pot.eval(pos.detach().contiguous(), Z, _box9(box), forces=False)
        fr = Fref.detach().to(torch.float64).contiguous() if torch.is_tensor(Fref) else Fref
        L, g = pot.force_match_grad(Fref=fr, want_loss=True)
        ctx.save_for_backward(torch.as_tensor(g, dtype=torch.float64))
        return torch.tensor(L, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gL):
        (g,) = ctx.saved_tensors
        return g * gL, None, None, None, None, None


def force_match_loss(pot: NNP, params, pos, Z, box, Fref) -> torch.Tensor:
    """L = |F - Fref|^2 / (3N), differentiable in the packed parameters."""
    return _ForceMatch.apply(params, pot, pos, Z, box, Fref)


class NVE:
    """Velocity-Verlet NVE integrator with device-resident state.

    r (n x 3, A), v (n x 3, A/fs) and the library forces stay on the GPU; one
    step costs one library evaluation plus four elementwise updates.
    """

    def __init__(self, pot: NNP, pos, Z, box, vel, dt_fs: float = 0.5, device="cuda"):
        # the elementwise updates must run on the library's stream
        if pot.torch_stream is None:
            raise ValueError("create the NNP with stream=<a torch.cuda.Stream> for NVE")
        self.stream = pot.torch_stream
        self.pot = pot
        self.retries = 0
        self.dt = dt_fs
        self.Z = torch.as_tensor(np.asarray(Z, dtype=np.int32), device=device)
        self.r = torch.as_tensor(np.asarray(pos, dtype=np.float64), device=device).clone()
        self.v = torch.as_tensor(np.asarray(vel, dtype=np.float64), device=device).clone()
        m = np.array([MASS[int(z)] for z in np.asarray(Z)])
        self.inv_m = torch.as_tensor(ACC_UNIT / m, device=device)[:, None]
        self.m = torch.as_tensor(m, device=device)[:, None]
        self.box = np.diag(np.asarray(box, dtype=np.float64))
        self.E = torch.zeros(1, dtype=torch.float64, device=device)
        self.F = torch.zeros_like(self.r)
        self.steps_done = 0
        torch.cuda.synchronize()
        self.pot.eval_into(self.r, self.Z, self.box, self.E, self.F, sync=True)

    def save(self, path):
        """Checkpoint of the state: positions, velocities, steps done, time
        step, atomic numbers and box (one .npz).  Forces are recomputed on
        restore, from the same positions."""
        self.stream.synchronize()
        np.savez(path, r=self.r.cpu().numpy(), v=self.v.cpu().numpy(), steps_done=np.int64(self.steps_done),
                 dt_fs=np.float64(self.dt), Z=self.Z.cpu().numpy(), box=np.diag(self.box))

    @classmethod
    def restore(cls, path, pot: NNP, device="cuda"):
        """An integrator that continues from a checkpoint of save()."""
        with np.load(path) as f:
            nve = cls(pot, f["r"], f["Z"], f["box"], f["v"], dt_fs=float(f["dt_fs"]), device=device)
            nve.steps_done = int(f["steps_done"])
        return nve

    def kinetic(self) -> torch.Tensor:
        with torch.cuda.stream(self.stream):
            return 0.5 * (self.m * self.v * self.v).sum() / ACC_UNIT  # eV

    def _chunk(self, n: int):
        half = 0.5 * self.dt
        with torch.cuda.stream(self.stream):
            for _ in range(n):
                self.v.add_(self.F * self.inv_m, alpha=half)
                self.r.add_(self.v, alpha=self.dt)
                self.pot.eval_into(self.r, self.Z, self.box, self.E, self.F, sync=False)
                self.v.add_(self.F * self.inv_m, alpha=half)

    def step(self, n: int = 1, check_every: int = 100, max_retries: int = 4):
        """n steps.  Device flags are checked every check_every steps; if the
        neighbour lists overflowed (capacity is then grown by the library),
        the state rolls back to the last check and the chunk is redone."""
        from . import NNPError
        done = 0
        while done < n:
            k = min(check_every, n - done) if check_every else n - done
            snap = [t.clone() for t in (self.r, self.v, self.F, self.E)]
            for attempt in range(max_retries + 1):
                self._chunk(k)
                try:
                    self.pot.sync()
                    break
                except NNPError as e:
                    if e.code != 4 or attempt == max_retries:
                        raise
                    self.retries += 1
                    with torch.cuda.stream(self.stream):
                        for t, s in zip((self.r, self.v, self.F, self.E), snap):
                            t.copy_(s)
                    self.stream.synchronize()
            done += k
            self.steps_done += k

    def total_energy(self) -> float:
        ek = self.kinetic()
        self.stream.synchronize()
        return float(self.E[0]) + float(ek)
