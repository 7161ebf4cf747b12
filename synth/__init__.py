"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only *generates inputs*: atom positions, atomic numbers, boxes,
network weights and initial velocities.  It holds none of the descriptor,
network or force arithmetic of the potential, so neither side of a parity
test can inherit a mistake from the other through it.

Workloads are shaped after the paper's bulk-water performance benchmark
(Results, "Performance Scaling of Different NNP Architectures", and
Tables S3/S4): full-NNP cubic water boxes at 1 g/cm^3.  Units: Angstrom,
amu, eV.

Recipes
-------
water_box(n):      n rigid waters (O-H 0.9572 A, HOH 104.52 deg) whose centres
                   sit on a k^3 lattice (k = ceil(n^(1/3)); n of the k^3 sites
                   drawn at random when n is not a cube), spacing L/k with
                   L = (n * 29.915 A^3)^(1/3); each centre jittered U(+-0.3 A)
                   per axis, re-drawn while an O-O distance (minimum image)
                   is below 2.5 A; orientations are uniform random rotations.
water_batch(B):    B boxes of round(exp(U(ln 16, ln 2048))) waters each.
hcno_box():        random covalent-like H/C/N/O trees (20-60 atoms, bond
                   lengths U(1.0, 1.5) A, element probabilities
                   H .45 / C .35 / N .10 / O .10) up to 2,000 atoms in a 40 A
                   box, then waters on the 1 g/cm^3 lattice filling the rest.
                   With elements=ANI2X_Z, probs=ANI2X_P: the seven elements
                   of the ANI-2x model (H .40 / C .30 / N .08 / O .08 / F .05
                   / S .05 / Cl .04), same trees.
xavier_weights():  per-species MLP weights, Xavier-uniform (gain 1), biases 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Physical constants of the synthetic water model (inputs, not method maths).
WATER_VOLUME_A3 = 29.915          # A^3 per molecule at 1 g/cm^3
OH_BOND_A = 0.9572
HOH_ANGLE_DEG = 104.52
MASS_AMU = {1: 1.008, 6: 12.011, 7: 14.007, 8: 15.999, 9: 18.998, 16: 32.06, 17: 35.45}

# Seeds per workload: geometry 1000 + k, weights 2000 + k.
GEOM_SEED = {1: 1001, 2: 1002, 3: 1003, 4: 1004, 5: 1005, 6: 1006}
WEIGHT_SEED = {1: 2001, 2: 2002, 3: 2003, 4: 2004, 5: 2005, 6: 2006}

HIDDEN = (160, 128, 96)


@dataclass
class System:
    """One periodic (or isolated) system: positions (n,3) f64, Z (n,) i32,
    box (3,) f64 edge lengths of an orthorhombic cell, or None if isolated."""
    pos: np.ndarray
    Z: np.ndarray
    box: np.ndarray | None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotation matrices from uniform unit quaternions."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _water_template() -> np.ndarray:
    """Rigid water in its own frame: O at the origin, H's in the xy plane."""
    half = math.radians(HOH_ANGLE_DEG) / 2.0
    return np.array([
        [0.0, 0.0, 0.0],
        [OH_BOND_A * math.sin(half), OH_BOND_A * math.cos(half), 0.0],
        [-OH_BOND_A * math.sin(half), OH_BOND_A * math.cos(half), 0.0],
    ])


def _min_image(d: np.ndarray, L: float) -> np.ndarray:
    return d - L * np.round(d / L)


def water_box(n_waters: int, seed: int, jitter: float = 0.3,
              min_oo: float = 2.5) -> System:
    """n rigid waters in a cubic box at 1 g/cm^3 (atom order O, H, H)."""
    if n_waters < 1:
        raise ValueError("n_waters must be >= 1")
    rng = np.random.default_rng(seed)
    L = (n_waters * WATER_VOLUME_A3) ** (1.0 / 3.0)
    k = int(math.ceil(n_waters ** (1.0 / 3.0) - 1e-9))
    a = L / k
    grid = np.stack(np.meshgrid(np.arange(k), np.arange(k), np.arange(k),
                                indexing="ij"), -1).reshape(-1, 3)
    if grid.shape[0] > n_waters:
        grid = grid[np.sort(rng.choice(grid.shape[0], n_waters, replace=False))]
    base = (grid + 0.5) * a
    centres = base + rng.uniform(-jitter, jitter, size=base.shape)
    # Re-draw the jitter of molecules that come closer than min_oo to an
    # earlier one (minimum image); lattice spacing >= 3.1 A so this ends fast.
    for _ in range(100):
        bad = _close_pairs(centres, L, min_oo)
        if not bad.size:
            break
        centres[bad] = base[bad] + rng.uniform(-jitter, jitter, size=(bad.size, 3))
    R = _random_rotations(rng, n_waters)
    mol = np.einsum("nij,aj->nai", R, _water_template()) + centres[:, None, :]
    pos = np.mod(mol.reshape(-1, 3), L)
    Z = np.tile(np.array([8, 1, 1], dtype=np.int32), n_waters)
    return System(pos=pos, Z=Z, box=np.array([L, L, L]),
                  meta={"kind": "water", "n_waters": n_waters, "seed": seed,
                        "L": L})


def _close_pairs(x: np.ndarray, L: float, rmin: float) -> np.ndarray:
    """Indices j of points that lie closer than rmin to some i < j (min image)."""
    from scipy.spatial import cKDTree
    tree = cKDTree(np.mod(x, L), boxsize=L)
    pairs = tree.query_pairs(rmin, output_type="ndarray")
    if pairs.size == 0:
        return np.zeros(0, dtype=np.int64)
    return np.unique(pairs.max(axis=1)).astype(np.int64)


def water_batch(n_systems: int, seed: int, lo: int = 16, hi: int = 2048
                ) -> list[System]:
    """Independent water boxes with log-uniform sizes in [lo, hi] waters."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi),
                                       size=n_systems))).astype(int)
    sub = rng.integers(0, 2**31 - 1, size=n_systems)
    return [water_box(int(s), int(sd)) for s, sd in zip(sizes, sub)]


HCNO_Z = np.array([1, 6, 7, 8], dtype=np.int32)
HCNO_P = np.array([0.45, 0.35, 0.10, 0.10])
ANI2X_Z = np.array([1, 6, 7, 8, 9, 16, 17], dtype=np.int32)
ANI2X_P = np.array([0.40, 0.30, 0.08, 0.08, 0.05, 0.05, 0.04])


def hcno_box(seed: int, L: float = 40.0, n_cluster_atoms: int = 2000,
             cluster_size: tuple[int, int] = (20, 60), max_waters: int = 3000,
             min_bonded: float = 0.95, min_between: float = 2.0,
             water_excl: float = 2.5, elements=HCNO_Z, probs=HCNO_P) -> System:
    """H/C/N/O clusters grown as random trees, solvated by lattice waters.

    Bonds: length U(1.0, 1.5) A along a uniform random direction from a
    random existing atom of the same cluster; a new atom is rejected if it
    comes closer than `min_bonded` to any atom of its cluster or closer than
    `min_between` to another cluster's atom (minimum image).  Waters sit on
    the 1 g/cm^3 lattice; a site is dropped if its O lies within
    `water_excl` A of a cluster atom.  Everything is an NNP atom.
    """
    rng = np.random.default_rng(seed)
    pos: list[np.ndarray] = []
    Z: list[int] = []
    cid: list[int] = []
    grid_n = max(1, int(L // 3.0))
    cellsz = L / grid_n
    grid: dict[tuple, list[int]] = {}

    def cell_of(p):
        c = np.floor(np.mod(p, L) / cellsz).astype(int) % grid_n
        return (int(c[0]), int(c[1]), int(c[2]))

    def ok(p, c_id):
        c = cell_of(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    key = ((c[0] + dx) % grid_n, (c[1] + dy) % grid_n,
                           (c[2] + dz) % grid_n)
                    for j in grid.get(key, ()):
                        d = _min_image(pos[j] - p, L)
                        r = math.sqrt(d @ d)
                        lim = min_bonded if cid[j] == c_id else min_between
                        if r < lim:
                            return False
        return True

    def add(p, z, c_id):
        pos.append(np.mod(p, L))
        Z.append(int(z))
        cid.append(c_id)
        grid.setdefault(cell_of(p), []).append(len(pos) - 1)

    c_id = 0
    while len(pos) < n_cluster_atoms:
        size = int(rng.integers(cluster_size[0], cluster_size[1] + 1))
        size = min(size, n_cluster_atoms - len(pos))
        for _ in range(1000):
            seedp = rng.uniform(0, L, size=3)
            if ok(seedp, c_id):
                break
        else:
            raise RuntimeError("could not place a cluster seed")
        members = [len(pos)]
        add(seedp, rng.choice(elements, p=probs), c_id)
        tries = 0
        while len(members) < size and tries < 20000:
            tries += 1
            parent = pos[members[int(rng.integers(len(members)))]]
            v = rng.normal(size=3)
            v /= np.linalg.norm(v)
            p = parent + v * rng.uniform(1.0, 1.5)
            if ok(p, c_id):
                members.append(len(pos))
                add(p, rng.choice(elements, p=probs), c_id)
        c_id += 1
    n_clu = len(pos)
    cl = np.array(pos)
    # waters on the 1 g/cm^3 lattice, skipping sites near cluster atoms
    k = int(round(L / (WATER_VOLUME_A3 ** (1.0 / 3.0))))
    a = L / k
    tmpl = _water_template()
    wat = []
    sites = np.stack(np.meshgrid(np.arange(k), np.arange(k), np.arange(k),
                                 indexing="ij"), -1).reshape(-1, 3)
    rng.shuffle(sites)
    for s in sites:
        if len(wat) >= max_waters:
            break
        c = (s + 0.5) * a + rng.uniform(-0.3, 0.3, size=3)
        d = _min_image(cl - c, L)
        if np.min(np.einsum("ij,ij->i", d, d)) < water_excl ** 2:
            continue
        R = _random_rotations(rng, 1)[0]
        wat.append(tmpl @ R.T + c)
    n_w = len(wat)
    allpos = np.concatenate([cl] + [w for w in wat]) if wat else cl
    allZ = np.concatenate([np.array(Z, dtype=np.int32),
                           np.tile(np.array([8, 1, 1], dtype=np.int32), n_w)])
    return System(pos=np.mod(allpos, L), Z=allZ.astype(np.int32),
                  box=np.array([L, L, L]),
                  meta={"kind": "hcno", "seed": seed, "L": L,
                        "n_cluster_atoms": n_clu, "n_waters": n_w,
                        "n_clusters": c_id})


def xavier_weights(n_species: int, d_in: int, seed: int,
                   hidden: tuple[int, ...] = HIDDEN,
                   final_scale: float = 1.0) -> list[list[tuple[np.ndarray, np.ndarray]]]:
    """Per-species MLP weights [(W1, b1), ..., (W4, b4)], W_l of shape
    (fan_in, fan_out) row-major, Xavier-uniform U(+-sqrt(6/(in+out))),
    biases zero.  Species s draws from its own spawned stream of `seed`.
    `final_scale` multiplies the output layer (documented per workload)."""
    widths = (d_in,) + tuple(hidden) + (1,)
    streams = np.random.SeedSequence(seed).spawn(n_species)
    out = []
    for s in range(n_species):
        rng = np.random.default_rng(streams[s])
        layers = []
        for li in range(len(widths) - 1):
            fi, fo = widths[li], widths[li + 1]
            lim = math.sqrt(6.0 / (fi + fo))
            W = rng.uniform(-lim, lim, size=(fi, fo))
            if li == len(widths) - 2:
                W = W * final_scale
            layers.append((W, np.zeros(fo)))
        out.append(layers)
    return out


def random_biases(weights, seed: int, scale: float = 0.1):
    """Copy of `weights` with U(+-scale) biases (tests exercise bias paths)."""
    rng = np.random.default_rng(seed)
    return [[(W.copy(), rng.uniform(-scale, scale, size=b.shape)) for W, b in sp]
            for sp in weights]


def maxwell_boltzmann(Z: np.ndarray, temperature_K: float, seed: int
                      ) -> np.ndarray:
    """Velocities (A/fs) drawn at `temperature_K` with zero net momentum."""
    kB_eV = 8.617333262e-5
    # 1 eV/amu = 9.64853e-3 A^2/fs^2
    m = np.array([MASS_AMU[int(z)] for z in Z])
    rng = np.random.default_rng(seed)
    sigma = np.sqrt(kB_eV * temperature_K / m * 9.64853321e-3)
    v = rng.normal(size=(Z.shape[0], 3)) * sigma[:, None]
    v -= (m[:, None] * v).sum(0) / m.sum()
    return v


def masses(Z: np.ndarray) -> np.ndarray:
    return np.array([MASS_AMU[int(z)] for z in Z])


def aev_length(n_species: int, n_rad: int = 16, n_ang: int = 32) -> int:
    """Length of the descriptor: per-species radial blocks plus one angular
    block per unordered species pair."""
    return n_rad * n_species + n_ang * n_species * (n_species + 1) // 2


def workload(k: int) -> dict:
    """The six named synthetic workloads (1..6) with their seeds."""
    if k == 1:
        s = water_box(64, GEOM_SEED[1])
        return dict(name="water-64 (192 atoms, 12.42 A)", systems=[s],
                    atomic_numbers=(1, 8), weight_seed=WEIGHT_SEED[1])
    if k == 2:
        s = water_box(4096, GEOM_SEED[2])
        return dict(name="water-4096 (12,288 atoms, 49.7 A)", systems=[s],
                    atomic_numbers=(1, 8), weight_seed=WEIGHT_SEED[2])
    if k == 3:
        s = water_box(32768, GEOM_SEED[3])
        return dict(name="water-32768 (98,304 atoms, 99.4 A)", systems=[s],
                    atomic_numbers=(1, 8), weight_seed=WEIGHT_SEED[3])
    if k == 4:
        b = water_batch(256, GEOM_SEED[4])
        return dict(name="batch-256 water boxes (16-2,048 waters)", systems=b,
                    atomic_numbers=(1, 8), weight_seed=WEIGHT_SEED[4])
    if k == 5:
        s = hcno_box(GEOM_SEED[5])
        return dict(name="HCNO-40A (2,000 cluster atoms + waters)", systems=[s],
                    atomic_numbers=(1, 6, 7, 8), weight_seed=WEIGHT_SEED[5])
    if k == 6:
        s = hcno_box(GEOM_SEED[6], elements=ANI2X_Z, probs=ANI2X_P)
        return dict(name="HCNOFSCl-40A (2,000 cluster atoms of 7 elements + waters)", systems=[s],
                    atomic_numbers=tuple(int(z) for z in ANI2X_Z), weight_seed=WEIGHT_SEED[6])
    raise ValueError(k)
