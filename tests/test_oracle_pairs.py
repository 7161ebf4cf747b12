"""Pins of the oracle's neighbour enumeration (pairs under periodic images).

* simple cubic lattices: every atom has sum_{1<=k<(rc/a)^2} r_3(k) neighbours
  (r_3 from tests/golden/lattice_shells.txt), also in boxes shorter than the
  cutoff, where an atom meets its own periodic images;
* the cell-list enumeration returns exactly the brute-force pair set;
* pairs come in mirrored couples (i, j, d) <-> (j, i, -d);
* bulk counts match 4/3 pi rc^3 rho.
"""
import math
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lattice_shells.txt")


def r3_table():
    t = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        t[int(k)] = int(v)
    return t


def lattice(a, k):
    g = np.stack(np.meshgrid(*[np.arange(k)] * 3, indexing="ij"), -1).reshape(-1, 3)
    return (g + 0.5) * a, np.array([k * a] * 3)


@pytest.mark.parametrize("a,k,rc", [(2.0, 8, 5.2), (2.0, 8, 3.5), (2.0, 3, 5.2),
                                    (2.0, 2, 5.2), (1.7, 5, 5.2), (3.1, 1, 5.2)])
def test_simple_cubic_shell_counts(oracle_mod, a, k, rc):
    r3 = r3_table()
    kmax = (rc / a) ** 2
    assert kmax < max(r3) + 1
    expected = sum(v for kk, v in r3.items() if 1 <= kk < kmax)
    pos, box = lattice(a, k)
    for fn in (oracle_mod.pairs_brute, oracle_mod.pairs_cells):
        pi, pj, pd = fn(pos, box, rc)
        counts = np.bincount(pi, minlength=pos.shape[0])
        assert np.all(counts == expected), (fn.__name__, counts[:5], expected)


def _canon(p):
    pi, pj, pd = p
    key = np.round(pd, 9)
    order = np.lexsort((key[:, 2], key[:, 1], key[:, 0], pj, pi))
    return pi[order], pj[order], pd[order]


@pytest.mark.parametrize("n_waters,seed", [(8, 1), (27, 2), (64, 1001), (200, 3)])
def test_cells_equal_brute(oracle_mod, n_waters, seed):
    s = synth.water_box(n_waters, seed)
    for rc in (3.5, 5.2):
        a = _canon(oracle_mod.pairs_brute(s.pos, s.box, rc))
        b = _canon(oracle_mod.pairs_cells(s.pos, s.box, rc))
        assert len(a[0]) == len(b[0])
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert np.allclose(a[2], b[2], atol=1e-12)


def test_orthorhombic_and_unwrapped(oracle_mod):
    rng = np.random.default_rng(7)
    box = np.array([7.3, 11.9, 16.4])
    pos = rng.uniform(0, 1, size=(90, 3)) * box
    shifted = pos + rng.integers(-3, 4, size=pos.shape) * box  # unwrapped copies
    a = _canon(oracle_mod.pairs_brute(pos, box, 5.2))
    b = _canon(oracle_mod.pairs_cells(shifted, box, 5.2))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.allclose(a[2], b[2], atol=1e-9)


def test_mirrored_pairs(oracle_mod):
    s = synth.water_box(27, 5)
    pi, pj, pd = oracle_mod.pairs_cells(s.pos, s.box, 5.2)
    fwd = {(int(i), int(j), tuple(np.round(d, 9))) for i, j, d in zip(pi, pj, pd)}
    for i, j, d in zip(pi, pj, pd):
        assert (int(j), int(i), tuple(np.round(-d, 9))) in fwd


def test_isolated_pairs(oracle_mod):
    rng = np.random.default_rng(3)
    pos = rng.uniform(0, 8, size=(40, 3))
    pi, pj, pd = oracle_mod.pairs_cells(pos, None, 5.2)
    n = 0
    for i in range(40):
        for j in range(40):
            if i != j and np.linalg.norm(pos[j] - pos[i]) < 5.2:
                n += 1
    assert len(pi) == n
    assert np.allclose(pd, pos[pj] - pos[pi])


def test_bulk_density_count(oracle_mod):
    rng = np.random.default_rng(11)
    L = 30.0
    rho = 0.1003
    n = int(rho * L ** 3)
    pos = rng.uniform(0, L, size=(n, 3))
    pi, _, _ = oracle_mod.pairs_cells(pos, np.array([L, L, L]), 5.2)
    expect = (n - 1) / L ** 3 * 4.0 / 3.0 * math.pi * 5.2 ** 3
    assert abs(len(pi) / n - expect) / expect < 0.02
