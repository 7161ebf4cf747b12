"""Pins of the oracle's descriptor (AEV).

Special geometries where every factor of a term takes a known value:
* fc(Rc/2) = 1/2, fc(Rc/3) = 3/4 (cos(pi/2) = 0, cos(pi/3) = 1/2);
* an angle with 0.95 cos(theta) = cos(theta_z) puts theta' exactly on sector
  z, where 2^(1-zeta) (1 + cos 0)^zeta = 2; neighbouring sectors then carry
  2^(1-zeta) (1 + cos(k pi / 8))^zeta;
* a distance equal to an angular shift makes its Gaussian exactly 1.
Plus the block layout (which entries are non-zero for which species) and
invariance under translation, rotation and permutation.
"""
import math

import numpy as np
import pytest

import synth

SHF_R = [0.9 + 0.26875 * m for m in range(16)]
SHF_A = [0.9, 1.55, 2.2, 2.85]
SHF_Z = [(2 * z + 1) * math.pi / 16 for z in range(8)]


def test_documented_constants(oracle_mod):
    p = oracle_mod.Params()
    assert np.allclose(p.shf_r, [0.9, 1.16875, 1.4375, 1.70625, 1.975, 2.24375, 2.5125,
                                 2.78125, 3.05, 3.31875, 3.5875, 3.85625, 4.125, 4.39375,
                                 4.6625, 4.93125])
    assert np.allclose(p.shf_a, SHF_A)
    assert np.allclose(p.shf_z, [0.19634954, 0.58904862, 0.9817477, 1.3744468, 1.7671459,
                                 2.1598449, 2.552544, 2.9452431])
    assert (p.rc_r, p.eta_r, p.rc_a, p.eta_a, p.zeta, p.celu_alpha) == (5.2, 16.0, 3.5, 8.0, 32.0, 0.1)
    assert p.aev_length == 128
    assert oracle_mod.Params(atomic_numbers=(1, 6, 7, 8)).aev_length == 384


def _model(oracle_mod, Zs=(1, 8)):
    p = oracle_mod.Params(atomic_numbers=Zs)
    w = synth.xavier_weights(p.n_species, p.aev_length, 1)
    return p, oracle_mod.Model(p, w)


def _aev_isolated(oracle_mod, m, pos, Z):
    sp = m.p.species_of(Z)
    pairs = oracle_mod.pairs_cells(pos, None, 5.2)
    return oracle_mod.aev(m, sp, pairs)


@pytest.mark.parametrize("r,fcval", [(2.6, 0.5), (5.2 / 3, 0.75)])
def test_radial_dimer_closed_form(oracle_mod, r, fcval):
    p, m = _model(oracle_mod)
    pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    G = _aev_isolated(oracle_mod, m, pos, [1, 8])     # H, O
    expect = np.array([0.25 * fcval * math.exp(-16.0 * (r - R) ** 2) for R in SHF_R])
    # H sees an O neighbour: block of neighbour species O (index 1)
    assert np.allclose(G[0, 16:32], expect, rtol=1e-13, atol=0)
    assert np.all(G[0, :16] == 0)
    # O sees an H neighbour: block of species H (index 0)
    assert np.allclose(G[1, :16], expect, rtol=1e-13, atol=0)
    assert np.all(G[1, 16:32] == 0)
    # one neighbour: no angular pair
    assert np.all(G[:, 32:] == 0)
    # the largest feature sits at the shift closest to r
    assert int(np.argmax(G[0, 16:32])) == int(np.argmin([abs(r - R) for R in SHF_R]))


def test_radial_cutoff_is_strict(oracle_mod):
    p, m = _model(oracle_mod)
    G = _aev_isolated(oracle_mod, m, np.array([[0, 0, 0], [5.2, 0, 0.0]]), [1, 1])
    assert np.all(G == 0)
    G = _aev_isolated(oracle_mod, m, np.array([[0, 0, 0], [5.2 - 1e-7, 0, 0.0]]), [1, 1])
    assert 0 < G.max() < 1e-15


def _triatomic(r1, r2, theta):
    return np.array([[0.0, 0.0, 0.0], [r1, 0.0, 0.0],
                     [r2 * math.cos(theta), r2 * math.sin(theta), 0.0]])


@pytest.mark.parametrize("zstar", [1, 2, 5, 6])  # theta' never reaches sectors 0 and 7
def test_angular_sector_closed_form(oracle_mod, zstar):
    """Centre O, two H at Rc_A/2 (fc = 1/2 each), angle placing theta' on
    sector zstar.  Then feature (a, zstar) = 2 * (1/2)^2 * exp(-8 (1.75 - R_a)^2)
    and sector z carries 2^-31 (1 + cos((zstar - z) pi/8))^32 instead of 2."""
    p, m = _model(oracle_mod)
    c = math.cos(SHF_Z[zstar]) / 0.95
    theta = math.acos(c)
    pos = _triatomic(1.75, 1.75, theta)
    G = _aev_isolated(oracle_mod, m, pos, [8, 1, 1])
    blk = G[0, 32:64].reshape(4, 8)  # block p(H,H) = 0
    for a in range(4):
        gauss = math.exp(-8.0 * (1.75 - SHF_A[a]) ** 2)
        for z in range(8):
            A = 2.0 if z == zstar else 2.0 ** -31 * (1 + math.cos((zstar - z) * math.pi / 8)) ** 32
            assert blk[a, z] == pytest.approx(A * 0.25 * gauss, rel=1e-11)
    assert np.all(G[0, 64:] == 0)       # p(H,O), p(O,O) blocks empty for this centre


def test_angular_gaussian_at_shift(oracle_mod):
    """r_ij + r_ik = 2 R_a makes the angular Gaussian exactly 1."""
    p, m = _model(oracle_mod)
    Ra = SHF_A[2]
    r1, r2 = 2.0, 2 * Ra - 2.0
    c = math.cos(SHF_Z[3]) / 0.95
    pos = _triatomic(r1, r2, math.acos(c))
    G = _aev_isolated(oracle_mod, m, pos, [8, 1, 1])
    f1 = 0.5 * math.cos(math.pi * r1 / 3.5) + 0.5
    f2 = 0.5 * math.cos(math.pi * r2 / 3.5) + 0.5
    assert G[0, 32 + 2 * 8 + 3] == pytest.approx(2.0 * f1 * f2, rel=1e-12)


def test_block_placement_four_species(oracle_mod):
    """Centre H (species 0) with a C (1) and an O (3) neighbour: only angular
    block p(1,3) = 6 and radial blocks 1 and 3 are non-zero."""
    p, m = _model(oracle_mod, (1, 6, 7, 8))
    assert [oracle_mod.pair_index(4, a, b) for a in range(4) for b in range(a, 4)] == list(range(10))
    pos = _triatomic(1.2, 1.4, 1.9)
    G = _aev_isolated(oracle_mod, m, pos, [1, 6, 8])
    g = G[0]
    nz = set(np.nonzero(g)[0].tolist())
    assert nz <= set(range(16, 32)) | set(range(48, 64)) | set(range(64 + 6 * 32, 64 + 7 * 32))
    assert g[16:32].max() > 0 and g[48:64].max() > 0 and g[64 + 192:64 + 224].max() > 0
    # the O centre sees H (0) and C (1): block p(0,1) = 1
    g = G[2]
    nz = set(np.nonzero(g)[0].tolist())
    assert nz <= set(range(0, 32)) | set(range(64 + 32, 64 + 64))


def test_aev_invariances(oracle_mod):
    p, m = _model(oracle_mod)
    s = synth.water_box(27, 9)
    sp = p.species_of(s.Z)
    G0 = oracle_mod.aev(m, sp, oracle_mod.pairs_cells(s.pos, s.box, 5.2))
    # translation (with wrap)
    t = np.array([3.3, -17.1, 0.4])
    G1 = oracle_mod.aev(m, sp, oracle_mod.pairs_cells(s.pos + t, s.box, 5.2))
    assert np.allclose(G0, G1, rtol=1e-10, atol=1e-12)
    # permutation
    perm = np.random.default_rng(0).permutation(s.n)
    G2 = oracle_mod.aev(m, sp[perm], oracle_mod.pairs_cells(s.pos[perm], s.box, 5.2))
    assert np.allclose(G0[perm], G2, rtol=1e-10, atol=1e-12)
    # rotation of an isolated cluster
    x = s.pos[:30]
    q = np.linalg.qr(np.random.default_rng(1).normal(size=(3, 3)))[0]
    Ga = oracle_mod.aev(m, sp[:30], oracle_mod.pairs_cells(x, None, 5.2))
    Gb = oracle_mod.aev(m, sp[:30], oracle_mod.pairs_cells(x @ q.T, None, 5.2))
    assert np.allclose(Ga, Gb, rtol=1e-10, atol=1e-12)
