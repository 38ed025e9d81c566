"""Composition of the seeded workloads: centre and AO counts as the
configurations state them, and no two centres closer than a stated floor
modulo the lattice (a centre that sits on a periodic image of another would
give a linearly dependent basis).  Pure numpy, no device."""
import itertools

import numpy as np
import pytest

from paper_2509_16460_gb300 import workloads as W


def min_separation(A, xyz, reach=2):
    """Smallest |x_i - x_j + T| over centre pairs and lattice translations T
    with |T_i| <= reach (T != 0 when i == j), by brute force."""
    A = np.asarray(A, float)
    T = np.array(list(itertools.product(range(-reach, reach + 1), repeat=3)), float) @ A
    best = np.inf
    n = len(xyz)
    for i in range(n):
        for j in range(i, n):
            d = np.linalg.norm(xyz[i] - xyz[j] + T, axis=1)
            if i == j:
                d = d[np.any(T != 0.0, axis=1)]
            best = min(best, float(d.min()))
    return best


def counts(w):
    return len(w.xyz), w.nao


def test_cfg1_composition():
    w = W.cfg1()
    assert counts(w) == (2, 18)
    assert min_separation(w.A, w.xyz) == pytest.approx(1.4)


def test_cfg2_composition():
    w = W.cfg2()
    assert counts(w) == (8, 240)
    # diamond: nearest neighbours at a sqrt(3)/4
    assert min_separation(w.A, w.xyz) == pytest.approx(6.74 * np.sqrt(3.0) / 4.0)
    assert w.Dk.shape == (1, 64, 240, 240)


def test_cfg3_composition():
    w = W.cfg3()
    # 24 C-like (30 AOs) + 24 H-like (14 AOs)
    assert counts(w) == (48, 24 * 30 + 24 * 14)
    assert w.nao == 1056
    assert w.Dk.shape == (2, 8, 1056, 1056)
    # inside a ring: C-C 2.64, C-H 2.05; between rings no contact below 1.5 bohr
    sep = min_separation(w.A, w.xyz)
    assert sep >= 1.5
    c = w.xyz[:6]
    h = w.xyz[24:30]
    assert np.linalg.norm(c[0] - c[1]) == pytest.approx(2.64)
    assert np.linalg.norm(c[0] - h[0]) == pytest.approx(2.05)


def test_cfg5_slab_composition():
    """4 rock-salt (001) layers of 8 sites (16 Mg-like + 16 O-like) and a CO
    molecule: 34 centres, 16 x 25 + 16 x 30 + 2 x 30 = 940 AOs, no centre on a
    periodic image of another."""
    w = W.cfg5()
    kinds = w.meta["kinds"]
    assert counts(w) == (34, 940)
    assert kinds.count("Mg") == 16
    assert kinds[:32].count("O") == 16
    assert kinds[32:] == ["C", "O"]
    slab = w.xyz[:32]
    # nearest neighbours inside the slab at the rock-salt spacing
    assert min_separation(w.A, slab) == pytest.approx(3.98, abs=1e-9)
    # every layer: 4 Mg + 4 O, alternating with their neighbours
    zs = np.round(slab[:, 2], 6)
    for z in np.unique(zs):
        layer = [k for k, zz in zip(kinds[:32], zs) if zz == z]
        assert layer.count("Mg") == 4 and layer.count("O") == 4
    # C 4.3 bohr above a top-layer cation, C-O 2.13 bohr
    top = zs.max()
    cation = [x for x, k, zz in zip(slab, kinds, zs) if k == "Mg" and zz == top]
    assert any(np.allclose(w.xyz[32] - x, [0.0, 0.0, 4.3]) for x in cation)
    assert np.linalg.norm(w.xyz[33] - w.xyz[32]) == pytest.approx(2.13)
    assert min_separation(w.A, w.xyz) >= 2.13 - 1e-9


def test_cfg4_cells_composition():
    """64 triclinic cells: 2-24 centres, minimum separation 1.5 bohr modulo the
    lattice, edges in 6-16 bohr, angles in 60-120 degrees, AO counts from the
    Z templates (H 14, C 30, O 30, Mg 25), k-meshes from 1^3 to 3^3."""
    per_z = {1: 14, 6: 30, 8: 30, 12: 25}
    cells = W.cfg4()
    assert len(cells) == 64
    for w in cells:
        n = w.meta["ncentre"]
        assert 2 <= n <= 24 and len(w.xyz) == n
        assert w.nao == sum(per_z[z] for z in w.meta["z"])
        assert min_separation(w.A, w.xyz) >= 1.5
        edges = np.linalg.norm(w.A, axis=1)
        assert np.all(edges >= 6.0) and np.all(edges <= 16.0)
        for i, j in ((1, 2), (0, 2), (0, 1)):
            ang = np.degrees(np.arccos(w.A[i] @ w.A[j] / (edges[i] * edges[j])))
            assert 60.0 - 1e-9 <= ang <= 120.0 + 1e-9
        assert all(1 <= k <= 3 for k in w.kmesh)
        assert 0.3 <= w.omega <= 0.5


def test_min_image_distance_helper():
    """The generator's minimum-image distance against the brute force above,
    on a skewed cell where rounding fractional differences alone is wrong."""
    A = np.array([[6.0, 0.0, 0.0], [5.0, 3.0, 0.0], [0.0, 0.0, 7.0]])
    rng = np.random.default_rng(0)
    for _ in range(20):
        f1, f2 = rng.uniform(0, 1, 3), rng.uniform(0, 1, 3)
        T = np.array(list(itertools.product(range(-3, 4), repeat=3)), float) @ A
        want = np.linalg.norm(f1 @ A - f2 @ A + T, axis=1).min()
        got = W.min_image_distance(A, f1, f2)
        assert got == pytest.approx(want)
