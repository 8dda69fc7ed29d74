"""Pins of the oracle's inclusion pattern generator (Sec. 3.4).

The rotation of each inclusion is checked against scipy's quaternion
rotation (an independent library routine), and the bounding-box generator
against a brute-force scan of every site with the scipy-based inside test.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_1409_8340_gb300 import inputs as I

P, OP = 0, 1


def scipy_q(G, inc, sites):
    """Inside value q for an array of (i, j, k) sites, via scipy rotations."""
    r = sites * np.array([G.hx, G.hy, G.hz])
    d = r - inc[:3]
    for ax in range(3):
        if G.bc[ax] == P:
            L = (G.nx, G.ny, G.nz)[ax] * (G.hx, G.hy, G.hz)[ax]
            d[:, ax] -= L * np.floor(d[:, ax] / L + 0.5)
    w, x, y, z = inc[6:10]
    rot = Rotation.from_quat([x, y, z, w])          # scipy: scalar last
    e = rot.inv().apply(d)                           # body-frame coordinates R^T d
    return np.sum((e / inc[3:6]) ** 2, axis=1)


def all_sites(G):
    k, j, i = np.meshgrid(np.arange(G.nz), np.arange(G.ny), np.arange(G.nx), indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)


@pytest.mark.parametrize("bc", [(P, P, P), (OP, P, P)])
def test_inside_value_matches_scipy_rotation(O, bc):
    G = O.Grid(20, 18, 16, bc=bc)
    incs = I.ellipsoids(12, (G.length(0), G.length(1), G.length(2)), 1.5, 5.0, seed=7)
    sites = all_sites(G)[::37]
    for inc in incs:
        ref = scipy_q(G, inc, sites.astype(float))
        got = np.array([O.inside_q(G, inc, *s) for s in sites])
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("bc,kind,frac", [((P, P, P), "spheres", 0.0), ((OP, P, P), "ellipsoids", 0.08),
                                           ((OP, OP, OP), "ellipsoids", 0.05)])
def test_generator_matches_brute_force_scan(O, bc, kind, frac):
    G = O.Grid(24, 20, 16, bc=bc)
    box = (G.length(0), G.length(1), G.length(2))
    if kind == "spheres":
        incs = I.spheres(10, box, 2.0, 2.0, seed=1)
    else:
        incs = I.ellipsoids(400, box, 1.5, 5.0, seed=3)
    target = I.target_sites(frac, G.N)
    alpha, used, marked = O.pattern(G, incs, target, -1.0, 1.0)
    sites = all_sites(G).astype(float)
    mark = np.zeros(G.N, dtype=bool)
    counts = []
    for n, inc in enumerate(incs):
        if target > 0 and mark.sum() >= target:
            break
        mark |= scipy_q(G, inc, sites) <= 1.0
        counts.append(mark.sum())
    assert used == len(counts)
    assert marked == mark.sum()
    np.testing.assert_array_equal(alpha.ravel(), np.where(mark, -1.0, 1.0))
    if target > 0:
        assert marked >= target and (used == 1 or counts[-2] < target)


def test_periodic_wrap_and_open_clip(O):
    inc = np.array([[0.0, 0.0, 0.0, 1.6, 1.6, 1.6, 1.0, 0.0, 0.0, 0.0]])
    Gp = O.Grid(16, 16, 16, bc=(P, P, P))
    ap, _, mp = O.pattern(Gp, inc)
    Go = O.Grid(16, 16, 16, bc=(OP, OP, OP))
    ao, _, mo = O.pattern(Go, inc)
    # the periodic sphere is split over the 8 corners; the open one keeps one octant
    assert ap[-1, -1, -1] == -1.0 and ap[0, 0, 0] == -1.0
    assert ao[-1, -1, -1] == 1.0 and ao[0, 0, 0] == -1.0
    # lattice points of a sphere of radius 1.6 xi on a 0.5 xi grid
    pts = np.arange(-4, 5) * 0.5
    X, Y, Z = np.meshgrid(pts, pts, pts, indexing="ij")
    full = int(np.sum(X ** 2 + Y ** 2 + Z ** 2 <= 1.6 ** 2))
    octant = int(np.sum((X ** 2 + Y ** 2 + Z ** 2 <= 1.6 ** 2) & (X >= 0) & (Y >= 0) & (Z >= 0)))
    assert mp == full and mo == octant
