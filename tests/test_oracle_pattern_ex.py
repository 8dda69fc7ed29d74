"""The full pattern generator of the oracle (Sec. 3.4) against what geometry fixes.

Pins: axis-aligned cuboid site counts in closed form (including periodic wrap);
every shape kind against an independent evaluation (scipy Rotation for the body
frame, the distance to a line for rotated cylinders); set identities (a cross is
the union of two bars, eight octants rotated by the octahedral group tile a
sphere, an inverted shape claims the complement); lattice coordination shells
(square, triangular, honeycomb, kagome, rectangular, hexagonal); checkerboard
structure and the draw fraction of the random checkerboard; Voronoi owners
against scipy's cKDTree for the Euclidean, absolute and maximum distances
(periodic and open axes); the target rule and the insulating mask.
"""
import math

import numpy as np
import pytest

P, OP = 0, 1


def shape(kind, c, a, q=(1.0, 0.0, 0.0, 0.0), value=-1.0, flags=0):
    return np.array([kind, flags, *c, *a, *q, value], dtype=np.float64)


def quat_axis_angle(axis, ang):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    return (math.cos(ang / 2), *(math.sin(ang / 2) * axis))


def site_positions(G):
    k, j, i = np.meshgrid(np.arange(G.nz), np.arange(G.ny), np.arange(G.nx), indexing="ij")
    return i, j, k, np.stack([i * G.hx, j * G.hy, k * G.hz], axis=-1)


def min_image(G, d):
    d = d.copy()
    for ax in range(3):
        if G.bc[ax] == P:
            L = G.length(ax)
            d[..., ax] -= L * np.floor(d[..., ax] / L + 0.5)
    return d


def claimed(O, G, shapes):
    alpha, _, _, _ = O.pattern_ex(G, shapes, background={"kind": O.BG_CONSTANT, "value": 7.0})
    return alpha != 7.0


def count_in(lo, hi, h, n, periodic):
    """sites i h (i in 0..n-1, wrapped when periodic) inside [lo, hi]"""
    if not periodic:
        return sum(1 for i in range(n) if lo <= i * h <= hi)
    L = n * h
    return sum(1 for i in range(n) if any(lo <= i * h + s * L <= hi for s in (-1, 0, 1)))


@pytest.mark.parametrize("bc", [(P, P, P), (OP, OP, OP), (P, OP, P)])
def test_axis_aligned_cuboid_counts(O, bc):
    G = O.Grid(20, 14, 10, bc=bc, hx=0.5, hy=0.7, hz=0.4)
    for c, a in [((4.05, 3.1, 1.93), (2.1, 1.1, 1.55)), ((0.31, 0.2, 0.13), (1.27, 2.02, 0.91)),
                 ((9.6, 8.8, 3.7), (0.74, 0.5, 0.5))]:
        got = int(claimed(O, G, [shape(O.CUBOID, c, a)]).sum())
        want = 1
        for ax, (h, n) in enumerate(((G.hx, G.nx), (G.hy, G.ny), (G.hz, G.nz))):
            want *= count_in(c[ax] - a[ax], c[ax] + a[ax], h, n, bc[ax] == P)
        assert got == want, (c, a)


def test_every_kind_against_an_independent_evaluation(O):
    from scipy.spatial.transform import Rotation
    G = O.Grid(24, 20, 16, bc=(P, OP, P), hx=0.5, hy=0.5, hz=0.5)
    i, j, k, r = site_positions(G)
    rng = np.random.default_rng(11)
    for trial in range(10):
        c = rng.uniform(0, 1, 3) * np.array([G.length(0), G.length(1), G.length(2)])
        a = rng.uniform(0.8, 3.5, 3)
        qv = Rotation.random(random_state=trial + 3).as_quat()          # (x, y, z, w)
        q = (qv[3], qv[0], qv[1], qv[2])
        e = min_image(G, r - c) @ Rotation.from_quat(qv).as_matrix()     # body coordinates R^T d
        s = e / a
        ell = (s ** 2).sum(-1)
        box = np.all(np.abs(e) <= a, axis=-1)
        want = {
            O.ELLIPSOID: ell <= 1,
            O.CUBOID: box,
            O.CYLINDER: (s[..., 0] ** 2 + s[..., 1] ** 2 <= 1) & (np.abs(e[..., 2]) <= a[2]),
            O.CROSS: box | ((np.abs(e[..., 0]) <= a[1]) & (np.abs(e[..., 1]) <= a[0]) & (np.abs(e[..., 2]) <= a[2])),
            O.OCTANT: (ell <= 1) & np.all(e >= 0, axis=-1),
        }
        # margin to every decision surface, so rounding order cannot matter
        near = (np.abs(ell - 1) < 1e-9) | np.any(np.abs(np.abs(e) - a) < 1e-9, axis=-1) | np.any(
            np.abs(e) < 1e-9, axis=-1) | (np.abs(e[..., 0] ** 2 / a[0] ** 2 + e[..., 1] ** 2 / a[1] ** 2 - 1) < 1e-9)
        for kind, w in want.items():
            got = claimed(O, G, [shape(kind, c, a, q)])
            assert np.array_equal(got[~near], w[~near]), (trial, kind)
            assert w.sum() > 0 or kind == O.OCTANT


def test_rotated_cylinder_is_a_distance_to_a_line(O):
    """columnar defects at +-45 degrees (Sec. 3.4): sites within r of the axis line and
    within the half-length of the centre along it"""
    G = O.Grid(40, 24, 40, bc=(P, P, OP), hx=0.5, hy=0.5, hz=0.5)
    _, _, _, r = site_positions(G)
    for ang in (math.pi / 4, -math.pi / 4):
        c = np.array([10.13, 6.07, 9.71])
        rad, half = 1.7, 6.3
        q = quat_axis_angle((0, 1, 0), ang)                              # body z tilted in the xz plane
        axis = np.array([math.sin(ang), 0.0, math.cos(ang)])
        d = min_image(G, r - c)
        along = d @ axis
        perp = np.linalg.norm(np.cross(d, axis), axis=-1)
        want = (perp <= rad) & (np.abs(along) <= half)
        near = (np.abs(perp - rad) < 1e-9) | (np.abs(np.abs(along) - half) < 1e-9)
        got = claimed(O, G, [shape(O.CYLINDER, c, (rad, rad, half), q)])
        assert np.array_equal(got[~near], want[~near])
        # volume: pi r^2 (2 half) within the surface layer
        vol = got.sum() * G.hx * G.hy * G.hz
        assert abs(vol - math.pi * rad ** 2 * 2 * half) < 0.25 * math.pi * rad ** 2 * 2 * half


def test_set_identities(O):
    G = O.Grid(30, 26, 22, bc=(P, P, OP), hx=0.5, hy=0.5, hz=0.5)
    c = (7.1234, 6.377, 5.2221)
    q = quat_axis_angle((1, 2, 3), 0.7)
    cross = claimed(O, G, [shape(O.CROSS, c, (4.3, 1.2, 2.1), q)])
    bars = claimed(O, G, [shape(O.CUBOID, c, (4.3, 1.2, 2.1), q),
                          shape(O.CUBOID, c, (4.3, 1.2, 2.1), tuple(
                              np.array(_qmul(q, quat_axis_angle((0, 0, 1), math.pi / 2)))))])
    assert np.array_equal(cross, bars)
    # eight octants of a sphere under 90-degree rotations tile the sphere
    rots = [(1.0, 0.0, 0.0, 0.0), quat_axis_angle((0, 0, 1), math.pi / 2), quat_axis_angle((0, 0, 1), math.pi),
            quat_axis_angle((0, 0, 1), -math.pi / 2)]
    flip = quat_axis_angle((1, 0, 0), math.pi)
    octs = [shape(O.OCTANT, c, (3.3, 3.3, 3.3), r) for r in rots] + \
           [shape(O.OCTANT, c, (3.3, 3.3, 3.3), _qmul(r, flip)) for r in rots]
    assert np.array_equal(claimed(O, G, octs), claimed(O, G, [shape(O.ELLIPSOID, c, (3.3, 3.3, 3.3))]))
    # an inverted shape claims exactly the complement
    e = shape(O.ELLIPSOID, c, (5.0, 3.0, 2.5), q)
    inv = e.copy()
    inv[1] = O.INVERT
    assert np.array_equal(claimed(O, G, [inv]), ~claimed(O, G, [e]))


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return (w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
            w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2)


@pytest.mark.parametrize("kind,nb,shell", [
    ("SQUARE", 1, [(4, 1.0)]), ("TRIANGULAR", 1, [(6, 1.0)]), ("HONEYCOMB", 2, [(3, 1 / math.sqrt(3))]),
    ("KAGOME", 3, [(4, 0.5)]), ("RECTANGULAR", 1, [(2, 1.0), (2, 1.3), (2, 1.6)]),
    ("HEXAGONAL", 1, [(6, 1.0), (2, 1.6)])])
def test_lattice_coordination(O, kind, nb, shell):
    a = 2.0
    lat = {"kind": getattr(O, kind), "count": (7, 7, 5), "origin": (0.3, 0.2, 0.1), "spacing": (a, 1.3 * a, 1.6 * a)
           if kind != "HEXAGONAL" else (a, 0, 1.6 * a), "motif": shape(O.ELLIPSOID, (0, 0, 0), (0.5, 0.5, 0.5))}
    if kind in ("SQUARE", "TRIANGULAR", "HONEYCOMB", "KAGOME"):
        lat["spacing"] = (a, 0.0, 1.6 * a)
    pts = O.lattice_shapes(lat)[:, 2:5]
    assert pts.shape[0] == 7 * 7 * 5 * nb
    # a point deep inside the finite lattice: its nearest shells
    centre = pts.mean(axis=0)
    p0 = pts[np.argmin(np.linalg.norm(pts - centre, axis=1))]
    dist = np.sort(np.linalg.norm(pts - p0, axis=1))[1:]
    at = 0
    for count, rel in shell:
        assert np.allclose(dist[at:at + count], rel * a, rtol=1e-12), (kind, dist[:12])
        at += count
    if kind in ("SQUARE", "TRIANGULAR", "HONEYCOMB", "KAGOME"):
        # the next shell is further out than the last listed one (except the stacking c)
        assert dist[at] > shell[-1][1] * a * (1 + 1e-9)


def test_lattice_of_motifs_equals_the_explicit_shapes(O):
    G = O.Grid(32, 28, 1, bc=(P, P, P), hx=0.5, hy=0.5, hz=0.5)
    motif = shape(O.ELLIPSOID, (0.11, 0.07, 0.0), (1.2, 1.2, 1.0), value=-0.5)
    lat = {"kind": O.KAGOME, "count": (4, 4, 1), "origin": (0.2, 0.3, 0.0), "spacing": (4.0, 0.0, 1.0), "motif": motif}
    a1, _, used, _ = O.pattern_ex(G, None, [lat])
    a2, _, _, _ = O.pattern_ex(G, O.lattice_shapes(lat))
    assert used == 48 and np.array_equal(a1, a2)
    assert set(np.unique(a1)) == {-0.5, 1.0}


def test_checkerboards(O):
    G = O.Grid(24, 16, 8, bc=(P, P, P), hx=0.5, hy=0.5, hz=0.5)
    bg = {"kind": O.BG_CHECKER, "cell": (2.0, 2.0, 0.0), "values": (0.3, 0.9), "p_odd": -1.0}
    a, _, _, _ = O.pattern_ex(G, None, background=bg)
    # 4x4-site cells, constant inside, alternating across every cell face
    cells = a.reshape(G.nz, G.ny // 4, 4, G.nx // 4, 4)
    assert np.all(cells == cells[:, :, :1, :, :1])
    v = cells[:, :, 0, :, 0]
    assert np.all(v[:, 1:, :] != v[:, :-1, :]) and np.all(v[:, :, 1:] != v[:, :, :-1])
    assert np.all(v == v[:1])
    # random checkerboard (Sec. 3.4 figure: two values with equal probability)
    Gb = O.Grid(256, 256, 1, bc=(P, P, P), hx=0.5, hy=0.5, hz=0.5)
    bg = {"kind": O.BG_CHECKER, "cell": (1.0, 1.0, 0.0), "values": (0.5, 1.0), "p_odd": 0.5, "seed": 99}
    a, _, _, _ = O.pattern_ex(Gb, None, background=bg)
    v = a.reshape(128, 2, 128, 2)[:, 0, :, 0]
    assert np.all(a.reshape(128, 2, 128, 2) == v[:, None, :, None])
    frac = np.mean(v == 1.0)
    assert abs(frac - 0.5) < 5 * math.sqrt(0.25 / v.size)
    # neighbouring cells independent, seeds matter
    assert abs(np.corrcoef(v[:, 1:].ravel(), v[:, :-1].ravel())[0, 1]) < 5 / math.sqrt(v.size)
    b, _, _, _ = O.pattern_ex(Gb, None, background=dict(bg, seed=100))
    assert np.mean(a != b) > 0.3
    c, _, _, _ = O.pattern_ex(Gb, None, background=dict(bg, p_odd=0.2))
    assert abs(np.mean(c.reshape(128, 2, 128, 2)[:, 0, :, 0] == 1.0) - 0.2) < 5 * math.sqrt(0.16 / v.size)


@pytest.mark.parametrize("bc,nz", [((P, P, P), 12), ((OP, P, OP), 10), ((P, OP, P), 1)])
@pytest.mark.parametrize("metric,p", [("EUCLIDEAN", 2), ("ABSOLUTE", 1), ("MAXIMUM", np.inf)])
def test_voronoi_against_kdtree(O, bc, nz, metric, p):
    from scipy.spatial import cKDTree
    G = O.Grid(28, 22, nz, bc=bc, hx=0.5, hy=0.5, hz=0.5)
    ext = np.array([G.length(a) if G.length(a) > 0 else 0.0 for a in range(3)])
    rng = np.random.default_rng(5)
    n = 40
    seeds = np.zeros((n, 4))
    seeds[:, :3] = rng.uniform(0, 1, (n, 3)) * ext
    seeds[:, 3] = np.arange(n) + 0.25
    a, _, _, _ = O.pattern_ex(G, None, background={"kind": O.BG_VORONOI, "metric": getattr(O, metric),
                                                   "seeds": seeds})
    _, _, _, r = site_positions(G)
    box = np.array([G.length(ax) if bc[ax] == P else 1e6 for ax in range(3)])
    tree = cKDTree(np.mod(seeds[:, :3], box), boxsize=box)
    dd, idx = tree.query(r.reshape(-1, 3), k=2, p=p)
    clear = (dd[:, 1] - dd[:, 0]) > 1e-9                                   # no near-ties
    owner = (a.ravel() - 0.25).round().astype(int)
    assert clear.mean() > 0.99
    assert np.array_equal(owner[clear], idx[clear, 0])


def test_target_rule_and_insulating_mask(O):
    G = O.Grid(40, 30, 12, bc=(P, P, P), hx=0.5, hy=0.5, hz=0.5)
    rng = np.random.default_rng(3)
    shapes = []
    for n in range(60):
        c = rng.uniform(0, 1, 3) * np.array([20, 15, 6])
        shapes.append(shape(O.ELLIPSOID if n % 2 else O.CUBOID, c, rng.uniform(0.8, 2.0, 3), value=-1.0 - (n % 3),
                            flags=O.INSULATING if n % 5 == 0 else 0))
    full, ins, used, marked = O.pattern_ex(G, shapes)
    assert used == 60
    target = marked // 3
    a, ins_t, used_t, marked_t = O.pattern_ex(G, shapes, target=target)
    assert marked_t >= target
    b, _, _, marked_b = O.pattern_ex(G, shapes[:used_t - 1])
    assert marked_b < target
    c, ins_c, _, _ = O.pattern_ex(G, shapes[:used_t])
    assert np.array_equal(a, c) and np.array_equal(ins_t, ins_c)
    # the mask marks exactly the sites whose first claimant is insulating
    own = np.full(G.shape, -1)
    for n, sh in enumerate(shapes):
        got = claimed(O, G, [sh]) & (own < 0)
        own[got] = n
    want = np.zeros(G.shape, dtype=bool)
    for n in range(0, 60, 5):
        want |= own == n
    assert np.array_equal(ins.astype(bool), want)
