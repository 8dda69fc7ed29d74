"""The full pattern generator (Sec. 3.4) on the GPU against the FP64 oracle.

Integer decisions taken in FP64 on both sides in the same operation order, so
the comparison is bit-exact: eps at every site, the insulating mask, the number
of shapes taken and of sites claimed.  Cases: every shape kind, rotated, across
periodic wraps and open faces, inverted (domain shaping), insulating, the
target rule; every lattice kind; alternating and random checkerboards; Voronoi
tessellations with the three metrics (few and many seeds, seeds outside the
box); a combined landscape; and a full-size 512x512x256 Voronoi checked at
sampled sites against the oracle's brute-force owner.
"""
import math

import numpy as np
import pytest

from paper_1409_8340_gb300 import inputs as I

pytestmark = pytest.mark.gpu

P, OP = 0, 1


def shape(kind, c, a, q=(1.0, 0.0, 0.0, 0.0), value=-1.0, flags=0):
    return np.array([kind, flags, *c, *a, *q, value], dtype=np.float64)


def rand_quat(rng):
    q = rng.normal(size=4)
    return tuple(q / np.linalg.norm(q))


def quat_axis_angle(axis, ang):
    axis = np.asarray(axis, dtype=np.float64) / np.linalg.norm(axis)
    return (math.cos(ang / 2), *(math.sin(ang / 2) * axis))


def run_both(O, p, shapes=None, lattices=(), background=None, target=0):
    from _helpers import oracle_grid
    from paper_1409_8340_gb300.solver import pattern_ex
    a_g, ins_g, used_g, marked_g = pattern_ex(p, shapes, lattices, background, target, insulating=True)
    a_o, ins_o, used_o, marked_o = O.pattern_ex(oracle_grid(O, p), shapes, lattices, background, target)
    assert (used_g, marked_g) == (used_o, marked_o)
    np.testing.assert_array_equal(a_g.cpu().numpy(), a_o.astype(np.float32))
    np.testing.assert_array_equal(ins_g.cpu().numpy(), ins_o)
    return a_o, ins_o


def params(nx, ny, nz, bc, h=(0.5, 0.5, 0.5)):
    from paper_1409_8340_gb300.solver import Params
    return Params(nx, ny, nz, bc=bc, hx=h[0], hy=h[1], hz=h[2])


@pytest.mark.parametrize("bc", [(P, P, P), (OP, P, OP), (OP, OP, OP)])
def test_every_shape_kind_rotated_and_wrapped(O, bc):
    p = params(45, 38, 27, bc, h=(0.5, 0.45, 0.6))
    rng = np.random.default_rng(7)
    box = np.array([p.length(0), p.length(1), p.length(2)])
    shapes = []
    for n in range(150):
        kind = n % 5
        c = rng.uniform(-0.1, 1.1, 3) * box                  # some centres outside: wrap or clip
        a = rng.uniform(0.6, 4.0, 3)
        flags = (O.INSULATING if n % 7 == 0 else 0)
        shapes.append(shape(kind, c, a, rand_quat(rng), value=-1.0 + 0.01 * n, flags=flags))
    run_both(O, p, shapes)
    a, ins = run_both(O, p, shapes, target=p.N // 6)
    assert ins.any()


def test_inverted_domain_and_columnar_defects(O):
    """a cylindrical integration domain (outside claimed first) holding columnar
    defects at +-45 degrees in a film stack (Sec. 3.4 and its figure)"""
    p = params(64, 60, 40, (P, P, OP))
    dom = shape(O.CYLINDER, (16.0, 15.0, 10.0), (14.0, 13.0, 50.0), value=0.0, flags=O.INVERT)
    rng = np.random.default_rng(9)
    cols = [dom]
    for n in range(40):
        ang = math.pi / 4 if n % 2 else -math.pi / 4
        c = (rng.uniform(0, 32), rng.uniform(0, 30), 10.0)
        cols.append(shape(O.CYLINDER, c, (1.1, 1.1, 20.0), quat_axis_angle((0, 1, 0), ang), value=-1.0,
                          flags=O.INSULATING if n % 3 == 0 else 0))
    run_both(O, p, cols)


@pytest.mark.parametrize("kind", ["SQUARE", "TRIANGULAR", "HONEYCOMB", "KAGOME", "RECTANGULAR", "HEXAGONAL"])
def test_lattices(O, kind):
    p = params(80, 70, 1, (P, P, P)) if kind in ("SQUARE", "TRIANGULAR", "HONEYCOMB", "KAGOME") \
        else params(48, 44, 36, (P, OP, P))
    motif = shape(O.ELLIPSOID, (0.05, 0.03, 0.0), (1.1, 0.9, 1.3), quat_axis_angle((0, 0, 1), 0.3), value=-0.7)
    lat = {"kind": getattr(O, kind), "count": (11, 12, 1 if p.nz == 1 else 4), "origin": (0.7, 0.4, 0.2),
           "spacing": (3.6, 2.9, 4.4), "motif": motif}
    a, _ = run_both(O, p, None, [lat], {"kind": O.BG_CONSTANT, "value": 0.9})
    assert (a == -0.7).any() and (a == 0.9).any()
    # the same lattice given as explicit shapes
    run_both(O, p, O.lattice_shapes(lat), (), {"kind": O.BG_CONSTANT, "value": 0.9})


@pytest.mark.parametrize("p_odd", [-1.0, 0.5, 0.15])
def test_checkerboards(O, p_odd):
    p = params(50, 44, 18, (P, OP, P))
    bg = {"kind": O.BG_CHECKER, "cell": (1.3, 2.1, 0.0 if p_odd < 0 else 1.7), "values": (0.5, 1.0),
          "p_odd": p_odd, "seed": (1 << 37) + 11}
    a, _ = run_both(O, p, None, (), bg)
    assert set(np.unique(a)) == {0.5, 1.0}


@pytest.mark.parametrize("metric", ["EUCLIDEAN", "ABSOLUTE", "MAXIMUM"])
@pytest.mark.parametrize("bc,dims,n_seeds", [((P, P, P), (40, 36, 28), 300), ((OP, P, OP), (41, 30, 25), 37),
                                             ((P, OP, P), (96, 88, 1), 900), ((OP, OP, OP), (20, 18, 9), 1),
                                             ((P, P, P), (33, 30, 22), 2)])
def test_voronoi(O, metric, bc, dims, n_seeds):
    p = params(*dims, bc)
    rng = np.random.default_rng(n_seeds)
    ext = np.array([p.length(0), p.length(1), max(p.length(2), 0.0)])
    seeds = np.zeros((n_seeds, 4))
    seeds[:, :3] = rng.uniform(-0.05, 1.05, (n_seeds, 3)) * ext     # a few outside the box
    seeds[:, 3] = rng.uniform(0.3, 1.0, n_seeds)
    bg = {"kind": O.BG_VORONOI, "metric": getattr(O, metric), "seeds": seeds}
    run_both(O, p, None, (), bg)


def test_voronoi_ties_go_to_the_lower_seed(O):
    """seeds on grid points at equal distances from many sites"""
    p = params(24, 24, 8, (P, P, P))
    seeds = np.array([[2.0, 2.0, 1.0, 0.1], [6.0, 2.0, 1.0, 0.2], [2.0, 6.0, 1.0, 0.3], [6.0, 6.0, 1.0, 0.4],
                      [4.0, 4.0, 3.0, 0.5], [10.0, 10.0, 2.0, 0.6]])
    for metric in (O.EUCLIDEAN, O.ABSOLUTE, O.MAXIMUM):
        run_both(O, p, None, (), {"kind": O.BG_VORONOI, "metric": metric, "seeds": seeds})


def test_combined_landscape(O):
    """domain mask, insulating spheres, a kagome lattice of cylinders and a polycrystalline
    (Voronoi) background with a different eps per grain"""
    p = params(72, 64, 20, (P, P, OP))
    rng = np.random.default_rng(12)
    dom = shape(O.ELLIPSOID, (18.0, 16.0, 5.0), (17.0, 15.0, 40.0), value=-1.0, flags=O.INVERT)
    sph = [shape(O.ELLIPSOID, rng.uniform(0, 1, 3) * (36, 32, 10), (1.5, 1.5, 1.5), value=-1.0,
                 flags=O.INSULATING) for _ in range(12)]
    lat = {"kind": O.KAGOME, "count": (7, 7, 1), "origin": (1.0, 1.0, 5.0), "spacing": (5.0, 0.0, 1.0),
           "motif": shape(O.CYLINDER, (0, 0, 0), (0.8, 0.8, 6.0), value=-0.5)}
    seeds = np.zeros((60, 4))
    seeds[:, :3] = rng.uniform(0, 1, (60, 3)) * (36, 32, 9.5)
    seeds[:, 3] = rng.uniform(0.4, 1.0, 60)
    run_both(O, p, [dom] + sph, [lat], {"kind": O.BG_VORONOI, "metric": O.EUCLIDEAN, "seeds": seeds})


def test_full_size_voronoi_sampled(O):
    """512x512x256 (open x, periodic y z) with 20 000 grains: every sampled site's eps
    is the value of the oracle's brute-force nearest seed"""
    from _helpers import oracle_grid
    from paper_1409_8340_gb300.solver import pattern_ex
    p = params(512, 512, 256, (OP, P, P))
    rng = np.random.default_rng(20)
    n = 20000
    seeds = np.zeros((n, 4))
    seeds[:, :3] = rng.uniform(0, 1, (n, 3)) * (p.length(0), p.length(1), p.length(2))
    seeds[:, 3] = np.arange(n) / n
    alpha, _, _, _ = pattern_ex(p, None, (), {"kind": 2, "metric": 0, "seeds": seeds})
    G = oracle_grid(O, p)
    a = alpha.cpu().numpy()
    idx = I.uniform(21, "t.sample", 3000)
    sites = (idx * p.N).astype(np.int64)
    for m in sites[:600]:
        i, j, k = m % p.nx, (m // p.nx) % p.ny, m // (p.nx * p.ny)
        own = O.voronoi_owner(G, seeds, O.EUCLIDEAN, int(i), int(j), int(k))
        assert a[k, j, i] == np.float32(seeds[own, 3]), (i, j, k)


def test_invalid_arguments_fail_before_device_work():
    import ctypes
    from paper_1409_8340_gb300 import _lib
    from paper_1409_8340_gb300._lib import TdglError
    from paper_1409_8340_gb300.solver import pattern_ex
    p = params(16, 16, 8, (P, P, P))
    bad = [
        [shape(7, (1, 1, 1), (1, 1, 1))],                                  # kind
        [shape(0, (1, 1, 1), (0.0, 1, 1))],                                # size
        [shape(0, (1, 1, 1), (1, 1, 1), q=(1.0, 0.1, 0.0, 0.0))],          # not a unit quaternion
        [shape(0, (1, 1, 1), (1, 1, 1), flags=8)],                         # flags
    ]
    for sh in bad:
        with pytest.raises(TdglError):
            pattern_ex(p, sh)
    with pytest.raises(TdglError):
        pattern_ex(p, None, (), {"kind": 2, "seeds": np.zeros((0, 4))})
    with pytest.raises(TdglError):
        pattern_ex(p, None, [{"kind": 9, "count": (1, 1, 1), "spacing": (1, 1, 1),
                              "motif": shape(0, (0, 0, 0), (1, 1, 1))}])
