"""Host model of the index arithmetic of the tiles staged by asynchronous copies
(csrc/staged_tile.cuh): which grid pair every stage element holds, and the ring of plane
stages.  No GPU.

A tile is 64 x-sites (32 pairs) by 8 rows.  Each psi stage row holds the pairs x0/2 - 1 ..
x0/2 + 32 of grid row j0 - 1 + rr, with the periodic wraps applied (open faces clamp), and
a thread copies an element only where some site of the tile reads it.  The model checks,
for every boundary combination and ragged tiles, that every copy address lies inside the
array and that every site of the tile reads its x, y neighbours (and itself) from stage
elements holding exactly the pairs the sweep's boundary rules name; and that the ring
(plane p of a tile in stage p % NS, the lower neighbour carried in a register, plane
t + NS - 1 issued once every thread has finished plane t - 1, waits leaving NS - 3 newer
copy groups in flight) never refills a stage a thread may still read.
"""
import itertools

import pytest

KBX, KBY, KPX = 32, 8, 64


def woc(c, n, per):
    return c % n if per else min(max(c, 0), n - 1)


def plane_of(nz, zper, z):
    if z < 0:
        return z + nz if zper else (1 if nz >= 2 else 0)
    if z >= nz:
        return z - nz if zper else (nz - 2 if nz >= 2 else 0)
    return z


def check_tile(nx, ny, nz, xper, yper, zper, kz, bx, by, bz):
    rowq, plq = nx // 2, (nx // 2) * ny
    n4 = plq * nz
    x0, j0 = bx * KPX, by * KBY
    k0 = bz * kz
    k1 = min(k0 + kz, nz)
    npl = k1 - k0 + 2
    for t in range(npl):
        base = plq * plane_of(nz, zper, k0 - 1 + t)
        stage = {}
        for r in range(KBY):
            for tx in range(KBX):
                x, j = x0 + 2 * tx, j0 + r
                cq = woc(x0 // 2 + tx, rowq, xper)
                own = woc(j, ny, yper) * rowq + cq
                yh = (woc(j0 - 1, ny, yper) if r == 0 else woc(j0 + KBY, ny, yper)) * rowq + cq
                xh = woc(j, ny, yper) * rowq + woc(x0 // 2 - 1 if tx == 0 else x0 // 2 + KBX, rowq, xper)
                need = x <= nx and j <= ny
                for off, key, cond in ((own, (r + 1, tx + 1), need), (yh, (0, tx + 1), r == 0),
                                       (yh, (KBY + 1, tx + 1), r == KBY - 1), (xh, (r + 1, 0), tx == 0),
                                       (xh, (r + 1, KBX + 1), tx == KBX - 1)):
                    if cond:
                        assert 0 <= base + off < n4
                        assert key not in stage
                        stage[key] = base + off
        if t == 0 or t == npl - 1:
            continue
        k = k0 - 1 + t
        for r in range(KBY):
            for tx in range(KBX):
                x, j = x0 + 2 * tx, j0 + r
                if not (x < nx and j < ny):
                    continue
                xlo, xhi = x == 0, x + 2 >= nx
                ylo, yhi = j == 0, j == ny - 1
                jp = (0 if yper else j) if yhi else j + 1
                jm = (ny - 1 if yper else j) if ylo else j - 1
                at = lambda xq, jj: xq + rowq * jj + plq * k
                assert stage[(r + 1, tx + 1)] == at(x // 2, j)
                assert stage[(r + 2, tx + 1)] == at(x // 2, jp)
                assert stage[(r, tx + 1)] == at(x // 2, jm)
                if not xlo:
                    assert stage[(r + 1, tx)] == at((x - 2) // 2, j)
                elif xper:
                    assert stage[(r + 1, tx)] == at((nx - 2) // 2, j)
                if not xhi:
                    assert stage[(r + 1, tx + 2)] == at((x + 2) // 2, j)
                elif xper:
                    assert stage[(r + 1, tx + 2)] == at(0, j)


GRIDS = [(34, 22, 13), (16, 16, 8), (40, 18, 11), (132, 10, 7), (136, 12, 6), (96, 20, 5), (2, 1, 1), (2, 3, 2),
         (66, 9, 1), (4, 4, 4)]


@pytest.mark.parametrize("nx,ny,nz", GRIDS)
def test_stage_elements_hold_the_named_neighbours(nx, ny, nz):
    for xper, yper, zper in itertools.product((False, True), repeat=3):
        for kz in sorted({1, 3, nz}):
            gx, gy, gz = (nx + KPX - 1) // KPX, (ny + KBY - 1) // KBY, (nz + kz - 1) // kz
            for bx, by, bz in itertools.product(range(gx), range(gy), range(gz)):
                check_tile(nx, ny, nz, xper, yper, zper, kz, bx, by, bz)


@pytest.mark.parametrize("ns", [5, 8])
def test_ring_never_refills_a_stage_in_use(ns):
    for npl in range(3, 3 * ns + 4):
        stage_plane = {}
        issued = 0

        def issue(t):
            nonlocal issued
            if t < npl:
                stage_plane[t % ns] = t
            issued += 1   # one commit group per call, empty past the last plane

        for t in range(1, ns):
            issue(t)
        done_upto = 0   # every thread has finished planes below this one
        for t in range(1, npl - 1):
            # the wait leaves ns - 3 newer groups in flight: planes 1 .. t + 1 have landed
            landed = issued - (ns - 3)
            assert landed >= t + 1
            done_upto = t - 1   # after the barrier every thread finished plane t - 1
            # the refill takes the stage of plane t - 1 (kept in registers from now on)
            tgt = (t + ns - 1) % ns
            assert tgt not in (t % ns, (t + 1) % ns)
            if tgt in stage_plane:
                assert stage_plane[tgt] <= done_upto
            issue(t + ns - 1)
            # this step reads planes t (stage) and t + 1 (stage); both present
            assert stage_plane[t % ns] == t and stage_plane[(t + 1) % ns] == t + 1
