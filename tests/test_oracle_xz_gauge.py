"""The xz-plane field gauge of the oracle (Eq. B_xz, Eq. A_xz, Sec. 3.3.1 y-wrap).

Pins: every plaquette carries the flux of B = (Bx, 0, Bz) (xy: hx hy Bz, yz:
hy hz Bx, xz: 0), the y-wrap plaquettes included; with B along z the xz gauge
and the (already pinned) yz gauge are related by an explicit lattice gauge
transform, and the FP64 time steps in the two gauges agree on every gauge
invariant; the signed xy winding of a periodic box equals the flux quanta.
"""
import math

import numpy as np
import pytest

from paper_1409_8340_gb300 import inputs as I

P, OP = 0, 1


def plaquette_phase(theta, a, b, bc):
    """sum of link phases around the (a, b) plaquettes at every site (forward a, forward b),
    periodic wraps included; axes of theta arrays are (z, y, x) = (2, 1, 0) for a = 0, 1, 2."""
    arr = {0: 2, 1: 1, 2: 0}
    ta, tb = theta[a], theta[b]
    s = ta + np.roll(tb, -1, axis=arr[a]) - np.roll(ta, -1, axis=arr[b]) - tb
    # keep plaquettes whose four sites exist (open axes: drop the last layer)
    sl = [slice(None)] * 3
    for ax in (a, b):
        if bc[ax] == OP:
            sl[arr[ax]] = slice(0, -1)
    return s[tuple(sl)]


@pytest.mark.parametrize("bc", [(P, P, P), (OP, P, P), (P, P, OP), (OP, OP, OP)])
def test_every_plaquette_carries_the_flux(O, bc):
    G = O.Grid(10, 8, 6, bc=bc, hx=0.5, hy=0.5, hz=0.5)
    G.Bz = 0.37
    Bx = 0.21
    if bc[0] == P and bc[1] == P:
        G.Bz = 2 * math.pi * 3 / (G.length(0) * G.length(1))
    if bc[1] == P and bc[2] == P:
        Bx = 2 * math.pi * 1 / (G.length(1) * G.length(2))
    th = O.xz_link_phases(G, Bx)
    for (a, b), flux in (((0, 1), G.hx * G.hy * G.Bz), ((1, 2), G.hy * G.hz * Bx), ((0, 2), 0.0)):
        ph = plaquette_phase(th, a, b, bc)
        np.testing.assert_allclose(np.exp(1j * ph), np.exp(-1j * flux), rtol=0, atol=1e-11)


def test_xz_and_yz_gauges_give_the_same_physics(O):
    """B = (0, 0, Bz), open x and y: theta_yz = theta_xz + chi_m - chi_{m+a} with
    chi_{i,j} = Bz (i hx ybar_j - j hy Lx / 2); time steps from psi0 (xz) and
    exp(i chi) psi0 (yz) agree on |psi|, mu, E_x and the sweep counts."""
    G = O.Grid(9, 8, 5, bc=(OP, OP, P), hx=0.5, hy=0.5, hz=0.5, Bz=0.31, Jext=0.015, ht=0.1)
    th_xz = O.xz_link_phases(G, 0.0)
    th_yz = O.landau_link_phases(G)
    ii = np.arange(G.nx)[None, None, :]
    jj = np.arange(G.ny)[None, :, None]
    ybar = jj * G.hy - 0.5 * G.length(1)
    chi = np.broadcast_to(G.Bz * (ii * G.hx * ybar - jj * G.hy * G.length(0) / 2), G.shape).astype(np.float64)
    # the transform maps the link tables onto each other (links inside the box)
    for ax, arr in ((0, 2), (1, 1), (2, 0)):
        d = th_xz[ax] + chi - np.roll(chi, -1, axis=arr) - th_yz[ax]
        sl = [slice(None)] * 3
        if G.bc[ax] == OP:
            sl[arr] = slice(0, -1)
        np.testing.assert_allclose(np.exp(1j * d[tuple(sl)]), 1.0, rtol=0, atol=1e-11)
    psi0 = I.random_psi(G.nx, G.ny, G.nz, 3)
    alpha = np.where(I.uniform(4, "t.al", G.N).reshape(G.shape) < 0.1, -1.0, 1.0)
    a = O.State(psi0.copy(), np.zeros(G.shape))
    b = O.State(psi0 * np.exp(1j * chi), np.zeros(G.shape))
    for _ in range(8):
        sa = O.step(G, a, alpha, theta=th_xz, eps=1e-11)
        sb = O.step(G, b, alpha, theta=th_yz, eps=1e-11)
        assert sa.sweeps == sb.sweeps
        assert abs(sa.Ex - sb.Ex) < 1e-12
        np.testing.assert_allclose(np.abs(a.psi), np.abs(b.psi), rtol=0, atol=1e-12)
        np.testing.assert_allclose(a.mu, b.mu, rtol=0, atol=1e-12)


@pytest.mark.parametrize("nz_quanta,nx_quanta", [(3, 0), (-2, 1), (5, -2)])
def test_signed_winding_equals_flux_quanta_xz(O, nz_quanta, nx_quanta):
    G = O.Grid(14, 12, 6, bc=(P, P, P))
    G.Bz = 2 * math.pi * nz_quanta / (G.length(0) * G.length(1))
    Bx = 2 * math.pi * nx_quanta / (G.length(1) * G.length(2))
    th = O.xz_link_phases(G, Bx)
    for seed in (1, 2):
        psi = I.random_psi(G.nx, G.ny, G.nz, seed)
        for K in (0.0, 0.9):
            n, tot = O.winding(G, psi, K, th)
            assert tot == nz_quanta * G.nz
