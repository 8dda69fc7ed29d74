"""Invariant pins of the FP64 oracle.

  * Lattice gauge invariance: psi -> exp(i chi) psi with
    U_{a,m} -> exp(i chi_m) U_{a,m} exp(-i chi_{m+a}) leaves |psi|, the link
    currents, mu, F, E_x and the sweep counts unchanged (Sec. 3.1, link variables).
  * Topology: the signed winding of all xy plaquettes of a periodic box equals
    the number of flux quanta n_z = Bz Lx Ly / 2 pi for ANY psi (Sec. 3.3.1,
    flux quantisation).
  * Gradient flow: at mu = K = 0 the linearised Crank-Nicolson step decreases
    the discrete free energy strictly when h_t beta max|psi|^2 < 1.
  * Charge conservation: after the Poisson solve the total link current
    J_s - grad mu is divergence free at every site, including the current
    injected through open faces (Eq. Poisson, Eq. J).
"""
import math

import numpy as np
import pytest

from paper_1409_8340_gb300 import inputs as I

P, OP = 0, 1


def gauge_transform(G, theta, chi):
    """theta'_{a,m} = theta_{a,m} + chi_m - chi_{m+a} (forward links, periodic wrap)."""
    out = theta.copy()
    for ax, arr_ax in ((0, 2), (1, 1), (2, 0)):
        out[ax] = theta[ax] + chi - np.roll(chi, -1, axis=arr_ax)
    return out


@pytest.mark.parametrize("bc", [(P, P, P), (OP, P, P), (OP, OP, P)])
def test_gauge_invariance_over_20_steps(O, bc):
    G = O.Grid(10, 8, 6, bc=bc, ht=0.1, By=0.0, Jext=0.01)
    G.Bz = 2 * math.pi * 2 / (G.length(0) * G.length(1))
    if bc[0] == P and bc[2] == P:
        G.By = 2 * math.pi * 1 / (G.length(0) * G.length(2))
    theta = O.landau_link_phases(G)
    chi = I.gauge_angles(G.nx, G.ny, G.nz, 21)
    theta2 = gauge_transform(G, theta, chi)
    psi0 = I.random_psi(G.nx, G.ny, G.nz, 22)
    alpha = np.where(I.uniform(23, "t.al", G.N).reshape(G.shape) < 0.15, -1.0, 1.0)
    a = O.State(psi0.copy(), np.zeros(G.shape))
    b = O.State(psi0 * np.exp(1j * chi), np.zeros(G.shape))
    for _ in range(20):
        sa = O.step(G, a, alpha, theta=theta, eps=1e-10)
        sb = O.step(G, b, alpha, theta=theta2, eps=1e-10)
        assert sa.sweeps == sb.sweeps
        assert abs(sa.Ex - sb.Ex) < 1e-12
        np.testing.assert_allclose(np.abs(a.psi), np.abs(b.psi), rtol=0, atol=1e-12)
        np.testing.assert_allclose(b.psi, a.psi * np.exp(1j * chi), rtol=0, atol=1e-12)
        np.testing.assert_allclose(a.mu, b.mu, rtol=0, atol=1e-12)
    assert abs(O.energy(G, a.psi, alpha, a.K, theta) - O.energy(G, b.psi, alpha, b.K, theta2)) < 1e-10
    # the Landau-mode oracle and explicit Landau links are the same computation
    c = O.State(psi0.copy(), np.zeros(G.shape))
    for _ in range(3):
        O.step(G, c, alpha, eps=1e-10)
    d = O.State(psi0.copy(), np.zeros(G.shape))
    for _ in range(3):
        O.step(G, d, alpha, theta=theta, eps=1e-10)
    np.testing.assert_allclose(c.psi, d.psi, rtol=0, atol=1e-12)


@pytest.mark.parametrize("nz_quanta,ny_quanta", [(4, 0), (-3, 0), (7, 2), (1, -1)])
def test_signed_winding_equals_flux_quanta(O, nz_quanta, ny_quanta):
    G = O.Grid(16, 12, 6, hx=0.5, hy=0.5, hz=0.5, bc=(P, P, P))
    G.Bz = 2 * math.pi * nz_quanta / (G.length(0) * G.length(1))
    G.By = 2 * math.pi * ny_quanta / (G.length(0) * G.length(2))
    for seed in (1, 2):
        psi = I.random_psi(G.nx, G.ny, G.nz, seed)
        for K in (0.0, 1.7):
            n, tot = O.winding(G, psi, K)
            assert tot == nz_quanta * G.nz
            # every plaquette carries an integer of small magnitude
            assert np.abs(n).max() <= 2


@pytest.mark.parametrize("bc", [(P, P, P), (OP, P, P), (OP, OP, OP)])
def test_free_energy_decreases_at_zero_current(O, bc):
    G = O.Grid(12, 10, 6, bc=bc, ht=0.1, beta=1.0)
    if bc[0] == P and bc[1] == P:
        G.Bz = 2 * math.pi * 3 / (G.length(0) * G.length(1))
    else:
        G.Bz = 0.3
    alpha = np.where(I.uniform(31, "t.al", G.N).reshape(G.shape) < 0.1, -1.0, 1.0)
    st = O.State(I.random_psi(G.nx, G.ny, G.nz, 32), np.zeros(G.shape))
    F = [O.energy(G, st.psi, alpha)]
    for _ in range(40):
        assert G.ht * G.beta * np.max(np.abs(st.psi)) ** 2 < 1.0
        O.step(G, st, alpha, fixed_sweeps=60, freeze_mu_K=True)
        F.append(O.energy(G, st.psi, alpha))
    dF = np.diff(F)
    assert np.all(dF < 0), dF.max()


@pytest.mark.parametrize("bc", [(P, P, P), (OP, P, P), (OP, OP, OP)])
def test_total_current_is_divergence_free(O, bc):
    J = 0.02
    G = O.Grid(9, 7, 5, bc=bc, Jext=J, g=1.2)
    G.Bz = 0.4 if bc[0] == OP else 2 * math.pi * 2 / (G.length(0) * G.length(1))
    psi = I.random_psi(G.nx, G.ny, G.nz, 41)
    K = 0.4 if bc[0] == P else 0.0
    f = O.poisson_rhs(G, psi, K)
    mu = O.poisson_solve(G, f)
    theta = O.landau_link_phases(G)
    cs = (1 / G.hx ** 2, 1 / G.hy ** 2, 1 / (G.g ** 2 * G.hz ** 2))
    div = np.zeros(G.shape)
    for ax, aa in ((0, 2), (1, 1), (2, 0)):
        U = np.exp(1j * theta[ax])
        if ax == 0:
            U = U * np.exp(1j * G.hx * K)
        nxt = np.roll(psi, -1, axis=aa)
        mnx = np.roll(mu, -1, axis=aa)
        # total current on the link m -> m+a, times h_a (so that its difference over h_a^2 is a divergence)
        jl = cs[ax] * (np.imag(np.conj(psi) * U * nxt) - (mnx - mu))
        jin = np.roll(jl, 1, axis=aa)
        d = jl - jin
        if G.bc[ax] == OP:
            n = jl.shape[aa]
            sl = [slice(None)] * 3
            # open faces: the link beyond the face is the mirror image of the inner link,
            # plus the injected normal current on the x faces
            inj = 2 * J / G.hx if ax == 0 else 0.0
            sl[aa] = 0
            d[tuple(sl)] = 2 * jl[tuple(sl)] - inj
            sl2 = list(sl); sl2[aa] = n - 2
            sl[aa] = n - 1
            d[tuple(sl)] = -2 * jl[tuple(sl2)] + inj
        div += d
    assert np.max(np.abs(div)) < 1e-10
