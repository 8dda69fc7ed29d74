"""Closed-form pins of the FP64 oracle.

Each case has an exact answer that follows from the mathematics of the scheme,
not from the oracle's code:
  * a uniform state with a constant potential obeys a scalar Crank-Nicolson
    recurrence (pins alpha, beta, the u*mu term and the linearisation of Sec. 3.1);
  * the zero-field uniform state |psi|^2 = alpha/beta is an exact fixed point;
  * plane waves exp(i k x) are eigenvectors of the gauge Laplacian with
    eigenvalue -(4/h^2) sin^2((k+K) h/2), so psi, J_av and the K ODE follow a
    scalar recurrence (Sec. 2.2, Eq. K_ODE, J_av);
  * the Neumann cosine modes of an open axis are eigenvectors with
    eigenvalue -(4/h^2) sin^2(pi m / (2(N-1))) (Sec. 3.3.2);
  * the normal state (alpha = -1, psi = 0) under applied current is Ohmic:
    E_x = J exactly, in both current formulations.
"""
import math

import numpy as np
import pytest

from paper_1409_8340_gb300 import inputs as I

P, OP = 0, 1


def test_uniform_state_with_constant_potential(O):
    G = O.Grid(5, 4, 3, bc=(P, P, P), u=1.7, beta=1.3, ht=0.1)
    a0, phi, alpha, c = 0.6, 0.4, 0.9, 0.35
    psi = np.full(G.shape, a0 * np.exp(1j * phi))
    mu = np.full(G.shape, c)
    al = np.full(G.shape, alpha)
    sol, *_ = O.solve_psi(G, psi, mu, al, 0.0, fixed_sweeps=80)
    z = alpha - G.beta * a0 ** 2 - 1j * G.u * c
    expect = a0 * np.exp(1j * phi) * (1 + G.ht / 2 * z) / (1 - G.ht / 2 * z)
    np.testing.assert_allclose(sol, expect, rtol=0, atol=1e-15)


@pytest.mark.parametrize("bc", [(P, P, P), (OP, P, P), (OP, OP, OP)])
def test_zero_field_uniform_fixed_point(O, bc):
    G = O.Grid(8, 6, 4, bc=bc, beta=1.25)
    alpha = 0.8
    psi = np.full(G.shape, math.sqrt(alpha / G.beta) * np.exp(0.7j), dtype=complex)
    st = O.State(psi.copy(), np.zeros(G.shape))
    for _ in range(5):
        O.step(G, st, np.full(G.shape, alpha), fixed_sweeps=80)
    assert np.max(np.abs(st.psi - psi)) < 1e-14
    assert np.max(np.abs(st.mu)) < 1e-13


def test_relaxes_to_uniform_state_from_small_perturbation(O):
    G = O.Grid(8, 8, 8, bc=(P, P, P), beta=1.0)
    alpha = 0.7
    base = math.sqrt(alpha) * np.exp(0.3j)
    noise = I.random_psi(8, 8, 8, 3) - 0.5
    st = O.State(base * (1 + 0.01 * noise), np.zeros(G.shape))
    O.run(G, st, np.full(G.shape, alpha), 300, fixed_sweeps=60)
    assert np.max(np.abs(np.abs(st.psi) ** 2 - alpha)) < 1e-6


def plane_wave_recurrence(G, a0, kvec, K0, alpha, nsteps):
    """Scalar recurrence for psi = a exp(i k.r) on a field-free periodic box."""
    hs = (G.hx, G.hy, G.hz)
    cs = (1 / G.hx ** 2, 1 / G.hy ** 2, 1 / (G.g ** 2 * G.hz ** 2))
    a, K = a0, K0
    out = []
    for _ in range(nsteps):
        kk = (kvec[0] + K, kvec[1], kvec[2])
        lam = sum(4 * cs[d] * math.sin(kk[d] * hs[d] / 2) ** 2 for d in range(3))
        c = alpha - lam - G.beta * a * a
        a = a * (1 + G.ht / 2 * c) / (1 - G.ht / 2 * c)
        jav = a * a * math.sin((kvec[0] + K) * G.hx) / G.hx
        Kn = K + G.u * G.ht * (G.Jext - jav)
        Ex = (Kn - K) / (G.u * G.ht)
        Kn = Kn - (2 * math.pi / G.hx) * math.floor(Kn * G.hx / (2 * math.pi))
        out.append((a, jav, Ex, Kn))
        K = Kn
    return out


@pytest.mark.parametrize("mvec,Jext", [((1, 0, 0), 0.02), ((2, 1, 0), -0.01), ((0, 0, 1), 0.0), ((1, 1, 2), 0.05)])
def test_plane_wave_and_K_ode(O, mvec, Jext):
    G = O.Grid(16, 8, 6, hx=0.5, hy=0.45, hz=0.6, bc=(P, P, P), g=1.4, u=1.3, beta=0.9, ht=0.1, Jext=Jext)
    kvec = tuple(2 * math.pi * m / G.length(d) for d, m in enumerate(mvec))
    z, y, x = np.meshgrid(np.arange(G.nz) * G.hz, np.arange(G.ny) * G.hy, np.arange(G.nx) * G.hx, indexing="ij")
    phase = np.exp(1j * (kvec[0] * x + kvec[1] * y + kvec[2] * z))
    a0, alpha, K0 = 0.55, 0.9, 0.13
    st = O.State(a0 * phase, np.zeros(G.shape), K=K0)
    ref = plane_wave_recurrence(G, a0, kvec, K0, alpha, 20)
    for n in range(20):
        s = O.step(G, st, np.full(G.shape, alpha), fixed_sweeps=80)
        a, jav, Ex, Kn = ref[n]
        np.testing.assert_allclose(st.psi, a * phase, rtol=0, atol=1e-13)
        assert abs(s.Jav - jav) < 1e-13
        assert abs(s.Ex - Ex) < 1e-11
        assert abs(st.K - Kn) < 1e-11
        assert np.max(np.abs(st.mu)) < 1e-12


@pytest.mark.parametrize("m", [1, 3])
def test_neumann_cosine_mode(O, m):
    G = O.Grid(11, 4, 3, hx=0.5, bc=(OP, P, P), beta=0.0, ht=0.1)
    i = np.arange(G.nx)
    mode = np.cos(math.pi * m * i / (G.nx - 1))
    psi = np.broadcast_to(0.3 * mode, G.shape).astype(complex)
    alpha = 0.6
    lam = 4 / G.hx ** 2 * math.sin(math.pi * m / (2 * (G.nx - 1))) ** 2
    factor = (1 + G.ht / 2 * (alpha - lam)) / (1 - G.ht / 2 * (alpha - lam))
    st = O.State(psi.copy(), np.zeros(G.shape))
    for n in range(1, 6):
        O.step(G, st, np.full(G.shape, alpha), fixed_sweeps=120)
        np.testing.assert_allclose(st.psi, psi * factor ** n, rtol=0, atol=1e-14)


@pytest.mark.parametrize("bcx", [OP, P])
def test_normal_state_is_ohmic(O, bcx):
    J = 0.013
    G = O.Grid(12, 6, 4, bc=(bcx, P, P), Jext=J, Bz=0.0)
    st = O.State(np.zeros(G.shape, dtype=complex), np.zeros(G.shape))
    for n in range(4):
        s = O.step(G, st, np.full(G.shape, -1.0), eps=1e-12)
        assert abs(s.Ex - J) < 1e-12
    if bcx == OP:
        # mu is linear in x with slope -J: the normal current -d mu/dx equals J everywhere
        slope = np.diff(st.mu, axis=2) / G.hx
        np.testing.assert_allclose(slope, -J, rtol=0, atol=1e-12)
    else:
        assert abs(st.K - 4 * G.u * G.ht * J) < 1e-13
