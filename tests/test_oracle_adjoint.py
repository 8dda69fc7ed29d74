"""Pins of the FP64 adjoint (gradient of time-averaged E_x with respect to alpha).

  * central finite differences of the forward oracle at 32 seeded sites, with
    every solve converged (60 Jacobi sweeps, exact Poisson), on a 16x16x8 grid;
    a second case with open y and z exercises the transposed boundary rows;
  * the dot-product identity <a, NS b> = <NS^H a, b> for the transposed stencil.
"""
import numpy as np
import pytest

from paper_1409_8340_gb300 import inputs as I

P, OP = 0, 1


@pytest.mark.parametrize("bc", [(OP, P, P), (OP, OP, OP)])
def test_ns_adjoint_dot_product(O, bc):
    G = O.Grid(9, 7, 5, bc=bc, Bz=0.3, By=0.1, g=1.3)
    a = I.random_psi(9, 7, 5, 1) - 0.3
    b = I.random_psi(9, 7, 5, 2) - 0.4
    lhs = np.vdot(a, O.ns(G, b))
    rhs = np.vdot(O.ns_adj(G, a), b)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("bc,steps", [((OP, P, P), 30), ((OP, OP, OP), 20)])
def test_adjoint_matches_finite_differences(O, bc, steps):
    from oracle import adjoint as A
    G = O.Grid(16, 16, 8, bc=bc, Bz=0.1, Jext=0.01)
    alpha = I.smoothed_field(16, 16, 8, seed=5, sigma_sites=2.0)
    psi0 = I.random_psi(16, 16, 8, 7) * 0.5 + 0.5
    mu0 = np.zeros(G.shape)
    ws = steps // 2
    traj, ex = A.forward(G, psi0, mu0, alpha, steps)
    g = A.adjoint_gradient(G, traj, alpha, ws)
    sites = np.sort((I.uniform(11, "fd.sites", 32) * G.N).astype(int))
    fd = A.fd_gradient(G, psi0, mu0, alpha, steps, ws, sites)
    err = np.abs(g.ravel()[sites] - fd)
    assert err.max() <= 1e-6 * np.abs(fd).max(), (err.max(), np.abs(fd).max())
