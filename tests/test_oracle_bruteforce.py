"""Brute-force pins of the FP64 oracle on tiny grids.

The sparse matrix M, the vector b (Sec. 3.1, matrix M and Eq. b, with the
boundary rows of Sec. 3.3) and the scalar Laplacian (Sec. 3.2) are assembled
here as DENSE matrices, site row by site row, and solved with numpy.linalg.
The oracle's stencil code must agree with the dense assembly entry by entry,
its Jacobi iteration must converge to numpy's dense solution, and its Poisson
solve must match the dense least-squares solution.  Non-cubic grids catch axis
mix-ups; every boundary combination is covered.
"""
import itertools
import math

import numpy as np
import pytest

from paper_1409_8340_gb300 import inputs as I

P, OP = 0, 1


def dense_laplacian_U(G, K):
    """Dense gauge Laplacian Lap_U (Eq. LaplUV_yz with Sec. 3.3 boundary rows)."""
    nx, ny, nz = G.nx, G.ny, G.nz
    N = nx * ny * nz
    Lx = nx * G.hx if G.bc[0] == P else (nx - 1) * G.hx
    idx = lambda i, j, k: i + nx * (j + ny * k)

    def Ux(i, j, k):
        U = np.exp(1j * G.hx * K)
        if G.bc[0] == P and i == nx - 1:
            U *= np.conj(np.exp(1j * (-j * G.hy * Lx * G.Bz + k * G.hz * Lx * G.By)))
        return U

    Uy = lambda i: np.exp(-1j * G.hy * G.Bz * (i * G.hx - Lx / 2))
    Uz = lambda i: np.exp(1j * G.hz * G.By * (i * G.hx - Lx / 2))
    c = (1 / G.hx ** 2, 1 / G.hy ** 2, 1 / (G.g ** 2 * G.hz ** 2))
    L = np.zeros((N, N), dtype=complex)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                m = idx(i, j, k)
                pos = [i, j, k]
                for ax, n in enumerate((nx, ny, nz)):
                    if n < 2:
                        continue
                    L[m, m] -= 2 * c[ax]
                    pp = list(pos); pp[ax] = (pos[ax] + 1) % n
                    pm = list(pos); pm[ax] = (pos[ax] - 1) % n
                    if ax == 0:
                        uf, ub = Ux(i, j, k), np.conj(Ux(pm[0], j, k))
                    elif ax == 1:
                        uf, ub = Uy(i), np.conj(Uy(i))
                    else:
                        uf, ub = Uz(i), np.conj(Uz(i))
                    if G.bc[ax] == P:
                        L[m, idx(*pp)] += c[ax] * uf
                        L[m, idx(*pm)] += c[ax] * ub
                    elif pos[ax] == 0:
                        L[m, idx(*pp)] += 2 * c[ax] * uf
                    elif pos[ax] == n - 1:
                        L[m, idx(*pm)] += 2 * c[ax] * ub
                    else:
                        L[m, idx(*pp)] += c[ax] * uf
                        L[m, idx(*pm)] += c[ax] * ub
    return L


def dense_system(G, psi_prev, mu, alpha, K):
    L = dense_laplacian_U(G, K)
    p = psi_prev.ravel()
    a2 = np.abs(p) ** 2
    mu = mu.ravel(); al = alpha.ravel()
    ht2 = G.ht / 2
    M = np.eye(len(p), dtype=complex) + ht2 * (np.diag(G.beta * a2 + 1j * G.u * mu - al) - L)
    b = p + ht2 * ((al - 1j * G.u * mu) * p - G.beta * a2 * p + L @ p)
    return M, b


def dense_scalar_laplacian(G):
    nx, ny, nz = G.nx, G.ny, G.nz
    N = nx * ny * nz
    idx = lambda i, j, k: i + nx * (j + ny * k)
    c = (1 / G.hx ** 2, 1 / G.hy ** 2, 1 / (G.g ** 2 * G.hz ** 2))
    L = np.zeros((N, N))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                m = idx(i, j, k)
                pos = [i, j, k]
                for ax, n in enumerate((nx, ny, nz)):
                    if n < 2:
                        continue
                    pp = list(pos); pp[ax] = (pos[ax] + 1) % n
                    pm = list(pos); pm[ax] = (pos[ax] - 1) % n
                    if G.bc[ax] == OP and pos[ax] == 0:
                        pm = pp
                    if G.bc[ax] == OP and pos[ax] == n - 1:
                        pp = pm
                    L[m, idx(*pp)] += c[ax]
                    L[m, idx(*pm)] += c[ax]
                    L[m, m] -= 2 * c[ax]
    return L


BCS = [(P, P, P), (OP, P, P), (OP, OP, OP), (P, OP, P), (P, P, OP)]


def make_grid(O, bc, nx=6, ny=5, nz=4, By=0.3, Bz=0.7, g=1.3, K=0.0):
    G = O.Grid(nx, ny, nz, hx=0.5, hy=0.6, hz=0.45, bc=bc, g=g, u=1.7, beta=1.1, ht=0.1, By=By, Bz=Bz)
    if bc[0] == P and bc[1] == P:   # flux quantisation Bz Lx Ly = 2 pi n
        G.Bz = 2 * math.pi * 2 / (G.length(0) * G.length(1))
    if bc[0] == P and bc[2] == P:
        G.By = 2 * math.pi * 1 / (G.length(0) * G.length(2))
    return G


def random_state(G, seed):
    psi = I.random_psi(G.nx, G.ny, G.nz, seed)
    mu = (I.uniform(seed, "t.mu", G.N).reshape(G.shape) - 0.5) * 0.4
    alpha = np.where(I.uniform(seed, "t.al", G.N).reshape(G.shape) < 0.2, -1.0, 0.8)
    return psi, mu, alpha


@pytest.mark.parametrize("bc", BCS)
def test_init_matches_dense_assembly(O, bc):
    G = make_grid(O, bc)
    K = 0.37 if bc[0] == P else 0.0
    psi, mu, alpha = random_state(G, 11)
    M, b_dense = dense_system(G, psi, mu, alpha, K)
    b, D = O.init(G, psi, mu, alpha, K)
    np.testing.assert_allclose(b.ravel(), b_dense, rtol=0, atol=1e-13)
    np.testing.assert_allclose(D.ravel(), np.diag(M), rtol=0, atol=1e-13)


@pytest.mark.parametrize("bc", BCS)
def test_jacobi_sweep_matches_dense(O, bc):
    G = make_grid(O, bc)
    K = -0.21 if bc[0] == P else 0.0
    psi, mu, alpha = random_state(G, 12)
    it = I.random_psi(G.nx, G.ny, G.nz, 99)
    M, bd = dense_system(G, psi, mu, alpha, K)
    b, D = O.init(G, psi, mu, alpha, K)
    nxt, r2 = O.sweep(G, it, b, D, K)
    Dd = np.diag(np.diag(M))
    R = M - Dd
    expect = (bd - R @ it.ravel()) / np.diag(M)
    np.testing.assert_allclose(nxt.ravel(), expect, rtol=0, atol=1e-13)
    r = bd - M @ it.ravel()
    assert abs(r2 - np.max(np.abs(r) ** 2)) < 1e-12


@pytest.mark.parametrize("bc", BCS)
def test_jacobi_converges_to_dense_solution(O, bc):
    G = make_grid(O, bc)
    K = 0.5 if bc[0] == P else 0.0
    psi, mu, alpha = random_state(G, 13)
    M, bd = dense_system(G, psi, mu, alpha, K)
    exact = np.linalg.solve(M, bd)
    sol, nsw, r2, hist = O.solve_psi(G, psi, mu, alpha, K, eps=1e-28, max_iter=500)
    assert np.max(np.abs(M @ sol.ravel() - bd)) < 1e-12
    np.testing.assert_allclose(sol.ravel(), exact, rtol=0, atol=1e-12)
    # residual history: Jacobi on a diagonally dominant M contracts
    assert hist[-1] < hist[0] * 1e-20


@pytest.mark.parametrize("bc", BCS)
def test_poisson_matches_dense_least_squares(O, bc):
    G = make_grid(O, bc)
    L = dense_scalar_laplacian(G)
    rng_f = I.uniform(5, "t.F", G.N) - 0.5
    w = O.site_weights(G).ravel()
    F = rng_f - (w @ rng_f) / w.sum()          # compatible right-hand side
    mu = O.poisson_solve(G, F.reshape(G.shape)).ravel()
    assert abs(w @ mu) < 1e-12 * max(1.0, np.abs(mu).max())
    np.testing.assert_allclose(L @ mu, F, rtol=0, atol=1e-11)
    ls = np.linalg.lstsq(L, F, rcond=None)[0]
    ls -= (w @ ls) / w.sum()
    np.testing.assert_allclose(mu, ls, rtol=0, atol=1e-10)
    # the oracle's own Laplacian agrees with the dense one
    np.testing.assert_allclose(O.laplacian_mu(G, mu.reshape(G.shape)).ravel(), L @ mu, atol=1e-11)


@pytest.mark.parametrize("bc", BCS)
def test_poisson_rhs_is_divergence_of_link_currents(O, bc):
    """f_m equals the lattice divergence of the supercurrent on links (Eq. Poisson):
    (J_{m->m+a} - J_{m-a->m})/h_a with J = Im[psi* U psi']/h_a (z with 1/g^2),
    where at an open face the outer link is the mirror image of the inner one."""
    G = make_grid(O, bc)
    K = 0.3 if bc[0] == P else 0.0
    psi, _, _ = random_state(G, 14)
    Ld = dense_laplacian_U(G, K)
    p = psi.ravel()
    f_dense = np.imag(np.conj(p) * ((Ld @ p) - np.diag(Ld) * p))
    f = O.poisson_rhs(G, psi, K)
    np.testing.assert_allclose(f.ravel(), f_dense, rtol=0, atol=1e-12)
    # telescoping: the weighted sum of a divergence vanishes
    w = O.site_weights(G).ravel()
    assert abs(w @ f.ravel()) < 1e-11
