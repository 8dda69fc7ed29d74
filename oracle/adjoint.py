"""FP64 adjoint of the implicit TDGL time loop (test infrastructure only).

Objective: J = mean of E_x over the steps window_start+1 .. T of a run of T
steps (open x, applied current injected through the x faces, K = 0).  The
paper has no adjoint; this module differentiates the discrete step the paper
defines (Sec. 3.1 and 3.2), with every linear solve taken as exact.

Writing H(psi, mu, alpha) = diag(beta|psi|^2 + i u mu - alpha) - Lap_U, the
Crank-Nicolson step of Sec. 3.1 is R = psi' - psi + (ht/2) H(psi,mu,alpha) (psi'
+ psi) = 0 and M = I + (ht/2) H.  With the real inner product <a,b> = Re sum
conj(a) b, one reverse step n (from psi^n, mu^n back to psi^{n-1}, mu^{n-1}) is
  w          = W * G(mubar^n / W)           (adjoint of the Poisson solve G,
                                            W the trapezoid weights)
  psibar^n  += i [NS^H(w psi^n) - w NS(psi^n)]      (adjoint of f = Im[psi* NS psi])
  M^H lam    = psibar^n                              (adjoint implicit solve)
  dJ/dalpha += (ht/2) Re[conj(lam) (psi^n + psi^{n-1})]
  mubar^{n-1} = (ht/2) u Im[conj(lam) (psi^n + psi^{n-1})] (+ v / |window|)
  psibar^{n-1} = lam - (ht/2) H^H lam - ht beta Re[conj(lam)(psi^n + psi^{n-1})] psi^{n-1}
with v the voltage weights (E_x = v . mu).
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def forward(G: O.Grid, psi0, mu0, alpha, nsteps, fixed_sweeps=60, eps=1e-6):
    """Run nsteps; return the trajectory of (psi, mu) and the E_x of each step."""
    st = O.State(np.asarray(psi0, dtype=np.complex128).copy(), np.asarray(mu0, dtype=np.float64).copy())
    traj = [(st.psi.copy(), st.mu.copy())]
    ex = []
    for _ in range(nsteps):
        s = O.step(G, st, alpha, fixed_sweeps=fixed_sweeps, eps=eps)
        traj.append((st.psi.copy(), st.mu.copy()))
        ex.append(s.Ex)
    return traj, ex


def objective(ex, window_start):
    return float(np.mean(ex[window_start:]))


def adjoint_gradient(G: O.Grid, traj, alpha, window_start, adj_sweeps=80):
    T = len(traj) - 1
    nwin = T - window_start
    v = O.voltage_weights(G)
    W = O.site_weights(G)
    S = sum((1.0 / G.hx ** 2, 1.0 / G.hy ** 2, (1.0 / (G.g ** 2 * G.hz ** 2)) if G.nz >= 2 else 0.0))
    ht2 = 0.5 * G.ht
    grad = np.zeros(G.shape)
    psibar = np.zeros(G.shape, dtype=np.complex128)
    mubar = np.zeros(G.shape)
    for n in range(T, 0, -1):
        psi_n, _ = traj[n]
        psi_p, mu_p = traj[n - 1]
        if n > window_start:
            mubar = mubar + v / nwin
        # mu^n = G(f(psi^n) + injection): adjoint Poisson, then the quadratic f
        w = W * O.poisson_solve(G, mubar / W)
        g = psibar + 1j * (O.ns_adj(G, w * psi_n) - w * O.ns(G, psi_n))
        # psi^n solves M psi^n = b with M, b from (psi^{n-1}, mu^{n-1}, alpha)
        _, D = O.init(G, psi_p, mu_p, alpha)
        Dc = np.conj(D)
        lam = g / Dc
        for _ in range(adj_sweeps):
            lam = (g + ht2 * O.ns_adj(G, lam)) / Dc
        s = psi_n + psi_p
        c = np.real(np.conj(lam) * s)
        grad += ht2 * c
        a2 = np.abs(psi_p) ** 2
        Hh_lam = (G.beta * a2 - 1j * G.u * mu_p - alpha + 2.0 * S) * lam - O.ns_adj(G, lam)
        mubar = ht2 * G.u * np.imag(np.conj(lam) * s)
        psibar = lam - ht2 * Hh_lam - G.ht * G.beta * c * psi_p
    return grad


def fd_gradient(G: O.Grid, psi0, mu0, alpha, nsteps, window_start, sites, delta=1e-4, fixed_sweeps=60):
    """Central finite differences of J at the given flat site indices."""
    out = []
    for m in sites:
        a_p = alpha.copy().ravel()
        a_m = alpha.copy().ravel()
        a_p[m] += delta
        a_m[m] -= delta
        _, ex_p = forward(G, psi0, mu0, a_p.reshape(G.shape), nsteps, fixed_sweeps)
        _, ex_m = forward(G, psi0, mu0, a_m.reshape(G.shape), nsteps, fixed_sweeps)
        out.append((objective(ex_p, window_start) - objective(ex_m, window_start)) / (2 * delta))
    return np.array(out)
