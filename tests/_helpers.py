"""Shared helpers for the GPU parity tests (oracle <-> CUDA path on the same inputs)."""
import math

import numpy as np

from paper_1409_8340_gb300 import inputs as I

P, OP = 0, 1


def oracle_grid(O, p):
    return O.Grid(p.nx, p.ny, p.nz, hx=p.hx, hy=p.hy, hz=p.hz, bc=tuple(p.bc), g=p.g, u=p.u, beta=p.beta,
                  ht=p.ht, By=p.By, Bz=p.Bz, Jext=p.Jext)


def inclusion_alpha(p, seed, frac=0.08):
    """A cheap alpha map for stencil tests: iid sites flipped to -1 (not the pattern generator)."""
    u = I.uniform(seed, "test.alpha", p.N).reshape(p.shape)
    return np.where(u < frac, -1.0, 1.0).astype(np.float32)


def make_solver(p, alpha_np, psi0=None, mu0=None, K=0.0, link_phase=None):
    import torch
    from paper_1409_8340_gb300.solver import Solver
    alpha = torch.as_tensor(np.ascontiguousarray(alpha_np, dtype=np.float32)).cuda()
    lp = None if link_phase is None else torch.as_tensor(np.ascontiguousarray(link_phase, dtype=np.float32)).cuda()
    s = Solver(p, alpha, link_phase=lp)
    if psi0 is not None:
        s.set_state(torch.as_tensor(np.ascontiguousarray(psi0).astype(np.complex64)),
                    None if mu0 is None else torch.as_tensor(np.asarray(mu0, dtype=np.float32)), K)
    return s


def gpu_state(s):
    psi, mu = s.state()
    return psi.cpu().numpy().astype(np.complex128), mu.cpu().numpy().astype(np.float64)


def quantised(p, nz_quanta=0, ny_quanta=0):
    if p.bc[0] == P and p.bc[1] == P:
        p.Bz = 2 * math.pi * nz_quanta / (p.length(0) * p.length(1))
    if p.bc[0] == P and p.bc[2] == P and p.nz >= 2:
        p.By = 2 * math.pi * ny_quanta / (p.length(0) * p.length(2))
    return p
