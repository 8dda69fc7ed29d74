"""Full-size workloads, in the launch configuration the benchmark times.

512x512x256 mesoscopic sample (67.1M sites): the inclusion map is bit-exact
with the oracle's; init + first sweep match the FP64 oracle at every site; a
convergence-tested step leaves a residual below the tolerance when the oracle
recomputes it; the multigrid potential matches the oracle's exact discrete
solution of the same right-hand side.  64x64x32 adjoint case: 400 steps with
checkpoints every 20, gradient checked along a random smooth direction against
central differences of the objective.
"""
import math

import numpy as np
import pytest

from _helpers import gpu_state, oracle_grid
from paper_1409_8340_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c3(O):
    import torch
    from paper_1409_8340_gb300 import presets
    from paper_1409_8340_gb300.solver import Solver, pattern
    w = presets.mesoscopic_512x512x256(0.025)
    p = w.params
    alpha, used, marked = pattern(p, w.candidates, w.target_sites, w.alpha_in, w.alpha_out)
    G = oracle_grid(O, p)
    alpha_o, used_o, marked_o = O.pattern(G, w.candidates, w.target_sites, w.alpha_in, w.alpha_out)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, w.seed).astype(np.complex64)
    s = Solver(p, alpha)
    s.set_state(torch.as_tensor(psi0))
    return {"p": p, "G": G, "alpha": alpha, "alpha_o": alpha_o, "counts": (used, marked, used_o, marked_o),
            "psi0": psi0, "s": s}


def test_c3_pattern_bit_exact(c3):
    used, marked, used_o, marked_o = c3["counts"]
    assert (used, marked) == (used_o, marked_o)
    assert marked >= 0.10 * c3["p"].N
    a = c3["alpha"].cpu().numpy()
    assert np.array_equal(a, c3["alpha_o"].astype(np.float32))


def test_c3_init_and_first_sweep_every_site(O, c3):
    import dataclasses

    import torch
    from paper_1409_8340_gb300.solver import Solver
    p = dataclasses.replace(c3["p"], fixed_sweeps=1)
    s = Solver(p, c3["alpha"])
    s.set_state(torch.as_tensor(c3["psi0"]))
    assert s.solve_psi() == 1
    b_g, D_g, _ = s.internals()
    psi1_g, _ = s.state()
    psi0 = c3["psi0"].astype(np.complex128)
    mu0 = np.zeros(p.shape)
    b_o, D_o = O.init(c3["G"], psi0, mu0, c3["alpha_o"], 0.0)
    assert np.max(np.abs(b_g.cpu().numpy() - b_o)) <= 3e-6
    assert np.max(np.abs(D_g.cpu().numpy() - D_o)) <= 3e-6
    del D_g
    psi1_o, _ = O.sweep(c3["G"], psi0, b_o, D_o, 0.0)
    assert np.max(np.abs(psi1_g.cpu().numpy() - psi1_o)) <= 3e-6
    s.close()


def test_c3_converged_step_residual_and_potential(O, c3):
    """One full step with the convergence test (eps = 1e-6), then: the oracle
    recomputes max|b - M psi|^2 of the GPU's psi from the GPU's b and diag M;
    the GPU potential after extra V-cycles matches the oracle's exact solve of the
    GPU's right-hand side."""
    s, p = c3["s"], c3["p"]
    s.step(1)
    b_g, D_g, _ = s.internals()
    psi_g, _ = gpu_state(s)
    r = O.residual(c3["G"], psi_g, b_g.cpu().numpy().astype(np.complex128), D_g.cpu().numpy().astype(np.complex128), 0.0)
    assert np.max(np.abs(r) ** 2) < p.eps
    obs = s.observables()
    assert 1 <= obs["last_sweeps"] <= 60
    assert math.isfinite(obs["Ex"])
    # the step ran p.poisson_cycles V-cycles from mu = 0; more solves of the same right-hand
    # side (10 V-cycles in all, each solve warm-started from the last) take the multigrid to
    # its FP32 floor
    for _ in range(-(-(10 - p.poisson_cycles) // p.poisson_cycles)):
        s.solve_mu()
    _, mu_g = gpu_state(s)
    f = s.internals()[2].cpu().numpy().astype(np.float64)
    mu_o = O.poisson_solve(c3["G"], f)
    err = np.max(np.abs(mu_g - mu_o)) / max(1.0, np.max(np.abs(mu_o)))
    assert err <= 1e-4, err


def test_c5_adjoint_directional_derivative():
    """400 steps, checkpoints every 20: <dJ/dalpha, v> against the central
    difference of J along a smooth random direction v.  The adjoint is the
    derivative of the step with exact linear solves, so the forward runs here
    solve tightly (psi: max|r|^2 < 1e-10; mu: relative residual 1e-6)."""
    import torch
    from paper_1409_8340_gb300 import presets
    from paper_1409_8340_gb300.solver import Solver
    w = presets.adjoint_64x64x32()
    p = w.params
    p.eps = 1e-10
    p.poisson_tol = 1e-6
    p.poisson_max_cycles = 40
    alpha = torch.as_tensor(w.alpha_field).cuda()
    psi0 = torch.as_tensor(I.random_psi(p.nx, p.ny, p.nz, w.seed).astype(np.complex64))
    s = Solver(p, alpha)
    s.set_state(psi0)
    J, grad, st = s.adjoint(400, checkpoint_every=20, adj_eps=1e-10, poisson_tol=1e-6)
    assert st["adjoint_sweeps"] > 0
    v = torch.as_tensor(I.smoothed_field(p.nx, p.ny, p.nz, seed=55, sigma_sites=4.0).astype(np.float32)).cuda()
    dJ = float((grad.double() * v.double()).sum())

    def J_of(a):
        t = Solver(p, a)
        t.set_state(psi0)
        ex = []
        for _ in range(400):
            t.step(1)
            ex.append(t.observables()["Ex"])
        t.close()
        return float(np.mean(ex[200:]))

    assert abs(J - J_of(alpha)) <= 1e-6 * abs(J) + 1e-9
    fds = []
    for delta in (0.01, 0.005):
        fds.append((J_of(alpha + delta * v) - J_of(alpha - delta * v)) / (2 * delta))
    fd = fds[-1]
    assert abs(fd - dJ) <= 0.05 * abs(fd) + 1e-7, (fds, dJ)
