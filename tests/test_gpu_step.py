"""GPU parity of the implicit psi step against the FP64 oracle (element by element).

Grids span several 32x8 tiles with ragged tails, every boundary combination,
a film (Nz = 1), anisotropy g != 1 and both field components.  Tolerance:
per-step max |psi_GPU - psi_oracle| <= 2e-5 (FP32 arithmetic against FP64).
"""
import dataclasses
import math

import numpy as np
import pytest

from _helpers import OP, P, gpu_state, inclusion_alpha, make_solver, oracle_grid, quantised
from paper_1409_8340_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_PSI = 2e-5


def cases():
    from paper_1409_8340_gb300.solver import Params
    out = []
    out.append(("periodic_40x20x12", quantised(Params(40, 20, 12, bc=(P, P, P)), 3, 1)))
    out.append(("openx_45x19x10_J", Params(45, 19, 10, bc=(OP, P, P), Bz=0.23, By=0.07, Jext=0.01, g=1.3)))
    out.append(("film_36x17x1", Params(36, 17, 1, bc=(OP, P, P), Bz=0.3, Jext=0.02)))
    out.append(("allopen_33x9x7", Params(33, 9, 7, bc=(OP, OP, OP), Bz=0.4, By=0.1)))
    out.append(("periodicx_openyz_64x24x16", Params(64, 24, 16, bc=(P, OP, OP), Bz=0.15, Jext=0.01)))
    out.append(("cube32_4quanta", quantised(Params(32, 32, 32, bc=(P, P, P), eps=1e-8), 4)))
    return out


CASES = cases()


def fresh(p):
    """Each test works on its own copy of the case parameters."""
    return dataclasses.replace(p)


@pytest.mark.parametrize("name,p", CASES, ids=[c[0] for c in CASES])
def test_init_and_first_sweep(O, name, p):
    p = fresh(p)
    p.fixed_sweeps = 1
    G = oracle_grid(O, p)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 7)
    mu0 = (I.uniform(8, "t.mu", p.N).reshape(p.shape) - 0.5) * 0.2
    alpha = inclusion_alpha(p, 9)
    K = 0.3 if p.bc[0] == P else 0.0
    s = make_solver(p, alpha, psi0, mu0, K)
    n = s.solve_psi()
    assert n == 1
    b_g, D_g, _ = s.internals()
    psi1, _ = gpu_state(s)
    b_o, D_o = O.init(G, psi0.astype(np.complex64).astype(np.complex128), mu0.astype(np.float32), alpha, K)
    np.testing.assert_allclose(b_g.cpu().numpy(), b_o, rtol=0, atol=3e-6)
    np.testing.assert_allclose(D_g.cpu().numpy(), D_o, rtol=0, atol=3e-6)
    psi1_o, _ = O.sweep(G, psi0.astype(np.complex64).astype(np.complex128), b_o, D_o, K)
    np.testing.assert_allclose(psi1, psi1_o, rtol=0, atol=3e-6)


@pytest.mark.parametrize("name,p", CASES, ids=[c[0] for c in CASES])
def test_fixed_sweeps_trajectory(O, name, p):
    """10 full steps (psi, K, mu) with exactly 40 sweeps per step on both sides."""
    p = fresh(p)
    p.fixed_sweeps = 40
    p.poisson_tol = 1e-5
    p.poisson_max_cycles = 60
    G = oracle_grid(O, p)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 17).astype(np.complex64).astype(np.complex128)
    alpha = inclusion_alpha(p, 19)
    s = make_solver(p, alpha, psi0)
    st = O.State(psi0.copy(), np.zeros(p.shape))
    for n in range(10):
        s.step(1)
        O.step(G, st, alpha.astype(np.float64), fixed_sweeps=40)
        psi_g, mu_g = gpu_state(s)
        err = np.max(np.abs(psi_g - st.psi))
        assert err <= TOL_PSI, (n, err)
        scale = max(1.0, np.max(np.abs(st.mu)))
        assert np.max(np.abs(mu_g - st.mu)) <= 2e-5 * scale, (n, np.max(np.abs(mu_g - st.mu)))
    obs = s.observables()
    assert abs(obs["K"] - st.K) < 1e-5


@pytest.mark.parametrize("name,p", CASES[:3] + CASES[5:], ids=[c[0] for c in CASES[:3] + CASES[5:]])
def test_tolerance_mode_per_step(O, name, p):
    """Convergence-tested steps: from the same input state, the oracle and the GPU
    take the same number of sweeps and produce the same psi."""
    p = fresh(p)
    if p.eps > 1e-8:
        p.eps = 1e-7
    p.poisson_tol = 1e-5
    p.poisson_max_cycles = 60
    G = oracle_grid(O, p)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 27).astype(np.complex64).astype(np.complex128)
    alpha = inclusion_alpha(p, 29)
    s = make_solver(p, alpha, psi0)
    mism = 0
    for n in range(10):
        psi_in, mu_in = gpu_state(s)
        K_in = s.observables()["K"]
        st = O.State(psi_in, mu_in, K=K_in)
        so = O.step(G, st, alpha.astype(np.float64), eps=p.eps)
        s.step(1)
        ng = s.observables()["last_sweeps"]
        psi_g, _ = gpu_state(s)
        if ng != so.sweeps:
            # r2 met eps within FP32 rounding on one side only: the two results differ by one
            # sweep of the iteration, so compare with the oracle run to the GPU's count
            mism += 1
            assert abs(ng - so.sweeps) <= 1
            st = O.State(psi_in, mu_in, K=K_in)
            O.step(G, st, alpha.astype(np.float64), fixed_sweeps=ng)
        assert np.max(np.abs(psi_g - st.psi)) <= TOL_PSI, (n, ng, so.sweeps)
    assert mism <= 2


def test_check_every_k_runs_whole_passes(O):
    from paper_1409_8340_gb300.solver import Params
    p = Params(48, 16, 8, bc=(OP, P, P), Bz=0.2, Jext=0.01, eps=1e-6, check_every=3)
    G = oracle_grid(O, p)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 37).astype(np.complex64).astype(np.complex128)
    alpha = inclusion_alpha(p, 39)
    s = make_solver(p, alpha, psi0)
    n = s.solve_psi()
    assert n % 3 == 0
    psi_o, no, _, _ = O.solve_psi(G, psi0, np.zeros(p.shape), alpha.astype(np.float64), 0.0, eps=p.eps,
                                  check_every=3)
    assert no == n
    assert np.max(np.abs(gpu_state(s)[0] - psi_o)) <= TOL_PSI


@pytest.mark.parametrize("name,p", CASES, ids=[c[0] for c in CASES])
def test_two_sweep_passes_match_single_sweeps(name, p):
    """Temporal blocking (two sweeps per pass over memory) keeps the per-sweep test:
    from the same state, the sweep counts are those of one sweep per pass and the
    states agree to FP32 rounding (the compiler may contract the same complex
    products into FMAs differently in the two kernels)."""
    base = fresh(p)
    base.poisson_tol = 0.0
    alpha = inclusion_alpha(base, 41)
    psi0 = I.random_psi(base.nx, base.ny, base.nz, 42)
    one = dataclasses.replace(base, sweeps_per_pass=1)
    two = dataclasses.replace(base, sweeps_per_pass=2)
    s1 = make_solver(one, alpha, psi0)
    s2 = make_solver(two, alpha, psi0)
    odd = even = 0
    for n in range(8):
        s1.step(1)
        s2.step(1)
        n1, n2 = s1.observables()["last_sweeps"], s2.observables()["last_sweeps"]
        assert n1 == n2, (n, n1, n2)
        odd += n1 % 2
        even += 1 - n1 % 2
        a, b = gpu_state(s1), gpu_state(s2)
        assert np.max(np.abs(a[0] - b[0])) <= 1e-6, (n, np.max(np.abs(a[0] - b[0])))
        assert np.max(np.abs(a[1] - b[1])) <= 1e-6 * max(1.0, np.max(np.abs(a[1]))), n
    # fixed sweep counts of both parities end on either stage of a pass
    for fs in (2, 3, 6, 7):
        t1 = make_solver(dataclasses.replace(one, fixed_sweeps=fs), alpha, psi0)
        t2 = make_solver(dataclasses.replace(two, fixed_sweeps=fs), alpha, psi0)
        t1.step(2)
        t2.step(2)
        a, b = gpu_state(t1), gpu_state(t2)
        assert np.max(np.abs(a[0] - b[0])) <= 1e-6, fs
    assert odd > 0 and even > 0   # both stages of a pass ended a solve
