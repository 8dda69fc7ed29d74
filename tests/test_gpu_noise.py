"""Thermal noise (Sec. 3.1.2) on the GPU against the FP64 oracle: the same
counter-based random numbers (site, step, seed) enter b on both sides, so b,
the first sweep and whole trajectories match to FP32 rounding."""
import dataclasses

import numpy as np
import pytest

from _helpers import OP, P, gpu_state, inclusion_alpha, make_solver, oracle_grid, quantised
from paper_1409_8340_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_PSI = 2e-5


def cases():
    from paper_1409_8340_gb300.solver import Params
    return [
        ("openx_34x22x13", Params(34, 22, 13, bc=(OP, P, P), Bz=0.21, Jext=0.02, noise_T=0.004, noise_seed=77)),
        ("periodic_16x16x8", quantised(Params(16, 16, 8, bc=(P, P, P), noise_T=0.01, noise_seed=(1 << 40) + 5), 2)),
        ("odd_nx_33x9x7", Params(33, 9, 7, bc=(OP, OP, OP), Bz=0.3, noise_T=0.002, noise_seed=3)),
        ("film_36x17x1", Params(36, 17, 1, bc=(OP, P, P), Bz=0.3, Jext=0.02, noise_T=0.003, noise_seed=11)),
    ]


CASES = cases()


def oracle_grid_noise(O, p):
    G = oracle_grid(O, p)
    G.noise_T = p.noise_T
    G.noise_seed = p.noise_seed
    return G


@pytest.mark.parametrize("name,p", CASES, ids=[c[0] for c in CASES])
def test_init_with_noise_every_step(O, name, p):
    p = dataclasses.replace(p, fixed_sweeps=1)
    G = oracle_grid_noise(O, p)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 5).astype(np.complex64)
    alpha = inclusion_alpha(p, 6)
    s = make_solver(p, alpha, psi0)
    for step in range(3):
        psi_in, mu_in = gpu_state(s)
        K = s.observables()["K"]
        s.solve_psi()
        b_g, _, _ = s.internals()
        b_o, _ = O.init(G, psi_in, mu_in, alpha, K)
        O.add_noise(G, b_o, step)
        assert np.max(np.abs(b_g.cpu().numpy() - b_o)) <= 3e-6, step


@pytest.mark.parametrize("name,p", CASES, ids=[c[0] for c in CASES])
def test_noisy_trajectory_matches_oracle(O, name, p):
    p = dataclasses.replace(p, fixed_sweeps=40, poisson_tol=1e-6, poisson_max_cycles=60)
    G = oracle_grid_noise(O, p)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 15).astype(np.complex64).astype(np.complex128)
    alpha = inclusion_alpha(p, 16)
    s = make_solver(p, alpha, psi0)
    st = O.State(psi0.copy(), np.zeros(p.shape))
    for n in range(6):
        s.step(1)
        O.step(G, st, alpha.astype(np.float64), fixed_sweeps=40)
        psi_g, mu_g = gpu_state(s)
        assert np.max(np.abs(psi_g - st.psi)) <= TOL_PSI, (n, np.max(np.abs(psi_g - st.psi)))
        assert np.max(np.abs(mu_g - st.mu)) <= 2e-5 * max(1.0, np.max(np.abs(st.mu))), n


def test_noise_counter_restarts_with_the_state_and_seed_matters():
    p = CASES[0][1]
    alpha = inclusion_alpha(p, 21)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 22).astype(np.complex64)
    a = make_solver(p, alpha, psi0)
    a.step(2)
    first = gpu_state(a)
    a.set_state(__import__("torch").as_tensor(psi0))
    a.step(2)
    again = gpu_state(a)
    assert np.array_equal(first[0], again[0])
    b = make_solver(dataclasses.replace(p, noise_seed=p.noise_seed + 1), alpha, psi0)
    b.step(2)
    assert np.max(np.abs(gpu_state(b)[0] - first[0])) > 1e-3


def test_batch_with_noise_matches_plain_handles():
    import torch
    from paper_1409_8340_gb300.solver import Batch
    ps = [CASES[0][1], CASES[1][1], dataclasses.replace(CASES[0][1], noise_seed=999)]
    alphas = [inclusion_alpha(p, 30 + i) for i, p in enumerate(ps)]
    psi0s = [I.random_psi(p.nx, p.ny, p.nz, 40 + i).astype(np.complex64) for i, p in enumerate(ps)]
    b = Batch(ps, [torch.as_tensor(a).cuda() for a in alphas])
    for i, s in enumerate(b.instances):
        s.set_state(torch.as_tensor(psi0s[i]))
    plain = [make_solver(p, a, x) for p, a, x in zip(ps, alphas, psi0s)]
    b.step(4)
    b.check()
    for i, s in enumerate(plain):
        s.step(4)
        x, y = gpu_state(b.instances[i]), gpu_state(s)
        assert np.max(np.abs(x[0] - y[0])) <= 1e-6, i


def test_adjoint_refuses_noise():
    from paper_1409_8340_gb300._lib import TdglError
    p = CASES[0][1]
    s = make_solver(p, inclusion_alpha(p, 50), I.random_psi(p.nx, p.ny, p.nz, 51))
    with pytest.raises(TdglError):
        s.adjoint(4, checkpoint_every=2)


@pytest.mark.parametrize("noise_T", [0.0, 0.004], ids=["no_noise", "noise"])
def test_checkpoint_resume_is_bitwise_continuous(noise_T):
    """100 straight steps equal 50 steps, a checkpoint to host memory (psi, mu, K, the
    previous step's mu that the extrapolated Poisson guess reads, and the step index,
    which is the noise counter), a fresh handle restored from it, and 50 more steps:
    bit for bit, with and without thermal noise."""
    from paper_1409_8340_gb300.solver import Params
    p = Params(64, 24, 12, bc=(OP, P, P), Bz=0.2, Jext=0.02, noise_T=noise_T, noise_seed=91)
    alpha = inclusion_alpha(p, 92)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 93)
    a = make_solver(p, alpha, psi0)
    a.step(100)
    b = make_solver(p, alpha, psi0)
    b.step(50)
    ck = b.checkpoint()
    assert ck["step"] == 50 and ck["mu_prev"] is not None
    b.close()
    c = make_solver(p, alpha)
    c.restore(ck)
    c.step(50)
    assert c.observables()["step"] == 100
    pa, ma = gpu_state(a)
    pc, mc = gpu_state(c)
    np.testing.assert_array_equal(pa, pc)
    np.testing.assert_array_equal(ma, mc)
    assert a.observables()["K"] == c.observables()["K"]
