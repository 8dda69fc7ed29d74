"""The xz-plane field gauge (Eq. B_xz, Eq. A_xz, y-wrap of Sec. 3.3.1) on the GPU.

The device builds its link table from FP64 phases; the oracle takes the same
gauge from its own link-phase routine (pinned on the CPU by plaquette fluxes,
gauge equivalence and winding).  Parity: init and first sweep at every site,
fixed-sweep trajectories of full steps (psi, K, mu), convergence-tested steps;
then the gauge invariants of the GPU path itself: with B along z the xz and yz
gauges give the same |psi|, mu, E_x and sweep counts, and a periodic box holds
its flux quanta as vortices.
"""
import dataclasses
import math

import numpy as np
import pytest

from _helpers import OP, P, gpu_state, inclusion_alpha, make_solver, oracle_grid
from paper_1409_8340_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_PSI = 2e-5


def xz(p, nz_quanta=None, nx_quanta=None):
    """Quantise Bz (periodic x and y) and Bx (periodic y and z) where the y wrap needs it."""
    p.xz_gauge = True
    if p.bc[1] == P and p.bc[0] == P and nz_quanta is not None:
        p.Bz = 2 * math.pi * nz_quanta / (p.length(0) * p.length(1))
    if p.bc[1] == P and p.bc[2] == P and p.nz >= 2 and nx_quanta is not None:
        p.Bx = 2 * math.pi * nx_quanta / (p.length(1) * p.length(2))
    return p


def cases():
    from paper_1409_8340_gb300.solver import Params
    return [
        ("periodic_40x20x12", xz(Params(40, 20, 12, bc=(P, P, P), Jext=0.01), 3, 1)),
        ("openx_45x19x10_J", xz(Params(45, 19, 10, bc=(OP, P, P), Bz=0.23, Jext=0.01, g=1.3), None, -1)),
        ("periodicx_openy_48x17x9", xz(Params(48, 17, 9, bc=(P, OP, P), Bz=0.3, Bx=0.12, Jext=0.015))),
        ("film_36x18x1", xz(Params(36, 18, 1, bc=(P, P, P), Jext=0.02), 2)),
        ("allopen_33x9x7", xz(Params(33, 9, 7, bc=(OP, OP, OP), Bz=0.4, Bx=0.2))),
        ("openz_32x24x9", xz(Params(32, 24, 9, bc=(P, P, OP), Bx=0.17, Jext=0.01), -2)),
    ]


CASES = cases()
IDS = [c[0] for c in CASES]


def theta_of(O, p):
    return O.xz_link_phases(oracle_grid(O, p), p.Bx)


@pytest.mark.parametrize("name,p", CASES, ids=IDS)
def test_init_and_first_sweep(O, name, p):
    p = dataclasses.replace(p, fixed_sweeps=1)
    G = oracle_grid(O, p)
    th = theta_of(O, p)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 7).astype(np.complex64).astype(np.complex128)
    mu0 = ((I.uniform(8, "t.mu", p.N).reshape(p.shape) - 0.5) * 0.2).astype(np.float32)
    alpha = inclusion_alpha(p, 9)
    K = 0.3 if p.bc[0] == P else 0.0
    s = make_solver(p, alpha, psi0, mu0, K)
    assert s.solve_psi() == 1
    b_g, D_g, _ = s.internals()
    b_o, D_o = O.init(G, psi0, mu0, alpha, K, theta=th)
    np.testing.assert_allclose(b_g.cpu().numpy(), b_o, rtol=0, atol=3e-6)
    np.testing.assert_allclose(D_g.cpu().numpy(), D_o, rtol=0, atol=3e-6)
    psi1_o, _ = O.sweep(G, psi0, b_o, D_o, K, theta=th)
    np.testing.assert_allclose(gpu_state(s)[0], psi1_o, rtol=0, atol=3e-6)


@pytest.mark.parametrize("name,p", CASES, ids=IDS)
def test_fixed_sweeps_trajectory(O, name, p):
    p = dataclasses.replace(p, fixed_sweeps=40, poisson_tol=1e-5, poisson_max_cycles=60)
    G = oracle_grid(O, p)
    th = theta_of(O, p)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 17).astype(np.complex64).astype(np.complex128)
    alpha = inclusion_alpha(p, 19)
    s = make_solver(p, alpha, psi0)
    st = O.State(psi0.copy(), np.zeros(p.shape))
    for n in range(10):
        s.step(1)
        so = O.step(G, st, alpha.astype(np.float64), theta=th, fixed_sweeps=40)
        psi_g, mu_g = gpu_state(s)
        assert np.max(np.abs(psi_g - st.psi)) <= TOL_PSI, (n, np.max(np.abs(psi_g - st.psi)))
        scale = max(1.0, np.max(np.abs(st.mu)))
        assert np.max(np.abs(mu_g - st.mu)) <= 2e-5 * scale, n
    obs = s.observables()
    assert abs(obs["K"] - st.K) < 1e-5
    assert abs(obs["Ex"] - so.Ex) < 1e-4 * max(1.0, abs(so.Ex))


@pytest.mark.parametrize("name,p", CASES[:3], ids=IDS[:3])
def test_tolerance_mode_per_step(O, name, p):
    p = dataclasses.replace(p, eps=1e-7, poisson_tol=1e-5, poisson_max_cycles=60)
    G = oracle_grid(O, p)
    th = theta_of(O, p)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 27).astype(np.complex64).astype(np.complex128)
    alpha = inclusion_alpha(p, 29)
    s = make_solver(p, alpha, psi0)
    mism = 0
    for n in range(8):
        psi_in, mu_in = gpu_state(s)
        K_in = s.observables()["K"]
        st = O.State(psi_in, mu_in, K=K_in)
        so = O.step(G, st, alpha.astype(np.float64), theta=th, eps=p.eps)
        s.step(1)
        ng = s.observables()["last_sweeps"]
        if ng != so.sweeps:
            # the test passed within FP32 rounding on one side only: compare with the
            # oracle run to the GPU's sweep count from the same input
            mism += 1
            assert abs(ng - so.sweeps) <= 1
            st = O.State(psi_in, mu_in, K=K_in)
            O.step(G, st, alpha.astype(np.float64), theta=th, fixed_sweeps=ng)
        assert np.max(np.abs(gpu_state(s)[0] - st.psi)) <= TOL_PSI, (n, ng, so.sweeps)
    assert mism <= 2


@pytest.mark.parametrize("name,p", [CASES[0], CASES[5]], ids=[IDS[0], IDS[5]])
def test_table_free_path_equals_the_link_table_path(O, name, p):
    """Even nx: the tiled kernels take the xz links from j-indexed tables; the same
    phases given as a 3N general-link table (per-site kernels) give the same steps."""
    p = dataclasses.replace(p, fixed_sweeps=30, poisson_tol=1e-5, poisson_max_cycles=60)
    q = dataclasses.replace(p, xz_gauge=False, general_links=True, Bx=0.0)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 37)
    alpha = inclusion_alpha(p, 38)
    a = make_solver(p, alpha, psi0)
    b = make_solver(q, alpha, psi0, link_phase=theta_of(O, p).astype(np.float32))
    for n in range(6):
        a.step(1)
        b.step(1)
        (xa, ma), (xb, mb) = gpu_state(a), gpu_state(b)
        assert np.max(np.abs(xa - xb)) < 5e-6, n
        assert np.max(np.abs(ma - mb)) < 5e-6, n


def test_xz_and_yz_gauges_agree_on_the_gpu():
    """B = (0, 0, Bz), open x and y, current injected through the x faces: the xz run from
    psi0 and the yz run from exp(i chi) psi0, chi_{i,j} = Bz (i hx ybar_j - j hy Lx / 2),
    give the same |psi|, mu, E_x and sweep counts."""
    from paper_1409_8340_gb300.solver import Params
    base = Params(48, 33, 12, bc=(OP, OP, P), Bz=0.27, Jext=0.015, eps=1e-8, poisson_tol=1e-5)
    pa = dataclasses.replace(base, xz_gauge=True)
    pb = dataclasses.replace(base)
    ii = np.arange(base.nx)[None, None, :]
    jj = np.arange(base.ny)[None, :, None]
    ybar = jj * base.hy - 0.5 * base.length(1)
    chi = np.broadcast_to(base.Bz * (ii * base.hx * ybar - jj * base.hy * base.length(0) / 2), base.shape)
    psi0 = I.random_psi(base.nx, base.ny, base.nz, 81)
    alpha = inclusion_alpha(base, 82)
    a = make_solver(pa, alpha, psi0)
    b = make_solver(pb, alpha, psi0 * np.exp(1j * chi))
    for n in range(15):
        a.step(1)
        b.step(1)
        (xa, ma), (xb, mb) = gpu_state(a), gpu_state(b)
        assert np.max(np.abs(np.abs(xa) - np.abs(xb))) < 2e-5, n
        assert np.max(np.abs(ma - mb)) < 2e-5, n
        oa, ob = a.observables(), b.observables()
        assert abs(oa["last_sweeps"] - ob["last_sweeps"]) <= 1
        assert abs(oa["Ex"] - ob["Ex"]) < 2e-5 + 1e-3 * abs(ob["Ex"])
    assert abs(oa["energy"] - ob["energy"]) < 1e-4 * abs(ob["energy"])


@pytest.mark.parametrize("nz_quanta,nx_quanta", [(3, 1), (-2, 2)])
def test_flux_quanta_become_vortices(O, nz_quanta, nx_quanta):
    """A periodic box relaxed in the xz gauge: the signed xy winding per z layer equals
    the flux quanta through the xy face (the topological charge of the y wrap)."""
    from paper_1409_8340_gb300.solver import Params
    p = xz(Params(32, 32, 8, bc=(P, P, P), hx=0.7, hy=0.7, hz=0.7, eps=1e-6), nz_quanta, nx_quanta)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 90)
    s = make_solver(p, np.ones(p.shape, np.float32), psi0)
    for _ in range(3):
        s.step(1)
        assert round(s.observables()["vortex_signed"]) == nz_quanta
    G = oracle_grid(O, p)
    psi, _ = gpu_state(s)
    assert O.winding(G, psi, s.observables()["K"], theta_of(O, p))[1] == nz_quanta * p.nz


def test_batch_and_adjoint_refuse_the_xz_gauge():
    import torch
    from paper_1409_8340_gb300._lib import TdglError
    from paper_1409_8340_gb300.solver import Batch
    p = CASES[1][1]
    alpha = inclusion_alpha(p, 95)
    with pytest.raises(TdglError):
        Batch([p], [torch.as_tensor(alpha).cuda()])
    s = make_solver(p, alpha, I.random_psi(p.nx, p.ny, p.nz, 96))
    with pytest.raises(TdglError):
        s.adjoint(4, checkpoint_every=2)
