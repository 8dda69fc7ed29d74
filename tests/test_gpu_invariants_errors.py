"""GPU checks of invariants and closed forms, and of the error paths of the C ABI.

Failures are made on the host: a sweep cap that is too small, a NaN written
into a small psi.  No test provokes a GPU fault, trap or hang.
"""
import math

import numpy as np
import pytest

from _helpers import OP, P, gpu_state, inclusion_alpha, make_solver, oracle_grid, quantised
from paper_1409_8340_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def gauge_transform(theta, chi):
    out = theta.copy()
    for ax, aa in ((0, 2), (1, 1), (2, 0)):
        out[ax] = theta[ax] + chi - np.roll(chi, -1, axis=aa)
    return out


def test_gauge_invariance_fp32(O):
    from paper_1409_8340_gb300.solver import Params
    p = quantised(Params(40, 24, 12, bc=(P, P, P), Jext=0.01, eps=1e-8, general_links=True,
                         poisson_tol=1e-5), 3, 1)
    G = oracle_grid(O, p)
    theta = O.landau_link_phases(G)
    chi = I.gauge_angles(p.nx, p.ny, p.nz, 71)
    theta2 = gauge_transform(theta, chi)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 72)
    alpha = inclusion_alpha(p, 73)
    a = make_solver(p, alpha, psi0, link_phase=theta.astype(np.float32))
    b = make_solver(p, alpha, psi0 * np.exp(1j * chi), link_phase=theta2.astype(np.float32))
    for n in range(20):
        a.step(1)
        b.step(1)
        pa, ma = gpu_state(a)
        pb, mb = gpu_state(b)
        assert np.max(np.abs(np.abs(pa) - np.abs(pb))) < 1e-5, n
        assert np.max(np.abs(ma - mb)) < 1e-5, n
        oa, ob = a.observables(), b.observables()
        assert oa["last_sweeps"] == ob["last_sweeps"]
    assert abs(oa["energy"] - ob["energy"]) < 1e-5 * abs(oa["energy"])
    # general-link mode with Landau phases equals the built-in Landau tables
    p2 = quantised(Params(40, 24, 12, bc=(P, P, P), Jext=0.01, eps=1e-8, poisson_tol=1e-5), 3, 1)
    c = make_solver(p2, alpha, psi0)
    c.step(20)
    assert np.max(np.abs(gpu_state(c)[0] - pa)) < 2e-5


def test_uniform_fixed_point_and_plane_wave(O):
    from paper_1409_8340_gb300.solver import Params
    # zero field, zero current: |psi|^2 = alpha/beta is a fixed point
    p0 = Params(32, 8, 8, bc=(P, P, P), fixed_sweeps=60, Jext=0.0, beta=1.0, poisson_tol=1e-6)
    alpha = 0.8
    psi = np.full(p0.shape, math.sqrt(alpha) * np.exp(0.4j), dtype=np.complex64)
    s = make_solver(p0, np.full(p0.shape, alpha, np.float32), psi)
    # plane wave exp(i k x), k = 2 pi / Lx, under current: amplitude and K follow the scalar recurrence
    p = Params(32, 8, 8, bc=(P, P, P), fixed_sweeps=60, Jext=0.02, beta=1.0, poisson_tol=1e-6)
    k = 2 * math.pi / p.length(0)
    x = np.arange(p.nx) * p.hx
    pw = (0.55 * np.exp(1j * k * x))[None, None, :] * np.ones(p.shape)
    s2 = make_solver(p, np.full(p.shape, 0.9, np.float32), pw.astype(np.complex64), K=0.13)
    s.step(5)
    assert np.max(np.abs(gpu_state(s)[0] - psi)) < 2e-6
    a, K = 0.55, 0.13
    cx = 1 / p.hx ** 2
    for n in range(10):
        lam = 4 * cx * math.sin((k + K) * p.hx / 2) ** 2
        c = 0.9 - lam - a * a
        a = a * (1 + p.ht / 2 * c) / (1 - p.ht / 2 * c)
        jav = a * a * math.sin((k + K) * p.hx) / p.hx
        K = K + p.ht * (p.Jext - jav)
        K -= (2 * math.pi / p.hx) * math.floor(K * p.hx / (2 * math.pi))
        s2.step(1)
        ps, _ = gpu_state(s2)
        assert np.max(np.abs(np.abs(ps) - a)) < 2e-6
        assert abs(s2.observables()["K"] - K) < 2e-6


def test_energy_decreases_with_frozen_mu_K(O):
    from paper_1409_8340_gb300.solver import Params
    p = quantised(Params(48, 32, 8, bc=(P, P, P), fixed_sweeps=40, freeze_mu_K=True), 3)
    alpha = inclusion_alpha(p, 81)
    s = make_solver(p, alpha, I.random_psi(p.nx, p.ny, p.nz, 82))
    F = [s.observables()["energy"]]
    for _ in range(30):
        s.step(1)
        F.append(s.observables()["energy"])
    assert np.all(np.diff(F) < 0), np.diff(F).max()


def test_not_converged_leaves_state(O):
    from paper_1409_8340_gb300._lib import TdglError
    from paper_1409_8340_gb300.solver import Params
    p = Params(40, 16, 8, bc=(OP, P, P), Bz=0.2, Jext=0.01, eps=1e-12, max_iter=2)
    s = make_solver(p, inclusion_alpha(p, 91), I.random_psi(p.nx, p.ny, p.nz, 92))
    before = gpu_state(s)
    with pytest.raises(TdglError) as e:
        s.step(1)
    assert e.value.code == -2
    after = gpu_state(s)
    np.testing.assert_array_equal(before[0], after[0])
    np.testing.assert_array_equal(before[1], after[1])
    # a feasible tolerance works again from the same state
    p.eps = 1e-6
    p.max_iter = 200
    s2 = make_solver(p, inclusion_alpha(p, 91), after[0], after[1])
    s2.step(2)


def test_nonfinite_is_reported(O):
    from paper_1409_8340_gb300._lib import TdglError
    from paper_1409_8340_gb300.solver import Params
    p = Params(40, 16, 8, bc=(OP, P, P), Bz=0.2, eps=1e-6)
    psi = I.random_psi(p.nx, p.ny, p.nz, 93).astype(np.complex64)
    psi[3, 5, 7] = np.nan
    s = make_solver(p, inclusion_alpha(p, 94), psi)
    with pytest.raises(TdglError) as e:
        s.step(1)
    assert e.value.code == -3
    # the next step from a clean state succeeds (status is reset per step)
    import torch
    s.set_state(torch.as_tensor(I.random_psi(p.nx, p.ny, p.nz, 95).astype(np.complex64)))
    s.step(1)


def test_host_buffers_round_trip(O):
    from paper_1409_8340_gb300.solver import Params
    p = Params(40, 16, 8, bc=(OP, P, P), Bz=0.2, Jext=0.01)
    s = make_solver(p, inclusion_alpha(p, 96))
    psi = I.random_psi(p.nx, p.ny, p.nz, 97).astype(np.complex64)
    mu = (I.uniform(98, "t", p.N).reshape(p.shape) - 0.5).astype(np.float32)
    s.upload_state(psi, mu, 0.0)
    psi2, mu2, K = s.download_state()
    np.testing.assert_array_equal(psi2.numpy(), psi)
    np.testing.assert_array_equal(mu2.numpy(), mu)
