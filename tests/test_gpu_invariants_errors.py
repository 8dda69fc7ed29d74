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


def _timeout_case():
    """512-site x lines, so that the Jacobi sweep, the Poisson right-hand side and the
    finest multigrid level all run on the staged kernels."""
    from paper_1409_8340_gb300.solver import Params
    p = Params(512, 32, 16, bc=(OP, P, P), Bz=0.2, Jext=0.01, eps=1e-6)
    alpha = inclusion_alpha(p, 111)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 112).astype(np.complex64)
    return p, alpha, psi0


def test_staged_sweep_timeout_is_reported_and_handle_recovers(O):
    """The first block of every staged sweep waits for bytes that never come: its waits
    run out after 20 ms (no copy faults), the step reports TDGL_ERR_TIMEOUT, the state
    stays at the last completed step, and the last-block reductions of the handle stay
    intact (the timed-out block still took its ticket): the observables of the same
    state equal those of an untouched handle.  The error persists until a state is
    loaded; then the handle steps exactly as the untouched one."""
    import torch
    from paper_1409_8340_gb300._lib import TDGL_ERR_TIMEOUT, TdglError
    p, alpha, psi0 = _timeout_case()
    s = make_solver(p, alpha, psi0)
    ref = make_solver(p, alpha, psi0)
    o_ref = ref.observables()
    s.test_staged_waits(20_000_000, 64)
    with pytest.raises(TdglError) as e:
        s.step(1)
    assert e.value.code == TDGL_ERR_TIMEOUT
    s.test_staged_waits(0, 0)
    psi_s, _ = gpu_state(s)
    np.testing.assert_array_equal(psi_s, psi0.astype(np.complex128))
    o = s.observables()
    for k in ("psi2_mean", "energy", "vortex_unsigned", "vortex_signed"):
        assert o[k] == pytest.approx(o_ref[k], rel=1e-12, abs=1e-12), k
    with pytest.raises(TdglError) as e:
        s.step(1)
    assert e.value.code == TDGL_ERR_TIMEOUT
    s.set_state(torch.as_tensor(psi0))
    s.step(3)
    ref.step(3)
    a, b = gpu_state(s), gpu_state(ref)
    np.testing.assert_allclose(a[0], b[0], rtol=0, atol=1e-6)
    np.testing.assert_allclose(a[1], b[1], rtol=0, atol=1e-5)


def test_staged_poisson_timeout_is_reported_and_handle_recovers(O):
    """The same for the Poisson solve: the first block of the staged right-hand side and
    the first warp of every staged smoother launch time out; the solve itself returns
    (it is asynchronous) and the next step reports TDGL_ERR_TIMEOUT; after a state load
    the handle steps as an untouched one."""
    import torch
    from paper_1409_8340_gb300._lib import TDGL_ERR_TIMEOUT, TdglError
    p, alpha, psi0 = _timeout_case()
    s = make_solver(p, alpha, psi0)
    ref = make_solver(p, alpha, psi0)
    s.step(1)
    ref.step(1)
    psi1, mu1 = gpu_state(s)
    s.test_staged_waits(20_000_000, 64)
    s.solve_mu()
    s.test_staged_waits(0, 0)
    with pytest.raises(TdglError) as e:
        s.step(1)
    assert e.value.code == TDGL_ERR_TIMEOUT
    # both handles load the same state (which also drops the previous mu that the
    # extrapolated Poisson guess reads), then step alike
    K1 = ref.observables()["K"]
    for h in (s, ref):
        h.set_state(torch.as_tensor(psi1.astype(np.complex64)), torch.as_tensor(mu1.astype(np.float32)), K1)
    s.step(2)
    ref.step(2)
    a, b = gpu_state(s), gpu_state(ref)
    np.testing.assert_allclose(a[0], b[0], rtol=0, atol=1e-6)
    np.testing.assert_allclose(a[1], b[1], rtol=0, atol=1e-5)


def test_vortex_count_of_known_defects_on_the_gpu():
    """Vortices and antivortices at known plaquette centres (zero field, open x and y):
    the GPU's unsigned count per layer is the number of defects, the signed count their
    net charge (the oracle's winding is pinned on the same state)."""
    import torch
    from test_oracle_pins import DEFECTS, vortex_state
    from paper_1409_8340_gb300.solver import Params
    p = Params(24, 22, 3, bc=(OP, OP, P))
    s = make_solver(p, np.ones(p.shape, dtype=np.float32))
    s.set_state(torch.as_tensor(vortex_state(p.nx, p.ny, p.nz, DEFECTS).astype(np.complex64)))
    o = s.observables()
    assert o["vortex_unsigned"] == len(DEFECTS)
    assert o["vortex_signed"] == sum(sg for _, _, sg in DEFECTS)
