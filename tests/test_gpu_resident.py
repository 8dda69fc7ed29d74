"""The device-resident step loop (tdgl_step_resident): n steps as one CUDA graph of
conditional nodes, against the host-driven tdgl_step on twin handles.

Both run the same kernels with the same arguments in the same order (Sec. 4.1's loop:
init, Jacobi sweeps until Eq. 11 holds, K ODE, Poisson solve, voltage); only where the
loop's decisions are taken differs (on the device against after a host read of the
control block).  So the results must agree bit for bit: psi, mu (with its pending
projection applied), K, E_x, the sweeps of the last step, the total sweeps and the step
count.  The host-driven path is pinned to the oracle elsewhere (the step, batch and
default-configuration parity tests); the one oracle check here runs the resident loop
on the benchmark's default configuration.
"""
import numpy as np
import pytest

from _helpers import OP, P, gpu_state, inclusion_alpha, make_solver, oracle_grid, quantised
from paper_1409_8340_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def twins(p, seed=11, mu0=False):
    alpha = inclusion_alpha(p, seed)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, seed + 1).astype(np.complex64)
    m0 = ((I.uniform(seed + 2, "res.mu", p.N).reshape(p.shape) - 0.5) * 0.1).astype(np.float32) if mu0 else None
    a, b = make_solver(p, alpha, psi0, m0), make_solver(p, alpha, psi0, m0)
    a.profile_enable(True)
    b.profile_enable(True)
    return a, b


def assert_same(a, b, tag):
    pa, ma = gpu_state(a)
    pb, mb = gpu_state(b)
    assert np.array_equal(pa, pb), (tag, np.max(np.abs(pa - pb)))
    assert np.array_equal(ma, mb), (tag, np.max(np.abs(ma - mb)))
    oa, ob = a.observables(), b.observables()
    for k in ("K", "Ex", "last_sweeps", "step", "javg", "poisson_cycles"):
        assert oa[k] == ob[k], (tag, k, oa[k], ob[k])
    ra, rb = a.profile(), b.profile()
    assert ra["steps"] == rb["steps"] and ra["sweeps"] == rb["sweeps"], (tag, ra, rb)


def cases():
    from paper_1409_8340_gb300.solver import Params
    return {
        # the benchmark's defaults: open x, extrapolated Poisson guess, one V-cycle, staged sweeps
        "openx_512x32x16": Params(512, 32, 16, bc=(OP, P, P), Bz=0.2, Jext=0.025),
        # K ODE (periodic x) with a field in two directions
        "periodic_64x32x16_K": quantised(Params(64, 32, 16, bc=(P, P, P), Jext=0.02), 8, 2),
        # the previous step's mu as the guess (the mu buffers never swap), two V-cycles
        "guess_prev_96x40x12": Params(96, 40, 12, bc=(OP, P, OP), Bz=0.2, Jext=0.02, poisson_guess=1,
                                      poisson_cycles=2),
        # thermal noise (the init's counter-based draws advance with the step counter)
        "noise_64x24x10": Params(64, 24, 10, bc=(OP, P, P), Bz=0.2, Jext=0.02, noise_T=0.02, noise_seed=5),
        # odd x extent: the register-tiled sweep kernel instead of the staged one
        "oddx_63x20x9": Params(63, 20, 9, bc=(OP, OP, P), Bz=0.25, Jext=0.02),
        # psi only: no K update and no Poisson solve
        "frozen_48x24x8": quantised(Params(48, 24, 8, bc=(P, P, P), freeze_mu_K=True), 6),
        # a sweep decision every third sweep
        "check3_64x32x8": Params(64, 32, 8, bc=(OP, P, P), Bz=0.2, Jext=0.02, check_every=3),
        # the xz-plane field (Eq. A_xz): staged sweeps with the j-indexed link tables
        "xz_gauge_128x32x16": Params(128, 32, 16, bc=(OP, P, OP), Bz=0.2, Bx=0.15, xz_gauge=True, Jext=0.01),
        # a tighter tolerance: more passes of the sweep loop per step
        "tight_eps_64x32x16": Params(64, 32, 16, bc=(OP, P, P), Bz=0.2, Jext=0.02, eps=1e-9, max_iter=400),
    }


@pytest.mark.parametrize("name", list(cases()))
def test_resident_steps_equal_host_steps(name):
    p = cases()[name]
    a, b = twins(p)
    for n in (1, 1, 5, 13):
        a.step(n)
        b.step_resident(n)
        assert_same(a, b, (name, n))


def test_resident_after_state_loads_and_checkpoints():
    """A state load mid-run (the first step after it runs launch by launch), a checkpoint
    restore with the previous mu, and host and resident steps interleaved."""
    import torch
    p = cases()["openx_512x32x16"]
    a, b = twins(p, seed=21)
    a.step(6)
    b.step_resident(6)
    ck = a.checkpoint()
    psi_new = torch.as_tensor(I.random_psi(p.nx, p.ny, p.nz, 23).astype(np.complex64))
    a.set_state(psi_new)
    b.set_state(psi_new)
    a.step(4)
    b.step_resident(4)
    assert_same(a, b, "after set_state")
    a.restore(ck)
    b.restore(ck)
    a.step(3)
    b.step(1)
    b.step_resident(1)
    b.step(1)
    assert_same(a, b, "after restore")
    a.step(7)
    b.step_resident(7)
    assert_same(a, b, "interleaved")


def test_resident_failure_stops_where_the_host_path_stops():
    """A Jacobi solve that does not converge within max_iter: both paths stop at the same
    step with TDGL_ERR_NOT_CONVERGED and the state of the step before."""
    from paper_1409_8340_gb300 import _lib
    from paper_1409_8340_gb300._lib import TdglError
    from paper_1409_8340_gb300.solver import Params
    p = Params(64, 32, 8, bc=(OP, P, P), Bz=0.2, Jext=0.02, eps=1e-6, max_iter=6)
    a, b = twins(p, seed=31)
    ea = eb = None
    try:
        a.step(40)
    except TdglError as e:
        ea = e
    try:
        b.step_resident(40)
    except TdglError as e:
        eb = e
    assert ea is not None and eb is not None, "max_iter 6 must fail within 40 steps"
    assert ea.code == eb.code == _lib.TDGL_ERR_NOT_CONVERGED, (str(ea), str(eb))
    pa, ma = gpu_state(a)
    pb, mb = gpu_state(b)
    assert a.observables()["step"] == b.observables()["step"] < 40
    assert np.array_equal(pa, pb) and np.array_equal(ma, mb)


def test_resident_refuses_what_it_does_not_cover_and_accepts_zero_steps():
    from paper_1409_8340_gb300 import _lib
    from paper_1409_8340_gb300.solver import Params
    L = _lib.load()
    base = dict(bc=(OP, P, P), Bz=0.2, Jext=0.02)
    for kw in (dict(poisson_tol=1e-6), dict(fixed_sweeps=4), dict(sweeps_per_pass=2)):
        p = Params(64, 32, 8, **base, **kw)
        s = make_solver(p, inclusion_alpha(p, 41), I.random_psi(p.nx, p.ny, p.nz, 42))
        assert L.tdgl_step_resident(s._h, 2) == _lib.TDGL_ERR_INVALID_ARG, kw
        assert L.tdgl_step_resident(s._h, -1) == _lib.TDGL_ERR_INVALID_ARG
    p = Params(64, 32, 8, **base)
    s = make_solver(p, inclusion_alpha(p, 43), I.random_psi(p.nx, p.ny, p.nz, 44))
    before = gpu_state(s)
    assert L.tdgl_step_resident(s._h, 0) == 0
    after = gpu_state(s)
    assert np.array_equal(before[0], after[0]) and s.observables()["step"] == 0


def test_resident_default_configuration_against_the_oracle(O):
    """The benchmark's defaults stepped by the resident loop into flux flow, then per step:
    mu against the oracle's exact solve of the GPU's own right-hand side, within a tenth
    of the one-step lag of mu plus 1e-4 max|mu| (the bound of the default-configuration
    parity test), and E_x within 1e-3 relative."""
    import torch
    from paper_1409_8340_gb300.solver import Params, Solver, pattern
    p = Params(512, 64, 32, bc=(OP, P, P), Bz=0.2, Jext=0.025)
    box = (p.length(0), p.length(1), p.length(2))
    cand = I.ellipsoids(max(200, int(20000 * p.N / (512 * 512 * 256))), box, 1.5, 5.0, seed=3)
    alpha, _, _ = pattern(p, cand, I.target_sites(0.10, p.N))
    G = oracle_grid(O, p)
    s = Solver(p, alpha)
    s.set_state(torch.as_tensor(I.random_psi(p.nx, p.ny, p.nz, 3).astype(np.complex64)))
    s.step_resident(100)
    for n in range(10):
        _, mu_prev = gpu_state(s)
        s.step_resident(1)
        o = s.observables()
        f = s.internals()[2].cpu().numpy().astype(np.float64)
        _, mu = gpu_state(s)
        mu_ex = O.poisson_solve(G, f)
        lag = np.max(np.abs(mu_ex - mu_prev))
        assert np.max(np.abs(mu - mu_ex)) <= 0.1 * lag + 1e-4 * np.max(np.abs(mu_ex)), n
        ex_ex = O.voltage_open_x(G, mu_ex)
        assert abs(o["Ex"] - ex_ex) <= 1e-3 * abs(ex_ex), (n, o["Ex"], ex_ex)


def test_enqueued_steps_equal_host_steps():
    """tdgl_step_enqueue: chained enqueues without waiting, then tdgl_sync (or any other
    call, which accounts for the pending steps first) -- the same bits as tdgl_step."""
    p = cases()["openx_512x32x16"]
    a, b = twins(p, seed=51)
    a.step(12)
    b.step_enqueue(3)
    b.step_enqueue(4)
    b.step_enqueue(5)
    b.sync()
    assert_same(a, b, "chained enqueues")
    a.step(6)
    b.step_enqueue(6)
    assert_same(a, b, "implicit sync")        # gpu_state reads the state: the pending steps first
    a.step(2)
    b.step_enqueue(1)
    b.step(1)                                 # a host-driven step after pending resident ones
    assert_same(a, b, "host step after enqueue")


def test_enqueued_failure_halts_the_later_steps():
    """A failure inside the graph halts every step enqueued after it: sync raises the error
    and the state is that of the host-driven path's last good step.  The failure is a staged
    sweep's bounded wait made to run out (the test hook of the timeout tests)."""
    from paper_1409_8340_gb300._lib import TDGL_ERR_TIMEOUT, TdglError
    p = cases()["openx_512x32x16"]
    a, b = twins(p, seed=61)
    a.step(2)
    b.step(2)
    for s in (a, b):
        s.test_staged_waits(20_000_000, 64)
    with pytest.raises(TdglError) as ea:
        a.step(5)
    b.step_enqueue(3)
    b.step_enqueue(3)
    with pytest.raises(TdglError) as eb:
        b.sync()
    assert ea.value.code == eb.value.code == TDGL_ERR_TIMEOUT
    b.sync()                                  # the error is reported once
    for s in (a, b):
        s.test_staged_waits(0, 0)
    pa, ma = gpu_state(a)
    pb, mb = gpu_state(b)
    assert a.observables()["step"] == b.observables()["step"] == 2
    assert np.array_equal(pa, pb) and np.array_equal(ma, mb)


def test_enqueued_not_converged_matches_the_host_path():
    """A solve that cannot converge within max_iter: the error comes from the enqueue (its
    first, launch-by-launch step) or from sync, and the state is the host path's."""
    from paper_1409_8340_gb300 import _lib
    from paper_1409_8340_gb300._lib import TdglError
    from paper_1409_8340_gb300.solver import Params
    p = Params(64, 32, 8, bc=(OP, P, P), Bz=0.2, Jext=0.02, eps=1e-6, max_iter=6)
    a, b = twins(p, seed=62)
    with pytest.raises(TdglError) as ea:
        a.step(60)
    with pytest.raises(TdglError) as eb:
        b.step_enqueue(30)
        b.step_enqueue(30)
        b.sync()
    assert ea.value.code == eb.value.code == _lib.TDGL_ERR_NOT_CONVERGED
    pa, ma = gpu_state(a)
    pb, mb = gpu_state(b)
    assert a.observables()["step"] == b.observables()["step"] < 60
    assert np.array_equal(pa, pb) and np.array_equal(ma, mb)
