"""Batched persistent step: every instance of a batch must follow the same
trajectory as a plain single-instance handle (and the FP64 oracle), whatever
the launch shape, graph replay or tuning; failures stay per instance; the
grid barrier's bounded wait reports a timeout instead of hanging.

Instances span both x boundary conditions, ragged tiles (sizes not multiples
of the 64 x 8 sweep tile), a frozen-mu instance and per-instance tolerances.
"""
import dataclasses

import numpy as np
import pytest

from _helpers import OP, P, gpu_state, inclusion_alpha, make_solver, oracle_grid, quantised
from paper_1409_8340_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_PSI = 2e-5


def batch_cases():
    from paper_1409_8340_gb300.solver import Params
    return [
        Params(34, 22, 13, bc=(OP, P, P), Bz=0.21, Jext=0.02, eps=1e-7, poisson_cycles=3),
        quantised(Params(16, 16, 8, bc=(P, P, P), eps=1e-6, poisson_cycles=2), 2),
        Params(40, 18, 11, bc=(OP, OP, P), Bz=0.35, Jext=0.01, eps=3e-7, poisson_cycles=2),
        Params(32, 16, 16, bc=(P, OP, OP), Bz=0.12, Jext=0.015, eps=1e-6, poisson_cycles=2),
        Params(24, 20, 9, bc=(OP, P, P), Bz=0.3, freeze_mu_K=True, eps=1e-6),
    ]


def make_batch(ps, alphas, psi0s, mu0s=None):
    import torch
    from paper_1409_8340_gb300.solver import Batch
    b = Batch(ps, [torch.as_tensor(a).cuda() for a in alphas])
    for i, s in enumerate(b.instances):
        mu = None if mu0s is None else torch.as_tensor(np.asarray(mu0s[i], dtype=np.float32))
        s.set_state(torch.as_tensor(psi0s[i].astype(np.complex64)), mu, 0.0)
    return b


def inputs(ps, seed):
    alphas = [inclusion_alpha(p, seed + 3 * i) for i, p in enumerate(ps)]
    psi0s = [I.random_psi(p.nx, p.ny, p.nz, seed + 3 * i + 1) for i, p in enumerate(ps)]
    mu0s = [((I.uniform(seed + 3 * i + 2, "t.mu", p.N).reshape(p.shape) - 0.5) * 0.1).astype(np.float32)
            for i, p in enumerate(ps)]
    return alphas, psi0s, mu0s


@pytest.mark.parametrize("guess", [1, 2], ids=["previous_mu", "extrapolated_mu"])
def test_batch_matches_plain_handles(guess):
    """Both Poisson starting guesses: the previous mu, and 2 mu^(n-1) - mu^(n-2)."""
    ps = [dataclasses.replace(p, poisson_guess=guess) for p in batch_cases()]
    alphas, psi0s, mu0s = inputs(ps, 100)
    b = make_batch(ps, alphas, psi0s, mu0s)
    plain = [make_solver(dataclasses.replace(p), a, psi, mu) for p, a, psi, mu in zip(ps, alphas, psi0s, mu0s)]
    for n in range(6):
        b.step(1)
        b.check()
        obs_b = b.observables()
        for i, s in enumerate(plain):
            s.step(1)
            pg, mg = gpu_state(s)
            pb, mb = gpu_state(b.instances[i])
            assert np.max(np.abs(pb - pg)) <= 1e-6, (n, i, np.max(np.abs(pb - pg)))
            scale = max(1.0, np.max(np.abs(mg)))
            assert np.max(np.abs(mb - mg)) <= 1e-6 * scale, (n, i, np.max(np.abs(mb - mg)))
            o = s.observables()
            assert obs_b[i]["last_sweeps"] == o["last_sweeps"], (n, i)
            assert abs(obs_b[i]["K"] - o["K"]) <= 1e-9
            assert abs(obs_b[i]["Ex"] - o["Ex"]) <= 1e-6 * max(1.0, abs(o["Ex"])), (n, i, obs_b[i]["Ex"], o["Ex"])
    st = b.stats()
    assert st["steps"] == 6
    assert st["sweeps"] == sum(st["instance_sweeps"]) and st["sweeps"] > 6 * len(ps)


def test_batch_against_oracle(O):
    """Two instances, 4 steps, convergence-tested sweeps, each step checked against the
    oracle from the batch's own input state at the per-step tolerance of the plain path
    (2e-5); the oracle's mu is the exact Poisson solution and the batch runs enough fixed
    V-cycles to reach it (within the FP32 floor of the multigrid, 1e-4 max|mu|).  Where the
    convergence test passed within FP32 rounding on one side only, the oracle is run to
    the batch's sweep count."""
    from paper_1409_8340_gb300.solver import Params
    ps = [Params(34, 22, 13, bc=(OP, P, P), Bz=0.21, Jext=0.02, eps=1e-7, poisson_cycles=12),
          quantised(Params(16, 16, 8, bc=(P, P, P), eps=1e-7, poisson_cycles=12), 2)]
    alphas, psi0s, _ = inputs(ps, 200)
    psi0s = [p.astype(np.complex64).astype(np.complex128) for p in psi0s]
    b = make_batch(ps, alphas, psi0s)
    Gs = [oracle_grid(O, p) for p in ps]
    mism = 0
    for n in range(4):
        ins = []
        for i in range(len(ps)):
            psi_in, mu_in = gpu_state(b.instances[i])
            ins.append((psi_in, mu_in, b.observables()[i]["K"]))
        b.step(1)
        b.check()
        obs = b.observables()
        for i, p in enumerate(ps):
            a = alphas[i].astype(np.float64)
            st = O.State(ins[i][0], ins[i][1], K=ins[i][2])
            so = O.step(Gs[i], st, a, eps=p.eps)
            ng = obs[i]["last_sweeps"]
            if ng != so.sweeps:
                mism += 1
                assert abs(ng - so.sweeps) <= 1
                st = O.State(ins[i][0], ins[i][1], K=ins[i][2])
                O.step(Gs[i], st, a, fixed_sweeps=ng)
            psi_b, mu_b = gpu_state(b.instances[i])
            assert np.max(np.abs(psi_b - st.psi)) <= TOL_PSI, (n, i, np.max(np.abs(psi_b - st.psi)))
            scale = max(1.0, np.max(np.abs(st.mu)))
            assert np.max(np.abs(mu_b - st.mu)) <= 1e-4 * scale, (n, i, np.max(np.abs(mu_b - st.mu)))
            assert abs(obs[i]["K"] - st.K) <= 1e-5
    assert mism <= 2


def test_staged_and_register_tiled_tiles_agree():
    """The tiles staged in shared memory and the register-tiled ones compute every
    site with the same arithmetic in the same order.  After one step (the sweeps
    alone decide psi) psi agrees bit for bit, with the same sweep counts; over five
    steps, where the right-hand side feeds mu back (its products may be contracted
    into fused multiply-adds differently in the two code paths, an ulp apart), psi
    and mu agree to 1e-6 like any two launch shapes."""
    from paper_1409_8340_gb300.solver import Params
    # and two grids wider than one tile (x halo pairs from the neighbouring tiles, a
    # ragged last tile), open and periodic in x
    ps = batch_cases() + [Params(132, 10, 7, bc=(OP, P, P), Bz=0.2, Jext=0.02, eps=1e-6, poisson_cycles=2),
                          Params(136, 12, 6, bc=(P, OP, OP), Bz=0.12, Jext=0.015, eps=1e-6, poisson_cycles=2)]
    alphas, psi0s, mu0s = inputs(ps, 310)
    one, five = {}, {}
    for kind in (0, 1):
        b = make_batch(ps, alphas, psi0s, mu0s)
        b.set_tuning(sweep_kernel=kind, kz=[1, 2, 3, 16, 5, 7, 4])
        assert b.tuning()["sweep_kernel"] == kind
        b.step(1)
        b.check()
        one[kind] = ([gpu_state(s)[0] for s in b.instances], b.stats()["instance_sweeps"])
        b.step(4)
        b.check()
        five[kind] = [gpu_state(s) for s in b.instances]
    assert one[0][1] == one[1][1]
    for i in range(len(ps)):
        assert np.array_equal(one[0][0][i], one[1][0][i]), i
        (p0, m0), (p1, m1) = five[0][i], five[1][i]
        assert np.max(np.abs(p0 - p1)) <= 1e-6, (i, np.max(np.abs(p0 - p1)))
        assert np.max(np.abs(m0 - m1)) <= 1e-6 * max(1.0, np.max(np.abs(m1))), i


def test_graph_replay_and_launch_shapes_agree():
    """Plain launches and graph replays, 1..3 blocks per SM and any sweep tile
    depth give identical psi (every site is computed the same way)."""
    ps = batch_cases()[:4]
    alphas, psi0s, mu0s = inputs(ps, 300)
    ref = None
    for tune in ({"graph_steps": 0}, {"graph_steps": 3}, {"graph_steps": 2, "blocks_per_sm": 1},
                 {"graph_steps": 0, "blocks_per_sm": 3, "kz": [1, 2, 3, 16]},
                 {"graph_steps": 2, "sweep_kernel": 1, "kz": [4, 1, 5, 2]}):
        b = make_batch(ps, alphas, psi0s, mu0s)
        b.set_tuning(**tune)
        b.step(5)
        b.check()
        st = b.stats()
        if tune["graph_steps"] > 0:
            assert st["graph"] == 1
        out = [gpu_state(s) for s in b.instances]
        if ref is None:
            ref = out
            continue
        for i in range(len(ps)):
            assert np.max(np.abs(out[i][0] - ref[i][0])) <= 1e-6, (tune, i)
            assert np.max(np.abs(out[i][1] - ref[i][1])) <= 1e-6 * max(1.0, np.max(np.abs(ref[i][1])))
        b.close()


def test_autotune_leaves_state_and_keeps_trajectory():
    ps = batch_cases()
    alphas, psi0s, mu0s = inputs(ps, 400)
    b = make_batch(ps, alphas, psi0s, mu0s)
    before = [gpu_state(s) for s in b.instances]
    rep = b.autotune(trial_steps=2)
    assert rep["candidates"] >= 3 and rep["classes"] == len(ps)
    assert rep["ms_best"] <= rep["ms_default"]
    after = [gpu_state(s) for s in b.instances]
    for x, y in zip(before, after):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
    assert b.stats()["steps"] == 0
    c = make_batch(ps, alphas, psi0s, mu0s)
    b.step(3)
    c.step(3)
    b.check()
    c.check()
    for i in range(len(ps)):
        x, y = gpu_state(b.instances[i]), gpu_state(c.instances[i])
        assert np.max(np.abs(x[0] - y[0])) <= 1e-6
        assert np.max(np.abs(x[1] - y[1])) <= 1e-6 * max(1.0, np.max(np.abs(y[1])))


def test_failed_instance_is_frozen_others_advance():
    from paper_1409_8340_gb300._lib import TDGL_ERR_NOT_CONVERGED
    ps = batch_cases()[:3]
    ps[1] = dataclasses.replace(ps[1], eps=1e-14, max_iter=3)   # cannot converge in 3 sweeps
    alphas, psi0s, mu0s = inputs(ps, 500)
    b = make_batch(ps, alphas, psi0s, mu0s)
    frozen_before = gpu_state(b.instances[1])
    plain = make_solver(dataclasses.replace(ps[0]), alphas[0], psi0s[0], mu0s[0])
    b.step(3)
    plain.step(3)
    rc, st = b.status()
    assert rc == TDGL_ERR_NOT_CONVERGED
    assert st == [0, TDGL_ERR_NOT_CONVERGED, 0]
    x = gpu_state(b.instances[1])
    assert np.array_equal(x[0], frozen_before[0]) and np.array_equal(x[1], frozen_before[1])
    assert np.max(np.abs(gpu_state(b.instances[0])[0] - gpu_state(plain)[0])) <= 1e-6
    assert b.stats()["instance_sweeps"][1] == 3


def test_plain_stepping_of_batch_instances_is_refused():
    from paper_1409_8340_gb300._lib import TdglError
    ps = batch_cases()[:2]
    alphas, psi0s, _ = inputs(ps, 600)
    b = make_batch(ps, alphas, psi0s)
    with pytest.raises(TdglError):
        b.instances[0].step(1)
    with pytest.raises(TdglError):
        b.instances[1].solve_psi()


def test_barrier_timeout_is_reported_and_context_survives():
    """Every barrier waits for one block that does not exist: each wait ends at
    its 30 ms bound, the launch returns, the error is sticky, and the context
    stays usable."""
    import torch
    from paper_1409_8340_gb300._lib import TDGL_ERR_TIMEOUT
    ps = batch_cases()[:2]
    alphas, psi0s, _ = inputs(ps, 700)
    b = make_batch(ps, alphas, psi0s)
    b.set_tuning(timeout_ms=30, test_extra_arrivals=1, graph_steps=0)
    b.step(2)
    rc, _ = b.status()
    assert rc == TDGL_ERR_TIMEOUT
    torch.cuda.synchronize()
    s = make_solver(dataclasses.replace(ps[0]), alphas[0], psi0s[0])
    s.step(1)
    assert np.isfinite(gpu_state(s)[0]).all()


def test_ensemble_64_full_size_sampled():
    """The 64-member ensemble of uneven sizes, as the benchmark runs it (default
    tuning, graph replay): 2 steps, then three members checked against plain
    handles started from the same state."""
    import torch
    from paper_1409_8340_gb300 import presets
    from paper_1409_8340_gb300.solver import Batch, pattern
    members = presets.ensemble_64()
    ps = [w.params for w in members]
    alphas = [pattern(w.params, w.candidates, w.target_sites, w.alpha_in, w.alpha_out)[0] for w in members]
    b = Batch(ps, alphas)
    psi0s = []
    for i, s in enumerate(b.instances):
        psi0 = I.random_psi(ps[i].nx, ps[i].ny, ps[i].nz, 900 + i).astype(np.complex64)
        psi0s.append(psi0)
        s.set_state(torch.as_tensor(psi0), None, 0.0)
    b.step(2)
    b.check()
    sizes = sorted({p.shape for p in ps})
    picks = [next(i for i, p in enumerate(ps) if p.shape == sz) for sz in sizes][:3]
    for i in picks:
        s = make_solver(dataclasses.replace(ps[i]), alphas[i].cpu().numpy(), psi0s[i])
        s.step(2)
        x, y = gpu_state(b.instances[i]), gpu_state(s)
        assert np.max(np.abs(x[0] - y[0])) <= 1e-6, i
        assert np.max(np.abs(x[1] - y[1])) <= 1e-6 * max(1.0, np.max(np.abs(y[1]))), i


def test_phase_log_accounts_for_the_launch():
    import torch
    ps = batch_cases()[:4]
    alphas, psi0s, mu0s = inputs(ps, 800)
    b = make_batch(ps, alphas, psi0s, mu0s)
    b.set_tuning(graph_steps=0)
    b.phase_log(True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b.step(1)
    e1.record()
    torch.cuda.synchronize()
    prof = b.phase_profile()
    total = sum(v[0] for v in prof.values())
    assert 0.3 * e0.elapsed_time(e1) <= total <= 1.05 * e0.elapsed_time(e1) + 0.05
    obs = b.observables()
    assert prof["init"][1] == 1
    assert prof["sweep"][1] == max(o["last_sweeps"] for o in obs) - 1
    assert prof["smooth"][1] > 0 and prof["shift"][1] == 1
