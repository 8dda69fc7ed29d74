"""tdgl_autotune on a single handle: every candidate sweep (staged, register-tiled, two
sweeps per pass) runs trial steps from the current state, which is restored after each;
the handle keeps the fastest.

Checks: the state after the call is the state before it, bit for bit (psi, mu, K, the
step and noise counters); the candidates the grid supports were timed; and the run then
continues exactly as a handle created with the chosen sweep and loaded from a checkpoint
taken before the call.
"""
import numpy as np
import pytest

from _helpers import OP, P, gpu_state, inclusion_alpha, make_solver
from paper_1409_8340_gb300 import inputs as I

pytestmark = pytest.mark.gpu

KERNEL = {"staged": (2, 1), "register_tiled": (1, 1), "two_sweeps_per_pass": (0, 2)}


def cases():
    from paper_1409_8340_gb300.solver import Params
    return {
        "openx_128x64x32": (Params(128, 64, 32, bc=(OP, P, P), Bz=0.2, Jext=0.02), 3),
        "noise_64x32x16": (Params(64, 32, 16, bc=(OP, P, P), Bz=0.2, Jext=0.02, noise_T=0.02, noise_seed=3), 3),
        "xz_gauge_64x32x16": (Params(64, 32, 16, bc=(OP, P, OP), Bz=0.2, Bx=0.15, xz_gauge=True, Jext=0.01), 2),
    }


@pytest.mark.parametrize("name", list(cases()))
def test_autotune_keeps_the_state_and_continues_as_the_chosen_sweep(name):
    import dataclasses
    p, n_cand = cases()[name]
    alpha = inclusion_alpha(p, 71)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 72).astype(np.complex64)
    a = make_solver(p, alpha, psi0)
    a.step(3)
    ck = a.checkpoint()
    before = gpu_state(a)
    o_before = a.observables()
    rep = a.autotune(2)
    assert rep["candidates"] == n_cand and len(rep["ms_per_step"]) == n_cand, rep
    assert rep["chosen"] in rep["ms_per_step"]
    after = gpu_state(a)
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    o_after = a.observables()
    for k in ("step", "K", "Ex", "last_sweeps"):
        assert o_after[k] == o_before[k], (k, o_before[k], o_after[k])
    kernel, spp = KERNEL[rep["chosen"]]
    b = make_solver(dataclasses.replace(p, sweep_kernel=kernel, sweeps_per_pass=spp), alpha)
    b.restore(ck)
    a.step(4)
    b.step(4)
    (pa, ma), (pb, mb) = gpu_state(a), gpu_state(b)
    assert np.array_equal(pa, pb) and np.array_equal(ma, mb)
    assert a.observables()["step"] == b.observables()["step"] == o_before["step"] + 4
