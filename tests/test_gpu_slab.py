"""The z-slab decomposition on the GPU: slab handles (the library's sweep, init and
right-hand-side kernels over each slab's planes between halo planes) and a
Poisson-only handle for the whole grid, driven by SlabStep in one process (the
ranks of a multi-GPU job emulated as consecutive slabs of one process, whose halo
planes are device copies).  Against one undivided handle on the same inputs: the
same sweep counts and E_x, psi within 1e-6 and mu within 1e-5 max(1, |mu|) at every
step (the per-site arithmetic is the same; the whole-grid Poisson solve sums the
right-hand side's mean in another order).
"""
import numpy as np
import pytest

from _helpers import OP, P, gpu_state, inclusion_alpha, make_solver
from paper_1409_8340_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def cases():
    from paper_1409_8340_gb300.solver import Params
    return [("64x24x12_3slabs", Params(64, 24, 12, bc=(OP, P, P), Bz=0.2, Jext=0.02), 3),
            ("512x32x16_2slabs", Params(512, 32, 16, bc=(OP, P, P), Bz=0.2, Jext=0.025), 2)]


@pytest.mark.parametrize("name,p,nslab", cases(), ids=[c[0] for c in cases()])
def test_slabs_match_the_undivided_handle(name, p, nslab):
    import torch
    from paper_1409_8340_gb300.slab import GpuPoisson, GpuSlab, LocalComm, SlabStep
    alpha = inclusion_alpha(p, 301)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 302).astype(np.complex64)
    ref = make_solver(p, alpha, psi0)
    n = p.nz // nslab
    slabs = []
    for q in range(nslab):
        idx = [(q * n - 1 + t) % p.nz for t in range(n + 2)]
        s = GpuSlab(p, q * n, n, torch.as_tensor(alpha[idx].copy()).cuda())
        s.set_state(torch.as_tensor(psi0[idx].copy()).cuda())
        slabs.append(s)
    stepper = SlabStep(slabs, LocalComm(), eps=p.eps, max_iter=p.max_iter, poisson=GpuPoisson(p))
    for step in range(5):
        sweeps, ex = stepper.step()
        ref.step(1)
        o = ref.observables()
        assert sweeps == o["last_sweeps"], (step, sweeps, o["last_sweeps"])
        assert abs(ex - o["Ex"]) <= 1e-5 * max(1e-3, abs(o["Ex"])), (step, ex, o["Ex"])
        psi_r, mu_r = gpu_state(ref)
        psi = np.concatenate([s.state()[0][1:-1].cpu().numpy() for s in slabs])
        mu = np.concatenate([s.state()[1][1:-1].cpu().numpy() for s in slabs])
        assert np.max(np.abs(psi - psi_r)) <= 1e-6, (step, np.max(np.abs(psi - psi_r)))
        assert np.max(np.abs(mu - mu_r)) <= 1e-5 * max(1.0, np.max(np.abs(mu_r))), step


def test_slab_and_poisson_handles_refuse_the_plain_calls():
    import ctypes

    import torch
    from paper_1409_8340_gb300 import _lib
    from paper_1409_8340_gb300.slab import GpuPoisson, GpuSlab
    p = cases()[0][1]
    s = GpuSlab(p, 0, 4, torch.ones((6, p.ny, p.nx), dtype=torch.float32, device="cuda"))
    L = _lib.load()
    assert L.tdgl_step(s._h, 1) == _lib.TDGL_ERR_INVALID_ARG
    assert L.tdgl_solve_psi(s._h, None) == _lib.TDGL_ERR_INVALID_ARG
    o = _lib.Obs()
    assert L.tdgl_observables(s._h, ctypes.byref(o)) == _lib.TDGL_ERR_INVALID_ARG
    g = GpuPoisson(p)
    assert L.tdgl_step(g._h, 1) == _lib.TDGL_ERR_INVALID_ARG
    assert L.tdgl_solve_mu(g._h) == _lib.TDGL_ERR_INVALID_ARG


@pytest.mark.parametrize("shape,bc", [((512, 32, 16), (OP, P, P)), ((64, 24, 12), (OP, OP, P)), ((48, 20, 10), (P, P, OP))],
                         ids=["512x32x16_openx", "64x24x12_openxy", "48x20x10_openz"])
def test_poisson_only_handle_matches_the_exact_solve(O, shape, bc):
    """The Poisson-only handle (tdgl_poisson_create, tdgl_solve_mu_f) on a right-hand side
    written by the caller, solved to a relative residual of 1e-6: mu within 2e-4 max|mu| of
    the oracle's exact discrete solution (Sec. 3.2), E_x within 1e-4 relative."""
    import torch
    from _helpers import oracle_grid
    from paper_1409_8340_gb300.slab import GpuPoisson
    from paper_1409_8340_gb300.solver import Params
    nx, ny, nz = shape
    p = Params(nx, ny, nz, bc=bc, Bz=0.0, Jext=0.0, poisson_tol=1e-6, poisson_max_cycles=40)
    G = oracle_grid(O, p)
    f = (I.uniform(311, "slab.f", p.N).reshape(p.shape) - 0.5) * 0.2
    f -= (O.site_weights(G) * f).sum() / O.site_weights(G).sum()      # compatible right-hand side
    solver = GpuPoisson(p)
    mu, ex = solver(torch.as_tensor(f.astype(np.float32)).cuda())
    mu = mu.cpu().numpy().astype(np.float64)
    mu_o = O.poisson_solve(G, f.astype(np.float32).astype(np.float64))
    assert np.max(np.abs(mu - mu_o)) <= 2e-4 * np.max(np.abs(mu_o)), np.max(np.abs(mu - mu_o))
    if bc[0] == OP:
        ex_o = O.voltage_open_x(G, mu_o)
        assert abs(ex - ex_o) <= 1e-4 * max(abs(ex_o), 1e-3), (ex, ex_o)
