"""Long runs: FP32 GPU against the FP64 oracle on time-averaged observables.

Over a long run the two trajectories separate by rounding, so they are
compared on time averages over the second half of the run: <|psi|^2>, the
vortex count per layer and the voltage E_x, each within 1 % (E_x with an
absolute floor of 1e-4 J when the state is pinned), as the method's
statistical parity requires.
"""
import numpy as np
import pytest

from _helpers import OP, P, oracle_grid, quantised
from paper_1409_8340_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def run_both(O, p, alpha, psi0, steps):
    import torch
    from paper_1409_8340_gb300.solver import Solver
    G = oracle_grid(O, p)
    st = O.State(psi0.astype(np.complex128), np.zeros(p.shape))
    s = Solver(p, torch.as_tensor(alpha).cuda())
    s.set_state(torch.as_tensor(psi0.astype(np.complex64)))
    rec_o, rec_g = [], []
    for n in range(steps):
        so = O.step(G, st, alpha.astype(np.float64), eps=p.eps)
        s.step(1)
        if n >= steps // 2:
            rec_o.append((float(np.mean(np.abs(st.psi) ** 2)), O.vortex_count(G, st.psi, st.K)[0], so.Ex))
            o = s.observables()
            rec_g.append((o["psi2_mean"], o["vortex_unsigned"], o["Ex"]))
    return np.mean(rec_o, axis=0), np.mean(rec_g, axis=0)


def test_periodic_cube_32_long_run(O):
    """The 32^3 periodic cube: 4 flux quanta, 10 spheres r = 2, eps = 1e-8, 300 steps."""
    from paper_1409_8340_gb300 import presets
    from paper_1409_8340_gb300.solver import pattern
    w = presets.periodic_cube_32()
    p = w.params
    p.poisson_tol = 1e-6
    alpha = pattern(p, w.candidates, w.target_sites, w.alpha_in, w.alpha_out)[0].cpu().numpy()
    psi0 = I.random_psi(p.nx, p.ny, p.nz, w.seed)
    avg_o, avg_g = run_both(O, p, alpha, psi0, 300)
    assert abs(avg_g[0] - avg_o[0]) <= 0.01 * abs(avg_o[0]), (avg_g, avg_o)
    assert abs(avg_g[1] - avg_o[1]) <= 0.01 * max(abs(avg_o[1]), 1.0), (avg_g, avg_o)
    assert abs(avg_g[2] - avg_o[2]) <= 1e-6, (avg_g, avg_o)


def test_transport_flux_flow_long_run(O):
    """Open x with injected current and a vortex lattice driven across a sample
    with sparse inclusions: 400 steps."""
    from paper_1409_8340_gb300.solver import Params
    p = Params(64, 32, 16, bc=(OP, P, P), Bz=0.4, Jext=0.04, eps=1e-6, poisson_tol=1e-6)
    u = I.uniform(31, "long.alpha", p.N).reshape(p.shape)
    alpha = np.where(u < 0.02, -1.0, 1.0).astype(np.float32)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 32)
    avg_o, avg_g = run_both(O, p, alpha, psi0, 400)
    assert abs(avg_g[0] - avg_o[0]) <= 0.01 * abs(avg_o[0]), (avg_g, avg_o)
    assert abs(avg_g[1] - avg_o[1]) <= 0.01 * max(abs(avg_o[1]), 1.0), (avg_g, avg_o)
    assert abs(avg_g[2] - avg_o[2]) <= max(0.01 * abs(avg_o[2]), 1e-4 * p.Jext), (avg_g, avg_o)
