"""GPU parity of the scalar-potential solve, the pattern generator and the observables."""
import math

import numpy as np
import pytest

from _helpers import OP, P, gpu_state, inclusion_alpha, make_solver, oracle_grid, quantised
from paper_1409_8340_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def poisson_cases():
    from paper_1409_8340_gb300.solver import Params
    return [
        ("periodic_32", quantised(Params(32, 32, 32, bc=(P, P, P)), 4)),
        ("openx_128x128x64_J", Params(128, 128, 64, bc=(OP, P, P), Bz=0.1, Jext=0.01)),
        ("openx_45x24x10_J", Params(45, 24, 10, bc=(OP, P, P), Bz=0.3, Jext=0.02, g=1.4)),
        ("allopen_33x17x9", Params(33, 17, 9, bc=(OP, OP, OP), Bz=0.2)),
        ("film_64x48x1", Params(64, 48, 1, bc=(OP, P, P), Bz=0.2, Jext=0.01)),
        ("uneven_96x96x48", Params(96, 96, 48, bc=(OP, P, P), Bz=0.3, Jext=0.02)),
        # nx = 512: the finest level's lines are solved by the recursive (two-pass) exact solve
        ("recursive_openx_512x24x12_J", Params(512, 24, 12, bc=(OP, P, P), Bz=0.2, Jext=0.02)),
        ("recursive_periodic_512x16x16", quantised(Params(512, 16, 16, bc=(P, P, P)), 2)),
        ("recursive_allopen_512x17x9", Params(512, 17, 9, bc=(OP, OP, OP), Bz=0.25)),
        # nx = 512 with smoothed coarser levels (rho = 0.38, 0.61, ...): their lines are
        # solved by the exact scan over the lanes
        ("recursive_scan_openx_512x48x24_J", Params(512, 48, 24, bc=(OP, P, P), Bz=0.2, Jext=0.02)),
        ("recursive_scan_periodic_512x32x32", quantised(Params(512, 32, 32, bc=(P, P, P)), 2)),
        ("recursive_scan_allopen_512x33x17", Params(512, 33, 17, bc=(OP, OP, OP), Bz=0.25)),
        ("recursive_scan_openx_512x96x48_J", Params(512, 96, 48, bc=(OP, P, P), Bz=0.2, Jext=0.02)),
        # a film (no z neighbours): the finest level itself (rho = 0.27) takes the exact scan
        ("recursive_scan_film_512x256x1_J", Params(512, 256, 1, bc=(OP, P, P), Bz=0.2, Jext=0.02)),
        ("recursive_scan_film_periodic_512x256x1", quantised(Params(512, 256, 1, bc=(P, P, P)), 3)),
        # 1024-site lines: 32 sites per lane, the register-only recursive kernel
        ("recursive_openx_1024x24x12_J", Params(1024, 24, 12, bc=(OP, P, P), Bz=0.2, Jext=0.02)),
        ("recursive_periodic_1024x32x16", quantised(Params(1024, 32, 16, bc=(P, P, P)), 2)),
    ]


PC = poisson_cases()


@pytest.mark.parametrize("name,p", PC, ids=[c[0] for c in PC])
def test_poisson_matches_exact_solution(O, name, p):
    p.poisson_cycles = 1
    p.poisson_tol = 1e-6
    p.poisson_max_cycles = 40
    G = oracle_grid(O, p)
    psi = I.random_psi(p.nx, p.ny, p.nz, 51).astype(np.complex64).astype(np.complex128)
    s = make_solver(p, np.ones(p.shape, np.float32), psi)
    s.solve_mu()
    _, mu_g = gpu_state(s)
    _, _, f_g = s.internals()
    f_o = O.poisson_rhs(G, psi, 0.0)
    np.testing.assert_allclose(f_g.cpu().numpy(), f_o, rtol=0, atol=2e-5 * max(1.0, np.abs(f_o).max()))
    mu_o = O.poisson_solve(G, f_o)
    err = np.max(np.abs(mu_g - mu_o)) / max(1e-30, np.max(np.abs(mu_o)))
    assert err < 2e-4, err
    obs = s.observables()
    assert obs["poisson_res"] < 1e-4


@pytest.mark.parametrize("bcx", [OP, P])
def test_normal_state_ohmic(O, bcx):
    from paper_1409_8340_gb300.solver import Params
    J = 0.013
    p = Params(64, 16, 8, bc=(bcx, P, P), Jext=J, eps=1e-8, poisson_tol=1e-6)
    s = make_solver(p, -np.ones(p.shape, np.float32), np.zeros(p.shape, np.complex64))
    for _ in range(3):
        s.step(1)
        assert abs(s.observables()["Ex"] - J) < 1e-5 * J + 1e-9


def test_mg_converges_fast_from_cold(O):
    """Residual reduction per V-cycle on a 128x128x64 open-x problem (cold start)."""
    from paper_1409_8340_gb300.solver import Params
    psi = I.random_psi(128, 128, 64, 52)
    res = []
    for c in range(1, 6):
        p = Params(128, 128, 64, bc=(OP, P, P), Bz=0.1, Jext=0.01, poisson_cycles=c, poisson_max_cycles=c,
                   poisson_tol=1e-12)
        s = make_solver(p, np.ones(p.shape, np.float32), psi)
        s.solve_mu()
        res.append(s.observables()["poisson_res"])
        s.close()
    # at least a factor 4 per cycle until the FP32 floor
    for a, b in zip(res[:-1], res[1:]):
        assert b < max(a / 4.0, 3e-6), res


@pytest.mark.parametrize("bc,ny,nz", [((OP, P, P), 48, 24), ((OP, OP, OP), 33, 17), ((OP, P, P), 96, 48)])
def test_mg_scan_levels_converge_fast(O, bc, ny, nz):
    """512 x-sites with smoothed coarser levels, whose lines the exact scan over the
    lanes solves: the same reduction per V-cycle from a cold start."""
    from paper_1409_8340_gb300.solver import Params
    psi = I.random_psi(512, ny, nz, 53)
    res = []
    for c in range(1, 5):
        p = Params(512, ny, nz, bc=bc, Bz=0.2, Jext=0.01, poisson_cycles=c, poisson_max_cycles=c, poisson_tol=1e-12)
        s = make_solver(p, np.ones(p.shape, np.float32), psi)
        s.solve_mu()
        res.append(s.observables()["poisson_res"])
        s.close()
    for a, b in zip(res[:-1], res[1:]):
        assert b < max(a / 4.0, 3e-6), res


PAT = [
    ("spheres_periodic_32", (32, 32, 32), (P, P, P), "spheres", 10, 2.0, 2.0, 0.0, 1),
    ("spheres_openx_96x80x40", (96, 80, 40), (OP, P, P), "spheres", 300, 2.0, 4.0, 0.05, 2),
    ("ellipsoids_openx_100x60x36", (100, 60, 36), (OP, P, P), "ellipsoids", 3000, 1.5, 5.0, 0.10, 3),
    ("ellipsoids_allopen_41x33x17", (41, 33, 17), (OP, OP, OP), "ellipsoids", 500, 1.5, 5.0, 0.10, 4),
]


@pytest.mark.parametrize("name,shape,bc,kind,count,a0,a1,frac,seed", PAT, ids=[c[0] for c in PAT])
def test_pattern_bit_exact(O, name, shape, bc, kind, count, a0, a1, frac, seed):
    from paper_1409_8340_gb300.solver import Params, pattern
    p = Params(*shape, bc=bc)
    box = (p.length(0), p.length(1), p.length(2))
    cand = (I.spheres if kind == "spheres" else I.ellipsoids)(count, box, a0, a1, seed=seed)
    target = I.target_sites(frac, p.N)
    alpha_g, used_g, marked_g = pattern(p, cand, target, -1.0, 1.0)
    alpha_o, used_o, marked_o = O.pattern(oracle_grid(O, p), cand, target, -1.0, 1.0)
    assert used_g == used_o and marked_g == marked_o
    np.testing.assert_array_equal(alpha_g.cpu().numpy(), alpha_o.astype(np.float32))


def test_observables_match_oracle(O):
    from paper_1409_8340_gb300.solver import Params
    p = quantised(Params(48, 32, 16, bc=(P, P, P), Jext=0.02), 5)
    G = oracle_grid(O, p)
    alpha = inclusion_alpha(p, 61)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 62)
    s = make_solver(p, alpha, psi0)
    s.step(30)
    psi_g, mu_g = gpu_state(s)
    obs = s.observables()
    K = obs["K"]
    assert abs(obs["psi2_mean"] - np.mean(np.abs(psi_g) ** 2)) < 1e-6
    F_o = O.energy(G, psi_g, alpha.astype(np.float64), K)
    assert abs(obs["energy"] - F_o) <= 1e-5 * abs(F_o) + 1e-6
    n_o, tot_o = O.winding(G, psi_g, K)
    assert obs["vortex_signed"] * p.nz == pytest.approx(5 * p.nz)
    assert tot_o == 5 * p.nz
    assert abs(obs["vortex_unsigned"] - np.abs(n_o).sum() / p.nz) <= 0.01 * max(1.0, np.abs(n_o).sum() / p.nz)


@pytest.mark.parametrize("bc", [(OP, P, P), (OP, OP, OP), (P, P, P)])
def test_fused_mean_projection(O, bc):
    """With a fixed number of V-cycles on a 512-site line, the closing finest-level passes
    also sum the trapezoid-weighted mu; the projection then removes that mean.  A start
    shifted by a constant (which the V-cycles keep) must come out with zero weighted
    mean, on the direct path (first solve) and the graph-replayed one (later solves),
    and equal the exact solution."""
    import torch
    from paper_1409_8340_gb300.solver import Params
    ny, nz = (48, 24) if bc[1] == P else (33, 17)
    p = Params(512, ny, nz, bc=bc, Bz=0.2, Jext=0.02 if bc[0] == OP else 0.0, poisson_cycles=8)
    if bc == (P, P, P):
        p = quantised(p, 2)
    G = oracle_grid(O, p)
    w = O.site_weights(G)
    psi = I.random_psi(p.nx, p.ny, p.nz, 61).astype(np.complex64).astype(np.complex128)
    s = make_solver(p, np.ones(p.shape, np.float32), psi)
    mu0 = (I.uniform(62, "t.mu", p.N).reshape(p.shape) + 0.5).astype(np.float32)
    # the shift is applied in FP32: each site may keep half an ulp of the raw values
    bound = w.sum() * 0.5 * np.spacing(np.float32(2.0))
    for n in range(3):
        s.set_state(torch.as_tensor(psi.astype(np.complex64)), torch.as_tensor(mu0), 0.0)
        s.solve_mu()
        _, mu_g = gpu_state(s)
        assert abs((w * mu_g).sum()) <= bound + 1e-6 * (w * np.abs(mu_g)).sum(), n
        f = s.internals()[2].cpu().numpy().astype(np.float64)
        mu_o = O.poisson_solve(G, f)
        err = np.max(np.abs(mu_g - mu_o)) / max(1e-30, np.max(np.abs(mu_o)))
        assert err < 2e-4, (n, err)
