"""The allocation-free sweep (tdgl_sweep_noalloc) against the oracle and the handle path.

tdgl_sweep_noalloc serves callers that cannot call cudaMalloc (a host
application whose memory manager owns the device heap, a real-time loop that
must not allocate once running): its scratch is a static device array.  Here it
is called twice in a row through the C ABI, each call fed with the previous
output, and each output is compared with the oracle's sweep (Eq. final) of the
same input, b and diag M, and with the 2nd and 3rd sweeps of tdgl_solve_psi on
the same start, within the tolerances of the other GPU tests.  The cases cover
open, periodic and all-open boxes, a film (nz = 1) and an odd nx (the per-site
kernel).  This file is collected last so that a run stopping at the first failure
has run everything else.
"""
import ctypes
import dataclasses
import math

import numpy as np
import pytest

from _helpers import OP, P, inclusion_alpha, make_solver, oracle_grid
from paper_1409_8340_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_PSI = 2e-5        # against the handle path (the parity tolerance of the step)
TOL_ORACLE = 3e-6     # one FP32 sweep against the FP64 oracle on the same inputs


def cases():
    from paper_1409_8340_gb300.solver import Params
    p1 = Params(48, 20, 12, bc=(OP, P, P), Bz=0.2, By=0.05, Jext=0.01, g=1.2)
    p2 = Params(40, 24, 10, bc=(P, P, P))
    p2.Bz = 2 * math.pi * 3 / (p2.length(0) * p2.length(1))
    p2.By = 2 * math.pi * 1 / (p2.length(0) * p2.length(2))
    p3 = Params(36, 18, 10, bc=(OP, OP, OP), Bz=0.3, By=0.1)
    p4 = Params(44, 20, 1, bc=(OP, P, P), Bz=0.25, Jext=0.02)
    p5 = Params(33, 20, 12, bc=(OP, P, P), Bz=0.2, Jext=0.01)
    return [("openx_48x20x12", p1, 0.0), ("periodic_40x24x10", p2, 0.37), ("allopen_36x18x10", p3, 0.0),
            ("film_44x20x1", p4, 0.0), ("oddnx_33x20x12", p5, 0.0)]


def noalloc_sweep(L, p, cur, b, D, K, stream):
    import torch
    cfg = p.to_c(0)
    out = torch.empty_like(cur)
    r2 = ctypes.c_double(-1.0)
    rc = L.tdgl_sweep_noalloc(ctypes.byref(cfg), ctypes.c_void_p(cur.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                              ctypes.c_void_p(D.data_ptr()), K, ctypes.c_void_p(out.data_ptr()),
                              ctypes.byref(r2), ctypes.c_void_p(stream))
    return rc, out, r2.value


@pytest.mark.parametrize("name,p,K", cases(), ids=[c[0] for c in cases()])
def test_noalloc_sweep_matches_oracle_and_handle_path(O, name, p, K):
    import torch
    from paper_1409_8340_gb300 import _lib
    L = _lib.load()
    G = oracle_grid(O, p)
    psi0 = I.random_psi(p.nx, p.ny, p.nz, 201)
    mu0 = (I.uniform(202, "t.mu", p.N).reshape(p.shape) - 0.5) * 0.2
    alpha = inclusion_alpha(p, 203)
    ref = {}
    for n in (1, 2, 3):
        s = make_solver(dataclasses.replace(p, fixed_sweeps=n), alpha, psi0, mu0, K)
        s.solve_psi()
        psi_n, _ = s.state()
        ref[n] = (psi_n.clone(), s.observables()["last_r2"])
        if n == 1:
            b, D, _ = s.internals()
            b, D = b.clone(), D.clone()
        s.close()
    b_o, D_o = b.cpu().numpy().astype(np.complex128), D.cpu().numpy().astype(np.complex128)
    stream = torch.cuda.current_stream().cuda_stream
    cur = ref[1][0]
    for n in (2, 3):
        rc, out, r2 = noalloc_sweep(L, p, cur, b, D, K, stream)
        assert rc == 0
        nxt_o, r2_o = O.sweep(G, cur.cpu().numpy().astype(np.complex128), b_o, D_o, K)
        err_o = np.max(np.abs(out.cpu().numpy() - nxt_o))
        assert err_o <= TOL_ORACLE, (n, err_o)
        assert abs(r2 - r2_o) <= 1e-5 * max(1.0, r2_o), (n, r2, r2_o)
        err = (out - ref[n][0]).abs().max().item()
        assert err <= TOL_PSI, (n, err)
        assert abs(r2 - ref[n][1]) <= 1e-6 * max(1.0, ref[n][1])
        cur = out


def test_noalloc_reports_a_nonfinite_residual():
    import torch
    from paper_1409_8340_gb300 import _lib
    from paper_1409_8340_gb300.solver import Params
    L = _lib.load()
    p = Params(48, 20, 12, bc=(OP, P, P), Bz=0.2)
    psi = I.random_psi(p.nx, p.ny, p.nz, 211).astype(np.complex64)
    psi[4, 7, 9] = np.nan
    cur = torch.as_tensor(psi).cuda()
    b = torch.as_tensor(I.random_psi(p.nx, p.ny, p.nz, 212).astype(np.complex64)).cuda()
    D = torch.full(p.shape, 2.0 + 0.1j, dtype=torch.complex64, device="cuda")
    rc, _, _ = noalloc_sweep(L, p, cur, b, D, 0.0, torch.cuda.current_stream().cuda_stream)
    assert rc == _lib.TDGL_ERR_NONFINITE


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_1409_8340_gb300 import _lib
    from paper_1409_8340_gb300.solver import Params
    L = _lib.load()
    p = Params(5000, 4, 4, bc=(OP, P, P))
    cfg = p.to_c(0)
    r2 = ctypes.c_double()
    rc = L.tdgl_sweep_noalloc(ctypes.byref(cfg), ctypes.c_void_p(256), ctypes.c_void_p(512), ctypes.c_void_p(768), 0.0,
                              ctypes.c_void_p(1024), ctypes.byref(r2), None)
    assert rc == -6
