"""The allocation-free sweep (tdgl_sweep_noalloc) against the handle path.

tdgl_sweep_noalloc serves callers that cannot call cudaMalloc (a host
application whose memory manager owns the device heap, a real-time loop that
must not allocate once running): its scratch is a static device array.  Here it
is called twice in a row through the C ABI, each call fed with the previous
output, and compared with the 2nd and 3rd sweeps of tdgl_solve_psi on the same
input, within the tolerance of the other GPU tests.  This file is collected
last so that a run stopping at the first failure has run everything else.
"""
import ctypes
import dataclasses
import math

import numpy as np
import pytest

from _helpers import OP, P, gpu_state, inclusion_alpha, make_solver
from paper_1409_8340_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_PSI = 2e-5


def cases():
    from paper_1409_8340_gb300.solver import Params
    p1 = Params(48, 20, 12, bc=(OP, P, P), Bz=0.2, By=0.05, Jext=0.01, g=1.2)
    p2 = Params(40, 24, 10, bc=(P, P, P))
    p2.Bz = 2 * math.pi * 3 / (p2.length(0) * p2.length(1))
    p2.By = 2 * math.pi * 1 / (p2.length(0) * p2.length(2))
    return [("openx_48x20x12", p1, 0.0), ("periodic_40x24x10", p2, 0.37)]


@pytest.mark.parametrize("name,p,K", cases(), ids=[c[0] for c in cases()])
def test_noalloc_sweep_matches_handle_path(name, p, K):
    import torch
    from paper_1409_8340_gb300 import _lib
    L = _lib.load()
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
    cfg = p.to_c(0)
    stream = torch.cuda.current_stream().cuda_stream
    cur = ref[1][0]
    for n in (2, 3):
        out = torch.empty_like(cur)
        r2 = ctypes.c_double(-1.0)
        rc = L.tdgl_sweep_noalloc(ctypes.byref(cfg), ctypes.c_void_p(cur.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                  ctypes.c_void_p(D.data_ptr()), K, ctypes.c_void_p(out.data_ptr()),
                                  ctypes.byref(r2), ctypes.c_void_p(stream))
        assert rc == 0
        err = (out - ref[n][0]).abs().max().item()
        assert err <= TOL_PSI, (n, err)
        assert abs(r2.value - ref[n][1]) <= 1e-6 * max(1.0, ref[n][1])
        cur = out


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
