"""Pins of three oracle functions against something other than the oracle itself.

  * Free energy (reading of Sec. 2.1: trapezoid-weighted discrete F).  Its gradient
    must be the weighted residual of the stencil that the brute-force dense
    assembly pins: dF/d(psi*_m) = dV w_m (-alpha psi + beta |psi|^2 psi - Lap_U psi)_m,
    so that the scheme is a weighted gradient flow.  Central differences of F in
    Re psi_m and Im psi_m at random sites are compared with that expression, with
    Lap_U psi read from the oracle's own b at mu = 0: (b - psi)/(h_t/2) = alpha psi -
    beta |psi|^2 psi + Lap_U psi.  Every boundary combination, a film, anisotropy,
    a K phase on periodic x and insulating sites.  A wrong face or edge weight, a
    missing link or a wrong coefficient fails it.
  * Philox4x32-10 (Salmon et al., SC'11; the generator of the thermal noise of
    Sec. 3.1.2).  The oracle's C implementation is compared word for word with an
    independent implementation of the same published generator: the one in Triton's
    language library, run on the CPU by Triton's interpreter.  A wrong multiplier,
    Weyl constant, word order or round count fails it.
  * Vortex count (reading of the winding of xy plaquettes).  A state built from
    vortices and antivortices at known plaquette centres (zero field, open x and y)
    must give n_p = +-1 exactly at those plaquettes and 0 elsewhere: the unsigned
    count is the number of defects, the signed count their net charge.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1409_8340_gb300 import inputs as I

P, OP = 0, 1


def energy_cases(O):
    cs = []
    cs.append(("periodic", O.Grid(8, 6, 5, bc=(P, P, P), Bz=2 * np.pi * 2 / (4.0 * 3.0), ht=0.1), 0.0, None))
    cs.append(("openx_K0", O.Grid(9, 6, 5, bc=(OP, P, P), Bz=0.3, By=0.1, g=1.3), 0.0, None))
    cs.append(("allopen", O.Grid(7, 6, 5, bc=(OP, OP, OP), Bz=0.4, By=0.2), 0.0, None))
    cs.append(("periodicx_K", O.Grid(10, 6, 5, bc=(P, OP, OP), Bz=0.25), 0.7, None))
    cs.append(("film", O.Grid(9, 7, 1, bc=(OP, OP, P), Bz=0.35), 0.0, None))
    ins = (I.uniform(41, "pin.ins", 9 * 7 * 6).reshape(6, 7, 9) < 0.15).astype(np.uint8)
    cs.append(("insulating", O.Grid(9, 7, 6, bc=(OP, P, P), Bz=0.3, insulating=ins), 0.0, ins))
    return cs


@pytest.mark.parametrize("case", range(6))
def test_energy_gradient_is_the_weighted_stencil_residual(O, case):
    name, G, K, ins = energy_cases(O)[case]
    psi = I.random_psi(G.nx, G.ny, G.nz, 50 + case).astype(np.complex128)
    if ins is not None:
        psi[ins != 0] = 0.0
    alpha = (I.uniform(60 + case, "pin.alpha", G.N).reshape(G.shape) * 2.0 - 1.0)
    b, _ = O.init(G, psi, np.zeros(G.shape), alpha, K)
    lap_part = (b - psi) / (0.5 * G.ht)          # alpha psi - beta |psi|^2 psi + Lap_U psi
    dV = G.hx * G.hy * (G.hz if G.nz >= 2 else 1.0)
    w = O.site_weights(G)
    pred = -2.0 * dV * w * lap_part              # 2 dF/dpsi* = dF/dRe + i dF/dIm
    cond = G.conducting()
    rng = np.random.default_rng(70 + case)
    sites = [tuple(s) for s in np.argwhere(cond)]
    picks = [sites[q] for q in rng.choice(len(sites), size=min(24, len(sites)), replace=False)]
    d = 1e-5
    scale = np.max(np.abs(pred[cond]))
    for s in picks:
        fd = []
        for e in (1.0, 1j):
            pp, pm = psi.copy(), psi.copy()
            pp[s] += d * e
            pm[s] -= d * e
            fd.append((O.energy(G, pp, alpha, K) - O.energy(G, pm, alpha, K)) / (2 * d))
        got = fd[0] + 1j * fd[1]
        assert abs(got - pred[s]) <= 1e-7 * scale + 1e-8, (name, s, got, pred[s])


_TRITON_SCRIPT = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np
import torch
import triton
import triton.language as tl

@triton.jit
def kern(c_ptr, out_ptr, seed, N: tl.constexpr):
    q = tl.arange(0, N)
    c0 = tl.load(c_ptr + 4 * q)
    c1 = tl.load(c_ptr + 4 * q + 1)
    c2 = tl.load(c_ptr + 4 * q + 2)
    c3 = tl.load(c_ptr + 4 * q + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + 4 * q, a.to(tl.int32, bitcast=True))
    tl.store(out_ptr + 4 * q + 1, b.to(tl.int32, bitcast=True))
    tl.store(out_ptr + 4 * q + 2, c.to(tl.int32, bitcast=True))
    tl.store(out_ptr + 4 * q + 3, d.to(tl.int32, bitcast=True))

req = json.loads(sys.stdin.read())
res = []
for seed, ctrs in req:
    c = torch.tensor(np.array(ctrs, dtype=np.uint32).view(np.int32).reshape(-1))
    out = torch.zeros_like(c)
    kern[(1,)](c, out, seed, len(ctrs))
    res.append(out.numpy().view(np.uint32).reshape(-1, 4).tolist())
print(json.dumps(res))
"""


def test_philox_matches_an_independent_implementation(O):
    pytest.importorskip("triton")
    rng = np.random.default_rng(2024)
    edge = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 0, 0, 0], [0, 0, 0, 1], [0x12345678, 0x9ABCDEF0, 7, 0x80000000],
            [5, 0, 3, 0], [0xDEADBEEF, 0, 0xFFFFFFFF, 0x7FFFFFFF], [2, 2, 2, 2]]
    reqs = []
    for seed in (0, 1, 77, (1 << 40) + 5, 0x7FFFFFFFFFFFFFFF, int(rng.integers(0, 1 << 62))):
        ctrs = edge + rng.integers(0, 1 << 32, size=(8, 4), dtype=np.uint64).tolist()
        reqs.append((int(seed), [[int(v) for v in c] for c in ctrs]))
    env = dict(os.environ, TRITON_INTERPRET="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(reqs), capture_output=True,
                       text=True, env=env, timeout=600)
    if r.returncode != 0:
        pytest.skip(f"Triton interpreter unavailable: {r.stderr.strip().splitlines()[-1:]}")
    lib_out = json.loads(r.stdout.strip().splitlines()[-1])
    for (seed, ctrs), got in zip(reqs, lib_out):
        key = (seed & 0xFFFFFFFF, seed >> 32)
        for c, x in zip(ctrs, got):
            assert O.philox4x32_10(c, key) == [int(v) for v in x], (seed, c)


def vortex_state(nx, ny, nz, defects):
    """psi = prod_v ((x - X_v) + i s_v (y - Y_v)) / |...| on sites (i, j); defects at
    plaquette centres (X, Y, s)."""
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    z = np.ones((ny, nx), dtype=np.complex128)
    for X, Y, sgn in defects:
        f = (i - X) + 1j * sgn * (j - Y)
        z *= f / np.abs(f)
    return np.broadcast_to(z, (nz, ny, nx)).copy()


DEFECTS = [(5.5, 4.5, 1), (15.5, 12.5, -1), (8.5, 14.5, 1), (18.5, 5.5, 1), (3.5, 17.5, -1)]


@pytest.mark.parametrize("nz,bcz", [(3, P), (1, P), (4, OP)])
def test_vortex_count_of_known_defects(O, nz, bcz):
    G = O.Grid(24, 22, nz, bc=(OP, OP, bcz))
    psi = vortex_state(G.nx, G.ny, G.nz, DEFECTS)
    n, tot = O.winding(G, psi)
    expect = np.zeros(G.shape, dtype=np.int32)
    for X, Y, sgn in DEFECTS:
        expect[:, int(Y), int(X)] = sgn
    np.testing.assert_array_equal(n, expect)
    uns, sig = O.vortex_count(G, psi)
    assert uns == len(DEFECTS)
    assert sig == sum(s for _, _, s in DEFECTS)
