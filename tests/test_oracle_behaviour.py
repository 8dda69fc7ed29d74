"""Solver behaviour the paper reports (Sec. 4.1 and 4.3), checked on the oracle.

The numbers come from tests/golden/paper_solver_behaviour.json, which quotes
the paper's text.  A small quasi-2D box in flux flow stands in for the paper's
free-flowing vortex lattice.
"""
import copy
import json
import math
import os

import numpy as np

from paper_1409_8340_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_solver_behaviour.json")))


def flux_flow_state(O, h=0.5, steps=400):
    n = int(round(16 / h))
    G = O.Grid(n, n, 4, hx=h, hy=h, hz=0.5, bc=(0, 0, 0), Jext=0.03, ht=GOLD["ht"])
    G.Bz = 2 * math.pi * 6 / (G.length(0) * G.length(1))
    st = O.State(I.random_psi(n, n, 4, 5), np.zeros(G.shape))
    al = np.ones(G.shape)
    O.run(G, st, al, steps, eps=GOLD["eps"])
    return G, st, al


def test_sweeps_per_step_in_flux_flow(O):
    G, st, al = flux_flow_state(O, h=GOLD["h"])
    s = [O.step(G, st, al, eps=GOLD["eps"]) for _ in range(20)]
    lo, hi = GOLD["jacobi_sweeps_steady_flux_flow"]
    assert all(lo <= x.sweeps <= hi for x in s), [x.sweeps for x in s]
    assert s[-1].Ex > 0.0            # vortices flow: dissipation under current


def test_sweeps_grow_linearly_in_log_eps(O):
    G, st, al = flux_flow_state(O, h=GOLD["h"])
    counts = []
    for eps in (1e-4, 1e-6, 1e-8, 1e-10):
        st2 = copy.deepcopy(st)
        counts.append(O.step(G, st2, al, eps=eps).sweeps)
    d = np.diff(counts)
    assert np.all(d >= 2) and np.all(d <= 6), counts


def test_sweeps_grow_as_h_decreases(O):
    G1, st1, al1 = flux_flow_state(O, h=0.5, steps=200)
    G2, st2, al2 = flux_flow_state(O, h=0.25, steps=200)
    n1 = O.step(G1, st1, al1, eps=GOLD["eps"]).sweeps
    n2 = O.step(G2, st2, al2, eps=GOLD["eps"]).sweeps
    assert n2 > n1
