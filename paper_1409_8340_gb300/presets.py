"""Named workloads (parameters and synthetic-input recipes).

  periodic_cube_32        32^3, periodic, 4 flux quanta, 10 spheres r = 2 xi, no current
  transport_128x128x64    open x / periodic y,z, Bz = 0.1, spheres r ~ U[2,4] to 5 %, J = 0.01
  mesoscopic_512x512x256  open x / periodic y,z, Bz = 0.2, random ellipsoids U[1.5,5] to 10 %,
                          J stepped 0 .. 0.05 in 11 increments
  ensemble_64             64 instances drawn from {32^3, 64^3, 96x96x48, 128x128x64}
  adjoint_64x64x32        open x / periodic y,z, Bz = 0.1, J = 0.01, smoothed random alpha
All inputs are seeded and synthetic (no dataset exists for this solver).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import inputs
from .solver import OPEN, PERIODIC, Params


@dataclasses.dataclass
class Workload:
    name: str
    params: Params
    seed: int
    steps: int
    candidates: np.ndarray | None      # inclusion candidates (None: alpha given directly)
    target_sites: int
    alpha_in: float = -1.0
    alpha_out: float = 1.0
    alpha_field: np.ndarray | None = None


def periodic_cube_32() -> Workload:
    p = Params(32, 32, 32, bc=(PERIODIC, PERIODIC, PERIODIC), eps=1e-8, ht=0.1).quantise_Bz(4)
    cand = inputs.spheres(10, (p.length(0), p.length(1), p.length(2)), 2.0, 2.0, seed=1)
    return Workload("periodic_cube_32", p, 1, 100, cand, 0)


def transport_128x128x64() -> Workload:
    p = Params(128, 128, 64, bc=(OPEN, PERIODIC, PERIODIC), Bz=0.1, Jext=0.01, eps=1e-6, ht=0.1)
    cand = inputs.spheres(400, (p.length(0), p.length(1), p.length(2)), 2.0, 4.0, seed=2)
    return Workload("transport_128x128x64", p, 2, 2000, cand, inputs.target_sites(0.05, p.N))


def mesoscopic_512x512x256(J: float = 0.0) -> Workload:
    p = Params(512, 512, 256, bc=(OPEN, PERIODIC, PERIODIC), Bz=0.2, Jext=J, eps=1e-6, ht=0.1)
    cand = inputs.ellipsoids(20000, (p.length(0), p.length(1), p.length(2)), 1.5, 5.0, seed=3)
    return Workload("mesoscopic_512x512x256", p, 3, 500, cand, inputs.target_sites(0.10, p.N))


MESOSCOPIC_CURRENTS = tuple(0.005 * n for n in range(11))


def ensemble_member(m: inputs.EnsembleMember) -> Workload:
    nx, ny, nz = m.shape
    p = Params(nx, ny, nz, bc=(OPEN, PERIODIC, PERIODIC), Bz=m.Bz, Jext=m.Jext, eps=1e-6, ht=0.1)
    cand = inputs.spheres(800, (p.length(0), p.length(1), p.length(2)), 2.0, 4.0, seed=m.seed)
    return Workload(f"ensemble_member_{nx}x{ny}x{nz}", p, m.seed, 1000, cand, inputs.target_sites(m.fraction, p.N),
                    alpha_in=-m.alpha_scale, alpha_out=m.alpha_scale)


def ensemble_64(seed: int = 4) -> list[Workload]:
    return [ensemble_member(m) for m in inputs.ensemble(64, seed)]


def adjoint_64x64x32() -> Workload:
    p = Params(64, 64, 32, bc=(OPEN, PERIODIC, PERIODIC), Bz=0.1, Jext=0.01, eps=1e-6, ht=0.1, poisson_cycles=2)
    field = inputs.smoothed_field(64, 64, 32, seed=5, sigma_sites=4.0).astype(np.float32)
    return Workload("adjoint_64x64x32", p, 5, 400, None, 0, alpha_field=field)
