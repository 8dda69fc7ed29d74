"""Seeded synthetic inputs for the TDGL solver (shared by tests, bench and users).

This module only draws random numbers and shapes them into *inputs*: initial
order parameters, candidate inclusion lists, gauge angles, a smoothed random
pinning field and ensemble descriptors.  It contains none of the solver's
arithmetic (no stencil, no link variables, no inside test, no Poisson solve),
so the FP64 oracle and the CUDA path can both consume it without sharing code.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), re-implemented here with numpy
uint64 arithmetic.  Every purpose gets its own stream, keyed by (seed, tag).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _tag_hash(tag: str) -> int:
    # FNV-1a over the tag bytes, used only to separate streams.
    h = 0xCBF29CE484222325
    for ch in tag.encode():
        h ^= ch
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def splitmix64(seed: int, tag: str, count: int) -> np.ndarray:
    """Return `count` uint64 outputs of the SplitMix64 stream keyed by (seed, tag)."""
    with np.errstate(over="ignore"):
        base = _mix(np.array([(seed ^ _tag_hash(tag)) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        idx = np.arange(1, count + 1, dtype=np.uint64)
        state = base + idx * _GAMMA
        return _mix(state)


def uniform(seed: int, tag: str, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits each."""
    bits = splitmix64(seed, tag, count) >> np.uint64(11)
    return bits.astype(np.float64) * (1.0 / 9007199254740992.0)


# --------------------------------------------------------------------------
# Initial order parameter: |psi| ~ U[0,1], arg psi ~ U[0, 2pi), per site.
# --------------------------------------------------------------------------
def random_psi(nx: int, ny: int, nz: int, seed: int) -> np.ndarray:
    """complex128 array of shape (nz, ny, nx) (x fastest in memory)."""
    n = nx * ny * nz
    amp = uniform(seed, "psi0.amp", n)
    ph = uniform(seed, "psi0.phase", n) * (2.0 * math.pi)
    return (amp * np.exp(1j * ph)).reshape(nz, ny, nx)


# --------------------------------------------------------------------------
# Candidate inclusion lists.  Each row: cx, cy, cz, a, b, c, q0, q1, q2, q3
# (centre in units of xi, semi-axes, unit quaternion of the body rotation).
# The pattern generator consumes the rows in order.
# --------------------------------------------------------------------------
INCLUSION_FIELDS = 10


def _shoemake_quaternions(u1, u2, u3):
    """Uniformly random unit quaternions from three uniforms (Shoemake, Graphics Gems III, 1992)."""
    s1 = np.sqrt(1.0 - u1)
    s2 = np.sqrt(u1)
    t1 = 2.0 * math.pi * u2
    t2 = 2.0 * math.pi * u3
    return np.stack([s2 * np.cos(t2), s1 * np.sin(t1), s1 * np.cos(t1), s2 * np.sin(t2)], axis=1)


def spheres(count: int, box: tuple[float, float, float], rmin: float, rmax: float,
            seed: int, tag: str = "spheres") -> np.ndarray:
    """`count` spheres, centres uniform in [0,Lx)x[0,Ly)x[0,Lz), radius U[rmin, rmax]."""
    u = uniform(seed, tag, 4 * count).reshape(count, 4)
    out = np.zeros((count, INCLUSION_FIELDS), dtype=np.float64)
    out[:, 0] = u[:, 0] * box[0]
    out[:, 1] = u[:, 1] * box[1]
    out[:, 2] = u[:, 2] * box[2]
    r = rmin + (rmax - rmin) * u[:, 3]
    out[:, 3] = r
    out[:, 4] = r
    out[:, 5] = r
    out[:, 6] = 1.0  # identity rotation
    return out


def ellipsoids(count: int, box: tuple[float, float, float], amin: float, amax: float,
               seed: int, tag: str = "ellipsoids") -> np.ndarray:
    """`count` ellipsoids, semi-axes each U[amin, amax], uniformly random orientation."""
    u = uniform(seed, tag, 9 * count).reshape(count, 9)
    out = np.zeros((count, INCLUSION_FIELDS), dtype=np.float64)
    out[:, 0] = u[:, 0] * box[0]
    out[:, 1] = u[:, 1] * box[1]
    out[:, 2] = u[:, 2] * box[2]
    out[:, 3:6] = amin + (amax - amin) * u[:, 3:6]
    out[:, 6:10] = _shoemake_quaternions(u[:, 6], u[:, 7], u[:, 8])
    return out


def target_sites(fraction: float, n_sites: int) -> int:
    """Number of inside sites a volume-fraction target asks for (ceil(f*N))."""
    return int(math.ceil(fraction * n_sites - 1e-9)) if fraction > 0 else 0


# --------------------------------------------------------------------------
# Random lattice gauge angles chi_m ~ U[0, 2pi).
# --------------------------------------------------------------------------
def gauge_angles(nx: int, ny: int, nz: int, seed: int) -> np.ndarray:
    return (uniform(seed, "gauge.chi", nx * ny * nz) * (2.0 * math.pi)).reshape(nz, ny, nx)


# --------------------------------------------------------------------------
# Smoothed random pinning field in [-1, 1]: iid U[-1,1] per site, separable
# Gaussian smoothing (periodic along y,z, mirror-reflected along x), affine
# rescale so that min -> -1 and max -> +1.
# --------------------------------------------------------------------------
def _smooth_axis(a: np.ndarray, axis: int, sigma_sites: float, periodic: bool) -> np.ndarray:
    n = a.shape[axis]
    rad = int(math.ceil(3.0 * sigma_sites))
    offs = np.arange(-rad, rad + 1)
    w = np.exp(-0.5 * (offs / sigma_sites) ** 2)
    w /= w.sum()
    out = np.zeros_like(a)
    idx = np.arange(n)
    for o, wo in zip(offs, w):
        src = idx + o
        if periodic:
            src = src % n
        else:  # reflect about the end points (..., 2, 1, 0, 1, 2, ...)
            period = 2 * (n - 1) if n > 1 else 1
            src = np.abs(src) % period
            src = np.where(src > n - 1, period - src, src)
        out += wo * np.take(a, src, axis=axis)
    return out


def smoothed_field(nx: int, ny: int, nz: int, seed: int, sigma_sites: float = 4.0,
                   periodic=(False, True, True)) -> np.ndarray:
    raw = uniform(seed, "alpha.field", nx * ny * nz).reshape(nz, ny, nx) * 2.0 - 1.0
    a = _smooth_axis(raw, 2, sigma_sites, periodic[0])
    a = _smooth_axis(a, 1, sigma_sites, periodic[1])
    a = _smooth_axis(a, 0, sigma_sites, periodic[2])
    lo, hi = a.min(), a.max()
    return (2.0 * (a - lo) / (hi - lo) - 1.0)


# --------------------------------------------------------------------------
# Ensemble descriptors (64 instances of uneven sizes).
# --------------------------------------------------------------------------
ENSEMBLE_SIZES = ((32, 32, 32), (64, 64, 64), (96, 96, 48), (128, 128, 64))


@dataclasses.dataclass
class EnsembleMember:
    shape: tuple[int, int, int]
    seed: int
    Bz: float
    alpha_scale: float
    Jext: float
    fraction: float


def ensemble(count: int, seed: int) -> list[EnsembleMember]:
    u = uniform(seed, "ensemble", 5 * count).reshape(count, 5)
    members = []
    for n in range(count):
        shape = ENSEMBLE_SIZES[min(int(u[n, 0] * len(ENSEMBLE_SIZES)), len(ENSEMBLE_SIZES) - 1)]
        members.append(EnsembleMember(
            shape=shape,
            seed=seed * 1000 + n,
            Bz=0.05 + 0.45 * u[n, 1],
            alpha_scale=0.5 + 0.5 * u[n, 2],
            Jext=0.03 * u[n, 3],
            fraction=0.03 + 0.05 * u[n, 4],
        ))
    return members
