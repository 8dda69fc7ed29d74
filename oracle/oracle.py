"""FP64 CPU oracle of the implicit TDGL step (arXiv:1409.8340).

TEST INFRASTRUCTURE ONLY: imported by `tests/`, by `__graft_entry__.smoke()`
and by the CPU-baseline leg of `bench.py`.  The CUDA library never imports,
links or calls anything here.

Per-site arithmetic lives in `tdgl_oracle.c` (plain C, double precision);
this module adds the time-step driver in the paper's order (Sec. 3: psi, then
K, then mu), the exact discrete Poisson solve, and observables.

Where the paper is silent the readings used here are:
  * u is absorbed in h_t (footnote of Eq. GL_numCN); the K ODE advances by u*h_t.
  * Jacobi starts from psi^- and the convergence test of Eq. convergence uses
    the residual of the sweep's input iterate; the iterate returned is the
    output of the sweep whose input passed.  `check_every = k` evaluates the
    test only after every k-th sweep (k = 1 is the paper).
  * K is integrated by explicit Euler with J_av of the new psi and the old K,
    then rewound (Sec. 2.2, the floor rule).
  * The scalar potential is the exact discrete solution of Lap mu = f with
    zero weighted mean (the fixed point of the paper's pseudo-time relaxation,
    Sec. 3.2); it is computed here by diagonalising the separable discrete
    Laplacian (FFT along periodic axes, DCT-I along open axes).
  * Open x carries the applied current as normal current injected through the
    faces: Neumann ghosts mu_{-1} = mu_1 + 2 hx J, mu_Nx = mu_{Nx-2} - 2 hx J,
    K = 0, and E_x = (<mu>_{i=0} - <mu>_{i=Nx-1}) / ((Nx-1) hx).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import sys

import numpy as np
import scipy.fft as sfft

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libtdgl_oracle.so")
SRC_PATH = os.path.join(HERE, "tdgl_oracle.c")

PERIODIC = 0
OPEN = 1


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, FP64, no FMA contraction)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC_PATH):
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", LIB_PATH, SRC_PATH, "-lm"]
        subprocess.run(cmd, check=True)
    return LIB_PATH


class _Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("bc", ctypes.c_int32 * 3), ("h", ctypes.c_double * 3),
                ("g", ctypes.c_double), ("u", ctypes.c_double), ("beta", ctypes.c_double),
                ("ht", ctypes.c_double), ("By", ctypes.c_double), ("Bz", ctypes.c_double),
                ("Jext", ctypes.c_double), ("ins", ctypes.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        d = ctypes.c_double
        dp = P(ctypes.c_double)
        gp = P(_Grid)
        L.or_landau_link_phases.argtypes = [gp, dp]
        L.or_init.argtypes = [gp, dp, d, dp, dp, dp, dp, dp]
        L.or_xz_link_phases.argtypes = [gp, d, dp]
        u32p = P(ctypes.c_uint32)
        L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.or_noise.argtypes = [gp, d, ctypes.c_uint64, ctypes.c_int64, dp]
        L.or_sweep.argtypes = [gp, dp, d, dp, dp, dp, dp]
        L.or_sweep.restype = d
        L.or_residual.argtypes = [gp, dp, d, dp, dp, dp, dp]
        L.or_javg.argtypes = [gp, dp, d, dp]
        L.or_javg.restype = d
        L.or_poisson_rhs.argtypes = [gp, dp, d, dp, dp]
        L.or_laplacian_mu.argtypes = [gp, dp, dp]
        L.or_energy.argtypes = [gp, dp, d, dp, dp]
        L.or_energy.restype = d
        L.or_winding.argtypes = [gp, dp, d, dp, P(ctypes.c_int32)]
        L.or_winding.restype = ctypes.c_int64
        L.or_pattern.argtypes = [gp, dp, ctypes.c_int64, ctypes.c_int64, d, d, dp, P(ctypes.c_int64)]
        L.or_pattern.restype = ctypes.c_int64
        L.or_inside_q.argtypes = [gp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.or_inside_q.restype = d
        L.or_threads.restype = ctypes.c_int
        L.or_set_threads.argtypes = [ctypes.c_int]
        L.or_set_threads.restype = ctypes.c_int
        i64 = ctypes.c_int64
        L.or_shape_contains.argtypes = [gp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.or_shape_contains.restype = ctypes.c_int
        L.or_lattice_shapes.argtypes = [dp, dp]
        L.or_lattice_shapes.restype = i64
        L.or_voronoi_owner.argtypes = [gp, dp, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.or_voronoi_owner.restype = i64
        L.or_pattern_ex.argtypes = [gp, dp, i64, i64, ctypes.c_int, ctypes.c_int, d, dp, dp, d, ctypes.c_uint64,
                                    dp, i64, dp, P(ctypes.c_uint8), P(i64)]
        L.or_pattern_ex.restype = i64
        _lib = L
    return _lib


@dataclasses.dataclass
class Grid:
    """Grid, boundary conditions and physical parameters (Sec. 2-3)."""
    nx: int
    ny: int
    nz: int
    hx: float = 0.5
    hy: float = 0.5
    hz: float = 0.5
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC)
    g: float = 1.0
    u: float = 1.0
    beta: float = 1.0
    ht: float = 0.1
    By: float = 0.0
    Bz: float = 0.0
    Jext: float = 0.0
    noise_T: float = 0.0          # grid-independent noise parameter T_zeta (Sec. 3.1.2); 0: no noise
    noise_seed: int = 0
    insulating: object = None     # u8 array of the grid's shape: insulating sites (Sec. 3.4 (ii)); None: none

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def N(self):
        return self.nx * self.ny * self.nz

    def c(self):
        g = _Grid()
        g.n[:] = [self.nx, self.ny, self.nz]
        g.bc[:] = list(self.bc)
        g.h[:] = [self.hx, self.hy, self.hz]
        g.g, g.u, g.beta, g.ht = self.g, self.u, self.beta, self.ht
        g.By, g.Bz, g.Jext = self.By, self.Bz, self.Jext
        if self.insulating is not None:
            self._ins = np.ascontiguousarray(self.insulating, dtype=np.uint8).reshape(self.shape)
            g.ins = self._ins.ctypes.data
        return g

    def conducting(self):
        return np.ones(self.shape, dtype=bool) if self.insulating is None else \
            (np.asarray(self.insulating).reshape(self.shape) == 0)

    def length(self, ax):
        n = (self.nx, self.ny, self.nz)[ax]
        h = (self.hx, self.hy, self.hz)[ax]
        return n * h if self.bc[ax] == PERIODIC else (n - 1) * h


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _cplx(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


def _theta_ptr(theta):
    if theta is None:
        return None
    return _dp(theta)


# --------------------------------------------------------------------------
# Elementary operations (thin wrappers over the C routines)
# --------------------------------------------------------------------------
def threads() -> int:
    """OpenMP threads used by the C loops."""
    return int(lib().or_threads())


def set_threads(n: int) -> int:
    """Run the C loops on n OpenMP threads; returns the count now in use."""
    return int(lib().or_set_threads(int(n)))


def landau_link_phases(G: Grid) -> np.ndarray:
    th = np.zeros((3,) + G.shape, dtype=np.float64)
    lib().or_landau_link_phases(ctypes.byref(G.c()), _dp(th))
    return th


def xz_link_phases(G: Grid, Bx: float) -> np.ndarray:
    """Link phases of the Landau gauge of Eq. A_xz (field (Bx, 0, Bz)), quasi-periodic in y."""
    th = np.zeros((3,) + G.shape, dtype=np.float64)
    lib().or_xz_link_phases(ctypes.byref(G.c()), float(Bx), _dp(th))
    return th


def init(G: Grid, psi_prev, mu, alpha, K=0.0, theta=None):
    """b and diag(M) of Sec. 3.1 (Eq. b and the matrix M)."""
    psi_prev = _cplx(psi_prev)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.empty(G.shape, dtype=np.complex128)
    D = np.empty(G.shape, dtype=np.complex128)
    lib().or_init(ctypes.byref(G.c()), _theta_ptr(theta), K, _dp(psi_prev), _dp(mu), _dp(alpha), _dp(b), _dp(D))
    return b, D


def sweep(G: Grid, psi, b, D, K=0.0, theta=None):
    """One Jacobi sweep (Eq. final); returns (psi_next, max|r|^2 of psi)."""
    psi = _cplx(psi)
    out = np.empty(G.shape, dtype=np.complex128)
    r2 = lib().or_sweep(ctypes.byref(G.c()), _theta_ptr(theta), K, _dp(psi), _dp(_cplx(b)), _dp(_cplx(D)), _dp(out))
    return out, r2


def residual(G: Grid, psi, b, D, K=0.0, theta=None):
    out = np.empty(G.shape, dtype=np.complex128)
    lib().or_residual(ctypes.byref(G.c()), _theta_ptr(theta), K, _dp(_cplx(psi)), _dp(_cplx(b)), _dp(_cplx(D)), _dp(out))
    return out


def javg(G: Grid, psi, K=0.0, theta=None) -> float:
    return lib().or_javg(ctypes.byref(G.c()), _theta_ptr(theta), K, _dp(_cplx(psi)))


def poisson_rhs(G: Grid, psi, K=0.0, theta=None):
    """f = div Im[psi*(grad - iA)psi] (Sec. 3.2), plus the open-x injection terms."""
    f = np.empty(G.shape, dtype=np.float64)
    lib().or_poisson_rhs(ctypes.byref(G.c()), _theta_ptr(theta), K, _dp(_cplx(psi)), _dp(f))
    if G.bc[0] == OPEN and G.Jext != 0.0:
        cond = G.conducting()      # no current enters an insulating face site
        f[:, :, 0] -= 2.0 * G.Jext / G.hx * cond[:, :, 0]
        f[:, :, -1] += 2.0 * G.Jext / G.hx * cond[:, :, -1]
    return f


def laplacian_mu(G: Grid, mu):
    out = np.empty(G.shape, dtype=np.float64)
    lib().or_laplacian_mu(ctypes.byref(G.c()), _dp(np.ascontiguousarray(mu, dtype=np.float64)), _dp(out))
    return out


def _axis_eigs(n, h, c, bc):
    k = np.arange(n)
    if n < 2:
        return np.zeros(n)
    if bc == PERIODIC:
        return -4.0 * c * np.sin(math.pi * k / n) ** 2
    return -4.0 * c * np.sin(math.pi * k / (2.0 * (n - 1))) ** 2


def poisson_solve(G: Grid, F):
    """Exact solution of Lap mu = F (Sec. 3.2 operator, periodic or Neumann per
    axis) with the zero mode removed (sum_m w_m mu_m = 0).  The component of F
    along the null space is discarded, which is the compatibility projection."""
    if G.insulating is not None:
        return poisson_solve_insulating(G, F)
    F = np.asarray(F, dtype=np.float64)
    ns = (G.nx, G.ny, G.nz)
    hs = (G.hx, G.hy, G.hz)
    cs = [1.0 / (h * h) for h in hs]
    cs[2] /= G.g * G.g
    arr_axis = {0: 2, 1: 1, 2: 0}   # array axis of x, y, z
    X = F.astype(np.complex128)
    for ax in range(3):
        if ns[ax] >= 2 and G.bc[ax] == OPEN:
            X = sfft.dct(X.real, type=1, axis=arr_axis[ax]) + 1j * sfft.dct(X.imag, type=1, axis=arr_axis[ax])
    for ax in range(3):
        if ns[ax] >= 2 and G.bc[ax] == PERIODIC:
            X = sfft.fft(X, axis=arr_axis[ax])
    lam = np.zeros(G.shape)
    for ax in range(3):
        e = _axis_eigs(ns[ax], hs[ax], cs[ax], G.bc[ax])
        shape = [1, 1, 1]
        shape[arr_axis[ax]] = ns[ax]
        lam = lam + e.reshape(shape)
    lam_safe = np.where(lam == 0.0, 1.0, lam)
    X = np.where(lam == 0.0, 0.0, X / lam_safe)
    for ax in range(3):
        if ns[ax] >= 2 and G.bc[ax] == PERIODIC:
            X = sfft.ifft(X, axis=arr_axis[ax])
    for ax in range(3):
        if ns[ax] >= 2 and G.bc[ax] == OPEN:
            X = sfft.idct(X.real, type=1, axis=arr_axis[ax]) + 1j * sfft.idct(X.imag, type=1, axis=arr_axis[ax])
    return X.real.copy()


def masked_laplacian_matrix(G: Grid):
    """The Poisson operator of Sec. 3.2 with the links next to insulating sites removed
    (Sec. 3.4 (ii)), as a sparse matrix over all sites: for every link joining two
    conducting sites, c_a (2 c_a for the inner link of an open face, the Neumann ghost)
    on the neighbour and minus the same on the diagonal; rows of insulating sites empty."""
    import scipy.sparse as sp
    cond = G.conducting()
    ns = (G.nx, G.ny, G.nz)
    hs = (G.hx, G.hy, G.hz)
    k, j, i = np.meshgrid(np.arange(G.nz), np.arange(G.ny), np.arange(G.nx), indexing="ij")
    idx = (i, j, k)
    m = (i + G.nx * (j + G.ny * k)).ravel()
    rows, cols, vals = [], [], []
    for ax in range(3):
        n = ns[ax]
        if n < 2:
            continue
        c = 1.0 / (hs[ax] * hs[ax]) / (G.g * G.g if ax == 2 else 1.0)
        for sgn in (1, -1):
            t = [a.copy() for a in idx]
            t[ax] = t[ax] + sgn
            exists = np.ones(G.shape, dtype=bool)
            if G.bc[ax] == OPEN:
                exists = (t[ax] >= 0) & (t[ax] < n)
            t[ax] = t[ax] % n
            nb = (t[0] + G.nx * (t[1] + G.ny * t[2]))
            ok = exists & cond & cond.ravel()[nb.ravel()].reshape(G.shape)
            wt = np.ones(G.shape)
            if G.bc[ax] == OPEN:
                face = (idx[ax] == 0) if sgn > 0 else (idx[ax] == n - 1)
                wt = np.where(face, 2.0, 1.0)
            v = (c * wt * ok).ravel()
            sel = v != 0
            rows += [m[sel], m[sel]]
            cols += [nb.ravel()[sel], m[sel]]
            vals += [v[sel], -v[sel]]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(G.N, G.N))


def conducting_components(G: Grid):
    """Labels of the connected components of the conducting sites (joined by the links
    that remain), -1 on insulating sites; and the number of components."""
    from scipy.sparse.csgraph import connected_components
    cond = G.conducting().ravel()
    idx = np.nonzero(cond)[0]
    A = masked_laplacian_matrix(G)[idx][:, idx]
    n, lab = connected_components(A, directed=False)
    out = np.full(G.N, -1)
    out[idx] = lab
    return out.reshape(G.shape), int(n)


def poisson_solve_insulating(G: Grid, F):
    """Lap mu = F on the conducting sites with no flux through links next to insulating
    sites (Sec. 3.4 (ii)), mu = 0 on insulating sites.  Each connected component of the
    conducting sites carries its own constant: F is made compatible on each (sum w F = 0
    over the component) and mu has zero weighted mean on each.  W Lap is symmetric (w the
    trapezoid weights), so CG on -W Lap in FP64 to 1e-14 gives the solution."""
    import scipy.sparse.linalg as sla
    cond = G.conducting().ravel()
    w = site_weights(G).ravel()
    lab, ncomp = conducting_components(G)
    lab = lab.ravel()
    idx = np.nonzero(cond)[0]
    A = masked_laplacian_matrix(G)
    Ac = A[idx][:, idx]
    wc = w[idx]
    lc = lab[idx]
    wsum = np.bincount(lc, weights=wc, minlength=ncomp)
    f = np.asarray(F, dtype=np.float64).ravel()[idx]
    f = f - (np.bincount(lc, weights=wc * f, minlength=ncomp) / wsum)[lc]
    Wm = -(Ac.multiply(wc[:, None])).tocsr()
    sol, info = sla.cg(Wm, -wc * f, rtol=1e-14, atol=0.0, maxiter=20000)
    if info != 0:
        raise RuntimeError(f"masked Poisson CG did not converge ({info})")
    sol = sol - (np.bincount(lc, weights=wc * sol, minlength=ncomp) / wsum)[lc]
    mu = np.zeros(G.N)
    mu[idx] = sol
    return mu.reshape(G.shape)


def site_weights(G: Grid):
    """Trapezoid weights w_m: product of 1/2 per open face the site lies on."""
    w = np.ones(G.shape)
    for ax, aa in ((0, 2), (1, 1), (2, 0)):
        n = (G.nx, G.ny, G.nz)[ax]
        if G.bc[ax] == OPEN and n >= 2:
            sl = [slice(None)] * 3
            sl[aa] = 0
            w[tuple(sl)] *= 0.5
            sl[aa] = n - 1
            w[tuple(sl)] *= 0.5
    return w


def energy(G: Grid, psi, alpha, K=0.0, theta=None) -> float:
    return lib().or_energy(ctypes.byref(G.c()), _theta_ptr(theta), K, _dp(_cplx(psi)),
                           _dp(np.ascontiguousarray(alpha, dtype=np.float64)))


def winding(G: Grid, psi, K=0.0, theta=None):
    """Per-plaquette winding numbers (xy plaquettes) and their signed total."""
    n = np.zeros(G.shape, dtype=np.int32)
    tot = lib().or_winding(ctypes.byref(G.c()), _theta_ptr(theta), K, _dp(_cplx(psi)),
                           n.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return n, int(tot)


def vortex_count(G: Grid, psi, K=0.0, theta=None):
    """(unsigned count per z layer averaged over layers, signed total per layer averaged)."""
    n, tot = winding(G, psi, K, theta)
    return float(np.abs(n).sum() / G.nz), float(tot / G.nz)


def pattern(G: Grid, inclusions, target=0, alpha_in=-1.0, alpha_out=1.0):
    """Inclusion map alpha (Sec. 3.4); returns (alpha, candidates used, marked sites)."""
    inc = np.ascontiguousarray(inclusions, dtype=np.float64)
    alpha = np.empty(G.shape, dtype=np.float64)
    marked = ctypes.c_int64(0)
    used = lib().or_pattern(ctypes.byref(G.c()), _dp(inc), inc.shape[0], int(target), alpha_in, alpha_out,
                            _dp(alpha), ctypes.byref(marked))
    return alpha, int(used), int(marked.value)


def inside_q(G: Grid, inclusion, i, j, k) -> float:
    inc = np.ascontiguousarray(inclusion, dtype=np.float64)
    return lib().or_inside_q(ctypes.byref(G.c()), _dp(inc), i, j, k)


# Full pattern generator (Sec. 3.4).  A shape is 13 numbers: kind, flags, centre[3],
# semi-axes[3], unit quaternion (w, x, y, z)[4], value.
ELLIPSOID, CUBOID, CYLINDER, CROSS, OCTANT = 0, 1, 2, 3, 4
INVERT, INSULATING = 1, 2
BG_CONSTANT, BG_CHECKER, BG_VORONOI = 0, 1, 2
EUCLIDEAN, ABSOLUTE, MAXIMUM = 0, 1, 2
SQUARE, TRIANGULAR, HONEYCOMB, KAGOME, RECTANGULAR, HEXAGONAL = 0, 1, 2, 3, 4, 5


def shape_contains(G: Grid, shape, i, j, k) -> bool:
    """Whether the shape's set (before its invert flag) holds site (i, j, k)."""
    sh = np.ascontiguousarray(shape, dtype=np.float64)
    return bool(lib().or_shape_contains(ctypes.byref(G.c()), _dp(sh), i, j, k))


def _lattice_record(lat: dict) -> np.ndarray:
    rec = np.zeros(24, dtype=np.float64)
    rec[0] = lat["kind"]
    rec[1:4] = lat["count"]
    rec[4:7] = lat.get("origin", (0.0, 0.0, 0.0))
    rec[7:10] = lat["spacing"]
    rec[10:23] = lat["motif"]
    return rec


def lattice_shapes(lat: dict) -> np.ndarray:
    """The shapes of one lattice: {kind, count[3], origin[3], spacing[3] (a, b, c), motif[13]}."""
    rec = _lattice_record(lat)
    n = lib().or_lattice_shapes(_dp(rec), None)
    out = np.zeros((n, 13), dtype=np.float64)
    lib().or_lattice_shapes(_dp(rec), _dp(out))
    return out


def voronoi_owner(G: Grid, seeds, metric, i, j, k) -> int:
    sd = np.ascontiguousarray(seeds, dtype=np.float64).reshape(-1, 4)
    return int(lib().or_voronoi_owner(ctypes.byref(G.c()), _dp(sd), sd.shape[0], int(metric), i, j, k))


def pattern_ex(G: Grid, shapes=None, lattices=(), background=None, target=0):
    """Pinning landscape: explicit shapes, then each lattice's shapes, first claim wins;
    the rest takes the background {kind, metric, value, cell[3], values[2], p_odd, seed,
    seeds (n, 4)}.  Returns (alpha, insulating (uint8), shapes used, sites claimed)."""
    parts = [np.asarray(shapes, dtype=np.float64).reshape(-1, 13)] if shapes is not None else []
    parts += [lattice_shapes(lat) for lat in lattices]
    allsh = np.ascontiguousarray(np.concatenate(parts) if parts else np.zeros((0, 13)), dtype=np.float64)
    bg = dict(background or {})
    cell = np.ascontiguousarray(bg.get("cell", (0.0, 0.0, 0.0)), dtype=np.float64)
    vals = np.ascontiguousarray(bg.get("values", (0.0, 0.0)), dtype=np.float64)
    seeds = np.ascontiguousarray(bg.get("seeds", np.zeros((0, 4))), dtype=np.float64).reshape(-1, 4)
    alpha = np.empty(G.shape, dtype=np.float64)
    ins = np.empty(G.shape, dtype=np.uint8)
    marked = ctypes.c_int64(0)
    used = lib().or_pattern_ex(ctypes.byref(G.c()), _dp(allsh), allsh.shape[0], int(target),
                               int(bg.get("kind", BG_CONSTANT)), int(bg.get("metric", EUCLIDEAN)),
                               float(bg.get("value", 1.0)), _dp(cell), _dp(vals), float(bg.get("p_odd", -1.0)),
                               int(bg.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF, _dp(seeds), seeds.shape[0],
                               _dp(alpha), ins.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), ctypes.byref(marked))
    return alpha, ins, int(used), int(marked.value)


def voltage_open_x(G: Grid, mu) -> float:
    """E_x from the mean potential of each x face.  With insulating sites: over the face
    sites of the largest conducting component (an island enclosed by insulators carries
    its own constant in mu and no current from face to face)."""
    if G.insulating is None:
        return float((mu[:, :, 0].mean() - mu[:, :, -1].mean()) / ((G.nx - 1) * G.hx))
    lab, _ = conducting_components(G)
    main = np.bincount(lab[lab >= 0]).argmax()
    c = lab == main
    m0 = mu[:, :, 0][c[:, :, 0]].mean()
    m1 = mu[:, :, -1][c[:, :, -1]].mean()
    return float((m0 - m1) / ((G.nx - 1) * G.hx))


# --------------------------------------------------------------------------
# The implicit psi solve and the time step
# --------------------------------------------------------------------------
class NotConverged(RuntimeError):
    pass


def philox4x32_10(counter, key):
    """Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): four 32-bit outputs."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in counter])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    out = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, out)
    return [int(v) for v in out]


def noise_amplitude(G: Grid) -> float:
    """h_t zeta_max with zeta_max = (T_zeta / (h_t hx hy hz))^(1/2) (Sec. 3.1.2); a film
    (Nz = 1) drops hz."""
    if G.noise_T <= 0:
        return 0.0
    vol = G.hx * G.hy * (G.hz if G.nz >= 2 else 1.0)
    return G.ht * math.sqrt(G.noise_T / (G.ht * vol))


def add_noise(G: Grid, b, step: int):
    """b += h_t zeta(step) in place (the 2 zeta_m term of Eq. b times h_t/2)."""
    amp = noise_amplitude(G)
    if amp > 0:
        lib().or_noise(ctypes.byref(G.c()), amp, int(G.noise_seed) & 0xFFFFFFFFFFFFFFFF, int(step), _dp(b))
    return b


def solve_psi(G: Grid, psi_prev, mu, alpha, K=0.0, theta=None, eps=1e-6, max_iter=200,
              check_every=1, fixed_sweeps=0, step=0):
    """Linear solve M psi = b by Jacobi (Eq. final) from psi^(0) = psi^-.

    Returns (psi, sweeps, r2 of the last tested residual, list of per-sweep r2)."""
    b, D = init(G, psi_prev, mu, alpha, K, theta)
    add_noise(G, b, step)
    cur = _cplx(psi_prev)
    hist = []
    for l in range(max_iter):
        nxt, r2 = sweep(G, cur, b, D, K, theta)
        hist.append(r2)
        if fixed_sweeps > 0:
            if l + 1 == fixed_sweeps:
                return nxt, l + 1, r2, hist
        elif (l + 1) % check_every == 0 and r2 < eps:
            return nxt, l + 1, r2, hist
        cur = nxt
    raise NotConverged(f"Jacobi did not reach |r|^2 < {eps} in {max_iter} sweeps")


@dataclasses.dataclass
class State:
    psi: np.ndarray
    mu: np.ndarray
    K: float = 0.0
    step: int = 0


@dataclasses.dataclass
class StepStats:
    sweeps: int
    r2: float
    Jav: float
    Ex: float
    K: float


def rewind(K: float, hx: float) -> float:
    """K -> K - (2 pi/hx) floor(K hx / 2 pi) (Sec. 2.2)."""
    return K - (2.0 * math.pi / hx) * math.floor(K * hx / (2.0 * math.pi))


def step(G: Grid, st: State, alpha, theta=None, eps=1e-6, max_iter=200, check_every=1,
         fixed_sweeps=0, freeze_mu_K=False) -> StepStats:
    """One time step in the paper's order: psi, then K (E_x), then mu (Sec. 3)."""
    psi, nsw, r2, _ = solve_psi(G, st.psi, st.mu, alpha, st.K, theta, eps, max_iter, check_every, fixed_sweeps,
                                st.step)
    Kold = st.K
    Knew = Kold
    Jav = 0.0
    Ex = 0.0
    if G.bc[0] == PERIODIC:
        Jav = javg(G, psi, Kold, theta)
        if not freeze_mu_K:
            dtK = G.u * G.ht
            Knew = Kold + dtK * (G.Jext - Jav)
            Ex = (Knew - Kold) / dtK
            Knew = rewind(Knew, G.hx)
    mu = st.mu
    if not freeze_mu_K:
        f = poisson_rhs(G, psi, Knew, theta)
        mu = poisson_solve(G, f)
    if G.bc[0] == OPEN:
        Ex = voltage_open_x(G, mu)
    st.psi, st.mu, st.K = psi, mu, Knew
    st.step += 1
    return StepStats(nsw, r2, Jav, Ex, Knew)


def run(G: Grid, st: State, alpha, nsteps, **kw):
    stats = []
    for _ in range(nsteps):
        stats.append(step(G, st, alpha, **kw))
    return stats


# --------------------------------------------------------------------------
# Pieces used by the adjoint
# --------------------------------------------------------------------------
def ns(G: Grid, psi, K=0.0, theta=None):
    """Neighbour sum NS_m(psi): the off-diagonal part of the gauge Laplacian."""
    out = np.empty(G.shape, dtype=np.complex128)
    L = lib()
    L.or_ns.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.or_ns(ctypes.byref(G.c()), _theta_ptr(theta), K, _dp(_cplx(psi)), _dp(out))
    return out


def ns_adj(G: Grid, lam, K=0.0, theta=None):
    """Conjugate transpose of the neighbour-sum operator applied to lam."""
    out = np.empty(G.shape, dtype=np.complex128)
    L = lib()
    L.or_ns_adj.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.or_ns_adj(ctypes.byref(G.c()), _theta_ptr(theta), K, _dp(_cplx(lam)), _dp(out))
    return out


def voltage_weights(G: Grid):
    """v with E_x = sum(v * mu) for open x (the face-mean voltage)."""
    v = np.zeros(G.shape)
    s = 1.0 / (G.ny * G.nz * (G.nx - 1) * G.hx)
    v[:, :, 0] = s
    v[:, :, -1] -= s
    return v
