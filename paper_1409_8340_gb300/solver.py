"""Python front end of the GB300 TDGL solver.

PyTorch only provides device memory and the stream: the workspace is one
uint8 CUDA tensor handed to tdgl_create(), and the state arrays are exposed as
zero-copy tensor views into it.  All arithmetic runs in libtdgl_gb300.so.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math

import numpy as np
import torch

from . import _lib
from ._lib import OPEN, PERIODIC, TdglError, check


@dataclasses.dataclass
class Params:
    """Problem description (see include/tdgl.h, struct tdgl_config)."""
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
    eps: float = 1e-6
    max_iter: int = 200
    check_every: int = 1
    fixed_sweeps: int = 0
    freeze_mu_K: bool = False
    poisson_cycles: int = 1
    poisson_max_cycles: int = 50
    poisson_tol: float = 0.0
    poisson_guess: int = 0         # 1 previous mu, 2 linear extrapolation in time, 0 default (2)
    general_links: bool = False
    xz_gauge: bool = False         # field (Bx, 0, Bz) in the Landau gauge of Eq. A_xz (By must be 0)
    Bx: float = 0.0
    sweeps_per_pass: int = 1       # 2: temporal blocking, two Jacobi sweeps per pass over memory
    sweep_kernel: int = 0          # 1 register-tiled, 2 staged in shared memory by bulk copies, 0 default
    noise_T: float = 0.0           # thermal noise parameter T_zeta (Sec. 3.1.2); 0: none
    noise_seed: int = 0

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def N(self):
        return self.nx * self.ny * self.nz

    def length(self, ax):
        n = (self.nx, self.ny, self.nz)[ax]
        h = (self.hx, self.hy, self.hz)[ax]
        return n * h if self.bc[ax] == PERIODIC else (n - 1) * h

    def quantise_Bz(self, n_quanta: int):
        """Set Bz to n flux quanta through the xy face (Sec. 3.3.1)."""
        self.Bz = 2 * math.pi * n_quanta / (self.length(0) * self.length(1))
        return self

    def to_c(self, d_alpha: int, d_link_phase: int = 0) -> _lib.Config:
        c = _lib.Config()
        c.nx, c.ny, c.nz = self.nx, self.ny, self.nz
        c.bc[:] = list(self.bc)
        c.hx, c.hy, c.hz = self.hx, self.hy, self.hz
        c.g, c.u, c.beta, c.ht = self.g, self.u, self.beta, self.ht
        c.By, c.Bz, c.Jext = self.By, self.Bz, self.Jext
        c.eps = self.eps
        c.max_iter = self.max_iter
        c.check_every = self.check_every
        c.fixed_sweeps = self.fixed_sweeps
        c.freeze_mu_K = int(bool(self.freeze_mu_K))
        c.poisson_cycles = self.poisson_cycles
        c.poisson_max_cycles = max(self.poisson_max_cycles, self.poisson_cycles)
        c.poisson_tol = self.poisson_tol
        c.links_mode = (_lib.LINKS_GENERAL if self.general_links else
                        _lib.LINKS_XZ if self.xz_gauge else _lib.LINKS_LANDAU)
        c.Bx = float(self.Bx)
        c.sweeps_per_pass = int(self.sweeps_per_pass)
        c.sweep_kernel = int(self.sweep_kernel)
        c.poisson_guess = int(self.poisson_guess)
        c.noise_T = float(self.noise_T)
        c.noise_seed = int(self.noise_seed) & 0xFFFFFFFFFFFFFFFF
        c.d_alpha = d_alpha
        c.d_link_phase = d_link_phase or None
        return c


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Solver:
    """One TDGL problem on one GPU.  alpha: CUDA float32 tensor of shape (nz, ny, nx)."""

    def __init__(self, p: Params, alpha: torch.Tensor, link_phase: torch.Tensor | None = None, stream=None,
                 device=None, insulating: torch.Tensor | None = None):
        """insulating: optional CUDA uint8 tensor of shape (nz, ny, nx), nonzero on insulating
        sites (Sec. 3.4 (ii)); read once at creation."""
        L = _lib.load()
        self.p = p
        self.device = alpha.device if device is None else torch.device(device)
        if alpha.dtype != torch.float32 or not alpha.is_cuda or alpha.numel() != p.N:
            raise ValueError("alpha must be a CUDA float32 tensor with nx*ny*nz elements")
        self.alpha = alpha.contiguous()
        self.link_phase = None
        if p.general_links:
            if link_phase is None or link_phase.numel() != 3 * p.N:
                raise ValueError("general links need a float32 phase tensor of 3*N elements")
            self.link_phase = link_phase.contiguous().to(torch.float32)
        self._cfg = p.to_c(self.alpha.data_ptr(), self.link_phase.data_ptr() if self.link_phase is not None else 0)
        self.insulating = None
        if insulating is not None:
            if insulating.dtype != torch.uint8 or not insulating.is_cuda or insulating.numel() != p.N:
                raise ValueError("insulating must be a CUDA uint8 tensor with nx*ny*nz elements")
            self.insulating = insulating.contiguous()
            self._cfg.d_insulating = self.insulating.data_ptr()
        nbytes = L.tdgl_workspace_bytes(ctypes.byref(self._cfg))
        if nbytes == 0:
            raise TdglError(-1, "tdgl_workspace_bytes")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        check(L.tdgl_create(ctypes.byref(self._cfg), ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                            ctypes.c_void_p(_stream_ptr(self.stream)), ctypes.byref(h)), "tdgl_create")
        self._h = h
        self._L = L
        self._owned = True

    @classmethod
    def _attach(cls, p: Params, alpha: torch.Tensor, handle: ctypes.c_void_p, workspace: torch.Tensor, stream, L):
        """A view of a handle owned by someone else (a batch instance)."""
        obj = cls.__new__(cls)
        obj.p = p
        obj.device = alpha.device
        obj.alpha = alpha
        obj.link_phase = None
        obj.insulating = None
        obj.stream = stream
        obj.workspace = workspace
        obj._h = handle
        obj._L = L
        obj._owned = False
        return obj

    # ------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                self._L.tdgl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _view(self, ptr: int, dtype, shape):
        off = ptr - self.workspace.data_ptr()
        n = int(np.prod(shape)) * torch.empty((), dtype=dtype).element_size()
        return self.workspace[off:off + n].view(dtype).view(shape)

    def state(self):
        """(psi complex64, mu float32) zero-copy views of the current state."""
        sp = _lib.StatePtrs()
        check(self._L.tdgl_get_state(self._h, ctypes.byref(sp)), "tdgl_get_state")
        return self._view(sp.psi, torch.complex64, self.p.shape), self._view(sp.mu, torch.float32, self.p.shape)

    def internals(self):
        """Views of b, diag M and the Poisson right-hand side of the last step."""
        sp = _lib.StatePtrs()
        check(self._L.tdgl_get_state(self._h, ctypes.byref(sp)), "tdgl_get_state")
        return (self._view(sp.b, torch.complex64, self.p.shape), self._view(sp.D, torch.complex64, self.p.shape),
                self._view(sp.f, torch.float32, self.p.shape))

    def set_state(self, psi: torch.Tensor, mu: torch.Tensor | None = None, K: float = 0.0):
        psi = psi.to(device=self.device, dtype=torch.complex64).contiguous()
        mu_ptr = None
        if mu is not None:
            mu = mu.to(device=self.device, dtype=torch.float32).contiguous()
            mu_ptr = ctypes.c_void_p(mu.data_ptr())
        check(self._L.tdgl_set_state(self._h, ctypes.c_void_p(psi.data_ptr()), mu_ptr, float(K)), "tdgl_set_state")

    def upload_state(self, psi: np.ndarray | torch.Tensor, mu=None, K: float = 0.0):
        """Copy a state in from host memory (numpy or CPU tensor)."""
        psi_t = torch.as_tensor(psi).to(torch.complex64).contiguous()
        mu_t = None if mu is None else torch.as_tensor(mu).to(torch.float32).contiguous()
        check(self._L.tdgl_upload_state(self._h, ctypes.c_void_p(psi_t.data_ptr()),
                                        None if mu_t is None else ctypes.c_void_p(mu_t.data_ptr()), float(K)),
              "tdgl_upload_state")

    def download_state(self, psi_out: torch.Tensor | None = None, mu_out: torch.Tensor | None = None):
        psi_out = torch.empty(self.p.shape, dtype=torch.complex64) if psi_out is None else psi_out
        mu_out = torch.empty(self.p.shape, dtype=torch.float32) if mu_out is None else mu_out
        K = ctypes.c_double()
        check(self._L.tdgl_download_state(self._h, ctypes.c_void_p(psi_out.data_ptr()),
                                          ctypes.c_void_p(mu_out.data_ptr()), ctypes.byref(K)), "tdgl_download_state")
        return psi_out, mu_out, K.value

    def set_step(self, n: int):
        """Set the step index and the noise counter of the next step (tdgl_set_step)."""
        check(self._L.tdgl_set_step(self._h, int(n)), "tdgl_set_step")

    def checkpoint(self) -> dict:
        """The resumable state in host memory: psi, mu, K, the previous step's mu (read by
        the extrapolated Poisson guess; None when the handle holds none) and the step index
        (which is also the counter of the thermal noise)."""
        psi, mu, K = self.download_state()
        prev = torch.empty(self.p.shape, dtype=torch.float32)
        rc = self._L.tdgl_get_mu_prev(self._h, ctypes.c_void_p(prev.data_ptr()), 1)
        if rc < 0:
            check(rc, "tdgl_get_mu_prev")
        return {"psi": psi, "mu": mu, "K": K, "mu_prev": prev if rc == 1 else None,
                "step": int(self.observables()["step"])}

    def restore(self, ck: dict):
        """Load a checkpoint(): the run continues exactly as it would have, noise included."""
        self.upload_state(ck["psi"], ck["mu"], ck["K"])
        prev = ck.get("mu_prev")
        if prev is not None:
            prev = torch.as_tensor(prev).to(torch.float32).contiguous()
            check(self._L.tdgl_set_mu_prev(self._h, ctypes.c_void_p(prev.data_ptr()), 1), "tdgl_set_mu_prev")
        self.set_step(ck["step"])

    def step(self, n: int = 1):
        check(self._L.tdgl_step(self._h, int(n)), "tdgl_step")

    def step_resident(self, n: int = 1):
        """n steps as one CUDA graph launch (conditional nodes), one synchronisation."""
        check(self._L.tdgl_step_resident(self._h, int(n)), "tdgl_step_resident")

    def step_enqueue(self, n: int = 1):
        """n resident steps enqueued without waiting; errors surface at sync() or at the
        next call on the solver."""
        check(self._L.tdgl_step_enqueue(self._h, int(n)), "tdgl_step_enqueue")

    def sync(self):
        """Wait for the enqueued steps; raises their error."""
        check(self._L.tdgl_sync(self._h), "tdgl_sync")

    def autotune(self, trial_steps: int = 3) -> dict:
        """Time the staged sweep, the register-tiled sweep and two sweeps per pass from the
        current state (restored after every trial) and keep the fastest."""
        r = _lib.TuneReport()
        check(self._L.tdgl_autotune(self._h, int(trial_steps), ctypes.byref(r)), "tdgl_autotune")
        names = ("staged", "register_tiled", "two_sweeps_per_pass")
        return {"ms_per_step": {names[c]: r.ms[c] for c in range(3) if r.ms[c] > 0}, "chosen": names[r.chosen],
                "candidates": r.candidates}

    def solve_psi(self) -> int:
        n = ctypes.c_int32()
        check(self._L.tdgl_solve_psi(self._h, ctypes.byref(n)), "tdgl_solve_psi")
        return n.value

    def solve_mu(self):
        check(self._L.tdgl_solve_mu(self._h), "tdgl_solve_mu")

    def adjoint(self, n_steps: int, checkpoint_every: int = 20, window_start: int | None = None,
                adj_eps: float = 1e-8, adj_max_iter: int = 500, poisson_cycles: int = 2, poisson_tol: float = 0.0):
        """Run n_steps forward from the current state and return (J, dJ/dalpha, stats),
        J = mean E_x over steps window_start+1..n_steps (default: the second half)."""
        ws_start = n_steps // 2 if window_start is None else window_start
        ac = _lib.AdjointConfig(n_steps, checkpoint_every, ws_start, adj_max_iter, adj_eps, poisson_cycles, 0,
                                poisson_tol)
        nbytes = self._L.tdgl_adjoint_workspace_bytes(self._h, ctypes.byref(ac))
        if nbytes == 0:
            raise TdglError(-1, "tdgl_adjoint_workspace_bytes")
        ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        grad = torch.empty(self.p.shape, dtype=torch.float32, device=self.device)
        J = ctypes.c_double()
        st = _lib.AdjointStats()
        check(self._L.tdgl_adjoint(self._h, ctypes.byref(ac), ctypes.c_void_p(ws.data_ptr()), nbytes,
                                   ctypes.c_void_p(grad.data_ptr()), ctypes.byref(J), ctypes.byref(st)),
              "tdgl_adjoint")
        return J.value, grad, st.as_dict()

    def profile_enable(self, on: bool = True):
        check(self._L.tdgl_profile_enable(self._h, int(bool(on))), "tdgl_profile_enable")

    def test_staged_waits(self, wait_ns: int = 0, extra_tx_bytes: int = 0):
        """Test hook (tdgl_test_staged_waits): bound the staged kernels' waits by wait_ns and
        add extra_tx_bytes to every stage's expected bytes, so that the waits run out;
        (0, 0) is normal use."""
        check(self._L.tdgl_test_staged_waits(self._h, int(wait_ns), int(extra_tx_bytes)), "tdgl_test_staged_waits")

    def profile(self) -> dict:
        pr = _lib.Profile()
        check(self._L.tdgl_profile_read(self._h, ctypes.byref(pr)), "tdgl_profile_read")
        return pr.as_dict()

    def observables(self) -> dict:
        o = _lib.Obs()
        check(self._L.tdgl_observables(self._h, ctypes.byref(o)), "tdgl_observables")
        return o.as_dict()


class Batch:
    """Independent TDGL problems (own sizes, fields, currents, time steps and alpha
    maps) advanced together: one persistent launch per time step for all of them,
    replayed from a CUDA graph.  instances[i] is a Solver view of instance i for
    state access and observables; stepping goes through the batch."""

    def __init__(self, params: list[Params], alphas: list[torch.Tensor], stream=None):
        L = _lib.load()
        if len(params) != len(alphas) or not params:
            raise ValueError("one alpha map per instance is needed")
        n = len(params)
        self.params = list(params)
        self.alphas = []
        for p, a in zip(params, alphas):
            if a.dtype != torch.float32 or not a.is_cuda or a.numel() != p.N:
                raise ValueError("alpha must be a CUDA float32 tensor with nx*ny*nz elements")
            self.alphas.append(a.contiguous())
        self.device = self.alphas[0].device
        self._cfgs = (_lib.Config * n)(*[p.to_c(a.data_ptr()) for p, a in zip(params, self.alphas)])
        nbytes = L.tdgl_batch_workspace_bytes(self._cfgs, n)
        if nbytes == 0:
            raise TdglError(-1, "tdgl_batch_workspace_bytes")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        b = ctypes.c_void_p()
        check(L.tdgl_batch_create(self._cfgs, n, ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                  ctypes.c_void_p(_stream_ptr(self.stream)), ctypes.byref(b)), "tdgl_batch_create")
        self._b = b
        self._L = L
        self.n = n
        self.instances = []
        for i in range(n):
            h = ctypes.c_void_p()
            check(L.tdgl_batch_instance(b, i, ctypes.byref(h)), "tdgl_batch_instance")
            self.instances.append(Solver._attach(params[i], self.alphas[i], h, self.workspace, self.stream, L))

    def close(self):
        if getattr(self, "_b", None):
            for s in self.instances:
                s._h = None
            self._L.tdgl_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        """Enqueue n batch steps (asynchronous; errors surface in status())."""
        check(self._L.tdgl_batch_step(self._b, int(n)), "tdgl_batch_step")

    def status(self) -> tuple[int, list[int]]:
        st = (ctypes.c_int32 * self.n)()
        rc = self._L.tdgl_batch_status(self._b, st)
        return rc, list(st)

    def check(self):
        rc, _ = self.status()
        check(rc, "tdgl_batch_status")

    def observables(self) -> list[dict]:
        out = (_lib.Obs * self.n)()
        check(self._L.tdgl_batch_observables(self._b, out), "tdgl_batch_observables")
        return [o.as_dict() for o in out]

    def stats(self) -> dict:
        st = _lib.BatchStats()
        sw = (ctypes.c_int64 * self.n)()
        check(self._L.tdgl_batch_stats_read(self._b, ctypes.byref(st), sw), "tdgl_batch_stats_read")
        d = st.as_dict()
        d["instance_sweeps"] = list(sw)
        return d

    def tuning(self) -> dict:
        t = _lib.BatchTuning()
        check(self._L.tdgl_batch_get_tuning(self._b, ctypes.byref(t)), "tdgl_batch_get_tuning")
        return {"blocks_per_sm": t.blocks_per_sm, "graph_steps": t.graph_steps, "timeout_ms": t.timeout_ms,
                "test_extra_arrivals": t.test_extra_arrivals, "sweep_kernel": t.sweep_kernel,
                "kz": list(t.kz)[:self.n]}

    def set_tuning(self, **kw):
        t = _lib.BatchTuning()
        check(self._L.tdgl_batch_get_tuning(self._b, ctypes.byref(t)), "tdgl_batch_get_tuning")
        for k, v in kw.items():
            if k == "kz":
                for i, z in enumerate(v):
                    t.kz[i] = int(z)
            else:
                setattr(t, k, int(v))
        check(self._L.tdgl_batch_set_tuning(self._b, ctypes.byref(t)), "tdgl_batch_set_tuning")

    def phase_log(self, on: bool = True):
        """Record the phase timings of every launch (tdgl_batch_phase_log)."""
        check(self._L.tdgl_batch_phase_log(self._b, int(bool(on))), "tdgl_batch_phase_log")

    def phase_profile(self) -> dict:
        """Per phase kind of the last launch: (ms, number of phases)."""
        n = len(_lib.BATCH_OPS)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int32 * n)()
        check(self._L.tdgl_batch_phase_read(self._b, ms, cnt, n), "tdgl_batch_phase_read")
        return {name: (ms[q], cnt[q]) for q, name in enumerate(_lib.BATCH_OPS)}

    def phase_list(self, cap: int = 512) -> list[tuple[str, float]]:
        """The last launch's phases in order: (kind, ms)."""
        ms = (ctypes.c_double * cap)()
        ops = (ctypes.c_int32 * cap)()
        n = ctypes.c_int32()
        check(self._L.tdgl_batch_phase_list(self._b, ms, ops, cap, ctypes.byref(n)), "tdgl_batch_phase_list")
        return [(_lib.BATCH_OPS[ops[q]], ms[q]) for q in range(min(n.value, cap))]

    def autotune(self, trial_steps: int = 3) -> dict:
        r = _lib.BatchTuneReport()
        check(self._L.tdgl_batch_autotune(self._b, int(trial_steps), ctypes.byref(r)), "tdgl_batch_autotune")
        return r.as_dict()


def pattern(p: Params, candidates: np.ndarray, target_sites: int = 0, alpha_in: float = -1.0,
            alpha_out: float = 1.0, device="cuda", stream=None):
    """Inclusion map alpha on the device (tdgl_pattern).  Returns (alpha, n_used, n_marked)."""
    L = _lib.load()
    cand = np.ascontiguousarray(candidates, dtype=np.float64).reshape(-1, 10)
    alpha = torch.empty(p.shape, dtype=torch.float32, device=device)
    cfg = p.to_c(alpha.data_ptr())
    nb = L.tdgl_pattern_scratch_bytes(ctypes.byref(cfg), cand.shape[0])
    scratch = torch.empty(max(nb, 256), dtype=torch.uint8, device=device)
    used = ctypes.c_int64()
    marked = ctypes.c_int64()
    st = stream if stream is not None else torch.cuda.current_stream(alpha.device)
    check(L.tdgl_pattern(ctypes.byref(cfg), cand.ctypes.data_as(ctypes.c_void_p), cand.shape[0], int(target_sites),
                         float(alpha_in), float(alpha_out), ctypes.c_void_p(alpha.data_ptr()),
                         ctypes.c_void_p(scratch.data_ptr()), nb, ctypes.c_void_p(st.cuda_stream),
                         ctypes.byref(used), ctypes.byref(marked)), "tdgl_pattern")
    return alpha, used.value, marked.value


def _shape_struct(row, out: _lib.Shape):
    row = np.asarray(row, dtype=np.float64).ravel()
    out.kind, out.flags = int(row[0]), int(row[1])
    out.c[:] = list(row[2:5])
    out.a[:] = list(row[5:8])
    out.q[:] = list(row[8:12])
    out.value = float(row[12])


def pattern_ex(p: Params, shapes=None, lattices=(), background=None, target_sites: int = 0, insulating: bool = False,
               device="cuda", stream=None):
    """Pinning landscape on the device (tdgl_pattern_ex, Sec. 3.4).

    shapes: (n, 13) rows (kind, flags, centre[3], semi-axes[3], quaternion (w, x, y, z)[4],
    value); lattices: dicts {kind, count[3], origin[3], spacing[3], motif (13 numbers)};
    background: dict {kind, metric, value, cell[3], values[2], p_odd, seed, seeds (n, 4)}
    (None: constant 1).  Returns (alpha, insulating mask or None, n_used, n_marked)."""
    L = _lib.load()
    sh = np.asarray(shapes if shapes is not None else np.zeros((0, 13)), dtype=np.float64).reshape(-1, 13)
    ns = sh.shape[0]
    sarr = (_lib.Shape * max(1, ns))()
    for n in range(ns):
        _shape_struct(sh[n], sarr[n])
    lats = list(lattices)
    larr = (_lib.Lattice * max(1, len(lats)))()
    for n, lat in enumerate(lats):
        larr[n].kind = int(lat["kind"])
        larr[n].count[:] = [int(v) for v in lat["count"]]
        larr[n].origin[:] = [float(v) for v in lat.get("origin", (0.0, 0.0, 0.0))]
        larr[n].spacing[:] = [float(v) for v in lat["spacing"]]
        _shape_struct(lat["motif"], larr[n].motif)
    bg = dict(background or {})
    B = _lib.Background()
    B.kind = int(bg.get("kind", _lib.BG_CONSTANT))
    B.metric = int(bg.get("metric", _lib.METRIC_EUCLIDEAN))
    B.value = float(bg.get("value", 1.0))
    B.cell[:] = [float(v) for v in bg.get("cell", (0.0, 0.0, 0.0))]
    B.values[:] = [float(v) for v in bg.get("values", (0.0, 0.0))]
    B.p_odd = float(bg.get("p_odd", -1.0))
    B.seed = int(bg.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    seeds = np.ascontiguousarray(bg.get("seeds", np.zeros((0, 4))), dtype=np.float64).reshape(-1, 4)
    B.host_seeds = seeds.ctypes.data if seeds.shape[0] else None
    B.n_seeds = seeds.shape[0]
    alpha = torch.empty(p.shape, dtype=torch.float32, device=device)
    ins = torch.empty(p.shape, dtype=torch.uint8, device=device) if insulating else None
    cfg = p.to_c(alpha.data_ptr())
    nb = L.tdgl_pattern_ex_scratch_bytes(ctypes.byref(cfg), ns, ctypes.addressof(larr), len(lats), ctypes.byref(B))
    if nb == 0:
        raise TdglError(-1, "tdgl_pattern_ex_scratch_bytes")
    scratch = torch.empty(nb, dtype=torch.uint8, device=device)
    used = ctypes.c_int64()
    marked = ctypes.c_int64()
    st = stream if stream is not None else torch.cuda.current_stream(alpha.device)
    check(L.tdgl_pattern_ex(ctypes.byref(cfg), ctypes.addressof(sarr), ns, ctypes.addressof(larr), len(lats),
                            ctypes.byref(B), int(target_sites), ctypes.c_void_p(alpha.data_ptr()),
                            ctypes.c_void_p(ins.data_ptr()) if ins is not None else None,
                            ctypes.c_void_p(scratch.data_ptr()), nb, ctypes.c_void_p(st.cuda_stream),
                            ctypes.byref(used), ctypes.byref(marked)), "tdgl_pattern_ex")
    return alpha, ins, used.value, marked.value


class TimeAveragedVoltage(torch.autograd.Function):
    """J(alpha) = time-averaged E_x of a run of n_steps from (psi0, mu0), differentiable
    in the pinning map alpha through the hand-written adjoint (tdgl_adjoint).

    The forward pass runs the checkpointed forward and, when alpha requires a
    gradient, the reverse pass too (checkpoint-and-recompute inside the library);
    backward scales the stored dJ/dalpha by the incoming gradient."""

    @staticmethod
    def forward(ctx, alpha, params: Params, psi0, mu0=None, n_steps: int = 400, checkpoint_every: int = 20,
                window_start: int | None = None, adj_eps: float = 1e-8):
        s = Solver(params, alpha.detach().contiguous())
        s.set_state(psi0, mu0, 0.0)
        if alpha.requires_grad:
            J, grad, _ = s.adjoint(n_steps, checkpoint_every, window_start, adj_eps)
            ctx.save_for_backward(grad)
        else:
            ws = n_steps // 2 if window_start is None else window_start
            ex = []
            for _ in range(n_steps):
                s.step(1)
                ex.append(s.observables()["Ex"])
            J = float(np.mean(ex[ws:]))
        s.close()
        return torch.tensor(J, dtype=torch.float64, device=alpha.device)

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        return (grad * gJ.to(grad.dtype), None, None, None, None, None, None, None)
