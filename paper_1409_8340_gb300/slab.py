"""z-slab decomposition of the time step over several GPUs or processes.

The paper names runs on several GPUs as future work (Sec. 5).  A grid that is
periodic in z is split into consecutive z-slabs; each process holds one or more
consecutive slabs (its share of the planes), each a slab handle of the C ABI
(tdgl_slab_*): the slab's planes between two halo planes that hold copies of the
neighbouring slabs' edge planes.  One time step, in the paper's order (Sec. 3.1:
psi; Sec. 3.2: mu):

  1. halo exchange of the state psi;
  2. init and first Jacobi sweep on every slab; the maximum of the slabs'
     max |r|^2 over the whole job (an all-reduce) is tested against eps
     (Eq. convergence); while it fails: halo exchange of the latest iterate and the
     next sweep;
  3. the result becomes the state; halo exchange;
  4. every slab writes the Poisson right-hand side of its planes; the parts are
     gathered on rank 0, which solves the potential of the whole grid (a Poisson-only
     handle) and scatters the slabs' parts back into their mu, with E_x.

The sweeps, the right-hand side and the Poisson solve are the library's kernels;
this module only moves planes and scalars between slabs (torch.distributed between
processes: NCCL for device tensors, gloo for host tensors) and takes the
convergence decision.  Slabs are given by a small protocol (planes, sweep, accept,
rhs, set_mu), implemented here for slab handles on the GPU.
"""
from __future__ import annotations

import ctypes
import math

import torch

from . import _lib
from ._lib import TdglError, check


# ---------------------------------------------------------------------------
# communication between the processes of one job
# ---------------------------------------------------------------------------
class LocalComm:
    """One process holding every slab: the periodic wrap joins its own top and bottom slabs."""
    rank = 0
    world = 1

    def exchange(self, send_up, send_down):
        """(plane for the bottom slab's lower halo, plane for the top slab's upper halo)."""
        return send_up, send_down

    def allreduce_max(self, x: float) -> float:
        return x

    def gather(self, t):
        return [t]

    def scatter(self, parts, like):
        return parts[0]

    def bcast(self, x: float) -> float:
        return x


class TorchComm:
    """torch.distributed between processes, one group of consecutive slabs per rank in rank
    order (rank r's top slab lies below rank r+1's bottom slab; the last rank's top slab below
    rank 0's bottom slab).  Every rank holds the same number of planes."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def exchange(self, send_up, send_down):
        d = self.dist
        if self.world == 1:
            return send_up, send_down
        up, down = (self.rank + 1) % self.world, (self.rank - 1) % self.world
        from_below = torch.empty_like(send_up)
        from_above = torch.empty_like(send_down)
        # the same order on every rank, so that the messages between one pair match in order
        ops = [d.P2POp(d.isend, send_up.contiguous(), up, self.group, 1),
               d.P2POp(d.isend, send_down.contiguous(), down, self.group, 2),
               d.P2POp(d.irecv, from_below, down, self.group, 1),
               d.P2POp(d.irecv, from_above, up, self.group, 2)]
        for r in d.batch_isend_irecv(ops):
            r.wait()
        return from_below, from_above

    def allreduce_max(self, x: float) -> float:
        dev = "cuda" if self.dist.get_backend(self.group) == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return float(t.item())

    def gather(self, t):
        t = t.contiguous()
        parts = [torch.empty_like(t) for _ in range(self.world)] if self.rank == 0 else None
        self.dist.gather(t, parts, dst=0, group=self.group)
        return parts

    def scatter(self, parts, like):
        out = torch.empty_like(like)
        self.dist.scatter(out, [p.contiguous() for p in parts] if self.rank == 0 else None, src=0, group=self.group)
        return out

    def bcast(self, x: float) -> float:
        dev = "cuda" if self.dist.get_backend(self.group) == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.dist.broadcast(t, src=0, group=self.group)
        return float(t.item())


# ---------------------------------------------------------------------------
# the step over all slabs
# ---------------------------------------------------------------------------
class NotConverged(RuntimeError):
    pass


class SlabStep:
    """One time step of the decomposed grid.  slabs: this process's slabs, bottom to top;
    poisson (rank 0 only): f of the whole grid (nz, ny, nx) -> (mu, E_x)."""

    def __init__(self, slabs, comm, eps: float, max_iter: int = 200, poisson=None):
        self.slabs = list(slabs)
        self.comm = comm
        self.eps = float(eps)
        self.max_iter = int(max_iter)
        self.poisson = poisson
        if comm.rank == 0 and poisson is None:
            raise ValueError("rank 0 needs the Poisson solver of the whole grid")

    def exchange(self, latest: bool):
        P = [s.planes(latest) for s in self.slabs]           # (first, last, halo below, halo above)
        for lower, upper in zip(P[:-1], P[1:]):
            upper[2].copy_(lower[1])
            lower[3].copy_(upper[0])
        below, above = self.comm.exchange(P[-1][1], P[0][0])
        P[0][2].copy_(below)
        P[-1][3].copy_(above)

    def step(self):
        """Returns (Jacobi sweeps, E_x)."""
        self.exchange(False)
        r2 = max(s.sweep(True) for s in self.slabs)
        sweeps = 1
        while True:
            g = self.comm.allreduce_max(r2)
            if not math.isfinite(g):
                raise TdglError(_lib.TDGL_ERR_NONFINITE, "slab step")
            if g < self.eps:          # the input of the last sweep passed: its output is the result
                break
            if sweeps >= self.max_iter:
                raise NotConverged(f"no convergence in {sweeps} sweeps")
            self.exchange(True)
            r2 = max(s.sweep(False) for s in self.slabs)
            sweeps += 1
        for s in self.slabs:
            s.accept()
        self.exchange(False)
        f = torch.cat([s.rhs() for s in self.slabs], dim=0)
        parts = self.comm.gather(f)
        mu_parts, ex = None, 0.0
        if self.comm.rank == 0:
            mu, ex = self.poisson(torch.cat(parts, dim=0))
            mu_parts = list(torch.split(mu, f.shape[0], dim=0))
        mu_local = self.comm.scatter(mu_parts, f)
        off = 0
        for s in self.slabs:
            n = s.nz_local
            s.set_mu(mu_local[off:off + n])
            off += n
        return sweeps, self.comm.bcast(ex)


# ---------------------------------------------------------------------------
# slabs and the whole-grid Poisson solve on the GPU (the library's kernels)
# ---------------------------------------------------------------------------
def _view(workspace: torch.Tensor, ptr: int, dtype, shape):
    off = ptr - workspace.data_ptr()
    n = 1
    for d in shape:
        n *= d
    n *= torch.empty((), dtype=dtype).element_size()
    return workspace[off:off + n].view(dtype).view(shape)


class GpuSlab:
    """A slab handle: planes z0 .. z0 + nz_local - 1 of the grid p (a solver.Params, periodic in
    z).  alpha: CUDA float32 (nz_local + 2, ny, nx), the slab with its halo planes."""

    def __init__(self, p, z0: int, nz_local: int, alpha: torch.Tensor, stream=None):
        L = _lib.load()
        self.p, self.z0, self.nz_local = p, int(z0), int(nz_local)
        if alpha.dtype != torch.float32 or not alpha.is_cuda or alpha.numel() != p.nx * p.ny * (nz_local + 2):
            raise ValueError("alpha must be a CUDA float32 tensor of the slab with its halo planes")
        self.alpha = alpha.contiguous()
        self._cfg = p.to_c(self.alpha.data_ptr())
        nbytes = L.tdgl_slab_workspace_bytes(ctypes.byref(self._cfg), self.z0, self.nz_local)
        if nbytes == 0:
            raise TdglError(-1, "tdgl_slab_workspace_bytes")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.alpha.device)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.alpha.device)
        h = ctypes.c_void_p()
        check(L.tdgl_slab_create(ctypes.byref(self._cfg), self.z0, self.nz_local,
                                 ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                 ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), "tdgl_slab_create")
        self._h, self._L = h, L
        self.shape = (self.nz_local + 2, p.ny, p.nx)

    def close(self):
        if getattr(self, "_h", None):
            self._L.tdgl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ptrs(self):
        sp = _lib.StatePtrs()
        check(self._L.tdgl_get_state(self._h, ctypes.byref(sp)), "tdgl_get_state")
        return sp

    def state(self):
        """(psi complex64, mu float32) views of the slab's state with its halo planes."""
        sp = self._ptrs()
        return (_view(self.workspace, sp.psi, torch.complex64, self.shape),
                _view(self.workspace, sp.mu, torch.float32, self.shape))

    def set_state(self, psi: torch.Tensor, mu: torch.Tensor | None = None):
        """psi, mu: the slab's planes with halos ((nz_local + 2, ny, nx)) on the device."""
        psi = psi.to(device=self.workspace.device, dtype=torch.complex64).contiguous()
        mu_ptr = None
        if mu is not None:
            mu = mu.to(device=self.workspace.device, dtype=torch.float32).contiguous()
            mu_ptr = ctypes.c_void_p(mu.data_ptr())
        check(self._L.tdgl_set_state(self._h, ctypes.c_void_p(psi.data_ptr()), mu_ptr, 0.0), "tdgl_set_state")

    def planes(self, latest: bool):
        arr = (ctypes.c_void_p * 4)()
        check(self._L.tdgl_slab_planes(self._h, int(bool(latest)), arr), "tdgl_slab_planes")
        return tuple(_view(self.workspace, arr[q], torch.complex64, (self.p.ny, self.p.nx)) for q in range(4))

    def sweep(self, first: bool) -> float:
        r2 = ctypes.c_double()
        check(self._L.tdgl_slab_sweep(self._h, int(bool(first)), ctypes.byref(r2)), "tdgl_slab_sweep")
        return r2.value

    def accept(self):
        check(self._L.tdgl_slab_accept(self._h), "tdgl_slab_accept")

    def rhs(self) -> torch.Tensor:
        check(self._L.tdgl_slab_rhs(self._h), "tdgl_slab_rhs")
        sp = self._ptrs()
        return _view(self.workspace, sp.f, torch.float32, self.shape)[1:-1]

    def set_mu(self, mu: torch.Tensor):
        self.state()[1][1:-1].copy_(mu)


class GpuPoisson:
    """The whole grid's Poisson solve on one GPU (a Poisson-only handle): f -> (mu, E_x)."""

    def __init__(self, p, device="cuda", stream=None):
        L = _lib.load()
        self.p = p
        self._cfg = p.to_c(0)
        nbytes = L.tdgl_poisson_workspace_bytes(ctypes.byref(self._cfg))
        if nbytes == 0:
            raise TdglError(-1, "tdgl_poisson_workspace_bytes")
        self.stream = stream if stream is not None else torch.cuda.current_stream(torch.device(device))
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        h = ctypes.c_void_p()
        check(L.tdgl_poisson_create(ctypes.byref(self._cfg), ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                    ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), "tdgl_poisson_create")
        self._h, self._L = h, L

    def close(self):
        if getattr(self, "_h", None):
            self._L.tdgl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ptrs(self):
        sp = _lib.StatePtrs()
        check(self._L.tdgl_get_state(self._h, ctypes.byref(sp)), "tdgl_get_state")
        return sp

    def __call__(self, f: torch.Tensor):
        shape = (self.p.nz, self.p.ny, self.p.nx)
        _view(self.workspace, self._ptrs().f, torch.float32, shape).copy_(f)
        check(self._L.tdgl_solve_mu_f(self._h), "tdgl_solve_mu_f")
        ex = ctypes.c_double()
        check(self._L.tdgl_read_ctl_scalars(self._h, ctypes.byref(ex), None), "tdgl_read_ctl_scalars")
        return _view(self.workspace, self._ptrs().mu, torch.float32, shape), ex.value
