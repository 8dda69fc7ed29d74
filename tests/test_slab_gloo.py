"""The z-slab decomposition's host logic on two processes (gloo, CPU).

paper_1409_8340_gb300.slab.SlabStep moves the halo planes between slabs (within a
process and between processes), takes the convergence decision on the maximum of
the slabs' residuals over the job (Eq. convergence), gathers the Poisson right-hand
side on rank 0 and scatters the potential back.  Here each slab computes with the
FP64 oracle (init, sweep and residual of its planes between the two halo planes;
the right-hand side of its planes), rank 0 solves the whole grid's Poisson equation
with the oracle's exact solve, and the run must equal the oracle's undivided steps
bit for bit: psi, mu, the sweep counts and E_x.  Two processes with two slabs each
exercise both kinds of halo copy (inside a process and between processes) and the
periodic wrap.
"""
import os
import socket

import numpy as np
import pytest

P, OP = 0, 1
NX, NY, NZ, SLABS_PER_RANK, WORLD, STEPS = 16, 12, 8, 2, 2, 4


def grid(O, nz):
    return O.Grid(NX, NY, nz, bc=(OP, P, P), Bz=0.3, Jext=0.02)


def inputs():
    from paper_1409_8340_gb300 import inputs as I
    u = I.uniform(71, "slab.alpha", NX * NY * NZ).reshape(NZ, NY, NX)
    alpha = np.where(u < 0.1, -1.0, 1.0)
    psi0 = I.random_psi(NX, NY, NZ, 72).astype(np.complex128)
    return alpha, psi0


class OracleSlab:
    """A slab of the oracle grid: planes z0 .. z0 + n - 1 between two halo planes (a grid of
    n + 2 planes, periodic in z, whose halo planes are only read)."""

    def __init__(self, O, z0, n, alpha, psi0):
        import torch
        self.O, self.z0, self.nz_local = O, z0, n
        self.G = grid(O, n + 2)
        idx = [(z0 - 1 + q) % NZ for q in range(n + 2)]
        self.alpha = alpha[idx].copy()
        self.psi = torch.from_numpy(psi0[idx].copy())          # state with halos
        self.mu = np.zeros((n + 2, NY, NX))
        self.it = None                                          # latest iterate
        self.b = self.D = None

    def planes(self, latest):
        a = self.it if latest else self.psi
        return a[1], a[-2], a[0], a[-1]

    def sweep(self, first):
        import torch
        O = self.O
        if first:
            self.b, self.D = O.init(self.G, self.psi.numpy(), self.mu, self.alpha, 0.0)
            cur = self.psi.numpy()
        else:
            cur = self.it.numpy()
        nxt, _ = O.sweep(self.G, cur, self.b, self.D, 0.0)
        r = O.residual(self.G, cur, self.b, self.D, 0.0)[1:-1]
        self.it = torch.from_numpy(nxt)
        return float(np.max(r.real ** 2 + r.imag ** 2))

    def accept(self):
        self.psi = self.it.clone()

    def rhs(self):
        import torch
        return torch.from_numpy(self.O.poisson_rhs(self.G, self.psi.numpy(), 0.0)[1:-1].copy())

    def set_mu(self, mu):
        self.mu[1:-1] = mu.numpy()


def _worker(rank, port, out_dir):
    import torch
    import torch.distributed as dist

    from oracle import oracle as O
    from paper_1409_8340_gb300.slab import SlabStep, TorchComm
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        alpha, psi0 = inputs()
        n = NZ // (WORLD * SLABS_PER_RANK)
        slabs = [OracleSlab(O, (rank * SLABS_PER_RANK + q) * n, n, alpha, psi0) for q in range(SLABS_PER_RANK)]
        G = grid(O, NZ)

        def poisson(f):
            mu = O.poisson_solve(G, f.numpy())
            return torch.from_numpy(mu), O.voltage_open_x(G, mu)

        stepper = SlabStep(slabs, TorchComm(), eps=1e-7, poisson=poisson if rank == 0 else None)
        rec = [stepper.step() for _ in range(STEPS)]
        psi = np.concatenate([s.psi.numpy()[1:-1] for s in slabs])
        mu = np.concatenate([s.mu[1:-1] for s in slabs])
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), psi=psi, mu=mu, sweeps=[r[0] for r in rec],
                 ex=[r[1] for r in rec])
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_process_slab_step_equals_the_undivided_oracle(O, tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_worker, args=(_free_port(), str(tmp_path)), nprocs=WORLD, join=True)
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(WORLD)]
    psi = np.concatenate([r["psi"] for r in res])
    mu = np.concatenate([r["mu"] for r in res])
    alpha, psi0 = inputs()
    G = grid(O, NZ)
    st = O.State(psi0.copy(), np.zeros((NZ, NY, NX)))
    sweeps, ex = [], []
    for _ in range(STEPS):
        s = O.step(G, st, alpha, eps=1e-7)
        sweeps.append(s.sweeps)
        ex.append(s.Ex)
    for r in res:
        assert list(r["sweeps"]) == sweeps
        assert list(r["ex"]) == ex
    np.testing.assert_array_equal(psi, st.psi)
    np.testing.assert_array_equal(mu, st.mu)
