"""Benchmark of the implicit TDGL time step on GB300.

Workload (default): the 512 x 512 x 256 mesoscopic sample -- open x, periodic
y and z, Bz = 0.2, random ellipsoidal inclusions (semi-axes U[1.5, 5] xi,
random orientation) to 10 % volume, alpha = +1 / -1, one increment of the
current sweep (J = 0.025), h = 0.5, h_t = 0.1, eps = 1e-6.  Synthetic seeded
inputs; the state is relaxed for a number of untimed steps before timing.

A step is one full time step: fused init + Jacobi sweeps to convergence
(residual reductions included), voltage, Poisson right-hand side, multigrid
V-cycles and zero-mode projection.  `value` is Jacobi site-updates per second
over whole steps (Gsite-iter/s), inputs resident in HBM; each array (512 MiB
per complex64 field) is far larger than the 129 MB L2, so no flush is needed.

Multi-GPU: every rank advances its own replica (weak scaling, no collective on
the data path); value = all ranks' site-updates / max-over-ranks time.

--impl reference times the FP64 CPU oracle on the host cores instead, each
step being one oracle time step on a bounded slab of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gsite-iter/s"
BYTES_PER_SITE_ITER = 32          # read psi 8 + b 8 + D 8, write psi 8
# the rest of a default time step, per site: the init (read psi 8, mu 4, alpha 4, the
# previous mu on half the rows 2; write b 8, D 8, psi 8, the Poisson guess on half the
# rows 2) and the Poisson solve (right-hand side 12; per multigrid level and site of it:
# four smoothing passes of 6, residual and restriction 9, prolongation 5, summed over the
# levels' 1 + 1/4 + 1/16 + ... = 4/3: 51)
INIT_BYTES_PER_SITE = 44
POISSON_BYTES_PER_SITE = 63
SLAB_NZ = 8                       # CPU sample: full x-y extent, 8 z planes


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--relax", type=int, default=150, help="untimed steps from the random start")
    ap.add_argument("--J", type=float, default=0.025)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-modes", action="store_true", help="skip the batched and adjoint measurements")
    ap.add_argument("--batch-steps", type=int, default=30)
    ap.add_argument("--batch-relax", type=int, default=20)
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default kernels (no sweep or batch autotuning); for profiling captures")
    ap.add_argument("--only", default="all", choices=["all", "batched", "adjoint", "xz", "pattern", "insulating"],
                    help="run one mode alone and print its dictionary (profiling captures)")
    # profiling captures only (a number printed with these changed is not a bench value)
    ap.add_argument("--nz", type=int, default=256, help="z planes of the grid (profiling captures: a smaller case)")
    ap.add_argument("--fixed-sweeps", type=int, default=0, help="exactly this many sweeps per step (profiling)")
    ap.add_argument("--sweep-kernel", type=int, default=0, choices=[0, 1, 2],
                    help="Jacobi sweep kernel: 1 register-tiled, 2 staged in shared memory, 0 library default")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("k_sweep_tma.cu", "sweep_tile.cuh", "tma_util.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1409_8340_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profile():
    """dram bytes per sweep launch from the committed ncu summary, if it was taken
    on the current sweep kernel source; None otherwise."""
    path = os.path.join(ROOT, "profiles", "sweep_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return d.get("dram_bytes_per_launch_full_size")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            cmd = ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "100"]
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        for line in open(self.file.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            if self.uuid and parts[1] != self.uuid:
                continue
            rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for n, v in zip(names, r[6:10]):
                if v.lower() == "active":
                    reasons.add(n)
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        pw = [float(r[4]) for r in rows if r[4].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------------------
# workload construction
# ---------------------------------------------------------------------------
def workload(J: float, nz_override: int | None = None):
    from paper_1409_8340_gb300 import inputs
    from paper_1409_8340_gb300.presets import mesoscopic_512x512x256
    w = mesoscopic_512x512x256(J)
    if nz_override is not None:
        p = w.params
        p.nz = nz_override
        box = (p.length(0), p.length(1), p.length(2))
        count = max(200, int(w.candidates.shape[0] * nz_override / 256))
        w.candidates = inputs.ellipsoids(count, box, 1.5, 5.0, seed=w.seed)
        w.target_sites = inputs.target_sites(0.10, p.N)
    return w


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def cpu_oracle_run(J: float, budget_s: float, max_steps: int | None = None, case: str = "slab",
                   threads: int | None = None, warm: bool = True):
    """Time the FP64 oracle on a bounded sample: `slab` = a 512x512x8 slab of the
    512x512x256 workload, `transport` = the 128x128x64 transport workload in full
    size (a bounded number of its steps).  threads: OpenMP threads (None: all).  warm: one
    untimed step first.  Returns (value, info, seconds, steps, sweeps)."""
    import numpy as np

    from oracle import oracle as O
    from paper_1409_8340_gb300 import inputs
    if case == "transport":
        from paper_1409_8340_gb300.presets import transport_128x128x64
        w = transport_128x128x64()
        label = "the 128x128x64 transport workload (full size; open x, periodic y z, Bz 0.1, J 0.01)"
    else:
        w = workload(J, SLAB_NZ)
        label = (f"a 512x512x{SLAB_NZ} slab of the 512x512x256 workload (same h, BCs, field, current, "
                 f"inclusion recipe)")
    p = w.params
    G = O.Grid(p.nx, p.ny, p.nz, hx=p.hx, hy=p.hy, hz=p.hz, bc=tuple(p.bc), Bz=p.Bz, Jext=p.Jext, ht=p.ht)
    alpha, _, _ = O.pattern(G, w.candidates, w.target_sites, w.alpha_in, w.alpha_out)
    n_all = os.cpu_count() or 1
    O.set_threads(threads if threads else n_all)
    st = O.State(inputs.random_psi(p.nx, p.ny, p.nz, w.seed), np.zeros(p.shape))
    if warm:
        O.step(G, st, alpha, eps=p.eps)        # one untimed step (first-touch, build)
    t0 = time.perf_counter()
    sweeps = steps = 0
    while True:
        s = O.step(G, st, alpha, eps=p.eps)
        sweeps += s.sweeps
        steps += 1
        el = time.perf_counter() - t0
        if (max_steps is not None and steps >= max_steps) or (max_steps is None and el >= budget_s):
            break
    used = O.threads()
    O.set_threads(n_all)
    value = sweeps * p.N / el / 1e9
    info = {"value": value, "unit": METRIC, "cores": used, "kind": "oracle",
            "sample": f"{steps} FP64 oracle time steps ({sweeps} Jacobi sweeps) on {label}; "
                      f"{el:.1f} s wall, OpenMP threads = {used}"}
    return value, info, el, steps, sweeps


def cpu_baseline_report(J: float, budget_s: float):
    """The oracle on the host cores: the 512x512x256 slab sample on all cores (the
    headline cpu_baseline), the same on one core, and the 128x128x64 transport workload
    on all cores and on one core; with the CPU model and core count."""
    value, info, _, _, _ = cpu_oracle_run(J, budget_s)
    info["cpu_model"] = cpu_model()
    info["host_cores"] = os.cpu_count()
    _, one, _, _, _ = cpu_oracle_run(J, budget_s / 3, threads=1, warm=False)
    info["one_thread"] = one
    _, tr_all, _, _, _ = cpu_oracle_run(J, budget_s / 3, case="transport")
    _, tr_one, _, _, _ = cpu_oracle_run(J, budget_s / 3, case="transport", threads=1, warm=False)
    info["transport_128x128x64"] = {"all_cores": tr_all, "one_thread": tr_one}
    return value, info


# ---------------------------------------------------------------------------
# batched and adjoint modes, reported against the plain single-instance step
# ---------------------------------------------------------------------------
def batched_mode(dev, steps: int, relax: int = 20, seq_steps: int = 5, autotune: bool = True):
    """The 64-member ensemble of uneven sizes in one persistent launch per step,
    replayed from a CUDA graph, after the autotuner; then the same members
    stepped one after another through plain handles from the same states."""
    import numpy as np
    import torch

    from paper_1409_8340_gb300 import inputs, presets
    from paper_1409_8340_gb300.solver import Batch, Solver, pattern
    members = presets.ensemble_64()
    ps = [w.params for w in members]
    alphas = [pattern(w.params, w.candidates, w.target_sites, w.alpha_in, w.alpha_out, device=dev)[0]
              for w in members]
    b = Batch(ps, alphas)
    for i, s in enumerate(b.instances):
        s.set_state(torch.as_tensor(inputs.random_psi(ps[i].nx, ps[i].ny, ps[i].nz, members[i].seed)
                                    .astype(np.complex64)))
    b.step(relax)
    b.check()
    rep = b.autotune(trial_steps=8) if autotune else None
    tun = b.tuning()
    kz_by_size = {f"{p.nx}x{p.ny}x{p.nz}": kz for p, kz in zip(ps, tun["kz"])}
    b.step(3)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    st0 = b.stats()
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st1 = b.stats()
    rc, _ = b.status()
    # phase breakdown of one more step (logged separately from the timed steps)
    b.phase_log(True)
    b.step(1)
    phases = {k: {"ms": round(v[0], 4), "phases": v[1]} for k, v in b.phase_profile().items() if v[1]}
    plist = b.phase_list()
    by_kind = {}
    for kind, pms in plist:
        by_kind.setdefault(kind, []).append(round(pms, 4))
    b.phase_log(False)
    site_iters = st1["site_iters"] - st0["site_iters"]
    value = site_iters / (ms * 1e-3) / 1e9
    # the same members, one after another, through plain handles from the batch's states
    plain = []
    for i, s in enumerate(b.instances):
        psi, mu = s.state()
        h = Solver(ps[i], alphas[i])
        h.set_state(psi.clone(), mu.clone(), s.observables()["K"])
        plain.append(h)
    for h in plain:
        h.step(1)
        h.profile_enable(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for h in plain:
        h.step(seq_steps)
    torch.cuda.synchronize()
    seq_s = time.perf_counter() - t0
    seq_iters = sum(h.profile()["sweeps"] * h.p.N for h in plain)
    launches = sum(h.profile()["kernel_launches"] for h in plain)
    sizes = {}
    for p in ps:
        sizes[f"{p.nx}x{p.ny}x{p.nz}"] = sizes.get(f"{p.nx}x{p.ny}x{p.nz}", 0) + 1
    return {
        "workload": "ensemble_64: 64 instances from {32^3, 64^3, 96x96x48, 128x128x64}, own seed, Bz in "
                    "[0.05,0.5], alpha scale in [0.5,1], J in [0,0.03], 3-8 % spheres; open x, periodic y z",
        "sizes": sizes, "sites": sum(p.N for p in ps), "steps": steps, "ms_per_step": ms / steps,
        "value": value, "unit": METRIC, "status": rc,
        "sweep_bytes_gbs": BYTES_PER_SITE_ITER * site_iters / (ms * 1e-3) / 1e9,
        "launches_per_step": 1, "graph": st1["graph"], "grid_blocks": st1["grid_blocks"],
        "blocks_per_sm": st1["blocks_per_sm"], "autotune": rep,
        "sweep_tiles": "staged" if tun["sweep_kernel"] == 0 else "register_tiled", "kz_by_size": kz_by_size,
        "phase_ms_one_step": phases,
        "phase_ms_in_order": {k: by_kind[k] for k in ("sweep", "smooth", "residual", "restrict", "prolong")
                              if k in by_kind},
        "sequential_plain": {"value": seq_iters / seq_s / 1e9, "unit": METRIC, "steps": seq_steps,
                             "ms_per_batch_step": 1e3 * seq_s / seq_steps,
                             "launches_per_batch_step": launches / seq_steps},
        "speedup_vs_sequential": value / (seq_iters / seq_s / 1e9),
    }


def adjoint_mode(dev, n_steps: int = 400, every: int = 20, relax: int = 50):
    """Gradient of the time-averaged E_x with respect to alpha on the 64x64x32
    transport case: 400 steps, checkpoints every 20, recompute; against 400 plain
    forward steps from the same state.  Twice: at the library's default tolerances,
    and at the accuracy the gradient is validated at (forward psi solves to
    max|r|^2 < 1e-10, Poisson solves to a relative residual of 1e-6, adjoint solves to
    1e-10 relative)."""
    import dataclasses

    import numpy as np
    import torch

    from paper_1409_8340_gb300 import inputs, presets
    from paper_1409_8340_gb300.solver import Solver
    w = presets.adjoint_64x64x32()

    def run(p, **adj):
        s = Solver(p, torch.as_tensor(w.alpha_field).to(dev))
        s.set_state(torch.as_tensor(inputs.random_psi(p.nx, p.ny, p.nz, w.seed).astype(np.complex64)))
        s.step(relax)
        ck = s.checkpoint()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(n_steps)
        torch.cuda.synchronize()
        fwd_s = time.perf_counter() - t0
        s.restore(ck)
        t0 = time.perf_counter()
        J, grad, st = s.adjoint(n_steps, checkpoint_every=every, **adj)
        torch.cuda.synchronize()
        adj_s = time.perf_counter() - t0
        s.close()
        return {"objective_mean_Ex": J, "grad_norm": float(grad.norm()), "forward_ms": 1e3 * fwd_s,
                "adjoint_total_ms": 1e3 * adj_s,
                "phases_ms": {"forward": st["ms_forward"], "recompute": st["ms_recompute"],
                              "reverse": st["ms_reverse"]},
                "adjoint_sweeps_per_step": st["adjoint_sweeps"] / n_steps,
                "cost_vs_forward": adj_s / fwd_s,
                "reverse_step_vs_forward_step": (st["ms_reverse"] / n_steps) / (1e3 * fwd_s / n_steps)}

    out = {"workload": "adjoint_64x64x32: open x, periodic y z, Bz 0.1, J 0.01, smoothed random alpha in [-1,1]",
           "steps": n_steps, "checkpoint_every": every}
    out["default_tolerances"] = run(w.params)
    tight = dataclasses.replace(w.params, eps=1e-10, poisson_tol=1e-6, poisson_max_cycles=40)
    out["validated_accuracy"] = run(tight, adj_eps=1e-10, poisson_tol=1e-6)
    out["validated_accuracy"]["tolerances"] = "psi max|r|^2 < 1e-10, Poisson relative residual 1e-6, adjoint 1e-10"
    # headline figures of the mode: the default-tolerance run
    out["cost_vs_forward"] = out["default_tolerances"]["cost_vs_forward"]
    out["reverse_step_vs_forward_step"] = out["default_tolerances"]["reverse_step_vs_forward_step"]
    return out


def xz_mode(dev, steps: int = 20, relax: int = 20, quanta_x: int = 600):
    """The mesoscopic workload with the field tilted in the xz plane, B = (Bx, 0, 0.2) with
    Bx Ly Lz = 2 pi * 600 (about 30 degrees from z), in the Landau gauge of Eq. A_xz:
    the link phases vary along y only, so the sweep takes them from j-indexed tables and
    moves the same 32 B/site as in the yz gauge."""
    import math

    import numpy as np
    import torch

    from paper_1409_8340_gb300 import inputs
    from paper_1409_8340_gb300.solver import Solver, pattern
    w = workload(0.025)
    p = w.params
    p.xz_gauge = True
    p.Bx = 2 * math.pi * quanta_x / (p.length(1) * p.length(2))
    alpha, _, _ = pattern(p, w.candidates, w.target_sites, w.alpha_in, w.alpha_out, device=dev)
    s = Solver(p, alpha)
    s.set_state(torch.as_tensor(inputs.random_psi(p.nx, p.ny, p.nz, w.seed).astype(np.complex64)))
    s.step(relax)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    s.profile_enable(True)
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = s.profile()
    s.profile_enable(False)
    obs = s.observables()
    n_plain = prof["sweeps"] - prof["steps"]
    sweep_ms = prof["ms_sweeps"] / max(1, n_plain)
    bpl = BYTES_PER_SITE_ITER * p.N
    peak, peak_kind = measured_peaks()
    del s
    torch.cuda.empty_cache()
    return {"workload": f"mesoscopic_512x512x256 in the xz gauge: B = ({p.Bx:.5f}, 0, {p.Bz}), J 0.025",
            "value": prof["sweeps"] * p.N / (ms * 1e-3) / 1e9, "unit": METRIC, "steps": steps,
            "ms_per_step": ms / steps, "sweeps_per_step": prof["sweeps"] / max(1, prof["steps"]),
            "phase_ms_per_step": {"init_sweep": prof["ms_init"] / steps, "sweeps": prof["ms_sweeps"] / steps,
                                  "K": prof["ms_K"] / steps, "poisson": prof["ms_poisson"] / steps},
            "sweep_roofline": {"kernel": "sweep_tma_kernel<XZ>", "bound": "hbm", "bytes_per_launch": bpl,
                               "avg_launch_ms": sweep_ms, "achieved": bpl / (sweep_ms * 1e-3) / 1e9,
                               "peak": peak, "unit": "GB/s", "frac": bpl / (sweep_ms * 1e-3) / 1e9 / peak,
                               "peak_source": peak_kind},
            "observables": {"Ex": obs["Ex"], "psi2_mean": obs["psi2_mean"],
                            "vortex_unsigned_per_layer": obs["vortex_unsigned"]}}


def insulating_mode(dev, steps: int = 20, relax: int = 20, nz: int = 256):
    """The mesoscopic workload with insulating inclusions (Sec. 3.4 (ii)): the same
    ellipsoids as the metallic ones, every fourth marked insulating (links next to them
    removed), the rest eps = -1; the Poisson solve is 2 CG iterations preconditioned by
    V-cycles per step (warm start).  The tiled sweep reads one link byte per site more
    (33 B/site)."""
    import numpy as np
    import torch

    from paper_1409_8340_gb300 import inputs
    from paper_1409_8340_gb300.solver import Solver, pattern_ex
    w = workload(0.025, None if nz == 256 else nz)
    p = w.params
    p.poisson_cycles = 2          # two CG iterations per step, each preconditioned by a V-cycle
    cand = np.asarray(w.candidates)
    sh = np.zeros((cand.shape[0], 13))
    sh[:, 2:5] = cand[:, 0:3]
    sh[:, 5:8] = cand[:, 3:6]
    sh[:, 8:12] = cand[:, 6:10]
    sh[:, 12] = w.alpha_in
    sh[::4, 1] = 2                                   # insulating
    alpha, ins, used, marked = pattern_ex(p, sh, (), {"kind": 0, "value": w.alpha_out}, w.target_sites,
                                          insulating=True, device=dev)
    s = Solver(p, alpha, insulating=ins)
    s.set_state(torch.as_tensor(inputs.random_psi(p.nx, p.ny, p.nz, w.seed).astype(np.complex64)))
    s.step(relax)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    s.profile_enable(True)
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = s.profile()
    s.profile_enable(False)
    obs = s.observables()
    n_plain = prof["sweeps"] - prof["steps"]
    sweep_ms = prof["ms_sweeps"] / max(1, n_plain)
    bpl = (BYTES_PER_SITE_ITER + 1) * p.N
    peak, peak_kind = measured_peaks()
    frac_ins = float(ins.float().mean())
    del s, alpha, ins
    torch.cuda.empty_cache()
    return {"workload": f"mesoscopic_512x512x{nz} with insulating inclusions (every 4th ellipsoid), J 0.025",
            "insulating_fraction": frac_ins, "inclusion_fraction": marked / p.N,
            "value": prof["sweeps"] * p.N / (ms * 1e-3) / 1e9, "unit": METRIC, "steps": steps,
            "ms_per_step": ms / steps, "sweeps_per_step": prof["sweeps"] / max(1, prof["steps"]),
            "phase_ms_per_step": {"init_sweep": prof["ms_init"] / steps, "sweeps": prof["ms_sweeps"] / steps,
                                  "K": prof["ms_K"] / steps, "poisson": prof["ms_poisson"] / steps},
            "sweep_roofline": {"kernel": "sweep_tma_kernel<MASK>", "bound": "hbm", "bytes_per_launch": bpl,
                               "avg_launch_ms": sweep_ms, "achieved": bpl / (sweep_ms * 1e-3) / 1e9,
                               "peak": peak, "unit": "GB/s", "frac": bpl / (sweep_ms * 1e-3) / 1e9 / peak,
                               "peak_source": peak_kind},
            "observables": {"Ex": obs["Ex"], "psi2_mean": obs["psi2_mean"]}}


def pattern_mode(dev, reps: int = 5):
    """The pattern generator (Sec. 3.4) at 512x512x256 (open x, periodic y z): the
    mesoscopic ellipsoids to 10 % (20 000 candidates), a polycrystalline Voronoi
    background of 20 000 grains, a random checkerboard, and a cylindrical domain mask
    with a kagome lattice of +-45 degree columnar insulating cylinders over the Voronoi
    grains.  Each timed with CUDA events over `reps` runs (the call synchronises)."""
    import math

    import numpy as np
    import torch

    from paper_1409_8340_gb300.solver import pattern, pattern_ex
    w = workload(0.0)
    p = w.params
    rng = np.random.default_rng(33)
    seeds = np.zeros((20000, 4))
    seeds[:, :3] = rng.uniform(0, 1, (20000, 3)) * (p.length(0), p.length(1), p.length(2))
    seeds[:, 3] = rng.uniform(0.5, 1.0, 20000)
    vor = {"kind": 2, "metric": 0, "seeds": seeds}
    dom = [1, 1, 128.0, 128.0, 64.0, 120.0, 120.0, 1e3, 1.0, 0.0, 0.0, 0.0, -1.0]          # inverted cylinder
    q45 = [math.cos(math.pi / 8), 0.0, math.sin(math.pi / 8), 0.0]
    motif = [2, 2, 0.0, 0.0, 0.0, 1.5, 1.5, 60.0] + q45 + [-1.0]
    lat = {"kind": 3, "count": (25, 29, 3), "origin": (2.0, 2.0, 40.0), "spacing": (10.0, 0.0, 40.0), "motif": motif}
    cases = {
        "ellipsoids_10pct": lambda: pattern(p, w.candidates, w.target_sites, w.alpha_in, w.alpha_out, device=dev),
        "voronoi_20000": lambda: pattern_ex(p, None, (), vor, device=dev),
        "random_checkerboard": lambda: pattern_ex(p, None, (), {"kind": 1, "cell": (2.0, 2.0, 2.0),
                                                                "values": (0.5, 1.0), "p_odd": 0.5, "seed": 7},
                                                  device=dev),
        "domain_kagome_columns_voronoi": lambda: pattern_ex(p, [dom], [lat], vor, insulating=True, device=dev),
    }
    out = {}
    for name, fn in cases.items():
        r = fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            r = fn()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        a = r[0]
        out[name] = {"ms": float(np.median(ms)), "gsites_per_s": p.N / (np.median(ms) * 1e-3) / 1e9,
                     "fraction_below_1": float((a < 1.0).float().mean())}
        del r, a
    torch.cuda.empty_cache()
    return {"workload": "pattern generator at 512x512x256, open x, periodic y z", "sites": p.N, "cases": out}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    # warmup steps, then K timed steps (each one oracle step on the slab sample)
    cpu_oracle_run(args.J, 0.0, max_steps=max(1, args.warmup))
    value, info, el, steps, sweeps = cpu_oracle_run(args.J, 0.0, max_steps=args.steps)
    line = {"metric": METRIC, "value": value, "unit": METRIC, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(1, steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"mesoscopic_512x512x256 (CPU slab nz={SLAB_NZ})",
                                            "J": args.J, "grid": [512, 512, SLAB_NZ]},
            "cpu_baseline": info,
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_native(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1409_8340_gb300 import build as B
    from paper_1409_8340_gb300 import inputs
    from paper_1409_8340_gb300.solver import Solver, pattern

    B.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    w = workload(args.J, None if args.nz == 256 else args.nz)
    p = w.params
    p.fixed_sweeps = args.fixed_sweeps
    p.sweep_kernel = args.sweep_kernel
    alpha, used, marked = pattern(p, w.candidates, w.target_sites, w.alpha_in, w.alpha_out, device=dev)
    psi0 = inputs.random_psi(p.nx, p.ny, p.nz, w.seed + rank).astype(np.complex64)
    s = Solver(p, alpha)
    s.set_state(torch.as_tensor(psi0))
    s.step(args.relax)
    # the sweep kernel by timing (staged, register-tiled, two sweeps per pass), from this
    # state and restored after each trial; the timed steps use the choice
    tune = s.autotune(3) if args.fixed_sweeps == 0 and not args.no_autotune else None
    s.step(args.warmup)
    # the device-resident loop's graph is built here, untimed; the timed steps start from
    # a checkpoint, so that the resident loop can repeat exactly the same steps below (the
    # loop runs one sweep per pass: not with two sweeps per pass, nor a fixed sweep count)
    ck = None
    if args.fixed_sweeps == 0 and (tune is None or tune["chosen"] != "two_sweeps_per_pass"):
        s.step_resident(args.warmup)
        ck = s.checkpoint()
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.3)

    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    s.profile_enable(True)
    e0.record(stream)
    s.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    prof = s.profile()
    s.profile_enable(False)
    clk = clocks.stop()
    obs = s.observables()

    # the same steps as one CUDA graph launch with conditional nodes (tdgl_step_resident):
    # the graph is built by the untimed warm-up call (the loop decides convergence on the
    # device, so a fixed sweep count is not run through it)
    resident = None
    if ck is not None:
        resident = resident_mode(s, p, args, stream, ck)

    site_iters = prof["sweeps"] * p.N
    t = torch.tensor([ms, float(site_iters)], dtype=torch.float64, device=dev)
    if dist:
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        tsum = t.clone()
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        ms_max, total_iters = float(tmax[0]), float(tsum[1])
    else:
        ms_max, total_iters = ms, float(site_iters)
    value = total_iters / (ms_max * 1e-3) / 1e9

    # roofline of the dominant kernel: the Jacobi sweep (sweeps 2..n of each step)
    n_plain = prof["sweeps"] - prof["steps"]
    avg_sweep_ms = prof["ms_sweeps"] / max(1, n_plain)
    bytes_per_launch = BYTES_PER_SITE_ITER * p.N
    achieved = bytes_per_launch / (avg_sweep_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    implicit_ms = prof["ms_init"] + prof["ms_sweeps"]

    # end to end through the C ABI with pinned host buffers: upload, step, download
    host_psi = torch.empty(p.shape, dtype=torch.complex64).pin_memory()
    host_mu = torch.empty(p.shape, dtype=torch.float32).pin_memory()
    _, _, K_now = s.download_state(host_psi, host_mu)
    e2e_value = None
    if args.e2e_steps > 0:
        # each step: H2D of the state from pinned memory, one time step, D2H of the new state
        s.profile_enable(True)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            s.upload_state(host_psi, host_mu, K_now)
            s.step(1)
            _, _, K_now = s.download_state(host_psi, host_mu)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        pe = s.profile()
        s.profile_enable(False)
        e2e_iters = pe["sweeps"] * p.N
        e2e_value = e2e_iters * world / e2e_s / 1e9

    modes = {}
    if rank == 0 and world == 1 and not args.no_modes:
        modes["batched"] = batched_mode(dev, args.batch_steps, args.batch_relax, autotune=not args.no_autotune)
        modes["batched"]["vs_plain_step"] = modes["batched"]["value"] / value
        modes["adjoint"] = adjoint_mode(dev)
        modes["xz_gauge"] = xz_mode(dev)
        modes["pattern"] = pattern_mode(dev)
        modes["insulating"] = insulating_mode(dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        _, cpu = cpu_baseline_report(args.J, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": ("mesoscopic_512x512x256" if (args.nz == 256 and args.fixed_sweeps == 0)
                                    else f"profiling case 512x512x{p.nz}, fixed_sweeps={args.fixed_sweeps}"),
                       "grid": [p.nx, p.ny, p.nz], "sites": p.N,
                       "bc": "open x, periodic y z", "Bz": p.Bz, "J": p.Jext, "h": p.hx, "ht": p.ht, "eps": p.eps,
                       "inclusions": {"kind": "ellipsoids", "used": used, "sites": marked,
                                      "fraction": marked / p.N},
                       "relax_steps": args.relax, "poisson_cycles": p.poisson_cycles,
                       "poisson_guess": "2 mu^(n-1) - mu^(n-2)" if p.poisson_guess in (0, 2) else "mu^(n-1)",
                       "l2": "inputs larger than L2 (512 MiB per complex64 array vs 129 MB L2); no flush",
                       "parallelism": f"replicas x{world}"},
            "sweeps_per_step": prof["sweeps"] / max(1, prof["steps"]),
            "phase_ms_per_step": {"init_sweep": prof["ms_init"] / args.steps,
                                  "sweeps": prof["ms_sweeps"] / args.steps, "K": prof["ms_K"] / args.steps,
                                  "poisson": prof["ms_poisson"] / args.steps},
            "implicit_step_gsite_iter_s": site_iters / (implicit_ms * 1e-3) / 1e9 if implicit_ms > 0 else None,
            # the whole step against the bandwidth bound of all its algorithmic bytes
            "step_roofline": step_roofline(p, prof, ms_max / args.steps, peak),
            "roofline": {"kernel": "sweep_tma_kernel" if p.sweep_kernel != 1 else "sweep2_kernel<0>", "bound": "hbm", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                         "bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_sweep_ms,
                         "traffic": traffic_from_profile()},
            "e2e": {"value": e2e_value, "unit": METRIC, "steps": args.e2e_steps,
                    "h2d_bytes_per_step": 12 * p.N, "d2h_bytes_per_step": 12 * p.N + 128},
            "gpu_launches": prof["kernel_launches"],
            "resident_step": dict(resident, vs_host_step=resident["value"] / value) if resident else None,
            "sweep_autotune": tune,
            "clocks": clk,
            "observables": {"Ex": obs["Ex"], "psi2_mean": obs["psi2_mean"],
                            "vortex_unsigned_per_layer": obs["vortex_unsigned"], "last_sweeps": obs["last_sweeps"],
                            "poisson_res": obs["poisson_res"], "poisson_cycles": obs["poisson_cycles"]},
            "cpu_baseline": cpu,
        }
        line.update(modes)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def step_roofline(p, prof, ms_step, peak):
    """Algorithmic bytes of one default step (init, the sweeps after it, the Poisson
    solve) over the step's time, against the measured copy bandwidth."""
    sweeps = prof["sweeps"] / max(1, prof["steps"])
    per_site = INIT_BYTES_PER_SITE + BYTES_PER_SITE_ITER * (sweeps - 1) + POISSON_BYTES_PER_SITE
    gbs = per_site * p.N / (ms_step * 1e-3) / 1e9
    return {"bound": "hbm", "bytes_per_site_step": per_site, "achieved": gbs, "peak": peak, "unit": "GB/s",
            "frac": gbs / peak}


def resident_mode(s, p, args, stream, ck):
    """The timed steps again, from the same checkpoint (so the same steps, bit for bit),
    through tdgl_step_resident: one graph launch (conditional nodes for the sweep loop and
    the buffer choices) and one synchronisation."""
    import torch
    s.restore(ck)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    s.profile_enable(True)      # counters only: the resident loop records no phase events
    e0.record(stream)
    s.step_resident(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    pr = s.profile()
    s.profile_enable(False)
    return {"value": pr["sweeps"] * p.N / (ms * 1e-3) / 1e9, "unit": METRIC, "ms_per_step": ms / args.steps,
            "sweeps_per_step": pr["sweeps"] / max(1, pr["steps"]), "gpu_launches": pr["kernel_launches"],
            "graph_launches": 1, "host_syncs": 1, "same_steps_as_host_timed": True}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.only != "all":
        import torch

        from paper_1409_8340_gb300 import build as B
        B.build()
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        if args.only == "batched":
            out = batched_mode(dev, args.batch_steps, args.batch_relax, autotune=not args.no_autotune)
        elif args.only == "xz":
            out = xz_mode(dev)
        elif args.only == "pattern":
            out = pattern_mode(dev)
        elif args.only == "insulating":
            out = insulating_mode(dev, min(args.steps, 20), min(args.relax, 20), args.nz)
        else:
            out = adjoint_mode(dev)
        print(json.dumps({"mode": args.only, **out}), flush=True)
        return 0
    return run_native(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
