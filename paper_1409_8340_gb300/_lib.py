"""ctypes binding of libtdgl_gb300.so (argument marshalling only).

Every function here forwards to the C ABI declared in include/tdgl.h.  There
is no fallback: if the CUDA library is missing or cannot be loaded, loading
raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtdgl_gb300.so")

PERIODIC = 0
OPEN = 1
LINKS_LANDAU = 0
LINKS_GENERAL = 1
LINKS_XZ = 2

TDGL_OK = 0
TDGL_ERR_INVALID_ARG = -1
TDGL_ERR_NOT_CONVERGED = -2
TDGL_ERR_NONFINITE = -3
TDGL_ERR_TIMEOUT = -4
TDGL_ERR_CUDA = -5
TDGL_ERR_WORKSPACE = -6

ERRORS = {0: "ok", -1: "invalid argument", -2: "not converged", -3: "non-finite residual", -4: "timeout",
          -5: "CUDA error", -6: "workspace"}


class TdglError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, 'unknown')} ({code})")


class Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("bc", ctypes.c_int32 * 3),
        ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double),
        ("g", ctypes.c_double), ("u", ctypes.c_double), ("beta", ctypes.c_double), ("ht", ctypes.c_double),
        ("By", ctypes.c_double), ("Bz", ctypes.c_double),
        ("Jext", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("max_iter", ctypes.c_int32),
        ("check_every", ctypes.c_int32),
        ("fixed_sweeps", ctypes.c_int32),
        ("freeze_mu_K", ctypes.c_int32),
        ("poisson_cycles", ctypes.c_int32),
        ("poisson_max_cycles", ctypes.c_int32),
        ("poisson_tol", ctypes.c_double),
        ("links_mode", ctypes.c_int32),
        ("sweeps_per_pass", ctypes.c_int32), ("noise_T", ctypes.c_double), ("noise_seed", ctypes.c_uint64),
        ("Bx", ctypes.c_double),
        ("d_alpha", ctypes.c_void_p),
        ("d_link_phase", ctypes.c_void_p),
        ("d_insulating", ctypes.c_void_p),
        ("sweep_kernel", ctypes.c_int32), ("poisson_guess", ctypes.c_int32),
    ]


class Obs(ctypes.Structure):
    _fields_ = [
        ("psi2_mean", ctypes.c_double), ("energy", ctypes.c_double), ("javg", ctypes.c_double),
        ("K", ctypes.c_double), ("Ex", ctypes.c_double),
        ("vortex_unsigned", ctypes.c_double), ("vortex_signed", ctypes.c_double),
        ("last_r2", ctypes.c_double), ("poisson_res", ctypes.c_double),
        ("last_sweeps", ctypes.c_int32), ("poisson_cycles", ctypes.c_int32), ("step", ctypes.c_int64),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class StatePtrs(ctypes.Structure):
    _fields_ = [("psi", ctypes.c_void_p), ("mu", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("D", ctypes.c_void_p), ("f", ctypes.c_void_p)]


class Profile(ctypes.Structure):
    _fields_ = [("ms_init", ctypes.c_double), ("ms_sweeps", ctypes.c_double), ("ms_K", ctypes.c_double),
                ("ms_poisson", ctypes.c_double), ("steps", ctypes.c_int64), ("sweeps", ctypes.c_int64),
                ("sweep_launches", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("vcycles", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class AdjointConfig(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int32), ("checkpoint_every", ctypes.c_int32), ("window_start", ctypes.c_int32),
                ("adj_max_iter", ctypes.c_int32), ("adj_eps", ctypes.c_double), ("poisson_cycles", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("poisson_tol", ctypes.c_double)]


class AdjointStats(ctypes.Structure):
    _fields_ = [("ms_forward", ctypes.c_double), ("ms_recompute", ctypes.c_double), ("ms_reverse", ctypes.c_double),
                ("adjoint_sweeps", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


BATCH_MAX = 256
BATCH_OPS = ("init", "sweep", "javg", "rhs", "smooth", "residual", "restrict", "coarse_fwd", "coarse_conv",
             "coarse_inv", "prolong", "mean", "shift")


class BatchTuning(ctypes.Structure):
    _fields_ = [("blocks_per_sm", ctypes.c_int32), ("graph_steps", ctypes.c_int32), ("timeout_ms", ctypes.c_int32),
                ("test_extra_arrivals", ctypes.c_int32), ("sweep_kernel", ctypes.c_int32),
                ("kz", ctypes.c_int32 * BATCH_MAX)]


class BatchStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("sweeps", ctypes.c_int64), ("site_iters", ctypes.c_double),
                ("grid_blocks", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class BatchTuneReport(ctypes.Structure):
    _fields_ = [("ms_default", ctypes.c_double), ("ms_best", ctypes.c_double), ("candidates", ctypes.c_int32),
                ("classes", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# Pattern generator, full form (include/tdgl.h, tdgl_pattern_ex)
SHAPE_ELLIPSOID, SHAPE_CUBOID, SHAPE_CYLINDER, SHAPE_CROSS, SHAPE_OCTANT = 0, 1, 2, 3, 4
SHAPE_INVERT, SHAPE_INSULATING = 1, 2
LATTICE_SQUARE, LATTICE_TRIANGULAR, LATTICE_HONEYCOMB, LATTICE_KAGOME = 0, 1, 2, 3
LATTICE_RECTANGULAR, LATTICE_HEXAGONAL = 4, 5
BG_CONSTANT, BG_CHECKER, BG_VORONOI = 0, 1, 2
METRIC_EUCLIDEAN, METRIC_ABSOLUTE, METRIC_MAXIMUM = 0, 1, 2


class Shape(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("flags", ctypes.c_int32), ("c", ctypes.c_double * 3),
                ("a", ctypes.c_double * 3), ("q", ctypes.c_double * 4), ("value", ctypes.c_double)]


class Lattice(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("count", ctypes.c_int32 * 3), ("origin", ctypes.c_double * 3),
                ("spacing", ctypes.c_double * 3), ("motif", Shape)]


class Background(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("metric", ctypes.c_int32), ("value", ctypes.c_double),
                ("cell", ctypes.c_double * 3), ("values", ctypes.c_double * 2), ("p_odd", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("host_seeds", ctypes.c_void_p), ("n_seeds", ctypes.c_int64)]


class TuneReport(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 3), ("chosen", ctypes.c_int32), ("candidates", ctypes.c_int32)]


# order of tdgl_abi_struct_size's argument
ABI_STRUCTS = (Config, Obs, StatePtrs, Profile, AdjointConfig, AdjointStats, BatchTuning, BatchStats,
               BatchTuneReport, Shape, Lattice, Background, TuneReport)

# name -> (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "tdgl_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "tdgl_abi_struct_size": (ctypes.c_size_t, [ctypes.c_int32]),
    "tdgl_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(Config)]),
    "tdgl_create": (ctypes.c_int, [ctypes.POINTER(Config), _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    "tdgl_destroy": (None, [_P]),
    "tdgl_set_state": (ctypes.c_int, [_P, _P, _P, ctypes.c_double]),
    "tdgl_upload_state": (ctypes.c_int, [_P, _P, _P, ctypes.c_double]),
    "tdgl_download_state": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "tdgl_get_state": (ctypes.c_int, [_P, ctypes.POINTER(StatePtrs)]),
    "tdgl_set_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "tdgl_get_mu_prev": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "tdgl_slab_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(Config), ctypes.c_int32, ctypes.c_int32]),
    "tdgl_slab_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_size_t, _P,
                                        ctypes.POINTER(_P)]),
    "tdgl_slab_sweep": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "tdgl_slab_accept": (ctypes.c_int, [_P]),
    "tdgl_slab_planes": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    "tdgl_slab_rhs": (ctypes.c_int, [_P]),
    "tdgl_poisson_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(Config)]),
    "tdgl_poisson_create": (ctypes.c_int, [ctypes.POINTER(Config), _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    "tdgl_solve_mu_f": (ctypes.c_int, [_P]),
    "tdgl_read_ctl_scalars": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "tdgl_set_mu_prev": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "tdgl_step": (ctypes.c_int, [_P, ctypes.c_int]),
    "tdgl_step_resident": (ctypes.c_int, [_P, ctypes.c_int32]),
    "tdgl_step_enqueue": (ctypes.c_int, [_P, ctypes.c_int32]),
    "tdgl_sync": (ctypes.c_int, [_P]),
    "tdgl_autotune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(TuneReport)]),
    "tdgl_solve_psi": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "tdgl_solve_mu": (ctypes.c_int, [_P]),
    "tdgl_observables": (ctypes.c_int, [_P, ctypes.POINTER(Obs)]),
    "tdgl_adjoint_workspace_bytes": (ctypes.c_size_t, [_P, ctypes.POINTER(AdjointConfig)]),
    "tdgl_adjoint": (ctypes.c_int, [_P, ctypes.POINTER(AdjointConfig), _P, ctypes.c_size_t, _P,
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(AdjointStats)]),
    "tdgl_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "tdgl_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(Profile)]),
    "tdgl_test_staged_waits": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32]),
    "tdgl_sweep_noalloc": (ctypes.c_int, [ctypes.POINTER(Config), _P, _P, _P, ctypes.c_double, _P,
                                          ctypes.POINTER(ctypes.c_double), _P]),
    "tdgl_batch_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(Config), ctypes.c_int32]),
    "tdgl_batch_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int32, _P, ctypes.c_size_t, _P,
                                         ctypes.POINTER(_P)]),
    "tdgl_batch_destroy": (None, [_P]),
    "tdgl_batch_instance": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(_P)]),
    "tdgl_batch_step": (ctypes.c_int, [_P, ctypes.c_int32]),
    "tdgl_batch_status": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "tdgl_batch_observables": (ctypes.c_int, [_P, ctypes.POINTER(Obs)]),
    "tdgl_batch_stats_read": (ctypes.c_int, [_P, ctypes.POINTER(BatchStats), ctypes.POINTER(ctypes.c_int64)]),
    "tdgl_batch_get_tuning": (ctypes.c_int, [_P, ctypes.POINTER(BatchTuning)]),
    "tdgl_batch_set_tuning": (ctypes.c_int, [_P, ctypes.POINTER(BatchTuning)]),
    "tdgl_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(BatchTuneReport)]),
    "tdgl_batch_phase_log": (ctypes.c_int, [_P, ctypes.c_int32]),
    "tdgl_batch_phase_read": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                                             ctypes.c_int32]),
    "tdgl_batch_phase_list": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                                             ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "tdgl_pattern_scratch_bytes": (ctypes.c_size_t, [ctypes.POINTER(Config), ctypes.c_int64]),
    "tdgl_pattern_ex_scratch_bytes": (ctypes.c_size_t, [ctypes.POINTER(Config), ctypes.c_int64, _P, ctypes.c_int32,
                                                        ctypes.POINTER(Background)]),
    "tdgl_pattern_ex": (ctypes.c_int, [ctypes.POINTER(Config), _P, ctypes.c_int64, _P, ctypes.c_int32,
                                       ctypes.POINTER(Background), ctypes.c_int64, _P, _P, _P, ctypes.c_size_t, _P,
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "tdgl_pattern": (ctypes.c_int, [ctypes.POINTER(Config), _P, ctypes.c_int64, ctypes.c_int64, ctypes.c_float,
                                    ctypes.c_float, _P, _P, ctypes.c_size_t, _P, ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_int64)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises OSError when it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError(f"CUDA library not built: {path} (run paper_1409_8340_gb300/build.py)")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        for which, cls in enumerate(ABI_STRUCTS):
            if L.tdgl_abi_struct_size(which) != ctypes.sizeof(cls):
                raise OSError(f"{cls.__name__}: binding layout ({ctypes.sizeof(cls)} bytes) differs from "
                              f"the library's ({L.tdgl_abi_struct_size(which)} bytes)")
        _lib = L
    return _lib


def check(code: int, where: str):
    if code != 0:
        raise TdglError(code, where)
