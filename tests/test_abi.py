"""The C ABI library loads and exports every entry point include/tdgl.h declares,
and host-side validation rejects bad configurations (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1409_8340_gb300 import build
    build.build()
    from paper_1409_8340_gb300 import _lib
    return _lib.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tdgl.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tdgl_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layouts_match_the_library(lib):
    from paper_1409_8340_gb300 import _lib
    for which, cls in enumerate(_lib.ABI_STRUCTS):
        assert lib.tdgl_abi_struct_size(which) == ctypes.sizeof(cls), cls.__name__
    assert lib.tdgl_abi_struct_size(len(_lib.ABI_STRUCTS)) == 0
    assert lib.tdgl_abi_struct_size(-1) == 0


def _cfg(**kw):
    from paper_1409_8340_gb300.solver import Params
    p = Params(32, 16, 8)
    for k, v in kw.items():
        setattr(p, k, v)
    return p.to_c(d_alpha=0x1000)


def test_workspace_size_and_validation(lib):
    from paper_1409_8340_gb300._lib import Config
    good = _cfg(bc=(1, 0, 0), Bz=0.1)
    assert lib.tdgl_workspace_bytes(ctypes.byref(good)) > 8 * 3 * 32 * 16 * 8
    bad = [
        _cfg(nx=1), _cfg(hx=0.0), _cfg(ht=-0.1), _cfg(max_iter=0), _cfg(check_every=0),
        _cfg(bc=(0, 0, 0), Bz=0.1),            # periodic x and y need whole flux quanta
        _cfg(bc=(2, 0, 0)), _cfg(poisson_cycles=0),
    ]
    for c in bad:
        assert lib.tdgl_workspace_bytes(ctypes.byref(c)) == 0
        h = ctypes.c_void_p()
        assert lib.tdgl_create(ctypes.byref(c), ctypes.c_void_p(0x100000), 1 << 30, None, ctypes.byref(h)) == -1
    nul = _cfg(bc=(1, 0, 0))
    nul.d_alpha = None
    assert lib.tdgl_workspace_bytes(ctypes.byref(nul)) == 0


def test_xz_gauge_validation(lib):
    import math
    ok = [
        _cfg(xz_gauge=True, bc=(1, 1, 1), Bx=0.3, Bz=0.2),                 # open y: no wrap, no quantisation
        _cfg(xz_gauge=True, bc=(0, 1, 0), Bx=0.3, Bz=0.2),                 # periodic x without y wrap: any field
        _cfg(xz_gauge=True, bc=(0, 0, 1), Bz=2 * math.pi * 3 / (16 * 8), Bx=0.4),
        _cfg(xz_gauge=True, bc=(1, 0, 0), Bz=0.2, Bx=2 * math.pi * 1 / (8 * 4)),
    ]
    for c in ok:
        assert lib.tdgl_workspace_bytes(ctypes.byref(c)) > 3 * 8 * 32 * 16 * 8
    bad = [
        _cfg(xz_gauge=True, bc=(0, 0, 1), Bz=0.2),                         # Bz Lx Ly not 2 pi n
        _cfg(xz_gauge=True, bc=(1, 0, 0), Bx=0.3),                         # Bx Ly Lz not 2 pi n
        _cfg(xz_gauge=True, bc=(1, 1, 1), By=0.1),                         # the xz gauge has no By
        _cfg(bc=(1, 1, 1), Bx=0.1),                                        # the yz gauge has no Bx
        _cfg(bc=(1, 1, 1), Bx=float("nan")),
    ]
    for c in bad:
        assert lib.tdgl_workspace_bytes(ctypes.byref(c)) == 0
    # the batch takes yz Landau links only
    c = (type(ok[0]) * 1)(ok[0])
    assert lib.tdgl_batch_workspace_bytes(c, 1) == 0


def test_insulating_validation(lib):
    good = _cfg(bc=(1, 0, 0), Bz=0.1)
    good.d_insulating = 0x2000
    assert lib.tdgl_workspace_bytes(ctypes.byref(good)) > lib.tdgl_workspace_bytes(ctypes.byref(_cfg(bc=(1, 0, 0))))
    odd = _cfg(nx=33, bc=(1, 0, 0))
    odd.d_insulating = 0x2000
    gen = _cfg(bc=(1, 0, 0), general_links=True)
    gen.d_link_phase = 0x3000
    gen.d_insulating = 0x2000
    for c in (odd, gen):
        assert lib.tdgl_workspace_bytes(ctypes.byref(c)) == 0
    arr = (type(good) * 1)(good)
    assert lib.tdgl_batch_workspace_bytes(arr, 1) == 0


def test_workspace_errors_before_device_work(lib):
    c = _cfg(bc=(1, 0, 0), Bz=0.1)
    h = ctypes.c_void_p()
    n = lib.tdgl_workspace_bytes(ctypes.byref(c))
    assert lib.tdgl_create(ctypes.byref(c), ctypes.c_void_p(0x100001), n, None, ctypes.byref(h)) == -6
    assert lib.tdgl_create(ctypes.byref(c), ctypes.c_void_p(0x100000), n - 1, None, ctypes.byref(h)) == -6
    assert lib.tdgl_error_string(-2).decode().startswith("Jacobi")


def test_batch_validation_before_device_work(lib):
    from paper_1409_8340_gb300._lib import Config
    good = [_cfg(bc=(1, 0, 0), Bz=0.1), _cfg(nx=16, ny=16, nz=4, bc=(1, 0, 0), Bz=0.2, Jext=0.01)]
    arr = (Config * 2)(*good)
    n = lib.tdgl_batch_workspace_bytes(arr, 2)
    assert n > lib.tdgl_workspace_bytes(ctypes.byref(good[0])) + lib.tdgl_workspace_bytes(ctypes.byref(good[1]))
    assert lib.tdgl_batch_workspace_bytes(arr, 0) == 0
    assert lib.tdgl_batch_workspace_bytes(arr, 257) == 0
    for bad in (_cfg(nx=33, bc=(1, 0, 0)),                 # the batched sweep pairs x sites
                _cfg(bc=(1, 0, 0), poisson_tol=1e-6),     # fixed V-cycles only
                _cfg(bc=(1, 0, 0), general_links=True)):
        if bad.links_mode == 1:
            bad.d_link_phase = 0x2000
        one = (Config * 1)(bad)
        assert lib.tdgl_batch_workspace_bytes(one, 1) == 0
        b = ctypes.c_void_p()
        assert lib.tdgl_batch_create(one, 1, ctypes.c_void_p(0x100000), 1 << 30, None, ctypes.byref(b)) == -1
    b = ctypes.c_void_p()
    assert lib.tdgl_batch_create(arr, 2, ctypes.c_void_p(0x100001), n, None, ctypes.byref(b)) == -6
    assert lib.tdgl_batch_create(arr, 2, ctypes.c_void_p(0x100000), n - 1, None, ctypes.byref(b)) == -6


def test_slab_and_poisson_only_workspaces_validate_on_the_host(lib):
    """The z-slab handles need a grid periodic in z, open in x, Landau links, even nx, no
    noise, and a slab inside the grid; the Poisson-only handle reads no alpha."""
    good = _cfg(nx=32, ny=16, nz=12, bc=(1, 0, 0), Bz=0.1)
    assert lib.tdgl_slab_workspace_bytes(ctypes.byref(good), 4, 4) > 0
    assert lib.tdgl_slab_workspace_bytes(ctypes.byref(good), 8, 4) > 0
    bad = [(good, 10, 4), (good, 0, 0), (good, -1, 4),
           (_cfg(nx=32, ny=16, nz=12, bc=(1, 0, 1), Bz=0.1), 0, 4),      # open z
           (_cfg(nx=33, ny=16, nz=12, bc=(1, 0, 0), Bz=0.1), 0, 4),      # odd nx
           (_cfg(nx=32, ny=16, nz=12, bc=(1, 0, 0), Bz=0.1, noise_T=0.01), 0, 4)]
    for c, z0, n in bad:
        assert lib.tdgl_slab_workspace_bytes(ctypes.byref(c), z0, n) == 0, (z0, n)
    pc = _cfg(nx=32, ny=16, nz=12, bc=(1, 0, 0), Bz=0.1)
    pc.d_alpha = None
    full = lib.tdgl_workspace_bytes(ctypes.byref(_cfg(nx=32, ny=16, nz=12, bc=(1, 0, 0), Bz=0.1)))
    assert 0 < lib.tdgl_poisson_workspace_bytes(ctypes.byref(pc)) < full - 40 * 32 * 16 * 12 + 4096
