"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads, and
exports every entry point include/afns.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "afns.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(af[a-z0-9_]*)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2609_29081_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("af_create", "af_set_state", "af_step", "af_advance", "af_get_state", "af_dt_max",
              "af_residual", "af_destroy"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_binding_names_match_header():
    from paper_2609_29081_b300 import _native
    declared = set(declared_symbols())
    bound = set(_native.EXPORTED) | set(_native.BATCH_EXPORTED)
    # every entry point the header declares has a binding, and the binding names
    # nothing the header does not declare
    assert declared == bound, (sorted(declared - bound), sorted(bound - declared))


def test_defaults_and_argument_checks_without_gpu(lib):
    """Host-only entry points: defaults and argument validation need no GPU."""
    from paper_2609_29081_b300 import _native as N
    L = N.load()
    o = N.Opts()
    assert L.af_opts_default(2, ctypes.byref(o)) == N.AF_OK
    assert o.cfl_c == pytest.approx(0.52) and o.cfl_v == 0.13 and o.eps == 1e-13
    assert o.limiter == N.LIM_S_PP and o.max_halvings == 30
    assert L.af_opts_default(3, ctypes.byref(o)) == N.AF_EINVAL
    g = N.Grid()
    g.dim, g.n[0], g.n[1] = 2, 64, 32
    g.lo[0], g.lo[1], g.hi[0], g.hi[1] = 0, 0, 1, 1
    nb = ctypes.c_size_t(0)
    assert L.af_workspace_bytes(ctypes.byref(g), None, ctypes.byref(nb)) == N.AF_OK
    assert nb.value > 5 * 16 * 64 * 32 * 8
    b = N.BC()
    ctx = ctypes.c_void_p()
    # a periodic side without a periodic partner is rejected before any device call
    b.side[0], b.side[1] = 0, 1
    st = L.af_create(ctypes.byref(g), 1.4, 0.01, 0.72, ctypes.byref(b), None, None, None, 0, ctypes.byref(ctx))
    assert st == N.AF_EINVAL and not ctx.value
    assert b"periodic" in L.af_last_error(None)   # the refusal is described, nothing printed
    g.n[0] = 3
    b.side[1] = 0
    st = L.af_create(ctypes.byref(g), 1.4, 0.01, 0.72, ctypes.byref(b), None, None, None, 0, ctypes.byref(ctx))
    assert st == N.AF_EINVAL
    # exact boundary data (AF_BC_EXACT = 4) exist only in 1D
    g.n[0] = 64
    b.side[0] = b.side[1] = 4
    b.side[2] = b.side[3] = 2
    st = L.af_create(ctypes.byref(g), 1.4, 0.01, 0.75, ctypes.byref(b), None, None, None, 0, ctypes.byref(ctx))
    assert st == N.AF_EINVAL and not ctx.value
    assert L.af_opts_default(1, ctypes.byref(o)) == N.AF_OK
    assert o.ex_M0 == 3.0 and o.ex_uinf == 0.2 and o.cfl_v == pytest.approx(0.33)
    # the stage kernel's CTA size: 128 (default) or 256; anything else is refused
    assert L.af_opts_default(2, ctypes.byref(o)) == N.AF_OK and o.threads == 128
    b.side[0] = b.side[1] = b.side[2] = b.side[3] = 0
    o.threads = 64
    st = L.af_create(ctypes.byref(g), 1.4, 0.01, 0.72, ctypes.byref(b), ctypes.byref(o), None, None, 0,
                     ctypes.byref(ctx))
    assert st == N.AF_EINVAL and not ctx.value
    assert o.kappa_off == 0
    o.threads, o.kappa_off = 128, 2
    st = L.af_create(ctypes.byref(g), 1.4, 0.01, 0.72, ctypes.byref(b), ctypes.byref(o), None, None, 0,
                     ctypes.byref(ctx))
    assert st == N.AF_EINVAL and not ctx.value
    # a moving wall is two-dimensional and needs a finite speed
    o.kappa_off = 0
    g1 = N.Grid()
    g1.dim, g1.n[0], g1.n[1] = 1, 32, 1
    g1.lo[0], g1.hi[0] = 0.0, 1.0
    b.side[0], b.side[1] = 5, 3
    st = L.af_create(ctypes.byref(g1), 1.4, 0.01, 0.72, ctypes.byref(b), None, None, None, 0, ctypes.byref(ctx))
    assert st == N.AF_EINVAL and not ctx.value
    b.side[0], b.side[1], b.side[2], b.side[3] = 1, 1, 1, 5
    b.wall_speed[3] = float("nan")
    st = L.af_create(ctypes.byref(g), 1.4, 0.01, 0.72, ctypes.byref(b), None, None, None, 0, ctypes.byref(ctx))
    assert st == N.AF_EINVAL and not ctx.value
    # a grid whose per-site element index would leave 32 bits is refused up front
    b.side[0] = b.side[1] = b.side[2] = b.side[3] = 0
    g.n[0], g.n[1] = 50000, 50000
    st = L.af_create(ctypes.byref(g), 1.4, 0.01, 0.72, ctypes.byref(b), None, None, None, 0, ctypes.byref(ctx))
    assert st == N.AF_EINVAL and not ctx.value
