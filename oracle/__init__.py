"""ctypes binding of the plain FP64 CPU oracle (``afns_oracle.c``).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference leg of ``bench.py`` may import this package. The CUDA
library never imports, links or calls it, and it shares no code with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "afns_oracle.c")
_HDR = os.path.join(_HERE, "afns_oracle.h")
_LIB = os.path.join(_HERE, "liboracle_afns.so")

BC_PERIODIC, BC_WALL, BC_SYMMETRY, BC_TRANSMISSIVE = 0, 1, 2, 3
LIM_NONE, LIM_PP, LIM_S_PP = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, no fast-math)."""
    stale = not os.path.exists(_LIB) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n1", ctypes.c_int), ("n2", ctypes.c_int),
                ("lo1", ctypes.c_double), ("hi1", ctypes.c_double),
                ("lo2", ctypes.c_double), ("hi2", ctypes.c_double),
                ("gamma", ctypes.c_double), ("mu", ctypes.c_double), ("Pr", ctypes.c_double),
                ("bc", ctypes.c_int * 4), ("limiter", ctypes.c_int),
                ("c_s", ctypes.c_double), ("cfl_c", ctypes.c_double),
                ("cfl_v", ctypes.c_double), ("eps", ctypes.c_double),
                ("source", ctypes.c_int), ("src_p0", ctypes.c_double), ("time", ctypes.c_double),
                ("ex_M0", ctypes.c_double), ("ex_uinf", ctypes.c_double),
                ("wall_speed", ctypes.c_double * 4)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        pp = ctypes.POINTER(Problem)
        L.orc_defaults.argtypes = [pp]
        L.orc_state_len.argtypes = [pp]
        L.orc_state_len.restype = ctypes.c_size_t
        L.orc_face_len.argtypes = [pp]
        L.orc_face_len.restype = ctypes.c_size_t
        L.orc_residual.argtypes = [pp, dp, ctypes.c_double, dp, dp, dp, ip]
        L.orc_dt_max.argtypes = [pp, dp]
        L.orc_dt_max.restype = ctypes.c_double
        L.orc_step.argtypes = [pp, dp, ctypes.c_double, ctypes.c_int, dp, ip]
        L.orc_point_low_order.argtypes = [pp, dp, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp]
        L.orc_point_low_order.restype = None
        L.orc_face_low_order.argtypes = [pp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        L.orc_face_low_order.restype = None
        L.orc_advance.argtypes = [pp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_int, ip, ip]
        L.orc_rk_table.argtypes = [dp, dp]
        for f in ("orc_op_dplus", "orc_op_dminus", "orc_op_dcentral"):
            getattr(L, f).argtypes = [dp, ctypes.c_double, dp]
        L.orc_op_bmatrix.argtypes = [dp]
        L.orc_op_d2_scalar.argtypes = [dp, dp, ctypes.c_double, dp]
        L.orc_inviscid_flux.argtypes = [pp, dp, ctypes.c_int, dp]
        L.orc_viscous_flux.argtypes = [pp, dp, dp, ctypes.c_int, dp]
        L.orc_visc_bound.argtypes = [pp, dp, dp, ctypes.c_int]
        L.orc_visc_bound.restype = ctypes.c_double
        L.orc_pressure.argtypes = [pp, dp]
        L.orc_pressure.restype = ctypes.c_double
        L.orc_wave_speed.argtypes = [pp, dp, ctypes.c_int]
        L.orc_wave_speed.restype = ctypes.c_double
        L.orc_theta.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_theta.restype = ctypes.c_double
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def problem(dim, n1, n2=1, lo=(0.0, 0.0), hi=(1.0, 1.0), gamma=1.4, mu=0.0, Pr=0.72,
            bc=(0, 0, 0, 0), limiter=LIM_S_PP, **kw) -> Problem:
    P = Problem()
    P.dim, P.n1, P.n2 = dim, n1, (n2 if dim == 2 else 1)
    P.lo1, P.hi1 = lo[0], hi[0]
    P.lo2, P.hi2 = (lo[1], hi[1]) if dim == 2 else (0.0, 1.0)
    P.gamma, P.mu, P.Pr = gamma, mu, Pr
    for k in range(4):
        P.bc[k] = bc[k]
    lib().orc_defaults(ctypes.byref(P))
    P.limiter = limiter
    for k, v in kw.items():
        if k == "wall_speed":
            for i in range(4):
                P.wall_speed[i] = v[i]
        else:
            setattr(P, k, v)
    return P


def state_len(P):
    return lib().orc_state_len(ctypes.byref(P))


def face_len(P):
    return lib().orc_face_len(ctypes.byref(P))


def residual(P, state, dt, with_theta=False):
    """Limited residual L(u) (same packed layout as the state)."""
    s = np.ascontiguousarray(state, dtype=np.float64)
    L = np.zeros_like(s)
    nb = ctypes.c_int(0)
    if with_theta:
        ts = np.zeros(face_len(P))
        tp = np.zeros(face_len(P))
        lib().orc_residual(ctypes.byref(P), _dp(s), dt, _dp(L), _dp(ts), _dp(tp), ctypes.byref(nb))
        return L, ts, tp, nb.value
    lib().orc_residual(ctypes.byref(P), _dp(s), dt, _dp(L), None, None, ctypes.byref(nb))
    return L, nb.value


def dt_max(P, state):
    s = np.ascontiguousarray(state, dtype=np.float64)
    return lib().orc_dt_max(ctypes.byref(P), _dp(s))


def point_low_order(P, state, dt, a0, a1=0):
    """Low-order point update (reading R7) of lattice node (a0, a1)."""
    s = np.ascontiguousarray(state, dtype=np.float64)
    out = np.zeros(P.dim + 2)
    lib().orc_point_low_order(ctypes.byref(P), _dp(s), dt, a0, a1, _dp(out))
    return out


def face_low_order(P, state, l, f0, f1=0):
    """Low-order LLF face flux of Eq. (19) of face (f0, f1) in direction l."""
    s = np.ascontiguousarray(state, dtype=np.float64)
    out = np.zeros(P.dim + 2)
    lib().orc_face_low_order(ctypes.byref(P), _dp(s), l, f0, f1, _dp(out))
    return out


def step(P, state, dt, max_halvings=30):
    """One SSP-RK54 step in place; returns (status, dt_taken, halvings)."""
    assert state.dtype == np.float64 and state.flags.c_contiguous
    taken = ctypes.c_double(0)
    h = ctypes.c_int(0)
    rc = lib().orc_step(ctypes.byref(P), _dp(state), dt, max_halvings, ctypes.byref(taken), ctypes.byref(h))
    return rc, taken.value, h.value


def advance(P, state, t, t_end, max_halvings=30, max_steps=0):
    """Advance in place with CFL steps; returns (status, steps, restarts)."""
    assert state.dtype == np.float64 and state.flags.c_contiguous
    ns = ctypes.c_int(0)
    nr = ctypes.c_int(0)
    rc = lib().orc_advance(ctypes.byref(P), _dp(state), t, t_end, max_halvings, max_steps,
                           ctypes.byref(ns), ctypes.byref(nr))
    return rc, ns.value, nr.value


def rk_table():
    a = np.zeros((5, 5))
    b = np.zeros((5, 5))
    lib().orc_rk_table(_dp(a), _dp(b))
    return a, b


def op(name, z5, dx):
    z = np.ascontiguousarray(z5, dtype=np.float64)
    out = ctypes.c_double(0)
    getattr(lib(), "orc_op_" + name)(_dp(z), dx, ctypes.byref(out))
    return out.value


def bmatrix():
    b = np.zeros(25)
    lib().orc_op_bmatrix(_dp(b))
    return b.reshape(5, 5)


def d2_scalar(k5, z5, dx):
    k = np.ascontiguousarray(k5, dtype=np.float64)
    z = np.ascontiguousarray(z5, dtype=np.float64)
    out = ctypes.c_double(0)
    lib().orc_op_d2_scalar(_dp(k), _dp(z), dx, ctypes.byref(out))
    return out.value


def inviscid_flux(P, U, l):
    U = np.ascontiguousarray(U, dtype=np.float64)
    F = np.zeros(P.dim + 2)
    lib().orc_inviscid_flux(ctypes.byref(P), _dp(U), l, _dp(F))
    return F


def viscous_flux(P, U, grad, l):
    U = np.ascontiguousarray(U, dtype=np.float64)
    g = np.ascontiguousarray(grad, dtype=np.float64).ravel()
    F = np.zeros(P.dim + 2)
    lib().orc_viscous_flux(ctypes.byref(P), _dp(U), _dp(g), l, _dp(F))
    return F


def visc_bound(P, U, grad, l):
    U = np.ascontiguousarray(U, dtype=np.float64)
    g = np.ascontiguousarray(grad, dtype=np.float64).ravel()
    return lib().orc_visc_bound(ctypes.byref(P), _dp(U), _dp(g), l)


def pressure(P, U):
    U = np.ascontiguousarray(U, dtype=np.float64)
    return lib().orc_pressure(ctypes.byref(P), _dp(U))


def wave_speed(P, U, l):
    U = np.ascontiguousarray(U, dtype=np.float64)
    return lib().orc_wave_speed(ctypes.byref(P), _dp(U), l)


def theta(zL, zH, eps):
    return lib().orc_theta(zL, zH, eps)


# ---------------------------------------------------------------------------
# Operation counts (opcount.cpp: this source compiled as C++ with a counting
# scalar). Categories and kinds as documented there.
# ---------------------------------------------------------------------------
_OPC_SRC = os.path.join(_HERE, "opcount.cpp")
_OPC_LIB = os.path.join(_HERE, "liboracle_opcount.so")
OPC_CATEGORIES = ("add", "mul", "div", "sqrt", "trans", "other")
OPC_KINDS = ("counted", "repeated", "trivial")
OPC_NPH = 12
OPC_PHASES = {0: "ghost fill", 1: "centres + centre limiter", 2: "node primitives",
              3: "point residual", 4: "high-order face flux", 5: "low-order cell and face quantities",
              6: "face limiter", 7: "point scaling limiter", 8: "cell residual", 9: "CFL bound",
              10: "RK combination", 11: "other"}

_opc = None


def opcount_build(force: bool = False) -> str:
    stale = not os.path.exists(_OPC_LIB) or any(
        os.path.getmtime(p) > os.path.getmtime(_OPC_LIB) for p in (_SRC, _HDR, _OPC_SRC))
    if force or stale:
        tmp = _OPC_LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _OPC_SRC])
        os.replace(tmp, _OPC_LIB)
    return _OPC_LIB


def _opc_lib():
    global _opc
    if _opc is None:
        L = ctypes.CDLL(opcount_build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(Problem)
        L.orc_opcount_reset.argtypes = []
        L.orc_opcount_get.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
        L.orc_opcount_residual.argtypes = [pp, dp, ctypes.c_double, dp]
        L.orc_opcount_step.argtypes = [pp, dp, ctypes.c_double]
        L.orc_opcount_dt_max.argtypes = [pp, dp]
        L.orc_opcount_dt_max.restype = ctypes.c_double
        _opc = L
    return _opc


def _opc_tally():
    L = _opc_lib()
    n = OPC_NPH * len(OPC_CATEGORIES) * len(OPC_KINDS)
    buf = (ctypes.c_longlong * n)()
    L.orc_opcount_get(buf)
    return np.array(buf, dtype=np.int64).reshape(OPC_NPH, len(OPC_CATEGORIES), len(OPC_KINDS))


def opcount(P, state, what="step", dt=None, out=None):
    """Operation tallies [phase, category, kind] of one stage residual
    (what="residual"; its values go to `out` if given), one SSP-RK54 step
    ("step", five residuals plus the combinations) or the CFL bound ("dt")."""
    L = _opc_lib()
    s = np.ascontiguousarray(state, dtype=np.float64).copy()
    if dt is None:
        dt = dt_max(P, s)
    L.orc_opcount_reset()
    if what == "residual":
        rc = L.orc_opcount_residual(ctypes.byref(P), _dp(s), dt, _dp(out) if out is not None else None)
    elif what == "step":
        rc = L.orc_opcount_step(ctypes.byref(P), _dp(s), dt)
    else:
        L.orc_opcount_dt_max(ctypes.byref(P), _dp(s))
        rc = 0
    assert rc == 0
    return _opc_tally()
