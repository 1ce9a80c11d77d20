"""ctypes binding of libafns (include/afns.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module allocates the
device workspace through PyTorch, passes pointers and sizes, and converts
between the packed state layout and the per-site pointers of the C-ABI.
There is no CPU fallback: a missing library or GPU raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import workloads

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libafns.so")

AF_OK, AF_EINVAL, AF_ENOMEM, AF_ECUDA, AF_ENOTPP, AF_ESTATE = range(6)
FP64, MIXED = 0, 1
LIM_NONE, LIM_PP, LIM_S_PP = 0, 1, 2

EXPORTED = ["af_opts_default", "af_workspace_bytes", "af_create", "af_destroy", "af_set_state",
            "af_get_state", "af_dt_max", "af_step", "af_advance", "af_residual", "af_get_limiter",
            "af_sizes", "af_set_profiling", "af_get_profile", "af_tune", "af_dt_max_noalloc",
            "af_alu_peak", "af_set_state_f32", "af_get_state_f32", "af_debug_tile_wait", "af_last_error"]


class AfnsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libafns status %d: %s" % (status, msg))
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 2), ("lo", ctypes.c_double * 2),
                ("hi", ctypes.c_double * 2)]


class BC(ctypes.Structure):
    _fields_ = [("side", ctypes.c_int * 4), ("wall_speed", ctypes.c_double * 4)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("limiter", ctypes.c_int), ("c_s", ctypes.c_double),
                ("cfl_c", ctypes.c_double), ("cfl_v", ctypes.c_double), ("eps", ctypes.c_double),
                ("max_halvings", ctypes.c_int), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
                ("source", ctypes.c_int), ("src_p0", ctypes.c_double),
                ("ex_M0", ctypes.c_double), ("ex_uinf", ctypes.c_double), ("threads", ctypes.c_int),
                ("kappa_off", ctypes.c_int)]


_libs = {}


def load(path: str = LIB_PATH):
    """Load libafns.so, or the build at `path` (raises if it was not built)."""
    if path in _libs:
        return _libs[path]
    if not os.path.exists(path):
        raise RuntimeError("%s is missing: build it with paper_2609_29081_b300.build.build()"
                           % os.path.basename(path))
    L = ctypes.CDLL(path)
    vp, dp, ip, sp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), \
        ctypes.POINTER(ctypes.c_size_t)
    P4 = ctypes.c_void_p * 4
    L.af_opts_default.argtypes = [ctypes.c_int, ctypes.POINTER(Opts)]
    L.af_workspace_bytes.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Opts), sp]
    L.af_create.argtypes = [ctypes.POINTER(Grid), ctypes.c_double, ctypes.c_double, ctypes.c_double,
                            ctypes.POINTER(BC), ctypes.POINTER(Opts), vp, vp, ctypes.c_size_t,
                            ctypes.POINTER(vp)]
    L.af_destroy.argtypes = [vp]
    L.af_set_state.argtypes = [vp, P4, ctypes.c_int, ctypes.c_double]
    L.af_get_state.argtypes = [vp, P4, ctypes.c_int, dp]
    L.af_set_state_f32.argtypes = [vp, P4, ctypes.c_int, ctypes.c_double]
    L.af_debug_tile_wait.argtypes = [vp, ctypes.c_int]
    L.af_get_state_f32.argtypes = [vp, P4, ctypes.c_int, dp]
    L.af_dt_max.argtypes = [vp, dp]
    L.af_step.argtypes = [vp, ctypes.c_double, dp, ip]
    L.af_advance.argtypes = [vp, ctypes.c_double, ip, ip]
    L.af_residual.argtypes = [vp, ctypes.c_double, P4, ctypes.c_int, ip]
    L.af_get_limiter.argtypes = [vp, vp, vp]
    L.af_sizes.argtypes = [vp, sp, sp, sp]
    L.af_tune.argtypes = [vp, ip, ip, ip]
    L.af_dt_max_noalloc.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, vp, vp, vp, vp]
    L.af_alu_peak.argtypes = [ctypes.c_int, dp]
    L.af_set_profiling.argtypes = [vp, ctypes.c_int]
    L.af_get_profile.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    L.af_last_error.argtypes = [vp]
    L.af_last_error.restype = ctypes.c_char_p
    for f in EXPORTED:
        if f != "af_last_error":
            getattr(L, f).restype = ctypes.c_int
    _libs[path] = L
    return L


def alu_peak(precision) -> float:
    """Measured FMA throughput of the current device in TFLOP/s (FP32 for MIXED,
    FP64 for FP64): the ALU roofline denominator of the stage kernels."""
    v = ctypes.c_double(0.0)
    rc = load().af_alu_peak(precision, ctypes.byref(v))
    if rc != AF_OK:
        raise AfnsError("af_alu_peak failed (status %d)" % rc)
    return v.value


def default_opts(dim, precision=FP64, limiter=LIM_S_PP, lib=None, **kw) -> Opts:
    o = Opts()
    (lib or load()).af_opts_default(dim, ctypes.byref(o))
    o.precision = precision
    o.limiter = limiter
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Solver:
    """One AF-NS problem on cuda:0 (device memory owned by a torch tensor)."""

    def __init__(self, dim, n, lo, hi, gamma, mu, Pr, bc, precision=FP64, limiter=LIM_S_PP, stream=None,
                 wall_speed=(0.0, 0.0, 0.0, 0.0), lib_path=LIB_PATH, **opts):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libafns needs a CUDA GPU; none is available")
        self.torch = torch
        self.lib = load(lib_path)
        self.dim = dim
        self.n = (int(n[0]), int(n[1]) if dim == 2 else 1)
        g = Grid()
        g.dim = dim
        g.n[0], g.n[1] = self.n
        g.lo[0], g.hi[0] = lo[0], hi[0]
        g.lo[1], g.hi[1] = (lo[1], hi[1]) if dim == 2 else (0.0, 1.0)
        b = BC()
        for k in range(4):
            b.side[k] = bc[k] if k < len(bc) else 0
            b.wall_speed[k] = wall_speed[k]
        self.opts = default_opts(dim, precision, limiter, lib=self.lib, **opts)
        nbytes = ctypes.c_size_t(0)
        self._check(self.lib.af_workspace_bytes(ctypes.byref(g), ctypes.byref(self.opts), ctypes.byref(nbytes)))
        self.ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device="cuda")
        base = self.ws.data_ptr()
        base = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ctx = ctypes.c_void_p()
        st = self._check(self.lib.af_create(ctypes.byref(g), gamma, mu, Pr, ctypes.byref(b), ctypes.byref(self.opts),
                                            ctypes.c_void_p(self.stream.cuda_stream), ctypes.c_void_p(base),
                                            nbytes.value, ctypes.byref(ctx)))
        self.ctx = ctx
        self.shapes = workloads.site_shapes(dim, *self.n)
        self.size = workloads.state_len(dim, *self.n)
        cells, faces = ctypes.c_size_t(0), ctypes.c_size_t(0)
        self.lib.af_sizes(self.ctx, ctypes.byref(cells), ctypes.byref(faces), None)
        self.faces = faces.value

    @classmethod
    def from_workload(cls, w, **kw):
        if getattr(w, "source", 0) and "source" not in kw:
            kw.update(source=w.source, src_p0=w.src_p0)
        if workloads.BC_EXACT in tuple(w.bc) and "ex_M0" not in kw:
            kw.update(ex_M0=w.ex_M0, ex_uinf=w.ex_uinf)
        if "wall_speed" not in kw:
            kw["wall_speed"] = tuple(w.wall_speed)
        return cls(w.dim, w.n, w.lo, w.hi, w.gamma, w.mu, w.Pr, w.bc, **kw)

    def _check(self, st):
        if st != AF_OK:
            # without a context: why the last af_create refused its arguments
            msg = self.lib.af_last_error(getattr(self, "ctx", None) or None)
            raise AfnsError(st, (msg or b"").decode())
        return st

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.af_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- site pointer arrays of a packed buffer (numpy host array or torch tensor)
    def _ptrs(self, buf, f32=False):
        P4 = ctypes.c_void_p * 4
        p = P4()
        if isinstance(buf, np.ndarray):
            assert buf.dtype == (np.float32 if f32 else np.float64) and buf.flags.c_contiguous and buf.size == self.size
            base, on_dev = buf.ctypes.data, 0
        else:
            assert buf.dtype == (self.torch.float32 if f32 else self.torch.float64)
            assert buf.is_contiguous() and buf.numel() == self.size
            base, on_dev = buf.data_ptr(), int(buf.is_cuda)
        o, esz = 0, 4 if f32 else 8
        for k, shp in enumerate(self.shapes):
            p[k] = base + esz * o
            o += int(np.prod(shp))
        return p, on_dev

    def set_state_f32(self, state, t=0.0):
        """FP32 site arrays (mixed-precision contexts only)."""
        if isinstance(state, np.ndarray):
            state = np.ascontiguousarray(state, dtype=np.float32)
        p, dev = self._ptrs(state, f32=True)
        self._check(self.lib.af_set_state_f32(self.ctx, p, dev, t))

    def get_state_f32(self, out=None):
        if out is None:
            out = np.empty(self.size, dtype=np.float32)
        p, dev = self._ptrs(out, f32=True)
        t = ctypes.c_double(0)
        self._check(self.lib.af_get_state_f32(self.ctx, p, dev, ctypes.byref(t)))
        self.t = t.value
        return out

    def set_state(self, state, t=0.0):
        if isinstance(state, np.ndarray):
            state = np.ascontiguousarray(state, dtype=np.float64)
        p, dev = self._ptrs(state)
        self._check(self.lib.af_set_state(self.ctx, p, dev, t))

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.size, dtype=np.float64)
        p, dev = self._ptrs(out)
        t = ctypes.c_double(0)
        self._check(self.lib.af_get_state(self.ctx, p, dev, ctypes.byref(t)))
        self.t = t.value
        return out

    def dt_max(self):
        d = ctypes.c_double(0)
        self._check(self.lib.af_dt_max(self.ctx, ctypes.byref(d)))
        return d.value

    def step(self, dt=0.0):
        d, h = ctypes.c_double(0), ctypes.c_int(0)
        self._check(self.lib.af_step(self.ctx, dt, ctypes.byref(d), ctypes.byref(h)))
        return d.value, h.value

    def advance(self, t_end):
        ns, nr = ctypes.c_int(0), ctypes.c_int(0)
        self._check(self.lib.af_advance(self.ctx, t_end, ctypes.byref(ns), ctypes.byref(nr)))
        return ns.value, nr.value

    def residual(self, dt, out=None):
        if out is None:
            out = np.empty(self.size, dtype=np.float64)
        p, dev = self._ptrs(out)
        nb = ctypes.c_int(0)
        self._check(self.lib.af_residual(self.ctx, dt, p, dev, ctypes.byref(nb)))
        return out, nb.value

    def limiter(self):
        ts = np.empty(self.faces)
        tp = np.empty(self.faces)
        self._check(self.lib.af_get_limiter(self.ctx, ts.ctypes.data_as(ctypes.c_void_p),
                                            tp.ctypes.data_as(ctypes.c_void_p)))
        return ts, tp

    def tune(self):
        tx, ty, th = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        self._check(self.lib.af_tune(self.ctx, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(th)))
        return {"tile_x": tx.value, "tile_y": ty.value, "threads": th.value}

    def set_profiling(self, on=True):
        self._check(self.lib.af_set_profiling(self.ctx, int(on)))

    def profile(self):
        ms, ns, nl = ctypes.c_double(0), ctypes.c_longlong(0), ctypes.c_longlong(0)
        self._check(self.lib.af_get_profile(self.ctx, ctypes.byref(ms), ctypes.byref(ns), ctypes.byref(nl)))
        return {"stage_ms": ms.value, "stage_launches": ns.value, "launches": nl.value}


BATCH_EXPORTED = ["afb_workspace_bytes", "afb_create", "afb_destroy", "afb_set_state", "afb_get_state", "afb_tune",
                  "afb_step_all", "afb_stats", "afb_sync", "afb_last_error"]


def _load_batch():
    L = load()
    if getattr(L, "_batch_ready", False):
        return L
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    P4 = ctypes.c_void_p * 4
    L.afb_workspace_bytes.argtypes = [ctypes.c_int, vp, vp, ctypes.POINTER(ctypes.c_size_t)]
    L.afb_create.argtypes = [ctypes.c_int, vp, dp, dp, dp, vp, vp, vp, vp, ctypes.c_size_t, ctypes.POINTER(vp)]
    L.afb_destroy.argtypes = [vp]
    L.afb_set_state.argtypes = [vp, ctypes.c_int, P4, ctypes.c_int, ctypes.c_double]
    L.afb_get_state.argtypes = [vp, ctypes.c_int, P4, ctypes.c_int, dp]
    L.afb_tune.argtypes = [vp, ip, ip, ip, ip]
    L.afb_step_all.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.afb_stats.argtypes = [vp, ctypes.c_int, ip, ip, ip, dp]
    L.afb_sync.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.afb_last_error.argtypes = [vp]
    L.afb_last_error.restype = ctypes.c_char_p
    for f in BATCH_EXPORTED:
        if f != "afb_last_error":
            getattr(L, f).restype = ctypes.c_int
    L._batch_ready = True
    return L


class BatchSolver:
    """Many independent 2D problems (workloads.Workload list) on cuda:0."""

    def __init__(self, wls, precision=MIXED, limiter=LIM_S_PP, stream=None, **opts):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libafns needs a CUDA GPU; none is available")
        self.torch = torch
        self.lib = _load_batch()
        self.wls = list(wls)
        n = len(self.wls)
        grids = (Grid * n)()
        bcs = (BC * n)()
        gam = (ctypes.c_double * n)(*[w.gamma for w in self.wls])
        mu = (ctypes.c_double * n)(*[w.mu for w in self.wls])
        pr = (ctypes.c_double * n)(*[w.Pr for w in self.wls])
        for k, w in enumerate(self.wls):
            assert w.dim == 2
            grids[k].dim = 2
            grids[k].n[0], grids[k].n[1] = w.n
            grids[k].lo[0], grids[k].lo[1] = w.lo
            grids[k].hi[0], grids[k].hi[1] = w.hi
            for s in range(4):
                bcs[k].side[s] = w.bc[s]
                bcs[k].wall_speed[s] = w.wall_speed[s]
        self.opts = default_opts(2, precision, limiter, **opts)
        nb = ctypes.c_size_t(0)
        self._check(self.lib.afb_workspace_bytes(n, ctypes.cast(grids, ctypes.c_void_p),
                                                 ctypes.cast(ctypes.byref(self.opts), ctypes.c_void_p),
                                                 ctypes.byref(nb)))
        self.ws = torch.empty(nb.value + 256, dtype=torch.uint8, device="cuda")
        base = (self.ws.data_ptr() + 255) // 256 * 256
        # a stream of its own: a CUDA graph cannot be captured on the legacy default stream
        self.stream = stream if stream is not None else torch.cuda.Stream()
        ctx = ctypes.c_void_p()
        self._check(self.lib.afb_create(n, ctypes.cast(grids, ctypes.c_void_p), gam, mu, pr,
                                        ctypes.cast(bcs, ctypes.c_void_p),
                                        ctypes.cast(ctypes.byref(self.opts), ctypes.c_void_p),
                                        ctypes.c_void_p(self.stream.cuda_stream), ctypes.c_void_p(base), nb.value,
                                        ctypes.byref(ctx)))
        self.ctx = ctx

    def _check(self, st):
        if st != AF_OK:
            c = getattr(self, "ctx", None)
            msg = self.lib.afb_last_error(c) if c else b""
            raise AfnsError(st, (msg or b"").decode())
        return st

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.afb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ptrs(self, i, buf):
        shapes = workloads.site_shapes(2, *self.wls[i].n)
        P4 = ctypes.c_void_p * 4
        p = P4()
        base = buf.ctypes.data
        o = 0
        for k, shp in enumerate(shapes):
            p[k] = base + 8 * o
            o += int(np.prod(shp))
        assert o == buf.size
        return p

    def set_state(self, i, state, t=0.0):
        s = np.ascontiguousarray(state, dtype=np.float64)
        self._check(self.lib.afb_set_state(self.ctx, i, self._ptrs(i, s), 0, t))

    def get_state(self, i):
        out = np.empty(workloads.state_len(2, *self.wls[i].n))
        t = ctypes.c_double(0)
        self._check(self.lib.afb_get_state(self.ctx, i, self._ptrs(i, out), 0, ctypes.byref(t)))
        return out, t.value

    def tune(self):
        v = [ctypes.c_int(0) for _ in range(4)]
        self._check(self.lib.afb_tune(self.ctx, *[ctypes.byref(x) for x in v]))
        return {"tile_x": v[0].value, "tile_y": v[1].value, "threads": v[2].value, "schedule": v[3].value}

    def step_all(self, nsteps=1, graph=True):
        self._check(self.lib.afb_step_all(self.ctx, nsteps, int(graph)))

    def sync(self):
        n = ctypes.c_longlong(0)
        self._check(self.lib.afb_sync(self.ctx, ctypes.byref(n)))
        return n.value

    def stats(self, i):
        a, r, f, t = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0)
        self._check(self.lib.afb_stats(self.ctx, i, ctypes.byref(a), ctypes.byref(r), ctypes.byref(f),
                                       ctypes.byref(t)))
        return {"accepted": a.value, "restarts": r.value, "failed": f.value, "t": t.value}
