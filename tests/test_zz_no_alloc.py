"""The allocation-free CFL entry point, checked through the C-ABI against the
context-based af_dt_max on the same state, on two calls in a row.

af_dt_max_noalloc exists for callers that must not allocate device memory: code
whose device memory is fully owned by a host framework's pool, or that runs where
a cudaMalloc (and its implicit device synchronisation) is not allowed. Its scratch
is a fixed device array inside the library."""
import ctypes

import numpy as np
import pytest

from conftest import cuda_ok
from paper_2609_29081_b300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


def _grid(N, w):
    g = N.Grid()
    g.dim, g.n[0], g.n[1] = 2, w.n[0], w.n[1]
    g.lo[0], g.lo[1], g.hi[0], g.hi[1] = w.lo[0], w.lo[1], w.hi[0], w.hi[1]
    return g


def _call(lib, g, w, opts, avg, out, stream):
    return lib.af_dt_max_noalloc(ctypes.byref(g), w.gamma, w.mu, w.Pr,
                                 ctypes.byref(opts) if opts is not None else None,
                                 ctypes.c_void_p(avg.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_dt_matches_context_dt_twice():
    import torch
    from paper_2609_29081_b300 import Solver, _native as N
    lib = N.load()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for k, w in enumerate([W.random_smooth_2d((70, 45), seed=40), W.smooth_2d(96)]):
        S = Solver.from_workload(w)
        S.set_state(w.state)
        if k == 1:
            S.step(0.0)      # a state that differs from the first call's
        ref = S.dt_max()
        state = torch.from_numpy(S.get_state()).cuda()
        avg = state[: 4 * w.n[0] * w.n[1]]
        g = _grid(N, w)
        assert _call(lib, g, w, None, avg, out, stream) == N.AF_OK
        torch.cuda.synchronize()
        assert out.item() == pytest.approx(ref, rel=1e-14)
    g.n[0], g.n[1] = 1 << 14, 1 << 13   # beyond the fixed scratch: rejected, nothing launched
    assert _call(lib, g, w, None, avg, out, stream) == N.AF_EINVAL


def test_noalloc_honours_kappa_off():
    """With kappa_off the bound has no conduction term, as a kappa_off context's."""
    import torch
    from paper_2609_29081_b300 import Solver, _native as N
    lib = N.load()
    w = W.random_smooth_2d((40, 24), seed=41)
    w.mu = 0.5   # a bound dominated by the viscous term, where the conduction term matters
    S = Solver.from_workload(w, kappa_off=1)
    S.set_state(w.state)
    ref = S.dt_max()
    avg = torch.from_numpy(np.ascontiguousarray(w.state[: 4 * w.n[0] * w.n[1]])).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    o = N.default_opts(2, kappa_off=1)
    assert _call(lib, _grid(N, w), w, o, avg, out, stream) == N.AF_OK
    torch.cuda.synchronize()
    assert out.item() == pytest.approx(ref, rel=1e-14)
    o0 = N.default_opts(2)
    assert _call(lib, _grid(N, w), w, o0, avg, out, stream) == N.AF_OK
    torch.cuda.synchronize()
    assert out.item() < ref * (1 - 1e-3)   # with conduction the step is smaller


@pytest.mark.parametrize("kind", ["nan", "negative_density", "negative_pressure"])
def test_noalloc_flags_inadmissible_cells(kind):
    """An inadmissible or non-finite cell average gives NaN, not a finite step
    taken from the other cells; the next call on a valid state is unaffected."""
    import torch
    from paper_2609_29081_b300 import _native as N
    lib = N.load()
    w = W.random_smooth_2d((50, 30), seed=42)
    nc = w.n[0] * w.n[1]
    avg = np.ascontiguousarray(w.state[: 4 * nc]).copy()
    good = torch.from_numpy(avg.copy()).cuda()
    cell = 777
    if kind == "nan":
        avg[2 * nc + cell] = np.nan
    elif kind == "negative_density":
        avg[cell] = -1e-3
    else:
        avg[3 * nc + cell] = 0.0   # E = 0 with nonzero momentum: p < 0
    bad = torch.from_numpy(avg).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    g = _grid(N, w)
    assert _call(lib, g, w, None, bad, out, stream) == N.AF_OK
    torch.cuda.synchronize()
    assert np.isnan(out.item())
    assert _call(lib, g, w, None, good, out, stream) == N.AF_OK
    torch.cuda.synchronize()
    assert np.isfinite(out.item()) and out.item() > 0
