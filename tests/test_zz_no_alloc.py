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


def test_noalloc_dt_matches_context_dt_twice():
    import torch
    from paper_2609_29081_b300 import Solver, _native as N
    lib = N.load()
    lib.af_dt_max_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.af_dt_max_noalloc.restype = ctypes.c_int
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
        g = N.Grid()
        g.dim, g.n[0], g.n[1] = 2, w.n[0], w.n[1]
        g.lo[0], g.lo[1], g.hi[0], g.hi[1] = w.lo[0], w.lo[1], w.hi[0], w.hi[1]
        st = lib.af_dt_max_noalloc(ctypes.byref(g), w.gamma, w.mu, w.Pr, None, ctypes.c_void_p(avg.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == N.AF_OK
        torch.cuda.synchronize()
        assert out.item() == pytest.approx(ref, rel=1e-14)
    g.n[0], g.n[1] = 1 << 14, 1 << 13   # beyond the fixed scratch: rejected, nothing launched
    st = lib.af_dt_max_noalloc(ctypes.byref(g), 1.4, 0.01, 0.72, None, ctypes.c_void_p(avg.data_ptr()),
                               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert st == N.AF_EINVAL
