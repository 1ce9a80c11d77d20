"""Failure detection without a GPU fault: the stage kernel's bounded tile-load
wait. A test hook arms the tile-load barrier with more bytes than the copies
deliver, so every wait runs out (after 2 s of the GPU's global timer); the
kernel flags the stage instead of hanging, the call returns AF_ECUDA with a
message, and the context keeps working once the hook is cleared."""
import time

import numpy as np
import pytest

from conftest import cuda_ok
from paper_2609_29081_b300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_tile_load_timeout_is_reported_and_context_recovers(prec):
    from paper_2609_29081_b300 import FP64, MIXED, AfnsError, Solver
    w = W.random_smooth_2d((16, 8), seed=2)   # one tile: one CTA waits
    S = Solver.from_workload(w, precision=MIXED if prec == "mixed" else FP64)
    S.set_state(w.state)
    ref, _ = S.residual(1e-3)
    assert S.lib.af_debug_tile_wait(S.ctx, 16) == 0
    t0 = time.time()
    with pytest.raises(AfnsError) as e:
        S.residual(1e-3)
    assert "timed out" in str(e.value)
    assert time.time() - t0 < 30
    assert S.lib.af_debug_tile_wait(S.ctx, 0) == 0
    again, _ = S.residual(1e-3)
    assert np.array_equal(again, ref)
    S.step(0.0)   # and a whole step goes through
