"""GPU checks of the batched form: many independent 2D problems of uneven sizes
and parameters advanced by one persistent stage kernel per RK stage, with the
batch step captured in a CUDA graph. Each problem must evolve exactly as it does
alone (same fused stage code, same CFL step), restarts stay per problem, and the
autotuner's choice does not change any result (the per-face and per-node
arithmetic does not depend on the tile shape)."""
import numpy as np
import pytest

from conftest import cuda_ok
from paper_2609_29081_b300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


def problems():
    out = []
    for k, (n, mu) in enumerate([((24, 16), 0.01), ((33, 17), 0.003), ((16, 40), 0.02), ((20, 20), 0.001)]):
        w = W.random_smooth_2d(n, seed=20 + k, mu=mu)
        out.append(w)
    w = W.random_smooth_2d((18, 22), seed=30, bc=(1, 1, 2, 3), mu=0.01)
    out.append(w)
    return out


def run_single(w, precision, steps):
    from paper_2609_29081_b300 import Solver
    S = Solver.from_workload(w, precision=precision)
    S.set_state(w.state)
    for _ in range(steps):
        S.step(0.0)
    return S.get_state(), S.t


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_single(prec, graph):
    from paper_2609_29081_b300 import FP64, MIXED, BatchSolver
    p = MIXED if prec == "mixed" else FP64
    wls = problems()
    B = BatchSolver(wls, precision=p)
    for i, w in enumerate(wls):
        B.set_state(i, w.state)
    B.step_all(6, graph=graph)
    B.sync()
    for i, w in enumerate(wls):
        st = B.stats(i)
        assert st["accepted"] == 6 and st["restarts"] == 0 and st["failed"] == 0
        got, t = B.get_state(i)
        ref, tref = run_single(w, p, 6)
        assert t == tref
        assert np.array_equal(got, ref)


def test_batch_tuned_config_same_results():
    from paper_2609_29081_b300 import MIXED, BatchSolver
    wls = problems()
    B = BatchSolver(wls, precision=MIXED)
    for i, w in enumerate(wls):
        B.set_state(i, w.state)
    cfg = B.tune()
    assert cfg["tile_x"] in (16, 32) and cfg["threads"] in (128, 256)
    B.step_all(4)
    B.sync()
    for i, w in enumerate(wls):
        got, _ = B.get_state(i)
        ref, _ = run_single(w, MIXED, 4)
        assert np.array_equal(got, ref)


def test_batch_restarts_stay_per_problem():
    """A near-vacuum blast in the batch restarts (Remark 3.2) without touching the
    others; every DoF of every problem stays admissible."""
    from paper_2609_29081_b300 import MIXED, BatchSolver
    wls = problems()[:3] + [W.blast_2d((32, 32), seed=2, rho_min=1e-10, p_min=1e-12)]
    B = BatchSolver(wls, precision=MIXED)
    for i, w in enumerate(wls):
        B.set_state(i, w.state)
    B.step_all(20)
    B.sync()
    st = [B.stats(i) for i in range(len(wls))]
    assert st[3]["restarts"] > 0 and st[3]["accepted"] + st[3]["restarts"] == 20
    for i in range(3):
        assert st[i]["accepted"] == 20 and st[i]["restarts"] == 0
    for i, w in enumerate(wls):
        s, _ = B.get_state(i)
        for U in W.split_sites(s, 2, *w.n):
            p = 0.4 * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0])
            assert np.isfinite(U).all() and U[0].min() > 0 and p.min() > 0
