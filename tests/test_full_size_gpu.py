"""GPU parity at the benchmark's full sizes, in the launch configurations the
benchmark times, through the C-ABI.

- The 2D smooth periodic flow at 1024^2: the mixed path's first-stage output in
  both launch configurations the autotuner picks between (16x8 tiles / 128
  threads and 32x8 / 256) against the FP64 oracle, every DoF, at the mixed
  bound (1e-5 of each component's scale); the two configurations bit-identical.
- The walled viscous shock tube at 2000 x 1000 (discontinuous data, the limiters
  active): the FP64 residual of every DoF against the oracle (stage output 1e-12,
  raw residual 1e-10, limiter fire sets) and the mixed stage output at 1e-5.
- The batched workload at its full size (256 problems, 13.5 M cells), autotuned
  as the benchmark runs it: one FP64 batch step, and the oracle's step of four
  sampled problems (the largest, the smallest, a near-vacuum blast and one more
  flow) to 1e-12 with equal restart counts.
"""
import numpy as np
import pytest

from conftest import cuda_ok
from paper_2609_29081_b300 import workloads as W
from parity_util import fire_sets_agree, max_rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

C1 = 0.391752226571890   # first SSP-RK54 stage weight
TOL_STAGE = 1e-12
TOL_RES = 1e-10
TOL_MIXED = 1e-5


def oracle_problem(orc, w, lim=2):
    return orc.problem(2, *w.n, lo=w.lo, hi=w.hi, mu=w.mu, Pr=w.Pr, bc=w.bc, gamma=w.gamma, limiter=lim,
                       wall_speed=w.wall_speed)


def stage(state, dt, L):
    return state + C1 * dt * L


@pytest.fixture(scope="module")
def smooth_1024(orc):
    w = W.smooth_2d(1024)
    P = oracle_problem(orc, w)
    dt = orc.dt_max(P, w.state)
    Lr, _ = orc.residual(P, w.state, dt)
    return w, dt, Lr


@pytest.mark.parametrize("cfg", [(16, 8, 128), (32, 8, 256)])
def test_mixed_full_size_stage_in_bench_launch_configs(smooth_1024, cfg):
    from paper_2609_29081_b300 import MIXED, Solver
    w, dt, Lr = smooth_1024
    S = Solver.from_workload(w, precision=MIXED, tile_x=cfg[0], tile_y=cfg[1], threads=cfg[2])
    S.set_state(w.state)
    Lg, _ = S.residual(dt)
    err, where = max_rel_err(stage(w.state, dt, Lg), stage(w.state, dt, Lr), 2, w.n)
    assert err < TOL_MIXED, (cfg, err, where)
    S.close()


def test_mixed_full_size_launch_configs_bit_identical(smooth_1024):
    from paper_2609_29081_b300 import MIXED, Solver
    w, dt, _ = smooth_1024
    out = []
    for cfg in ((16, 8, 128), (32, 8, 256)):
        S = Solver.from_workload(w, precision=MIXED, tile_x=cfg[0], tile_y=cfg[1], threads=cfg[2])
        S.set_state(w.state)
        for _ in range(2):
            S.step(0.0)
        out.append(S.get_state())
        S.close()
    assert np.array_equal(out[0], out[1])


def test_walled_tube_full_size_parity(orc):
    """2000 x 1000, no-slip walls and a symmetry side, pressure ratio 100: every
    DoF of the FP64 residual against the oracle, and the mixed stage output."""
    from paper_2609_29081_b300 import FP64, MIXED, Solver
    w = W.shock_tube_2d()
    assert w.n == (2000, 1000)
    P = oracle_problem(orc, w)
    dt = orc.dt_max(P, w.state)
    Lr, ts_r, tp_r, nb_r = orc.residual(P, w.state, dt, with_theta=True)
    S = Solver.from_workload(w, precision=FP64)
    S.set_state(w.state)
    Lg, nb_g = S.residual(dt)
    err, where = max_rel_err(stage(w.state, dt, Lg), stage(w.state, dt, Lr), 2, w.n)
    assert err < TOL_STAGE, (err, where)
    err, where = max_rel_err(Lg, Lr, 2, w.n)
    assert err < TOL_RES, (err, where)
    ts_g, tp_g = S.limiter()
    assert fire_sets_agree(ts_g, ts_r)[0] and fire_sets_agree(tp_g, tp_r)[0]
    S.close()
    M = Solver.from_workload(w, precision=MIXED)
    M.set_state(w.state)
    Lm, _ = M.residual(dt)
    err, where = max_rel_err(stage(w.state, dt, Lm), stage(w.state, dt, Lr), 2, w.n)
    assert err < TOL_MIXED, (err, where)
    M.close()


def test_batch_full_workload_sampled_problems(orc):
    """The batched workload as benchmarked (256 problems, seed 5), autotuned;
    one FP64 batch step; four sampled problems against the oracle's step."""
    from paper_2609_29081_b300 import FP64, BatchSolver
    wls = W.batch_problems(nprob=256, seed=5)
    B = BatchSolver(wls, precision=FP64)
    for i, w in enumerate(wls):
        B.set_state(i, w.state)
    B.tune()
    B.step_all(1, graph=True)
    B.sync()
    cells = [w.n[0] * w.n[1] for w in wls]
    blasts = [i for i, w in enumerate(wls) if w.state[: w.n[0] * w.n[1]].min() < 1e-3]
    assert blasts
    flows = [i for i in range(len(wls)) if i not in blasts]
    picks = sorted({int(np.argmax(cells)), int(np.argmin(cells)), blasts[0], flows[len(flows) // 2]})
    for i in picks:
        w = wls[i]
        st = B.stats(i)
        assert st["accepted"] + st["restarts"] >= 1 and not st["failed"]
        P = oracle_problem(orc, w)
        s = w.state.copy()
        dt = orc.dt_max(P, s)
        rc, taken, halv = orc.step(P, s, dt)
        assert rc == 0
        if st["accepted"] == 1:
            assert halv == st["restarts"], (i, halv, st)
            got = B.get_state(i)[0]
            err, where = max_rel_err(got, s, 2, w.n)
            assert err < TOL_STAGE, (i, w.n, err, where)
        else:
            # the step is still being halved: the oracle needed at least as many
            assert halv >= st["restarts"], (i, halv, st)
    B.close()
