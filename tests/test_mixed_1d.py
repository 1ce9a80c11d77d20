"""GPU checks of the mixed-precision 1D path (FP32 storage and stencils, FP64
limiters and FP64-formed compensated cell updates) against the FP64 oracle:
the smooth periodic wave and the viscous shock tube of Sec. 4 (N = 4096).

The error against the FP64 oracle is bounded by FP32 roundoff (1e-5 of each
component's scale after one stage and after 10 steps), mass is conserved to
1e-13 on a periodic grid, and the shock tube keeps rho, p > 0.
"""
import numpy as np
import pytest

from conftest import cuda_ok
from paper_2609_29081_b300 import workloads as W
from parity_util import max_rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

C1 = 0.391752226571890

CASES = {
    "smooth_128": lambda: W.smooth_1d(128),
    "smooth_ragged_200": lambda: W.smooth_1d(200, mu=0.05),
    "tube_4096": lambda: W.shock_tube_1d(4096),
}


def mixed(w, lim=2):
    from paper_2609_29081_b300 import MIXED, Solver
    S = Solver.from_workload(w, precision=MIXED, limiter=lim)
    S.set_state(w.state)
    return S


@pytest.mark.parametrize("case", sorted(CASES))
def test_mixed_1d_stage_against_fp64_oracle(orc, case):
    w = CASES[case]()
    P = orc.problem(1, w.n[0], lo=w.lo, hi=w.hi, mu=w.mu, Pr=w.Pr, bc=w.bc, gamma=w.gamma)
    S = mixed(w)
    dt = 0.8 * orc.dt_max(P, w.state)
    Lr, nb_r = orc.residual(P, w.state, dt)
    Lg, nb_g = S.residual(dt)
    err, where = max_rel_err(w.state + C1 * dt * Lg, w.state + C1 * dt * Lr, 1, w.n)
    assert err < 1e-5, (err, where)
    assert nb_g == nb_r


@pytest.mark.parametrize("case", sorted(CASES))
def test_mixed_1d_ten_steps_against_fp64_oracle(orc, case):
    w = CASES[case]()
    P = orc.problem(1, w.n[0], lo=w.lo, hi=w.hi, mu=w.mu, Pr=w.Pr, bc=w.bc, gamma=w.gamma)
    S = mixed(w)
    s = w.state.copy()
    rc, ns, nr = orc.advance(P, s, 0.0, 1e9, max_steps=10)
    for _ in range(10):
        S.step(0.0)
    g = S.get_state()
    err, where = max_rel_err(g, s, 1, w.n)
    assert rc == 0 and err < 2e-5, (err, where)
    ga, sa = W.split_sites(g, 1, *w.n)[0], W.split_sites(s, 1, *w.n)[0]
    assert np.abs(ga - sa).sum() / np.abs(sa).sum() < 2e-6


def test_mixed_1d_conserves_and_tube_stays_positive():
    w = W.smooth_1d(128)
    S = mixed(w)
    m0 = W.split_sites(w.state, 1, 128)[0].sum(axis=1)
    for _ in range(100):
        S.step(0.0)
    m1 = W.split_sites(S.get_state(), 1, 128)[0].sum(axis=1)
    scale = np.abs(W.split_sites(w.state, 1, 128)[0]).sum(axis=1)
    assert np.all(np.abs(m1 - m0) < 1e-13 * scale), (m1 - m0) / scale
    t = W.shock_tube_1d(4096)
    S = mixed(t)
    S.advance(0.02)
    for U in W.split_sites(S.get_state(), 1, 4096):
        p = 0.4 * (U[2] - 0.5 * U[1] ** 2 / U[0])
        assert np.isfinite(U).all() and U[0].min() > 0 and p.min() > 0
