"""GPU parity of the 1D CUDA path against the CPU oracle, through the C-ABI
(configurations: smooth periodic N=128 to t=0.5; viscous shock tube N=4096)."""
import numpy as np
import pytest

from conftest import cuda_ok
from paper_2609_29081_b300 import workloads as W
from parity_util import max_rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

C1 = 0.391752226571890


def make(orc, w, lim=2):
    from paper_2609_29081_b300 import Solver
    P = orc.problem(1, w.n[0], lo=w.lo, hi=w.hi, mu=w.mu, Pr=w.Pr, bc=w.bc, limiter=lim, gamma=w.gamma)
    S = Solver.from_workload(w, limiter=lim)
    S.set_state(w.state)
    return P, S


def walled_tube(n):
    w = W.shock_tube_1d(n)
    w.bc = (1, 2, 0, 0)
    return w


CASES = {
    "smooth_128": lambda: W.smooth_1d(128),
    "smooth_ragged_37": lambda: W.smooth_1d(37),
    "smooth_ragged_200": lambda: W.smooth_1d(200, mu=0.05),
    "tube_4096": lambda: W.shock_tube_1d(4096),
    "tube_walls_130": lambda: walled_tube(130),
    "entropy_70": lambda: W.entropy_wave_1d(70),
    "tiny_4": lambda: W.smooth_1d(4),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("lim", [0, 1, 2])
def test_residual_parity_1d(orc, case, lim):
    w = CASES[case]()
    P, S = make(orc, w, lim)
    dt = 0.9 * orc.dt_max(P, w.state)
    assert S.dt_max() == pytest.approx(orc.dt_max(P, w.state), rel=1e-14)
    Lr, ts, tp, nb_r = orc.residual(P, w.state, dt, with_theta=True)
    Lg, nb_g = S.residual(dt)
    assert max_rel_err(Lg, Lr, 1, w.n)[0] < 1e-10
    err, where = max_rel_err(w.state + C1 * dt * Lg, w.state + C1 * dt * Lr, 1, w.n)
    assert err < 1e-12, (err, where)
    assert nb_g == nb_r
    if lim:
        tsg, tpg = S.limiter()
        assert np.abs(tsg - ts).max() < 1e-10 and np.abs(tpg - tp).max() < 1e-10


@pytest.mark.parametrize("case", sorted(CASES))
def test_one_step_parity_1d(orc, case):
    w = CASES[case]()
    P, S = make(orc, w)
    dt = orc.dt_max(P, w.state)
    s = w.state.copy()
    rc, taken, h = orc.step(P, s, dt)
    tg, hg = S.step(dt)
    assert rc == 0 and (tg, hg) == (taken, h)
    err, where = max_rel_err(S.get_state(), s, 1, w.n)
    assert err < 1e-12, (err, where)


def test_smooth_periodic_to_t_end(orc):
    """Configuration 1 in full: N = 128 to t = 0.5 with CFL steps."""
    w = W.smooth_1d(128)
    P, S = make(orc, w)
    s = w.state.copy()
    rc, ns, nr = orc.advance(P, s, 0.0, 0.5)
    ns_g, nr_g = S.advance(0.5)
    assert rc == 0 and (ns_g, nr_g) == (ns, nr)
    err, where = max_rel_err(S.get_state(), s, 1, w.n)
    assert err < 1e-10, (err, where)


def test_shock_tube_first_100_steps(orc):
    """Configuration 2 (N = 4096, limiters active): 100 CFL steps against the oracle."""
    w = W.shock_tube_1d(4096)
    P, S = make(orc, w)
    s = w.state.copy()
    rc, ns, nr = orc.advance(P, s, 0.0, 1e9, max_steps=100)
    for _ in range(100):
        S.step(0.0)
    err, where = max_rel_err(S.get_state(), s, 1, w.n)
    assert rc == 0 and err < 1e-10, (err, where)


def test_shock_tube_full_run_positive():
    """Configuration 2 in full on the GPU (to t = 0.2): positivity of every DoF,
    mass change only through the shock's thermal precursor at the right end."""
    from paper_2609_29081_b300 import Solver
    w = W.shock_tube_1d(4096)
    S = Solver.from_workload(w)
    S.set_state(w.state)
    m0 = W.split_sites(w.state, 1, 4096)[0][0].sum()
    ns, nr = S.advance(0.2)
    s = S.get_state()
    avg, pt = W.split_sites(s, 1, 4096)
    for U in (avg, pt):
        p = 0.4 * (U[2] - 0.5 * U[1] ** 2 / U[0])
        assert np.isfinite(U).all() and U[0].min() > 0 and p.min() > 0
    assert abs(avg[0].sum() - m0) < 1e-6 * m0
    assert S.t == pytest.approx(0.2, abs=1e-14) and ns > 1000
