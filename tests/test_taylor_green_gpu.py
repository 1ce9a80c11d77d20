"""GPU checks with the manufactured Taylor-Green energy source (Sec. 4 example):
parity with the FP64 oracle at a stage time (residual) and over steps, and
convergence of the GPU path to the exact solution."""
import numpy as np
import pytest

from conftest import cuda_ok
from paper_2609_29081_b300 import workloads as W
from parity_util import max_rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

C1 = 0.391752226571890


def oracle_problem(orc, w, t=0.0):
    return orc.problem(2, *w.n, lo=w.lo, hi=w.hi, mu=w.mu, Pr=w.Pr, gamma=w.gamma, source=1,
                       src_p0=w.src_p0, time=t)


def solver(w, prec="fp64", t=0.0):
    from paper_2609_29081_b300 import FP64, MIXED, Solver
    S = Solver.from_workload(w, precision=FP64 if prec == "fp64" else MIXED)
    S.set_state(w.state, t)
    return S


@pytest.mark.parametrize("n", [20, 37])
def test_source_residual_parity(orc, n):
    """L(u) with the source at t = 0.05 (a ragged grid included): 1e-12 on
    u + c dt L. The raw energy residual is the O(mu) time derivative of a nearly
    steady flow, formed from flux differences and a source of size O(1)-O(10^3),
    so it is held to 1e-7 of its own scale (roundoff of the terms / the result)."""
    t = 0.05
    w = W.taylor_green_2d(n, t=t)
    P = oracle_problem(orc, w, t)
    S = solver(w, t=t)
    dt = 0.8 * orc.dt_max(P, w.state)
    Lr, nb_r = orc.residual(P, w.state, dt)
    Lg, nb_g = S.residual(dt)
    assert max_rel_err(Lg, Lr, 2, w.n)[0] < 1e-7
    err, where = max_rel_err(w.state + C1 * dt * Lg, w.state + C1 * dt * Lr, 2, w.n)
    assert err < 1e-12, (err, where)


def test_source_ten_steps_parity(orc):
    """Ten CFL steps from t = 0 (stage times of every RK stage enter the source)."""
    w = W.taylor_green_2d(24)
    P = oracle_problem(orc, w)
    s = w.state.copy()
    rc, ns, nr = orc.advance(P, s, 0.0, 1e9, max_steps=10)
    S = solver(w)
    for _ in range(10):
        S.step(0.0)
    err, where = max_rel_err(S.get_state(), s, 2, w.n)
    assert rc == 0 and err < 1e-10, (err, where)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gpu_converges_to_exact_taylor_green(prec):
    """L1 error of the cell averages against the exact solution at t = 0.2.
    FP64 on 32^2, 64^2, 128^2: observed order above 3.5 in every component
    (measured 3.84/4.91/4.91/3.74, then 3.97/4.77/4.77/3.93). Mixed on 16^2, 32^2,
    64^2: the FP32 point values (E ~ 625, FP32 spacing ~6e-5) put a floor of a
    few 1e-8 (density) and 1e-5 (energy) under the error, reached from 32^2 on;
    above it the mixed errors stay within 1.6x of the FP64 ones and the momentum
    order is above 4 (measured 4.85)."""
    T = 0.2
    ns = (32, 64, 128) if prec == "fp64" else (16, 32)
    errs = []
    for n in ns:
        w = W.taylor_green_2d(n)
        S = solver(w, prec)
        S.advance(T)
        ex = W.taylor_green_2d(n, t=T).state
        g = W.split_sites(S.get_state(), 2, n, n)[0]
        errs.append(np.abs(g - W.split_sites(ex, 2, n, n)[0]).sum(axis=(1, 2)) / n ** 2)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    print(prec, "L1 errors", errs, "orders", orders)
    if prec == "fp64":
        assert orders[-1].min() > 3.5, (errs, orders)
    else:
        ref = []
        for n in ns:
            w = W.taylor_green_2d(n)
            S = solver(w, "fp64")
            S.advance(T)
            g = W.split_sites(S.get_state(), 2, n, n)[0]
            ref.append(np.abs(g - W.split_sites(W.taylor_green_2d(n, t=T).state, 2, n, n)[0]).sum(axis=(1, 2)) / n ** 2)
        assert np.all(np.array(errs) < 1.6 * np.array(ref)), (errs, ref)
        assert orders[-1][1:3].min() > 4.0, (errs, orders)
