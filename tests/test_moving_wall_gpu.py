"""GPU checks of the moving no-slip wall (the lid of the Sec. 4 cavity) and of
the low-Mach Sec. 4 workloads built on it: Couette flow as a closed-form residual,
the impulsively started plate against erfc, the lid-driven cavity and the double
shear layer against the FP64 oracle, and the batched form on a mix of them."""
from math import erfc, sqrt

import numpy as np
import pytest

from conftest import cuda_ok
from paper_2609_29081_b300 import workloads as W
from parity_util import max_rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


def oracle_problem(orc, w, limiter=2):
    return orc.problem(2, *w.n, lo=w.lo, hi=w.hi, mu=w.mu, Pr=w.Pr, bc=w.bc, gamma=w.gamma, limiter=limiter,
                       wall_speed=w.wall_speed)


def solver(w, prec="fp64", limiter=2):
    from paper_2609_29081_b300 import FP64, MIXED, Solver
    S = Solver.from_workload(w, precision=FP64 if prec == "fp64" else MIXED, limiter=limiter)
    S.set_state(w.state)
    return S


@pytest.mark.parametrize("n", [12, 17])
@pytest.mark.parametrize("limiter", [0, 2])
def test_couette_residual_on_gpu(orc, n, limiter):
    """Couette flow u = U y under a lid moving with U: the GPU residual is
    (0, 0, 0, mu U^2) at every DoF to 1e-12, as the oracle's."""
    w = W.couette_2d(n, U=0.5, mu=1e-2)
    P = oracle_problem(orc, w, limiter)
    dt = 0.5 * orc.dt_max(P, w.state)
    L, nb = solver(w, limiter=limiter).residual(dt)
    assert nb == 0
    for part in W.split_sites(L, 2, n, n):
        assert np.abs(part[:3]).max() < 1e-12
        assert np.abs(part[3] - 1e-2 * 0.25).max() < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_moving_plate_matches_erfc_on_gpu(prec):
    """Rayleigh's plate (U = 0.1, mu = 1e-3, 4 x 100 cells, t = 1): within 2e-4 of
    U erfc(y / (2 sqrt(mu t))) (oracle: 4.7e-5), uniform in x."""
    w = W.moving_plate_2d(100, U=0.1, mu=1e-3)
    S = solver(w, prec)
    S.advance(1.0)
    avg = W.split_sites(S.get_state(), 2, *w.n)[0]
    u = avg[1] / avg[0]
    y = (np.arange(100) + 0.5) / 100
    ex = np.array([0.1 * erfc(yy / (2 * sqrt(1e-3))) for yy in y])
    assert np.abs(u - u[:, :1]).max() < (1e-15 if prec == "fp64" else 1e-6)
    assert np.abs(u[:, 0] - ex).max() < 2e-4


@pytest.mark.parametrize("n", [(24, 24), (21, 19)])
def test_cavity_parity(orc, n):
    """Lid-driven cavity (Re = 100, Mach 0.01): 20 CFL steps of the GPU FP64 path
    within 1e-10 of the oracle, a ragged grid included; the wall point values
    carry the wall velocities (the top corners that of the lid)."""
    w = W.lid_driven_cavity(n, Re=100.0)
    P = oracle_problem(orc, w)
    s = w.state.copy()
    rc, ns, nr = orc.advance(P, s, 0.0, 1e9, max_steps=20)
    S = solver(w)
    for _ in range(20):
        S.step(0.0)
    got = S.get_state()
    err, where = max_rel_err(got, s, 2, w.n)
    assert rc == 0 and err < 1e-10, (err, where)
    vx = W.split_sites(got, 2, *w.n)[3]
    assert np.all(vx[1][-1] == vx[0][-1]) and np.all(vx[2][-1] == 0.0)
    assert np.all(vx[1][:-1, 0] == 0.0) and np.all(vx[1][:-1, -1] == 0.0)


def test_cavity_mixed_tracks_fp64():
    """The mixed path on the cavity: 20 steps within 1e-4 (relative to each
    component's scale) of the GPU FP64 path. At Mach 0.01 the energy (~1.8e4) is
    10^4 times the kinetic energy, so the FP32 point values give the pressure an
    absolute error of ~1e-3 whose differences drive the momentum: the measured
    gap is 2.2e-5 of the momentum scale, a floor of the FP32 storage at low Mach
    (FP64 is the precision for low-Mach accuracy runs)."""
    w = W.lid_driven_cavity(32, Re=1000.0)
    a, b = solver(w), solver(w, "mixed")
    for _ in range(20):
        a.step(0.0)
        b.step(0.0)
    err, where = max_rel_err(b.get_state(), a.get_state(), 2, w.n)
    assert err < 1e-4, (err, where)


def test_double_shear_layer_parity(orc):
    """Double shear layer on 32^2 (mu = 2e-4, Mach 0.01): 10 CFL steps within 1e-10
    of the oracle; mass and momentum of the cell averages conserved to roundoff."""
    w = W.double_shear_layer(32)
    P = oracle_problem(orc, w)
    s = w.state.copy()
    rc, ns, nr = orc.advance(P, s, 0.0, 1e9, max_steps=10)
    S = solver(w)
    for _ in range(10):
        S.step(0.0)
    got = S.get_state()
    err, where = max_rel_err(got, s, 2, w.n)
    assert rc == 0 and err < 1e-10, (err, where)
    a0, a1 = W.split_sites(w.state, 2, *w.n)[0], W.split_sites(got, 2, *w.n)[0]
    for c in range(3):
        assert abs(a1[c].sum() - a0[c].sum()) < 1e-11 * max(1.0, np.abs(a0[c]).sum())


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_of_lid_and_shear_problems_equals_single(prec):
    """A batch of cavities (two Reynolds numbers, two sizes), a double shear layer
    and a Couette problem: each evolves in the batch exactly as alone."""
    from paper_2609_29081_b300 import FP64, MIXED, BatchSolver, Solver
    p = MIXED if prec == "mixed" else FP64
    wls = [W.lid_driven_cavity(24, Re=100.0), W.lid_driven_cavity((40, 32), Re=1000.0),
           W.double_shear_layer(32), W.couette_2d(20)]
    B = BatchSolver(wls, precision=p)
    for i, w in enumerate(wls):
        B.set_state(i, w.state)
    B.step_all(5)
    B.sync()
    for i, w in enumerate(wls):
        got, t = B.get_state(i)
        S = Solver.from_workload(w, precision=p)
        S.set_state(w.state)
        for _ in range(5):
            S.step(0.0)
        ref = S.get_state()
        assert t == S.t and np.array_equal(got, ref), w.name
