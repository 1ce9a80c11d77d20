"""GPU checks of the mixed-precision 2D path (FP32 stencils and storage, FP64
positivity islands, float-float cell averages) against the FP64 oracle.

The mixed path is not expected to reproduce FP64 to 1e-12; its error against the
FP64 oracle is measured and bounded by FP32 roundoff (stage: 1e-5 of each
component's scale), it must conserve mass to 1e-12 (compensated averages), keep
positivity, and stay far below the discretisation error of the grid.
"""
import numpy as np
import pytest

from conftest import cuda_ok
from paper_2609_29081_b300 import workloads as W
from parity_util import max_rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

C1 = 0.391752226571890


def solver(w, precision, lim=2):
    from paper_2609_29081_b300 import MIXED, FP64, Solver
    S = Solver.from_workload(w, precision=MIXED if precision == "mixed" else FP64, limiter=lim)
    S.set_state(w.state)
    return S


def l1_rel(a, b, n):
    sa = W.split_sites(a, 2, *n)[0]
    sb = W.split_sites(b, 2, *n)[0]
    return float(np.abs(sa - sb).sum() / np.abs(sb).sum())


CASES = {
    "periodic_ragged_33x17": lambda: W.random_smooth_2d((33, 17), seed=3),
    "walls_16x8": lambda: W.random_smooth_2d((16, 8), seed=2, bc=(1, 1, 1, 2)),
    "outflow_sym_35x19": lambda: W.random_smooth_2d((35, 19), seed=4, bc=(3, 3, 2, 2)),
    "shock_tube_36x18": lambda: W.shock_tube_2d((36, 18)),
    "smooth_2d_64": lambda: W.smooth_2d(64),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_mixed_stage_against_fp64_oracle(orc, case):
    w = CASES[case]()
    P = orc.problem(2, *w.n, lo=w.lo, hi=w.hi, mu=w.mu, Pr=w.Pr, bc=w.bc, gamma=w.gamma)
    S = solver(w, "mixed")
    dt = 0.8 * orc.dt_max(P, w.state)
    Lr, nb_r = orc.residual(P, w.state, dt)
    Lg, nb_g = S.residual(dt)
    err, where = max_rel_err(w.state + C1 * dt * Lg, w.state + C1 * dt * Lr, 2, w.n)
    assert err < 1e-5, (err, where)
    assert nb_g == nb_r


@pytest.mark.parametrize("case", sorted(CASES))
def test_mixed_ten_steps_against_fp64_oracle(orc, case):
    w = CASES[case]()
    P = orc.problem(2, *w.n, lo=w.lo, hi=w.hi, mu=w.mu, Pr=w.Pr, bc=w.bc, gamma=w.gamma)
    S = solver(w, "mixed")
    s = w.state.copy()
    rc, ns, nr = orc.advance(P, s, 0.0, 1e9, max_steps=10)
    for _ in range(10):
        S.step(0.0)
    g = S.get_state()
    err, where = max_rel_err(g, s, 2, w.n)
    assert rc == 0 and err < 2e-5, (err, where)
    assert l1_rel(g, s, w.n) < 2e-6


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_launch_configuration_does_not_change_results(prec):
    """Tile shape and CTA size (autotuned) change no bit of the result."""
    from paper_2609_29081_b300 import MIXED, FP64, Solver
    w = W.random_smooth_2d((70, 37), seed=13, bc=(1, 1, 2, 3))
    p = MIXED if prec == "mixed" else FP64
    outs = []
    for tx, ty in (((16, 8), (32, 8), (16, 16), (32, 16)) if prec == "mixed" else ((16, 8), (16, 16))):
        S = Solver.from_workload(w, precision=p, tile_x=tx, tile_y=ty)
        S.set_state(w.state)
        r0, _ = S.residual(1e-3)
        cfg = S.tune()
        r1, _ = S.residual(1e-3)
        assert np.array_equal(r0, r1), cfg
        for _ in range(3):
            S.step(0.0)
        outs.append(S.get_state())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_mixed_conserves_and_stays_positive():
    """Compensated cell averages: mass, momentum, energy conserved to 1e-12 on a
    periodic grid after 50 steps; a near-vacuum blast keeps positivity."""
    w = W.random_smooth_2d((48, 40), seed=12)
    S = solver(w, "mixed")
    m0 = W.split_sites(w.state, 2, *w.n)[0].sum(axis=(1, 2))
    for _ in range(50):
        S.step(0.0)
    m1 = W.split_sites(S.get_state(), 2, *w.n)[0].sum(axis=(1, 2))
    scale = np.abs(W.split_sites(w.state, 2, *w.n)[0]).sum(axis=(1, 2))
    assert np.all(np.abs(m1 - m0) < 1e-12 * scale), (m1 - m0) / scale
    b = W.blast_2d((32, 32), seed=3)
    S = solver(b, "mixed")
    restarts = 0
    for _ in range(30):
        restarts += S.step(0.0)[1]
    for U in W.split_sites(S.get_state(), 2, 32, 32):
        p = 0.4 * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0])
        assert np.isfinite(U).all() and U[0].min() > 0 and p.min() > 0


def test_mixed_error_below_discretisation_error():
    """On the smooth periodic workload the FP32 error (mixed vs FP64 on the same
    grid) must stay below the discretisation error, estimated as the distance
    between the FP64 solutions on N and 2N cells (2x2 restriction of averages).
    At 64^2 the discretisation error is ~1e-6; the FP32 error is ~1e-8. (The
    fourth-order discretisation error falls as N^-4 while FP32 roundoff does not,
    so on fine grids of smooth flows FP32 becomes the larger error; the benchmark
    states both.)"""
    n, t_end = 64, 0.2
    sol = {}
    for key, nn, prec in (("f64", n, "fp64"), ("mix", n, "mixed"), ("fine", 2 * n, "fp64")):
        w = W.smooth_2d(nn)
        S = solver(w, prec)
        S.advance(t_end)
        sol[key] = W.split_sites(S.get_state(), 2, nn, nn)[0]
    fine = sol["fine"]
    restr = 0.25 * (fine[:, 0::2, 0::2] + fine[:, 1::2, 0::2] + fine[:, 0::2, 1::2] + fine[:, 1::2, 1::2])
    disc = np.abs(sol["f64"] - restr).sum() / np.abs(restr).sum()
    fp32 = np.abs(sol["mix"] - sol["f64"]).sum() / np.abs(sol["f64"]).sum()
    assert fp32 < disc, (fp32, disc)


def test_f32_state_io():
    """FP32 site arrays in and out of a mixed context: the round trip is exact,
    stepping from FP32 input equals stepping from the same values given in FP64,
    and an FP64 context refuses FP32 arrays."""
    from paper_2609_29081_b300 import FP64, MIXED, AfnsError, Solver
    w = W.random_smooth_2d((33, 17), seed=3)
    s32 = w.state.astype(np.float32)
    S = Solver.from_workload(w, precision=MIXED)
    S.set_state_f32(s32)
    assert np.array_equal(S.get_state_f32(), s32)
    R = Solver.from_workload(w, precision=MIXED)
    R.set_state(s32.astype(np.float64))
    for _ in range(3):
        S.step(0.0)
        R.step(0.0)
    assert np.array_equal(S.get_state(), R.get_state())
    F = Solver.from_workload(w, precision=FP64)
    with pytest.raises(AfnsError):
        F.set_state_f32(s32)


def test_f32_upload_checks_values():
    """An FP32 upload is checked as it is unpacked: a negative density, a negative
    pressure or a NaN anywhere, and a periodic duplicate point that differs from
    its partner, are refused; a clean state after a refused one is accepted
    (the check starts from zero on every call)."""
    from paper_2609_29081_b300 import MIXED, AfnsError, Solver
    w = W.random_smooth_2d((33, 17), seed=4)
    S = Solver.from_workload(w, precision=MIXED)
    n1, n2 = w.n
    avg = 4 * n1 * n2
    xe = avg + 4 * n2 * (n1 + 1)
    for where, value in ((5, -1.0), (avg + 7, np.nan), (3 * n1 * n2 + 11, -50.0)):
        bad = w.state.astype(np.float32)
        bad[where] = value
        with pytest.raises(AfnsError):
            S.set_state_f32(bad)
        S.set_state_f32(w.state.astype(np.float32))
    bad = w.state.astype(np.float32)
    bad[xe - 4 * n2 * (n1 + 1) + n1] *= 1.001     # x-edge density at i = n1 (duplicate of i = 0), row 0
    with pytest.raises(AfnsError):
        S.set_state_f32(bad)
    S.set_state_f32(w.state.astype(np.float32))
    assert np.array_equal(S.get_state_f32(), w.state.astype(np.float32))


def test_f32_upload_check_is_exact_at_zero_pressure():
    """The FP32 upload check decides p > 0 exactly, also where 2 rho E and |m|^2
    agree to FP32 rounding (its FP32 screen leaves those to FP64): E = 1/2 + 2^-24
    with rho = m_x = 1 has p > 0 and is accepted; E = 1/2 (p = 0) and
    E = 1/2 - 2^-25 (p < 0) are refused, for a cell average and for a vertex."""
    from paper_2609_29081_b300 import MIXED, AfnsError, Solver
    w = W.random_smooth_2d((33, 17), seed=6)
    S = Solver.from_workload(w, precision=MIXED)
    n1, n2 = w.n
    vert = 4 * n1 * n2 + 4 * (n1 + 1) * n2 + 4 * n1 * (n2 + 1)
    for base, stride in ((0, n1 * n2), (vert, (n1 + 1) * (n2 + 1))):
        k = base + 2 * (n1 + (1 if base else 0)) + 3      # (i, j) = (3, 2)
        for E, ok in ((0.5 + 2.0 ** -24, True), (0.5, False), (0.5 - 2.0 ** -25, False)):
            s = w.state.astype(np.float32)
            s[k], s[k + stride], s[k + 2 * stride], s[k + 3 * stride] = 1.0, 1.0, 0.0, E
            assert float(np.float32(E)) == E
            if ok:
                S.set_state_f32(s)
                assert np.array_equal(S.get_state_f32(), s)
            else:
                with pytest.raises(AfnsError):
                    S.set_state_f32(s)
