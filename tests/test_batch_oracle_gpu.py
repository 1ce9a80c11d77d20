"""GPU parity of the batched persistent path (afb_*) against the CPU oracle
directly, through the C-ABI.

The batched kernel is separate code around the single-problem tile function
(a work list over problems, per-problem tensor maps, descriptors and tile
constants, a device-side commit / halving kernel), so it is held to the oracle
itself, not only to the single path: FP64 after one batch step to 1e-12 and after several
to 1e-10 of each component's scale, with each problem's accepted steps and
restarts (Remark 3.2) equal to the oracle's; the mixed form against the FP64
oracle at the single-path mixed bounds. The batch holds problems of the
batched workload's recipe at multi-tile sizes (non-square, 128 x 192 cells),
a near-vacuum blast that restarts, a walled box, a lid-driven cavity (moving
wall) and uneven mu / Pr.
"""
import numpy as np
import pytest

from conftest import cuda_ok
from paper_2609_29081_b300 import workloads as W
from parity_util import max_rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

TOL_STEP = 1e-12
TOL_STEPS = 1e-10


def batch_cases():
    """(name, workload) pairs; sizes span several 16 x 8 tiles with ragged tails."""
    flows = [w for w in W.batch_problems(nprob=24, seed=5, sizes=(128, 192), blast_frac=0.0)
             if w.n[0] != w.n[1]]
    flow = flows[0]
    flow.Pr = 0.9
    blast = W.blast_2d((64, 48), seed=2, mu=3e-4, rho_min=1e-10, p_min=1e-12)
    walls = W.random_smooth_2d((40, 28), seed=31, bc=(1, 1, 2, 3), mu=0.004, Pr=0.5)
    cavity = W.lid_driven_cavity((36, 30), Re=400.0)
    small = W.random_smooth_2d((21, 19), seed=32, mu=0.02, Pr=1.3)
    return [("flow_%dx%d" % flow.n, flow), ("blast_64x48", blast), ("walls_40x28", walls),
            ("cavity_36x30", cavity), ("smooth_21x19", small)]


def oracle_problem(orc, w):
    return orc.problem(2, *w.n, lo=w.lo, hi=w.hi, mu=w.mu, Pr=w.Pr, bc=w.bc, gamma=w.gamma, limiter=2,
                       wall_speed=w.wall_speed)


def run_batch(cases, precision, nsteps):
    """Advance the batch one graph-replayed step at a time; returns per problem
    the states after the first step and at the end, the final counters, and the
    number of trailing rejected steps (restarts of a step not yet accepted)."""
    from paper_2609_29081_b300 import BatchSolver
    wls = [w for _, w in cases]
    B = BatchSolver(wls, precision=precision)
    for i, w in enumerate(wls):
        B.set_state(i, w.state)
    first, trailing = [], [0] * len(wls)
    prev = [0] * len(wls)
    for k in range(nsteps):
        B.step_all(1, graph=True)
        B.sync()
        for i in range(len(wls)):
            a = B.stats(i)["accepted"]
            trailing[i] = 0 if a > prev[i] else trailing[i] + 1
            prev[i] = a
        if k == 0:
            first = [B.get_state(i)[0] for i in range(len(wls))]
    final = [B.get_state(i)[0] for i in range(len(wls))]
    stats = [B.stats(i) for i in range(len(wls))]
    return first, final, stats, trailing


def oracle_run(orc, w, steps):
    P = oracle_problem(orc, w)
    s = w.state.copy()
    rc, ns, nr = orc.advance(P, s, 0.0, 1e9, max_steps=steps)
    assert rc == 0 and ns == steps
    return s, nr


NSTEPS = 8


@pytest.fixture(scope="module")
def fp64_run():
    from paper_2609_29081_b300 import FP64
    cases = batch_cases()
    return cases, run_batch(cases, FP64, NSTEPS)


@pytest.mark.parametrize("k", range(5))
def test_batch_fp64_first_step_matches_oracle(orc, fp64_run, k):
    cases, (first, _, stats, _) = fp64_run
    name, w = cases[k]
    got = first[k]
    # the oracle's step holds its halvings; a first batch step that was rejected
    # instead leaves u^n and halves in the next batch step
    P = oracle_problem(orc, w)
    s = w.state.copy()
    rc, taken, halv = orc.step(P, s, orc.dt_max(P, s))
    assert rc == 0
    if halv:
        assert np.array_equal(got, w.state)   # the batch kept u^n and halves in its next step
        return
    err, where = max_rel_err(got, s, 2, w.n)
    assert err < TOL_STEP, (name, err, where)


@pytest.mark.parametrize("k", range(5))
def test_batch_fp64_steps_match_oracle_with_equal_restarts(orc, fp64_run, k):
    cases, (_, final, stats, trailing) = fp64_run
    name, w = cases[k]
    acc, rst = stats[k]["accepted"], stats[k]["restarts"]
    assert stats[k]["failed"] == 0 and acc + rst == NSTEPS
    ref, nr = oracle_run(orc, w, acc)
    assert nr == rst - trailing[k], (name, nr, rst, trailing[k])
    err, where = max_rel_err(final[k], ref, 2, w.n)
    assert err < TOL_STEPS, (name, err, where)


def test_batch_blast_restarts(fp64_run):
    """The near-vacuum member does restart, and only it."""
    cases, (_, _, stats, _) = fp64_run
    names = [c[0] for c in cases]
    b = names.index("blast_64x48")
    assert stats[b]["restarts"] > 0
    for i, st in enumerate(stats):
        if i != b:
            assert st["restarts"] == 0 and st["accepted"] == NSTEPS


def test_batch_mixed_tracks_fp64_oracle(orc):
    """Mixed batch against the FP64 oracle at the single-path mixed bounds
    (max 2e-5 of each component's scale, relative L1 of the cell averages 2e-6)
    on the problems whose step sequence matches the oracle's. The Mach 0.01
    cavity is held to its single-path bound (1e-4): its energy is 1e4 times its
    kinetic energy, so FP32 point values carry 1e-3 absolute pressure error."""
    from paper_2609_29081_b300 import MIXED
    cases = batch_cases()
    nsteps = 6
    _, final, stats, trailing = run_batch(cases, MIXED, nsteps)
    for k, (name, w) in enumerate(cases):
        acc = stats[k]["accepted"]
        ref, nr = oracle_run(orc, w, acc)
        if name.startswith("blast"):
            # positivity of every DoF; the restart sequence may differ from FP64's
            for U in W.split_sites(final[k], 2, *w.n):
                p = (w.gamma - 1) * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0])
                assert np.isfinite(U).all() and U[0].min() > 0 and p.min() > 0
            continue
        assert acc == nsteps and nr == 0
        err, where = max_rel_err(final[k], ref, 2, w.n)
        sa = W.split_sites(final[k], 2, *w.n)[0]
        sb = W.split_sites(ref, 2, *w.n)[0]
        l1 = float(np.abs(sa - sb).sum() / np.abs(sb).sum())
        if name.startswith("cavity"):
            assert err < 1e-4, (name, err, where)
        else:
            assert err < 2e-5 and l1 < 2e-6, (name, err, l1, where)


def test_batch_largest_problem_one_step_matches_oracle(orc):
    """The largest grid of the batched workload (sides up to 512), non-square, in
    a batch with a small problem: one FP64 batch step equals one oracle step to
    1e-12 (many full tiles in both directions and ragged work-list neighbours)."""
    from paper_2609_29081_b300 import FP64
    big = [w for w in W.batch_problems(nprob=40, seed=7, sizes=(384, 512), blast_frac=0.0) if w.n[0] != w.n[1]][0]
    small = W.random_smooth_2d((20, 13), seed=33)
    cases = [("big_%dx%d" % big.n, big), ("small_20x13", small)]
    first, _, stats, _ = run_batch(cases, FP64, 1)
    for k, (name, w) in enumerate(cases):
        assert stats[k]["accepted"] == 1 and stats[k]["restarts"] == 0
        P = oracle_problem(orc, w)
        s = w.state.copy()
        rc, taken, halv = orc.step(P, s, orc.dt_max(P, s))
        assert rc == 0 and halv == 0
        err, where = max_rel_err(first[k], s, 2, w.n)
        assert err < TOL_STEP, (name, err, where)
