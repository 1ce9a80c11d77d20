"""Fourth-order convergence of the GPU path on the smooth periodic 2D flow
(grid-refinement ladder, Sec. 4 accuracy tests; no exact solution exists for
the viscous flow, so the error of N cells is measured against the 2N solution
restricted by 2x2 averaging of the cell averages).

FP64 path, limiter off: the observed order between successive ladder rungs
approaches 4 (measured 4.09, 4.23). With the smoothness limiter on (s+pp),
theta_s = exp(-phi1 phi2) of Eq. (22) is 1 - O(dx^2) wherever the flow
compresses, which blends an O(dx^2) share of the first-order LLF flux into the
face flux, so the order degrades toward 3 on this flow (measured 3.61, 3.40);
the test holds it above 3.2. The mixed path is checked on the coarse rungs, where
the discretisation error is far above FP32 roundoff.
"""
import numpy as np
import pytest

from conftest import cuda_ok
from paper_2609_29081_b300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

T_END = 0.2


def averages(n, prec, lim):
    from paper_2609_29081_b300 import FP64, MIXED, Solver
    w = W.smooth_2d(n)
    S = Solver.from_workload(w, precision=FP64 if prec == "fp64" else MIXED, limiter=lim)
    S.set_state(w.state)
    S.advance(T_END)
    return W.split_sites(S.get_state(), 2, n, n)[0]


def restrict(a):
    return 0.25 * (a[:, 0::2, 0::2] + a[:, 1::2, 0::2] + a[:, 0::2, 1::2] + a[:, 1::2, 1::2])


def ladder_orders(ns, prec, lim):
    sol = {n: averages(n, prec, lim) for n in ns}
    err = [np.abs(sol[n] - restrict(sol[2 * n])).sum() / np.abs(sol[n]).sum() for n in ns[:-1]]
    return err, [float(np.log2(err[k] / err[k + 1])) for k in range(len(err) - 1)]


def test_fp64_fourth_order_ladder_unlimited():
    err, orders = ladder_orders([64, 128, 256, 512], "fp64", 0)
    print("fp64 lim 0 L1 errors", err, "orders", orders)
    assert min(orders) > 3.8, (err, orders)


def test_fp64_ladder_with_smoothness_limiter():
    err, orders = ladder_orders([64, 128, 256, 512], "fp64", 2)
    print("fp64 lim 2 L1 errors", err, "orders", orders)
    assert min(orders) > 3.2, (err, orders)


def test_mixed_fourth_order_on_coarse_rungs():
    err, orders = ladder_orders([32, 64, 128], "mixed", 2)
    print("mixed L1 errors", err, "orders", orders)
    assert orders[-1] > 3.5, (err, orders)
