"""Von Neumann analysis of the viscous part of the compact AF scheme, written
from the paper's formulas in numpy (it does not use the oracle or the CUDA
library): the stable viscous CFL number of Eq. (13) for SSP-RK54.

Linearised about a fluid at rest (rho = 1, u = v = 0), the viscous terms of
Eq. (1) split into the momentum system
    m_t = div(K grad (u, v)),  K_11 = diag(4/3, 1) mu, K_22 = diag(1, 4/3) mu,
    K_12 = [[0, -2/3], [1, 0]] mu, K_21 = [[0, 1], [-2/3, 0]] mu,
and the temperature equation T_t = (gamma mu / Pr) Lap T (Sec. 2.2). Both are
discretised exactly as the scheme does it:
  - cell centres by the Simpson inversion of Sec. 2.1 / Sec. 2.2;
  - point values by the compact D^2 of Eqs. (9)-(10) (the B matrix, with K at
    every stencil node) and the mixed terms D_c^(l)(K_lm D_c^(m) Z) of Eq. (12);
  - cell averages by the difference of the Simpson edge averages of the viscous
    flux K_l1 D_c^(1) Z + K_l2 D_c^(2) Z (Eq. (12)), D_c of Eq. (8) along the
    lattice lines through each node.
Per Fourier mode the operator is a small matrix on the DoFs of one cell (cell
average plus the point sites); its eigenvalues times dt must lie in the
stability region of SSP-RK54 (the Shu-Osher coefficients of Spiteri and Ruuth,
applied to y' = z y). With dt = C Delta x^2 / rho~ as in Eq. (13) the largest
stable C is found by bisection.

What this pins: in 1D the limit is the printed C^v = 0.33 (to 2 %); in 2D the
printed 0.33/2 is not stable for the scheme's own operator: the limit is 0.1307
where heat conduction dominates the bound (the largest eigenvalue of the 2D
operator is 40.8 / dx^2, against 2 x 16 / dx^2 for two 1D operators) and 0.149
where the 4/3 mu of the momentum system does; the 2D default of the oracle and
the library, 0.13, lies just below the smaller one.
"""
import numpy as np
import pytest

# B of Eq. (10): rows m = -2..2, columns n = -2..2, from
# B = [[0, 0], [0, M]] - [[M, 0], [0, 0]] with the 4 x 4 M printed there.
M10 = np.array([[1 / 8, -1 / 6, 1 / 24, 0.0],
                [-1 / 6, -3 / 8, 2 / 3, -1 / 8],
                [1 / 8, -2 / 3, 3 / 8, 1 / 6],
                [0.0, -1 / 24, 1 / 6, -1 / 8]])
B10 = np.zeros((5, 5))
B10[1:, 1:] += M10
B10[:4, :4] -= M10

# Shu-Osher form of SSP-RK54 (Spiteri & Ruuth 2002): u_k = sum_j a_kj u_j + b_k dt L(u_{s_k})
SSP54 = [
    ({0: 1.0}, 0.391752226571890, 0),
    ({0: 0.444370493651235, 1: 0.555629506348765}, 0.368410593050371, 1),
    ({0: 0.620101851488403, 2: 0.379898148511597}, 0.251891774271694, 2),
    ({0: 0.178079954393132, 3: 0.821920045606868}, 0.544974750228521, 3),
]


def rk_amplification(z):
    """R(z) of SSP-RK54 for y' = (z / dt) y."""
    u = [np.ones_like(z)]
    for coef, b, src in SSP54:
        u.append(sum(c * u[j] for j, c in coef.items()) + b * z * u[src])
    u5 = (0.517231671970585 * u[2] + 0.096059710526147 * u[3] + 0.063692468666290 * z * u[3]
          + 0.386708617503269 * u[4] + 0.226007483236906 * z * u[4])
    return u5


def test_rk_polynomial_is_fourth_order():
    """R(z) of a five-stage scheme is a degree-5 polynomial; for fourth order its
    first five coefficients are those of exp(z): 1, 1, 1/2, 1/6, 1/24."""
    z = np.linspace(-1.0, 1.0, 6)
    coef = np.polynomial.polynomial.polyfit(z, rk_amplification(z), 5)
    assert np.allclose(coef[:5], [1, 1, 1 / 2, 1 / 6, 1 / 24], atol=1e-12, rtol=0)
    assert 0 < coef[5] < 1 / 120
    z = np.linspace(-2.0, 2.0, 9)
    assert np.allclose(np.polynomial.polynomial.polyval(z, coef), rk_amplification(z), atol=1e-12)


class Lattice2D:
    """Bloch-wave evaluation of the 2D scheme's linear viscous operator.

    Lattice node (a, b) sits at (a dx/2, b dy/2); vertices at (even, even),
    x-edge points at (even, odd), y-edge points at (odd, even), cell centres at
    (odd, odd). For phases (px, py) per cell, the DoF family s has value
    A[s] exp(i (px a + py b)/2) at its nodes; A[0] is the cell average (placed at
    the centre). ncomp components per node."""

    def __init__(self, px, py, dx, dy, A):
        self.px, self.py, self.dx, self.dy, self.A = px, py, dx, dy, A

    def phase(self, a, b):
        return np.exp(0.5j * (self.px * a + self.py * b))

    def site(self, a, b):
        ea, eb = a % 2 == 0, b % 2 == 0
        return 3 if (ea and eb) else 1 if ea else 2 if eb else 0

    def z(self, a, b):
        s = self.site(a, b)
        if s != 0:
            return self.A[s] * self.phase(a, b)
        # Simpson inversion of Sec. 2.2: 16 z_c = 36 zbar - 4 sum(edges) - sum(vertices)
        edges = self.z(a - 1, b) + self.z(a + 1, b) + self.z(a, b - 1) + self.z(a, b + 1)
        verts = self.z(a - 1, b - 1) + self.z(a + 1, b - 1) + self.z(a - 1, b + 1) + self.z(a + 1, b + 1)
        return (36.0 * self.A[0] * self.phase(a, b) - 4.0 * edges - verts) / 16.0

    # D_c of Eq. (8) along x / y at node (a, b), applied to a node function g
    def dcx(self, g, a, b):
        return (g(a - 2, b) - 8 * g(a - 1, b) + 8 * g(a + 1, b) - g(a + 2, b)) / (6 * self.dx)

    def dcy(self, g, a, b):
        return (g(a, b - 2) - 8 * g(a, b - 1) + 8 * g(a, b + 1) - g(a, b + 2)) / (6 * self.dy)

    # compact second derivative of Eq. (9) with K evaluated at every node (constant here)
    def d2x(self, K, a, b):
        return 4 / self.dx ** 2 * sum(B10[m + 2, n + 2] * (K @ self.z(a + n, b))
                                      for m in range(-2, 3) for n in range(-2, 3))

    def d2y(self, K, a, b):
        return 4 / self.dy ** 2 * sum(B10[m + 2, n + 2] * (K @ self.z(a, b + n))
                                      for m in range(-2, 3) for n in range(-2, 3))


def operator_2d(K, px, py, dx=1.0, dy=1.0):
    """Matrix of the linear viscous residual on the DoFs of one cell (sites avg,
    x-edge, y-edge, vertex, each with ncomp components) for the Bloch phases."""
    K11, K12, K21, K22 = K
    nc = K11.shape[0]
    reps = {0: (1, 1), 1: (2, 1), 2: (1, 2), 3: (2, 2)}
    Mop = np.zeros((4 * nc, 4 * nc), complex)
    for s_in in range(4):
        for c_in in range(nc):
            A = np.zeros((4, nc), complex)
            A[s_in, c_in] = 1.0
            G = Lattice2D(px, py, dx, dy, A)
            gx = lambda a, b: G.dcx(G.z, a, b)   # noqa: E731
            gy = lambda a, b: G.dcy(G.z, a, b)   # noqa: E731

            def flux1(a, b):
                return K11 @ gx(a, b) + K12 @ gy(a, b)

            def flux2(a, b):
                return K21 @ gx(a, b) + K22 @ gy(a, b)

            for s_out, (a, b) in reps.items():
                if s_out == 0:
                    # cell average: Simpson edge averages of the viscous fluxes (Eq. (12))
                    f_e = (flux1(a + 1, b - 1) + 4 * flux1(a + 1, b) + flux1(a + 1, b + 1)) / 6
                    f_w = (flux1(a - 1, b - 1) + 4 * flux1(a - 1, b) + flux1(a - 1, b + 1)) / 6
                    f_n = (flux2(a - 1, b + 1) + 4 * flux2(a, b + 1) + flux2(a + 1, b + 1)) / 6
                    f_s = (flux2(a - 1, b - 1) + 4 * flux2(a, b - 1) + flux2(a + 1, b - 1)) / 6
                    r = (f_e - f_w) / dx + (f_n - f_s) / dy
                else:
                    # point value: compact D^2 plus the mixed terms of Eq. (12)
                    r = G.d2x(K11, a, b) + G.d2y(K22, a, b)
                    r = r + G.dcx(lambda a_, b_: K12 @ gy(a_, b_), a, b)
                    r = r + G.dcy(lambda a_, b_: K21 @ gx(a_, b_), a, b)
                r = r / G.phase(a, b)
                Mop[s_out * nc:(s_out + 1) * nc, s_in * nc + c_in] = r
    return Mop


def operator_1d(nu, p, dx=1.0):
    """1D scalar diffusion z_t = nu z_xx on the AF DoFs (cell average, point),
    Bloch phase p per cell: centres by Simpson (Sec. 2.1), points by Eq. (9)
    with the B matrix, averages by the difference of nu D_c z at the faces."""
    def val(A, a):
        ph = np.exp(0.5j * p * a)
        if a % 2 == 0:
            return A[1] * ph
        return (6 * A[0] * ph - val(A, a - 1) - val(A, a + 1)) / 4

    def dc(A, a):
        return (val(A, a - 2) - 8 * val(A, a - 1) + 8 * val(A, a + 1) - val(A, a + 2)) / (6 * dx)

    Mop = np.zeros((2, 2), complex)
    for s in range(2):
        A = np.zeros(2, complex)
        A[s] = 1.0
        cell = nu * (dc(A, 2) - dc(A, 0)) / dx / np.exp(0.5j * p * 1)
        pt = 4 / dx ** 2 * sum(B10[m + 2, n + 2] * nu * val(A, 2 + n) for m in range(-2, 3)
                               for n in range(-2, 3)) / np.exp(0.5j * p * 2)
        Mop[0, s], Mop[1, s] = cell, pt
    return Mop


def momentum_K(mu=1.0):
    K11 = mu * np.array([[4 / 3, 0.0], [0.0, 1.0]])
    K22 = mu * np.array([[1.0, 0.0], [0.0, 4 / 3]])
    K12 = mu * np.array([[0.0, -2 / 3], [1.0, 0.0]])
    K21 = mu * np.array([[0.0, 1.0], [-2 / 3, 0.0]])
    return K11, K12, K21, K22


def heat_K(nu=1.0):
    one = np.array([[nu]])
    zero = np.zeros((1, 1))
    return one, zero, zero, one


def spectrum_2d(K, nphase=33):
    ph = np.linspace(-np.pi, np.pi, nphase)
    return np.concatenate([np.linalg.eigvals(operator_2d(K, px, py)) for px in ph for py in ph])


def spectrum_1d(nphase=257):
    return np.concatenate([np.linalg.eigvals(operator_1d(1.0, p)) for p in np.linspace(-np.pi, np.pi, nphase)])


def stable_limit(lams, scale):
    """Largest C with |R(C lam / scale)| <= 1 for all eigenvalues lam (dx = 1):
    dt = C dx^2 / scale."""
    def ok(C):
        return np.all(np.abs(rk_amplification(C * lams / scale)) <= 1 + 1e-12)
    lo, hi = 0.0, 2.0
    assert ok(1e-6) and not ok(hi)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if ok(mid) else (lo, mid)
    return lo


@pytest.fixture(scope="module")
def spectra():
    return {"heat": spectrum_2d(heat_K()), "mom": spectrum_2d(momentum_K())}


def test_operators_are_consistent_and_dissipative(spectra):
    """Low modes: the symbols approach the continuous ones (-nu |k|^2 for heat;
    -mu |k|^2 and -(4/3) mu |k|^2 for momentum), and no eigenvalue has a
    positive real part (the semi-discrete operators are stable)."""
    k = 1e-2
    ev = np.linalg.eigvals(operator_2d(heat_K(), k, 0.0))
    assert np.min(np.abs(ev + k * k)) < 1e-6 * k * k + 1e-12
    ev = np.linalg.eigvals(operator_2d(momentum_K(), k, 0.0))
    for target in (-k * k, -4 / 3 * k * k):
        assert np.min(np.abs(ev - target)) < 1e-6 * k * k + 1e-12
    ev = np.linalg.eigvals(operator_1d(1.0, k))
    assert np.min(np.abs(ev + k * k)) < 1e-6 * k * k
    for lam in spectra.values():
        assert lam.real.max() < 1e-10


def test_viscous_cfl_limit_1d_is_the_printed_value():
    C = stable_limit(spectrum_1d(), 1.0)
    assert abs(C / 0.33 - 1) < 0.02, C


def test_viscous_cfl_limit_2d_reading(spectra):
    """dt = C^v dx^2 / rho~ with rho~ = max(4 mu / 3, gamma mu / Pr) (rho = 1).
    Temperature: rho~ >= gamma mu / Pr, worst when equal (scale 1 on the unit
    operator). Momentum: rho~ >= 4 mu / 3, worst when equal. The stable C^v of
    the scheme is the smaller limit: below the printed 0.33/2, and the default
    of both codes (0.13) lies within 1 % under it."""
    import oracle as orc
    c_heat = stable_limit(spectra["heat"], 1.0)
    c_mom = stable_limit(spectra["mom"], 4 / 3)
    c = min(c_heat, c_mom)
    print("2D viscous CFL limits: heat %.4f, momentum %.4f (printed 0.33/2 = 0.165)" % (c_heat, c_mom))
    assert abs(c_heat - 0.1307) < 5e-4 and abs(c_mom - 0.1493) < 5e-4
    assert c < 0.33 / 2
    default = orc.problem(2, 8, 8).cfl_v
    assert 0.99 * c <= default <= c
