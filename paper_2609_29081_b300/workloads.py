"""Seeded synthetic inputs shaped like the paper's test problems.

This module only builds initial data: it evaluates an initial condition, takes
cell averages by 5-point Gauss-Legendre quadrature per direction and samples the
point values. It holds none of the AF method's arithmetic, and it is the one
module that both the CUDA path (bench, tests) and the CPU oracle tests use.

Packed state layout (component-major, x index fastest), shared with the C-ABI:
  2D: avg[4][n2][n1], xe[4][n2][n1+1], ye[4][n2+1][n1], vx[4][n2+1][n1+1]
  1D: avg[3][n1],     pt[3][n1+1]
Components are conservative: (rho, rho*u, [rho*v,] E).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BC_PERIODIC, BC_WALL, BC_SYMMETRY, BC_TRANSMISSIVE, BC_EXACT, BC_MOVING = 0, 1, 2, 3, 4, 5


@dataclass
class Workload:
    name: str
    dim: int
    n: tuple
    lo: tuple
    hi: tuple
    gamma: float
    mu: float
    Pr: float
    bc: tuple
    t_end: float
    state: np.ndarray = field(repr=False)
    steps: int = 0          # nominal step count of the configuration (0: run to t_end)
    source: int = 0         # manufactured source (0: none, 1: Taylor-Green energy source)
    src_p0: float = 100.0   # p0 of the Taylor-Green source
    ex_M0: float = 3.0      # BC_EXACT: upstream Mach number of the viscous shock
    ex_uinf: float = 0.2    # BC_EXACT: translation velocity of the viscous shock
    wall_speed: tuple = (0.0, 0.0, 0.0, 0.0)  # BC_MOVING sides: tangential wall velocity

    def __post_init__(self):
        periodize(self.state, self.dim, self.n, self.bc)

    @property
    def cells(self) -> int:
        return int(np.prod(self.n[: self.dim]))


def site_shapes(dim, n1, n2=1):
    if dim == 1:
        return [(3, n1), (3, n1 + 1)]
    return [(4, n2, n1), (4, n2, n1 + 1), (4, n2 + 1, n1), (4, n2 + 1, n1 + 1)]


def split_sites(state, dim, n1, n2=1):
    """Views of the packed state, one per DoF site (avg, [xe, ye, vx] or [pt])."""
    out, o = [], 0
    for shp in site_shapes(dim, n1, n2):
        sz = int(np.prod(shp))
        out.append(state[o:o + sz].reshape(shp))
        o += sz
    assert o == state.size
    return out


def state_len(dim, n1, n2=1):
    return sum(int(np.prod(s)) for s in site_shapes(dim, n1, n2))


def periodize(state, dim, n, bc):
    """Make the duplicated last face of every periodic direction an exact copy of
    the first (sampling sin at 0 and at the period differs in the last bits)."""
    sites = split_sites(state, dim, *n)
    if dim == 1:
        if bc[0] == BC_PERIODIC:
            sites[1][:, -1] = sites[1][:, 0]
        return state
    if bc[0] == BC_PERIODIC:
        for k in (1, 3):
            sites[k][:, :, -1] = sites[k][:, :, 0]
    if bc[2] == BC_PERIODIC:
        for k in (2, 3):
            sites[k][:, -1, :] = sites[k][:, 0, :]
    return state


def _to_cons(gamma, rho, vel, p):
    m = [rho * v for v in vel]
    E = p / (gamma - 1.0) + 0.5 * rho * sum(v * v for v in vel)
    return [rho, *m, E]


def project(dim, n, lo, hi, gamma, prim_fn):
    """Packed state of a primitive initial condition prim_fn(x[,y]) -> (rho, vel list, p)."""
    gx, gw = np.polynomial.legendre.leggauss(5)
    gw = gw / 2.0
    if dim == 1:
        n1 = n[0]
        dx = (hi[0] - lo[0]) / n1
        xc = lo[0] + (np.arange(n1) + 0.5) * dx
        avg = np.zeros((3, n1))
        for q in range(5):
            rho, vel, p = prim_fn(xc + 0.5 * dx * gx[q])
            for c, v in enumerate(_to_cons(gamma, rho, vel, p)):
                avg[c] += gw[q] * v
        xf = lo[0] + np.arange(n1 + 1) * dx
        rho, vel, p = prim_fn(xf)
        pt = np.array(_to_cons(gamma, rho, vel, p))
        return np.concatenate([avg.ravel(), pt.ravel()])
    n1, n2 = n
    dx = (hi[0] - lo[0]) / n1
    dy = (hi[1] - lo[1]) / n2
    xc = lo[0] + (np.arange(n1) + 0.5) * dx
    yc = lo[1] + (np.arange(n2) + 0.5) * dy
    xf = lo[0] + np.arange(n1 + 1) * dx
    yf = lo[1] + np.arange(n2 + 1) * dy
    avg = np.zeros((4, n2, n1))
    for qy in range(5):
        Y = (yc + 0.5 * dy * gx[qy])[:, None]
        for qx in range(5):
            X = (xc + 0.5 * dx * gx[qx])[None, :]
            rho, vel, p = prim_fn(np.broadcast_to(X, (n2, n1)), np.broadcast_to(Y, (n2, n1)))
            for c, v in enumerate(_to_cons(gamma, rho, vel, p)):
                avg[c] += gw[qx] * gw[qy] * v

    def sample(x, y):
        X, Y = np.meshgrid(x, y)
        rho, vel, p = prim_fn(X, Y)
        return np.array([np.broadcast_to(v, X.shape) for v in _to_cons(gamma, rho, vel, p)])

    return np.concatenate([avg.ravel(), sample(xf, yc).ravel(), sample(xc, yf).ravel(),
                           sample(xf, yf).ravel()])


# ---------------------------------------------------------------------------
# Configurations
# ---------------------------------------------------------------------------

def smooth_1d(n=128, mu=0.01, Pr=0.72, gamma=1.4, t_end=0.5):
    """1D periodic smooth wave on [0, 2 pi): rho = 1 + 0.2 sin x, u = 1, p = 1."""
    lo, hi = (0.0,), (2 * np.pi,)

    def f(x):
        return 1.0 + 0.2 * np.sin(x), [np.ones_like(x)], np.ones_like(x)

    s = project(1, (n,), lo, hi, gamma, f)
    return Workload("smooth_1d_periodic_N%d" % n, 1, (n,), lo, hi, gamma, mu, Pr,
                    (BC_PERIODIC,) * 4, t_end, s)


def shock_tube_1d(n=4096, mu=1e-3, Pr=0.72, gamma=1.4, t_end=0.2):
    """1D viscous Sod-type tube on [0,1], transmissive ends."""
    lo, hi = (0.0,), (1.0,)

    def f(x):
        left = x < 0.5
        return (np.where(left, 1.0, 0.125), [np.zeros_like(x)], np.where(left, 1.0, 0.1))

    s = project(1, (n,), lo, hi, gamma, f)
    return Workload("shock_tube_1d_N%d" % n, 1, (n,), lo, hi, gamma, mu, Pr,
                    (BC_TRANSMISSIVE,) * 4, t_end, s)


def becker_prim(x, t, M0=3.0, mu=1e-2, Pr=0.75, gamma=1.4, u_inf=0.2):
    """Exact moving viscous shock (Sec. 4, Becker's solution) with rho_L = w_L =
    m0 = 1: (rho, u, p) at positions x (array) and time t. The relative velocity
    w(xi), xi = x - u_inf t, is found by bisection of the printed implicit law."""
    g = gamma
    wL, m0 = 1.0, 1.0
    wR = wL * ((g - 1.0) + 2.0 / M0 ** 2) / (g + 1.0)
    w0 = np.sqrt(wL * wR)
    k = 2.0 * mu * g / ((g + 1.0) * m0 * Pr)

    def xi_of(w):
        return k * (wL / (wL - wR) * np.log((wL - w) / (wL - w0)) - wR / (wL - wR) * np.log((w - wR) / (w0 - wR)))

    xi = np.asarray(x, dtype=float) - u_inf * t
    lo, hi = np.full_like(xi, wR), np.full_like(xi, wL)
    with np.errstate(divide="ignore"):
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            up = xi_of(mid) > xi
            lo, hi = np.where(up, mid, lo), np.where(up, hi, mid)
    w = 0.5 * (lo + hi)
    e = ((g + 1.0) / (g - 1.0) * w0 * w0 - w * w) / (2.0 * g)
    rho = m0 / w
    return rho, u_inf + w, (g - 1.0) * rho * e


def becker_1d(n=80, t=0.0, M0=3.0, mu=1e-2, Pr=0.75, gamma=1.4, u_inf=0.2, t_end=0.2, lo=-1.0, hi=1.5):
    """1D viscous shock wave (Sec. 4) on [lo, hi] (default [-1, 1.5]): the exact
    Becker profile at time t (shock at x = u_inf t), both ends prescribed from the
    exact solution (BC_EXACT). M0 = 3, mu = 1e-2 is the paper's unlimited accuracy
    case; M0 = 20, mu = 1e-3 the limited one."""
    lo, hi = (float(lo),), (float(hi),)

    def f(x):
        rho, u, p = becker_prim(x, t, M0, mu, Pr, gamma, u_inf)
        return rho, [u], p

    s = project(1, (n,), lo, hi, gamma, f)
    return Workload("becker_1d_N%d_M%g" % (n, M0), 1, (n,), lo, hi, gamma, mu, Pr, (BC_EXACT,) * 4, t_end, s,
                    ex_M0=M0, ex_uinf=u_inf)


def leblanc_1d(n=800, mu=0.0, Pr=0.75, gamma=5.0 / 3.0, t_end=0.4):
    """1D LeBlanc problem (Sec. 4 example) on [-0.5, 0.5], outflow ends:
    (rho, u, p) = (1, 0, 6.666667e-2) for x < -0.2, (1e-2, 0, 6.666667e-11)
    otherwise; gamma = 5/3 (p = (gamma-1) rho e with e = 0.1 and 1e-7)."""
    lo, hi = (-0.5,), (0.5,)

    def f(x):
        left = x < -0.2
        return (np.where(left, 1.0, 1e-2), [np.zeros_like(x)], np.where(left, 6.666667e-2, 6.666667e-11))

    s = project(1, (n,), lo, hi, gamma, f)
    return Workload("leblanc_1d_N%d_mu%g" % (n, mu), 1, (n,), lo, hi, gamma, mu, Pr,
                    (BC_TRANSMISSIVE,) * 4, t_end, s)


def stokes_first_problem(n=100, mu=1e-2, gamma=1.4, t_end=1.0, ny=4):
    """First problem of Stokes (Sec. 4 example): a tangential velocity jump that
    diffuses, on [-0.5, 0.5] with outflow ends; (rho, u, v, p) = (1, 0, -0.1,
    1/gamma) for x < 0, (1, 0, 0.1, 1/gamma) otherwise; kappa = 0. The solution
    depends on x only, so it runs as a 2D strip of n x ny cells, periodic in y.
    kappa = 0 is obtained through Pr = 1e30 (kappa = gamma mu / ((gamma-1) Pr),
    1e-30 times the viscosity; the heat-conduction term of the CFL bound vanishes
    likewise). In the incompressible limit v = 0.1 erf(x / (2 sqrt(mu t)))."""
    h = 1.0 / n
    lo, hi = (-0.5, 0.0), (0.5, ny * h)

    def f(x, y):
        return np.ones_like(x), [np.zeros_like(x), np.where(x < 0.0, -0.1, 0.1)], np.full_like(x, 1.0 / gamma)

    st = project(2, (n, ny), lo, hi, gamma, f)
    return Workload("stokes_first_%dx%d_mu%g" % (n, ny, mu), 2, (n, ny), lo, hi, gamma, mu, 1e30,
                    (BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_PERIODIC, BC_PERIODIC), t_end, st)


def fourier_modes(seed, nmodes=8, amp=0.05, kmax=4):
    """Seeded velocity perturbation: nmodes wavevectors from {1..kmax}^2 without
    replacement, random phases, per-mode amplitude amp / nmodes."""
    rng = np.random.default_rng(seed)
    ks = [(a, b) for a in range(1, kmax + 1) for b in range(1, kmax + 1)]
    pick = rng.choice(len(ks), size=nmodes, replace=False)
    ph = rng.uniform(0.0, 2 * np.pi, size=(nmodes, 2))
    return [(ks[p][0], ks[p][1], ph[q, 0], ph[q, 1], amp / nmodes) for q, p in enumerate(pick)]


def smooth_2d(n=1024, mu=0.01, Pr=0.72, gamma=1.4, seed=3, steps=200, mean=(1.0, 0.5), amp=0.05,
              t_end=0.0):
    """2D periodic smooth flow on [0, 2 pi)^2: rho = 1 + 0.2 sin(x + y),
    (u, v) = mean + 8-mode Fourier perturbation, p = 1."""
    lo, hi = (0.0, 0.0), (2 * np.pi, 2 * np.pi)
    modes = fourier_modes(seed, amp=amp)

    def f(x, y):
        du = np.zeros_like(x)
        dv = np.zeros_like(x)
        for k1, k2, p1, p2, a in modes:
            du = du + a * np.sin(k1 * x + k2 * y + p1)
            dv = dv + a * np.cos(k1 * x + k2 * y + p2)
        return 1.0 + 0.2 * np.sin(x + y), [mean[0] + du, mean[1] + dv], np.ones_like(x)

    nn = (n, n) if np.isscalar(n) else tuple(n)
    s = project(2, nn, lo, hi, gamma, f)
    return Workload("smooth_2d_periodic_%dx%d" % nn, 2, nn, lo, hi, gamma, mu, Pr,
                    (BC_PERIODIC,) * 4, t_end, s, steps)


SRC_TAYLOR_GREEN = 1


def taylor_green_2d(n=80, t=0.0, mu=1e-5, Pr=1.0, p0=100.0, gamma=1.4, t_end=0.2):
    """2D manufactured Taylor-Green vortex on [0, 2 pi]^2 (Sec. 4), the exact
    solution at time t: rho = 1, (u, v) = a (sin x cos y, -cos x sin y),
    p = p0/(gamma-1) + a^2 (cos 2x + cos 2y)/4 with a = exp(-2 mu t). The energy
    equation carries the manufactured source (Workload.source = 1)."""
    lo, hi = (0.0, 0.0), (2 * np.pi, 2 * np.pi)
    a = np.exp(-2.0 * mu * t)

    def f(x, y):
        u = a * np.sin(x) * np.cos(y)
        v = -a * np.cos(x) * np.sin(y)
        p = p0 / (gamma - 1.0) + a * a * (np.cos(2 * x) + np.cos(2 * y)) / 4.0
        return np.ones_like(x), [u, v], p

    nn = (n, n) if np.isscalar(n) else tuple(n)
    st = project(2, nn, lo, hi, gamma, f)
    return Workload("taylor_green_2d_%dx%d_t%g" % (nn[0], nn[1], t), 2, nn, lo, hi, gamma, mu, Pr,
                    (BC_PERIODIC,) * 4, t_end, st, 0, SRC_TAYLOR_GREEN, p0)


def couette_2d(n=16, U=0.5, mu=1e-2, Pr=0.72, gamma=1.4, p0=1.0, t_end=0.1):
    """Plane Couette flow on [0,1]^2, periodic in x, a no-slip wall at y = 0 and a
    wall moving with speed U in x at y = 1: rho = 1, u = U y, v = 0, p = p0. The
    momentum equations are steady for this field; the energy grows at the
    viscous-heating rate mu U^2."""
    lo, hi = (0.0, 0.0), (1.0, 1.0)

    def f(x, y):
        return np.ones_like(x), [U * y, np.zeros_like(x)], np.full_like(x, p0)

    nn = (n, n) if np.isscalar(n) else tuple(n)
    st = project(2, nn, lo, hi, gamma, f)
    return Workload("couette_2d_%dx%d" % nn, 2, nn, lo, hi, gamma, mu, Pr,
                    (BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_MOVING), t_end, st, wall_speed=(0.0, 0.0, 0.0, U))


def moving_plate_2d(n=100, U=0.1, mu=1e-2, gamma=1.4, t_end=1.0, nx=4):
    """Impulsively started plate (Rayleigh's problem): fluid at rest over y in
    [0, 1] (rho = 1, p = 1/gamma), the wall at y = 0 set moving with speed U in x
    at t = 0, outflow at y = 1; run as a strip of nx x n cells periodic in x.
    Incompressible limit: u = U erfc(y / (2 sqrt(mu t))). kappa = 0 through
    Pr = 1e30 as in the first problem of Stokes."""
    h = 1.0 / n
    lo, hi = (0.0, 0.0), (nx * h, 1.0)

    def f(x, y):
        return np.ones_like(x), [np.zeros_like(x), np.zeros_like(x)], np.full_like(x, 1.0 / gamma)

    st = project(2, (nx, n), lo, hi, gamma, f)
    return Workload("moving_plate_%dx%d_mu%g" % (nx, n, mu), 2, (nx, n), lo, hi, gamma, mu, 1e30,
                    (BC_PERIODIC, BC_PERIODIC, BC_MOVING, BC_TRANSMISSIVE), t_end, st,
                    wall_speed=(0.0, 0.0, U, 0.0))


def lid_driven_cavity(n=128, Re=100.0, Pr=0.72, gamma=1.4, t_end=40.0):
    """Lid-driven cavity (Sec. 4) on [0,1]^2: rho = 1, u = v = 0, p = 1e4/gamma
    (Mach 0.01 for the unit lid speed), no-slip adiabatic walls, the top one
    moving with velocity (1, 0); mu = 1/Re. The paper gives no Prandtl number
    for this case: 0.72 is taken."""
    lo, hi = (0.0, 0.0), (1.0, 1.0)

    def f(x, y):
        return np.ones_like(x), [np.zeros_like(x), np.zeros_like(x)], np.full_like(x, 1e4 / gamma)

    nn = (n, n) if np.isscalar(n) else tuple(n)
    st = project(2, nn, lo, hi, gamma, f)
    return Workload("lid_cavity_%dx%d_Re%g" % (nn[0], nn[1], Re), 2, nn, lo, hi, gamma, 1.0 / Re, Pr,
                    (BC_WALL, BC_WALL, BC_WALL, BC_MOVING), t_end, st, wall_speed=(0.0, 0.0, 0.0, 1.0))


def double_shear_layer(n=200, mu=2e-4, Pr=0.72, gamma=1.4, t_end=1.8):
    """Double shear layer (Sec. 4) on the periodic unit square: rho = 1,
    p = 1e4/gamma, u = tanh(30 (y - 1/4)) for y <= 1/2 and tanh(30 (3/4 - y))
    above, v = 0.05 sin(2 pi x); mu = 2e-4 (Re 1e4, Mach 0.01). No Prandtl number
    is given for this case: 0.72 is taken."""
    lo, hi = (0.0, 0.0), (1.0, 1.0)

    def f(x, y):
        u = np.where(y <= 0.5, np.tanh(30.0 * (y - 0.25)), np.tanh(30.0 * (0.75 - y)))
        return np.ones_like(x), [u, 0.05 * np.sin(2 * np.pi * x)], np.full_like(x, 1e4 / gamma)

    nn = (n, n) if np.isscalar(n) else tuple(n)
    st = project(2, nn, lo, hi, gamma, f)
    return Workload("double_shear_layer_%dx%d" % nn, 2, nn, lo, hi, gamma, mu, Pr, (BC_PERIODIC,) * 4, t_end, st)


def shock_tube_2d(n=(2000, 1000), mu=1e-3, Pr=0.73, gamma=1.4, t_end=1.0):
    """2D viscous shock tube in a walled box [0,1]x[0,0.5] (Daru-Tenaud setup):
    no-slip adiabatic walls at x=0, x=1, y=0; symmetry at y=0.5."""
    lo, hi = (0.0, 0.0), (1.0, 0.5)

    def f(x, y):
        left = x < 0.5
        rho = np.where(left, 120.0, 1.2)
        return rho, [np.zeros_like(x), np.zeros_like(x)], rho / gamma

    s = project(2, tuple(n), lo, hi, gamma, f)
    return Workload("shock_tube_2d_%dx%d" % tuple(n), 2, tuple(n), lo, hi, gamma, mu, Pr,
                    (BC_WALL, BC_WALL, BC_WALL, BC_SYMMETRY), t_end, s)


def entropy_wave_2d(n=32, gamma=1.4, mean=(1.0, 0.5), t=0.0, amp=0.2):
    """Exact Euler solution (mu = 0): rho = 1 + amp sin(x + y - (u+v) t), constant u, v, p."""
    lo, hi = (0.0, 0.0), (2 * np.pi, 2 * np.pi)

    def f(x, y):
        ph = x + y - (mean[0] + mean[1]) * t
        return 1.0 + amp * np.sin(ph), [np.full_like(x, mean[0]), np.full_like(x, mean[1])], np.ones_like(x)

    nn = (n, n) if np.isscalar(n) else tuple(n)
    s = project(2, nn, lo, hi, gamma, f)
    return Workload("entropy_wave_2d_%dx%d" % nn, 2, nn, lo, hi, gamma, 0.0, 0.72,
                    (BC_PERIODIC,) * 4, 0.0, s)


def entropy_wave_1d(n=32, gamma=1.4, u=1.0, t=0.0, amp=0.2):
    lo, hi = (0.0,), (2 * np.pi,)

    def f(x):
        return 1.0 + amp * np.sin(x - u * t), [np.full_like(x, u)], np.ones_like(x)

    s = project(1, (n,), lo, hi, gamma, f)
    return Workload("entropy_wave_1d_N%d" % n, 1, (n,), lo, hi, gamma, 0.0, 0.72,
                    (BC_PERIODIC,) * 4, 0.0, s)


def random_smooth_2d(n=(24, 20), seed=0, mu=0.01, Pr=0.72, gamma=1.4, bc=(0, 0, 0, 0), amp=0.1,
                     lo=(0.0, 0.0), hi=(2 * np.pi, 2 * np.pi)):
    """Seeded smooth periodic-in-shape fields for parity cases (uneven sizes)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, size=(4, 3, 2))
    L = (hi[0] - lo[0], hi[1] - lo[1])

    def f(x, y):
        X = 2 * np.pi * (x - lo[0]) / L[0]
        Y = 2 * np.pi * (y - lo[1]) / L[1]
        g = []
        for q in range(4):
            v = 0.0
            for k in range(3):
                v = v + c[q, k, 0] * np.sin((k + 1) * X + c[q, k, 1]) * np.cos(k * Y + 0.5 * c[q, k, 0])
            g.append(v)
        return 1.0 + amp * g[0], [0.3 + amp * g[1], -0.2 + amp * g[2]], 1.0 + amp * g[3]

    s = project(2, tuple(n), lo, hi, gamma, f)
    return Workload("random_smooth_2d_%dx%d_s%d" % (n[0], n[1], seed), 2, tuple(n), lo, hi, gamma,
                    mu, Pr, tuple(bc), 0.0, s)


def blast_2d(n=(32, 32), seed=0, mu=1e-3, Pr=0.72, gamma=1.4, rho_min=1e-6, p_min=1e-8):
    """Near-vacuum Gaussian blast on a periodic square (stresses both limiters)."""
    rng = np.random.default_rng(seed)
    lo, hi = (0.0, 0.0), (1.0, 1.0)
    cx, cy = rng.uniform(0.3, 0.7, size=2)
    sig = 1.0 / 16.0

    def f(x, y):
        r2 = (x - cx) ** 2 + (y - cy) ** 2
        g = np.exp(-r2 / (2 * sig * sig))
        return rho_min + g, [np.zeros_like(x), np.zeros_like(x)], p_min + g

    s = project(2, tuple(n), lo, hi, gamma, f)
    return Workload("blast_2d_%dx%d_s%d" % (n[0], n[1], seed), 2, tuple(n), lo, hi, gamma, mu, Pr,
                    (BC_PERIODIC,) * 4, 0.0, s)


def _sep_sin(k1, k2, ph, x, y):
    """sin(k1 x + k2 y + ph) on the grid x (columns) by y (rows), as outer products."""
    return np.outer(np.cos(k2 * y + ph), np.sin(k1 * x)) + np.outer(np.sin(k2 * y + ph), np.cos(k1 * x))


def project_separable(n, L, gamma, field_fn, quad=3):
    """Packed state of a field given by field_fn(x1d, y1d) -> (rho, u, v, p) 2D
    arrays on the tensor grid x1d (columns) by y1d (rows). Cell averages by
    quad-point Gauss-Legendre per direction."""
    n1, n2 = n
    dx, dy = L[0] / n1, L[1] / n2
    gx, gw = np.polynomial.legendre.leggauss(quad)
    gw = gw / 2.0
    xc = (np.arange(n1) + 0.5) * dx
    yc = (np.arange(n2) + 0.5) * dy
    xf = np.arange(n1 + 1) * dx
    yf = np.arange(n2 + 1) * dy

    def cons(x, y):
        rho, u, v, p = field_fn(x, y)
        return np.array([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])

    avg = np.zeros((4, n2, n1))
    for qy in range(quad):
        for qx in range(quad):
            avg += gw[qx] * gw[qy] * cons(xc + 0.5 * dx * gx[qx], yc + 0.5 * dy * gx[qy])
    return np.concatenate([avg.ravel(), cons(xf, yc).ravel(), cons(xc, yf).ravel(), cons(xf, yf).ravel()])


def batch_problems(nprob=256, seed=5, sizes=(64, 96, 128, 192, 256, 384, 512), blast_frac=0.25, gamma=1.4,
                   Pr=0.72):
    """Batched workload: nprob independent periodic problems on [0,1]^2 with grid
    sides drawn from `sizes` (uneven, seeded), mu log-uniform in [1e-4, 1e-2],
    background rho = 1, p = 1/gamma (sound speed 1), mean flow of Mach U[0.1, 3] at
    a random angle plus an 8-mode Fourier velocity perturbation (total amplitude
    0.05); a fraction blast_frac are near-vacuum Gaussian blasts instead
    (rho = 1e-6 + g, p = 1e-8 + g, g = exp(-r^2 / (2 sigma^2)), sigma = 1/16)."""
    rng = np.random.default_rng(seed)
    out = []
    nblast = int(round(blast_frac * nprob))
    blast_ids = set(rng.choice(nprob, size=nblast, replace=False).tolist())
    for p in range(nprob):
        n = (int(rng.choice(sizes)), int(rng.choice(sizes)))
        mu = float(10 ** rng.uniform(-4, -2))
        if p in blast_ids:
            cx, cy = rng.uniform(0.3, 0.7, size=2)
            sig = 1.0 / 16.0

            def f(x, y, cx=cx, cy=cy, sig=sig):
                g = np.outer(np.exp(-(y - cy) ** 2 / (2 * sig * sig)), np.exp(-(x - cx) ** 2 / (2 * sig * sig)))
                z = np.zeros_like(g)
                return 1e-6 + g, z, z, 1e-8 + g
            name = "blast"
        else:
            mach = rng.uniform(0.1, 3.0)
            ang = rng.uniform(0, 2 * np.pi)
            U0, V0 = mach * np.cos(ang), mach * np.sin(ang)
            modes = fourier_modes(int(rng.integers(1 << 30)))

            def f(x, y, U0=U0, V0=V0, modes=modes):
                du = np.zeros((len(y), len(x)))
                dv = np.zeros((len(y), len(x)))
                for k1, k2, p1, p2, a in modes:
                    du += a * _sep_sin(2 * np.pi * k1, 2 * np.pi * k2, p1, x, y)
                    dv += a * _sep_sin(2 * np.pi * k1, 2 * np.pi * k2, p2 + np.pi / 2, x, y)
                one = np.ones_like(du)
                return one, U0 + du, V0 + dv, one / gamma
            name = "flow"
        s = project_separable(n, (1.0, 1.0), gamma, f)
        out.append(Workload("batch%03d_%s_%dx%d" % (p, name, n[0], n[1]), 2, n, (0.0, 0.0), (1.0, 1.0), gamma, mu,
                            Pr, (BC_PERIODIC,) * 4, 0.0, s))
    return out
