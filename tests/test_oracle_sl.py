"""Pins for the oracle's SL discretisation against facts the paper and mathematics fix.

No test here re-types an oracle formula: each compares against a closed form,
an independent identity or an observed convergence order.
"""

import math

import numpy as np
import pytest

import workloads as W
from oracle import semi_lagrangian as sl

from closed_forms import exact_flow_cos_t_cos_x

TWO_PI = 2.0 * math.pi


@pytest.mark.parametrize("r", [1, 3, 5])
def test_erk_local_order_on_closed_form_flow(r):
    """One backward ERK step has local error O(dt^{r+1}) (Sec. 2.1), checked on the exact flow of eq. (alpha4)."""
    ws = sl.WaveSpeed("cos_t_cos_x")
    x = np.array([-0.9, -0.6, -0.37, 0.05, 0.11, 0.4, 0.63, 0.91])
    errs = []
    dts = [0.02, 0.01, 0.005]
    for dt in dts:
        nx = 64
        g = sl.Grid(nx, 10, cfl=dt / (2.0 / nx))
        n = 3
        s = sl.departure_offsets_1d(g, ws, n, r, x=x)
        xi = x - g.h * s
        exact = exact_flow_cos_t_cos_x(x, (n + 1) * dt, n * dt)
        errs.append(np.max(np.abs(xi - exact)))
    orders = [math.log(errs[i] / errs[i + 1], 2) for i in range(2)]
    assert orders[-1] > r + 1 - 0.35 and min(orders) > r, (errs, orders)


def test_departure_constant_alpha_is_exact():
    """For constant alpha every ERK is exact: s = alpha dt / h = alpha * cfl (Sec. 3.2)."""
    for r in (1, 3, 5):
        g = sl.Grid(32, 8, cfl=0.85)
        s = sl.departure_offsets_1d(g, sl.WaveSpeed("const", a=1.3), 2, r)
        assert np.allclose(s, 1.3 * 0.85, rtol=0, atol=1e-13)


@pytest.mark.parametrize("r", [1, 3, 5])
def test_departure_cos_t_closed_form(r):
    """alpha = cos(2 pi t): xi = x - [sin 2 pi t_{n+1} - sin 2 pi t_n] / (2 pi), local error O(dt^{r+1})."""
    ws = sl.WaveSpeed("cos_t")
    errs = []
    for nx in (64, 128, 256):
        g = sl.Grid(nx, 8)
        n = 5
        s = sl.departure_offsets_1d(g, ws, n, r)
        exact = (math.sin(TWO_PI * (n + 1) * g.dt) - math.sin(TWO_PI * n * g.dt)) / TWO_PI / g.h
        assert np.ptp(s) < 1e-14  # independent of x
        errs.append(abs(s[0] - exact) * g.h)
    orders = [math.log(errs[i] / errs[i + 1], 2) for i in range(2)]
    assert min(orders) > r + 1 - 0.35, (errs, orders)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_weights_reproduce_polynomials(p):
    """Interpolation of degree p is exact for polynomials of degree <= p (Sec. 2.1, proof of Lemma 3.1)."""
    eps = np.linspace(0.0, 0.999, 37)
    w = sl.lagrange_weights(eps, p)
    nodes = sl.stencil(p).astype(np.float64)
    for k in range(p + 1):
        assert np.allclose(w @ nodes**k, (-eps) ** k, rtol=0, atol=1e-12)
    assert np.allclose(w.sum(axis=1), 1.0, atol=1e-14)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_stencil_is_the_p_plus_1_nearest_nodes(p):
    """Odd p: nodes x_E + j h, j = -(p+1)/2 .. (p-1)/2 (Sec. 2.1)."""
    st = sl.stencil(p)
    assert len(st) == p + 1 and st[0] == -(p + 1) // 2 and st[-1] == (p - 1) // 2
    # for eps in (0,1) the departure point -eps lies in the middle cell (-1, 0)
    mid = len(st) // 2
    assert st[mid - 1] == -1 and st[mid] == 0


def test_decompose_east_neighbour():
    """xi = x_E - h eps with eps in [0,1); a point on a node has eps = 0 (eq. (depart_decompose))."""
    s = np.array([0.0, 0.85, 1.0, 2.5, -0.25, -1.0, 3.999999])
    fl, eps = sl.decompose(s)
    assert np.all((eps >= 0.0) & (eps < 1.0))
    assert np.allclose(fl + eps, s, atol=0)
    assert list(fl) == [0, 0, 1, 2, -1, -1, 3]


@pytest.mark.parametrize("cfl,shift", [(1.0, 1), (2.0, 2), (3.0, 3)])
def test_integer_courant_is_an_exact_shift(cfl, shift):
    """Constant alpha with integer Courant number: departure points are nodes and Phi is a cyclic shift."""
    nx = 40
    g = sl.Grid(nx, 4, cfl=cfl)
    u = np.random.default_rng(1).standard_normal(nx)
    for p in (1, 3, 5):
        s = sl.departure_offsets_1d(g, sl.WaveSpeed("const"), 0, p)
        # exact in exact arithmetic; the ERK weights sum to 1 only up to one rounding
        assert np.allclose(sl.sl_apply_1d(u, s, p), np.roll(u, shift), rtol=0, atol=1e-13)


def test_matrix_matches_apply():
    g = sl.Grid(24, 4)
    ws = sl.WaveSpeed("sin_kx_cos_t", a=0.5, k=2)
    u = np.random.default_rng(2).standard_normal(24)
    for p in (1, 3, 5):
        s = sl.departure_offsets_1d(g, ws, 1, p)
        assert np.allclose(sl.sl_matrix_1d(s, p) @ u, sl.sl_apply_1d(u, s, p), atol=1e-14)


@pytest.mark.parametrize("p", [1, 3])
def test_sequential_global_order(p):
    """Global error O(dt^r + h^{p+1}/dt) with dt = 0.85 h, r = p gives order p (Sec. 2.1), on the exact flow of eq. (alpha4)."""
    from oracle import mgrit as mg

    ws = sl.WaveSpeed("cos_t_cos_x")
    errs = []
    for nx in (64, 128, 256):
        nt = nx // 2  # T = nt * 0.85 * 2 / nx = 0.85
        g = sl.Grid(nx, nt)
        H = mg.Hierarchy(g, ws, p, [])
        U = mg.sequential_solve(H, W.u0_sin4(nx))
        T = nt * g.dt
        foot = exact_flow_cos_t_cos_x(g.x, T, 0.0)
        exact = np.sin(math.pi * foot) ** 4
        errs.append(np.sqrt(g.h) * np.linalg.norm(U[-1] - exact))
    orders = [math.log(errs[i] / errs[i + 1], 2) for i in range(2)]
    assert orders[-1] > p - 0.3, (errs, orders)


@pytest.mark.parametrize("kind", ["sin_cos2", "paper2"])
@pytest.mark.parametrize("r", [1, 3, 5])
def test_departure_2d_local_order_against_an_ode_solver(r, kind):
    """Eq. (SL2D_char1-2) by one backward ERK step: against scipy's adaptive RK integration of the
    characteristic ODE (velocities written out here: the 2D workload's field and eq. (alpha-var_2D)),
    local error O(dt^{r+1}).  A swapped component, a stage time slip or a wrong axis order of the
    [j][i] arrays changes the order."""
    integrate = pytest.importorskip("scipy.integrate")
    a = 0.5

    def velocity(x, y, t):
        if kind == "sin_cos2":
            return 1.0 + a * np.sin(TWO_PI * y) * math.cos(TWO_PI * t), 1.0 + a * np.cos(TWO_PI * x) * math.sin(TWO_PI * t)
        ct = math.cos(TWO_PI * t / 3.4)
        return np.sin(math.pi * y) ** 2 * ct, -(np.cos(math.pi * x) ** 2) * ct

    def rhs(t, z):
        return np.concatenate(velocity(z[: len(z) // 2], z[len(z) // 2:], t))

    ws = sl.WaveSpeed(kind, a=a, a2=a)
    pts = [(1, 2), (5, 3), (7, 12), (10, 6), (14, 9)]  # (i, j) on the 16-point grid
    errs = []
    for nx in (16, 32, 64):
        g = sl.Grid(nx, 4, dim=2)
        n = 2
        sx, sy = sl.departure_offsets_2d(g, ws, n, r)
        q = nx // 16
        x0 = np.array([g.x[i * q] for i, _ in pts])
        y0 = np.array([g.x[j * q] for _, j in pts])
        sol = integrate.solve_ivp(rhs, ((n + 1) * g.dt, n * g.dt), np.concatenate([x0, y0]), method="DOP853",
                                  rtol=1e-13, atol=1e-14)
        xe, ye = sol.y[: len(pts), -1], sol.y[len(pts):, -1]
        xi = np.array([x0[k] - g.h * sx[j * q, i * q] for k, (i, j) in enumerate(pts)])
        eta = np.array([y0[k] - g.h * sy[j * q, i * q] for k, (i, j) in enumerate(pts)])
        errs.append(max(np.max(np.abs(xi - xe)), np.max(np.abs(eta - ye))))
    orders = [math.log(errs[i] / errs[i + 1], 2) for i in range(2)]
    assert orders[-1] > r + 1 - 0.5 and min(orders) > r - 0.3, (errs, orders)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_sl2d_reproduces_polynomials(p):
    """Tensor-product interpolation is exact on x^a y^b, a, b <= p (Sec. 4.1)."""
    nx = 32
    rng = np.random.default_rng(3)
    sx = rng.uniform(-1.5, 1.5, (nx, nx))
    sy = rng.uniform(-1.5, 1.5, (nx, nx))
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(nx, dtype=float))
    inner = (slice(6, nx - 6), slice(6, nx - 6))  # stencils do not wrap here
    for a in range(p + 1):
        for b in range(p + 1):
            u = (X / nx) ** a * (Y / nx) ** b
            v = sl.sl_apply_2d(u, sx, sy, p)
            exact = ((X - sx) / nx) ** a * ((Y - sy) / nx) ** b
            assert np.allclose(v[inner], exact[inner], atol=1e-12)


def test_sl2d_integer_courant_shift_and_matrix():
    nx = 12
    g = sl.Grid(nx, 2, cfl=1.0, dim=2)
    ws = sl.WaveSpeed("const2", a=1.0, a2=2.0)
    sx, sy = sl.departure_offsets_2d(g, ws, 0, 3)
    u = np.random.default_rng(4).standard_normal((nx, nx))
    v = sl.sl_apply_2d(u, sx, sy, 3)
    assert np.allclose(v, np.roll(np.roll(u, 1, axis=1), 2, axis=0), rtol=0, atol=1e-13)
    sx, sy = sl.departure_offsets_2d(g, sl.WaveSpeed("sin_cos2", a=0.5), 1, 3)
    assert np.allclose(sl.sl_matrix_2d(sx, sy, 3) @ u.ravel(), sl.sl_apply_2d(u, sx, sy, 3).ravel(), atol=1e-13)
