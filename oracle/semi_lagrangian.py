"""Semi-Lagrangian discretisation of periodic linear advection (oracle, FP64, numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows Sec. 2.1 of the paper (eq. (ad), (LagForm), (depart_ODE),
(depart_decompose)) for 1D and Sec. 4.1 (eq. (ad_2D), (SL2D_char1-2)) for 2D.

Representation of a departure point.  The paper writes the departure point of
the characteristic arriving at x_i as xi_i = x_E - h eps with x_E the east
neighbour and eps in [0, 1).  The oracle stores the signed, unwrapped
displacement in grid units, s_i = (x_i - xi_i) / h.  Then x_E = x_i - h floor(s_i),
i.e. E = i - floor(s_i), and eps = s_i - floor(s_i).  This is the same
decomposition written without forming the absolute coordinate, which keeps
full precision in eps for large i.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

# ---------------------------------------------------------------------------
# Grid (Sec. 2.1: n_x equidistant nodes, x_{i+1} = x_i + h; t_{n+1} = t_n + dt)
# ---------------------------------------------------------------------------


@dataclasses.dataclass(frozen=True)
class Grid:
    """Periodic uniform grid on [xmin, xmax); nodes x_i = xmin + i h (left aligned).

    The paper does not say where the nodes sit inside the periodic cell; this
    reading places node 0 at xmin.  dt = cfl * h (the paper uses dt = 0.85 h).
    """

    nx: int
    nt: int
    cfl: float = 0.85
    xmin: float = -1.0
    xmax: float = 1.0
    dim: int = 1

    @property
    def length(self) -> float:
        return self.xmax - self.xmin

    @property
    def h(self) -> float:
        return self.length / self.nx

    @property
    def dt(self) -> float:
        return self.cfl * self.h

    @property
    def x(self) -> np.ndarray:
        return self.xmin + self.h * np.arange(self.nx, dtype=np.float64)

    @property
    def npts(self) -> int:
        return self.nx**self.dim


# ---------------------------------------------------------------------------
# Wave speeds (eq. (alpha1), (alpha2), (alpha4), (alpha-const_2D), (alpha-var_2D)
# and the variable-speed families of the synthetic workloads)
# ---------------------------------------------------------------------------

TWO_PI = 2.0 * math.pi


@dataclasses.dataclass(frozen=True)
class WaveSpeed:
    """An analytic wave speed alpha(x, t) (1D) or (alpha, beta)(x, y, t) (2D).

    kinds (1D): "const" alpha = a;  "cos_t" alpha = cos(2 pi t) (eq. alpha2);
      "cos_t_cos_x" alpha = cos(2 pi t) cos(2 pi x) (eq. alpha4);
      "sin_kx_cos_t" alpha = 1 + a sin(2 pi k x) cos(2 pi t).
    kinds (2D): "const2" (alpha, beta) = (a, a2) (eq. alpha-const_2D with a = a2 = 1);
      "paper2" eq. (alpha-var_2D): (sin^2(pi y) cos(2 pi t / 3.4), -cos^2(pi x) cos(2 pi t / 3.4));
      "sin_cos2" (1 + a sin(2 pi y) cos(2 pi t), 1 + a cos(2 pi x) sin(2 pi t)).
    """

    kind: str
    a: float = 1.0
    k: float = 1.0
    a2: float = 1.0

    @property
    def dim(self) -> int:
        return 2 if self.kind in ("const2", "paper2", "sin_cos2") else 1

    def alpha(self, x: np.ndarray, t: float) -> np.ndarray:
        if self.kind == "const":
            return np.full_like(x, self.a)
        if self.kind == "cos_t":
            return np.full_like(x, math.cos(TWO_PI * t))
        if self.kind == "cos_t_cos_x":
            return math.cos(TWO_PI * t) * np.cos(TWO_PI * x)
        if self.kind == "sin_kx_cos_t":
            return 1.0 + self.a * np.sin(TWO_PI * self.k * x) * math.cos(TWO_PI * t)
        raise ValueError(f"not a 1D wave speed: {self.kind}")

    def velocity(self, x: np.ndarray, y: np.ndarray, t: float) -> tuple[np.ndarray, np.ndarray]:
        if self.kind == "const2":
            return np.full_like(x, self.a), np.full_like(y, self.a2)
        if self.kind == "paper2":
            ct = math.cos(TWO_PI * t / 3.4)
            return np.sin(math.pi * y) ** 2 * ct, -(np.cos(math.pi * x) ** 2) * ct
        if self.kind == "sin_cos2":
            return (
                1.0 + self.a * np.sin(TWO_PI * y) * math.cos(TWO_PI * t),
                1.0 + self.a * np.cos(TWO_PI * x) * math.sin(TWO_PI * t),
            )
        raise ValueError(f"not a 2D wave speed: {self.kind}")


# ---------------------------------------------------------------------------
# Explicit Runge-Kutta tableaux (Sec. 2.1: one backward ERK step of order r).
# The paper takes its tableaux from a thesis that is not available; the reading
# used here is: r = 1 forward Euler; r = 3 Kutta's classical third-order method;
# r = 5 Butcher's six-stage fifth-order method (J. C. Butcher, J. Austral. Math.
# Soc. 4 (1964), the scheme with nodes 0, 1/4, 1/4, 1/2, 3/4, 1).
# ---------------------------------------------------------------------------


def erk_tableau(r: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Return (A, b, c) of the order-r explicit Runge-Kutta method."""
    if r == 1:
        return np.zeros((1, 1)), np.array([1.0]), np.array([0.0])
    if r == 3:
        A = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [-1.0, 2.0, 0.0]])
        return A, np.array([1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0]), np.array([0.0, 0.5, 1.0])
    if r == 5:
        A = np.zeros((6, 6))
        A[1, 0] = 1.0 / 4.0
        A[2, 0] = 1.0 / 8.0
        A[2, 1] = 1.0 / 8.0
        A[3, 1] = -1.0 / 2.0
        A[3, 2] = 1.0
        A[4, 0] = 3.0 / 16.0
        A[4, 3] = 9.0 / 16.0
        A[5, 0] = -3.0 / 7.0
        A[5, 1] = 2.0 / 7.0
        A[5, 2] = 12.0 / 7.0
        A[5, 3] = -12.0 / 7.0
        A[5, 4] = 8.0 / 7.0
        b = np.array([7.0, 0.0, 32.0, 12.0, 32.0, 7.0]) / 90.0
        c = np.array([0.0, 0.25, 0.25, 0.5, 0.75, 1.0])
        return A, b, c
    raise ValueError(f"ERK order {r} not supported (1, 3, 5)")


def departure_offsets_1d(grid: Grid, ws: WaveSpeed, n: int, r: int, x: np.ndarray | None = None) -> np.ndarray:
    """Fine departure offsets s_i = (x_i - xi_i) / h for the step t_n -> t_{n+1}.

    Eq. (depart_ODE): d xi / dt = alpha(xi, t), xi(t_{n+1}) = x_i, integrated
    backwards to t_n with one ERK step of size dt (Sec. 2.1).  Stage k_s =
    alpha(x_i - dt sum_j a_sj k_j, t_{n+1} - c_s dt), and x_i - xi = dt sum_s b_s k_s.
    """
    A, b, c = erk_tableau(r)
    if x is None:
        x = grid.x
    dt = grid.dt
    t1 = (n + 1) * dt
    ks: list[np.ndarray] = []
    for s in range(len(b)):
        xs = x.copy()
        for j in range(s):
            if A[s, j] != 0.0:
                xs = xs - dt * A[s, j] * ks[j]
        ks.append(ws.alpha(xs, t1 - c[s] * dt))
    disp = np.zeros_like(x)
    for s in range(len(b)):
        if b[s] != 0.0:
            disp = disp + b[s] * ks[s]
    return dt * disp / grid.h


def departure_offsets_2d(grid: Grid, ws: WaveSpeed, n: int, r: int) -> tuple[np.ndarray, np.ndarray]:
    """2D fine departure offsets (s_x, s_y) on the nx x nx grid, arrays [j][i] (y slow).

    Eq. (SL2D_char1-2): the characteristic (xi, eta) arriving at (x_i, y_j) at
    t_{n+1}, integrated back to t_n by one ERK step of size dt.
    """
    A, b, c = erk_tableau(r)
    X, Y = np.meshgrid(grid.x, grid.x)  # X[j][i] = x_i, Y[j][i] = y_j
    dt = grid.dt
    t1 = (n + 1) * dt
    kx: list[np.ndarray] = []
    ky: list[np.ndarray] = []
    for s in range(len(b)):
        xs, ys = X.copy(), Y.copy()
        for j in range(s):
            if A[s, j] != 0.0:
                xs = xs - dt * A[s, j] * kx[j]
                ys = ys - dt * A[s, j] * ky[j]
        vx, vy = ws.velocity(xs, ys, t1 - c[s] * dt)
        kx.append(vx)
        ky.append(vy)
    dx = np.zeros_like(X)
    dy = np.zeros_like(Y)
    for s in range(len(b)):
        if b[s] != 0.0:
            dx = dx + b[s] * kx[s]
            dy = dy + b[s] * ky[s]
    return dt * dx / grid.h, dt * dy / grid.h


# ---------------------------------------------------------------------------
# East-neighbour decomposition (eq. (depart_decompose)) and Lagrange weights
# ---------------------------------------------------------------------------


def stencil(p: int) -> np.ndarray:
    """Interpolation node offsets j = -l(p) .. r(p) relative to x_E (odd p: l = (p+1)/2, r = (p-1)/2)."""
    if p % 2 != 1:
        raise ValueError("only odd interpolation degrees are supported (Sec. 3.2, Case 3)")
    ell = (p + 1) // 2
    return np.arange(-ell, ell, dtype=np.int64)


def decompose(s: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Split offsets s into (floor(s), eps) with eps = s - floor(s) in [0, 1).

    The east node of the departure point is E = i - floor(s) (eq. (depart_decompose)).
    A departure point exactly on a node has eps = 0 and that node as E.
    """
    fl = np.floor(s)
    eps = s - fl
    bad = eps >= 1.0
    if np.any(bad):
        fl = np.where(bad, fl + 1.0, fl)
        eps = np.where(bad, eps - 1.0, eps)
    return fl.astype(np.int64), eps


def lagrange_weights(eps: np.ndarray, p: int) -> np.ndarray:
    """Lagrange weights for nodes j in stencil(p) at the point -eps: w_j = prod_{q != j} (-eps - q)/(j - q).

    Returns an array of shape eps.shape + (p + 1,).
    """
    nodes = stencil(p)
    z = -np.asarray(eps, dtype=np.float64)
    w = np.ones(z.shape + (len(nodes),))
    for a, j in enumerate(nodes):
        for q in nodes:
            if q != j:
                w[..., a] *= (z - q) / float(j - q)
    return w


def sl_apply_1d(u: np.ndarray, s: np.ndarray, p: int) -> np.ndarray:
    """One SL step (Phi u)_i = sum_j w_j(eps_i) u_{(E_i + j) mod nx} (Sec. 2.1, operator S_{p,r})."""
    nx = u.shape[-1]
    fl, eps = decompose(s)
    E = np.arange(nx, dtype=np.int64) - fl
    w = lagrange_weights(eps, p)
    idx = np.mod(E[:, None] + stencil(p)[None, :], nx)
    return np.sum(w * u[..., idx], axis=-1)


def sl_matrix_1d(s: np.ndarray, p: int) -> np.ndarray:
    """Dense nx x nx matrix of the SL step with offsets s (for small nx only)."""
    nx = s.shape[0]
    fl, eps = decompose(s)
    E = np.arange(nx, dtype=np.int64) - fl
    w = lagrange_weights(eps, p)
    M = np.zeros((nx, nx))
    for i in range(nx):
        for a, j in enumerate(stencil(p)):
            M[i, (E[i] + j) % nx] += w[i, a]
    return M


def sl_apply_2d(u: np.ndarray, sx: np.ndarray, sy: np.ndarray, p: int) -> np.ndarray:
    """2D SL step by tensor-product interpolation (Sec. 4.1): along x on each of the p+1 rows, then along y.

    u, sx, sy are [j][i] arrays (y slow).  The north-east node of the departure
    point is (E, N) = (i - floor(sx), j - floor(sy)) with (eps, nu) the fractional parts.
    """
    ny, nx = u.shape
    fx, eps = decompose(sx)
    fy, nu = decompose(sy)
    I = np.arange(nx, dtype=np.int64)[None, :]
    J = np.arange(ny, dtype=np.int64)[:, None]
    E = I - fx
    N = J - fy
    wx = lagrange_weights(eps, p)
    wy = lagrange_weights(nu, p)
    st = stencil(p)
    out = np.zeros_like(u)
    for b_, jb in enumerate(st):
        rows = np.mod(N + jb, ny)
        row_val = np.zeros_like(u)
        for a_, ja in enumerate(st):
            cols = np.mod(E + ja, nx)
            row_val += wx[..., a_] * u[rows, cols]
        out += wy[..., b_] * row_val
    return out


def sl_matrix_2d(sx: np.ndarray, sy: np.ndarray, p: int) -> np.ndarray:
    """Dense N x N matrix (N = nx^2, row-major index j*nx + i) of the 2D SL step (small nx only)."""
    ny, nx = sx.shape
    fx, eps = decompose(sx)
    fy, nu = decompose(sy)
    wx = lagrange_weights(eps, p)
    wy = lagrange_weights(nu, p)
    st = stencil(p)
    M = np.zeros((nx * ny, nx * ny))
    for j in range(ny):
        for i in range(nx):
            E = i - fx[j, i]
            N = j - fy[j, i]
            for b_, jb in enumerate(st):
                for a_, ja in enumerate(st):
                    M[j * nx + i, ((N + jb) % ny) * nx + (E + ja) % nx] += wy[j, i, b_] * wx[j, i, a_]
    return M
