"""Discrete adjoint of the SL one-step system (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no adjoint.  This module states the plain definitions used to check the library's
adjoint solve:
  J(u0, a) = 1/2 ||u_nt - u_target||^2 with u_{n+1} = Phi_n(a) u_n (eq. (one-step), g = 0);
  lambda_nt = u_nt - u_target, lambda_n = Phi_n^T lambda_{n+1};
  dJ/du0 = lambda_0,  dJ/da = sum_n lambda_{n+1}^T (dPhi_n/da) u_n.
dPhi_n/da acts through the departure offsets only: (dPhi u)_i = sum_j w_j'(eps_i) (ds_i/da) u_{E_i+j}
(E_i is locally constant), with ds/da from differentiating the ERK stages (tangent-linear ERK).
In 2D (Sec. 4.1) the step is the tensor-product interpolation with weights wx_a(eps) wy_b(nu), so
(dPhi u)_i = sum_{a,b} [wx_a'(eps_i) dsx_i/da wy_b(nu_i) + wx_a(eps_i) wy_b'(nu_i) dsy_i/da] u_{..}.
The adjoint MGRIT solve uses the reversed problem mu_k = lambda_{nt-k}, mu_{k+1} = Phi_{nt-1-k}^T mu_k,
whose coarse operators are the transposed coarse operators Psi^T of the forward hierarchy.
"""

from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import coarse as co
from . import mgrit as mg
from . import semi_lagrangian as sl

TWO_PI = 2.0 * math.pi

# ---------------------------------------------------------------------------
# transposed operators (plain definitions: scatter of the gather's weights)
# ---------------------------------------------------------------------------


def sl_matrix_sparse_1d(s: np.ndarray, p: int) -> sp.csr_matrix:
    """The SL step as a sparse matrix: row i has w_j(eps_i) at column (E_i + j) mod nx."""
    nx = s.shape[0]
    fl, eps = sl.decompose(s)
    E = np.arange(nx, dtype=np.int64) - fl
    w = sl.lagrange_weights(eps, p)
    st = sl.stencil(p)
    rows = np.repeat(np.arange(nx), len(st))
    cols = np.mod(E[:, None] + st[None, :], nx).ravel()
    return sp.csr_matrix((w.ravel(), (rows, cols)), shape=(nx, nx))


def sl_transpose_apply_1d(v: np.ndarray, s: np.ndarray, p: int) -> np.ndarray:
    """S^T v: every arrival point i adds w_j(eps_i) v_i to node (E_i + j) mod nx."""
    nx = v.shape[0]
    fl, eps = sl.decompose(s)
    E = np.arange(nx, dtype=np.int64) - fl
    w = sl.lagrange_weights(eps, p)
    out = np.zeros(nx)
    for a, j in enumerate(sl.stencil(p)):
        np.add.at(out, np.mod(E + j, nx), w[:, a] * v)
    return out


def sl_transpose_apply_2d(v: np.ndarray, sx: np.ndarray, sy: np.ndarray, p: int) -> np.ndarray:
    """S^T v in 2D: arrival point (i, j) adds wx_a wy_b v_{j,i} to node ((N + jb) mod ny, (E + ja) mod nx)."""
    ny, nx = v.shape
    fx, eps = sl.decompose(sx)
    fy, nu = sl.decompose(sy)
    E = np.arange(nx, dtype=np.int64)[None, :] - fx
    N = np.arange(ny, dtype=np.int64)[:, None] - fy
    wx = sl.lagrange_weights(eps, p)
    wy = sl.lagrange_weights(nu, p)
    st = sl.stencil(p)
    out = np.zeros_like(v)
    for b_, jb in enumerate(st):
        rows = np.mod(N + jb, ny)
        for a_, ja in enumerate(st):
            cols = np.mod(E + ja, nx)
            np.add.at(out, (rows, cols), wy[..., b_] * wx[..., a_] * v)
    return out


class TransposedSolver:
    """Applies M^{-T} (M = I - diag(sigma) D_{p+1}, or its 2D form) to vectors.

    mode "exact": sparse LU of M^T; mode "gmres": the same inexact GMRES as the forward solve
    (coarse.gmres_zero_guess), applied to M^T.
    """

    def __init__(self, M: sp.csc_matrix, mode: str = "exact", rtol: float = 1e-2, maxit: int = 10):
        self.MT = sp.csc_matrix(M.T)
        self.mode = mode
        self.rtol = rtol
        self.maxit = maxit
        self._lu = spla.splu(self.MT) if mode == "exact" else None

    def solve(self, v: np.ndarray) -> np.ndarray:
        shape = v.shape
        b = v.ravel()
        if self.mode == "exact":
            return self._lu.solve(b).reshape(shape)
        return co.gmres_zero_guess(self.MT, b, self.rtol, self.maxit).reshape(shape)


class ReversedTransposed:
    """The hierarchy of the reversed adjoint problem: step k of level l is Phi_{l, N_l-1-k}^T.

    Offers the interface mgrit.vcycle / mgrit.mgrit_solve use (levels, nlevels, step).
    """

    def __init__(self, H: mg.Hierarchy):
        self.H = H
        self.levels = H.levels
        self._tsolvers: dict[tuple[int, int], TransposedSolver] = {}

    @property
    def nlevels(self) -> int:
        return self.H.nlevels

    def step_T(self, l: int, n: int, v: np.ndarray) -> np.ndarray:
        """Phi_{l,n}^T v: S^T on level 0, (M^{-1} S)^T = S^T M^{-T} on coarse levels."""
        H = self.H
        lev = H.levels[l]
        if l > 0 and H.coarse == "bsl":
            key = (l, n)
            if key not in self._tsolvers:
                if H.dim == 1:
                    M = co.correction_matrix_1d(lev.sigma[n], H.p)
                else:
                    M = co.correction_matrix_2d(lev.sigma[0][n], lev.sigma[1][n], H.p)
                self._tsolvers[key] = TransposedSolver(M, H.solve_mode, H.gmres_rtol, H.gmres_maxit)
            v = self._tsolvers[key].solve(v)
        if H.dim == 1:
            return sl_transpose_apply_1d(v, lev.s[n], H.p)
        return sl_transpose_apply_2d(v, lev.s[0][n], lev.s[1][n], H.p)

    def step(self, l: int, k: int, v: np.ndarray) -> np.ndarray:
        return self.step_T(l, self.levels[l].nt - 1 - k, v)


def adjoint_sequential(H: mg.Hierarchy, lam_T: np.ndarray) -> np.ndarray:
    """lambda_n for n = 0..nt from lambda_nt by backward stepping with the transposed fine steps."""
    R = ReversedTransposed(H)
    nt = H.levels[0].nt
    lam = np.zeros((nt + 1,) + lam_T.shape)
    lam[nt] = lam_T
    for n in range(nt - 1, -1, -1):
        lam[n] = R.step_T(0, n, lam[n + 1])
    return lam


def adjoint_mgrit(H: mg.Hierarchy, lam_T: np.ndarray, M_init: np.ndarray, rtol: float = 1e-10,
                  max_iter: int = 200) -> tuple[np.ndarray, mg.SolveResult]:
    """Adjoint solve by MGRIT on the reversed problem (same cycle and convention as mgrit_solve)."""
    R = ReversedTransposed(H)
    res = mg.mgrit_solve(R, lam_T, M_init, rtol=rtol, max_iter=max_iter)
    lam = res.U[::-1].copy()  # lambda_n = mu_{nt - n}
    return lam, res


# ---------------------------------------------------------------------------
# the a-derivative of the departure offsets (tangent-linear ERK) and of the SL step
# ---------------------------------------------------------------------------


def dalpha(ws: sl.WaveSpeed, x: np.ndarray, t: float) -> tuple[np.ndarray, np.ndarray]:
    """(d alpha / d a, d alpha / d x) of the 1D families (a is the amplitude parameter)."""
    if ws.kind == "const":
        return np.ones_like(x), np.zeros_like(x)
    if ws.kind == "cos_t":
        return np.zeros_like(x), np.zeros_like(x)
    if ws.kind == "cos_t_cos_x":
        return np.zeros_like(x), -TWO_PI * math.cos(TWO_PI * t) * np.sin(TWO_PI * x)
    if ws.kind == "sin_kx_cos_t":
        ct = math.cos(TWO_PI * t)
        return np.sin(TWO_PI * ws.k * x) * ct, ws.a * TWO_PI * ws.k * np.cos(TWO_PI * ws.k * x) * ct
    raise ValueError(ws.kind)


def dvelocity(ws: sl.WaveSpeed, x: np.ndarray, y: np.ndarray, t: float):
    """Derivatives of the 2D families: ((dvx/da, dvx/dx, dvx/dy), (dvy/da, dvy/dx, dvy/dy)).

    The parameter a is the amplitude of "sin_cos2" (both components) and the x speed of "const2";
    "paper2" does not depend on it.
    """
    z = np.zeros_like(x)
    if ws.kind == "const2":
        return (np.ones_like(x), z, z), (z, z, z)
    if ws.kind == "paper2":
        ct = math.cos(TWO_PI * t / 3.4)
        return (z, z, 2.0 * math.pi * np.sin(math.pi * y) * np.cos(math.pi * y) * ct), \
               (z, 2.0 * math.pi * np.cos(math.pi * x) * np.sin(math.pi * x) * ct, z)
    if ws.kind == "sin_cos2":
        ct, st = math.cos(TWO_PI * t), math.sin(TWO_PI * t)
        return (np.sin(TWO_PI * y) * ct, z, ws.a * TWO_PI * np.cos(TWO_PI * y) * ct), \
               (np.cos(TWO_PI * x) * st, -ws.a * TWO_PI * np.sin(TWO_PI * x) * st, z)
    raise ValueError(ws.kind)


def departure_offsets_da_2d(grid: sl.Grid, ws: sl.WaveSpeed, n: int, r: int) -> tuple[np.ndarray, np.ndarray]:
    """(d sx / d a, d sy / d a) for the fine step t_n -> t_{n+1}: departure_offsets_2d's stages differentiated."""
    A, b, c = sl.erk_tableau(r)
    X, Y = np.meshgrid(grid.x, grid.x)
    dt = grid.dt
    t1 = (n + 1) * dt
    kx, ky, dkx, dky = [], [], [], []
    for s in range(len(b)):
        xs, ys = X.copy(), Y.copy()
        dxs, dys = np.zeros_like(X), np.zeros_like(Y)
        for j in range(s):
            if A[s, j] != 0.0:
                xs = xs - dt * A[s, j] * kx[j]
                ys = ys - dt * A[s, j] * ky[j]
                dxs = dxs - dt * A[s, j] * dkx[j]
                dys = dys - dt * A[s, j] * dky[j]
        ts = t1 - c[s] * dt
        vx, vy = ws.velocity(xs, ys, ts)
        (ax, xx, xy), (ay, yx, yy) = dvelocity(ws, xs, ys, ts)
        kx.append(vx)
        ky.append(vy)
        dkx.append(ax + xx * dxs + xy * dys)
        dky.append(ay + yx * dxs + yy * dys)
    dx = np.zeros_like(X)
    dy = np.zeros_like(Y)
    for s in range(len(b)):
        if b[s] != 0.0:
            dx = dx + b[s] * dkx[s]
            dy = dy + b[s] * dky[s]
    return dt * dx / grid.h, dt * dy / grid.h


def departure_offsets_da_1d(grid: sl.Grid, ws: sl.WaveSpeed, n: int, r: int) -> np.ndarray:
    """d s_i / d a for the fine step t_n -> t_{n+1}: the ERK stages of departure_offsets_1d differentiated."""
    A, b, c = sl.erk_tableau(r)
    x = grid.x
    dt = grid.dt
    t1 = (n + 1) * dt
    ks, dks = [], []
    for s in range(len(b)):
        xs = x.copy()
        dxs = np.zeros_like(x)
        for j in range(s):
            if A[s, j] != 0.0:
                xs = xs - dt * A[s, j] * ks[j]
                dxs = dxs - dt * A[s, j] * dks[j]
        ts = t1 - c[s] * dt
        da, dx = dalpha(ws, xs, ts)
        ks.append(ws.alpha(xs, ts))
        dks.append(da + dx * dxs)
    d = np.zeros_like(x)
    for s in range(len(b)):
        if b[s] != 0.0:
            d = d + b[s] * dks[s]
    return dt * d / grid.h


def lagrange_weights_deps(eps: np.ndarray, p: int) -> np.ndarray:
    """d w_j / d eps of lagrange_weights (product rule over the factors (-eps - q))."""
    nodes = sl.stencil(p)
    z = -np.asarray(eps, dtype=np.float64)
    out = np.zeros(z.shape + (len(nodes),))
    for a, j in enumerate(nodes):
        others = [q for q in nodes if q != j]
        denom = np.prod([float(j - q) for q in others])
        tot = np.zeros_like(z)
        for skip in others:
            term = np.ones_like(z)
            for q in others:
                if q != skip:
                    term = term * (z - q)
            tot = tot + term
        out[..., a] = -tot / denom  # d/d eps = - d/d z
    return out


def dphi_da_apply_1d(u: np.ndarray, s: np.ndarray, ds: np.ndarray, p: int) -> np.ndarray:
    """(dPhi/da) u = sum_j w_j'(eps_i) ds_i u_{E_i + j}."""
    nx = u.shape[0]
    fl, eps = sl.decompose(s)
    E = np.arange(nx, dtype=np.int64) - fl
    dw = lagrange_weights_deps(eps, p)
    idx = np.mod(E[:, None] + sl.stencil(p)[None, :], nx)
    return np.sum(dw * u[idx], axis=-1) * ds


def dphi_da_apply_2d(u: np.ndarray, sx: np.ndarray, sy: np.ndarray, dsx: np.ndarray, dsy: np.ndarray,
                     p: int) -> np.ndarray:
    """(dPhi/da) u in 2D: the product rule on wx_a(eps) wy_b(nu) with d eps/da = dsx, d nu/da = dsy."""
    ny, nx = u.shape
    fx, eps = sl.decompose(sx)
    fy, nu = sl.decompose(sy)
    E = np.arange(nx, dtype=np.int64)[None, :] - fx
    N = np.arange(ny, dtype=np.int64)[:, None] - fy
    wx, wy = sl.lagrange_weights(eps, p), sl.lagrange_weights(nu, p)
    dwx, dwy = lagrange_weights_deps(eps, p), lagrange_weights_deps(nu, p)
    st = sl.stencil(p)
    out = np.zeros_like(u)
    for b_, jb in enumerate(st):
        rows = np.mod(N + jb, ny)
        for a_, ja in enumerate(st):
            val = u[rows, np.mod(E + ja, nx)]
            out += (dwx[..., a_] * dsx * wy[..., b_] + wx[..., a_] * dwy[..., b_] * dsy) * val
    return out


# ---------------------------------------------------------------------------
# objective and gradients
# ---------------------------------------------------------------------------


def objective(grid: sl.Grid, ws: sl.WaveSpeed, p: int, u0: np.ndarray, u_target: np.ndarray) -> float:
    """J = 1/2 ||u_nt - u_target||^2 with sequential SL stepping (the oracle's forward)."""
    H = mg.Hierarchy(grid, ws, p, [])
    U = mg.sequential_solve(H, u0)
    d = U[-1] - u_target
    return 0.5 * float(np.sum(d * d))


def gradients(grid: sl.Grid, ws: sl.WaveSpeed, p: int, u0: np.ndarray, u_target: np.ndarray):
    """(dJ/du0, dJ/da) by the discrete adjoint with sequential forward and backward stepping."""
    H = mg.Hierarchy(grid, ws, p, [])
    U = mg.sequential_solve(H, u0)
    lam = adjoint_sequential(H, U[-1] - u_target)
    return lam[0], dJ_da(H, U, lam)


def dJ_da(H: mg.Hierarchy, U: np.ndarray, lam: np.ndarray) -> float:
    """sum_n lambda_{n+1} . (dPhi_n/da) u_n over the fine steps (U, lam: all nt+1 slices)."""
    grid, ws, p = H.grid, H.ws, H.p
    out = 0.0
    for n in range(grid.nt):
        if H.dim == 1:
            ds = departure_offsets_da_1d(grid, ws, n, H.r)
            out += float(lam[n + 1] @ dphi_da_apply_1d(U[n], H.levels[0].s[n], ds, p))
        else:
            dsx, dsy = departure_offsets_da_2d(grid, ws, n, H.r)
            v = dphi_da_apply_2d(U[n], H.levels[0].s[0][n], H.levels[0].s[1][n], dsx, dsy, p)
            out += float(np.sum(lam[n + 1] * v))
    return out
