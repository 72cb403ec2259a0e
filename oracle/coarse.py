"""Corrected semi-Lagrangian coarse-grid operators (oracle, FP64, numpy/scipy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 3 of the paper: D_{p+1} (eq. (Dp+1_def)), f_{p+1} (eq. (fpoly_def)),
phi_{p+1} (eq. (varphi_p_def), (varphi_p_multilevel_def)), the multilevel
sigma recursion (eq. (nu_p_def)) and the backward-Euler corrected operator
Psi = [I - diag(sigma) D_{p+1}]^{-1} S_{p,r*} (eq. (Bp_def), (Psi_Bp_def2),
(Phi_multilevel)); the backtracking estimate of coarse departure points
(eq. (coarse_depart_interp), Sec. 3.3.1) and its 2D bilinear version
(Sec. SM6, eq. (SM:poly_interp_1d), (SM:poly_interp_2d)); the 2D operator
(eq. (BEOper_2D)).

Offsets are displacements in grid units (see semi_lagrangian): the departure
point of the characteristic arriving at x_i is x_i - h s_i.
"""

from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .semi_lagrangian import decompose, stencil

# ---------------------------------------------------------------------------
# D_{p+1} and f_{p+1}
# ---------------------------------------------------------------------------


def second_difference(nx: int) -> sp.csr_matrix:
    """Periodic second difference: (T v)_i = v_{i-1} - 2 v_i + v_{i+1}."""
    e = np.ones(nx)
    T = sp.diags([e[:-1], -2.0 * e, e[:-1]], [-1, 0, 1], shape=(nx, nx), format="lil")
    T[0, nx - 1] = 1.0
    T[nx - 1, 0] = 1.0
    return T.tocsr()


def D_matrix(nx: int, p: int) -> sp.csr_matrix:
    """D_{p+1}: periodic, second-order (p+1)-th difference, h^{-(p+1)} D v ~ v^{(p+1)} (eq. (Dp+1_def)).

    The paper fixes only that it is periodic and second-order accurate
    (Sec. 3.2).  Reading: the centred stencil (delta^2)^{(p+1)/2}, i.e. the
    periodic second difference raised to the power (p+1)/2.
    """
    T = second_difference(nx)
    D = sp.identity(nx, format="csr")
    for _ in range((p + 1) // 2):
        D = D @ T
    return D.tocsr()


def f_poly(z: np.ndarray, p: int) -> np.ndarray:
    """f_{p+1}(z) = 1/(p+1)! prod_{q=-l(p)}^{r(p)} (q + z)  (eq. (fpoly_def))."""
    out = np.ones_like(np.asarray(z, dtype=np.float64))
    for q in stencil(p):
        out = out * (q + z)
    return out / math.factorial(p + 1)


def eps_of(s: np.ndarray) -> np.ndarray:
    """The east-neighbour distance eps in [0, 1) of offsets s (eq. (depart_decompose))."""
    return decompose(s)[1]


# ---------------------------------------------------------------------------
# Backtracking coarse departure points (Sec. 3.3.1 in 1D, Sec. SM6 in 2D)
# ---------------------------------------------------------------------------


def backtrack_1d(s_fine: np.ndarray, m: int) -> np.ndarray:
    """Coarse departure offsets from the fine ones by linear interpolation and backtracking.

    s_fine: (m * N, nx) offsets of the level above; returns (N, nx).
    Eq. (coarse_depart_interp): c^{(m-1)} = f^{(m-1)}; for k = m-2 .. 0,
    c^{(k)} = (f_E^{(k)} - f_W^{(k)})/h (c^{(k+1)} - x_E) + f_E^{(k)}, with x_E, x_W
    the east and west nodes of c^{(k+1)}.  Positions are written in grid units
    relative to the arrival node x_i (the formula is invariant under that
    translation and scaling), and the fine departure point arriving at node E is
    E - s^{(k)}_{E mod nx} in that frame (alpha is periodic).
    """
    nsteps, nx = s_fine.shape
    N = nsteps // m
    i = np.arange(nx, dtype=np.int64)
    out = np.zeros((N, nx))
    for n in range(N):
        c = -s_fine[m * n + m - 1]  # c^{(m-1)} = f^{(m-1)}, relative to x_i
        for k in range(m - 2, -1, -1):
            sk = s_fine[m * n + k]
            xE = np.ceil(c)  # east node of c (a node itself if c lies on one)
            E = i + xE.astype(np.int64)
            fE = xE - sk[np.mod(E, nx)]
            fW = (xE - 1.0) - sk[np.mod(E - 1, nx)]
            c = (fE - fW) * (c - xE) + fE
        out[n] = -c
    return out


def _p1d(x: np.ndarray, xE: np.ndarray, qE: np.ndarray, qW: np.ndarray) -> np.ndarray:
    """Eq. (SM:poly_interp_1d) in grid units: (q_E - q_W)(x - x_E) + q_E."""
    return (qE - qW) * (x - xE) + qE


def _p2d(x, y, xE, yN, rNE, rNW, rSE, rSW):
    """Eq. (SM:poly_interp_2d) in grid units: (p1d_N - p1d_S)(y - y_N) + p1d_N."""
    pN = _p1d(x, xE, rNE, rNW)
    pS = _p1d(x, xE, rSE, rSW)
    return (pN - pS) * (y - yN) + pN


def backtrack_2d(sx_fine: np.ndarray, sy_fine: np.ndarray, m: int) -> tuple[np.ndarray, np.ndarray]:
    """2D coarse departure offsets by bilinear backtracking (Sec. SM6).

    sx_fine, sy_fine: (m * N, ny, nx); returns two (N, ny, nx) arrays.  At each
    sub-step the x and y components are fitted separately with the bilinear
    function through the four fine characteristics arriving at the nodes NE,
    NW, SE, SW around (c^{(k+1)}, d^{(k+1)}).  (The definition of y_N in the
    paper reads "x_S + h"; the reading is y_N = y_S + h.)
    """
    nsteps, ny, nx = sx_fine.shape
    N = nsteps // m
    I = np.arange(nx, dtype=np.int64)[None, :]
    J = np.arange(ny, dtype=np.int64)[:, None]
    ox = np.zeros((N, ny, nx))
    oy = np.zeros((N, ny, nx))
    for n in range(N):
        c = -sx_fine[m * n + m - 1]
        d = -sy_fine[m * n + m - 1]
        for k in range(m - 2, -1, -1):
            kx = sx_fine[m * n + k]
            ky = sy_fine[m * n + k]
            xE = np.ceil(c)
            yN = np.ceil(d)
            E = np.mod(I + xE.astype(np.int64), nx)
            W = np.mod(I + xE.astype(np.int64) - 1, nx)
            Nn = np.mod(J + yN.astype(np.int64), ny)
            S = np.mod(J + yN.astype(np.int64) - 1, ny)
            xW = xE - 1.0
            yS = yN - 1.0
            cx = _p2d(c, d, xE, yN, xE - kx[Nn, E], xW - kx[Nn, W], xE - kx[S, E], xW - kx[S, W])
            cy = _p2d(c, d, xE, yN, yN - ky[Nn, E], yN - ky[Nn, W], yS - ky[S, E], yS - ky[S, W])
            c, d = cx, cy
        ox[n] = -c
        oy[n] = -d
    return ox, oy


# ---------------------------------------------------------------------------
# phi and sigma (eq. (varphi_p_def), (varphi_p_multilevel_def), (nu_p_def))
# ---------------------------------------------------------------------------


def phi(s_coarse: np.ndarray, s_fine: np.ndarray, m: int, p: int) -> np.ndarray:
    """phi[n][i] = (-1)^{p+1} (f(eps_coarse[n][i]) - sum_{k<m} f(eps_fine[m n + k][i])).

    The sum runs over the m fine steps at the same arrival index i, as the
    equation is written (not along the characteristic).
    """
    N = s_coarse.shape[0]
    fc = f_poly(eps_of(s_coarse), p)
    ff = f_poly(eps_of(s_fine), p).reshape((N, m) + s_fine.shape[1:]).sum(axis=1)
    return (-1.0) ** (p + 1) * (fc - ff)


def sigma_next(sigma_fine: np.ndarray | None, phi_coarse: np.ndarray, m: int) -> np.ndarray:
    """Eq. (nu_p_def): sigma_1 = phi_1; sigma_l[n] = sum_{k<m} sigma_{l-1}[m n + k] + phi_l[n]."""
    if sigma_fine is None:
        return phi_coarse.copy()
    N = phi_coarse.shape[0]
    return sigma_fine.reshape((N, m) + sigma_fine.shape[1:]).sum(axis=1) + phi_coarse


# ---------------------------------------------------------------------------
# The correction matrix and its solves (eq. (Bp_def), (Phi_multilevel), (BEOper_2D))
# ---------------------------------------------------------------------------


def correction_matrix_1d(sigma: np.ndarray, p: int) -> sp.csc_matrix:
    """M = I - diag(sigma) D_{p+1}."""
    nx = sigma.shape[0]
    return (sp.identity(nx) - sp.diags(sigma) @ D_matrix(nx, p)).tocsc()


def correction_matrix_2d(sigma_x: np.ndarray, sigma_y: np.ndarray, p: int) -> sp.csc_matrix:
    """M = I - diag(sigma_x)(I (x) D) - diag(sigma_y)(D (x) I), row-major [j][i] ordering (eq. (BEOper_2D))."""
    ny, nx = sigma_x.shape
    D = D_matrix(nx, p)
    Dx = sp.kron(sp.identity(ny), D)
    Dy = sp.kron(D_matrix(ny, p), sp.identity(nx))
    M = sp.identity(nx * ny) - sp.diags(sigma_x.ravel()) @ Dx - sp.diags(sigma_y.ravel()) @ Dy
    return M.tocsc()


class CorrectionSolver:
    """Applies [I - diag(sigma) D]^{-1} to vectors.

    mode "exact": sparse LU with partial pivoting (scipy SuperLU), the reading
      that keeps MGRIT linear.
    mode "gmres": the paper's inexact solve, unpreconditioned GMRES from a zero
      initial guess, stopped at relative residual `rtol` or `maxit` iterations
      (Sec. 3.3: 10 iterations; Sec. 3.4 and 4.3: rtol 1e-2 or 10 iterations).
    """

    def __init__(self, M: sp.csc_matrix, mode: str = "exact", rtol: float = 1e-2, maxit: int = 10):
        self.M = M
        self.mode = mode
        self.rtol = rtol
        self.maxit = maxit
        self._lu = spla.splu(M) if mode == "exact" else None

    def solve(self, v: np.ndarray) -> np.ndarray:
        shape = v.shape
        b = v.ravel()
        if self.mode == "exact":
            return self._lu.solve(b).reshape(shape)
        x = gmres_zero_guess(self.M, b, self.rtol, self.maxit)
        return x.reshape(shape)


def gmres_zero_guess(A, b: np.ndarray, rtol: float, maxit: int) -> np.ndarray:
    """Plain GMRES (Arnoldi with modified Gram-Schmidt, Givens-free least squares) from x0 = 0.

    Stops when ||b - A x|| <= rtol ||b|| or after maxit iterations.
    """
    n = b.shape[0]
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return np.zeros(n)
    V = np.zeros((maxit + 1, n))
    H = np.zeros((maxit + 1, maxit))
    V[0] = b / beta
    y = np.zeros(0)
    k_used = 0
    for k in range(maxit):
        w = A @ V[k]
        for j in range(k + 1):
            H[j, k] = np.dot(V[j], w)
            w = w - H[j, k] * V[j]
        H[k + 1, k] = np.linalg.norm(w)
        k_used = k + 1
        e1 = np.zeros(k + 2)
        e1[0] = beta
        y, *_ = np.linalg.lstsq(H[: k + 2, : k + 1], e1, rcond=None)
        res = np.linalg.norm(e1 - H[: k + 2, : k + 1] @ y)
        if res <= rtol * beta or H[k + 1, k] == 0.0:
            break
        V[k + 1] = w / H[k + 1, k]
    return V[:k_used].T @ y
