"""Sequential time stepping and linear MGRIT with FCF relaxation (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2.2 of the paper: the one-step system u_{n+1} = Phi_n u_n + g_{n+1}
(eq. (one-step)); F-relaxation (step from each C-point across its m-1
F-points), C-relaxation (one step into each C-point), FCF pre-relaxation,
the coarse residual equation e_{m(n+1)} = Psi e_{mn} + r_{m(n+1)}
(eq. (one-step-coarse)) with injection, post F-relaxation; recursion gives the
V-cycle (Sec. 3.4), the coarsest level is solved by sequential stepping.
Linear MGRIT (residual correction, not FAS) as in Sec. SM2.

Level rule (Sec. 3.4): coarsen by m until a further coarsening would leave
fewer than two time points; `max_coarsest` > 1 stops earlier, once a level has
at most that many steps.
"""

from __future__ import annotations

import dataclasses

import numpy as np

from . import coarse as co
from . import semi_lagrangian as sl


def coarsening_factors(nt: int, m, levels: int = 0, max_coarsest: int = 1) -> list[int]:
    """The coarsening factor of each coarse level (level l has nt / prod(factors[:l]) steps).

    m: an int (same factor on all levels) or a list (m_1, m_2, ...; the last is
    repeated).  levels > 0 fixes the number of levels; levels == 0 applies the
    rule "coarsen while the level has more than max_coarsest steps and the
    next level keeps at least one step".
    """
    ms = [m] if isinstance(m, int) else list(m)
    out: list[int] = []
    n = nt
    while True:
        if levels > 0 and len(out) + 1 >= levels:
            break
        f = ms[min(len(out), len(ms) - 1)]
        if levels == 0 and n <= max_coarsest:
            break
        if n % f != 0 or n // f < 1:
            if levels > 0:
                raise ValueError("nt is not divisible by the coarsening factors for the requested levels")
            break
        out.append(f)
        n //= f
    return out


@dataclasses.dataclass
class Level:
    index: int
    nt: int
    m: int  # coarsening factor from the level above (0 on level 0)
    s: object  # 1D: (nt, nx) offsets; 2D: (sx, sy) each (nt, nx, nx)
    sigma: object = None  # 1D: (nt, nx); 2D: (sigma_x, sigma_y)


class Hierarchy:
    """Departure data, sigma and correction solvers on every level.

    coarse: "bsl" the paper's corrected operator (eq. (Phi_multilevel), (BEOper_2D));
            "sl" the plain coarse SL step with the same departure points;
            "ideal" the product of the m operators of the level above (eq. below (one-step-coarse)).
    solve_mode: "exact" or "gmres" (see coarse.CorrectionSolver).
    """

    def __init__(self, grid: sl.Grid, ws: sl.WaveSpeed, p: int, factors: list[int], r: int | None = None,
                 coarse: str = "bsl", solve_mode: str = "exact", gmres_rtol: float = 1e-2, gmres_maxit: int = 10):
        self.grid = grid
        self.ws = ws
        self.p = p
        self.r = p if r is None else r
        self.dim = grid.dim
        self.coarse = coarse
        self.solve_mode = solve_mode
        self.gmres_rtol = gmres_rtol
        self.gmres_maxit = gmres_maxit
        self.factors = list(factors)
        self.levels: list[Level] = []
        self._solvers: dict[tuple[int, int], co.CorrectionSolver] = {}
        nt = grid.nt
        if self.dim == 1:
            s0 = np.stack([sl.departure_offsets_1d(grid, ws, n, self.r) for n in range(nt)])
        else:
            pairs = [sl.departure_offsets_2d(grid, ws, n, self.r) for n in range(nt)]
            s0 = (np.stack([a for a, _ in pairs]), np.stack([b for _, b in pairs]))
        self.levels.append(Level(0, nt, 0, s0))
        for l, m in enumerate(self.factors, start=1):
            prev = self.levels[-1]
            if self.dim == 1:
                s = co.backtrack_1d(prev.s, m)
                ph = co.phi(s, prev.s, m, p)
                sig = co.sigma_next(prev.sigma, ph, m)
            else:
                sx, sy = co.backtrack_2d(prev.s[0], prev.s[1], m)
                phx = co.phi(sx, prev.s[0], m, p)
                phy = co.phi(sy, prev.s[1], m, p)
                psx = None if prev.sigma is None else prev.sigma[0]
                psy = None if prev.sigma is None else prev.sigma[1]
                s = (sx, sy)
                sig = (co.sigma_next(psx, phx, m), co.sigma_next(psy, phy, m))
            self.levels.append(Level(l, prev.nt // m, m, s, sig))

    @property
    def nlevels(self) -> int:
        return len(self.levels)

    def slice_shape(self) -> tuple[int, ...]:
        return (self.grid.nx,) if self.dim == 1 else (self.grid.nx, self.grid.nx)

    def sl_step(self, l: int, n: int, u: np.ndarray) -> np.ndarray:
        lev = self.levels[l]
        if self.dim == 1:
            return sl.sl_apply_1d(u, lev.s[n], self.p)
        return sl.sl_apply_2d(u, lev.s[0][n], lev.s[1][n], self.p)

    def solver(self, l: int, n: int) -> co.CorrectionSolver:
        key = (l, n)
        if key not in self._solvers:
            lev = self.levels[l]
            if self.dim == 1:
                M = co.correction_matrix_1d(lev.sigma[n], self.p)
            else:
                M = co.correction_matrix_2d(lev.sigma[0][n], lev.sigma[1][n], self.p)
            self._solvers[key] = co.CorrectionSolver(M, self.solve_mode, self.gmres_rtol, self.gmres_maxit)
        return self._solvers[key]

    def step(self, l: int, n: int, u: np.ndarray) -> np.ndarray:
        """Phi_{l,n} u: the fine SL step on level 0, the coarse operator on levels l >= 1."""
        if l == 0:
            return self.sl_step(0, n, u)
        if self.coarse == "ideal":
            m = self.levels[l].m
            v = u
            for k in range(m):
                v = self.step(l - 1, m * n + k, v)
            return v
        v = self.sl_step(l, n, u)
        if self.coarse == "sl":
            return v
        return self.solver(l, n).solve(v)


def build_hierarchy(grid: sl.Grid, ws: sl.WaveSpeed, p: int, m, levels: int = 0, max_coarsest: int = 1, **kw) -> Hierarchy:
    return Hierarchy(grid, ws, p, coarsening_factors(grid.nt, m, levels, max_coarsest), **kw)


# ---------------------------------------------------------------------------
# Sequential stepping (eq. (one-step))
# ---------------------------------------------------------------------------


def sequential_solve(H: Hierarchy, u0: np.ndarray, level: int = 0, g: np.ndarray | None = None) -> np.ndarray:
    """u_{n+1} = Phi_n u_n + g_{n+1}, n = 0 .. N-1; returns all N+1 slices."""
    N = H.levels[level].nt
    U = np.zeros((N + 1,) + u0.shape)
    U[0] = u0
    for n in range(N):
        U[n + 1] = H.step(level, n, U[n]) + (0.0 if g is None else g[n + 1])
    return U


# ---------------------------------------------------------------------------
# MGRIT
# ---------------------------------------------------------------------------


def residual(H: Hierarchy, l: int, U: np.ndarray, g: np.ndarray) -> np.ndarray:
    """r_n = g_n + Phi_{n-1} u_{n-1} - u_n for n = 1 .. N (row 0 is zero)."""
    r = np.zeros_like(U)
    for n in range(1, U.shape[0]):
        r[n] = g[n] + H.step(l, n - 1, U[n - 1]) - U[n]
    return r


def f_relax(H: Hierarchy, l: int, U: np.ndarray, g: np.ndarray, m: int) -> None:
    """F-relaxation: from each C-point u_{jm}, step across the m-1 F-points after it."""
    N = U.shape[0] - 1
    for j in range(N // m):
        for k in range(1, m):
            n = j * m + k
            U[n] = H.step(l, n - 1, U[n - 1]) + g[n]


def c_relax(H: Hierarchy, l: int, U: np.ndarray, g: np.ndarray, m: int) -> None:
    """C-relaxation: one step from the last F-point into each C-point u_{jm}, j >= 1."""
    N = U.shape[0] - 1
    for j in range(1, N // m + 1):
        n = j * m
        U[n] = H.step(l, n - 1, U[n - 1]) + g[n]


def c_residual(H: Hierarchy, l: int, U: np.ndarray, g: np.ndarray, m: int) -> np.ndarray:
    """C-point residuals r_{jm} = g_{jm} + Phi u_{jm-1} - u_{jm}, returned as the coarse right-hand side."""
    N = U.shape[0] - 1
    Nc = N // m
    gc = np.zeros((Nc + 1,) + U.shape[1:])
    for j in range(1, Nc + 1):
        n = j * m
        gc[j] = g[n] + H.step(l, n - 1, U[n - 1]) - U[n]
    return gc


def relax(H: Hierarchy, l: int, U: np.ndarray, g: np.ndarray, m: int, mode: str) -> None:
    """The pre-relaxation of a cycle (Sec. 2.2): "FCF" (F, then C, then F) or "F" (F-relaxation only,
    the Parareal form)."""
    f_relax(H, l, U, g, m)
    if mode == "FCF":
        c_relax(H, l, U, g, m)
        f_relax(H, l, U, g, m)
    elif mode != "F":
        raise ValueError(mode)


def vcycle(H: Hierarchy, l: int, U: np.ndarray, g: np.ndarray, mode: str = "FCF") -> None:
    """One V-cycle on level l: relaxation, coarse residual by injection, recursive coarse solve,
    correction, F-relaxation."""
    if l == H.nlevels - 1:
        for n in range(1, U.shape[0]):
            U[n] = H.step(l, n - 1, U[n - 1]) + g[n]
        return
    m = H.levels[l + 1].m
    relax(H, l, U, g, m, mode)
    gc = c_residual(H, l, U, g, m)
    Ec = np.zeros_like(gc)
    vcycle(H, l + 1, Ec, gc, mode)
    N = U.shape[0] - 1
    for j in range(1, N // m + 1):
        U[j * m] += Ec[j]
    f_relax(H, l, U, g, m)


@dataclasses.dataclass
class SolveResult:
    U: np.ndarray
    iterations: int
    history: list[float]
    converged: bool
    final_errors: list[float] | None = None


def mgrit_solve(H: Hierarchy, u0: np.ndarray, U_init: np.ndarray, rtol: float = 1e-10, max_iter: int = 200,
                norm_mode: int = 1, mode: str = "FCF", u_final_ref: np.ndarray | None = None,
                final_tol: float = 0.0) -> SolveResult:
    """Iterate MGRIT V-cycles from U_init until the space-time residual drops by rtol (Sec. 2.2).

    norm_mode 0: r_0 is the 2-norm of the residual of the initial iterate over
      all n = 1..nt; r_k (k >= 1) is the residual after V-cycle k (post
      F-relaxation, so only C-points contribute).  Stop at the first k with
      r_k < rtol r_0 and report k.
    norm_mode 1 (the convention of the paper's tables): r_k is the C-point
      residual after the FCF relaxation of cycle k (k = 0, 1, ...), r_0 the
      first of these.  Every cycle completes its coarse correction and post
      F-relaxation; after cycle k the solve stops if k >= 1 and
      r_k < rtol r_0, and reports k + 1 cycles.  (With exact coarse solves this
      reproduces the constant-wave-speed columns of Table 2 exactly.)
    mode: "FCF" (the paper's relaxation) or "F" (F-relaxation only, every level).
    u_final_ref (norm_mode 1): the alternative stopping rule of Sec. SM4 -- after the correction and
      post F-relaxation of cycle k, e_k = (h^d sum (u(T) - u_final_ref)^2)^(1/2) (the discrete l2
      norm of the final time slice's distance to the reference, e.g. the exact PDE solution); the
      solve stops at the first e_k <= final_tol and reports k + 1 cycles (the residual test is not
      applied).  The e_k are returned in final_errors.
    """
    if H.nlevels < 2:
        raise ValueError("MGRIT needs at least two levels")
    U = U_init.copy()
    U[0] = u0
    g = np.zeros_like(U)
    hist: list[float] = []
    if norm_mode == 0:
        r0 = float(np.linalg.norm(residual(H, 0, U, g)))
        hist.append(r0)
        for it in range(1, max_iter + 1):
            vcycle(H, 0, U, g, mode)
            rk = float(np.linalg.norm(residual(H, 0, U, g)))
            hist.append(rk)
            if rk < rtol * r0:
                return SolveResult(U, it, hist, True)
        return SolveResult(U, max_iter, hist, False)
    m = H.levels[1].m
    N = U.shape[0] - 1
    errs: list[float] | None = None if u_final_ref is None else []
    wgt = None if u_final_ref is None else H.grid.h ** H.grid.dim
    for k in range(0, max_iter):
        relax(H, 0, U, g, m, mode)
        gc = c_residual(H, 0, U, g, m)
        rk = float(np.linalg.norm(gc))
        hist.append(rk)
        Ec = np.zeros_like(gc)
        vcycle(H, 1, Ec, gc, mode)
        for j in range(1, N // m + 1):
            U[j * m] += Ec[j]
        f_relax(H, 0, U, g, m)
        if errs is not None:
            ek = float(np.sqrt(wgt * np.sum((U[N] - u_final_ref) ** 2)))
            errs.append(ek)
            if ek <= final_tol:
                return SolveResult(U, k + 1, hist, True, errs)
        elif k >= 1 and rk < rtol * hist[0]:
            return SolveResult(U, k + 1, hist, True)
    return SolveResult(U, max_iter, hist, False, errs)
