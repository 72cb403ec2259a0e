"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the method itself: it only produces the
inputs a user would hand to a solver (initial conditions, the random initial
MGRIT iterate, wave-speed parameters and the batched problem list).  Both the
CUDA path and the CPU oracle receive these arrays, so neither side generates
its own random numbers.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: draw k of stream `seed` is mix(seed + (k + 1) * GOLDEN).
"""

from __future__ import annotations

import dataclasses

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_C2_BUMPS = 20260001
SEED_C3_BUMPS = 20260002
SEED_C4_PROBLEMS = 20260004
SEED_C5_BUMPS = 20260005
SEED_C5_TARGET = 20260006
SEED_INITIAL_ITERATE = 20260100


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """SplitMix64 output for each counter k of stream `seed` (uint64 array)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (counters.astype(np.uint64) + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """`count` doubles in [0, 1) from the top 53 bits of SplitMix64 draws."""
    k = np.arange(start, start + count, dtype=np.uint64)
    return (splitmix64(seed, k) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def grid_1d(nx: int, xmin: float = -1.0, xmax: float = 1.0) -> np.ndarray:
    """Left-aligned periodic nodes x_i = xmin + i h, h = (xmax - xmin) / nx."""
    h = (xmax - xmin) / nx
    return xmin + h * np.arange(nx, dtype=np.float64)


def u0_sin4(nx: int) -> np.ndarray:
    """The paper's 1D initial condition sin^4(pi x) on (-1, 1)."""
    x = grid_1d(nx)
    return np.sin(np.pi * x) ** 4


def u0_sin2_2d(nx: int) -> np.ndarray:
    """The paper's 2D initial condition sin^2[pi/2 (x-1)] sin^2[pi/2 (y-1)], row-major u[j][i] (y slow)."""
    x = grid_1d(nx)
    fx = np.sin(0.5 * np.pi * (x - 1.0)) ** 2
    return np.outer(fx, fx)


@dataclasses.dataclass(frozen=True)
class Bump:
    cx: float
    cy: float
    width: float


def bumps(seed: int, count: int) -> list[Bump]:
    """Gaussian bump parameters: centres U[-1, 1]^2, widths U[0.05, 0.2]."""
    r = uniform01(seed, 3 * count)
    return [Bump(-1.0 + 2.0 * r[3 * b], -1.0 + 2.0 * r[3 * b + 1], 0.05 + 0.15 * r[3 * b + 2]) for b in range(count)]


def _periodic_distance(x: np.ndarray, c: float) -> np.ndarray:
    d = np.mod(x - c + 1.0, 2.0) - 1.0
    return d


def u0_bumps_1d(nx: int, seed: int, count: int) -> np.ndarray:
    """Sum of unit-amplitude Gaussian bumps exp(-d^2 / (2 w^2)), d the periodic distance."""
    x = grid_1d(nx)
    u = np.zeros(nx)
    for b in bumps(seed, count):
        d = _periodic_distance(x, b.cx)
        u += np.exp(-(d * d) / (2.0 * b.width * b.width))
    return u


def u0_bumps_2d(nx: int, seed: int, count: int) -> np.ndarray:
    """2D sum of Gaussian bumps on the periodic square, row-major u[j][i] (y index j slow)."""
    x = grid_1d(nx)
    u = np.zeros((nx, nx))
    for b in bumps(seed, count):
        dx = _periodic_distance(x, b.cx)
        dy = _periodic_distance(x, b.cy)
        u += np.exp(-(dy[:, None] ** 2 + dx[None, :] ** 2) / (2.0 * b.width * b.width))
    return u


def initial_iterate(nt: int, npts: int, seed: int = SEED_INITIAL_ITERATE, rows: np.ndarray | None = None) -> np.ndarray:
    """Random initial MGRIT iterate with entries U[0, 1].

    Returns an (nt + 1) x npts array whose row n (n >= 1) holds draws
    (n - 1) * npts ... n * npts - 1 of the stream; row 0 is left at zero and is
    replaced by the initial condition by the solver.  With `rows` given, only
    those time rows are produced (for sampling large cases).
    """
    if rows is None:
        u = np.zeros((nt + 1, npts))
        u[1:] = uniform01(seed, nt * npts).reshape(nt, npts)
        return u
    rows = np.asarray(rows, dtype=np.int64)
    res = np.zeros((len(rows), npts))
    live = rows >= 1
    if live.any():
        counters = ((rows[live] - 1) * npts)[:, None] + np.arange(npts, dtype=np.int64)[None, :]
        draws = splitmix64(seed, counters.ravel().astype(np.uint64)) >> np.uint64(11)
        res[live] = (draws.astype(np.float64) * (1.0 / 9007199254740992.0)).reshape(-1, npts)
    return res


@dataclasses.dataclass(frozen=True)
class BatchedProblem:
    """One problem of the batched 1D workload: alpha = 1 + a sin(2 pi k x) cos(2 pi t)."""

    nx: int
    nt: int
    order: int
    a: float
    k: int
    m: int


def batched_problems(count: int = 256, seed: int = SEED_C4_PROBLEMS) -> list[BatchedProblem]:
    """The batched workload: nx, nt powers of two, order in {1,3,5}, a in [0.1,0.7], k in {1,2,3}, m in {4,8}."""
    r = uniform01(seed, 6 * count)
    out = []
    for q in range(count):
        u = r[6 * q : 6 * q + 6]
        nx = 256 << min(int(u[0] * 5), 4)
        nt = 1024 << min(int(u[1] * 5), 4)
        order = (1, 3, 5)[min(int(u[2] * 3), 2)]
        a = 0.1 + 0.6 * u[3]
        k = 1 + min(int(u[4] * 3), 2)
        m = (4, 8)[min(int(u[5] * 2), 1)]
        out.append(BatchedProblem(nx, nt, order, a, k, m))
    return out


def dof_count(nx: int, nt: int, dim: int = 1) -> int:
    """Space-time unknowns u_1 ... u_nt: nx^dim * nt."""
    return int(nx) ** dim * int(nt)


def cfl_dt(nx: int, cfl: float = 0.85, xmin: float = -1.0, xmax: float = 1.0) -> float:
    return cfl * (xmax - xmin) / nx

