"""Pins for the oracle's sequential stepping and MGRIT cycle (Sec. 2.2, 3.3, 3.4)."""

import concurrent.futures as cf
import multiprocessing
import os

import numpy as np
import pytest

import oracle_jobs
import workloads as W
from oracle import mgrit as mg
from oracle import semi_lagrangian as sl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALPHA = {"alpha1": "const", "alpha2": "cos_t", "alpha4": "cos_t_cos_x"}


def read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            a, p, m, it = line.split()
            rows.append((a, int(p), int(m), int(it)))
    return rows


def test_coarsening_rules():
    """Coarsen until a further level would have fewer than two time points (Sec. 3.4); or stop at <= 8 steps."""
    assert mg.coarsening_factors(1024, 4) == [4] * 5  # 1024 .. 4 .. 1
    assert mg.coarsening_factors(2048, 4) == [4] * 5  # .. 8 .. 2
    assert mg.coarsening_factors(16384, 8, max_coarsest=8) == [8] * 4  # .. 32 .. 4
    assert mg.coarsening_factors(256, 4, levels=2) == [4]
    assert mg.coarsening_factors(16384, [16, 4]) == [16, 4, 4, 4, 4, 4]


def _small(kind="sin_kx_cos_t", nx=48, nt=64, p=3, m=4, **kw):
    g = sl.Grid(nx, nt)
    ws = sl.WaveSpeed(kind, a=0.5, k=1)
    H = mg.build_hierarchy(g, ws, p, m, **kw)
    return g, H, W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3), W.initial_iterate(nt, nx)


def test_ideal_coarse_operator_converges_in_one_iteration():
    """Psi = Phi^m makes the coarse problem the exact Schur complement: one iteration (Sec. 2.2)."""
    g, H, u0, U0 = _small(levels=2, coarse="ideal")
    R = mg.mgrit_solve(H, u0, U0, norm_mode=0)
    assert R.iterations == 1 and R.history[1] < 1e-13 * R.history[0]


def test_integer_courant_converges_in_one_iteration():
    """alpha = 1, c = 1: phi = 0 and the coarse SL step is the exact m-shift, so Psi = Phi^m."""
    g = sl.Grid(32, 64, cfl=1.0)
    H = mg.build_hierarchy(g, sl.WaveSpeed("const"), 3, 4)
    R = mg.mgrit_solve(H, W.u0_sin4(32), W.initial_iterate(64, 32), norm_mode=0)
    assert R.iterations == 1


@pytest.mark.parametrize("norm_mode", [0, 1])
def test_fixed_point_is_sequential_solution(norm_mode):
    """MGRIT solves the same one-step system as sequential stepping (eq. (one-step))."""
    g, H, u0, U0 = _small()
    R = mg.mgrit_solve(H, u0, U0, norm_mode=norm_mode)
    assert R.converged
    Useq = mg.sequential_solve(H, u0)
    assert np.linalg.norm(R.U - Useq) / np.linalg.norm(Useq) < 1e-9


@pytest.mark.parametrize("solve_mode", ["exact", "gmres"])
def test_fixed_point_2d_is_sequential_solution(solve_mode):
    """2D (Sec. 4): with exact correction solves or the paper's inexact GMRES (rtol 1e-2, 10 iterations)
    the cycle converges to the solution of the fine one-step system, i.e. sequential stepping."""
    nx, nt = 8, 64
    g = sl.Grid(nx, nt, dim=2)
    H = mg.build_hierarchy(g, sl.WaveSpeed("sin_cos2", a=0.5, a2=0.5), 3, 2, solve_mode=solve_mode)
    u0 = W.u0_bumps_2d(nx, W.SEED_C5_BUMPS, 5)
    R = mg.mgrit_solve(H, u0, W.initial_iterate(nt, nx * nx).reshape(nt + 1, nx, nx), norm_mode=1)
    assert R.converged and R.iterations > 3
    Useq = mg.sequential_solve(H, u0)
    assert np.linalg.norm(R.U - Useq) / np.linalg.norm(Useq) < 1e-9


def test_residual_history_is_contracting():
    g, H, u0, U0 = _small(kind="cos_t_cos_x", p=1, m=8)
    R = mg.mgrit_solve(H, u0, U0)
    h = np.array(R.history)
    assert np.all(h[2:] < h[1:-1])


def test_rediscretised_coarse_operator_diverges_where_the_corrected_one_converges():
    """Constant alpha, c = 0.85, p = 3, m = 8: the plain coarse SL operator lets the residual grow
    (rho(c) > 1 in Fig. 2, Sec. 2.3) while the corrected operator converges (Fig. 3)."""
    g = sl.Grid(64, 1024, cfl=0.85)
    U0 = W.initial_iterate(1024, 64)
    res = {}
    for kind in ("bsl", "sl"):
        H = mg.build_hierarchy(g, sl.WaveSpeed("const"), 3, 8, levels=2, coarse=kind)
        res[kind] = mg.mgrit_solve(H, W.u0_sin4(64), U0, max_iter=20 if kind == "bsl" else 6)
    assert res["bsl"].converged and res["bsl"].iterations <= 18
    h = res["sl"].history
    assert not res["sl"].converged and h[-1] > 10.0 * h[1]


FAST_T2 = {("alpha1", 1, 4), ("alpha1", 1, 8), ("alpha1", 1, 16), ("alpha2", 1, 16), ("alpha4", 1, 8),
           ("alpha1", 3, 16), ("alpha4", 3, 16)}
# Cells where the exact coarse solve (the reading used here) differs from the paper's
# GMRES-based solve by one iteration; all other cells must match exactly.
KNOWN_OFF_BY_ONE = {("table2", "alpha4", 3, 4), ("table1", "alpha2", 1, 8), ("table1", "alpha4", 3, 4)}


def _check_count(table, a, p, m, expect, got):
    if (table, a, p, m) in KNOWN_OFF_BY_ONE:
        assert abs(got - expect) <= 1
    else:
        assert got == expect


def _table_case(table, a, p, m, expect, levels):
    nx, nt = 256, 1024
    g = sl.Grid(nx, nt)
    H = mg.build_hierarchy(g, sl.WaveSpeed(ALPHA[a]), p, m, levels=levels)
    R = mg.mgrit_solve(H, W.u0_sin4(nx), W.initial_iterate(nt, nx))
    _check_count(table, a, p, m, expect, R.iterations)


@pytest.mark.parametrize("a,p,m,expect", [r for r in read_table("table2_multilevel_iters.txt") if r[:3] in FAST_T2])
def test_table2_multilevel_iterations(a, p, m, expect):
    _table_case("table2", a, p, m, expect, levels=0)


@pytest.mark.parametrize("a,p,m,expect", [r for r in read_table("table1_two_level_iters.txt")
                                          if r[:3] in {("alpha1", 1, 16), ("alpha4", 1, 16), ("alpha2", 1, 8)}])
def test_table1_two_level_iterations(a, p, m, expect):
    _table_case("table1", a, p, m, expect, levels=2)


# The remaining cells of both tables (14 of Table 2, all 18 of Table 1): the oracle's solves run at once in
# a process pool started with `spawn`, one worker per core (about 50 s on 8 cores), then each cell is checked.
REST_T2 = [r for r in read_table("table2_multilevel_iters.txt") if r[:3] not in FAST_T2]
ALL_T1 = read_table("table1_two_level_iters.txt")


@pytest.fixture(scope="module")
def table_counts():
    jobs = [("table2", a, p, m, 0) for a, p, m, _ in REST_T2] + [("table1", a, p, m, 2) for a, p, m, _ in ALL_T1]
    workers = max(1, min(len(jobs), os.cpu_count() or 1))
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=multiprocessing.get_context("spawn")) as ex:
        futs = {j: ex.submit(oracle_jobs.table_cell_iterations, ALPHA[j[1]], j[2], j[3], j[4]) for j in jobs}
        return {j[:4]: f.result() for j, f in futs.items()}


@pytest.mark.parametrize("a,p,m,expect", REST_T2)
def test_table2_multilevel_iterations_remaining_cells(table_counts, a, p, m, expect):
    _check_count("table2", a, p, m, expect, table_counts[("table2", a, p, m)])


@pytest.mark.parametrize("a,p,m,expect", ALL_T1)
def test_table1_two_level_iterations_all(table_counts, a, p, m, expect):
    _check_count("table1", a, p, m, expect, table_counts[("table1", a, p, m)])


# ---------------------------------------------------------------------------
# F-relaxation only (the Parareal form of Sec. 2.2)
# ---------------------------------------------------------------------------


def _f_problem(nt=64, m=4, levels=2):
    g = sl.Grid(48, nt)
    ws = sl.WaveSpeed("sin_kx_cos_t", a=0.5, k=1.0)
    return mg.build_hierarchy(g, ws, 3, m, levels=levels)


def test_f_relaxation_two_level_is_exact_on_the_first_k_intervals_after_k_cycles():
    """Two-level MGRIT with F-relaxation is Parareal: after k cycles the C-points j m, j <= k, equal
    sequential stepping (and j = k + 1 does not yet)."""
    H = _f_problem()
    u0 = W.u0_bumps_1d(48, W.SEED_C2_BUMPS, 3)
    seq = mg.sequential_solve(H, u0)
    U0 = W.initial_iterate(64, 48)
    for k in (1, 2, 3):
        R = mg.mgrit_solve(H, u0, U0, max_iter=k, mode="F")
        for j in range(1, k + 1):
            assert np.max(np.abs(R.U[4 * j] - seq[4 * j])) < 1e-12
        assert np.max(np.abs(R.U[4 * (k + 1)] - seq[4 * (k + 1)])) > 1e-8


def test_f_relaxation_with_the_ideal_coarse_operator_converges_in_one_cycle():
    g = sl.Grid(48, 64)
    H = mg.build_hierarchy(g, sl.WaveSpeed("sin_kx_cos_t", a=0.5, k=1.0), 3, 4, levels=2, coarse="ideal")
    u0 = W.u0_bumps_1d(48, W.SEED_C2_BUMPS, 3)
    R = mg.mgrit_solve(H, u0, W.initial_iterate(64, 48), max_iter=1, mode="F")
    seq = mg.sequential_solve(H, u0)
    assert np.max(np.abs(R.U - seq)) < 1e-12


def test_f_and_fcf_relaxation_reach_the_same_fixed_point():
    H = _f_problem(nt=128, levels=0)
    u0 = W.u0_bumps_1d(48, W.SEED_C2_BUMPS, 3)
    U0 = W.initial_iterate(128, 48)
    a = mg.mgrit_solve(H, u0, U0, mode="F")
    b = mg.mgrit_solve(H, u0, U0, mode="FCF")
    seq = mg.sequential_solve(H, u0)
    assert a.converged and b.converged and a.iterations >= b.iterations
    assert np.linalg.norm(a.U - seq) / np.linalg.norm(seq) < 1e-9


# ---------------------------------------------------------------------------
# Stopping at discretisation accuracy (Sec. SM4)
# ---------------------------------------------------------------------------


def _cos_t_exact_final(grid, u0_fn):
    """alpha = cos(2 pi t): characteristics x(t) = x0 + sin(2 pi t) / (2 pi), so u(x, T) = u0(x - sin(2 pi T)/(2 pi))."""
    T = grid.nt * grid.dt
    x = grid.xmin + grid.h * np.arange(grid.nx)
    return u0_fn(x - np.sin(2 * np.pi * T) / (2 * np.pi))


def _sin4(x):
    return np.sin(np.pi * x) ** 4


def test_sl_discretisation_error_against_the_closed_form_flow_falls_with_order():
    """The sequential SL solution's error at T against the exact flow of alpha = cos(2 pi t) shrinks with p
    (Sec. SM4 reports the same ordering for its test problem)."""
    g = sl.Grid(128, 256)
    ws = sl.WaveSpeed("cos_t")
    u0 = _sin4(g.xmin + g.h * np.arange(g.nx))
    ref = _cos_t_exact_final(g, _sin4)
    errs = []
    for p in (1, 3, 5):
        seq = mg.sequential_solve(mg.Hierarchy(g, ws, p, []), u0)
        errs.append(float(np.sqrt(g.h * np.sum((seq[-1] - ref) ** 2))))
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10, errs


def test_stopping_at_discretisation_accuracy():
    """With u_final_ref = the exact final state and the tolerance just above the sequential solution's own
    error, MGRIT stops once u(T) is that accurate: the recorded final errors are the distances of the
    returned iterates, the last is within the tolerance and the one before is not, and (as in Sec. SM4 for
    p = 1, 3) fewer cycles are needed than for the 1e-10 residual reduction."""
    g = sl.Grid(128, 256)
    ws = sl.WaveSpeed("cos_t")
    u0 = _sin4(g.xmin + g.h * np.arange(g.nx))
    ref = _cos_t_exact_final(g, _sin4)
    for p in (1, 3):
        H = mg.build_hierarchy(g, ws, p, 4)
        seq = mg.sequential_solve(H, u0)
        disc = float(np.sqrt(g.h * np.sum((seq[-1] - ref) ** 2)))
        tol = 1.01 * disc
        U0 = W.initial_iterate(g.nt, g.nx)
        R = mg.mgrit_solve(H, u0, U0, u_final_ref=ref, final_tol=tol)
        full = mg.mgrit_solve(H, u0, U0)
        assert R.converged and R.iterations == len(R.final_errors)
        assert abs(R.final_errors[-1] - np.sqrt(g.h * np.sum((R.U[-1] - ref) ** 2))) < 1e-15
        assert R.final_errors[-1] <= tol and (R.iterations == 1 or R.final_errors[-2] > tol)
        assert R.iterations < full.iterations
