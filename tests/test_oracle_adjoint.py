"""Pins for the oracle's discrete adjoint: transposition identities against explicit matrices, the
tangent-linear ERK and weight derivatives against finite differences, and the gradients against
central finite differences of the sequential forward solve (FP64, step 1e-6)."""

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as adj
from oracle import coarse as co
from oracle import mgrit as mg
from oracle import semi_lagrangian as sl


def problem(nx=32, nt=32, p=3, a=0.5, kind="sin_kx_cos_t", m=4):
    g = sl.Grid(nx, nt)
    ws = sl.WaveSpeed(kind, a=a, k=1.0)
    return g, ws, mg.build_hierarchy(g, ws, p, m)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_transposed_gather_is_the_matrix_transpose(p):
    g, ws, H = problem(p=p)
    rng = np.random.default_rng(1)
    v = rng.standard_normal(g.nx)
    for l in range(H.nlevels):
        for n in (0, H.levels[l].nt - 1):
            s = H.levels[l].s[n]
            assert np.allclose(adj.sl_transpose_apply_1d(v, s, p), sl.sl_matrix_1d(s, p).T @ v, atol=1e-13)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_transposed_coarse_operator_dot_product(p):
    """<Psi u, v> = <u, Psi^T v> for the corrected coarse operators of every level."""
    g, ws, H = problem(p=p)
    R = adj.ReversedTransposed(H)
    rng = np.random.default_rng(2)
    for l in range(H.nlevels):
        for n in range(H.levels[l].nt):
            u, v = rng.standard_normal(g.nx), rng.standard_normal(g.nx)
            lhs = H.step(l, n, u) @ v
            rhs = u @ R.step_T(l, n, v)
            assert abs(lhs - rhs) < 1e-12 * (1 + abs(lhs))


def test_transposed_correction_solve_against_dense():
    g, ws, H = problem(p=5)
    sig = H.levels[1].sigma[0]
    M = co.correction_matrix_1d(sig, 5).toarray()
    v = np.random.default_rng(3).standard_normal(g.nx)
    x = adj.TransposedSolver(co.correction_matrix_1d(sig, 5)).solve(v)
    assert np.allclose(M.T @ x, v, atol=1e-12)


@pytest.mark.parametrize("r", [1, 3, 5])
def test_tangent_linear_departure_matches_finite_differences(r):
    g = sl.Grid(64, 16)
    for kind, a in (("sin_kx_cos_t", 0.5), ("const", 0.8)):
        ds = adj.departure_offsets_da_1d(g, sl.WaveSpeed(kind, a=a, k=2.0), 5, r)
        d = 1e-6
        fd = (sl.departure_offsets_1d(g, sl.WaveSpeed(kind, a=a + d, k=2.0), 5, r)
              - sl.departure_offsets_1d(g, sl.WaveSpeed(kind, a=a - d, k=2.0), 5, r)) / (2 * d)
        assert np.allclose(ds, fd, rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_weight_derivative_matches_finite_differences(p):
    eps = np.linspace(0.01, 0.99, 23)
    d = 1e-6
    fd = (sl.lagrange_weights(eps + d, p) - sl.lagrange_weights(eps - d, p)) / (2 * d)
    assert np.allclose(adj.lagrange_weights_deps(eps, p), fd, atol=1e-8)


@pytest.mark.parametrize("p", [1, 3])
def test_gradients_match_central_finite_differences(p):
    g = sl.Grid(32, 48)
    a0 = 0.5
    u0 = W.u0_bumps_1d(32, W.SEED_C5_BUMPS, 3)
    ut = W.u0_bumps_1d(32, W.SEED_C5_TARGET, 3)
    gu, ga = adj.gradients(g, sl.WaveSpeed("sin_kx_cos_t", a=a0, k=1.0), p, u0, ut)
    h = 1e-6
    J = lambda a, u: adj.objective(g, sl.WaveSpeed("sin_kx_cos_t", a=a, k=1.0), p, u, ut)  # noqa: E731
    fda = (J(a0 + h, u0) - J(a0 - h, u0)) / (2 * h)
    assert abs(ga - fda) <= 1e-6 * abs(fda)
    rng = np.random.default_rng(4)
    for _ in range(4):
        d = rng.standard_normal(32)
        fdu = (J(a0, u0 + h * d) - J(a0, u0 - h * d)) / (2 * h)
        assert abs(gu @ d - fdu) <= 1e-6 * max(abs(fdu), 1e-3)


def test_adjoint_mgrit_fixed_point_is_the_sequential_adjoint():
    g, ws, H = problem(nx=48, nt=64, p=3, m=4)
    lam_T = np.random.default_rng(5).standard_normal(48)
    seq = adj.adjoint_sequential(H, lam_T)
    lam, res = adj.adjoint_mgrit(H, lam_T, W.initial_iterate(64, 48))
    assert res.converged and np.linalg.norm(lam - seq) / np.linalg.norm(seq) < 1e-9


# ---------------------------------------------------------------------------
# 2D (Sec. 4.1 tensor-product step; the adjoint of the paper's 2D coarse operator)
# ---------------------------------------------------------------------------


def problem_2d(nx=8, nt=16, p=3, a=0.5, kind="sin_cos2", m=4, solve_mode="exact"):
    g = sl.Grid(nx, nt, dim=2)
    ws = sl.WaveSpeed(kind, a=a, a2=a)
    return g, ws, mg.build_hierarchy(g, ws, p, m, solve_mode=solve_mode)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_transposed_gather_2d_is_the_matrix_transpose(p):
    g, ws, H = problem_2d(nx=12, p=p)
    v = np.random.default_rng(11).standard_normal((12, 12))
    for l in range(H.nlevels):
        for n in (0, H.levels[l].nt - 1):
            sx, sy = H.levels[l].s[0][n], H.levels[l].s[1][n]
            ref = (sl.sl_matrix_2d(sx, sy, p).T @ v.ravel()).reshape(12, 12)
            assert np.allclose(adj.sl_transpose_apply_2d(v, sx, sy, p), ref, atol=1e-13)


@pytest.mark.parametrize("kind", ["sin_cos2", "paper2"])
def test_transposed_coarse_operator_dot_product_2d(kind):
    g, ws, H = problem_2d(kind=kind, a=0.5 if kind == "sin_cos2" else 1.0)
    R = adj.ReversedTransposed(H)
    rng = np.random.default_rng(12)
    for l in range(H.nlevels):
        for n in range(H.levels[l].nt):
            u, v = rng.standard_normal((8, 8)), rng.standard_normal((8, 8))
            lhs = float(np.sum(H.step(l, n, u) * v))
            rhs = float(np.sum(u * R.step_T(l, n, v)))
            assert abs(lhs - rhs) < 1e-12 * (1 + abs(lhs))


def test_transposed_gmres_solve_2d_meets_its_stopping_rule():
    g, ws, H = problem_2d(solve_mode="gmres")
    sx, sy = H.levels[1].sigma[0][0], H.levels[1].sigma[1][0]
    M = co.correction_matrix_2d(sx, sy, 3)
    v = np.random.default_rng(13).standard_normal(64)
    x = adj.TransposedSolver(M, "gmres", 1e-2, 10).solve(v)
    assert np.linalg.norm(M.T @ x - v) <= 1e-2 * np.linalg.norm(v) * (1 + 1e-12)


@pytest.mark.parametrize("r", [1, 3, 5])
@pytest.mark.parametrize("kind", ["sin_cos2", "const2"])
def test_tangent_linear_departure_2d_matches_finite_differences(r, kind):
    g = sl.Grid(16, 8, dim=2)
    a, d = 0.5, 1e-6
    dsx, dsy = adj.departure_offsets_da_2d(g, sl.WaveSpeed(kind, a=a, a2=0.7), 5, r)
    px, py = sl.departure_offsets_2d(g, sl.WaveSpeed(kind, a=a + d, a2=0.7), 5, r)
    mx, my = sl.departure_offsets_2d(g, sl.WaveSpeed(kind, a=a - d, a2=0.7), 5, r)
    assert np.allclose(dsx, (px - mx) / (2 * d), rtol=1e-7, atol=1e-9)
    assert np.allclose(dsy, (py - my) / (2 * d), rtol=1e-7, atol=1e-9)
    assert np.max(np.abs(dsx)) > 1e-3  # the parameter acts on the x speed in both families


@pytest.mark.parametrize("p", [1, 3, 5])
def test_dphi_da_1d_is_the_directional_derivative_of_the_step(p):
    """(dPhi/da) u equals the central difference of sl_apply_1d along ds away from floor switches."""
    rng = np.random.default_rng(13)
    nx = 24
    s = rng.uniform(0.2, 0.8, nx) + rng.integers(-3, 4, nx)
    ds, u = rng.standard_normal(nx), rng.standard_normal(nx)
    d = 1e-6
    fd = (sl.sl_apply_1d(u, s + d * ds, p) - sl.sl_apply_1d(u, s - d * ds, p)) / (2 * d)
    got = adj.dphi_da_apply_1d(u, s, ds, p)
    assert np.allclose(got, fd, atol=1e-7)
    assert np.max(np.abs(got)) > 1e-2


@pytest.mark.parametrize("p", [1, 3, 5])
def test_dphi_da_2d_is_the_directional_derivative_of_the_step(p):
    """(dPhi/da) u equals the central difference of sl_apply_2d along (dsx, dsy) away from floor switches."""
    rng = np.random.default_rng(14)
    nx = 12
    sx = rng.uniform(0.2, 0.8, (nx, nx)) + rng.integers(-2, 3, (nx, nx))
    sy = rng.uniform(0.2, 0.8, (nx, nx)) + rng.integers(-2, 3, (nx, nx))
    dsx, dsy, u = rng.standard_normal((nx, nx)), rng.standard_normal((nx, nx)), rng.standard_normal((nx, nx))
    d = 1e-6
    fd = (sl.sl_apply_2d(u, sx + d * dsx, sy + d * dsy, p) - sl.sl_apply_2d(u, sx - d * dsx, sy - d * dsy, p)) / (2 * d)
    assert np.allclose(adj.dphi_da_apply_2d(u, sx, sy, dsx, dsy, p), fd, atol=1e-7)


@pytest.mark.parametrize("p", [1, 3])
def test_gradients_2d_match_central_finite_differences(p):
    g = sl.Grid(16, 16, dim=2)
    a0 = 0.5
    u0 = W.u0_bumps_2d(16, W.SEED_C5_BUMPS, 5)
    ut = W.u0_bumps_2d(16, W.SEED_C5_TARGET, 5)
    gu, ga = adj.gradients(g, sl.WaveSpeed("sin_cos2", a=a0), p, u0, ut)
    h = 1e-6
    J = lambda a, u: adj.objective(g, sl.WaveSpeed("sin_cos2", a=a), p, u, ut)  # noqa: E731
    fda = (J(a0 + h, u0) - J(a0 - h, u0)) / (2 * h)
    assert abs(ga - fda) <= 1e-6 * abs(fda)
    rng = np.random.default_rng(15)
    for _ in range(4):
        d = rng.standard_normal((16, 16))
        fdu = (J(a0, u0 + h * d) - J(a0, u0 - h * d)) / (2 * h)
        assert abs(float(np.sum(gu * d)) - fdu) <= 1e-6 * max(abs(fdu), 1e-3)


@pytest.mark.parametrize("solve_mode", ["exact", "gmres"])
def test_adjoint_mgrit_2d_fixed_point_is_the_sequential_adjoint(solve_mode):
    g, ws, H = problem_2d(nx=8, nt=32, p=3, m=4, solve_mode=solve_mode)
    lam_T = np.random.default_rng(16).standard_normal((8, 8))
    seq = adj.adjoint_sequential(H, lam_T)
    lam, res = adj.adjoint_mgrit(H, lam_T, W.initial_iterate(32, 64).reshape(33, 8, 8))
    assert res.converged and np.linalg.norm(lam - seq) / np.linalg.norm(seq) < 1e-9
