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
