"""Pins for D_{p+1}, f_{p+1}, backtracking, phi/sigma and the corrected operator (oracle)."""

import math

import numpy as np
import pytest

from oracle import coarse as co
from oracle import semi_lagrangian as sl

from closed_forms import exact_flow_cos_t_cos_x


@pytest.mark.parametrize("p", [1, 3, 5])
def test_D_fourier_symbol(p):
    """D_{p+1} is circulant with symbol (-4 sin^2(w/2))^{(p+1)/2} (Sec. 3: periodic, second order)."""
    nx = 32
    D = co.D_matrix(nx, p).toarray()
    i = np.arange(nx)
    for kk in range(nx):
        w = 2.0 * math.pi * kk / nx
        mode = np.exp(1j * w * i)
        lam = (-4.0 * math.sin(w / 2.0) ** 2) ** ((p + 1) // 2)
        assert np.allclose(D @ mode, lam * mode, atol=1e-10)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_D_is_second_order(p):
    """h^{-(p+1)} D_{p+1} v = v^{(p+1)} + O(h^2) on a smooth periodic v (eq. (Dp+1_def), s = 2)."""
    errs = []
    for nx in (64, 128, 256):
        h = 2.0 / nx
        x = -1.0 + h * np.arange(nx)
        v = np.sin(math.pi * x)
        d = co.D_matrix(nx, p) @ v / h ** (p + 1)
        exact = (-1.0) ** ((p + 1) // 2) * math.pi ** (p + 1) * np.sin(math.pi * x)
        errs.append(np.max(np.abs(d - exact)))
    assert math.log(errs[1] / errs[2], 2) > 1.8


@pytest.mark.parametrize("p", [1, 3, 5])
def test_f_is_the_interpolation_error_of_the_node_polynomial(p):
    """v(z) = z^{p+1}: v(-eps) - sum_j w_j v(j) = (-1)^{p+1} (p+1)! f_{p+1}(eps) (proof of Lemma 3.1)."""
    eps = np.linspace(0.0, 1.0, 41)
    w = sl.lagrange_weights(eps, p)
    nodes = sl.stencil(p).astype(np.float64)
    err = (-eps) ** (p + 1) - w @ nodes ** (p + 1)
    assert np.allclose(err, (-1.0) ** (p + 1) * math.factorial(p + 1) * co.f_poly(eps, p), atol=1e-11)
    assert abs(co.f_poly(np.array(0.0), p)) < 1e-15 and abs(co.f_poly(np.array(1.0), p)) < 1e-15


def test_backtracking_equals_fine_steps_for_time_dependent_alpha():
    """For alpha = alpha(t) backtracking reproduces m fine ERK steps exactly (Sec. 3.3.1, footnote)."""
    g = sl.Grid(64, 32)
    ws = sl.WaveSpeed("cos_t")
    for r in (1, 3):
        s = np.stack([sl.departure_offsets_1d(g, ws, n, r) for n in range(g.nt)])
        for m in (2, 4, 8):
            c = co.backtrack_1d(s, m)
            ref = s.reshape(g.nt // m, m, g.nx).sum(axis=1)
            assert np.allclose(c, ref, atol=1e-12)


def test_backtracking_2d_equals_fine_steps_for_uniform_velocity():
    g = sl.Grid(16, 8, dim=2, cfl=0.7)
    ws = sl.WaveSpeed("const2", a=0.8, a2=-1.3)
    pairs = [sl.departure_offsets_2d(g, ws, n, 3) for n in range(g.nt)]
    sx = np.stack([a for a, _ in pairs])
    sy = np.stack([b for _, b in pairs])
    cx, cy = co.backtrack_2d(sx, sy, 4)
    assert np.allclose(cx, 4 * 0.8 * 0.7, atol=1e-12) and np.allclose(cy, 4 * -1.3 * 0.7, atol=1e-12)


def test_backtracking_1d_is_exact_for_affine_fine_maps():
    """Eq. (coarse_depart_interp) interpolates linearly between the fine characteristics through the east
    and west nodes, so affine fine offset fields (a different one per fine step) are followed exactly:
    the coarse departure point is the composition of the m fine departure maps (nodes away from the
    periodic seam)."""
    nx, m = 128, 8
    rng = np.random.default_rng(22)
    a = rng.uniform(0.3, 2.7, m)
    b = rng.uniform(-0.01, 0.01, m)
    X0 = np.arange(nx, dtype=np.float64)
    s = np.stack([a[k] + b[k] * X0 for k in range(m)])
    c = co.backtrack_1d(s, m)[0]
    X = X0.copy()
    for k in range(m - 1, -1, -1):
        X = X - (a[k] + b[k] * X)
    assert np.allclose(c[40:88], (X0 - X)[40:88], atol=1e-11)


def test_backtracking_2d_is_exact_for_bilinear_fine_maps():
    """Sec. SM6 fits each component bilinearly through the four fine characteristics around the current
    point, so when every fine offset field is bilinear in (x, y) the backtracked coarse departure point is
    the exact composition of the m fine departure maps.  Distinct x, y and xy coefficients per fine step
    make a swapped axis, a mixed-up corner or a reversed step order fail.  Nodes are taken away from the
    periodic seam, where a bilinear field on the torus is not bilinear."""
    nx, m = 64, 4
    rng = np.random.default_rng(21)
    coef = rng.uniform([0.6, 0.004, -0.006, 1e-4], [1.4, 0.012, 0.006, 3e-4], size=(2, m, 4))
    J, I = np.meshgrid(np.arange(nx, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")

    def field(axis, k, X, Y):
        a, b, c, e = coef[axis, k]
        return a + b * X + c * Y + e * X * Y

    sx = np.stack([field(0, k, I, J) for k in range(m)])
    sy = np.stack([-field(1, k, I, J) for k in range(m)])
    cx, cy = co.backtrack_2d(sx, sy, m)
    X, Y = I.copy(), J.copy()
    for k in range(m - 1, -1, -1):
        X, Y = X - field(0, k, X, Y), Y + field(1, k, X, Y)
    inner = (slice(20, 44), slice(20, 44))
    assert np.allclose(cx[0][inner], (I - X)[inner], atol=1e-10)
    assert np.allclose(cy[0][inner], (J - Y)[inner], atol=1e-10)


def test_backtracking_follows_a_varying_flow():
    """On eq. (alpha4) the backtracked coarse departure point tracks the exact coarse characteristic
    much better than one coarse ERK step (Sec. 3.3.1, Fig. 4)."""
    nx, m = 256, 8
    g = sl.Grid(nx, m)
    ws = sl.WaveSpeed("cos_t_cos_x")
    s = np.stack([sl.departure_offsets_1d(g, ws, n, 1) for n in range(m)])
    c = co.backtrack_1d(s, m)[0]
    exact = exact_flow_cos_t_cos_x(g.x, m * g.dt, 0.0)
    err_bt = np.max(np.abs(g.x - g.h * c - exact))
    coarse_grid = sl.Grid(nx, 1, cfl=m * g.cfl)
    one_step = sl.departure_offsets_1d(coarse_grid, ws, 0, 1)
    err_erk = np.max(np.abs(g.x - g.h * one_step - exact))
    assert err_bt < 0.2 * err_erk


def test_phi_vanishes_at_integer_courant():
    g = sl.Grid(32, 16, cfl=1.0)
    s = np.stack([sl.departure_offsets_1d(g, sl.WaveSpeed("const"), n, 1) for n in range(g.nt)])
    for p in (1, 3, 5):
        c = co.backtrack_1d(s, 4)
        assert np.max(np.abs(co.phi(c, s, 4, p))) < 1e-13


@pytest.mark.parametrize("p", [1, 3, 5])
def test_phi_constant_alpha(p):
    """Constant alpha: eps constant, phi independent of i and n (Sec. 3.2): f(frac(m c)) - m f(frac(c))."""
    cfl, m = 0.85, 4
    g = sl.Grid(32, 16, cfl=cfl)
    s = np.stack([sl.departure_offsets_1d(g, sl.WaveSpeed("const"), n, p) for n in range(g.nt)])
    c = co.backtrack_1d(s, m)
    ph = co.phi(c, s, m, p)
    expect = (-1.0) ** (p + 1) * (co.f_poly(np.array(math.fmod(m * cfl, 1.0)), p) - m * co.f_poly(np.array(cfl), p))
    assert np.allclose(ph, expect, atol=1e-13)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_backward_euler_correction_is_contractive_for_constant_alpha(p):
    """||B_{p+1}||_2 <= 1 for constant alpha (Sec. 3.2, Case 2): M = I - phi D has eigenvalues >= 1."""
    nx = 32
    for m in (2, 4, 8, 16):
        for cfl in np.linspace(0.05, 0.95, 19):
            ph = float(co.f_poly(np.array(math.fmod(m * cfl, 1.0)), p) - m * co.f_poly(np.array(cfl), p))
            M = co.correction_matrix_1d(np.full(nx, ph), p).toarray()
            assert np.linalg.norm(np.linalg.inv(M), 2) <= 1.0 + 1e-12


def test_sigma_recursion_sums_over_levels():
    """eq. (nu_p_def): sigma_1 = phi_1; sigma_2[n] = sum_k sigma_1[m n + k] + phi_2[n]."""
    rng = np.random.default_rng(5)
    ph1 = rng.standard_normal((16, 8))
    ph2 = rng.standard_normal((4, 8))
    s1 = co.sigma_next(None, ph1, 4)
    s2 = co.sigma_next(s1, ph2, 4)
    assert np.array_equal(s1, ph1)
    assert np.allclose(s2[1], ph1[4] + ph1[5] + ph1[6] + ph1[7] + ph2[1])


@pytest.mark.parametrize("p", [1, 3, 5])
def test_multilevel_sigma_telescopes_to_the_fine_level(p):
    """Eq. (nu_p_def) with eq. (varphi_p_multilevel_def) telescopes: on level l, sigma[n][i] equals
    (-1)^{p+1} (f(eps_l[n][i]) - the sum of f(eps_0[k][i]) over the fine steps k inside coarse step n),
    with no reference to the levels in between (variable alpha, uneven factors)."""
    from oracle import mgrit as mg

    H = mg.Hierarchy(sl.Grid(32, 64), sl.WaveSpeed("sin_kx_cos_t", a=0.5, k=1.0), p, [4, 2, 4])
    f0 = co.f_poly(co.eps_of(H.levels[0].s), p)
    span = 1
    for lev in H.levels[1:]:
        span *= lev.m
        fine_sum = f0.reshape(lev.nt, span, -1).sum(axis=1)
        expect = (-1.0) ** (p + 1) * (co.f_poly(co.eps_of(lev.s), p) - fine_sum)
        assert np.allclose(lev.sigma, expect, atol=1e-12)
        assert np.std(lev.sigma) > 1e-3  # sigma varies in n and i, so an index slip would show


def test_multilevel_sigma_2d_telescopes_to_the_fine_level():
    """The same telescoping for each axis of the 2D sigma (Sec. 4, eq. (BEOper_2D))."""
    from oracle import mgrit as mg

    p = 3
    H = mg.Hierarchy(sl.Grid(8, 16, dim=2), sl.WaveSpeed("sin_cos2", a=0.5, a2=0.5), p, [2, 4])
    for axis in (0, 1):
        f0 = co.f_poly(co.eps_of(H.levels[0].s[axis]), p)
        span = 1
        for lev in H.levels[1:]:
            span *= lev.m
            fine_sum = f0.reshape((lev.nt, span) + f0.shape[1:]).sum(axis=1)
            expect = co.f_poly(co.eps_of(lev.s[axis]), p) - fine_sum
            assert np.allclose(lev.sigma[axis], expect, atol=1e-12)


def test_correction_solvers():
    rng = np.random.default_rng(6)
    sig = rng.uniform(0.0, 2.0, 48)
    for p in (1, 3, 5):
        M = co.correction_matrix_1d(sig if p != 3 else -sig, p)
        v = rng.standard_normal(48)
        x = co.CorrectionSolver(M, "exact").solve(v)
        assert np.allclose(M @ x, v, atol=1e-12)
        z = co.gmres_zero_guess(M, v, 1e-13, 48)
        assert np.allclose(z, x, atol=1e-9)


def test_gmres_minimises_over_the_krylov_space():
    """GMRES from x0 = 0 returns argmin ||b - A x|| over span{b, Ab, ..., A^{k-1} b} (brute force)."""
    rng = np.random.default_rng(7)
    M = co.correction_matrix_1d(rng.uniform(0.0, 3.0, 40), 1)
    b = rng.standard_normal(40)
    for k in (1, 3, 6):
        x = co.gmres_zero_guess(M, b, 0.0, k)
        K = np.stack([np.linalg.matrix_power(M.toarray(), j) @ b for j in range(k)], axis=1)
        c, *_ = np.linalg.lstsq(M @ K, b, rcond=None)
        assert np.allclose(np.linalg.norm(b - M @ x), np.linalg.norm(b - M @ (K @ c)), rtol=1e-8)
    x = co.CorrectionSolver(M, "gmres", rtol=1e-2, maxit=10).solve(b)
    res = np.linalg.norm(M @ x - b) / np.linalg.norm(b)
    full = co.gmres_zero_guess(M, b, 0.0, 10)
    assert res <= 1e-2 or np.allclose(x, full)


def test_correction_2d_symbol():
    """Constant sigma: I - sx (I (x) D) - sy (D (x) I) has symbol 1 - sx l(wx) - sy l(wy) (eq. (BEOper_2D))."""
    nx, p = 8, 3
    M = co.correction_matrix_2d(np.full((nx, nx), -0.3), np.full((nx, nx), -0.7), p).toarray()
    I, J = np.meshgrid(np.arange(nx), np.arange(nx))
    for kx in range(nx):
        for ky in range(nx):
            wx, wy = 2 * math.pi * kx / nx, 2 * math.pi * ky / nx
            mode = np.exp(1j * (wx * I + wy * J)).ravel()
            lx = (4 * math.sin(wx / 2) ** 2) ** 2
            ly = (4 * math.sin(wy / 2) ** 2) ** 2
            assert np.allclose(M @ mode, (1 + 0.3 * lx + 0.7 * ly) * mode, atol=1e-10)
