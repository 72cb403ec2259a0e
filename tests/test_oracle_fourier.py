"""Pins of oracle/fourier.py (Sec. 2.3): the symbols are the eigenvalues of the oracle's own SL step and
corrected coarse operator on grid Fourier modes, rho has the symmetries the paper states for odd p, the
ideal coarse operator gives rho = 0, and measured two-level convergence factors follow rho."""

import numpy as np
import pytest

import workloads as W
from oracle import fourier as F
from oracle import mgrit as mg
from oracle import semi_lagrangian as sl


def modes(nx):
    k = np.array([1, 5, 17, nx // 4 + 3, nx // 2 - 1])
    return 2 * np.pi * k / nx


@pytest.mark.parametrize("p", [1, 3, 5])
@pytest.mark.parametrize("c", [0.3, 0.85, 1.7, 2.25])
def test_sl_symbol_is_the_eigenvalue_of_the_oracle_step(p, c):
    nx = 64
    idx = np.arange(nx)
    for w in modes(nx):
        v = np.exp(1j * w * idx)
        out = sl.sl_apply_1d(v.real, np.full(nx, c), p) + 1j * sl.sl_apply_1d(v.imag, np.full(nx, c), p)
        lam = F.sl_symbol(np.array([w]), c, p)[0]
        assert np.max(np.abs(out - lam * v)) < 1e-13


@pytest.mark.parametrize("p", [1, 3, 5])
@pytest.mark.parametrize("c", [0.55, 0.85])
def test_corrected_symbol_is_the_eigenvalue_of_the_oracle_coarse_operator(p, c):
    nx, nt, m = 64, 16, 4
    H = mg.build_hierarchy(sl.Grid(nx, nt, cfl=c), sl.WaveSpeed("const", a=1.0), p, m, levels=2)
    idx = np.arange(nx)
    for w in modes(nx):
        v = np.exp(1j * w * idx)
        out = H.step(1, 0, v.real) + 1j * H.step(1, 0, v.imag)
        mu = F.coarse_symbol(np.array([w]), c, p, m, "corrected")[0]
        assert np.max(np.abs(out - mu * v)) < 1e-11


@pytest.mark.parametrize("p", [1, 3])
def test_rho_symmetries_for_odd_p(p):
    """Sec. 2.3: for odd p, rho on [0, 0.5] mirrors rho on [0.5, 1] about c = 0.5, and rho is 1-periodic in c.
    The mirror maps w to -w, so it is exact on a frequency sampling symmetric about 0 (offset 1/2).  (p = 1, 3
    as in Fig. 2: for p = 5 both terms of the quotient fall below rounding level at the frequencies next to 0.)"""
    for kind in ("sl", "corrected"):
        for d in (0.05, 0.17, 0.31, 0.44):
            for m in (2, 4, 8):
                a, b = F.rho(0.5 - d, p, m, kind, offset=0.5), F.rho(0.5 + d, p, m, kind, offset=0.5)
                assert abs(a - b) <= 1e-9 * max(1.0, abs(a)), (kind, d, m)
                assert abs(F.rho(1.5 + d, p, m, kind) - F.rho(0.5 + d, p, m, kind)) <= 1e-9 * max(1.0, abs(b))


def test_rho_of_the_ideal_coarse_operator_is_zero():
    for p in (1, 3, 5):
        assert F.rho(0.63, p, 4, "ideal") < 1e-14


@pytest.mark.parametrize("p", [1, 3])
@pytest.mark.parametrize("c", [0.55, 0.65, 0.95])
def test_measured_two_level_factor_follows_rho(p, c):
    """Two-level MGRIT, alpha = 1: with the corrected operator the final-iteration factor is within
    [0.75, 1.05] rho; with the rediscretised one the residual grows where rho > 2 and falls where rho < 0.5
    (Fig. 2's reading of rho as a convergence estimate)."""
    nx, nt, m = 128, 2048, 4
    g = sl.Grid(nx, nt, cfl=c)
    for coarse in ("corrected", "sl"):
        H = mg.build_hierarchy(g, sl.WaveSpeed("const", a=1.0), p, m, levels=2, coarse=coarse)
        R = mg.mgrit_solve(H, W.u0_sin4(nx), W.initial_iterate(nt, nx), max_iter=8, rtol=1e-300)
        f = R.history[-1] / R.history[-2]
        r = F.rho(c, p, m, coarse)
        if coarse == "corrected":
            assert 0.75 * r <= f <= 1.05 * r, (f, r)
        elif r > 2:
            assert f > 1.0, (f, r)
        elif r < 0.5:
            assert f < 1.0, (f, r)
