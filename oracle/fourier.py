"""Fourier symbols of the constant-wave-speed SL operators and the two-level MGRIT convergence estimate
rho(c) of Sec. 2.3 (eq. (rho_MGRIT_asym)).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For alpha = 1 and the Courant number c = dt / h every arrival node has the departure offset s = c, so
the SL step is circulant: (Phi u)_i = sum_j w_j(eps) u_{i - floor(c) + j}, j in stencil(p), and the
grid Fourier mode e^{i w k} (k the node index) is an eigenvector with the eigenvalue
lambda(w; c) = sum_j w_j(eps) e^{i w (j - floor(c))}.  The coarse operators act on the same modes:
the rediscretised step over m dt has the symbol lambda(w; m c); the corrected operator of Sec. 3
(two levels, constant sigma = phi) has mu = lambda(w; m c) / (1 - sigma d(w)), where
d(w) = (-4 sin^2(w/2))^{(p+1)/2} is the symbol of D_{p+1}.

Reading: at w = 0 both operators keep the constant mode exactly (lambda = mu = 1), so the quotient of
eq. (rho_MGRIT_asym) is 0/0 there; such frequencies contribute 0 to the maximum.  (For p = 5 the
numerator and denominator also reach rounding level at the sampled frequencies next to 0, where the
quotient is then not reliable; the paper evaluates rho for p = 1, 3.)
"""

from __future__ import annotations

import numpy as np

from . import coarse
from . import semi_lagrangian as sl


def sl_symbol(omega: np.ndarray, c: float, p: int) -> np.ndarray:
    """lambda(w; c) of the SL step with constant offset c (Sec. 2.1 with alpha = 1)."""
    fl, eps = sl.decompose(np.array([float(c)]))
    w = sl.lagrange_weights(eps, p)[0]
    j = sl.stencil(p) - fl[0]
    return np.sum(w[None, :] * np.exp(1j * np.outer(np.asarray(omega, dtype=np.float64), j)), axis=1)


def d_symbol(omega: np.ndarray, p: int) -> np.ndarray:
    """Symbol of D_{p+1} = (delta^2)^{(p+1)/2}: (-4 sin^2(w/2))^{(p+1)/2}."""
    return (-4.0 * np.sin(np.asarray(omega, dtype=np.float64) / 2) ** 2) ** ((p + 1) // 2)


def coarse_symbol(omega: np.ndarray, c: float, p: int, m: int, kind: str) -> np.ndarray:
    """mu(w; c) of the coarse operator: "sl" the rediscretised step over m dt (Sec. 2.3), "corrected"
    Psi = M^{-1} S with sigma = phi (eq. (varphi_p_def), two levels, constant alpha), "ideal" Phi^m."""
    lam_m = sl_symbol(omega, m * c, p)
    if kind == "sl":
        return lam_m
    if kind == "ideal":
        return sl_symbol(omega, c, p) ** m
    if kind == "corrected":
        sig = float(coarse.phi(np.array([[m * c]]), np.full((m, 1), float(c)), m, p)[0, 0])
        return lam_m / (1.0 - sig * d_symbol(omega, p))
    raise ValueError(kind)


def rho(c: float, p: int, m: int, kind: str = "sl", npts: int = 512, offset: float = 0.0) -> float:
    """Eq. (rho_MGRIT_asym): max over npts equispaced w in [-pi, pi) of |lambda|^m |lambda^m - mu| / (1 - |mu|)
    (the paper's sampling w_k = -pi + 2 pi k / npts; offset shifts it to w_k = -pi + 2 pi (k + offset) / npts)."""
    omega = -np.pi + 2.0 * np.pi * (np.arange(npts) + offset) / npts
    lam = sl_symbol(omega, c, p)
    mu = coarse_symbol(omega, c, p, m, kind)
    num = np.abs(lam) ** m * np.abs(lam ** m - mu)
    den = 1.0 - np.abs(mu)
    zero = (num < 1e-14) & (np.abs(den) < 1e-14)
    with np.errstate(divide="ignore"):
        q = np.where(zero, 0.0, num / np.where(zero, 1.0, den))
    return float(np.max(q))
