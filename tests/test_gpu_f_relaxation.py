"""F-relaxation only (relax = 1, the Parareal form of Sec. 2.2) on the GPU against the oracle's mode "F":
multilevel 1D solves in FP64 and FP32 bulk, a 2D solve, and Parareal's exactness on the first k coarse
intervals after k two-level cycles."""

import numpy as np
import pytest

import workloads as W
from oracle import mgrit as omg
from oracle import semi_lagrangian as osl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2203_13382_gb300 as mg  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("p", [1, 3, 5])
@pytest.mark.parametrize("levels", [2, 0])
def test_f_relaxation_fp64_matches_the_oracle(p, levels):
    nx, nt, m = 128, 256, 4
    ws = osl.WaveSpeed("sin_kx_cos_t", a=0.5, k=1.0)
    H = omg.build_hierarchy(osl.Grid(nx, nt), ws, p, m, levels=levels)
    u0 = W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
    U0 = W.initial_iterate(nt, nx)
    ref = omg.mgrit_solve(H, u0, U0, mode="F")
    assert ref.converged
    h = mg.mgrit_setup(nx, nt, p, m, wave="sin_kx_cos_t", a=0.5, k=1.0, levels=levels, relax=1)
    out, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda())
    assert st["iterations"] == ref.iterations
    assert rel(out.cpu().numpy(), ref.U) < 1e-12
    hist = np.asarray(st["history"])
    assert np.allclose(hist, ref.history[: len(hist)], rtol=1e-8, atol=1e-13 * ref.history[0])


@pytest.mark.parametrize("p", [1, 3, 5])
def test_f_relaxation_fp32_bulk_matches_the_oracle(p):
    nx, nt, m = 256, 512, 4
    ws = osl.WaveSpeed("sin_kx_cos_t", a=0.5, k=1.0)
    H = omg.build_hierarchy(osl.Grid(nx, nt), ws, p, m)
    u0 = W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
    U0 = W.initial_iterate(nt, nx)
    ref = omg.mgrit_solve(H, u0, U0, mode="F")
    h = mg.mgrit_setup(nx, nt, p, m, wave="sin_kx_cos_t", a=0.5, k=1.0, precision=1, relax=1)
    out, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda())
    # the FP32 error cycle changes the per-cycle reduction slightly; the stopping test is in FP64
    assert st["converged"] and abs(st["iterations"] - ref.iterations) <= 1
    assert rel(out.cpu().numpy(), ref.U) < 1e-7


@pytest.mark.parametrize("precision", [0, 1])
def test_parareal_exact_on_the_first_k_intervals(precision):
    """Two levels, F-relaxation: after k cycles the C-points j m, j <= k, are the sequential solution (FP32
    bulk: up to the FP32 rounding of the last correction), and C-point (k + 1) m is not yet."""
    nx, nt, p, m = 256, 256, 3, 8
    ws = osl.WaveSpeed("sin_kx_cos_t", a=0.6, k=2.0)
    u0 = W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
    U0 = W.initial_iterate(nt, nx)
    seq = omg.sequential_solve(omg.Hierarchy(osl.Grid(nx, nt), ws, p, []), u0)
    for k in (1, 2, 5):
        # k cycles exactly: max_iter = k with a tolerance out of reach
        h = mg.mgrit_setup(nx, nt, p, m, wave="sin_kx_cos_t", a=0.6, k=2.0, levels=2, precision=precision,
                           relax=1, max_iter=k, rtol=1e-300)
        out, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda(), allow_not_converged=True)
        assert st["iterations"] == k
        got = out.cpu().numpy()
        scale = np.max(np.abs(seq))
        tol = 1e-12 if precision == 0 else 1e-6
        for j in range(1, k + 1):
            assert np.max(np.abs(got[j * m] - seq[j * m])) < tol * scale, (k, j)
        assert np.max(np.abs(got[(k + 1) * m] - seq[(k + 1) * m])) > 1e-4 * scale


def test_f_relaxation_2d_matches_the_oracle():
    nx, nt, p, m = 32, 32, 3, 4
    g = osl.Grid(nx, nt, dim=2)
    ws = osl.WaveSpeed("paper2", a=1.0, a2=1.0)
    H = omg.build_hierarchy(g, ws, p, m, levels=0, solve_mode="gmres", gmres_rtol=1e-2, gmres_maxit=10)
    u0 = W.u0_bumps_2d(nx, W.SEED_C3_BUMPS, 5)
    U0 = W.initial_iterate(nt, nx * nx)
    ref = omg.mgrit_solve(H, u0, U0.reshape(nt + 1, nx, nx), mode="F")
    h = mg.mgrit_setup(nx, nt, p, m, wave="paper2", a=1.0, a2=1.0, dim=2, relax=1)
    out, st = h.solve(torch.from_numpy(u0.ravel().copy()).cuda(), torch.from_numpy(U0).cuda())
    assert st["converged"] and st["iterations"] == ref.iterations
    assert rel(out.cpu().numpy(), ref.U.reshape(nt + 1, -1)) < 1e-9


def test_batched_solves_reject_f_relaxation():
    with pytest.raises(mg.MgritError):
        mg.mgrit_setup_batched([dict(nx=64, nt=64, order=3, m=4)], precision=1, relax=1)
