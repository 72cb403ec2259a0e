"""Edge cases of the GPU path against the oracle: the smallest grid (nx = 16: one 16-row partition of the
FP32 correction solve, no reduction levels), a time axis that is not a multiple of the departure kernel's
step block (nt = 100, two levels of 100 / 25 steps), the integer-Courant case (exact shifts, sigma = 0,
exact coarse operator), and argument errors."""

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
@pytest.mark.parametrize("precision", [0, 1])
def test_smallest_grid(p, precision):
    nx, nt, m = 16, 64, 4
    H = omg.build_hierarchy(osl.Grid(nx, nt), osl.WaveSpeed("sin_kx_cos_t", a=0.5, k=1.0), p, m)
    u0 = W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
    U0 = W.initial_iterate(nt, nx)
    ref = omg.mgrit_solve(H, u0, U0)
    h = mg.mgrit_setup(nx, nt, p, m, wave="sin_kx_cos_t", a=0.5, k=1.0, precision=precision)
    out, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda())
    assert st["iterations"] == ref.iterations
    assert rel(out.cpu().numpy(), ref.U) < (1e-12 if precision == 0 else 1e-5)


@pytest.mark.parametrize("precision", [0, 1])
def test_ragged_time_axis(precision):
    nx, nt, p, m = 256, 100, 3, 4
    H = omg.build_hierarchy(osl.Grid(nx, nt), osl.WaveSpeed("sin_kx_cos_t", a=0.6, k=2.0), p, m)
    assert [lv.nt for lv in H.levels] == [100, 25]
    u0 = W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
    U0 = W.initial_iterate(nt, nx)
    ref = omg.mgrit_solve(H, u0, U0)
    h = mg.mgrit_setup(nx, nt, p, m, wave="sin_kx_cos_t", a=0.6, k=2.0, precision=precision)
    assert h.nlevels == 2 and h.level_info(1)[0] == 25
    out, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda())
    assert st["iterations"] == ref.iterations
    assert rel(out.cpu().numpy(), ref.U) < (1e-12 if precision == 0 else 1e-5)
    seq = omg.sequential_solve(omg.Hierarchy(osl.Grid(nx, nt), osl.WaveSpeed("sin_kx_cos_t", a=0.6, k=2.0), p, []), u0)
    got = h.sequential(torch.from_numpy(u0).cuda()).cpu().numpy()
    assert rel(got, seq) < (1e-12 if precision == 0 else 1e-5)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_integer_courant_number(p):
    """alpha = 1 with dt = h: every departure point is a grid node, phi = sigma = 0, the coarse operator
    equals Phi^m, and MGRIT converges as fast as the oracle (one cycle to the exact solution)."""
    nx, nt, m = 128, 64, 4
    H = omg.build_hierarchy(osl.Grid(nx, nt, cfl=1.0), osl.WaveSpeed("const", a=1.0), p, m)
    u0 = W.u0_sin4(nx)
    U0 = W.initial_iterate(nt, nx)
    ref = omg.mgrit_solve(H, u0, U0)
    h = mg.mgrit_setup(nx, nt, p, m, wave="const", a=1.0, cfl=1.0)
    for l in range(1, h.nlevels):
        assert np.max(np.abs(h.sigma(l).cpu().numpy())) < 1e-12
    out, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda())
    assert st["iterations"] == ref.iterations
    exact = np.stack([np.roll(u0, n) for n in range(nt + 1)])
    assert rel(out.cpu().numpy(), exact) < 1e-12


def test_argument_errors():
    with pytest.raises(mg.MgritError):
        mg.mgrit_setup(24, 64, 3, 4)        # nx not a power of two
    with pytest.raises(mg.MgritError):
        mg.mgrit_setup(8, 64, 3, 4)         # nx below 16
    with pytest.raises(mg.MgritError):
        mg.mgrit_setup(8192, 64, 3, 4)      # 1D slices larger than shared memory holds
    with pytest.raises(mg.MgritError):
        mg.mgrit_setup(64, 1, 3, 4)         # fewer than two steps
    with pytest.raises(mg.MgritError):
        mg.mgrit_setup(64, 64, 2, 4)        # even order
    with pytest.raises(mg.MgritError):
        mg.mgrit_setup(64, 63, 3, 4, levels=2)  # nt not divisible by m for the requested levels


@pytest.mark.parametrize("p", [1, 3, 5])
@pytest.mark.parametrize("precision", [0, 1])
def test_variable_coarsening_first_level(p, precision):
    """Sec. 5's coarsening: factor 16 on the first level, 4 below (option m_first)."""
    nx, nt = 128, 1024
    H = omg.build_hierarchy(osl.Grid(nx, nt), osl.WaveSpeed("sin_kx_cos_t", a=0.4, k=1.0), p, [16, 4])
    u0 = W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
    U0 = W.initial_iterate(nt, nx)
    ref = omg.mgrit_solve(H, u0, U0)
    h = mg.mgrit_setup(nx, nt, p, 4, wave="sin_kx_cos_t", a=0.4, k=1.0, m_first=16, precision=precision)
    assert [h.level_info(l)[0] for l in range(h.nlevels)] == [lv.nt for lv in H.levels]
    out, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda())
    assert st["iterations"] == ref.iterations
    assert rel(out.cpu().numpy(), ref.U) < (1e-12 if precision == 0 else 1e-5)


def test_rediscretised_coarse_operator():
    """coarse_op = 1: the plain coarse SL step (no correction), as the oracle's coarse = "sl"."""
    nx, nt, p, m = 64, 256, 3, 4
    H = omg.build_hierarchy(osl.Grid(nx, nt, cfl=1.0), osl.WaveSpeed("const", a=1.0), p, m, coarse="sl")
    u0 = W.u0_sin4(nx)
    U0 = W.initial_iterate(nt, nx)
    ref = omg.mgrit_solve(H, u0, U0)
    h = mg.mgrit_setup(nx, nt, p, m, wave="const", a=1.0, cfl=1.0, coarse_op=1)
    out, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda())
    assert st["iterations"] == ref.iterations
    assert rel(out.cpu().numpy(), ref.U) < 1e-12
