"""The failure statuses of mgrit_solve, each made to happen without faulting the GPU.

- MGRIT_EDIVERGED: a NaN in the initial condition (the residual norm is not finite), and the rediscretised
  coarse operator of Sec. 2.3 on a problem where it lets the residual grow past diverge_ratio * r0.
- MGRIT_ENOTCONVERGED: max_iter = 2; the statistics and the last iterate are still returned and equal the
  oracle's after two cycles.
- MGRIT_ETIMEOUT: the test-only option test_wait_cycles makes the first bounded wait of every CTA of the
  staged FP32 passes run out on a barrier that nothing completes; the CTAs let their bulk copies land under
  the normal limit before they stop, and the GPU keeps working (the next solve matches the oracle).
"""

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

EDIVERGED, ENOTCONVERGED, ETIMEOUT = 5, 4, 6


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _solve_status(h, u0, U0):
    try:
        h.solve(u0, U0)
    except mg.MgritError as e:
        return e.status, str(e)
    return 0, ""


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_in_the_initial_condition_is_reported_as_divergence(precision):
    nx, nt = 128, 256
    u0 = W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
    u0[17] = np.nan
    h = mg.mgrit_setup(nx, nt, 3, 4, wave="sin_kx_cos_t", a=0.5, precision=precision)
    out, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(W.initial_iterate(nt, nx)).cuda(),
                      allow_not_converged=True)
    assert not st["converged"] and st["iterations"] == 1 and not np.isfinite(st["r_final"])
    status, msg = _solve_status(h, torch.from_numpy(u0).cuda(), None)
    assert status == EDIVERGED and "diverged" in msg
    h.destroy()


def test_rediscretised_coarse_operator_growth_is_reported_as_divergence():
    """Constant speed, c = 0.85, p = 3, m = 8, two levels: with the plain coarse SL step the residual grows
    past 1e3 r0 (the oracle's history gives the cycle), where the corrected operator converges."""
    nx, nt, p, m = 64, 4096, 3, 8
    u0 = W.u0_sin4(nx)
    U0 = W.initial_iterate(nt, nx)
    H = omg.build_hierarchy(osl.Grid(nx, nt), osl.WaveSpeed("const"), p, m, levels=2, coarse="sl")
    ref = omg.mgrit_solve(H, u0, U0, max_iter=12)
    ratio = np.array(ref.history) / ref.history[0]
    first = int(np.argmax(ratio > 1e3))
    assert ratio[first] > 1e3  # the oracle diverges within 12 cycles
    h = mg.mgrit_setup(nx, nt, p, m, wave="const", levels=2, coarse_op=1, diverge_ratio=1e3)
    _, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda(), allow_not_converged=True)
    assert not st["converged"] and st["iterations"] == first + 1
    assert np.allclose(st["history"], ref.history[: first + 1], rtol=1e-8, atol=0)
    assert _solve_status(h, torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda())[0] == EDIVERGED
    h.destroy()
    hc = mg.mgrit_setup(nx, nt, p, m, wave="const", levels=2)  # the corrected operator on the same problem
    _, st = hc.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda())
    assert st["converged"]
    hc.destroy()


@pytest.mark.parametrize("precision", [0, 1])
def test_max_iter_reached_returns_the_last_iterate(precision):
    nx, nt, p, m = 256, 512, 3, 4
    u0 = W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
    U0 = W.initial_iterate(nt, nx)
    H = omg.build_hierarchy(osl.Grid(nx, nt), osl.WaveSpeed("sin_kx_cos_t", a=0.5, k=1.0), p, m)
    ref = omg.mgrit_solve(H, u0, U0, max_iter=2)
    assert not ref.converged
    h = mg.mgrit_setup(nx, nt, p, m, wave="sin_kx_cos_t", a=0.5, k=1.0, precision=precision, max_iter=2)
    out, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda(), allow_not_converged=True)
    assert st["iterations"] == 2 and not st["converged"] and len(st["history"]) == 2
    assert st["r0"] == st["history"][0] and st["r_final"] == st["history"][1]
    assert np.allclose(st["history"], ref.history, rtol=1e-7 if precision else 1e-10, atol=0)
    assert rel(out.cpu().numpy(), ref.U) < (1e-12 if precision == 0 else 1e-5)
    status, msg = _solve_status(h, torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda())
    assert status == ENOTCONVERGED and "max_iter" in msg
    h.destroy()


def test_bounded_wait_timeout_is_reported_and_the_gpu_stays_usable():
    nx, nt, p, m = 256, 512, 3, 4
    u0 = W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
    U0 = W.initial_iterate(nt, nx)
    ut, Ut = torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda()
    h = mg.mgrit_setup(nx, nt, p, m, wave="sin_kx_cos_t", a=0.5, k=1.0, precision=1, test_wait_cycles=2000)
    for _ in range(2):  # also with the cycle's captured graph replayed
        status, msg = _solve_status(h, ut, Ut)
        assert status == ETIMEOUT and "bounded device wait" in msg
    h.destroy()
    torch.cuda.synchronize()
    H = omg.build_hierarchy(osl.Grid(nx, nt), osl.WaveSpeed("sin_kx_cos_t", a=0.5, k=1.0), p, m)
    ref = omg.mgrit_solve(H, u0, U0)
    h = mg.mgrit_setup(nx, nt, p, m, wave="sin_kx_cos_t", a=0.5, k=1.0, precision=1)
    out, st = h.solve(ut, Ut)
    assert st["iterations"] == ref.iterations and rel(out.cpu().numpy(), ref.U) < 1e-5
    h.destroy()
