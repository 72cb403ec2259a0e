"""GPU parity for the 2D path against the oracle (Sec. 4): departure offsets and sigma of every level,
single fine and coarse steps, sequential stepping and MGRIT.  Coarse correction solves use the paper's
inexact GMRES (zero guess, at most 10 iterations, relative residual 1e-2; Sec. 4.3) on both sides.

Tolerances: setup arrays, single steps and sequential stepping agree to 1e-12 (FP64, rounding order
only).  With the inexact solve the MGRIT iterates depend on rounding inside GMRES, so the converged
solutions are compared where the theory fixes them: both equal the unique fine-level solution to the
stopping tolerance (1e-9 relative), with identical iteration counts.  With exact correction solves
(solve_mode 2: restarted GMRES to 1e-14 on the GPU, sparse LU in the oracle) MGRIT is a linear iteration
again and the FP64 iterates are compared element by element (1e-12), residual histories included.
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

CASES = [
    # nx, nt, p, m, wave, a, levels
    (16, 32, 1, 4, "const2", 1.0, 0),
    (16, 32, 3, 4, "sin_cos2", 0.5, 0),
    (32, 32, 5, 4, "paper2", 1.0, 0),
    (32, 64, 3, 8, "sin_cos2", 0.5, 2),
]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def hier(nx, nt, p, m, wave, a, levels):
    g = osl.Grid(nx, nt, dim=2)
    ws = osl.WaveSpeed(wave, a=a, a2=a)
    return omg.build_hierarchy(g, ws, p, m, levels=levels, solve_mode="gmres", gmres_rtol=1e-2, gmres_maxit=10)


def gpu(nx, nt, p, m, wave, a, levels, **opt):
    return mg.mgrit_setup(nx, nt, p, m, wave=wave, a=a, a2=a, dim=2, levels=levels, **opt)


@pytest.mark.parametrize("case", CASES)
def test_setup_arrays_2d(case):
    H = hier(*case)
    h = gpu(*case)
    nx = case[0]
    assert h.nlevels == H.nlevels
    for l in range(H.nlevels):
        nt_l = H.levels[l].nt
        s = h.offsets(l).cpu().numpy().reshape(2, nt_l, nx, nx)
        for c in range(2):
            ref = H.levels[l].s[c]
            assert np.max(np.abs(s[c] - ref)) < 1e-11 * max(1.0, np.max(np.abs(ref)))
        if l > 0:
            sg = h.sigma(l).cpu().numpy().reshape(2, nt_l, nx, nx)
            for c in range(2):
                ref = H.levels[l].sigma[c]
                assert np.max(np.abs(sg[c] - ref)) < 1e-11 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("case", CASES)
def test_single_steps_2d(case):
    H = hier(*case)
    h = gpu(*case)
    nx = case[0]
    rng = np.random.default_rng(21)
    for l in range(H.nlevels):
        for n in sorted({0, H.levels[l].nt - 1}):
            x = rng.standard_normal((nx, nx))
            y = h.apply_step(l, n, torch.from_numpy(x.reshape(1, -1).copy()).cuda()).cpu().numpy()[0]
            ref = H.step(l, n, x).ravel()
            assert rel(y, ref) < (1e-12 if l == 0 else 1e-10), (l, n, rel(y, ref))


@pytest.mark.parametrize("case", CASES[:3])
def test_sequential_2d(case):
    H = hier(*case)
    h = gpu(*case)
    nx = case[0]
    u0 = W.u0_bumps_2d(nx, W.SEED_C3_BUMPS, 5)
    ref = omg.sequential_solve(H, u0).reshape(case[1] + 1, -1)
    out = h.sequential(torch.from_numpy(u0.ravel().copy()).cuda()).cpu().numpy()
    assert rel(out, ref) < 1e-12


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("precision", [0, 1])
def test_mgrit_2d(case, precision):
    H = hier(*case)
    h = gpu(*case, precision=precision)
    nx, nt = case[0], case[1]
    u0 = W.u0_bumps_2d(nx, W.SEED_C3_BUMPS, 5)
    U0 = W.initial_iterate(nt, nx * nx)
    ref = omg.mgrit_solve(H, u0, U0.reshape(nt + 1, nx, nx))
    seq = omg.sequential_solve(H, u0).reshape(nt + 1, -1)
    out, st = h.solve(torch.from_numpy(u0.ravel().copy()).cuda(), torch.from_numpy(U0).cuda())
    assert st["converged"] and st["iterations"] == ref.iterations
    tol = 1e-9 if precision == 0 else 1e-5
    assert rel(out.cpu().numpy(), seq) < tol
    assert rel(ref.U.reshape(nt + 1, -1), seq) < 1e-9


def test_graph_replay_matches_direct_launches_2d():
    case = CASES[1]
    nx, nt = case[0], case[1]
    u0 = torch.from_numpy(W.u0_bumps_2d(nx, W.SEED_C3_BUMPS, 5).ravel().copy()).cuda()
    U0 = torch.from_numpy(W.initial_iterate(nt, nx * nx)).cuda()
    outs = []
    for g in (0, 1):
        h = gpu(*case, precision=1, use_graph=g)
        out, st = h.solve(u0, U0)
        outs.append((out.cpu(), st["iterations"]))
    assert torch.equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


@pytest.mark.parametrize("case", CASES)
def test_mgrit_2d_exact_correction_solves(case):
    nx, nt, p, m, wave, a, levels = case
    H = omg.build_hierarchy(osl.Grid(nx, nt, dim=2), osl.WaveSpeed(wave, a=a, a2=a), p, m, levels=levels)
    h = gpu(*case, solve_mode=2)
    u0 = W.u0_bumps_2d(nx, W.SEED_C3_BUMPS, 5)
    U0 = W.initial_iterate(nt, nx * nx)
    ref = omg.mgrit_solve(H, u0, U0.reshape(nt + 1, nx, nx))
    out, st = h.solve(torch.from_numpy(u0.ravel().copy()).cuda(), torch.from_numpy(U0).cuda())
    assert st["converged"] and st["iterations"] == ref.iterations
    assert rel(out.cpu().numpy(), ref.U.reshape(nt + 1, -1)) < 1e-12
    assert np.allclose(st["history"], ref.history, rtol=1e-9, atol=0)
