"""Parity at the full size of the 1D benchmark workload (nx = 4096, nt = 16384, p = r = 3, m = 8 to at
most 8 coarsest steps, alpha = 1 + 0.5 sin(2 pi x) cos(2 pi t)) and of the 2D workload's fine level
(512^2, p = r = 5), on outputs the oracle computes one at a time: departure offsets, coarse offsets and
sigma of sampled rows, single steps of sampled rows on every relaxed level, and the MGRIT solution of the
benchmark's launch configuration against the oracle's sequential solution (its fixed point; MGRIT stops
at a 1e-10 residual, so the two agree to about that level, not to rounding)."""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import coarse as oc
from oracle import mgrit as omg
from oracle import semi_lagrangian as osl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2203_13382_gb300 as mg  # noqa: E402

NX, NT, P, M = 4096, 16384, 3, 8
WS = osl.WaveSpeed("sin_kx_cos_t", a=0.5, k=1.0)
GRID = osl.Grid(NX, NT)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def handle(precision):
    return mg.mgrit_setup(NX, NT, P, M, wave="sin_kx_cos_t", a=0.5, k=1.0, max_coarsest=8, precision=precision)


def fine_rows(n0, count):
    return np.stack([osl.departure_offsets_1d(GRID, WS, n, P) for n in range(n0, n0 + count)])


def coarse_row(level, n):
    """Offsets and sigma of coarse row n on `level` by the oracle's backtracking from the fine rows below."""
    if level == 0:
        return fine_rows(n, 1)[0], None
    rows = [coarse_row(level - 1, M * n + k) for k in range(M)]
    s_prev = np.stack([r[0] for r in rows])
    s = oc.backtrack_1d(s_prev, M)
    ph = oc.phi(s, s_prev, M, P)
    sig_prev = None if level == 1 else np.stack([r[1] for r in rows])
    return s[0], oc.sigma_next(sig_prev, ph, M)[0]


@pytest.fixture(scope="module")
def h64():
    h = handle(0)
    yield h
    h.destroy()


def test_level_structure(h64):
    assert [h64.level_info(l)[0] for l in range(h64.nlevels)] == [16384, 2048, 256, 32, 4]


@pytest.mark.parametrize("level,rows", [(0, [0, 777, 16383]), (1, [0, 1023, 2047]), (2, [5, 255]), (3, [31])])
def test_offsets_and_sigma_of_sampled_rows(h64, level, rows):
    s_all = h64.offsets(level)
    sg_all = h64.sigma(level) if level > 0 else None
    for n in rows:
        s, sg = coarse_row(level, n)
        got = s_all[n].cpu().numpy()
        assert np.max(np.abs(got - s)) < 1e-11 * max(1.0, np.max(np.abs(s)))
        if level > 0:
            g = sg_all[n].cpu().numpy()
            assert np.max(np.abs(g - sg)) < 1e-11 * max(1.0, np.max(np.abs(sg)))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("level,n", [(0, 9999), (1, 1500), (2, 200), (3, 17)])
def test_single_steps_of_sampled_rows(precision, level, n):
    h = handle(precision)
    rng = np.random.default_rng(40 + level)
    x = rng.standard_normal(NX)
    got = h.apply_step(level, n, torch.from_numpy(x.reshape(1, -1).copy()).cuda()).cpu().numpy()[0]
    s, sg = coarse_row(level, n)
    ref = osl.sl_apply_1d(x, s, P)
    if level > 0:
        ref = spla.spsolve(oc.correction_matrix_1d(sg, P), ref)
    tol = (1e-12 if level == 0 else 1e-10) if precision == 0 else 2e-6
    assert rel(got, ref) < tol
    h.destroy()


@pytest.fixture(scope="module")
def sequential_oracle():
    H = omg.Hierarchy(GRID, WS, P, [])
    return omg.sequential_solve(H, W.u0_bumps_1d(NX, W.SEED_C2_BUMPS, 3))


@pytest.mark.parametrize("precision", [1, 0])
def test_mgrit_solution_is_the_sequential_solution(precision, sequential_oracle):
    """The benchmark's solve (FP32 bulk: its launch configuration) converges to the oracle's sequential
    solution; the residual history falls by 1e-10 in the iteration count the benchmark reports."""
    u0 = W.u0_bumps_1d(NX, W.SEED_C2_BUMPS, 3)
    U0 = W.initial_iterate(NT, NX)
    h = mg.mgrit_setup(NX, NT, P, M, wave="sin_kx_cos_t", a=0.5, k=1.0, max_coarsest=8, precision=precision,
                       rtol=1e-10)
    out, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda())
    assert st["converged"] and st["history"][-1] < 1e-10 * st["history"][0]
    got = out.cpu().numpy()
    ref = sequential_oracle
    rows = [1, 7, 8, 4095, 8192, 12345, NT]
    assert rel(got[rows], ref[rows]) < 1e-9
    assert rel(got, ref) < 1e-9
    h.destroy()


# ---- 2D workload, fine level (512^2, p = r = 5) -------------------------------------------------------

NX2, NT2 = 512, 2048
WS2 = osl.WaveSpeed("sin_cos2", a=0.5, a2=0.5)
GRID2 = osl.Grid(NX2, NT2, dim=2)


@pytest.fixture(scope="module")
def h2d():
    h = mg.mgrit_setup(NX2, NT2, 5, 4, wave="sin_cos2", a=0.5, a2=0.5, dim=2, precision=1)
    yield h
    h.destroy()


@pytest.mark.parametrize("n", [0, 1234, 2047])
def test_2d_offsets_and_single_step_of_sampled_rows(h2d, n):
    sx, sy = osl.departure_offsets_2d(GRID2, WS2, n, 5)
    s_all = h2d.offsets(0)
    gx = s_all[n].cpu().numpy().reshape(NX2, NX2)
    gy = s_all[NT2 + n].cpu().numpy().reshape(NX2, NX2)
    assert np.max(np.abs(gx - sx)) < 1e-11 * max(1.0, np.max(np.abs(sx)))
    assert np.max(np.abs(gy - sy)) < 1e-11 * max(1.0, np.max(np.abs(sy)))
    x = np.random.default_rng(7).standard_normal((NX2, NX2))
    ref = osl.sl_apply_2d(x, sx, sy, 5)
    got = h2d.apply_step(0, n, torch.from_numpy(x.reshape(1, -1).copy()).cuda()).cpu().numpy()[0]
    assert rel(got, ref.ravel()) < 2e-6
