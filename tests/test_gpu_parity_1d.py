"""GPU parity for the 1D path: every setup array, single steps, sequential stepping and MGRIT solves are
compared with the CPU oracle on the same seeded inputs, through the C ABI.

Tolerances: FP64 results within 1e-12 relative L2 of the oracle (the paper fixes no precision; both
sides evaluate the same formulas in IEEE double and differ only in rounding order, libm vs CUDA
sin/cos and FMA contraction); FP32-bulk within 1e-5; MGRIT iteration counts identical.
"""

import numpy as np
import pytest

import workloads as W
from oracle import coarse as oco
from oracle import mgrit as omg
from oracle import semi_lagrangian as osl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2203_13382_gb300 as mg  # noqa: E402

CASES = [
    # (nx, nt, p, m, wave, a, k, levels, max_coarsest)
    (64, 64, 1, 4, "const", 1.0, 1.0, 0, 1),
    (128, 256, 3, 4, "sin_kx_cos_t", 0.5, 1.0, 0, 1),
    (128, 512, 3, 8, "sin_kx_cos_t", 0.5, 1.0, 0, 8),
    (64, 256, 5, 4, "cos_t_cos_x", 1.0, 1.0, 0, 1),
    (256, 256, 1, 4, "const", 1.0, 1.0, 2, 1),  # the two-level constant-speed workload
    (64, 128, 1, 16, "cos_t", 1.0, 1.0, 0, 1),
]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def oracle_hierarchy(nx, nt, p, m, wave, a, k, levels, max_coarsest):
    g = osl.Grid(nx, nt)
    ws = osl.WaveSpeed(wave, a=a, k=k)
    return omg.build_hierarchy(g, ws, p, m, levels=levels, max_coarsest=max_coarsest)


def gpu_handle(nx, nt, p, m, wave, a, k, levels, max_coarsest, **opt):
    return mg.mgrit_setup(nx, nt, p, m, wave=wave, a=a, k=k, levels=levels, max_coarsest=max_coarsest, **opt)


@pytest.mark.parametrize("case", CASES)
def test_setup_arrays_match_oracle(case):
    """Departure offsets of every level (ERK, backtracking) and sigma (eq. (nu_p_def))."""
    H = oracle_hierarchy(*case)
    h = gpu_handle(*case)
    assert h.nlevels == H.nlevels
    for l in range(H.nlevels):
        nt_l, m_l = h.level_info(l)
        assert nt_l == H.levels[l].nt and m_l == H.levels[l].m
        s = h.offsets(l).cpu().numpy()
        assert np.max(np.abs(s - H.levels[l].s)) < 1e-11 * max(1.0, np.max(np.abs(H.levels[l].s)))
        if l > 0:
            sg = h.sigma(l).cpu().numpy()
            assert np.max(np.abs(sg - H.levels[l].sigma)) < 1e-11 * max(1.0, np.max(np.abs(H.levels[l].sigma)))


@pytest.mark.parametrize("case", CASES)
def test_single_steps_match_oracle(case):
    """Phi on level 0 (SL step) and Psi = [I - diag(sigma) D]^{-1} S on every coarse level."""
    H = oracle_hierarchy(*case)
    h = gpu_handle(*case)
    rng = np.random.default_rng(11)
    for l in range(H.nlevels):
        nt_l = H.levels[l].nt
        steps = sorted(set([0, nt_l // 2, nt_l - 1]))
        x = rng.standard_normal((len(steps), case[0]))
        for c, n in enumerate(steps):
            y = h.apply_step(l, n, torch.from_numpy(x[c : c + 1].copy()).cuda()).cpu().numpy()[0]
            ref = H.step(l, n, x[c])
            assert rel(y, ref) < 1e-12, (l, n, rel(y, ref))


@pytest.mark.parametrize("case", CASES)
def test_single_steps_fp32_match_oracle(case):
    """FP32 levels: the gather and the correction matrix factorised on the fly from sigma (FP32)."""
    H = oracle_hierarchy(*case)
    h = gpu_handle(*case, precision=1)
    rng = np.random.default_rng(12)
    for l in range(H.nlevels):
        nt_l = H.levels[l].nt
        for n in sorted(set([0, nt_l // 3, nt_l - 1])):
            x = rng.standard_normal(case[0])
            y = h.apply_step(l, n, torch.from_numpy(x[None, :].copy()).cuda()).cpu().numpy()[0]
            ref = H.step(l, n, x)
            assert rel(y, ref) < 2e-6, (l, n, rel(y, ref))


@pytest.mark.parametrize("case", CASES[:4])
def test_sequential_matches_oracle(case):
    H = oracle_hierarchy(*case)
    h = gpu_handle(*case)
    nx = case[0]
    u0 = W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
    ref = omg.sequential_solve(H, u0)
    out = h.sequential(torch.from_numpy(u0).cuda()).cpu().numpy()
    assert rel(out, ref) < 1e-12
    last = h.sequential(torch.from_numpy(u0).cuda(), store_all=False).cpu().numpy()
    assert rel(last, ref[-1]) < 1e-12


@pytest.mark.parametrize("case", CASES)
def test_mgrit_fp64_matches_oracle(case):
    H = oracle_hierarchy(*case)
    h = gpu_handle(*case)
    nx, nt = case[0], case[1]
    u0 = W.u0_sin4(nx) if case[4] == "const" else W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
    U0 = W.initial_iterate(nt, nx)
    ref = omg.mgrit_solve(H, u0, U0)
    out, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda())
    assert st["iterations"] == ref.iterations and st["converged"]
    assert rel(out.cpu().numpy(), ref.U) < 1e-12
    hist = np.array(st["history"])
    assert np.allclose(hist, ref.history, rtol=1e-7, atol=1e-13 * ref.history[0])


@pytest.mark.parametrize("case", CASES[1:4])
def test_mgrit_fp32_bulk_matches_fp64_oracle(case):
    """FP32 relaxation and coarse cycle on the error, FP64 residual and C-point state."""
    H = oracle_hierarchy(*case)
    h = gpu_handle(*case, precision=1)
    nx, nt = case[0], case[1]
    u0 = W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
    U0 = W.initial_iterate(nt, nx)
    ref = omg.mgrit_solve(H, u0, U0)
    out, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda())
    assert st["converged"]
    assert rel(out.cpu().numpy(), ref.U) < 1e-5
    assert st["iterations"] == ref.iterations


def test_correction_solve_against_dense_inverse():
    """Psi on a coarse level equals the dense [I - diag(sigma) D]^{-1} S built by the oracle."""
    case = (32, 64, 5, 4, "sin_kx_cos_t", 0.7, 2.0, 0, 1)
    H = oracle_hierarchy(*case)
    h = gpu_handle(*case)
    l = 1
    x = np.random.default_rng(3).standard_normal(32)
    for n in (0, 7, 15):
        M = oco.correction_matrix_1d(H.levels[l].sigma[n], 5).toarray()
        S = osl.sl_matrix_1d(H.levels[l].s[n], 5)
        ref = np.linalg.solve(M, S @ x)
        y = h.apply_step(l, n, torch.from_numpy(x[None].copy()).cuda()).cpu().numpy()[0]
        assert rel(y, ref) < 1e-12


def test_setup_rejects_bad_arguments_on_gpu():
    with pytest.raises(mg.MgritError):
        mg.mgrit_setup(64, 100, 3, 8, levels=3)  # 100 not divisible
    with pytest.raises(mg.MgritError):
        mg.mgrit_setup(64, 64, 4, 4)


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_matches_direct_launches(precision):
    """use_graph = 1 (cycles captured once and replayed) and 0 (launched one by one) give identical
    solutions and residual histories."""
    case = CASES[2]
    nx, nt = case[0], case[1]
    u0 = torch.from_numpy(W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)).cuda()
    U0 = torch.from_numpy(W.initial_iterate(nt, nx)).cuda()
    res = []
    for g in (0, 1):
        h = gpu_handle(*case, precision=precision, use_graph=g, profile=1)
        out, st = h.solve(u0, U0)
        res.append((out.cpu(), st))
    assert torch.equal(res[0][0], res[1][0])
    assert res[0][1]["iterations"] == res[1][1]["iterations"]
    assert res[0][1]["history"] == res[1][1]["history"]
    assert res[0][1]["kernel_launches"] == res[1][1]["kernel_launches"]
