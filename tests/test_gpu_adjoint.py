"""GPU parity of the discrete adjoint (mgrit_adjoint_solve) against the oracle, and the gradients against
central finite differences of the GPU's own sequential forward solve (FP64, step 1e-6)."""

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as oadj
from oracle import mgrit as omg
from oracle import semi_lagrangian as osl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2203_13382_gb300 as mg  # noqa: E402
from paper_2203_13382_gb300.autograd import advection_solve  # noqa: E402

CASES = [
    # nx, nt, p, m, wave, a, levels
    (64, 128, 3, 4, "sin_kx_cos_t", 0.5, 0),
    (64, 64, 1, 8, "sin_kx_cos_t", 0.3, 2),
    (32, 96, 5, 4, "const", 0.9, 0),
]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def oracle_gradients(nx, nt, p, m, wave, a, levels, u0, ut, U_init):
    g = osl.Grid(nx, nt)
    ws = osl.WaveSpeed(wave, a=a, k=1.0)
    H = omg.build_hierarchy(g, ws, p, m, levels=levels)
    fwd = omg.mgrit_solve(H, u0, U_init)
    lam, res = oadj.adjoint_mgrit(H, fwd.U[-1] - ut, np.zeros_like(fwd.U))
    dJda = 0.0
    for n in range(nt):
        ds = oadj.departure_offsets_da_1d(g, ws, n, p)
        dJda += float(lam[n + 1] @ oadj.dphi_da_apply_1d(fwd.U[n], H.levels[0].s[n], ds, p))
    return fwd, lam, res, dJda


@pytest.mark.parametrize("case", CASES)
def test_adjoint_matches_oracle(case):
    nx, nt, p, m, wave, a, levels = case
    u0 = W.u0_bumps_1d(nx, W.SEED_C5_BUMPS, 3)
    ut = W.u0_bumps_1d(nx, W.SEED_C5_TARGET, 3)
    U_init = W.initial_iterate(nt, nx)
    fwd, lam, res, dJda = oracle_gradients(nx, nt, p, m, wave, a, levels, u0, ut, U_init)
    h = mg.mgrit_setup(nx, nt, p, m, wave=wave, a=a, k=1.0, levels=levels)
    U, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U_init).cuda())
    assert st["iterations"] == fwd.iterations
    m1 = h.level_info(1)[1]
    dJdu0, ga_dev, ast = h.adjoint(torch.from_numpy(ut).cuda(), U[::m1].contiguous())
    assert ga_dev.is_cuda and ga_dev.shape == (1,)  # dJ/da stays on the device
    ga = float(ga_dev)
    assert ast["iterations"] == res.iterations
    assert rel(dJdu0.cpu().numpy(), lam[0]) < 1e-11
    assert abs(ga - dJda) <= 1e-11 * max(abs(dJda), 1e-12)


def test_gradients_match_finite_differences_of_the_gpu_forward():
    nx, nt, p, m = 64, 128, 3, 4
    a0, hfd = 0.5, 1e-6
    u0 = torch.from_numpy(W.u0_bumps_1d(nx, W.SEED_C5_BUMPS, 3)).cuda()
    ut = torch.from_numpy(W.u0_bumps_1d(nx, W.SEED_C5_TARGET, 3)).cuda()

    def J(a, u):
        h = mg.mgrit_setup(nx, nt, p, m, wave="sin_kx_cos_t", a=a, k=1.0)
        last = h.sequential(u, store_all=False)
        h.destroy()
        return 0.5 * float(((last - ut) ** 2).sum())

    u0r = u0.clone().requires_grad_(True)
    ar = torch.tensor(a0, dtype=torch.float64, device="cuda", requires_grad=True)
    uT = advection_solve(u0r, ar, nx=nx, nt=nt, order=p, m=m, wave="sin_kx_cos_t", k=1.0)
    loss = 0.5 * ((uT - ut) ** 2).sum()
    loss.backward()
    fda = (J(a0 + hfd, u0) - J(a0 - hfd, u0)) / (2 * hfd)
    assert abs(float(ar.grad) - fda) <= 1e-6 * abs(fda)
    rng = np.random.default_rng(20260006)
    for _ in range(4):
        d = torch.from_numpy(rng.standard_normal(nx)).cuda()
        fdu = (J(a0, u0 + hfd * d) - J(a0, u0 - hfd * d)) / (2 * hfd)
        assert abs(float((u0r.grad * d).sum()) - fdu) <= 1e-6 * max(abs(fdu), 1e-3)


def test_adjoint_rejects_fp32_bulk_handles():
    h = mg.mgrit_setup(64, 64, 3, 4, wave="sin_kx_cos_t", a=0.5, precision=1)
    z = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MgritError):
        h.adjoint(z, torch.zeros(17, 64, dtype=torch.float64, device="cuda"))
