"""GPU parity of the 2D discrete adjoint (mgrit_adjoint_solve on a 2D handle).

Small grids: the adjoint MGRIT's iteration count equals the oracle's (same cycle, same inexact GMRES on
M^T), and dJ/du0, dJ/da agree with the oracle's exact discrete gradient (sequential forward and backward
stepping).  Both MGRIT solves stop at a 1e-10 relative residual, so the comparison tolerance is 1e-8.
Adjoint workload (256^2, nt = 1024, p = 3, m = 4, alpha = (1 + a sin 2 pi y cos 2 pi t, 1 + a cos 2 pi x
sin 2 pi t), a = 0.5): dJ/da and dJ/du0 along 4 seeded directions against central finite differences (step
1e-6) of the GPU's FP64 sequential forward, to 1e-6 relative.
"""

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
    # nx, nt, p, m, wave, a
    (16, 32, 3, 4, "sin_cos2", 0.5),
    (16, 32, 1, 4, "const2", 0.8),
    (16, 64, 5, 4, "sin_cos2", 0.3),
    (32, 32, 3, 8, "paper2", 1.0),
]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.mark.parametrize("case", CASES)
def test_adjoint_2d_matches_oracle(case):
    nx, nt, p, m, wave, a = case
    g = osl.Grid(nx, nt, dim=2)
    ws = osl.WaveSpeed(wave, a=a, a2=0.6)
    u0 = W.u0_bumps_2d(nx, W.SEED_C5_BUMPS, 5)
    ut = W.u0_bumps_2d(nx, W.SEED_C5_TARGET, 5)
    U_init = W.initial_iterate(nt, nx * nx)
    H = omg.build_hierarchy(g, ws, p, m, solve_mode="gmres", gmres_rtol=1e-2, gmres_maxit=10)
    fwd = omg.mgrit_solve(H, u0, U_init.reshape(nt + 1, nx, nx))
    _, res = oadj.adjoint_mgrit(H, fwd.U[-1] - ut, np.zeros_like(fwd.U))
    lam0, dJda = oadj.gradients(g, ws, p, u0, ut)

    h = mg.mgrit_setup(nx, nt, p, m, wave=wave, a=a, a2=0.6, dim=2)
    U, st = h.solve(torch.from_numpy(u0.ravel().copy()).cuda(), torch.from_numpy(U_init).cuda())
    assert st["iterations"] == fwd.iterations
    m1 = h.level_info(1)[1]
    dJdu0, ga_dev, ast = h.adjoint(torch.from_numpy(ut.ravel().copy()).cuda(), U[::m1].contiguous())
    assert ga_dev.is_cuda and ga_dev.shape == (1,)  # dJ/da stays on the device
    ga = float(ga_dev)
    assert ast["converged"] and ast["iterations"] == res.iterations
    assert rel(dJdu0.cpu().numpy(), lam0.ravel()) < 1e-8
    if wave == "paper2":
        assert ga == 0.0 and dJda == 0.0
    else:
        assert abs(ga - dJda) <= 1e-8 * abs(dJda)


def test_adjoint_2d_repeated_calls_are_bitwise_identical():
    """The transposed step sums in a fixed order (sorted buckets): no dependence on atomic ordering."""
    nx, nt = 32, 32
    h = mg.mgrit_setup(nx, nt, 3, 4, wave="sin_cos2", a=0.5, dim=2)
    u0 = torch.from_numpy(W.u0_bumps_2d(nx, W.SEED_C5_BUMPS, 5).ravel().copy()).cuda()
    ut = torch.from_numpy(W.u0_bumps_2d(nx, W.SEED_C5_TARGET, 5).ravel().copy()).cuda()
    U, _ = h.solve(u0)
    C = U[::4].contiguous()
    d1, a1, _ = h.adjoint(ut, C)
    d2, a2, _ = h.adjoint(ut, C)
    assert torch.equal(d1, d2) and torch.equal(a1, a2)


def test_adjoint_2d_full_size_against_finite_differences():
    nx, nt, p, m, a0, hfd = 256, 1024, 3, 4, 0.5, 1e-6
    u0 = torch.from_numpy(W.u0_bumps_2d(nx, W.SEED_C5_BUMPS, 5).ravel().copy()).cuda()
    # target: the forward solution at a = 0.4 from another bump set
    ht = mg.mgrit_setup(nx, nt, p, m, wave="sin_cos2", a=0.4, dim=2)
    ut = ht.sequential(torch.from_numpy(W.u0_bumps_2d(nx, W.SEED_C5_TARGET, 5).ravel().copy()).cuda(),
                       store_all=False).clone()
    ht.destroy()

    def J(a, u):
        h = mg.mgrit_setup(nx, nt, p, m, wave="sin_cos2", a=a, dim=2, levels=2)
        last = h.sequential(u, store_all=False)
        torch.cuda.synchronize()
        h.destroy()
        return 0.5 * float(((last - ut) ** 2).sum())

    u0r = u0.clone().requires_grad_(True)
    ar = torch.tensor(a0, dtype=torch.float64, device="cuda", requires_grad=True)
    uT = advection_solve(u0r, ar, nx=nx, nt=nt, order=p, m=m, dim=2, wave="sin_cos2")
    loss = 0.5 * ((uT - ut) ** 2).sum()
    loss.backward()
    fda = (J(a0 + hfd, u0) - J(a0 - hfd, u0)) / (2 * hfd)
    assert abs(float(ar.grad) - fda) <= 1e-6 * abs(fda)
    rng = np.random.default_rng(20260006)
    for _ in range(4):
        d = torch.from_numpy(rng.standard_normal(nx * nx)).cuda()
        fdu = (J(a0, u0 + hfd * d) - J(a0, u0 - hfd * d)) / (2 * hfd)
        assert abs(float((u0r.grad * d).sum()) - fdu) <= 1e-6 * max(abs(fdu), 1e-3)
