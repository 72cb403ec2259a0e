"""FP32 bulk with an FP64 coarse cycle (coarse_fp64 = 1): level 0's error relaxation in FP32, the coarse
levels (relaxation, coarse residuals, correction solves, coarsest solve) in FP64, against the FP64 oracle
with identical iteration counts; and the cluster split of FP64 coarse passes (cluster_coarse), equal bit
for bit to the one-CTA-per-interval kernels."""

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
@pytest.mark.parametrize("mode", ["FCF", "F"])
def test_coarse_fp64_1d_matches_the_oracle(p, mode):
    nx, nt, m = 256, 1024, 8
    ws = osl.WaveSpeed("sin_kx_cos_t", a=0.5, k=1.0)
    H = omg.build_hierarchy(osl.Grid(nx, nt), ws, p, m)
    u0 = W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
    U0 = W.initial_iterate(nt, nx)
    ref = omg.mgrit_solve(H, u0, U0, mode=mode)
    h = mg.mgrit_setup(nx, nt, p, m, wave="sin_kx_cos_t", a=0.5, k=1.0, precision=1, coarse_fp64=1,
                       relax=0 if mode == "FCF" else 1)
    out, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda())
    assert st["converged"] and st["iterations"] == ref.iterations
    assert rel(out.cpu().numpy(), ref.U) < 1e-5


def test_coarse_fp64_2d_matches_the_oracle():
    nx, nt, p, m = 32, 64, 3, 4
    g = osl.Grid(nx, nt, dim=2)
    ws = osl.WaveSpeed("sin_cos2", a=0.5, a2=0.5)
    H = omg.build_hierarchy(g, ws, p, m, levels=0, solve_mode="gmres", gmres_rtol=1e-2, gmres_maxit=10)
    u0 = W.u0_bumps_2d(nx, W.SEED_C3_BUMPS, 5)
    U0 = W.initial_iterate(nt, nx * nx)
    ref = omg.mgrit_solve(H, u0, U0.reshape(nt + 1, nx, nx))
    h = mg.mgrit_setup(nx, nt, p, m, wave="sin_cos2", a=0.5, a2=0.5, dim=2, precision=1, coarse_fp64=1)
    out, st = h.solve(torch.from_numpy(u0.ravel().copy()).cuda(), torch.from_numpy(U0).cuda())
    assert st["converged"] and st["iterations"] == ref.iterations
    assert rel(out.cpu().numpy(), ref.U.reshape(nt + 1, -1)) < 1e-5


def test_coarse_fp64_argument_errors():
    with pytest.raises(mg.MgritError):
        mg.mgrit_setup(64, 64, 3, 4, precision=0, coarse_fp64=1)
    with pytest.raises(mg.MgritError):
        mg.mgrit_setup_batched([dict(nx=64, nt=64, order=3, m=4)], precision=1, coarse_fp64=1)


@pytest.mark.parametrize("p", [1, 3, 5])
@pytest.mark.parametrize("nx,nt,m", [(4096, 2048, 8), (256, 1024, 4), (16, 256, 4)])
def test_cluster_split_coarse_levels_are_identical(p, nx, nt, m):
    """cluster_coarse = 1 splits FP64 coarse passes with few intervals (and the FP64 coarsest solve)
    over thread-block clusters; the results equal the one-CTA-per-interval kernels bit for bit."""
    ws = dict(wave="sin_kx_cos_t", a=0.5, k=1.0)
    u0 = torch.from_numpy(W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)).cuda()
    U0 = torch.from_numpy(W.initial_iterate(nt, nx)).cuda()
    outs = []
    for cl in (0, 1):
        h = mg.mgrit_setup(nx, nt, p, m, cluster_coarse=cl, **ws)
        out, st = h.solve(u0, U0)
        outs.append((out.cpu().numpy(), st["iterations"], st["history"]))
    assert outs[0][1] == outs[1][1]
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][2] == outs[1][2]


def test_cluster_split_matches_the_oracle_fp64():
    nx, nt, p, m = 512, 512, 3, 8
    ws = osl.WaveSpeed("sin_kx_cos_t", a=0.6, k=2.0)
    H = omg.build_hierarchy(osl.Grid(nx, nt), ws, p, m)
    u0 = W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
    U0 = W.initial_iterate(nt, nx)
    ref = omg.mgrit_solve(H, u0, U0)
    h = mg.mgrit_setup(nx, nt, p, m, wave="sin_kx_cos_t", a=0.6, k=2.0, cluster_coarse=1)
    out, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda())
    assert st["iterations"] == ref.iterations
    assert rel(out.cpu().numpy(), ref.U) < 1e-12
