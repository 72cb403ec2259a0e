"""Sequential SL stepping on the GPU (sl_step_sequential), the comparator of MGRIT: the thread-block
cluster kernel (nx >= 256) against the oracle's sequential stepping (eq. (one-step)), FP64 to 1e-12
and FP32 to 1e-5, every slice and final slice only, including the full 1D workload (nx = 4096,
nt = 16384, p = 3, alpha = 1 + 0.5 sin(2 pi x) cos(2 pi t))."""

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


def oracle_sequential(nx, nt, p, a, k, u0):
    H = omg.Hierarchy(osl.Grid(nx, nt), osl.WaveSpeed("sin_kx_cos_t", a=a, k=k), p, [])
    return omg.sequential_solve(H, u0)


@pytest.mark.parametrize("nx", [256, 512, 1024, 2048, 4096])
@pytest.mark.parametrize("p", [1, 3, 5])
@pytest.mark.parametrize("precision", [0, 1])
def test_cluster_sequential_matches_oracle(nx, p, precision):
    nt = 96
    u0 = W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
    ref = oracle_sequential(nx, nt, p, 0.5, 2.0, u0)
    h = mg.mgrit_setup(nx, nt, p, 4, wave="sin_kx_cos_t", a=0.5, k=2.0, precision=precision)
    tol = 1e-12 if precision == 0 else 1e-5
    out = h.sequential(torch.from_numpy(u0).cuda()).cpu().numpy()
    assert rel(out, ref) < tol
    last = h.sequential(torch.from_numpy(u0).cuda(), store_all=False).cpu().numpy()
    assert rel(last, ref[-1]) < tol
    if precision == 0:
        assert np.array_equal(last, out[-1])


def test_cluster_sequential_full_workload_matches_oracle():
    nx, nt, p = 4096, 16384, 3
    u0 = W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
    ref = oracle_sequential(nx, nt, p, 0.5, 1.0, u0)
    h = mg.mgrit_setup(nx, nt, p, 8, wave="sin_kx_cos_t", a=0.5, k=1.0, max_coarsest=8)
    out = h.sequential(torch.from_numpy(u0).cuda()).cpu().numpy()
    rows = [1, 2, 1000, 8191, 12345, nt]
    assert rel(out[rows], ref[rows]) < 1e-12
    assert rel(out, ref) < 1e-12
