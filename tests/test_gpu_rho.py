"""Two-level convergence factors of the GPU solver against the Fourier estimate rho(c) (Sec. 2.3, Fig. 2 for
the rediscretised coarse operator, Fig. 3 for the corrected one) at the paper's size nx x nt = 2^7 x 2^15,
and the measured factors against the oracle's on a shorter time axis."""

import numpy as np
import pytest

import workloads as W
from oracle import fourier as F
from oracle import mgrit as omg
from oracle import semi_lagrangian as osl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2203_13382_gb300 as mg  # noqa: E402


def gpu_history(nx, nt, p, m, c, coarse_op, iters):
    h = mg.mgrit_setup(nx, nt, p, m, wave="const", a=1.0, cfl=c, levels=2, coarse_op=coarse_op, max_iter=iters,
                       rtol=1e-300)
    _, st = h.solve(torch.from_numpy(W.u0_sin4(nx)).cuda(), torch.from_numpy(W.initial_iterate(nt, nx)).cuda(),
                    allow_not_converged=True)
    return st["history"]


@pytest.mark.parametrize("p", [1, 3])
@pytest.mark.parametrize("c", [0.55, 0.65, 0.85, 0.95])
def test_factors_follow_rho_at_the_paper_size(p, c):
    nx, nt, m = 128, 1 << 15, 4
    for coarse_op, kind in ((0, "corrected"), (1, "sl")):
        hist = gpu_history(nx, nt, p, m, c, coarse_op, 6)
        f = hist[-1] / hist[-2]
        r = F.rho(c, p, m, kind)
        if kind == "corrected":
            assert 0.75 * r <= f <= 1.05 * r, (f, r)
        elif r > 2:
            assert f > 1.0, (f, r)
        elif r < 0.5:
            assert f < 1.0, (f, r)


@pytest.mark.parametrize("p", [1, 3])
@pytest.mark.parametrize("coarse_op,kind", [(0, "corrected"), (1, "sl")])
def test_factors_equal_the_oracle(p, coarse_op, kind):
    nx, nt, m, c = 128, 2048, 4, 0.65
    g = osl.Grid(nx, nt, cfl=c)
    H = omg.build_hierarchy(g, osl.WaveSpeed("const", a=1.0), p, m, levels=2, coarse=kind)
    R = omg.mgrit_solve(H, W.u0_sin4(nx), W.initial_iterate(nt, nx), max_iter=5, rtol=1e-300)
    hist = gpu_history(nx, nt, p, m, c, coarse_op, 5)
    assert len(hist) == len(R.history)
    assert np.allclose(hist, R.history, rtol=1e-9, atol=0)
