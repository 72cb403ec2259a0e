"""The discretisation-accuracy stopping rule (mgrit_solve_to_reference, Sec. SM4) against the oracle's
u_final_ref rule: alpha = cos(2 pi t), whose exact flow gives the reference final state."""

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


def exact_final(g):
    x = g.xmin + g.h * np.arange(g.nx)
    T = g.nt * g.dt
    return np.sin(np.pi * (x - np.sin(2 * np.pi * T) / (2 * np.pi))) ** 4


@pytest.mark.parametrize("p", [3, 5])
@pytest.mark.parametrize("precision", [0, 1])
def test_stop_at_discretisation_accuracy(p, precision):
    g = osl.Grid(128, 256)
    ws = osl.WaveSpeed("cos_t")
    x = g.xmin + g.h * np.arange(g.nx)
    u0 = np.sin(np.pi * x) ** 4
    ref = exact_final(g)
    H = omg.build_hierarchy(g, ws, p, 4)
    seq = omg.sequential_solve(H, u0)
    tol = 1.01 * float(np.sqrt(g.h * np.sum((seq[-1] - ref) ** 2)))
    U0 = W.initial_iterate(g.nt, g.nx)
    R = omg.mgrit_solve(H, u0, U0, u_final_ref=ref, final_tol=tol)
    h = mg.mgrit_setup(g.nx, g.nt, p, 4, wave="cos_t", precision=precision)
    out, st = h.solve_to_reference(torch.from_numpy(u0).cuda(), torch.from_numpy(ref).cuda(), tol,
                                   u_init=torch.from_numpy(U0).cuda())
    assert st["converged"] and st["iterations"] == R.iterations
    # e is a distance between nearby vectors: compare it on the scale of the states themselves
    scale = float(np.sqrt(g.h * np.sum(ref ** 2)))
    assert abs(st["final_error"] - R.final_errors[-1]) <= (1e-12 if precision == 0 else 1e-5) * scale
    got = out.cpu().numpy()
    assert np.linalg.norm(got - R.U) / np.linalg.norm(R.U) < (1e-12 if precision == 0 else 1e-5)
    # the returned final slice is the one the rule measured
    assert abs(np.sqrt(g.h * np.sum((got[-1] - ref) ** 2)) - st["final_error"]) < 1e-12 * st["final_error"] + 1e-15


def test_stop_rule_argument_errors():
    h = mg.mgrit_setup(64, 64, 3, 4, wave="cos_t")
    u0 = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MgritError):
        h.solve_to_reference(u0, u0, -1.0)
