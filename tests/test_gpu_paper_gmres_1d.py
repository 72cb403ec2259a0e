"""1D coarse correction solves by the paper's inexact GMRES (solve_mode 1; Sec. 3.3: 10 iterations from a
zero guess in the two-level runs, Sec. 3.4: relative residual 1e-2 or 10 iterations in the multilevel ones).

- Parity with the oracle's "gmres" mode (oracle/coarse.py gmres_zero_guess): the same iteration counts and
  residual histories.  With an inexact inner solve MGRIT is no longer a linear iteration, and the oracle's
  modified Gram-Schmidt and the GPU's classical Gram-Schmidt in two passes round differently, so the
  iterates are compared where the theory fixes them: both converge to the unique solution of the
  fine-level one-step system (the oracle's sequential stepping) -- within 1e-9 relative, as two iterates
  at a 1e-10 residual.
- The paper's Table 1 (two levels) at 2^10 x 2^12 and 2^12 x 2^14 under its own coarse solve (10 GMRES
  iterations): every cell within one cycle of the printed count, and the number of exact cells reported.
"""

import os

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

HERE = os.path.join(os.path.dirname(__file__), "golden")
WAVES = {"alpha1": dict(wave="const", a=1.0), "alpha2": dict(wave="cos_t"), "alpha4": dict(wave="cos_t_cos_x")}
ORACLE_WAVES = {"alpha1": osl.WaveSpeed("const"), "alpha2": osl.WaveSpeed("cos_t"),
                "alpha4": osl.WaveSpeed("cos_t_cos_x")}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


# (nx, nt, p, m, levels, gmres_rtol, gmres_maxit, wave): two-level with a fixed 10 iterations, multilevel
# with the paper's rtol 1e-2 / 10 iterations, p = 1, 3, 5, constant and variable speeds
CASES = [
    (128, 512, 1, 4, 2, 0.0, 10, "alpha1"),
    (128, 512, 3, 8, 2, 0.0, 10, "alpha4"),
    (256, 256, 5, 4, 2, 0.0, 10, "alpha2"),
    (128, 1024, 3, 4, 0, 1e-2, 10, "alpha4"),
    (256, 512, 5, 8, 0, 1e-2, 10, "alpha1"),
    (64, 1024, 1, 4, 0, 1e-2, 10, "alpha2"),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"nx{c[0]}-nt{c[1]}-p{c[2]}-m{c[3]}-L{c[4]}-rtol{c[5]}-{c[7]}")
def test_paper_mode_matches_the_oracle(case):
    nx, nt, p, m, levels, rtol, maxit, a = case
    u0 = W.u0_sin4(nx)
    U0 = W.initial_iterate(nt, nx)
    H = omg.build_hierarchy(osl.Grid(nx, nt), ORACLE_WAVES[a], p, m, levels=levels, solve_mode="gmres",
                            gmres_rtol=rtol, gmres_maxit=maxit)
    R = omg.mgrit_solve(H, u0, U0)
    seq = omg.sequential_solve(omg.Hierarchy(osl.Grid(nx, nt), ORACLE_WAVES[a], p, []), u0)
    h = mg.mgrit_setup(nx, nt, p, m, levels=levels, solve_mode=1, gmres_rtol=rtol, gmres_maxit=maxit, **WAVES[a])
    assert h.nlevels == H.nlevels
    out, st = h.solve(torch.from_numpy(u0).cuda(), torch.from_numpy(U0).cuda())
    h.destroy()
    assert st["converged"] and st["iterations"] == R.iterations, (st["iterations"], R.iterations)
    # the first cycles agree closely; later residuals are rounding-sensitive (nonlinear iteration)
    assert np.allclose(st["history"][:3], R.history[:3], rtol=1e-6, atol=0)
    got = out.cpu().numpy()
    assert rel(got, seq) < 1e-9 and rel(R.U, seq) < 1e-9


def test_paper_mode_options_are_checked():
    with pytest.raises(mg.MgritError) as e:  # FP32 coarse levels have no GMRES path
        mg.mgrit_setup(64, 64, 3, 4, wave="const", precision=1, solve_mode=1)
    assert e.value.status == 7
    h = mg.mgrit_setup(64, 64, 3, 4, wave="const", solve_mode=1)
    z = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MgritError) as e:
        h.adjoint(z, torch.zeros(17, 64, dtype=torch.float64, device="cuda"))
    assert e.value.status == 7
    h.destroy()


def table1_cells():
    out = []
    with open(os.path.join(HERE, "table1_two_level_iters_large.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = line.split()
            out.append((int(v[0]), int(v[1]), v[2], int(v[3]), int(v[4]), int(v[5])))
    return out


@pytest.fixture(scope="module")
def table1_counts():
    res = {}
    for c in table1_cells():
        lnx, lnt, a, p, m, _ = c
        nx, nt = 1 << lnx, 1 << lnt
        h = mg.mgrit_setup(nx, nt, p, m, levels=2, solve_mode=1, gmres_rtol=0.0, gmres_maxit=10, **WAVES[a])
        _, st = h.solve(torch.from_numpy(W.u0_sin4(nx)).cuda(), torch.from_numpy(W.initial_iterate(nt, nx)).cuda())
        h.destroy()
        assert st["converged"]
        res[c] = st["iterations"]
    return res


@pytest.mark.parametrize("cell", table1_cells(), ids=lambda c: f"{c[2]}-p{c[3]}-m{c[4]}-2^{c[0]}x2^{c[1]}")
def test_table1_cell_under_the_papers_coarse_solve(table1_counts, cell):
    got, expect = table1_counts[cell], cell[5]
    print(f"Table 1 {cell[2]} p={cell[3]} m={cell[4]} 2^{cell[0]} x 2^{cell[1]}: paper {expect}, GPU (GMRES) {got}")
    assert abs(got - expect) <= 1


def test_table1_exact_cells_under_the_papers_coarse_solve(table1_counts):
    exact = sum(table1_counts[c] == c[5] for c in table1_counts)
    print(f"Table 1 with 10-iteration GMRES correction solves: {exact} of {len(table1_counts)} cells exact")
    assert exact >= 0.8 * len(table1_counts)
