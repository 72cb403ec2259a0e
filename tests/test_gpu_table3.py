"""The GPU's 2D MGRIT iteration counts against the paper's Table 3: both velocity fields (constant (1, 1)
and eq. (alpha-var_2D)), the corrected coarse operator at (2^6)^2 x 2^10, (2^7)^2 x 2^11 and (2^8)^2 x 2^12,
and the rediscretised coarse step (the parenthesised values) at the two smallest grids.

The golden values are the paper's printed counts (tests/golden/table3_2d_multilevel_iters_all.txt); the
paper's solver settings: FP64, linear MGRIT, FCF, coarsen until fewer than two time points remain, coarse
correction by GMRES with rtol 1e-2 / 10 iterations.  The exact count depends on the random initial
iterate and on rounding inside the inexact GMRES solves, so each cell must agree within a tolerance that
grows with the count (1 cycle, or 10% of the count when larger), most cells exactly; every pair is printed.
"""

import os

import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2203_13382_gb300 as mg  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table3_2d_multilevel_iters_all.txt")
VEL = {"const": dict(wave="const2", a=1.0, a2=1.0), "var": dict(wave="paper2", a=1.0, a2=1.0)}


def cells():
    out = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = line.split()
            out.append((v[0], v[1], int(v[2]), int(v[3]), int(v[4]), int(v[5]), int(v[6])))
    return out


def cell_id(c):
    return f"{c[0]}-{c[1]}-2^{c[2]}sq-x-2^{c[3]}-p{c[4]}-m{c[5]}"


@pytest.fixture(scope="module")
def counts():
    res = {}
    for c in cells():
        vel, coarse, lnx, lnt, p, m, _ = c
        nx, nt = 1 << lnx, 1 << lnt
        # the rediscretised operator grows the residual for many cycles before it converges: no growth cap
        h = mg.mgrit_setup(nx, nt, p, m, dim=2, coarse_op=0 if coarse == "corr" else 1, max_iter=400,
                           diverge_ratio=0.0, **VEL[vel])
        u0 = torch.from_numpy(W.u0_sin2_2d(nx).ravel().copy()).cuda()
        U0 = torch.from_numpy(W.initial_iterate(nt, nx * nx)).cuda()
        _, st = h.solve(u0, U0)
        h.destroy()
        assert st["converged"]
        res[c] = st["iterations"]
    return res


@pytest.mark.parametrize("cell", cells(), ids=cell_id)
def test_table3_cell(counts, cell):
    got, expect = counts[cell], cell[6]
    print(f"Table 3 {cell_id(cell)}: paper {expect}, GPU {got}")
    assert abs(got - expect) <= 1


def test_table3_most_cells_exact(counts):
    exact = sum(counts[c] == c[6] for c in counts)
    within1 = sum(abs(counts[c] - c[6]) <= 1 for c in counts)
    print(f"Table 3: {exact} of {len(counts)} cells equal the paper's printed count, {within1} within one")
    assert within1 == len(counts) and exact >= 0.85 * len(counts)
