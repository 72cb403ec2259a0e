"""The GPU's 1D MGRIT iteration counts against the paper's printed counts at its larger grids: Table 2
(multilevel, Sec. 3.4) and Table 1 (two levels, Sec. 3.3) at 2^10 x 2^12 and 2^12 x 2^14 (the oracle
reproduces their 2^8 x 2^10 rows in the CPU suite), and the strong-scaling problem of Sec. 5 / SM4
(2^12 x 2^14, coarsening 16 then 4).

The golden values are the paper's printed counts (tests/golden/table2_multilevel_iters_large.txt,
tests/golden/table1_two_level_iters_large.txt, tests/golden/sm4_strong_scaling_iters.txt), with the
paper's settings (Table 1: two levels; the paper's 10-iteration GMRES correction solves are exact here): FP64, linear MGRIT, FCF, the
corrected coarse operator with exact 1D correction solves, u0 = sin^4(pi x), a random U[0, 1] initial
iterate.  The paper's random iterate is not known, so a count may differ from the printed one by a
cycle; every cell must agree within one and most cells exactly.  Each cell's pair is printed.
"""

import os

import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2203_13382_gb300 as mg  # noqa: E402

HERE = os.path.join(os.path.dirname(__file__), "golden")
WAVES = {"alpha1": dict(wave="const", a=1.0), "alpha2": dict(wave="cos_t"), "alpha4": dict(wave="cos_t_cos_x")}


def cells():
    """(log2 nx, log2 nt, alpha, p, m_first, m, levels, printed count) of the golden files."""
    out = []
    for name, kind in (("table2_multilevel_iters_large.txt", "t2"), ("table1_two_level_iters_large.txt", "t1"),
                       ("sm4_strong_scaling_iters.txt", "sm4")):
        with open(os.path.join(HERE, name)) as f:
            for line in f:
                if line.startswith("#") or not line.strip():
                    continue
                v = line.split()
                if kind == "sm4":
                    out.append((int(v[0]), int(v[1]), v[2], int(v[3]), int(v[4]), int(v[5]), 0, int(v[6])))
                else:
                    out.append((int(v[0]), int(v[1]), v[2], int(v[3]), 0, int(v[4]), 2 if kind == "t1" else 0,
                                int(v[5])))
    return out


@pytest.fixture(scope="module")
def counts():
    res = {}
    for c in cells():
        lnx, lnt, a, p, mf, m, lv, _ = c
        nx, nt = 1 << lnx, 1 << lnt
        h = mg.mgrit_setup(nx, nt, p, m, levels=lv, m_first=mf, **WAVES[a])
        u0 = torch.from_numpy(W.u0_sin4(nx)).cuda()
        U0 = torch.from_numpy(W.initial_iterate(nt, nx)).cuda()
        _, st = h.solve(u0, U0)
        h.destroy()
        assert st["converged"]
        res[c] = st["iterations"]
    return res


def cell_id(c):
    m = f"{c[4]}-{c[5]}" if c[4] else f"{c[5]}"
    return f"{'two-level' if c[6] == 2 else 'multilevel'}-{c[2]}-p{c[3]}-m{m}-2^{c[0]}x2^{c[1]}"


@pytest.mark.parametrize("cell", cells(), ids=cell_id)
def test_cell_within_one_cycle(counts, cell):
    got, expect = counts[cell], cell[7]
    print(f"{cell_id(cell)}: paper {expect}, GPU {got}")
    assert abs(got - expect) <= 1


def test_most_cells_exact(counts):
    exact = sum(counts[c] == c[7] for c in counts)
    print(f"{exact} of {len(counts)} cells equal the paper's printed count")
    assert exact >= 0.8 * len(counts)
