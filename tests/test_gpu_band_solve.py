"""The banded separator inverse of the FP32 correction solves (mgrit_options.coarse_band).

On 1D FP32 coarse levels M = I - diag(sigma) D_{p+1} (eq. (Phi_multilevel)) is solved with 8-row
partitions whose separator system is inverted by a stored band of S^{-1} = (M^{-1}) restricted to the
separators, probed in setup and kept only where it is exact to 1e-9 of its diagonal blocks.  A coarse step
with the band must equal the FP64 coarse step within the FP32 tolerance of the single-step parity tests and
the step with the block cyclic reduction (coarse_band = 0); the band must actually be in use on the levels
whose sigma is moderate; MGRIT with and without the band takes the same number of cycles.
"""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2203_13382_gb300 as mg  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


CASES = [(4096, 2048, 3, 8), (1024, 1024, 1, 4), (2048, 512, 5, 4), (512, 4096, 3, 4), (128, 256, 3, 4)]


@pytest.mark.parametrize("nx,nt,p,m", CASES)
def test_band_step_matches_fp64_and_block_pcr(nx, nt, p, m):
    kw = dict(wave="sin_kx_cos_t", a=0.5, k=2.0)
    hb = mg.mgrit_setup(nx, nt, p, m, precision=1, **kw)
    hp = mg.mgrit_setup(nx, nt, p, m, precision=1, coarse_band=0, **kw)
    hd = mg.mgrit_setup(nx, nt, p, m, precision=0, **kw)
    rng = np.random.default_rng(20260601 + nx + p)
    used = []
    for level in range(1, hb.nlevels):
        used.append(hb.level_band(level))
        assert hp.level_band(level) == 0
        nt_l, _ = hb.level_info(level)
        count = min(4, nt_l)
        n0 = (nt_l - count) // 2
        x = torch.from_numpy(rng.standard_normal((count, nx))).cuda()
        yb = hb.apply_step(level, n0, x).cpu().numpy()
        yp = hp.apply_step(level, n0, x).cpu().numpy()
        yd = hd.apply_step(level, n0, x).cpu().numpy()
        # FP32 accuracy: the single-step tolerance, or twice the block cyclic reduction's own error on the deep
        # levels where sigma is large and the correction matrix less well conditioned
        tol = max(2e-6, 2.0 * rel(yp, yd))
        assert rel(yb, yd) <= tol, (level, used[-1], rel(yb, yd), rel(yp, yd))
        assert rel(yb, yp) <= tol, (level, used[-1], rel(yb, yp))
    print(f"nx={nx} p={p} m={m}: band half-widths per coarse level {used}")
    if nx >= 128:
        assert used[0] > 0  # level 1 (moderate sigma) takes the band
    for h in (hb, hp, hd):
        h.destroy()


@pytest.mark.parametrize("p", [1, 3, 5])
def test_mgrit_with_and_without_the_band(p):
    nx, nt, m = 1024, 2048, 4
    kw = dict(wave="sin_kx_cos_t", a=0.5, k=1.0, precision=1)
    u0 = torch.from_numpy(W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)).cuda()
    U0 = torch.from_numpy(W.initial_iterate(nt, nx)).cuda()
    res = {}
    for band in (1, 0):
        h = mg.mgrit_setup(nx, nt, p, m, coarse_band=band, **kw)
        out, st = h.solve(u0, U0)
        res[band] = (out.cpu().numpy(), st["iterations"], [h.level_band(l) for l in range(1, h.nlevels)])
        h.destroy()
    assert res[1][1] == res[0][1]
    assert rel(res[1][0], res[0][0]) < 1e-9  # both at a 1e-10 residual of the same FP64 system
    assert any(w > 0 for w in res[1][2])
