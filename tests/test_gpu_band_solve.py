"""The banded separator inverse of the FP32 correction solves (mgrit_options.coarse_band).

On 1D FP32 coarse levels M = I - diag(sigma) D_{p+1} (eq. (Phi_multilevel)) is solved with 8-row
partitions whose separator system is inverted by a stored band of S^{-1} = (M^{-1}) restricted to the
separators, probed in setup (8 colours, and 16 where the decay is slower) and kept only where the entries
it leaves out are below 1e-8 of its diagonal blocks (under the FP32 unit roundoff of the solve that applies
it).
- The probed decay of S^{-1} equals the oracle's: M^{-1} formed densely from the oracle's sigma of every
  step, its separator blocks at partition distance t = 1..3 relative to the diagonal block of the same
  partition, summed as the probe's eight colours sum them (partitions 8 apart share a colour; FP32 probe:
  1e-3 relative where the ratio is above 1e-6), and the band width the setup chose is the smallest one whose
  left-out entries are under the tolerance.
- A coarse step with the band equals the FP64 coarse step within the FP32 tolerance of the single-step parity
  tests and the step with the block cyclic reduction (coarse_band = 0); the band is in use on the levels
  whose sigma is moderate; MGRIT with and without the band takes the same number of cycles.
"""

import numpy as np
import pytest

import workloads as W
from oracle import coarse as oco
from oracle import mgrit as omg
from oracle import semi_lagrangian as osl

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


def oracle_decay(sigma_rows, nx, p):
    """What the probe measures, from the exact inverse: S^{-1} is the separator rows and columns (the first B
    rows of each 8-row partition) of M^{-1}; a probe of colour c (unit right-hand sides on every partition
    = c mod 8) returns at partition k the sum of S^{-1}[k, q] over the partitions q = c (mod 8).  Ratio at
    distance t = 1..3: the largest such sum for q = k +- t (mod 8) over the one for q = k (mod 8), maximised
    over k and the steps."""
    B, P = (p + 1) // 2, nx // 8
    sep = np.array([k * 8 + a for k in range(P) for a in range(B)])
    out = np.zeros(3)
    for sig in sigma_rows:
        Minv = np.linalg.inv(oco.correction_matrix_1d(sig, p).toarray())
        S = Minv[np.ix_(sep, sep)].reshape(P, B, P, B)
        alias = np.stack([S[:, :, c::8, :].sum(axis=2) for c in range(8)], axis=1)  # [k][colour][a][c]
        for k in range(P):
            dmax = np.abs(alias[k, k % 8]).max()
            for t in range(1, 4):
                v = max(np.abs(alias[k, (k + t) % 8]).max(), np.abs(alias[k, (k - t) % 8]).max())
                out[t - 1] = max(out[t - 1], v / dmax)
    return out


@pytest.mark.parametrize("p", [1, 3, 5])
def test_probed_decay_matches_the_oracle(p):
    nx, nt, m = 256, 256, 4
    kw = dict(wave="sin_kx_cos_t", a=0.5, k=2.0)
    H = omg.build_hierarchy(osl.Grid(nx, nt), osl.WaveSpeed("sin_kx_cos_t", a=0.5, k=2.0), p, m)
    h = mg.mgrit_setup(nx, nt, p, m, precision=1, **kw)
    assert h.nlevels == H.nlevels
    for level in range(1, h.nlevels):
        W_gpu, dec = h.level_band(level, decay=True)
        if nx // 8 < 16 or not any(dec):
            continue
        ref = oracle_decay(H.levels[level].sigma, nx, p)
        for t in range(3):
            if ref[t] > 1e-6:
                assert abs(dec[t] - ref[t]) <= 1e-3 * ref[t], (level, t + 1, dec[t], ref[t])
            else:
                assert dec[t] <= 1e-6 + 2.0 * ref[t], (level, t + 1, dec[t], ref[t])
        # the chosen width: the smallest whose left-out entries (distances W+1 .. 4) are under 1e-8, or 0;
        # levels this first probe rejects are probed again with 16 colours (widths up to 6)
        need = next((w for w in range(1, 4) if all(d < 1e-8 for d in dec[w:])), 0)
        assert W_gpu in (need, 0) or need == 0, (level, W_gpu, need, dec)
        print(f"p={p} level {level}: band {W_gpu}, probed {['%.2e' % d for d in dec]}, oracle {['%.2e' % r for r in ref]}")
    h.destroy()
