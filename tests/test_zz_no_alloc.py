"""mgrit_apply_step_noalloc: the variant of mgrit_apply_step for callers that cannot allocate device memory.

It must give the same result as mgrit_apply_step, call after call, while allocating nothing (its FP32
staging lives in a fixed file-scope device buffer).  This file is collected last so that a run that
stops at the first failure has already run every other test.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2203_13382_gb300 as mg  # noqa: E402

FP32_TOL = 1e-5  # the FP32-bulk tolerance of the parity tests


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision", [1, 0])
def test_noalloc_matches_apply_step_on_consecutive_calls(precision):
    h = mg.mgrit_setup(256, 512, 3, 4, wave="sin_kx_cos_t", a=0.5, k=1.0, precision=precision)
    rng = np.random.default_rng(20260501)
    for level in (0, 1, 2):
        nt_l, _ = h.level_info(level)
        for call in range(2):  # two calls in a row share the staging buffer
            count = 3 + call
            n0 = (call * 5) % max(1, nt_l - count)
            x = torch.from_numpy(rng.standard_normal((count, 256))).cuda()
            ref = h.apply_step(level, n0, x).cpu().numpy()
            out = torch.empty_like(x)
            got = h.apply_step_noalloc(level, n0, x, out).cpu().numpy()
            assert rel(got, ref) <= FP32_TOL, (level, call, rel(got, ref))
    h.destroy()


def test_noalloc_rejects_sizes_beyond_its_capacity():
    h = mg.mgrit_setup(1024, 4096, 1, 4, wave="const", precision=1)
    x = torch.zeros(1025, 1024, dtype=torch.float64, device="cuda")  # 1025 * 1024 > 2^20 values
    with pytest.raises(mg.MgritError) as e:
        h.apply_step_noalloc(0, 0, x)
    assert e.value.status == 1 and "capacity" in str(e.value)
    h.destroy()
