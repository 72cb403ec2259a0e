"""mgrit_apply_step_noalloc: the variant of mgrit_apply_step for callers that cannot allocate device memory.

Some callers cannot let a library allocate: a framework that has reserved the whole device memory pool
for itself (a cudaMalloc from the library would fail, or fragment that pool), or a latency-bound caller
that cannot accept the device-wide synchronisation a cudaFree implies.  The entry point stages its FP32
levels through a fixed file-scope device buffer instead.  It runs the same kernels in the same order as
mgrit_apply_step, so its results must be bitwise equal, call after call (the buffer keeps the previous
call's contents), in 1D and 2D, and the device's free memory must not move while it runs.  This file is
collected last so that a run that stops at the first failure has already run every other test; it also
passes when run alone in a fresh process.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2203_13382_gb300 as mg  # noqa: E402


@pytest.mark.parametrize("precision", [1, 0])
def test_noalloc_equals_apply_step_on_consecutive_calls(precision):
    h = mg.mgrit_setup(256, 512, 3, 4, wave="sin_kx_cos_t", a=0.5, k=1.0, precision=precision)
    rng = np.random.default_rng(20260501)
    for level in (0, 1, 2):
        nt_l, _ = h.level_info(level)
        for call in range(2):  # two calls in a row share the staging buffer
            count = 3 + call
            n0 = (call * 5) % max(1, nt_l - count)
            x = torch.from_numpy(rng.standard_normal((count, 256))).cuda()
            ref = h.apply_step(level, n0, x)
            out = torch.empty_like(x)
            got = h.apply_step_noalloc(level, n0, x, out)
            assert got.data_ptr() == out.data_ptr()
            assert torch.equal(got, ref), (level, call, float((got - ref).abs().max()))
    h.destroy()


def test_noalloc_equals_apply_step_2d():
    """A 2D FP32-bulk handle: the fine SL step and the GMRES-corrected coarse step, staged through the same
    buffer (count * 64^2 values)."""
    nx = 64
    h = mg.mgrit_setup(nx, 64, 3, 4, wave="sin_cos2", a=0.5, dim=2, precision=1)
    rng = np.random.default_rng(20260502)
    for level in (0, 1):
        for call in range(2):
            count = 2 + call
            x = torch.from_numpy(rng.standard_normal((count, nx * nx))).cuda()
            ref = h.apply_step(level, call, x)
            got = h.apply_step_noalloc(level, call, x, torch.empty_like(x))
            assert torch.equal(got, ref), (level, call, float((got - ref).abs().max()))
    h.destroy()


def test_noalloc_allocates_no_device_memory():
    h = mg.mgrit_setup(1024, 1024, 3, 4, wave="sin_kx_cos_t", a=0.5, precision=1)
    x = torch.randn(64, 1024, dtype=torch.float64, device="cuda")
    out = torch.empty_like(x)
    for level in (0, 1, 2):  # the CUDA runtime may load each kernel's code on its first use
        h.apply_step_noalloc(level, 0, x, out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for level in (0, 1, 2, 1, 0):
        h.apply_step_noalloc(level, 0, x, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    h.destroy()


def test_noalloc_rejects_sizes_beyond_its_capacity():
    h = mg.mgrit_setup(1024, 4096, 1, 4, wave="const", precision=1)
    x = torch.zeros(1025, 1024, dtype=torch.float64, device="cuda")  # 1025 * 1024 > 2^20 values
    with pytest.raises(mg.MgritError) as e:
        h.apply_step_noalloc(0, 0, x, torch.empty_like(x))
    assert e.value.status == 1 and "capacity" in str(e.value)
    h.destroy()


def test_noalloc_binding_rejects_mismatched_buffers():
    h = mg.mgrit_setup(256, 256, 3, 4, wave="const", precision=1)
    x = torch.zeros(3, 256, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        h.apply_step_noalloc(0, 0, x, torch.empty(2, 256, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        h.apply_step_noalloc(0, 0, torch.zeros(3, 128, dtype=torch.float64, device="cuda"))
    h.destroy()
