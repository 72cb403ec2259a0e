"""The C-ABI library loads without a GPU and exports every entry point declared in include/mgrit_sl.h."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mgrit_sl.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mgrit_[a-z_]+|sl_step_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2203_13382_gb300 import build

    build.build()
    import paper_2203_13382_gb300 as mg

    return mg.load_library()


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("mgrit_setup", "mgrit_solve", "sl_step_sequential", "mgrit_adjoint_solve", "mgrit_destroy",
                     "mgrit_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2203_13382_gb300 import build

    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_binding_covers_every_declared_symbol():
    import paper_2203_13382_gb300 as mg

    assert sorted(mg._SIGNATURES) == declared_functions()


def test_host_only_calls(lib):
    import ctypes

    import paper_2203_13382_gb300 as mg

    o = mg.default_options()
    assert o.norm_mode == 1 and o.max_iter == 200 and abs(o.rtol - 1e-10) < 1e-25 and o.profile == 0
    assert mg.mgrit_status_string(0) == "ok"
    assert mg.mgrit_status_string(8) == "singular correction matrix"
    # argument errors are detected before any CUDA call
    g = mg.MgritGrid(1, 100, 64, -1.0, 1.0, 0.85)  # nx not a power of two
    w = mg.MgritWavespeed(0, 1.0, 1.0, 1.0)
    h = ctypes.c_void_p()
    st = lib.mgrit_setup(ctypes.byref(g), ctypes.byref(w), 1, 4, 0, None, None, ctypes.byref(h))
    assert st == 1 and b"power of two" in lib.mgrit_last_error()
    g = mg.MgritGrid(1, 64, 64, -1.0, 1.0, 0.85)
    assert lib.mgrit_setup(ctypes.byref(g), ctypes.byref(w), 2, 4, 0, None, None, ctypes.byref(h)) == 1  # even p
    assert lib.mgrit_setup(ctypes.byref(g), ctypes.byref(w), 3, 1, 0, None, None, ctypes.byref(h)) == 1  # m = 1
    w2 = mg.MgritWavespeed(11, 1.0, 1.0, 1.0)
    assert lib.mgrit_setup(ctypes.byref(g), ctypes.byref(w2), 3, 4, 0, None, None, ctypes.byref(h)) == 1  # 2D kind
    assert lib.mgrit_setup(ctypes.byref(g), ctypes.byref(w), 3, 4, 0, None, None, None) == 1
    g3 = mg.MgritGrid(1, 64, 96, -1.0, 1.0, 0.85)
    assert lib.mgrit_setup(ctypes.byref(g3), ctypes.byref(w), 3, 64, 3, None, None, ctypes.byref(h)) == 1


@pytest.mark.parametrize("field,value,status,msg", [
    ("precision", 2, 1, b"precision"),
    ("coarse_op", 2, 1, b"coarse_op"),
    ("norm_mode", 0, 7, b"norm_mode"),
    ("max_iter", 0, 1, b"max_iter"),
    ("rtol", 1.0, 1, b"rtol"),
    ("max_coarsest", 0, 1, b"max_coarsest"),
    ("m_first", 1, 1, b"m_first"),
    ("coarse_fp64", 1, 1, b"precision 1 only"),  # with the default precision 0
    ("gmres_maxit", 11, 1, b"gmres_maxit"),
    ("gmres_rtol", -0.5, 1, b"gmres_rtol"),
    ("relax", 2, 1, b"relax"),
    ("cluster_coarse", 3, 1, b"cluster_coarse"),
    ("diverge_ratio", -1.0, 1, b"diverge_ratio"),
    ("test_wait_cycles", -1, 1, b"test_wait_cycles"),
    ("fine_only", 2, 1, b"fine_only"),
    ("solve_mode", 3, 1, b"solve_mode"),
    ("coarse_band", 2, 1, b"coarse_band"),
])
def test_option_errors_are_reported_before_any_cuda_call(lib, field, value, status, msg):
    """Every option is range-checked by mgrit_setup before it touches the device (here: no GPU at all)."""
    import ctypes

    import paper_2203_13382_gb300 as mg

    o = mg.default_options()
    setattr(o, field, value)
    g = mg.MgritGrid(1, 64, 64, -1.0, 1.0, 0.85)
    w = mg.MgritWavespeed(0, 1.0, 1.0, 1.0)
    h = ctypes.c_void_p()
    assert lib.mgrit_setup(ctypes.byref(g), ctypes.byref(w), 3, 4, 0, ctypes.byref(o), None, ctypes.byref(h)) == status
    assert msg in lib.mgrit_last_error() and not h.value


def test_level_count_errors(lib):
    import ctypes

    import paper_2203_13382_gb300 as mg

    w = mg.MgritWavespeed(0, 1.0, 1.0, 1.0)
    h = ctypes.c_void_p()
    g = mg.MgritGrid(1, 64, 64, -1.0, 1.0, 0.85)
    assert lib.mgrit_setup(ctypes.byref(g), ctypes.byref(w), 3, 4, 1, None, None, ctypes.byref(h)) == 1
    assert b"levels" in lib.mgrit_last_error()
    g = mg.MgritGrid(1, 64, 24, -1.0, 1.0, 0.85)  # 24 -> 6 -> (not divisible by 4)
    assert lib.mgrit_setup(ctypes.byref(g), ctypes.byref(w), 3, 4, 4, None, None, ctypes.byref(h)) == 1
    assert b"divisible" in lib.mgrit_last_error()


def test_batched_setup_rejects_what_it_does_not_run(lib):
    """mgrit_setup_batched runs FP32 bulk, FCF, FP32 coarse levels, the corrected operator, 1D only; other
    requests are refused before any device work (no GPU here)."""
    import ctypes

    import paper_2203_13382_gb300 as mg

    grids = (mg.MgritGrid * 2)(mg.MgritGrid(1, 64, 64, -1.0, 1.0, 0.85), mg.MgritGrid(1, 128, 64, -1.0, 1.0, 0.85))
    waves = (mg.MgritWavespeed * 2)(mg.MgritWavespeed(0, 1.0, 1.0, 1.0), mg.MgritWavespeed(0, 1.0, 1.0, 1.0))
    orders = (ctypes.c_int * 2)(3, 1)
    ms = (ctypes.c_int * 2)(4, 4)
    b = ctypes.c_void_p()
    for field, value in (("precision", 0), ("relax", 1), ("coarse_fp64", 1), ("coarse_op", 1)):
        o = mg.default_options()
        o.precision = 1
        setattr(o, field, value)
        assert lib.mgrit_setup_batched(2, grids, waves, orders, ms, ctypes.byref(o), None, ctypes.byref(b)) == 7
        assert not b.value
    o = mg.default_options()
    o.precision = 1
    assert lib.mgrit_setup_batched(0, grids, waves, orders, ms, ctypes.byref(o), None, ctypes.byref(b)) == 1
    grids[1].dim = 2
    assert lib.mgrit_setup_batched(2, grids, waves, orders, ms, ctypes.byref(o), None, ctypes.byref(b)) == 7
    assert b"1D" in lib.mgrit_last_error()


def test_null_handles_are_argument_errors(lib):
    """Every call that takes a handle returns MGRIT_EINVAL for a null one; the destroy calls accept it."""
    import ctypes

    import paper_2203_13382_gb300 as mg

    st = mg.MgritStats()
    a, b = ctypes.c_int(), ctypes.c_int()
    calls = [
        lambda: lib.mgrit_solve(None, None, None, None, ctypes.byref(st)),
        lambda: lib.sl_step_sequential(None, None, None, 0),
        lambda: lib.mgrit_solve_host(None, None, None, None, ctypes.byref(st)),
        lambda: lib.mgrit_solve_to_reference(None, None, None, None, None, 0.0, ctypes.byref(st)),
        lambda: lib.mgrit_adjoint_solve(None, None, None, None, None, ctypes.byref(st)),
        lambda: lib.mgrit_level_info(None, 0, ctypes.byref(a), ctypes.byref(b)),
        lambda: lib.mgrit_level_band(None, 0, ctypes.byref(a), None),
        lambda: lib.mgrit_copy_offsets(None, 0, None),
        lambda: lib.mgrit_copy_sigma(None, 0, None),
        lambda: lib.mgrit_apply_step(None, 0, 0, 1, None, None),
        lambda: lib.mgrit_apply_step_noalloc(None, 0, 0, 1, None, None),
        lambda: lib.mgrit_solve_batched(None, None, None, None, None),
        lambda: lib.mgrit_default_options(None),
    ]
    assert [c() for c in calls] == [1] * len(calls)
    lib.mgrit_destroy(None)
    lib.mgrit_destroy_batched(None)
    assert lib.mgrit_status_string(99) == b"unknown status"


def test_struct_layouts_match_the_header(tmp_path):
    """ctypes mirrors of the C structs have the C sizes and field offsets (compiled with gcc here)."""
    import ctypes
    import shutil

    import paper_2203_13382_gb300 as mg

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "mgrit_sl.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(mgrit_grid), sizeof(mgrit_wavespeed),"
        " sizeof(mgrit_options), sizeof(mgrit_stats), offsetof(mgrit_stats, device_bytes),"
        " offsetof(mgrit_stats, phase_ms), offsetof(mgrit_options, profile));return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(mg.MgritGrid), ctypes.sizeof(mg.MgritWavespeed), ctypes.sizeof(mg.MgritOptions),
            ctypes.sizeof(mg.MgritStats), mg.MgritStats.device_bytes.offset, mg.MgritStats.phase_ms.offset,
            mg.MgritOptions.profile.offset]
    assert got == want
