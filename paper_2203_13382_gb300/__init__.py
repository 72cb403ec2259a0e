"""Python binding of libmgrit_sl.so: MGRIT with modified semi-Lagrangian coarse-grid operators on GB300.

A thin ctypes layer over the C ABI declared in include/mgrit_sl.h; every computation runs in the
library's CUDA kernels.  PyTorch supplies device memory and the CUDA stream.  There is no CPU fallback:
the first call raises ImportError if the library has not been built (call `build.build()`), and solver
calls fail if no GPU is present.
"""

from __future__ import annotations

import ctypes
import os

from . import build as _build

WAVE_KINDS = {
    "const": 0,
    "cos_t": 1,
    "cos_t_cos_x": 2,
    "sin_kx_cos_t": 3,
    "const2": 10,
    "paper2": 11,
    "sin_cos2": 12,
}

STATUS = {
    0: "MGRIT_OK",
    1: "MGRIT_EINVAL",
    2: "MGRIT_ENOMEM",
    3: "MGRIT_ECUDA",
    4: "MGRIT_ENOTCONVERGED",
    5: "MGRIT_EDIVERGED",
    6: "MGRIT_ETIMEOUT",
    7: "MGRIT_EUNSUPPORTED",
    8: "MGRIT_ESINGULAR",
}


class MgritGrid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("nt", ctypes.c_int), ("xmin", ctypes.c_double),
                ("xmax", ctypes.c_double), ("cfl", ctypes.c_double)]


class MgritWavespeed(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("a", ctypes.c_double), ("k", ctypes.c_double), ("a2", ctypes.c_double)]


class MgritOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("coarse_op", ctypes.c_int), ("norm_mode", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("rtol", ctypes.c_double), ("max_coarsest", ctypes.c_int),
                ("m_first", ctypes.c_int), ("coarse_fp64", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("profile", ctypes.c_int), ("gmres_maxit", ctypes.c_int), ("gmres_rtol", ctypes.c_double),
                ("relax", ctypes.c_int), ("cluster_coarse", ctypes.c_int), ("diverge_ratio", ctypes.c_double),
                ("fine_only", ctypes.c_int), ("solve_mode", ctypes.c_int), ("coarse_band", ctypes.c_int),
                ("test_wait_cycles", ctypes.c_int)]


PHASES = ["departure", "backtrack", "tables", "factor", "fine64_fc", "fine64_res", "fine64_post", "fine32_res",
          "coarse", "coarsest", "misc", "sequential"]


class MgritStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("levels", ctypes.c_int),
                ("history_len", ctypes.c_int), ("r0", ctypes.c_double), ("r_final", ctypes.c_double),
                ("residual_history", ctypes.c_double * 256), ("setup_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("phase_ms", ctypes.c_double * 12),
                ("phase_launches", ctypes.c_int * 12), ("final_error", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {
            "iterations": self.iterations,
            "converged": bool(self.converged),
            "levels": self.levels,
            "r0": self.r0,
            "r_final": self.r_final,
            "history": list(self.residual_history[: self.history_len]),
            "setup_ms": self.setup_ms,
            "solve_ms": self.solve_ms,
            "device_bytes": self.device_bytes,
            "kernel_launches": self.kernel_launches,
            "phase_ms": {PHASES[i]: self.phase_ms[i] for i in range(12)},
            "phase_launches": {PHASES[i]: self.phase_launches[i] for i in range(12)},
            "final_error": self.final_error,
        }


# every entry point of include/mgrit_sl.h: name -> (restype, argtypes)
_VP = ctypes.c_void_p
_SIGNATURES = {
    "mgrit_default_options": (ctypes.c_int, [ctypes.POINTER(MgritOptions)]),
    "mgrit_setup": (ctypes.c_int, [ctypes.POINTER(MgritGrid), ctypes.POINTER(MgritWavespeed), ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, ctypes.POINTER(MgritOptions), _VP,
                                   ctypes.POINTER(_VP)]),
    "mgrit_solve": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.POINTER(MgritStats)]),
    "sl_step_sequential": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int]),
    "mgrit_solve_host": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.POINTER(MgritStats)]),
    "mgrit_solve_to_reference": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_double,
                                                ctypes.POINTER(MgritStats)]),
    "mgrit_adjoint_solve": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.POINTER(MgritStats)]),
    "mgrit_level_info": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int)]),
    "mgrit_level_band": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _VP]),
    "mgrit_copy_offsets": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    "mgrit_copy_sigma": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    "mgrit_apply_step": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP]),
    "mgrit_apply_step_noalloc": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP]),
    "mgrit_destroy": (None, [_VP]),
    "mgrit_setup_batched": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(MgritGrid), ctypes.POINTER(MgritWavespeed),
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(MgritOptions), _VP, ctypes.POINTER(_VP)]),
    "mgrit_solve_batched": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                           ctypes.POINTER(MgritStats)]),
    "mgrit_solve_batched_host": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                                ctypes.POINTER(MgritStats)]),
    "sl_step_sequential_batched": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
    "mgrit_destroy_batched": (None, [_VP]),
    "mgrit_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mgrit_last_error": (ctypes.c_char_p, []),
}

_LIB = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Loads libmgrit_sl.so (in-tree) and binds every C-ABI entry point."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or _build.LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"{p} is missing: build it with paper_2203_13382_gb300.build.build() (needs nvcc)")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _LIB = lib
    return lib


class MgritError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load_library()
        msg = lib.mgrit_last_error().decode() if status != 0 else ""
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(status: int, where: str, allow=()) -> int:
    if status != 0 and status not in allow:
        raise MgritError(status, where)
    return status


def _ptr(t) -> int | None:
    if t is None:
        return None
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("device buffers must be contiguous float64 CUDA tensors")
    return t.data_ptr()


def default_options(**overrides) -> MgritOptions:
    o = MgritOptions()
    _check(load_library().mgrit_default_options(ctypes.byref(o)), "mgrit_default_options")
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class Handle:
    """An MGRIT problem set up on the GPU (owns the device workspace)."""

    def __init__(self, ptr: int, grid: MgritGrid, order: int, options: MgritOptions):
        self._ptr = ptr
        self.grid = grid
        self.order = order
        self.options = options
        self.npts = grid.nx ** grid.dim

    def _h(self) -> int:
        if not self._ptr:
            raise RuntimeError("handle already destroyed")
        return self._ptr

    def destroy(self) -> None:
        if self._ptr:
            load_library().mgrit_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def level_info(self, level: int) -> tuple[int, int]:
        nt = ctypes.c_int()
        m = ctypes.c_int()
        _check(load_library().mgrit_level_info(self._h(), level, ctypes.byref(nt), ctypes.byref(m)), "level_info")
        return nt.value, m.value

    def level_band(self, level: int, decay: bool = False):
        """Half-width of the banded separator inverse of this level's FP32 correction solves (0: none);
        with decay=True also the probed decay at partition distances 1..4 (a list of 4 floats)."""
        w = ctypes.c_int()
        d = (ctypes.c_float * 4)()
        _check(load_library().mgrit_level_band(self._h(), level, ctypes.byref(w), d), "mgrit_level_band")
        return (w.value, list(d)) if decay else w.value

    @property
    def nlevels(self) -> int:
        nt = ctypes.c_int()
        load_library().mgrit_level_info(self._h(), -1, ctypes.byref(nt), None)
        return nt.value

    def _empty(self, *shape):
        import torch

        return torch.empty(*shape, dtype=torch.float64, device="cuda")

    def offsets(self, level: int):
        nt, _ = self.level_info(level)
        out = self._empty(self.grid.dim * nt, self.npts)
        _check(load_library().mgrit_copy_offsets(self._h(), level, _ptr(out)), "mgrit_copy_offsets")
        return out

    def sigma(self, level: int):
        nt, _ = self.level_info(level)
        out = self._empty(self.grid.dim * nt, self.npts)
        _check(load_library().mgrit_copy_sigma(self._h(), level, _ptr(out)), "mgrit_copy_sigma")
        return out

    def _check_slices(self, slices, out=None) -> None:
        """The C calls read and write count * npts values: refuse tensors of any other shape."""
        if slices.ndim != 2 or slices.shape[1] != self.npts:
            raise ValueError(f"slices must have shape (count, {self.npts}), got {tuple(slices.shape)}")
        if out is not None and (tuple(out.shape) != tuple(slices.shape) or out.device != slices.device):
            raise ValueError(f"out must have the shape and device of slices, got {tuple(out.shape)} on {out.device}")

    def apply_step(self, level: int, n0: int, slices):
        self._check_slices(slices)
        out = self._empty(*slices.shape)
        count = slices.shape[0]
        _check(load_library().mgrit_apply_step(self._h(), level, n0, count, _ptr(slices), _ptr(out)),
               "mgrit_apply_step")
        return out

    def apply_step_noalloc(self, level: int, n0: int, slices, out=None):
        """apply_step for callers that cannot allocate device memory: the library allocates nothing, and
        `out` (if given) must be preallocated by the caller."""
        self._check_slices(slices, out)
        if out is None:
            out = self._empty(*slices.shape)
        _check(load_library().mgrit_apply_step_noalloc(self._h(), level, n0, slices.shape[0], _ptr(slices),
                                                        _ptr(out)), "mgrit_apply_step_noalloc")
        return out

    def solve(self, u0, u_init=None, u_out=None, allow_not_converged: bool = False):
        if u_out is None:
            u_out = self._empty(self.grid.nt + 1, self.npts)
        st = MgritStats()
        allow = (4, 5) if allow_not_converged else ()  # not converged / diverged: stats still filled
        _check(load_library().mgrit_solve(self._h(), _ptr(u0), _ptr(u_init), _ptr(u_out), ctypes.byref(st)),
               "mgrit_solve", allow)
        return u_out, st.as_dict()

    def solve_to_reference(self, u0, u_final_ref, tol: float, u_init=None, u_out=None,
                           allow_not_converged: bool = False):
        """MGRIT until the final slice is within tol of u_final_ref (discrete l2 norm; Sec. SM4)."""
        if u_out is None:
            u_out = self._empty(self.grid.nt + 1, self.npts)
        st = MgritStats()
        allow = (4,) if allow_not_converged else ()
        _check(load_library().mgrit_solve_to_reference(self._h(), _ptr(u0), _ptr(u_init), _ptr(u_out),
                                                       _ptr(u_final_ref), float(tol), ctypes.byref(st)),
               "mgrit_solve_to_reference", allow)
        return u_out, st.as_dict()

    def solve_host(self, u0, u_init=None, u_out=None):
        """End-to-end solve from host (numpy float64) arrays: copies in, solves, copies back."""
        import numpy as np

        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        if u_init is not None:
            u_init = np.ascontiguousarray(u_init, dtype=np.float64)
        if u_out is None:
            u_out = np.empty((self.grid.nt + 1, self.npts))
        st = MgritStats()
        vp = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        _check(load_library().mgrit_solve_host(self._h(), vp(u0), vp(u_init), vp(u_out), ctypes.byref(st)),
               "mgrit_solve_host")
        return u_out, st.as_dict()

    def adjoint(self, u_target, checkpoints):
        """Discrete adjoint (mgrit_adjoint_solve): returns (dJ/du0, dJ/da, stats of the adjoint MGRIT); both
        gradients are CUDA tensors (dJ/da of shape [1])."""
        dJdu0 = self._empty(self.npts)
        dJda = self._empty(1)
        st = MgritStats()
        _check(load_library().mgrit_adjoint_solve(self._h(), _ptr(u_target), _ptr(checkpoints), _ptr(dJdu0),
                                                   _ptr(dJda), ctypes.byref(st)), "mgrit_adjoint_solve")
        return dJdu0, dJda, st.as_dict()

    def sequential(self, u0, u_out=None, store_all: bool = True):
        if u_out is None:
            u_out = self._empty(self.grid.nt + 1, self.npts) if store_all else self._empty(self.npts)
        _check(load_library().sl_step_sequential(self._h(), _ptr(u0), _ptr(u_out), 1 if store_all else 0),
               "sl_step_sequential")
        return u_out


def mgrit_setup(nx: int, nt: int, order: int, m: int, wave: str = "const", a: float = 1.0, k: float = 1.0,
                a2: float = 1.0, levels: int = 0, dim: int = 1, cfl: float = 0.85, xmin: float = -1.0,
                xmax: float = 1.0, stream=None, **options) -> Handle:
    """Set up a problem (see mgrit_setup in include/mgrit_sl.h); options are mgrit_options fields."""
    import torch

    g = MgritGrid(dim, nx, nt, xmin, xmax, cfl)
    w = MgritWavespeed(WAVE_KINDS[wave] if isinstance(wave, str) else int(wave), a, k, a2)
    o = default_options(**options)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    out = ctypes.c_void_p()
    _check(load_library().mgrit_setup(ctypes.byref(g), ctypes.byref(w), order, m, levels, ctypes.byref(o),
                                      ctypes.c_void_p(stream), ctypes.byref(out)), "mgrit_setup")
    return Handle(out.value, g, order, o)


class Batch:
    """Independent 1D problems solved together (mgrit_setup_batched / mgrit_solve_batched)."""

    def __init__(self, ptr: int, grids: list, options: MgritOptions):
        self._ptr = ptr
        self.grids = grids
        self.options = options

    def destroy(self) -> None:
        if self._ptr:
            load_library().mgrit_destroy_batched(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def solve(self, u0_list, u_init_list=None, out_list=None):
        import torch

        n = len(self.grids)
        if out_list is None:
            out_list = [torch.empty(g.nt + 1, g.nx, dtype=torch.float64, device="cuda") for g in self.grids]
        arr = lambda ts: (_VP * n)(*[_ptr(t) for t in ts])  # noqa: E731
        st = (MgritStats * n)()
        init = arr(u_init_list) if u_init_list is not None else None
        _check(load_library().mgrit_solve_batched(self._ptr, arr(u0_list), init, arr(out_list), st),
               "mgrit_solve_batched")
        return out_list, [s.as_dict() for s in st]

    def solve_host(self, u0_list, u_init_c_list=None, out_list=None):
        """End-to-end batched solve from host (numpy float64) arrays: u_init_c_list[q] holds the initial iterate
        at the C-points only ((nt/m_1 + 1) x nx, row 0 ignored); returns the full solutions (host arrays)."""
        import numpy as np

        n = len(self.grids)
        c = lambda a: np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
        u0_list = [c(a) for a in u0_list]
        if u_init_c_list is not None:
            u_init_c_list = [c(a) for a in u_init_c_list]
        if out_list is None:
            out_list = [np.empty((g.nt + 1, g.nx)) for g in self.grids]
        vp = lambda al: (_VP * n)(*[a.ctypes.data for a in al])  # noqa: E731
        st = (MgritStats * n)()
        init = vp(u_init_c_list) if u_init_c_list is not None else None
        _check(load_library().mgrit_solve_batched_host(self._ptr, vp(u0_list), init, vp(out_list), st),
               "mgrit_solve_batched_host")
        return out_list, [s.as_dict() for s in st]

    def sequential(self, u0_list, out_list=None):
        """sl_step_sequential_batched: the final slice of every problem by sequential SL stepping (FP32)."""
        import torch

        n = len(self.grids)
        if out_list is None:
            out_list = [torch.empty(g.nx, dtype=torch.float64, device="cuda") for g in self.grids]
        arr = lambda ts: (_VP * n)(*[_ptr(t) for t in ts])  # noqa: E731
        _check(load_library().sl_step_sequential_batched(self._ptr, arr(u0_list), arr(out_list)),
               "sl_step_sequential_batched")
        return out_list


def mgrit_setup_batched(problems: list, stream=None, **options) -> Batch:
    """problems: dicts with nx, nt, order, m and optionally wave, a, k, cfl (1D); options as mgrit_setup."""
    import torch

    n = len(problems)
    grids = (MgritGrid * n)(*[MgritGrid(1, p["nx"], p["nt"], -1.0, 1.0, p.get("cfl", 0.85)) for p in problems])
    waves = (MgritWavespeed * n)(*[MgritWavespeed(WAVE_KINDS[p.get("wave", "sin_kx_cos_t")], p.get("a", 1.0),
                                                  p.get("k", 1.0), 1.0) for p in problems])
    orders = (ctypes.c_int * n)(*[p["order"] for p in problems])
    ms = (ctypes.c_int * n)(*[p["m"] for p in problems])
    options.setdefault("precision", 1)
    o = default_options(**options)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    out = ctypes.c_void_p()
    _check(load_library().mgrit_setup_batched(n, grids, waves, orders, ms, ctypes.byref(o), ctypes.c_void_p(stream),
                                              ctypes.byref(out)), "mgrit_setup_batched")
    return Batch(out.value, list(grids), o)


def mgrit_solve(handle: Handle, u0, u_init=None, u_out=None):
    return handle.solve(u0, u_init, u_out)


def sl_step_sequential(handle: Handle, u0, u_out=None, store_all: bool = True):
    return handle.sequential(u0, u_out, store_all)


def mgrit_destroy(handle: Handle) -> None:
    handle.destroy()


def mgrit_status_string(status: int) -> str:
    return load_library().mgrit_status_string(status).decode()

