"""Oracle runs that tests hand to a process pool (started with `spawn`); this module imports neither
torch nor the CUDA library, so the pool's workers stay CPU-only."""

import workloads as W


def solve_batched_problem(p: dict, q: int):
    """The oracle's MGRIT solve of one 1D problem alpha = 1 + a sin(2 pi k x) cos(2 pi t), u0 = sin^4(pi x),
    random initial iterate of seed SEED_INITIAL_ITERATE + q: (iterations, solution, steps per level)."""
    from oracle import mgrit as omg
    from oracle import semi_lagrangian as osl

    H = omg.build_hierarchy(osl.Grid(p["nx"], p["nt"]), osl.WaveSpeed("sin_kx_cos_t", a=p["a"], k=p["k"]),
                            p["order"], p["m"])
    R = omg.mgrit_solve(H, W.u0_sin4(p["nx"]), W.initial_iterate(p["nt"], p["nx"], seed=W.SEED_INITIAL_ITERATE + q))
    return R.iterations, R.U, [lv.nt for lv in H.levels]


def table_cell_iterations(speed: str, p: int, m: int, levels: int) -> int:
    """Iterations of the oracle's MGRIT on the paper's table problem (Sec. 3.3 / 3.4: nx = 256, nt = 1024,
    u0 = sin^4(pi x), the shared random initial iterate) with wave speed `speed`, order p, factor m."""
    from oracle import mgrit as omg
    from oracle import semi_lagrangian as osl

    nx, nt = 256, 1024
    H = omg.build_hierarchy(osl.Grid(nx, nt), osl.WaveSpeed(speed), p, m, levels=levels)
    return omg.mgrit_solve(H, W.u0_sin4(nx), W.initial_iterate(nt, nx)).iterations
