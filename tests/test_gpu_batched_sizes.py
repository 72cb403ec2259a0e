"""The batched solve at the sizes of the 256-problem workload.

- Against the oracle: a batch whose problems span nx = 512 .. 4096 (the FP32 CTA classes of 64, 128, 256
  and 512 threads, one thread per 8 slice points, and the tuner's doublings), p = 1, 3, 5, m = 4, 8 and
  four to six levels.  Every problem equals its own mgrit_solve and the oracle (FP32-bulk tolerance 1e-5,
  identical iteration counts).  The oracle solves run in a process pool started with `spawn`.
- At full size: the 256-problem workload itself (2.8e9 space-time unknowns).  Every problem converges; its
  final slice equals the FP64 sequential solution of its own one-step system (sl_step_sequential, pinned to
  the oracle at full size elsewhere) to 1e-8 of the solution's scale, as an FP64 iterate at a 1e-10 residual
  must; the largest
  problem equals its own single-problem solve; and the FP64 batched sequential stepping equals the
  single-problem FP64 stepping.
"""

import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest

import oracle_jobs
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2203_13382_gb300 as mg  # noqa: E402

# nx 4096 / 2048 / 1024 / 512: FP32 CTA classes of 512 / 256 / 128 / 64 threads
PROBLEMS = [
    dict(nx=4096, nt=512, order=3, m=8, a=0.5, k=2.0),    # levels 512/64/8/1
    dict(nx=2048, nt=512, order=5, m=4, a=0.35, k=1.0),   # 512/128/32/8/2
    dict(nx=1024, nt=1024, order=1, m=8, a=0.7, k=3.0),   # 1024/128/16/2
    dict(nx=512, nt=2048, order=3, m=4, a=0.6, k=2.0),    # 2048/512/128/32/8/2
    dict(nx=4096, nt=256, order=5, m=4, a=0.2, k=3.0),    # 256/64/16/4/1
]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_batched_at_workload_sizes_equals_individual_solves_and_the_oracle():
    with cf.ProcessPoolExecutor(max_workers=len(PROBLEMS), mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(oracle_jobs.solve_batched_problem, p, q) for q, p in enumerate(PROBLEMS)]
        u0s = [W.u0_sin4(p["nx"]) for p in PROBLEMS]
        U0s = [W.initial_iterate(p["nt"], p["nx"], seed=W.SEED_INITIAL_ITERATE + q) for q, p in enumerate(PROBLEMS)]
        b = mg.mgrit_setup_batched(PROBLEMS)
        outs, stats = b.solve([torch.from_numpy(u).cuda() for u in u0s], [torch.from_numpy(U).cuda() for U in U0s])
        got = [o.cpu().numpy() for o in outs]
        b.destroy()
        for q, p in enumerate(PROBLEMS):
            h = mg.mgrit_setup(p["nx"], p["nt"], p["order"], p["m"], wave="sin_kx_cos_t", a=p["a"], k=p["k"],
                               precision=1)
            ref, st = h.solve(torch.from_numpy(u0s[q]).cuda(), torch.from_numpy(U0s[q]).cuda())
            h.destroy()
            assert stats[q]["iterations"] == st["iterations"] and stats[q]["converged"], q
            assert rel(got[q], ref.cpu().numpy()) < 1e-13, q
        for q, f in enumerate(futs):
            its, U, levels = f.result()
            assert stats[q]["levels"] == len(levels)
            assert stats[q]["iterations"] == its, (q, stats[q]["iterations"], its)
            assert rel(got[q], U) < 1e-5, (q, rel(got[q], U))


def test_full_batched_workload_reaches_every_problems_fp64_solution():
    probs = W.batched_problems(256)
    specs = [dict(nx=q.nx, nt=q.nt, order=q.order, m=q.m, a=q.a, k=float(q.k)) for q in probs]
    u0s = [torch.from_numpy(W.u0_sin4(q.nx)).cuda() for q in probs]
    inits = []
    for q in probs:
        U = torch.zeros(q.nt + 1, q.nx, dtype=torch.float64, device="cuda")
        rows = np.arange(q.m, q.nt + 1, q.m)  # the solver reads the C-points only
        U[torch.from_numpy(rows).cuda()] = torch.from_numpy(W.initial_iterate(q.nt, q.nx, rows=rows)).cuda()
        inits.append(U)
    b = mg.mgrit_setup_batched(specs)
    outs, stats = b.solve(u0s, inits)
    b.destroy()
    assert all(st["converged"] for st in stats)
    finals = [o[-1].clone() for o in outs]
    big = int(np.argmax([q.nx * q.nt for q in probs]))
    qb = probs[big]
    h = mg.mgrit_setup(qb.nx, qb.nt, qb.order, qb.m, wave="sin_kx_cos_t", a=qb.a, k=float(qb.k), precision=1)
    ref, st = h.solve(u0s[big], inits[big])
    h.destroy()
    assert st["iterations"] == stats[big]["iterations"]
    assert rel(outs[big].cpu().numpy(), ref.cpu().numpy()) < 1e-13
    del outs, ref
    worst = 0.0
    for q, p in enumerate(probs):
        h = mg.mgrit_setup(p.nx, p.nt, p.order, p.m, wave="sin_kx_cos_t", a=p.a, k=float(p.k), precision=0,
                           fine_only=1)
        seq = h.sequential(u0s[q], store_all=False)
        h.destroy()
        # measured against the solution's scale: some final slices have decayed far below it (a relative
        # difference of 1e-6 at |u(T)| = 3e-3 |u0| is an absolute 3e-9, the oracle's own MGRIT gives the same)
        f, r = finals[q].cpu().numpy(), seq.cpu().numpy()
        e = float(np.linalg.norm(f - r) / max(np.linalg.norm(r), np.linalg.norm(u0s[q].cpu().numpy())))
        worst = max(worst, e)
        assert e < 1e-8, (q, p, e)
    print(f"largest difference of a final slice from FP64 sequential stepping (scale max(|u(T)|, |u0|)): {worst:.2e}")


def test_fp64_batched_sequential_equals_single_problem_stepping():
    probs = W.batched_problems(256)[:12]
    specs = [dict(nx=q.nx, nt=q.nt, order=q.order, m=q.m, a=q.a, k=float(q.k)) for q in probs]
    u0s = [torch.from_numpy(W.u0_sin4(q.nx)).cuda() for q in probs]
    b = mg.mgrit_setup_batched(specs, precision=0, fine_only=1)
    got = b.sequential(u0s)
    with pytest.raises(mg.MgritError) as e:
        b.solve(u0s)
    assert e.value.status == 7  # a fine_only batch has no hierarchy
    b.destroy()
    for q, p in enumerate(probs):
        h = mg.mgrit_setup(p.nx, p.nt, p.order, p.m, wave="sin_kx_cos_t", a=p.a, k=float(p.k), precision=0)
        ref = h.sequential(u0s[q], store_all=False)
        h.destroy()
        assert rel(got[q].cpu().numpy(), ref.cpu().numpy()) < 1e-13, q
