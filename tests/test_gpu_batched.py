"""Batched independent problems (one launch per cycle phase): every problem of a heterogeneous batch gives
the result of its own mgrit_solve (same kernels, same order: identical iterates) and matches the oracle
(FP32-bulk tolerance 1e-5, identical iteration counts)."""

import numpy as np
import pytest

import workloads as W
from oracle import mgrit as omg
from oracle import semi_lagrangian as osl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2203_13382_gb300 as mg  # noqa: E402

PROBLEMS = [
    dict(nx=64, nt=256, order=1, m=4, a=0.3, k=1.0),
    dict(nx=128, nt=512, order=3, m=8, a=0.6, k=2.0),
    dict(nx=256, nt=128, order=5, m=4, a=0.2, k=3.0),
    dict(nx=64, nt=1024, order=3, m=4, a=0.7, k=1.0),
    dict(nx=128, nt=256, order=5, m=8, a=0.45, k=2.0),
    dict(nx=256, nt=512, order=1, m=8, a=0.1, k=3.0),
]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def inputs(p, q):
    u0 = W.u0_sin4(p["nx"])
    U0 = W.initial_iterate(p["nt"], p["nx"], seed=W.SEED_INITIAL_ITERATE + q)
    return u0, U0


def test_batched_equals_individual_solves_and_the_oracle():
    b = mg.mgrit_setup_batched(PROBLEMS)
    u0s, U0s = zip(*[inputs(p, q) for q, p in enumerate(PROBLEMS)])
    outs, stats = b.solve([torch.from_numpy(u).cuda() for u in u0s], [torch.from_numpy(U).cuda() for U in U0s])
    for q, p in enumerate(PROBLEMS):
        h = mg.mgrit_setup(p["nx"], p["nt"], p["order"], p["m"], wave="sin_kx_cos_t", a=p["a"], k=p["k"], precision=1)
        ref, st = h.solve(torch.from_numpy(u0s[q]).cuda(), torch.from_numpy(U0s[q]).cuda())
        assert stats[q]["iterations"] == st["iterations"] and stats[q]["converged"]
        assert rel(outs[q].cpu().numpy(), ref.cpu().numpy()) < 1e-13
        H = omg.build_hierarchy(osl.Grid(p["nx"], p["nt"]), osl.WaveSpeed("sin_kx_cos_t", a=p["a"], k=p["k"]),
                                p["order"], p["m"])
        R = omg.mgrit_solve(H, u0s[q], U0s[q])
        assert stats[q]["iterations"] == R.iterations
        assert rel(outs[q].cpu().numpy(), R.U) < 1e-5
    b.destroy()


def test_batched_workload_generator_is_valid():
    probs = W.batched_problems(256)
    assert len(probs) == 256
    for p in probs:
        assert p.nx in (256, 512, 1024, 2048, 4096) and p.nt in (1024, 2048, 4096, 8192, 16384)
        assert p.order in (1, 3, 5) and p.m in (4, 8) and 0.1 <= p.a <= 0.7 and p.k in (1, 2, 3)
