"""Batched descent (one persistent launch over many contexts) vs the
single-instance path and the oracle (marked gpu).  Exact equality of every
job's move log, final solution and counters."""
import numpy as np
import pytest

import oracle as O
from paper_2506_17357_gb300 import instances as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2506_17357_gb300 import tga as T  # noqa: E402


def _jobs(count, lo, hi, seed):
    sizes = I.uniform_int(I.splitmix64(seed, I.S_BATCH_SIZE, count), lo, hi)
    out = []
    for j in range(count):
        s = seed * 1000 + j
        inst = I.cvrp_uniform(int(sizes[j]), s) if j % 2 == 0 else I.vrptw(int(sizes[j]), s)
        sol = I.random_split_solution(inst, I.solution_seed(s))
        out.append((inst, sol, I.mask_for(inst)))
    return out


def _single(inst, sol, mask):
    ls = T.LocalSearch(inst, sol, mask, log_capacity=1 << 16).build()
    try:
        st = ls.descend()
        return st, ls.move_log(), ls.solution()
    finally:
        ls.close()


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_equals_single_instance(autotune):
    jobs = _jobs(24, 20, 400, seed=11 + int(autotune))
    stream = torch.cuda.Stream()
    lss = [T.LocalSearch(inst, sol, mask, stream=stream, log_capacity=1 << 16) for inst, sol, mask in jobs]
    try:
        ctxs = [ls.ctx for ls in lss]
        if autotune:
            rows = T.tga_batch_autotune(ctxs)
            assert all(r in (16, 32, 64) for r in rows)
        stats = T.tga_descend_batch(ctxs)
        for (inst, sol, mask), ls, st in zip(jobs, lss, stats):
            ref_st, ref_log, (ref_tour, ref_rs) = _single(inst, sol, mask)
            tour, rs = ls.solution()
            assert st["status"] == 0 and st["local_optimum"] == 1
            assert (st["steps"], st["candidates"], st["final_cost"]) == \
                   (ref_st["steps"], ref_st["candidates"], ref_st["final_cost"])
            assert np.array_equal(ls.move_log(), ref_log)
            assert np.array_equal(tour, ref_tour) and np.array_equal(rs, ref_rs)
    finally:
        for ls in lss:
            ls.close()


def test_batch_against_oracle_small():
    jobs = _jobs(10, 8, 60, seed=21)
    lss = [T.LocalSearch(inst, sol, mask, log_capacity=4096) for inst, sol, mask in jobs]
    try:
        T.tga_descend_batch([ls.ctx for ls in lss])
        for (inst, sol, mask), ls in zip(jobs, lss):
            final, steps, olog, _ = O.descend(inst, sol, mask, "def")
            assert np.array_equal(ls.move_log(), olog)
            tour, rs = ls.solution()
            assert np.array_equal(tour, final.tour) and np.array_equal(rs, final.route_start)
    finally:
        for ls in lss:
            ls.close()


def test_batch_step_limit_and_rerun():
    jobs = _jobs(6, 50, 200, seed=31)
    lss = [T.LocalSearch(inst, sol, mask) for inst, sol, mask in jobs]
    try:
        ctxs = [ls.ctx for ls in lss]
        st = T.tga_descend_batch(ctxs, max_steps=5)
        assert all(s["steps"] == 5 for s in st)
        st2 = T.tga_descend_batch(ctxs)           # resumes from the caller's (updated) solution
        for (inst, sol, mask), s in zip(jobs, st2):
            ref = _single(inst, sol, mask)[0]
            assert s["final_cost"] == ref["final_cost"] and s["steps"] == ref["steps"] - 5
    finally:
        for ls in lss:
            ls.close()
