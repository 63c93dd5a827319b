"""Small parity cases run against the index-checked build of libtga
(libtga_check.so: every indexed device access checked against its array's
extent).  Run as a child process by tests/test_gpu_index_checks.py, with
TGA_INDEX_CHECKS=1 so that the binding loads the checked library.

Every case compares the GPU path with the oracle (moves, solution, cost) and
then reads tga_get_bounds_report: a case passes only if the library reports
that it was built with the checks and that no check failed.  Prints one JSON
line: {"cases": [...], "ok": bool}.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2506_17357_gb300 import instances as I  # noqa: E402
from paper_2506_17357_gb300 import tga as T  # noqa: E402

assert os.path.basename(T.LIB_PATH) == "libtga_check.so", T.LIB_PATH


def _sol(tour, rs):
    return I.Solution(np.asarray(tour, np.int32), np.asarray(rs, np.int32))


def _case(kind, n, seed, extra_empty):
    if kind == "vrpspdtw":
        inst = I.vrpspdtw(n, seed)
    else:
        inst = I.vrptw(n, seed) if kind == "vrptw" else I.cvrp_uniform(n, seed)
    rng = np.random.default_rng(seed)
    if kind == "cvrp":
        inst.capacity = -(-int(inst.demand.sum()) // int(rng.integers(2, 6)))
    else:
        inst.capacity = int(rng.integers(60, 200))
    sol = I.random_split_solution(inst, seed + 17)
    rs = list(sol.route_start)
    for _ in range(extra_empty):
        at = int(rng.integers(0, len(rs)))
        rs.insert(at, rs[at] if at < len(rs) else n)
    rs = sorted(rs)
    rs[0], rs[-1] = 0, n
    return inst, _sol(sol.tour, rs)


def _report(ls):
    rep = T.tga_get_bounds_report(ls.ctx)
    assert rep["checked"], "the loaded library was built without index checks"
    assert rep["site"] == 0, f"index check failed: {rep}"
    return rep


def stepwise(inst, sol, mask, granular=None, max_steps=10 ** 6):
    """Evaluate / apply one step at a time, each step against the oracle."""
    ls = T.LocalSearch(inst, sol, mask, granular=granular).build()
    cur = sol.copy()
    steps = 0
    try:
        while steps < max_steps:
            mv = ls.eval_best_move()
            om = O.best_move(inst, cur, mask, "def", granular=granular)
            assert mv["valid"] == om["found"], (steps, mv, om)
            if not om["found"]:
                break
            assert (mv["delta"], mv["move_index"]) == (om["delta"], om["idx"]), (steps, mv, om)
            ls.apply_current_move()
            if om["delta"] >= 0:
                break
            cur = O.apply_move(inst, cur, om["op"], om["a"], om["b"])
            steps += 1
        tour, rs = ls.solution()
        assert np.array_equal(tour, cur.tour) and np.array_equal(rs, cur.route_start)
        st = ls.stats()
        assert st["status"] == 0, st
        _report(ls)
        return steps
    finally:
        ls.close()


def descent(inst, sol, mask, mode):
    """A whole descent on one path against the oracle's trajectory."""
    ls = T.LocalSearch(inst, sol, mask, log_capacity=1 << 14).build()
    try:
        ls.set_descent_mode(mode)
        st = ls.descend()
        final, steps, olog, _ = O.descend(inst, sol, mask, "def")
        assert st["status"] == 0, st
        assert st["steps"] == steps and np.array_equal(ls.move_log(), olog)
        tour, rs = ls.solution()
        assert np.array_equal(tour, final.tour) and np.array_equal(rs, final.route_start)
        _report(ls)
        return steps
    finally:
        ls.close()


def batch(jobs):
    """The batched launch on small jobs: each equals its single-job descent."""
    lss = [T.LocalSearch(inst, sol, I.mask_for(inst)) for inst, sol in jobs]
    try:
        stats = T.tga_descend_batch([ls.ctx for ls in lss])
        for ls, st, (inst, sol) in zip(lss, stats, jobs):
            final, steps, _, _ = O.descend(inst, sol, I.mask_for(inst), "def")
            assert st["status"] == 0 and st["steps"] == steps, st
            tour, rs = ls.solution()
            assert np.array_equal(tour, final.tour)
            _report(ls)
        return len(jobs)
    finally:
        for ls in lss:
            ls.close()


def main():
    cases = []

    def run(name, fn, *a, **k):
        cases.append({"case": name, "steps": int(fn(*a, **k))})

    rng = np.random.default_rng(4242)
    for kind in ("cvrp", "vrptw", "vrpspdtw"):
        for s in range(3):
            n = int(rng.integers(5, 61))
            inst, sol = _case(kind, n, 3100 + 10 * s + len(kind), extra_empty=int(rng.integers(0, 3)))
            run(f"stepwise {kind} n={n}", stepwise, inst, sol, I.MASK_ALL)
    for kind in ("cvrp", "vrptw"):
        inst, sol = _case(kind, 45, 3300 + len(kind), extra_empty=1)
        run(f"stepwise {kind} swaps of runs", stepwise, inst, sol, I.MASK_EXT | I.MASK_ALL)
        inst, sol = _case(kind, 50, 3400 + len(kind), extra_empty=2)
        nbr = I.granular_neighbors(inst, 6)
        run(f"stepwise {kind} granular theta=6", stepwise, inst, sol, I.MASK_ALL, granular=nbr)
    # routes longer than a warp (chunked scans) and than the intra tables (sweeps)
    inst = I.vrptw(105, 3)
    inst.capacity = 10 ** 6
    sol = I.random_split_solution(inst, 4)
    run("stepwise vrptw 35-customer routes", stepwise, inst, _sol(sol.tour, [0, 35, 70, 105, 105]), I.MASK_ALL,
        max_steps=20)
    cinst = I.cvrp_uniform(120, 9)
    cinst.capacity = int(cinst.demand.sum())
    csol = I.random_split_solution(cinst, 10)
    run("stepwise cvrp 60-customer routes", stepwise, cinst, _sol(csol.tour, [0, 60, 120]), I.MASK_ALL,
        max_steps=30)
    for mode, kind in ((T.DESCENT_PERSISTENT, "vrptw"), (T.DESCENT_GRAPH, "cvrp"), (T.DESCENT_HOST, "vrpspdtw"),
                       (T.DESCENT_PERSISTENT, "cvrp")):
        inst, sol = _case(kind, 120, 3500 + mode, extra_empty=1)
        run(f"descent {T.DESCENT_NAMES[mode]} {kind} n=120", descent, inst, sol, I.MASK_ALL, mode)
    jobs = []
    for j in range(4):
        inst = I.cvrp_uniform(60 + 20 * j, 3600 + j) if j % 2 == 0 else I.vrptw(60 + 20 * j, 3600 + j)
        jobs.append((inst, I.random_split_solution(inst, 3700 + j)))
    run("batched 4 jobs", batch, jobs)
    print(json.dumps({"cases": cases, "ok": True}))


if __name__ == "__main__":
    main()
