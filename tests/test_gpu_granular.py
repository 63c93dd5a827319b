"""Edge-based extraction (granular mask, Section 5.3.1) on the GPU vs the
oracle restricted to the same candidate set (marked gpu).

Bit-exact: every evaluation's (delta, move index) and its number of kept
candidates equal the oracle's, whole trajectories give the same move log,
solution and candidate total, and the 1000-customer VRPTW trajectory is
re-evaluated by the oracle at every step.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle as O
from paper_2506_17357_gb300 import instances as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2506_17357_gb300 import tga as T  # noqa: E402
from paper_2506_17357_gb300.tga import LocalSearch, TGAError  # noqa: E402


def _sol(tour, rs):
    return I.Solution(np.asarray(tour, np.int32), np.asarray(rs, np.int32))


def _case(kind, n, seed, extra_empty):
    inst = I.vrptw(n, seed) if kind == "vrptw" else I.cvrp_uniform(n, seed)
    rng = np.random.default_rng(seed)
    inst.capacity = int(rng.integers(60, 200)) if kind == "vrptw" else -(-int(inst.demand.sum()) // int(rng.integers(2, 6)))
    sol = I.random_split_solution(inst, seed + 17)
    rs = list(sol.route_start)
    for _ in range(extra_empty):
        at = int(rng.integers(0, len(rs)))
        rs.insert(at, rs[at] if at < len(rs) else n)
    rs = sorted(rs)
    rs[0], rs[-1] = 0, n
    return inst, _sol(sol.tour, rs)


@pytest.mark.parametrize("kind", ["cvrp", "vrptw"])
@pytest.mark.parametrize("seed", range(5))
def test_granular_stepwise_small_random(kind, seed):
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(6, 61))
    theta = int(rng.integers(1, min(12, n - 1) + 1))
    inst, sol = _case(kind, n, 900 + seed, extra_empty=int(rng.integers(0, 3)))
    nbr = I.granular_neighbors(inst, theta)
    ls = LocalSearch(inst, sol, I.MASK_ALL, granular=nbr).build()
    cur = sol.copy()
    steps = 0
    try:
        while True:
            before = ls.stats()["candidates"]
            mv = ls.eval_best_move()
            om = O.best_move(inst, cur, I.MASK_ALL, "def", granular=nbr)
            assert ls.stats()["candidates"] - before == om["candidates"], steps
            assert mv["valid"] == om["found"]
            if not om["found"]:
                break
            assert (mv["delta"], mv["move_index"]) == (om["delta"], om["idx"]), (steps, mv, om)
            ls.apply_current_move()
            if om["delta"] >= 0:
                break
            cur = O.apply_move(inst, cur, om["op"], om["a"], om["b"])
            tour, rs = ls.solution()
            assert np.array_equal(tour, cur.tour) and np.array_equal(rs, cur.route_start), steps
            steps += 1
        st = ls.stats()
        assert st["status"] == 0 and st["steps"] == steps
        assert st["final_cost"] == O.solution_cost(inst, cur)
    finally:
        ls.close()


@pytest.mark.parametrize("case", [("vrptw", 200, 10), ("cvrp", 300, 15), ("cvrp", 150, 1)])
def test_granular_full_trajectory(case):
    kind, n, theta = case
    inst = I.vrptw(n, 5) if kind == "vrptw" else I.cvrp_uniform(n, 5)
    sol = I.random_split_solution(inst, I.solution_seed(5))
    mask = I.mask_for(inst)
    nbr = I.granular_neighbors(inst, theta)
    ls = LocalSearch(inst, sol, mask, log_capacity=1 << 16, granular=nbr).build()
    try:
        ls.set_tile(0, 0)
        st = ls.descend()
        assert ls.descent_mode()[0] == T.DESCENT_GRAPH
        log = ls.move_log()
        tour, rs = ls.solution()
        ops = T.tga_get_op_candidates(ls.ctx)
    finally:
        ls.close()
    fin, steps, olog, ocands = O.descend(inst, sol, mask, "concat", granular=nbr)
    assert st["status"] == 0 and st["local_optimum"] == 1
    assert st["steps"] == steps and np.array_equal(log, olog)
    assert np.array_equal(tour, fin.tour) and np.array_equal(rs, fin.route_start)
    assert st["candidates"] == ocands == sum(ops)
    assert st["final_cost"] == O.solution_cost(inst, fin)


def test_granular_host_launched_equals_graph(monkeypatch):
    inst = I.vrptw(250, 6)
    sol = I.random_split_solution(inst, I.solution_seed(6))
    nbr = I.granular_neighbors(inst, 8)
    out = {}
    for mode in (T.DESCENT_GRAPH, T.DESCENT_HOST):
        ls = LocalSearch(inst, sol, I.MASK_ALL, log_capacity=1 << 16, granular=nbr).build()
        try:
            ls.set_descent_mode(mode)
            out[mode] = (ls.descend(), ls.move_log(), ls.solution())
        finally:
            ls.close()
    (a, la, (ta, ra)), (b, lb, (tb, rb)) = out[T.DESCENT_GRAPH], out[T.DESCENT_HOST]
    for k in ("steps", "evaluations", "candidates", "final_cost"):
        assert a[k] == b[k], k
    assert np.array_equal(la, lb) and np.array_equal(ta, tb) and np.array_equal(ra, rb)


def test_granular_refusals():
    inst = I.cvrp_uniform(40, 3)
    sol = I.random_split_solution(inst, 4)
    bad = I.granular_neighbors(inst, 4)
    bad[7, 2] = 7                                   # a customer in its own row
    with pytest.raises(TGAError) as e:
        LocalSearch(inst, sol, I.MASK_ALL, granular=bad)
    assert e.value.code == T.TGA_ERR_INVALID
    ls = LocalSearch(inst, sol, I.MASK_ALL, granular=I.granular_neighbors(inst, 4)).build()
    try:
        ls.set_descent_mode(T.DESCENT_PERSISTENT)
        with pytest.raises(TGAError) as e:
            ls.descend()
        assert e.value.code == T.TGA_ERR_STATE
        with pytest.raises(TGAError) as e:
            T.tga_descend_batch([ls.ctx])
        assert e.value.code == T.TGA_ERR_STATE
    finally:
        ls.close()


_W = {}


def _worker_init(seed, theta):
    _W["inst"], _ = I.config2(seed)
    _W["nbr"] = I.granular_neighbors(_W["inst"], theta)


def _worker_eval(args):
    tour, rs = args
    return O.best_move(_W["inst"], _sol(tour, rs), I.MASK_CONFIG2, "concat", granular=_W["nbr"])["key"]


def test_granular_config2_every_step():
    """1000-customer VRPTW, theta = 20: the GPU trajectory replayed with the
    oracle's route surgery and every state re-evaluated by the oracle."""
    inst, sol = I.config2(1)
    nbr = I.granular_neighbors(inst, 20)
    ls = LocalSearch(inst, sol, I.MASK_CONFIG2, log_capacity=1 << 16, granular=nbr).build()
    try:
        ls.set_tile(0, 0)
        st = ls.descend()
        log = ls.move_log()
        tour, rs = ls.solution()
    finally:
        ls.close()
    assert st["status"] == 0 and st["local_optimum"] == 1 and len(log) == st["steps"] + 1
    W = inst.n + 1 + sol.n_routes
    states = [sol]
    cur = sol
    for k in log[:-1]:
        delta, idx = O.unpack_key(int(k))
        assert delta < 0
        op, a, b = idx // (W * W), (idx % (W * W)) // W, idx % W
        cur = O.apply_move(inst, cur, op, a, b)
        states.append(cur)
    assert np.array_equal(states[-1].tour, tour) and np.array_equal(states[-1].route_start, rs)
    assert st["final_cost"] == O.solution_cost(inst, states[-1])
    procs = max(1, (os.cpu_count() or 2) - 1)
    with mp.get_context("spawn").Pool(procs, initializer=_worker_init, initargs=(1, 20)) as pool:
        keys = pool.map(_worker_eval, [(s.tour, s.route_start) for s in states], chunksize=4)
    for k, (key, got) in enumerate(zip(keys, log)):
        assert key == int(got), f"step {k}: gpu {int(got):#x} oracle {key:#x}"
