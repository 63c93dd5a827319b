"""Swaps of runs (op ranks 6 and 7: a customer with a run of two, two runs of
two; the Swap of Section 5.3.1 with run lengths N1, N2 in {1, 2}) on the GPU
path vs the CPU oracle, through the C-ABI (marked gpu).

Inter-route candidates come from the gather kernel over the position-ordered
distance copy, intra-route ones from the route kernels (subsequence tables,
the sweeps of long routes, the CVRP per-customer warps).  The bar is
bit-exact, as for the other ranks.
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

XS = 64 | 128


def _sol(tour, rs):
    return I.Solution(np.asarray(tour, np.int32), np.asarray(rs, np.int32))


def _case(kind, n, seed, extra_empty):
    inst = I.vrptw(n, seed) if kind == "vrptw" else I.cvrp_uniform(n, seed)
    rng = np.random.default_rng(seed)
    inst.capacity = (int(rng.integers(60, 200)) if kind == "vrptw"
                     else -(-int(inst.demand.sum()) // int(rng.integers(2, 6))))
    sol = I.random_split_solution(inst, seed + 17)
    rs = list(sol.route_start)
    for _ in range(extra_empty):
        at = int(rng.integers(0, len(rs)))
        rs.insert(at, rs[at] if at < len(rs) else n)
    rs = sorted(rs)
    rs[0], rs[-1] = 0, n
    return inst, _sol(sol.tour, rs)


def _stepwise(inst, sol, mask, max_steps=10 ** 6):
    ls = LocalSearch(inst, sol, mask).build()
    cur = sol.copy()
    steps = 0
    try:
        while steps < max_steps:
            mv = ls.eval_best_move()
            om = O.best_move(inst, cur, mask, "def")
            assert mv["valid"] == om["found"], (steps, mv, om, ls.stats())
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
        assert st["status"] == 0, st
        assert st["final_cost"] == O.solution_cost(inst, cur)
        assert st["steps"] == steps
        assert st["candidates"] == sum(T.tga_get_op_candidates(ls.ctx))
        return steps
    finally:
        ls.close()


@pytest.mark.parametrize("kind", ["cvrp", "vrptw"])
@pytest.mark.parametrize("seed", range(6))
def test_xswap_stepwise_small_random(kind, seed):
    """Every step on random instances with n in [3, 60], extra empty routes,
    all eight operator ranks."""
    rng = np.random.default_rng(3000 + seed)
    n = int(rng.integers(3, 61))
    inst, sol = _case(kind, n, 700 + seed, extra_empty=int(rng.integers(0, 3)))
    _stepwise(inst, sol, I.MASK_EXT)


@pytest.mark.parametrize("kind", ["cvrp", "vrptw"])
@pytest.mark.parametrize("mask", [64, 128, XS])
def test_xswap_stepwise_alone(kind, mask):
    inst, sol = _case(kind, 45, 51 + mask, extra_empty=1)
    _stepwise(inst, sol, mask)


def test_xswap_long_routes_sweeps_and_chunked_scans():
    """Time-window routes above 40 customers take the sweeps instead of the
    tables; above 30 the rebuilds run in chunks.  Small penalty weights keep
    the long routes inside the integer headroom."""
    inst = I.vrptw(135, 5)
    inst.w_tw, inst.w_load = 2, 10
    inst.capacity = 1200
    sol = I.random_split_solution(inst, 6)
    _stepwise(inst, _sol(sol.tour, [0, 45, 90, 135]), XS | 1, max_steps=25)
    cv = I.cvrp_uniform(120, 7)
    cv.capacity = int(cv.demand.sum())
    sol2 = I.random_split_solution(cv, 8)
    _stepwise(cv, _sol(sol2.tour, [0, 40, 80, 120]), XS, max_steps=25)


@pytest.mark.parametrize("kind,seed", [("vrptw", 2), ("cvrp", 3)])
def test_xswap_full_trajectory(kind, seed):
    inst = I.vrptw(150, seed) if kind == "vrptw" else I.cvrp_uniform(150, seed)
    sol = I.random_split_solution(inst, I.solution_seed(seed))
    ls = LocalSearch(inst, sol, I.MASK_EXT, log_capacity=1 << 16).build()
    try:
        st = ls.descend()
        log = ls.move_log()
        fin = _sol(*ls.solution())
        assert ls.descent_mode()[0] == T.DESCENT_GRAPH       # automatic: the per-step path
    finally:
        ls.close()
    ofin, steps, olog, ocands = O.descend(inst, sol, I.MASK_EXT, "concat")
    assert st["status"] == 0 and st["local_optimum"] == 1
    assert st["steps"] == steps and np.array_equal(log, olog)
    assert np.array_equal(fin.tour, ofin.tour) and np.array_equal(fin.route_start, ofin.route_start)
    assert st["candidates"] == ocands
    ops = [O.unpack_key(int(k))[1] // (inst.n + 1 + sol.n_routes) ** 2 for k in log[:-1]]
    assert {6, 7} & set(ops), "no swap of runs applied"


def test_xswap_paths_agree_and_persistent_refused():
    inst = I.vrptw(250, 4)
    sol = I.random_split_solution(inst, I.solution_seed(4))
    out = {}
    for mode in (T.DESCENT_GRAPH, T.DESCENT_HOST):
        ls = LocalSearch(inst, sol, I.MASK_EXT, log_capacity=1 << 16).build()
        try:
            ls.set_descent_mode(mode)
            out[mode] = (ls.descend(), ls.move_log(), ls.solution())
        finally:
            ls.close()
    (sg, lg, (tg, rg)), (sh, lh, (th, rh)) = out[T.DESCENT_GRAPH], out[T.DESCENT_HOST]
    for k in ("steps", "evaluations", "candidates", "final_cost", "local_optimum", "status"):
        assert sg[k] == sh[k], k
    assert np.array_equal(lg, lh) and np.array_equal(tg, th) and np.array_equal(rg, rh)
    ls = LocalSearch(inst, sol, I.MASK_EXT).build()
    try:
        ls.set_descent_mode(T.DESCENT_PERSISTENT)
        with pytest.raises(TGAError) as e:
            ls.descend(max_steps=3)
        assert e.value.code == T.TGA_ERR_STATE
    finally:
        ls.close()


def test_xswap_apply_arbitrary_candidates():
    """tga_apply_move on random improving candidates of ranks 6 and 7, in and
    across routes: the result equals the oracle's route surgery."""
    rng = np.random.default_rng(9)
    for kind in ("cvrp", "vrptw"):
        inst, sol = _case(kind, 30, 61, extra_empty=1)
        ls = LocalSearch(inst, sol, I.MASK_EXT).build()
        cur = sol.copy()
        cost = O.solution_cost(inst, cur)
        applied = 0
        try:
            for _ in range(120):
                idx, dl = O.list_moves(inst, cur, XS, "def")
                if len(idx) == 0:
                    break
                pick = int(rng.integers(0, len(idx)))
                W = inst.n + 1 + cur.n_routes
                ix, delta = int(idx[pick]), int(dl[pick])
                op, a, b = ix // (W * W), (ix % (W * W)) // W, ix % W
                if delta >= 0:
                    continue
                mv = torch.tensor([delta, np.int32(np.uint32(ix).view(np.int32)), op, a, b, 1],
                                  dtype=torch.int32, device="cuda:0")
                T.tga_apply_move(ls.ctx, mv.data_ptr())
                cur = O.apply_move(inst, cur, op, a, b)
                cost += delta
                applied += 1
                tour, rs = ls.solution()
                assert np.array_equal(tour, cur.tour) and np.array_equal(rs, cur.route_start)
                assert ls.stats()["final_cost"] == cost == O.solution_cost(inst, cur)
                mvb = ls.eval_best_move()
                om = O.best_move(inst, cur, I.MASK_EXT)
                assert (mvb["delta"], mvb["move_index"]) == (om["delta"], om["idx"])
        finally:
            ls.close()
        assert applied > 5


def test_xswap_refusals():
    inst = I.vrpspdtw(40, 3)
    sol = I.random_split_solution(inst, 4)
    with pytest.raises(TGAError) as e:
        LocalSearch(inst, sol, I.MASK_EXT)
    assert e.value.code == T.TGA_ERR_INVALID           # no pickup variant
    cv, csol = _case("cvrp", 40, 5, extra_empty=0)
    ls = LocalSearch(cv, csol, I.MASK_EXT).build()
    try:
        nbr = torch.from_numpy(I.granular_neighbors(cv, 5).reshape(-1)).to("cuda:0")
        with pytest.raises(TGAError) as e:
            T.tga_set_granular(ls.ctx, nbr.data_ptr(), 5)
        assert e.value.code == T.TGA_ERR_STATE
        with pytest.raises(TGAError) as e:
            T.tga_descend_batch([ls.ctx])
        assert e.value.code == T.TGA_ERR_STATE
    finally:
        ls.close()


# ---------------------------------------------------------------------------
# full size: VRPTW with 1000 customers and all eight ranks; sampled steps
# re-evaluated by the oracle from the replayed GPU move log

_W = {}


def _worker_init(seed):
    _W["inst"], _ = I.config2(seed)


def _worker_eval(args):
    tour, rs = args
    return O.best_move(_W["inst"], _sol(tour, rs), I.MASK_EXT, "concat")["key"]


def test_xswap_vrptw1000_sampled_steps():
    inst, sol = I.config2(1)
    ls = LocalSearch(inst, sol, I.MASK_EXT, log_capacity=1 << 16).build()
    try:
        st = ls.descend()
        log = ls.move_log()
        fin = _sol(*ls.solution())
    finally:
        ls.close()
    assert st["status"] == 0 and st["local_optimum"] == 1
    W = inst.n + 1 + sol.n_routes
    states = [sol]
    cur = sol
    for k in log[:-1]:
        delta, idx = O.unpack_key(int(k))
        assert delta < 0
        cur = O.apply_move(inst, cur, idx // (W * W), (idx % (W * W)) // W, idx % W)
        states.append(cur)
    assert np.array_equal(cur.tour, fin.tour) and np.array_equal(cur.route_start, fin.route_start)
    assert st["final_cost"] == O.solution_cost(inst, fin)
    n = len(log)
    picks = sorted(set(p for p in (0, 1, 2, n // 4, n // 2, 3 * n // 4, n - 2, n - 1) if 0 <= p < n))
    procs = min(len(picks), max(1, (os.cpu_count() or 2) - 1))
    with mp.get_context("spawn").Pool(procs, initializer=_worker_init, initargs=(1,)) as pool:
        keys = pool.map(_worker_eval, [(states[k].tour, states[k].route_start) for k in picks], chunksize=1)
    for k, key in zip(picks, keys):
        assert key == int(log[k]), f"step {k}: gpu {int(log[k]):#x} oracle {key:#x}"
