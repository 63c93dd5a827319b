"""Simultaneous pickup and delivery with time windows (VRPSPDTW) on the GPU
path vs the CPU oracle, through the C-ABI (marked gpu).

With pickups every load term penalises the largest load on board, which the
device evaluates from the L_I / L_O / L_M attributes of Section 4.3.2 (inter-
route constants, intra-route subsequence tables and sweeps).  The bar is the
same as without pickups: every evaluation's (delta, move index) equals the
oracle's, and the applied moves leave the same solution.
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


def _pd_case(n, seed, extra_empty, cap=None):
    inst = I.vrpspdtw(n, seed)
    rng = np.random.default_rng(seed)
    inst.capacity = int(rng.integers(60, 200)) if cap is None else cap
    sol = I.random_split_solution(inst, seed + 17)
    rs = list(sol.route_start)
    for _ in range(extra_empty):      # empty routes at random slots
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
        return steps
    finally:
        ls.close()


def _descend(inst, sol, mask, mode=None, cap=1 << 18):
    ls = LocalSearch(inst, sol, mask, log_capacity=cap).build()
    try:
        if mode is not None:
            ls.set_descent_mode(mode)
        st = ls.descend()
        return st, ls.move_log(), _sol(*ls.solution())
    finally:
        ls.close()


@pytest.mark.parametrize("seed", range(8))
def test_pd_stepwise_small_random(seed):
    """Every step on random instances with n in [3, 60], extra empty routes,
    all six operator ranks."""
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(3, 61))
    inst, sol = _pd_case(n, 600 + seed, extra_empty=int(rng.integers(0, 3)))
    _stepwise(inst, sol, I.MASK_ALL)


@pytest.mark.parametrize("mask", [1, 2, 4, 8, 16, 32])
def test_pd_stepwise_single_operators(mask):
    inst, sol = _pd_case(40, 91 + mask, extra_empty=1)
    _stepwise(inst, sol, mask)


def test_pd_long_routes_fallback_sweeps_and_chunked_scans():
    """Routes above 40 customers (intra-route sweeps instead of the tables)
    and above 30 (rebuilds in chunks with a carry).  Small penalty weights keep
    the long routes inside the integer headroom."""
    inst = I.vrpspdtw(135, 5)
    inst.w_tw, inst.w_load = 2, 10
    inst.capacity = 1100                             # the load terms stay active
    sol = I.random_split_solution(inst, 6)
    _stepwise(inst, _sol(sol.tour, [0, 45, 90, 135]), I.MASK_ALL, max_steps=25)


@pytest.mark.parametrize("seed", [2, 3])
def test_pd_full_trajectory(seed):
    inst = I.vrpspdtw(200, seed)
    sol = I.random_split_solution(inst, I.solution_seed(seed))
    st, log, fin = _descend(inst, sol, I.MASK_ALL)
    ofin, steps, olog, ocands = O.descend(inst, sol, I.MASK_ALL, "concat")
    assert st["status"] == 0 and st["local_optimum"] == 1
    assert st["steps"] == steps and np.array_equal(log, olog)
    assert np.array_equal(fin.tour, ofin.tour) and np.array_equal(fin.route_start, ofin.route_start)
    assert st["final_cost"] == O.solution_cost(inst, ofin)
    assert st["candidates"] == ocands


@pytest.mark.parametrize("limit", [1, 64, None])
def test_pd_descent_paths_agree(limit):
    """Persistent launch, graph loop and host-launched steps: same move log,
    solution and counters with pickups."""
    inst = I.vrpspdtw(300, 4)
    sol = I.random_split_solution(inst, I.solution_seed(4))
    out = {}
    for mode in (T.DESCENT_GRAPH, T.DESCENT_HOST, T.DESCENT_PERSISTENT):
        ls = LocalSearch(inst, sol, I.MASK_ALL, log_capacity=1 << 16).build()
        try:
            ls.set_descent_mode(mode)
            st = ls.descend() if limit is None else ls.descend(max_steps=limit)
            assert ls.descent_mode()[0] == mode
            out[mode] = (st, ls.move_log(), ls.solution())
        finally:
            ls.close()
    sg, lg, (tg, rg) = out[T.DESCENT_GRAPH]
    for mode in (T.DESCENT_HOST, T.DESCENT_PERSISTENT):
        sh, lh, (th, rh) = out[mode]
        for k in ("steps", "evaluations", "candidates", "final_cost", "local_optimum", "status"):
            assert sg[k] == sh[k], (mode, k)
        assert np.array_equal(lg, lh) and np.array_equal(tg, th) and np.array_equal(rg, rh), mode
    if limit is None:
        ofin, steps, olog, _ = O.descend(inst, sol, I.MASK_ALL, "concat")
        assert sg["steps"] == steps and np.array_equal(lg, olog)


def test_pd_apply_arbitrary_candidates():
    """tga_apply_move on random improving candidates of every op type: the
    result equals the oracle's route surgery, the cost follows the delta, and
    the rebuilt attributes drive the next evaluation correctly."""
    rng = np.random.default_rng(5)
    inst, sol = _pd_case(30, 41, extra_empty=1)
    ls = LocalSearch(inst, sol, I.MASK_ALL).build()
    cur = sol.copy()
    cost = O.solution_cost(inst, cur)
    applied = 0
    try:
        for _ in range(80):
            idx, dl = O.list_moves(inst, cur, I.MASK_ALL, "def")
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
            om = O.best_move(inst, cur, I.MASK_ALL)
            assert (mvb["delta"], mvb["move_index"]) == (om["delta"], om["idx"])
    finally:
        ls.close()
    assert applied > 5


def test_pd_without_pickups_matches_vrptw():
    """All-zero pickups: the largest load is the total delivery, so the
    trajectory equals the VRPTW one of the same instance."""
    inst = I.vrpspdtw(150, 8)
    inst.pickup = np.zeros_like(inst.pickup)
    plain = I.vrptw(150, 8)
    sol = I.random_split_solution(plain, 9)
    st1, log1, fin1 = _descend(inst, sol, I.MASK_ALL)
    st2, log2, fin2 = _descend(plain, sol, I.MASK_ALL)
    assert st1["steps"] == st2["steps"] > 0 and np.array_equal(log1, log2)
    assert np.array_equal(fin1.tour, fin2.tour)


def test_pd_refusals_and_invalid_pickups():
    inst, sol = _pd_case(50, 3, extra_empty=0)
    ls = LocalSearch(inst, sol, I.MASK_ALL).build()
    try:
        nbr = torch.from_numpy(I.granular_neighbors(inst, 5).reshape(-1)).to("cuda:0")
        with pytest.raises(TGAError) as e:
            T.tga_set_granular(ls.ctx, nbr.data_ptr(), 5)
        assert e.value.code == T.TGA_ERR_STATE
        with pytest.raises(TGAError) as e:
            T.tga_descend_batch([ls.ctx])
        assert e.value.code == T.TGA_ERR_STATE
    finally:
        ls.close()
    bad = I.vrpspdtw(50, 3)
    bad.pickup = bad.pickup.copy()
    bad.pickup[7] = -1
    ls = LocalSearch(bad, sol, I.MASK_ALL)
    try:
        with pytest.raises(TGAError) as e:
            ls.descend()
        assert e.value.code == T.TGA_ERR_INVALID
    finally:
        ls.close()


# ---------------------------------------------------------------------------
# full-size workload: VRPSPDTW with 1000 customers, sampled steps re-evaluated
# by the oracle in a spawn pool from the replayed GPU move log

_W = {}


def _worker_init(seed):
    _W["inst"], _ = I.config_spd(seed)


def _worker_eval(args):
    tour, rs = args
    return O.best_move(_W["inst"], _sol(tour, rs), I.MASK_ALL, "concat")["key"]


def test_pd_config_full_size_sampled_steps():
    inst, sol = I.config_spd(1)
    st, log, fin = _descend(inst, sol, I.MASK_ALL, cap=1 << 16)
    assert st["status"] == 0 and st["local_optimum"] == 1
    assert len(log) == st["steps"] + 1
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
    picks = sorted(set(p for p in (0, 1, 2, 3, n // 8, n // 4, n // 2, 3 * n // 4, n - 3, n - 2, n - 1)
                       if 0 <= p < n))
    procs = min(len(picks), max(1, (os.cpu_count() or 2) - 1))
    with mp.get_context("spawn").Pool(procs, initializer=_worker_init, initargs=(1,)) as pool:
        keys = pool.map(_worker_eval, [(states[k].tour, states[k].route_start) for k in picks], chunksize=1)
    for k, key in zip(picks, keys):
        assert key == int(log[k]), f"step {k}: gpu {int(log[k]):#x} oracle {key:#x}"
