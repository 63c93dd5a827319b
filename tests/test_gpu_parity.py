"""GPU path vs the CPU oracle, through the C-ABI (marked gpu).

The bar is bit-exact: every evaluation's (delta, move index) equals the
oracle's, every applied move leaves the same tour/route_start, and the final
cost equals the oracle's recomputation.  Full-size workloads are checked by
replaying the GPU's own move log with the oracle's route surgery and
re-evaluating the neighbourhood with the oracle at every (config 2) or at
sampled (config 3) steps in a spawn process pool.
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

from paper_2506_17357_gb300.tga import LocalSearch, TGAError  # noqa: E402


def _sol(tour, rs):
    return I.Solution(np.asarray(tour, np.int32), np.asarray(rs, np.int32))


def _random_case(kind, n, seed, extra_empty):
    inst = I.vrptw(n, seed) if kind == "vrptw" else I.cvrp_uniform(n, seed)
    rng = np.random.default_rng(seed)
    inst.capacity = int(rng.integers(60, 200)) if kind == "vrptw" else -(-int(inst.demand.sum()) // int(rng.integers(2, 6)))
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
            assert (mv["op"], mv["a"], mv["b"]) == (om["op"], om["a"], om["b"])
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


@pytest.mark.parametrize("kind", ["cvrp", "vrptw"])
@pytest.mark.parametrize("seed", range(8))
def test_stepwise_small_random(kind, seed):
    """Every step on random instances with n in [3, 60], extra empty routes,
    all six operator ranks."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(3, 61))
    inst, sol = _random_case(kind, n, 500 + seed, extra_empty=int(rng.integers(0, 3)))
    _stepwise(inst, sol, I.MASK_ALL)


@pytest.mark.parametrize("mask", [1, 2, 4, 8, 16, 32, I.MASK_CONFIG1, I.MASK_CONFIG3])
def test_stepwise_single_operators(mask):
    for kind in ("cvrp", "vrptw"):
        inst, sol = _random_case(kind, 40, 77 + mask, extra_empty=1)
        _stepwise(inst, sol, mask)


def test_long_routes_multi_chunk_scans():
    """Routes longer than a warp (scans run in chunks with a carry)."""
    inst = I.cvrp_uniform(150, 9)
    inst.capacity = int(inst.demand.sum())            # no capacity pressure
    sol = I.random_split_solution(inst, 10)
    assert sol.n_routes == 1
    _stepwise(inst, _sol(sol.tour, [0, 75, 150]), I.MASK_ALL, max_steps=60)
    inst2 = I.vrptw(105, 3)
    inst2.capacity = 10 ** 6
    sol2 = I.random_split_solution(inst2, 4)
    # 35-customer VRPTW routes (37 scan elements); the descent stays within the
    # integer headroom (no route above 57 customers) for its first 20 steps
    _stepwise(inst2, _sol(sol2.tour, [0, 35, 70, 105, 105]), I.MASK_ALL, max_steps=20)


def test_cvrp_route_kernel_with_one_long_route():
    """CVRP intra-route evaluation by route (at most 16 customers per route
    on average) with one route longer than a warp's distance block: that route
    falls back to a warp per moved customer, inside the per-route kernel, on
    the per-step and the persistent paths."""
    from paper_2506_17357_gb300 import tga as T
    inst = I.cvrp_uniform(120, 31)
    inst.capacity = int(inst.demand.sum())            # no capacity pressure
    sol = I.random_split_solution(inst, 32)
    rs = [0, 40, 52, 64, 76, 88, 100, 110, 120]        # 8 routes, the first of 40 customers
    case = _sol(sol.tour, rs)
    _stepwise(inst, case, I.MASK_CONFIG3, max_steps=40)
    st, log, fin = _descend_gpu(inst, case, I.MASK_CONFIG3, mode=T.DESCENT_PERSISTENT, pshape=(16, 4, 1))
    sg, lg, fg = _descend_gpu(inst, case, I.MASK_CONFIG3, mode=T.DESCENT_GRAPH)
    ofin, steps, olog, _ = O.descend(inst, case, I.MASK_CONFIG3, "def")
    for s_, l_, f_ in ((st, log, fin), (sg, lg, fg)):
        assert s_["status"] == 0 and s_["steps"] == steps and np.array_equal(l_, olog)
        assert np.array_equal(f_.tour, ofin.tour) and np.array_equal(f_.route_start, ofin.route_start)


def test_integer_headroom_is_enforced():
    """A VRPTW state whose routes are so long that a candidate route could
    cost 2^27 or more is refused with TGA_ERR_RANGE instead of risking int32
    overflow."""
    inst = I.vrptw(120, 3)
    inst.capacity = 10 ** 6
    sol = I.random_split_solution(inst, 4)
    ls = LocalSearch(inst, _sol(sol.tour, [0, 120, 120]), I.MASK_ALL)
    with pytest.raises(TGAError) as e:
        ls.descend(max_steps=10)
    assert e.value.code == 2
    ls.close()


def _descend_gpu(inst, sol, mask, cap=1 << 20, tile=None, mode=None, pshape=None):
    from paper_2506_17357_gb300 import tga as T
    ls = LocalSearch(inst, sol, mask, log_capacity=cap).build()
    try:
        if tile is not None:
            ls.set_tile(*tile)
        if mode is not None:
            ls.set_descent_mode(mode)
        if pshape is not None:
            T.tga_set_persistent_shape(ls.ctx, *pshape)
        st = ls.descend()
        log = ls.move_log()
        tour, rs = ls.solution()
        return st, log, _sol(tour, rs)
    finally:
        ls.close()


@pytest.mark.parametrize("mode", [0, 2])       # automatic (persistent at this size), graph
@pytest.mark.parametrize("tile", [None, (16, 2), (32, 4), (64, 8), (0, 0), (8, 2, 1), (16, 2, 2),
                                  (32, 2, 4), (64, 4, 2), (16, 4, 0), (32, 8, 0)])    # row split 0: strip-major
def test_config1_full_trajectory(tile, mode):
    inst, sol = I.config1(1)
    st, log, fin = _descend_gpu(inst, sol, I.MASK_CONFIG1, tile=tile, mode=mode)
    ofin, steps, olog, ocands = O.descend(inst, sol, I.MASK_CONFIG1, "def")
    assert st["status"] == 0 and st["local_optimum"] == 1
    assert st["steps"] == steps and np.array_equal(log, olog)
    assert np.array_equal(fin.tour, ofin.tour) and np.array_equal(fin.route_start, ofin.route_start)
    assert st["final_cost"] == O.solution_cost(inst, ofin)
    assert st["candidates"] == ocands


@pytest.mark.parametrize("kind", ["vrptw", "cvrp"])
@pytest.mark.parametrize("limit", [0, 1, 5, 63, 64, 65, None])
def test_descent_paths_agree(kind, limit):
    """The persistent launch, the graph loop and the host-launched per-step
    path (what profilers trace) give the same move log, solution and
    counters, and stop exactly at the step limit."""
    from paper_2506_17357_gb300 import tga as T
    if kind == "vrptw":
        inst = I.vrptw(300, 4)
        mask = I.MASK_ALL
    else:
        inst = I.cvrp_uniform(400, 6)
        mask = I.MASK_CONFIG3
    sol = I.random_split_solution(inst, I.solution_seed(4))
    out = {}
    for mode in (T.DESCENT_GRAPH, T.DESCENT_HOST, T.DESCENT_PERSISTENT):
        ls = LocalSearch(inst, sol, mask, log_capacity=1 << 16).build()
        try:
            ls.set_descent_mode(mode)
            st = ls.descend() if limit is None else ls.descend(max_steps=limit)
            if limit != 0:
                assert ls.descent_mode()[0] == mode
            out[mode] = (st, ls.move_log(), ls.solution())
        finally:
            ls.close()
    sg, lg, (tg, rg) = out[T.DESCENT_GRAPH]
    if limit is not None:
        assert sg["steps"] <= limit and (sg["local_optimum"] == 1 or sg["steps"] == limit)
    else:
        assert sg["local_optimum"] == 1
    for mode in (T.DESCENT_HOST, T.DESCENT_PERSISTENT):
        sh, lh, (th, rh) = out[mode]
        for k in ("steps", "evaluations", "candidates", "final_cost", "local_optimum", "status"):
            assert sg[k] == sh[k], (mode, k)
        assert np.array_equal(lg, lh) and np.array_equal(tg, th) and np.array_equal(rg, rh), mode


@pytest.mark.parametrize("kind", ["cvrp", "vrptw", "vrpspdtw"])
@pytest.mark.parametrize("shape", [(16, 4, 0), (32, 8, 0), (16, 4, 1), (8, 2, 2)])
def test_persistent_shapes_equal_the_graph_path(kind, shape):
    """The persistent descent under a set shape -- strip mode (row split 0:
    every CTA walks a share of the strip-major tile order) or one tile per
    item -- gives the graph path's move log, solution and counters."""
    from paper_2506_17357_gb300 import tga as T
    if kind == "vrptw":
        inst = I.vrptw(300, 14)
    elif kind == "vrpspdtw":
        inst = I.vrpspdtw(250, 15)
    else:
        inst = I.cvrp_uniform(450, 16)
    mask = I.MASK_CONFIG3 if kind == "cvrp" else I.MASK_ALL
    sol = I.random_split_solution(inst, I.solution_seed(14))
    out = {}
    for mode in (T.DESCENT_GRAPH, T.DESCENT_PERSISTENT):
        ls = LocalSearch(inst, sol, mask, log_capacity=1 << 16).build()
        try:
            ls.set_descent_mode(mode)
            if mode == T.DESCENT_PERSISTENT:
                T.tga_set_persistent_shape(ls.ctx, *shape)
                assert tuple(T.tga_get_persistent_shape(ls.ctx)) == shape
            st = ls.descend()
            assert ls.descent_mode()[0] == mode
            out[mode] = (st, ls.move_log(), ls.solution())
        finally:
            ls.close()
    sg, lg, (tg, rg) = out[T.DESCENT_GRAPH]
    sp, lp, (tp, rp) = out[T.DESCENT_PERSISTENT]
    assert sg["local_optimum"] == 1 and sg["status"] == 0
    for k in ("steps", "evaluations", "candidates", "final_cost", "local_optimum", "status"):
        assert sg[k] == sp[k], k
    assert np.array_equal(lg, lp) and np.array_equal(tg, tp) and np.array_equal(rg, rp)


def test_persistent_shape_setter_rejects_bad_shapes():
    from paper_2506_17357_gb300 import tga as T
    inst = I.cvrp_uniform(30, 3)
    ls = LocalSearch(inst, I.random_split_solution(inst, 4), I.MASK_ALL).build()
    try:
        for bad in ((12, 4, 1), (16, 3, 1), (16, 8, 2), (64, 4, 0), (16, 2, 0), (8, 2, 1)):
            with pytest.raises(TGAError):
                T.tga_set_persistent_shape(ls.ctx, *bad)
        T.tga_set_persistent_shape(ls.ctx, 0, 0, 0)                 # back to the automatic choice
    finally:
        ls.close()


@pytest.mark.parametrize("kind", ["cvrp", "vrptw", "vrpspdtw"])
@pytest.mark.parametrize("shape", [(16, 4), (16, 8), (32, 4), (32, 8)])
def test_strip_kernel_stepwise(kind, shape):
    """The strip-major inter-route kernel: every step against the oracle on
    random instances whose tile walks span several strips, CTAs that cross
    strip boundaries, and ragged last strips and row tiles."""
    from paper_2506_17357_gb300 import tga as T
    rng = np.random.default_rng(100 * ["cvrp", "vrptw", "vrpspdtw"].index(kind) + 10 * shape[0] + shape[1])
    for rep in range(2):
        n = int(rng.integers(40, 260))
        if kind == "vrpspdtw":
            inst = I.vrpspdtw(n, 500 + rep)
            inst.capacity = 120
            mask = I.MASK_ALL
        elif kind == "vrptw":
            inst = I.vrptw(n, 510 + rep)
            inst.capacity = 120
            mask = I.MASK_ALL
        else:
            inst = I.cvrp_uniform(n, 520 + rep)
            inst.capacity = -(-int(inst.demand.sum()) // 9)
            mask = I.MASK_CVRP_MIXED
        sol = I.random_split_solution(inst, 530 + rep)
        ls = LocalSearch(inst, sol, mask).build()
        cur = sol
        try:
            ls.set_tile(shape[0], shape[1], 0)
            assert ls.set_tile(shape[0], shape[1], 0) == (shape[0], shape[1], 0)
            for step in range(40):
                mv = ls.eval_best_move()
                om = O.best_move(inst, cur, mask, "concat")
                assert (mv["delta"], mv["move_index"]) == (om["delta"], om["idx"]), (n, step)
                if om["delta"] >= 0:
                    break
                ls.apply_current_move()
                cur = O.apply_move(inst, cur, om["op"], om["a"], om["b"])
            assert ls.stats()["status"] == 0
        finally:
            ls.close()


@pytest.mark.parametrize("kind", ["vrptw", "cvrp"])
def test_strip_kernel_full_descent_equals_tile_kernel(kind):
    """A whole descent on the graph path with the strip-major kernel gives the
    move log, solution and counters of the one-CTA-per-tile kernel."""
    from paper_2506_17357_gb300 import tga as T
    if kind == "vrptw":
        inst, sol = I.config2(2)
        mask = I.MASK_CONFIG2
    else:
        inst = I.cvrp_clustered(2500, 7)
        sol = I.random_split_solution(inst, I.solution_seed(7))
        mask = I.MASK_CONFIG3
    res = []
    for tile in ((32, 4), (32, 8, 0), (16, 8, 0)):
        st, log, fin = _descend_gpu(inst, sol, mask, tile=tile, mode=T.DESCENT_GRAPH)
        res.append((st, log, fin))
    st0, log0, fin0 = res[0]
    assert st0["status"] == 0 and st0["local_optimum"] == 1
    for st, log, fin in res[1:]:
        for k in ("steps", "evaluations", "candidates", "final_cost", "status"):
            assert st[k] == st0[k], k
        assert np.array_equal(log, log0)
        assert np.array_equal(fin.tour, fin0.tour) and np.array_equal(fin.route_start, fin0.route_start)


def test_persistent_descent_resumes_and_reports_its_grid():
    """A persistent descent stopped by the step limit resumes where it stopped
    (second call) and reaches the same local optimum as one uninterrupted call."""
    from paper_2506_17357_gb300 import tga as T
    inst, sol = I.config1(3)
    ref = _descend_gpu(inst, sol, I.MASK_CONFIG1, mode=T.DESCENT_GRAPH)
    ls = LocalSearch(inst, sol, I.MASK_CONFIG1, log_capacity=1 << 12).build()
    try:
        ls.set_descent_mode(T.DESCENT_PERSISTENT)
        a = ls.descend(max_steps=7)
        mode, grid = ls.descent_mode()
        assert mode == T.DESCENT_PERSISTENT and grid >= 1
        assert a["steps"] == min(7, ref[0]["steps"])
        b = ls.descend()
        assert b["steps"] == ref[0]["steps"] and b["final_cost"] == ref[0]["final_cost"]
        tour, rs = ls.solution()
        assert np.array_equal(tour, ref[2].tour) and np.array_equal(rs, ref[2].route_start)
    finally:
        ls.close()


@pytest.mark.parametrize("seed", [2, 3])
def test_small_vrptw_full_trajectory(seed):
    inst = I.vrptw(200, seed)
    sol = I.random_split_solution(inst, I.solution_seed(seed))
    st, log, fin = _descend_gpu(inst, sol, I.MASK_ALL)
    ofin, steps, olog, ocands = O.descend(inst, sol, I.MASK_ALL, "concat")
    assert st["steps"] == steps and np.array_equal(log, olog)
    assert np.array_equal(fin.tour, ofin.tour)
    assert st["candidates"] == ocands


def test_apply_arbitrary_candidates():
    """tga_apply_move on non-best candidates of every op type: the result
    equals the oracle's route surgery and the cost follows the delta."""
    rng = np.random.default_rng(3)
    for kind in ("cvrp", "vrptw"):
        inst, sol = _random_case(kind, 30, 31, extra_empty=1)
        ls = LocalSearch(inst, sol, I.MASK_ALL).build()
        cur = sol.copy()
        cost = O.solution_cost(inst, cur)
        try:
            for _ in range(60):
                idx, dl = O.list_moves(inst, cur, I.MASK_ALL, "def")
                pick = int(rng.integers(0, len(idx)))
                W = inst.n + 1 + cur.n_routes
                ix, delta = int(idx[pick]), int(dl[pick])
                op, a, b = ix // (W * W), (ix % (W * W)) // W, ix % W
                if delta >= 0:          # only improving moves change the solution
                    continue
                mv = torch.tensor([delta, np.int32(np.uint32(ix).view(np.int32)), op, a, b, 1],
                                  dtype=torch.int32, device="cuda:0")
                from paper_2506_17357_gb300.tga import tga_apply_move
                tga_apply_move(ls.ctx, mv.data_ptr())
                cur = O.apply_move(inst, cur, op, a, b)
                cost += delta
                tour, rs = ls.solution()
                assert np.array_equal(tour, cur.tour) and np.array_equal(rs, cur.route_start)
                assert ls.stats()["final_cost"] == cost == O.solution_cost(inst, cur)
                # attributes after the apply drive the next evaluation correctly
                mvb = ls.eval_best_move()
                om = O.best_move(inst, cur, I.MASK_ALL)
                assert (mvb["delta"], mvb["move_index"]) == (om["delta"], om["idx"])
        finally:
            ls.close()


def test_invalid_inputs_reported():
    inst, sol = I.config1(1)
    bad = I.Instance(**{**inst.__dict__})
    bad.dist = inst.dist.copy()
    bad.dist[3, 5] += 1                       # asymmetric
    ls = LocalSearch(bad, sol, I.MASK_CONFIG1)
    with pytest.raises(TGAError) as e:
        ls.descend()
    assert e.value.code == 1
    ls.close()
    dup = sol.copy()
    dup.tour = dup.tour.copy()
    dup.tour[1] = dup.tour[0]                 # not a permutation
    ls = LocalSearch(inst, dup, I.MASK_CONFIG1)
    with pytest.raises(TGAError):
        ls.descend()
    ls.close()


# ---------------------------------------------------------------------------
# full-size workloads: GPU trajectory verified by the oracle in a spawn pool

_W = {}


def _worker_init(cfg, seed):
    _W["inst"], _ = {2: I.config2, 3: I.config3}[cfg](seed)


def _worker_eval(args):
    tour, rs, mask, method = args
    return O.best_move(_W["inst"], _sol(tour, rs), mask, method)["key"]


def _replay(inst, sol, log, W):
    states = [sol]
    cur = sol
    for k in log[:-1]:
        delta, idx = O.unpack_key(int(k))
        assert delta < 0
        op, a, b = idx // (W * W), (idx % (W * W)) // W, idx % W
        cur = O.apply_move(inst, cur, op, a, b)
        states.append(cur)
    return states


def _verify_pool(cfg, seed, states, log, picks, mask, method):
    procs = min(len(picks), max(1, (os.cpu_count() or 2) - 1))
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs, initializer=_worker_init, initargs=(cfg, seed)) as pool:
        keys = pool.map(_worker_eval, [(states[k].tour, states[k].route_start, mask, method) for k in picks],
                        chunksize=1)
    for k, key in zip(picks, keys):
        assert key == int(log[k]), f"step {k}: gpu {int(log[k]):#x} oracle {key:#x}"


def test_config2_full_trajectory_every_step():
    inst, sol = I.config2(1)
    st, log, fin = _descend_gpu(inst, sol, I.MASK_CONFIG2)
    assert st["status"] == 0 and st["local_optimum"] == 1
    assert len(log) == st["steps"] + 1
    states = _replay(inst, sol, log, inst.n + 1 + sol.n_routes)
    assert np.array_equal(states[-1].tour, fin.tour) and np.array_equal(states[-1].route_start, fin.route_start)
    assert st["final_cost"] == O.solution_cost(inst, fin)
    assert O.check_solution(inst, fin) == 0
    budget = int(os.environ.get("TGA_C2_CHECK_STEPS", "0"))
    picks = list(range(len(log)))
    if budget and budget < len(picks):        # optional cap for slow hosts: first, last, spread
        picks = sorted(set(picks[:budget // 2] + picks[-1:] + picks[::max(1, len(picks) // (budget // 2))]))
    _verify_pool(2, 1, states, log, picks, I.MASK_CONFIG2, "concat")


def _replay_picks(inst, sol, log, W, picks):
    """Replay the GPU's move log with the oracle's route surgery, keeping only
    the states at the picked evaluations (and the final one)."""
    want = set(picks)
    kept = {}
    cur = sol
    for k, key in enumerate(log[:-1]):
        if k in want:
            kept[k] = cur
        delta, idx = O.unpack_key(int(key))
        assert delta < 0, k
        op, a, b = idx // (W * W), (idx % (W * W)) // W, idx % W
        cur = O.apply_move(inst, cur, op, a, b)
    if len(log) - 1 in want:
        kept[len(log) - 1] = cur
    return kept, cur


def config3_picks(n_evals):
    """Evaluations of the CVRP-10000 descent re-evaluated by the oracle:
    every one of the first 50, then every 200th, and the last two (the last
    one is the local optimum)."""
    picks = set(range(min(50, n_evals))) | set(range(0, n_evals, 200)) | {n_evals - 2, n_evals - 1}
    return sorted(p for p in picks if 0 <= p < n_evals)


def test_config3_sampled_steps_and_local_optimum():
    """Clustered CVRP-10000 (the per-step graph path at full size: the
    multi-wave inter-route grid, a 461 MB position-ordered distance copy
    beyond L2, move indices near 6 W^2): the whole move sequence is replayed
    by the oracle's route surgery (every logged move must improve), the final
    solution and cost are checked, and the oracle re-evaluates the
    neighbourhood from scratch at the picked evaluations."""
    inst, sol = I.config3(1)
    st, log, fin = _descend_gpu(inst, sol, I.MASK_CONFIG3)
    assert st["status"] == 0 and st["local_optimum"] == 1
    assert len(log) == st["steps"] + 1
    W = inst.n + 1 + sol.n_routes
    picks = config3_picks(len(log))
    kept, last = _replay_picks(inst, sol, log, W, picks)
    assert np.array_equal(last.tour, fin.tour) and np.array_equal(last.route_start, fin.route_start)
    assert st["final_cost"] == O.solution_cost(inst, fin)
    assert O.check_solution(inst, fin) == 0
    states = [kept[k] for k in picks]
    _verify_pool(3, 1, dict(zip(picks, states)), log, picks, I.MASK_CONFIG3, "concat")
    print(f"cvrp10000: {len(picks)} of {len(log)} evaluations re-evaluated by the oracle")
    # the persistent descent in strip mode (the path the timed bench takes at
    # this size) gives the same move log, solution and counters
    from paper_2506_17357_gb300 import tga as T
    sp, logp, finp = _descend_gpu(inst, sol, I.MASK_CONFIG3, mode=T.DESCENT_PERSISTENT, pshape=(32, 8, 0))
    assert np.array_equal(logp, log) and np.array_equal(finp.tour, fin.tour)
    assert np.array_equal(finp.route_start, fin.route_start)
    for k in ("steps", "evaluations", "candidates", "final_cost", "local_optimum", "status"):
        assert sp[k] == st[k], k
