"""Pins of the CPU oracle to things other than itself (CPU only).

* exhaustive rounding rule of the integer distances (number theory),
* hand-worked examples under tests/golden/ (each cites its passage),
* the paper's concatenation operator (Section 4.3) against the forward
  simulation of the time-warp definition and of the load on board, and its
  associativity; special cases of the pickup-and-delivery load profile,
* an independent pure-Python brute force over whole candidate sets,
* closed-form candidate counts, textbook CVRP deltas, and geometry
  (2-opt on points in convex position ends in convex order),
* invariants of a descent (cost bookkeeping, one visit per customer, load
  conservation, fixed fleet, local optimality).
"""
import json
import math
import os
import random

import numpy as np
import pytest

import oracle as O
from paper_2506_17357_gb300 import instances as I
from tests.brute import brute_moves, route_cost as py_route_cost

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _inst_from_golden(g):
    tw = "tw_early" in g
    return I.instance_from_arrays(
        "golden", np.array(g["dist"]), g["demand"], g["capacity"],
        service=g.get("service"), tw_early=g.get("tw_early"), tw_late=g.get("tw_late"),
        coords=g.get("coords")) if tw else I.instance_from_arrays(
        "golden", np.array(g["dist"]), g["demand"], g["capacity"], coords=g.get("coords"))


def _sol(tour, rs):
    return I.Solution(np.asarray(tour, np.int32), np.asarray(rs, np.int32))


def _tiny(kind, n, seed, m_extra_empty=1):
    if kind in ("vrpspdtw", "vrpspd"):
        inst = I.vrpspdtw(n, seed)
        inst.has_tw = kind == "vrpspdtw"
    else:
        inst = I.vrptw(n, seed) if kind == "vrptw" else I.cvrp_uniform(n, seed)
    # a few multi-customer routes even at tiny n
    inst.capacity = 100 if kind != "cvrp" else -(-int(inst.demand.sum()) // 3)
    sol = I.random_split_solution(inst, seed + 11)
    rs = list(sol.route_start) + [n] * m_extra_empty   # trailing empty routes
    return inst, _sol(sol.tour, rs)


# ----------------------------------------------------------------------------
def test_round_sqrt_exhaustive():
    """c = round(sqrt(S)) for every S up to 2*1000^2: the nearest integer c
    satisfies (c-1/2)^2 <= S < (c+1/2)^2, i.e. c^2-c < S <= c^2+c."""
    s = np.arange(0, 2 * 1000 * 1000 + 1, dtype=np.int64)
    c = I.round_sqrt(s)
    assert c[0] == 0
    ok = (c[1:] * c[1:] - c[1:] < s[1:]) & (s[1:] <= c[1:] * c[1:] + c[1:])
    assert bool(ok.all())
    for v in (1, 2, 3, 24, 25, 26, 2 * 10 ** 6, 999_999):
        assert int(c[v]) == int(math.floor(math.sqrt(v) + 0.5))


def test_distance_matrix_properties():
    inst = I.cvrp_uniform(50, 3)
    d = inst.dist.astype(np.int64)
    assert (d == d.T).all() and (np.diag(d) == 0).all()
    xy = inst.coords.astype(np.float64)
    exact = np.sqrt(((xy[:, None, :] - xy[None, :, :]) ** 2).sum(-1))
    assert np.abs(d - exact).max() <= 0.5


def test_generator_is_deterministic():
    a, sa = I.config1(7)
    b, sb = I.config1(7)
    assert (a.dist == b.dist).all() and (sa.tour == sb.tour).all()
    assert sorted(sa.tour.tolist()) == list(range(1, a.n + 1))
    assert a.capacity == -(-int(a.demand.sum()) // 8)


def test_pickup_generator_and_split_rule():
    """The VRPSPDTW recipe is the VRPTW one of the same seed plus pickups in
    [1, 50]; the initial split keeps every route's total delivery and total
    pickup within the capacity and opens a route only when the next customer
    would break one of them."""
    a, b, v = I.vrpspdtw(300, 9), I.vrpspdtw(300, 9), I.vrptw(300, 9)
    assert (a.pickup == b.pickup).all() and (a.dist == v.dist).all() and (a.demand == v.demand).all()
    assert a.pickup[0] == 0 and a.pickup[1:].min() >= 1 and a.pickup[1:].max() <= 50
    sol = I.random_split_solution(a, 10)
    routes = sol.routes()
    for k, r in enumerate(routes):
        sd = sum(int(a.demand[x]) for x in r)
        sp = sum(int(a.pickup[x]) for x in r)
        assert sd <= a.capacity and sp <= a.capacity
        if k + 1 < len(routes):
            nx = routes[k + 1][0]
            assert sd + a.demand[nx] > a.capacity or sp + a.pickup[nx] > a.capacity


# ----------------------------------------------------------------------------
def test_hand_cvrp_swap():
    g = _golden("hand_cvrp_swap.json")
    inst = _inst_from_golden(g)
    sol = _sol(g["tour"], g["route_start"])
    ex = g["expected"]
    assert O.solution_cost(inst, sol) == ex["solution_cost"]
    assert [O.route_cost(inst, r) for r in sol.routes()] == ex["route_costs"]
    assert O.count_candidates(inst, sol, g["op_mask"]) == ex["n_candidates"]
    W = inst.n + 1 + sol.n_routes
    for method in ("def", "concat"):
        idx, dl = O.list_moves(inst, sol, g["op_mask"], method)
        got = {}
        for i, d in zip(idx.tolist(), dl.tolist()):
            a, b = (i - W * W) // W, (i - W * W) % W
            got[f"{a},{b}"] = d
        assert got == ex["swap_deltas"]
        bm = O.best_move(inst, sol, g["op_mask"], method)
        assert {k: bm[k] for k in ("delta", "idx", "op", "a", "b")} == ex["best"]


def test_hand_vrptw_warp():
    g = _golden("hand_vrptw_warp.json")
    inst = _inst_from_golden(g)
    sol = _sol(g["tour"], g["route_start"])
    ex = g["expected"]
    assert O.route_warp(inst, [1, 2]) == ex["warp"]
    assert O.route_warp(inst, [2, 1]) == ex["reversed_warp"]
    assert [O.route_cost(inst, r) for r in sol.routes()] == ex["route_costs"]
    assert O.count_candidates(inst, sol, g["op_mask"]) == ex["n_candidates"]
    for method in ("def", "concat"):
        bm = O.best_move(inst, sol, g["op_mask"], method)
        assert {k: bm[k] for k in ("delta", "idx", "op", "a", "b")} == ex["best"]


# ----------------------------------------------------------------------------
def test_hand_vrpspd_load():
    g = _golden("hand_vrpspd_load.json")
    inst = I.instance_from_arrays("golden", np.array(g["dist"]), g["demand"], g["capacity"],
                                  pickup=g["pickup"])
    sol = _sol(g["tour"], g["route_start"])
    ex = g["expected"]
    for order, peak in ex["peak_loads"].items():
        route = [int(x) for x in order.split(",")]
        assert O.route_peak_load(inst, route) == peak
        from tests.brute import peak_load
        assert peak_load(inst, route) == peak
    assert [O.route_cost(inst, r) for r in sol.routes()] == ex["route_costs"]
    assert O.count_candidates(inst, sol, g["op_mask"]) == ex["n_candidates"]
    for method in ("def", "concat"):
        idx, dl = O.list_moves(inst, sol, g["op_mask"], method)
        assert {str(i): d for i, d in zip(idx.tolist(), dl.tolist())} == ex["deltas"]
        bm = O.best_move(inst, sol, g["op_mask"], method)
        assert {k: bm[k] for k in ("delta", "idx", "op", "a", "b")} == ex["best"]


@pytest.mark.parametrize("seed", range(3))
def test_peak_load_special_cases(seed):
    """Section 2 load profile: without pickups the largest load is the total
    delivery at departure; with deliveries all zero it is the total pickup on
    return; it always lies between max(sum d, sum p) and sum d + sum p; and
    driving the route backwards with the roles of d and p exchanged gives the
    same profile in reverse, so the same largest load."""
    inst = I.vrpspdtw(30, 500 + seed)
    no_pk = I.vrptw(30, 500 + seed)
    only_pk = I.vrpspdtw(30, 500 + seed)
    only_pk.demand = np.zeros_like(only_pk.demand)
    swapped = I.vrpspdtw(30, 500 + seed)
    swapped.demand, swapped.pickup = inst.pickup.copy(), inst.demand.copy()
    rng = random.Random(seed)
    for _ in range(100):
        route = rng.sample(range(1, inst.n + 1), rng.randint(1, 15))
        sd = sum(int(inst.demand[x]) for x in route)
        sp = sum(int(inst.pickup[x]) for x in route)
        peak = O.route_peak_load(inst, route)
        assert O.route_peak_load(no_pk, route) == sd
        assert O.route_peak_load(only_pk, route) == sp
        assert max(sd, sp) <= peak <= sd + sp
        assert O.route_peak_load(swapped, route[::-1]) == peak


def _fold(inst, nodes):
    s = O.seg_node(inst, nodes[0])
    for x in nodes[1:]:
        s = O.seg_concat(inst, s, O.seg_node(inst, x))
    return s


@pytest.mark.parametrize("kind", ["vrptw", "vrpspdtw"])
@pytest.mark.parametrize("seed", range(6))
def test_concat_equals_forward_simulation(kind, seed):
    """Section 4.3: folding the concatenation operator over (0, route, 0)
    gives the route's distance, loads and time warp of the forward simulation
    (travel time = distance, waiting allowed, late arrival warps back; the
    largest load on board from the load profile of Section 2)."""
    inst = I.vrptw(40, 100 + seed) if kind == "vrptw" else I.vrpspdtw(40, 100 + seed)
    pk = inst.pickup if inst.pickup is not None else np.zeros_like(inst.demand)
    rng = random.Random(seed)
    for _ in range(200):
        L = rng.randint(1, 12)
        route = rng.sample(range(1, inst.n + 1), L)
        s = _fold(inst, [0] + route + [0])
        seq = [0] + route + [0]
        assert s[0] == sum(int(inst.dist[seq[k], seq[k + 1]]) for k in range(len(seq) - 1))
        assert s[1] == sum(int(inst.demand[x]) for x in route)
        assert s[2] == sum(int(pk[x]) for x in route)
        assert s[3] == O.route_peak_load(inst, route)
        assert s[7] == O.route_warp(inst, route)
        assert py_route_cost(inst, route) == O.route_cost(inst, route)


@pytest.mark.parametrize("kind", ["vrptw", "vrpspdtw"])
@pytest.mark.parametrize("seed", range(4))
def test_concat_associative(kind, seed):
    inst = I.vrptw(30, 200 + seed) if kind == "vrptw" else I.vrpspdtw(30, 200 + seed)
    rng = random.Random(seed)
    for _ in range(300):
        nodes = rng.sample(range(0, inst.n + 1), rng.randint(3, 9))
        cut1 = rng.randint(1, len(nodes) - 2)
        cut2 = rng.randint(cut1 + 1, len(nodes) - 1)
        a, b, c = _fold(inst, nodes[:cut1]), _fold(inst, nodes[cut1:cut2]), _fold(inst, nodes[cut2:])
        left = O.seg_concat(inst, O.seg_concat(inst, a, b), c)
        right = O.seg_concat(inst, a, O.seg_concat(inst, b, c))
        assert (left == right).all()


# ----------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["cvrp", "vrptw", "vrpspdtw"])
@pytest.mark.parametrize("seed", range(5))
def test_swaps_of_runs_against_brute_force(kind, seed):
    """Ranks 6 and 7 (a customer with a run of two, two runs of two; Section
    5.3.1 Swap with N1 = 1, 2 and N2 = 2): every candidate and delta equals the
    independent Python statement of the exchange, in and across routes."""
    n = 6 + seed % 4
    inst, sol = _tiny(kind, n, 900 + seed, m_extra_empty=1)
    expect = brute_moves(inst, sol.routes(), 64 | 128)
    assert expect, "no run-swap candidates"
    for method in ("def", "concat"):
        idx, dl = O.list_moves(inst, sol, 64 | 128, method)
        assert dict(zip(idx.tolist(), dl.tolist())) == expect, method
    full = brute_moves(inst, sol.routes(), I.MASK_EXT)
    bm = O.best_move(inst, sol, I.MASK_EXT, "concat")
    assert (bm["delta"], bm["idx"]) == min((d, i) for i, d in full.items())


def test_swap_of_runs_hand_example():
    """One route (0, 1, 2, 3, 4, 0) on a line: node x at coordinate 10 x.
    Exchanging customer 1 with the run (3, 4) gives (0, 3, 4, 2, 1, 0):
    distance 30 + 10 + 20 + 10 + 10 = 80 instead of 80 for the straight
    route, delta 0; exchanging the runs (1, 2) and (3, 4) gives
    (0, 3, 4, 1, 2, 0): 30 + 10 + 30 + 10 + 20 = 100, delta +20."""
    pts = np.array([[10 * x, 0] for x in range(5)], np.int64)
    inst = I.instance_from_arrays("line", I.rounded_euclidean(pts), [0, 1, 1, 1, 1], 100)
    sol = _sol([1, 2, 3, 4], [0, 4])
    W = 4 + 1 + 1
    idx, dl = O.list_moves(inst, sol, 64 | 128, "def")
    got = dict(zip(idx.tolist(), dl.tolist()))
    assert got[6 * W * W + 1 * W + 3] == 0
    assert got[7 * W * W + 1 * W + 3] == 20
    # customer 4 with the run (1, 2): (0, 4, 3, 1, 2, 0): 40 + 10 + 20 + 10 + 20 = 100
    assert got[6 * W * W + 4 * W + 1] == 20
    # candidates: runs (1,2), (2,3), (3,4); singles not in the run: 2 each -> 6; run pairs: (1,2)-(3,4) -> 1
    assert len(got) == 7


@pytest.mark.parametrize("kind", ["cvrp", "vrptw", "vrpspdtw", "vrpspd"])
@pytest.mark.parametrize("seed", range(5))
def test_candidate_sets_against_brute_force(kind, seed):
    """Every candidate (move index -> delta) equals a from-scratch recompute of
    the whole neighbour solution built by independent Python list surgery."""
    n = 5 + seed % 4
    inst, sol = _tiny(kind, n, 300 + seed, m_extra_empty=1)
    routes = sol.routes()
    expect = brute_moves(inst, routes, I.MASK_ALL)
    for method in ("def", "concat"):
        idx, dl = O.list_moves(inst, sol, I.MASK_ALL, method)
        got = dict(zip(idx.tolist(), dl.tolist()))
        assert got == expect, method
    bm = O.best_move(inst, sol, I.MASK_ALL, "def")
    best = min((d, i) for i, d in expect.items())
    assert (bm["delta"], bm["idx"]) == best


def _closed_form_count(n, lens, mask):
    m = len(lens)
    A = n + m
    c = 0
    runs2 = sum(max(0, L - 1) for L in lens)          # runs of two consecutive customers
    if mask & 64:           # a customer with a run of two it is not part of
        c += runs2 * (n - 2)
    if mask & 128:          # unordered pairs of runs of two that share no customer
        c += runs2 * (runs2 - 1) // 2 - sum(max(0, L - 2) for L in lens)
    if mask & 1:
        c += n * (A - 2)
    if mask & 2:
        c += n * (n - 1) // 2
    if mask & 4:
        c += sum(L * (L - 1) // 2 for L in lens)
    if mask & 8:
        c += (A * A - sum((L + 1) ** 2 for L in lens)) // 2
    if mask & 16:
        c += sum(max(0, L - 1) for L in lens) * (A - 3)
    if mask & 32:
        c += sum(max(0, L - 2) for L in lens) * (A - 4)
    return c


@pytest.mark.parametrize("mask", [1, 2, 4, 8, 16, 32, 64, 128, I.MASK_ALL, I.MASK_EXT, I.MASK_CONFIG1,
                                  I.MASK_CONFIG3])
def test_candidate_counts_closed_form(mask):
    for kind, n, seed in (("cvrp", 40, 1), ("vrptw", 60, 2), ("cvrp", 7, 3)):
        inst, sol = _tiny(kind, n, seed, m_extra_empty=2)
        lens = [len(r) for r in sol.routes()]
        assert O.count_candidates(inst, sol, mask) == _closed_form_count(n, lens, mask)


def test_textbook_cvrp_deltas():
    """CVRP special cases that reduce to textbook edge formulas:
    2-opt: c(u-,v)+c(u,v+)-c(u-,u)-c(v,v+); inter-route relocate:
    c(u-,u+)-c(u-,u)-c(u,u+)+c(v,u)+c(u,v+)-c(v,v+) plus the load-penalty
    change of both routes."""
    inst, sol = _tiny("cvrp", 30, 9, m_extra_empty=0)
    c = inst.dist.astype(np.int64)
    routes = sol.routes()
    n, m = inst.n, len(routes)
    W = n + 1 + m
    idx, dl = O.list_moves(inst, sol, 4 | 1, "def")
    got = dict(zip(idx.tolist(), dl.tolist()))
    pos = {x: (r, i) for r, rt in enumerate(routes) for i, x in enumerate(rt)}
    loads = [sum(int(inst.demand[x]) for x in rt) for rt in routes]
    pen = lambda L: inst.w_load * max(0, L - inst.capacity)
    checked = 0
    for rt in routes:
        full = [0] + rt + [0]
        for i in range(1, len(full) - 1):
            for j in range(i + 1, len(full) - 1):
                u, v = full[i], full[j]
                want = c[full[i - 1], v] + c[u, full[j + 1]] - c[full[i - 1], u] - c[v, full[j + 1]]
                assert got[2 * W * W + u * W + v] == want
                checked += 1
    for u in range(1, n + 1):
        ra, i = pos[u]
        fa = [0] + routes[ra] + [0]
        um, up = fa[i], fa[i + 2]
        for rb in range(m):
            if rb == ra:
                continue
            fb = [0] + routes[rb] + [0]
            for j in range(len(fb) - 1):
                v, vp = fb[j], fb[j + 1]
                anchor = n + 1 + rb if j == 0 else v
                want = (c[um, up] - c[um, u] - c[u, up] + c[v, u] + c[u, vp] - c[v, vp]
                        + pen(loads[ra] - inst.demand[u]) - pen(loads[ra])
                        + pen(loads[rb] + inst.demand[u]) - pen(loads[rb]))
                assert got[u * W + anchor] == want
                checked += 1
    assert checked > 500


def test_two_opt_descent_reaches_convex_order():
    """Points in convex position: a tour is optimal iff it has no crossing
    edges, and every crossing can be removed by an improving 2-opt move, so
    a 2-opt local optimum is the angular order (either direction)."""
    k = 14
    pts = [(int(round(5000 + 5000 * math.cos(2 * math.pi * t / (k + 1)))),
            int(round(5000 + 5000 * math.sin(2 * math.pi * t / (k + 1))))) for t in range(k + 1)]
    dist = I.rounded_euclidean(np.array(pts, np.int64))     # node 0 (depot) is on the circle too
    inst = I.instance_from_arrays("circle", dist, [0] + [1] * (dist.shape[0] - 1), 10 ** 6)
    n = inst.n
    rng = random.Random(5)
    perm = list(range(1, n + 1))
    rng.shuffle(perm)
    sol = _sol(perm, [0, n])
    final, steps, log, _ = O.descend(inst, sol, 4, "def")
    tour = final.tour.tolist()
    assert steps > 0
    assert tour == sorted(tour) or tour == sorted(tour, reverse=True)


@pytest.mark.parametrize("kind,n,seed,mask", [
    ("cvrp", 25, 1, I.MASK_CONFIG1), ("vrptw", 30, 2, I.MASK_ALL),
    ("cvrp", 40, 3, I.MASK_CONFIG3), ("vrptw", 45, 4, I.MASK_ALL),
    ("vrpspdtw", 35, 5, I.MASK_ALL), ("vrpspd", 30, 6, I.MASK_ALL),
    ("cvrp", 30, 7, I.MASK_EXT), ("vrptw", 35, 8, I.MASK_EXT)])
def test_descent_invariants(kind, n, seed, mask):
    inst, sol = _tiny(kind, n, seed, m_extra_empty=1)
    c0 = O.solution_cost(inst, sol)
    final, steps, log, cands = O.descend(inst, sol, mask, "def")
    deltas = [O.unpack_key(k)[0] for k in log]
    assert len(log) == steps + 1
    assert all(d < 0 for d in deltas[:-1]) and deltas[-1] >= 0
    assert O.solution_cost(inst, final) == c0 + sum(deltas[:-1])
    assert O.check_solution(inst, final) == 0
    assert final.n_routes == sol.n_routes
    assert sorted(final.tour.tolist()) == list(range(1, n + 1))
    assert sum(int(inst.demand[x]) for x in final.tour) == int(inst.demand.sum())
    bm = O.best_move(inst, final, mask, "def")
    assert bm["delta"] >= 0 and bm["key"] == int(log[-1])
    # the concatenation evaluator follows the identical trajectory
    final2, steps2, log2, cands2 = O.descend(inst, sol, mask, "concat")
    assert steps2 == steps and (log2 == log).all() and cands2 == cands
    assert (final2.tour == final.tour).all()


def test_empty_neighbourhood():
    inst = I.instance_from_arrays("one", np.array([[0, 3], [3, 0]]), [0, 1], 5)
    sol = _sol([1], [0, 1])
    assert O.count_candidates(inst, sol, I.MASK_ALL) == 0
    assert O.best_move(inst, sol, I.MASK_ALL)["found"] is False
    final, steps, log, _ = O.descend(inst, sol, I.MASK_ALL)
    assert steps == 0 and int(log[0]) == O.NO_MOVE_KEY


def test_apply_rejects_non_candidates():
    inst, sol = _tiny("cvrp", 10, 1, m_extra_empty=0)
    route = next(r for r in sol.routes() if len(r) >= 2)
    u, pred = route[1], route[0]
    with pytest.raises(ValueError):
        O.apply_move(inst, sol, 0, u, pred)         # v == pred(u)
    with pytest.raises(ValueError):
        O.apply_move(inst, sol, 1, 5, 5)            # swap needs a < b


# ----------------------------------------------------------------------------
# edge-based extraction with a granular mask (Section 5.3.1)

def test_granular_neighbors_are_the_nearest_customers():
    inst = I.vrptw(40, 8)
    nbr = I.granular_neighbors(inst, 6)
    assert nbr.shape == (41, 6) and (nbr[0] == 0).all()
    for x in range(1, 41):
        order = sorted((int(inst.dist[x][y]), y) for y in range(1, 41) if y != x)
        assert nbr[x].tolist() == [y for _, y in order[:6]]


@pytest.mark.parametrize("kind", ["cvrp", "vrptw"])
@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("theta", [1, 2, 4])
def test_granular_candidate_sets_against_brute_force(kind, seed, theta):
    """The kept candidates and their deltas equal the brute force restricted by
    an independent Python statement of the same mask rule."""
    n = 6 + seed % 3
    inst, sol = _tiny(kind, n, 700 + seed, m_extra_empty=1)
    nbr = I.granular_neighbors(inst, theta)
    expect = brute_moves(inst, sol.routes(), I.MASK_ALL, nbr)
    for method in ("def", "concat"):
        idx, dl = O.list_moves(inst, sol, I.MASK_ALL, method, granular=nbr)
        assert dict(zip(idx.tolist(), dl.tolist())) == expect, method
        assert O.count_candidates(inst, sol, I.MASK_ALL, granular=nbr) == len(expect)
    bm = O.best_move(inst, sol, I.MASK_ALL, "def", granular=nbr)
    assert (bm["delta"], bm["idx"]) == min((d, i) for i, d in expect.items())


def test_granular_full_mask_is_the_node_based_set():
    """With every other customer in every row, the edge-based set is the full
    node-based set minus the 2-opt* exchanges of two whole routes."""
    inst, sol = _tiny("vrptw", 8, 31, m_extra_empty=1)
    n, m = inst.n, sol.n_routes
    W = n + 1 + m
    full_idx, full_dl = O.list_moves(inst, sol, I.MASK_ALL, "def")
    g_idx, g_dl = O.list_moves(inst, sol, I.MASK_ALL, "def", granular=I.granular_neighbors(inst, n - 1))
    full = {int(i): int(d) for i, d in zip(full_idx, full_dl)
            if not (i // (W * W) == 3 and (i % (W * W)) // W > n and i % W > n)}
    assert {int(i): int(d) for i, d in zip(g_idx, g_dl)} == full


def test_granular_descent_definition_equals_concatenation():
    inst = I.vrptw(35, 12)
    inst.capacity = 90
    sol = I.random_split_solution(inst, 13)
    nbr = I.granular_neighbors(inst, 5)
    f1, s1, l1, c1 = O.descend(inst, sol, I.MASK_ALL, "def", granular=nbr)
    f2, s2, l2, c2 = O.descend(inst, sol, I.MASK_ALL, "concat", granular=nbr)
    assert s1 == s2 > 0 and (l1 == l2).all() and c1 == c2
    assert (f1.tour == f2.tour).all() and O.check_solution(inst, f1) == 0
    # the restricted descent stops at a local optimum of the restricted set
    assert O.best_move(inst, f1, I.MASK_ALL, "def", granular=nbr)["delta"] >= 0


@pytest.mark.parametrize("kind,mask", [("cvrp", I.MASK_CONFIG3), ("vrptw", I.MASK_ALL), ("cvrp", I.MASK_EXT),
                                       ("vrpspdtw", I.MASK_ALL)])
@pytest.mark.parametrize("stride", [1, 3, 7])
def test_slices_partition_the_candidate_set(kind, mask, stride):
    """The interleaved slices the harness spreads over host processes: their
    counts add up to the full count, the smallest key among them is the full
    evaluation's best move, and each slice's best is the smallest key of its
    own candidates in the full listing (so no slice visits a candidate twice
    or misses one)."""
    inst, sol = _tiny(kind, 14, 5 + stride)
    full = O.best_move(inst, sol, mask, "concat")
    idx, delta = O.list_moves(inst, sol, mask, "concat")
    keys = {int(i): O.pack_key(int(d), int(i)) for i, d in zip(idx, delta)}
    parts = [O.best_move_slice(inst, sol, mask, ph, stride) for ph in range(stride)]
    assert sum(p["candidates"] for p in parts) == full["candidates"] == len(idx)
    assert min(p["key"] for p in parts) == full["key"]
    # the slice rule restated: the outermost index of (op, a, b)
    n, routes = inst.n, sol.routes()
    W = n + 1 + len(routes)
    route_of = {x: r for r, nodes in enumerate(routes) for x in nodes}
    route_of.update({n + 1 + r: r for r in range(len(routes))})

    def outer(i):
        op, a, b = i // (W * W), (i % (W * W)) // W, i % W
        if op in (2, 3):
            return route_of[a]
        return b if op in (6, 7) else a

    for ph, p in enumerate(parts):
        mine = [k for i, k in keys.items() if outer(i) % stride == ph]
        assert p["candidates"] == len(mine)
        assert p["key"] == (min(mine) if mine else O.NO_MOVE_KEY)
    with pytest.raises(ValueError):
        O.best_move_slice(inst, sol, mask, stride, stride)
