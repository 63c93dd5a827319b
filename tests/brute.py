"""Pure-Python brute force over one local-search step (test helper).

Written independently of the C oracle: every neighbour is produced by Python
list surgery on a deep copy of the route list, and scored by recomputing the
whole solution's cost from scratch with a fresh forward simulation.  Used only
on tiny instances.

Objective: Section 2 of the paper with the penalised capacity excess (of the
largest load on board when the instance has pickups) and the time-warp
relaxation of Section 4.3.3 (weights w_load, w_tw).  Operators:
Section 4.1 (relocate, swap, 2-opt, 2-opt*) plus or-opt of 2-3 customers,
and the swaps of Section 5.3.1 with unequal or longer runs: a customer with a
run of two, and two runs of two.
"""
import copy


def peak_load(inst, route):
    """Largest load on board: after serving the first k customers the vehicle
    carries the deliveries still owed to customers k+1.. plus the pickups of
    customers 1..k (Section 2); k = 0 is the departure."""
    pk = getattr(inst, "pickup", None)
    d = [int(inst.demand[x]) for x in route]
    p = [0 if pk is None else int(pk[x]) for x in route]
    return max(sum(d[k:]) + sum(p[:k]) for k in range(len(route) + 1))


def route_cost(inst, route):
    if not route:
        return 0
    c = inst.dist
    seq = [0] + list(route) + [0]
    dist = sum(int(c[seq[k]][seq[k + 1]]) for k in range(len(seq) - 1))
    load = peak_load(inst, route)
    cost = dist + inst.w_load * max(0, load - inst.capacity)
    if inst.has_tw:
        t = int(inst.tw_early[0])
        warp = 0
        for k in range(1, len(seq)):
            a, b = seq[k - 1], seq[k]
            t = t + int(inst.service[a]) + int(c[a][b])
            t = max(t, int(inst.tw_early[b]))
            if t > int(inst.tw_late[b]):
                warp += t - int(inst.tw_late[b])
                t = int(inst.tw_late[b])
        cost += inst.w_tw * warp
    return cost


def total_cost(inst, routes):
    return sum(route_cost(inst, r) for r in routes)


def _locate(routes, x):
    for r, route in enumerate(routes):
        if x in route:
            return r, route.index(x)
    raise KeyError(x)


def brute_moves(inst, routes, mask, nbr=None):
    """dict move_index -> delta over the whole candidate set.  ``nbr``: the
    granular mask of the edge-based extraction (Section 5.3.1) as neighbour
    rows; an inter-route candidate is kept by the rule of the edge-based
    reading (relocate/or-opt: destination a start depot or in the moved
    customer's row; swap: either in the other's row; 2-opt*: one start depot,
    or either in the other's row), intra-route candidates always."""
    n, m = inst.n, len(routes)
    W = n + 1 + m
    base = total_cost(inst, routes)
    depot_anchor = {n + 1 + r: r for r in range(m)}
    anchors = list(range(1, n + 1)) + list(depot_anchor)
    out = {}
    near = None if nbr is None else {x: set(int(y) for y in nbr[x]) for x in range(1, n + 1)}

    def route_of(x):
        return depot_anchor[x] if x in depot_anchor else _locate(routes, x)[0]

    def kept(op, a, b):
        if near is None or op == 2 or route_of(a) == route_of(b):
            return True
        if op in (0, 4, 5):
            return b in depot_anchor or b in near[a]
        if op == 1:
            return b in near[a] or a in near[b]
        if a in depot_anchor and b in depot_anchor:
            return False
        if a in depot_anchor or b in depot_anchor:
            return True
        return b in near[a] or a in near[b]

    def record(op, a, b, new_routes):
        if not kept(op, a, b):
            return
        idx = op * W * W + a * W + b
        assert idx not in out
        out[idx] = total_cost(inst, new_routes) - base

    def pred(u):
        r, i = _locate(routes, u)
        return n + 1 + r if i == 0 else routes[r][i - 1]

    for op, k in ((0, 1), (4, 2), (5, 3)):
        if not mask >> op & 1:
            continue
        for u in range(1, n + 1):
            r, i = _locate(routes, u)
            run = routes[r][i:i + k]
            if len(run) < k:
                continue
            for v in anchors:
                if v in run or v == pred(u):
                    continue
                nr = copy.deepcopy(routes)
                del nr[r][i:i + k]
                if v in depot_anchor:
                    rv = depot_anchor[v]
                    nr[rv][0:0] = run
                else:
                    rv, j = _locate(nr, v)
                    nr[rv][j + 1:j + 1] = run
                record(op, u, v, nr)
    if mask >> 1 & 1:
        for a in range(1, n + 1):
            for b in range(a + 1, n + 1):
                nr = copy.deepcopy(routes)
                ra, i = _locate(nr, a)
                rb, j = _locate(nr, b)
                nr[ra][i], nr[rb][j] = b, a
                record(1, a, b, nr)
    # ops 6 / 7: a customer (6) or a run of two starting at a (7, a < b)
    # exchanges places with the run of two starting at b; the runs stay in
    # order and must not share a customer
    for op, k1 in ((6, 1), (7, 2)):
        if not mask >> op & 1:
            continue
        for b in range(1, n + 1):
            rb, j = _locate(routes, b)
            if j + 2 > len(routes[rb]):
                continue
            for a in range(1, n + 1):
                if op == 7 and not a < b:
                    continue
                ra, i = _locate(routes, a)
                if i + k1 > len(routes[ra]):
                    continue
                run_a = routes[ra][i:i + k1]
                run_b = routes[rb][j:j + 2]
                if set(run_a) & set(run_b):
                    continue
                nr = copy.deepcopy(routes)
                if ra != rb:
                    nr[ra][i:i + k1] = run_b
                    nr[rb][j:j + 2] = run_a
                else:
                    # rebuild the route as a sequence of placeholders
                    seq = list(routes[ra])
                    first, second = (i, j) if i < j else (j, i)
                    lf, ls = (k1, 2) if i < j else (2, k1)
                    new = (seq[:first] + seq[second:second + ls] + seq[first + lf:second] +
                           seq[first:first + lf] + seq[second + ls:])
                    nr[ra] = new
                record(op, a, b, nr)
    if mask >> 2 & 1:
        for r, route in enumerate(routes):
            for i in range(len(route)):
                for j in range(i + 1, len(route)):
                    nr = copy.deepcopy(routes)
                    nr[r][i:j + 1] = list(reversed(nr[r][i:j + 1]))
                    record(2, route[i], route[j], nr)
    if mask >> 3 & 1:
        for a in anchors:
            for b in anchors:
                ra = depot_anchor[a] if a in depot_anchor else _locate(routes, a)[0]
                rb = depot_anchor[b] if b in depot_anchor else _locate(routes, b)[0]
                if not ra < rb:
                    continue
                ia = -1 if a in depot_anchor else routes[ra].index(a)
                ib = -1 if b in depot_anchor else routes[rb].index(b)
                nr = copy.deepcopy(routes)
                nr[ra] = routes[ra][:ia + 1] + routes[rb][ib + 1:]
                nr[rb] = routes[rb][:ib + 1] + routes[ra][ia + 1:]
                record(3, a, b, nr)
    return out
