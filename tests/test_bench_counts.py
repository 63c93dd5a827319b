"""bench.py's roofline work counts (CPU): the closed-form inter-route
candidate counts per operator rank, which the reported achieved rates are
built from, equal the oracle's enumeration minus its intra-route candidates
(counted here by brute force over the route lengths)."""
import numpy as np
import pytest

import bench
import oracle as O
from paper_2506_17357_gb300 import instances as I


def _intra(lens, op):
    """Intra-route candidates of rank ``op`` for route lengths ``lens``,
    counted by enumeration of index pairs."""
    c = 0
    for L in lens:
        for i in range(L):
            for j in range(L):
                if op == 0 and j != i and j != i - 1:
                    c += 1                      # relocate i after element j (j = -1: the depot)
                elif op == 1 and i < j:
                    c += 1
                elif op == 2 and i < j:
                    c += 1
                elif op in (4, 5):
                    k = op - 2
                    if i + k <= L and not (i - 1 <= j <= i + k - 1):
                        c += 1
                elif op == 6 and i + 2 <= L and not (i <= j <= i + 1):
                    c += 1                      # run at i, customer j outside it
                elif op == 7 and i + 2 <= L and j + 2 <= L and j >= i + 2:
                    c += 1
        if op == 0:
            c += max(0, L - 1)                  # after the start depot: every customer but the first
        elif op in (4, 5):
            k = op - 2
            c += max(0, L - k)                  # after the start depot: every run but the first
    return c


@pytest.mark.parametrize("seed", range(4))
def test_inter_candidate_counts_match_the_oracle(seed):
    inst = I.cvrp_uniform(24, 40 + seed)
    inst.capacity = -(-int(inst.demand.sum()) // 4)
    sol = I.random_split_solution(inst, 50 + seed)
    rs = list(sol.route_start) + [inst.n]       # one empty route
    sol = I.Solution(sol.tour, np.asarray(rs, np.int32))
    lens = np.diff(sol.route_start)
    inter = bench.inter_candidates(inst.n, lens, I.MASK_EXT)
    for op in (0, 1, 3, 4, 5, 6, 7):
        total = O.count_candidates(inst, sol, 1 << op)
        assert inter.get(op, 0) == total - _intra(lens.tolist(), op), op
