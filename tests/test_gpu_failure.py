"""Failure detection on the device (marked gpu): every device-side wait of
the library is bounded, and a wait that runs out stops the kernel, reports
TGA_ERR_TIMEOUT and leaves a context that a rebuild makes usable again.
The waits are made to run out with a zero time limit (tga_set_wait_limit),
so nothing here faults, traps or hangs a GPU: each wait checks its flag
once and gives up."""
import numpy as np
import pytest

import oracle as O
from paper_2506_17357_gb300 import instances as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2506_17357_gb300 import tga as T  # noqa: E402


def _case(n=80, seed=21):
    inst = I.cvrp_uniform(n, seed)
    inst.capacity = -(-int(inst.demand.sum()) // 6)
    return inst, I.random_split_solution(inst, seed + 1)


def _recovers(ls, inst, mask):
    """After a rebuild the context descends from the caller's current
    solution exactly like the oracle."""
    tour, rs = ls.solution()
    start = I.Solution(tour, rs)
    assert O.check_solution(inst, start) == 0          # the caller's arrays hold a whole solution
    T.tga_set_wait_limit(ls.ctx, -1)
    ls.build()
    st = ls.descend()
    fin, steps, _, _ = O.descend(inst, start, mask, "concat")
    assert st["status"] == 0 and st["steps"] == steps
    tour2, rs2 = ls.solution()
    assert np.array_equal(tour2, fin.tour) and np.array_equal(rs2, fin.route_start)


def test_batched_idle_wait_runs_out_and_the_context_recovers():
    """One small job in the batched launch: every CTA without a chunk polls
    idle, and with a zero limit its second poll gives up."""
    inst, sol = _case()
    mask = I.MASK_CVRP_MIXED
    ls = T.LocalSearch(inst, sol, mask).build()
    try:
        T.tga_set_wait_limit(ls.ctx, 0)
        with pytest.raises(T.TGAError) as e:
            T.tga_descend_batch([ls.ctx])
        assert e.value.code == T.TGA_ERR_TIMEOUT
        _recovers(ls, inst, mask)
    finally:
        ls.close()


def test_persistent_wait_runs_out_and_leaves_the_solution_untouched():
    """The persistent descent: CTAs that finish their share first wait for
    the step's plan (and later at the grid barrier); with a zero limit they
    give up at once, the descent stops with TGA_ERR_TIMEOUT and the caller's
    solution is not written back (it may be mid-update on the device)."""
    inst, sol = _case(120, 31)
    mask = I.MASK_CVRP_MIXED
    ls = T.LocalSearch(inst, sol, mask).build()
    try:
        ls.set_descent_mode(T.DESCENT_PERSISTENT)
        T.tga_set_wait_limit(ls.ctx, 0)
        with pytest.raises(T.TGAError) as e:
            ls.descend()
        assert e.value.code == T.TGA_ERR_TIMEOUT
        tour, rs = ls.solution()
        assert np.array_equal(tour, sol.tour) and np.array_equal(rs, sol.route_start)
        mode, grid = T.tga_get_descent_mode(ls.ctx)
        assert mode == T.DESCENT_PERSISTENT and grid > 1
        _recovers(ls, inst, mask)
    finally:
        ls.close()


def test_default_limits_are_restored():
    inst, sol = _case(60, 41)
    ls = T.LocalSearch(inst, sol, I.MASK_CVRP_MIXED).build()
    try:
        T.tga_set_wait_limit(ls.ctx, 0)
        T.tga_set_wait_limit(ls.ctx, -1)
        ls.set_descent_mode(T.DESCENT_PERSISTENT)
        st = ls.descend()
        assert st["status"] == 0 and st["local_optimum"] == 1
    finally:
        ls.close()
