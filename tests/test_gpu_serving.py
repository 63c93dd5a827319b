"""Continuous-batching serving loop (marked gpu): every result served in the
mix equals the same job descended alone (exact: move log, final solution,
cost), jobs admitted while others run overlap on the GPU, and the memory
budget bounds what is resident."""
import numpy as np
import pytest

from paper_2506_17357_gb300 import instances as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2506_17357_gb300 import serving as S  # noqa: E402
from paper_2506_17357_gb300 import tga as T  # noqa: E402


def _requests(count, lo, hi, seed, spread_s):
    sizes, kinds = I.serving_sizes(count, seed=seed, lo=lo, hi=hi)
    arr = np.linspace(0.0, spread_s, count)
    reqs = []
    for j in range(count):
        inst, sol = I.serving_job(j, int(sizes[j]), bool(kinds[j]), seed=seed)
        reqs.append(S.Request(j, float(arr[j]), inst, sol, I.mask_for(inst)))
    return reqs


def _alone(req):
    ls = T.LocalSearch(req.inst, req.sol, req.op_mask, log_capacity=1 << 15).build()
    try:
        st = ls.descend()
        return st, ls.move_log(), ls.solution()
    finally:
        ls.close()


@pytest.mark.parametrize("budget_mb,slots", [(256, 6), (60, 6)])   # 60 MiB: two or three jobs at a time
def test_served_results_equal_alone(budget_mb, slots):
    reqs = _requests(14, 30, 600, seed=7, spread_s=0.02)
    srv = S.Server(budget_bytes=budget_mb << 20, max_slots=slots, log_capacity=1 << 15)
    res = srv.serve(reqs)
    assert [r.rid for r in res] == [q.rid for q in reqs]
    for q, r in zip(reqs, res):
        st, log, (tour, rs) = _alone(q)
        assert r.status == 0
        assert (r.steps, r.final_cost, r.candidates) == (st["steps"], st["final_cost"], st["candidates"])
        assert np.array_equal(r.move_log, log)
        assert np.array_equal(r.tour, tour) and np.array_equal(r.route_start, rs)
        assert r.admitted_s >= r.arrival_s and r.finished_s >= r.admitted_s
    # the budget bounds the resident footprint at every admission
    events = sorted([(r.admitted_s, 1, r) for r in res] + [(r.finished_s, -1, r) for r in res],
                    key=lambda e: (e[0], e[1]))
    used, peak = 0, 0
    for _, kind, r in events:
        used += kind * S.footprint_bytes(r.n, int(np.asarray(reqs[r.rid].sol.route_start).size - 1))
        peak = max(peak, used)
    assert peak <= budget_mb << 20


def test_jobs_overlap_on_the_device():
    reqs = _requests(10, 200, 800, seed=8, spread_s=0.0)
    res = S.Server(budget_bytes=1 << 30, max_slots=8).serve(reqs)
    overlaps = sum(1 for a in res for b in res
                   if a.rid < b.rid and a.admitted_s < b.finished_s and b.admitted_s < a.finished_s)
    assert overlaps > 0
    one = S.Server(budget_bytes=1 << 30, max_slots=1).serve(reqs)
    assert [r.final_cost for r in one] == [r.final_cost for r in res]
    # one at a time: no two jobs are ever resident together
    for a in one:
        for b in one:
            if a.rid < b.rid:
                assert a.finished_s <= b.admitted_s or b.finished_s <= a.admitted_s


def test_request_above_budget_is_rejected():
    reqs = _requests(2, 500, 600, seed=9, spread_s=0.0)
    with pytest.raises(ValueError):
        S.Server(budget_bytes=1 << 20, max_slots=2).serve(reqs)


def test_admitted_job_holds_no_more_than_its_footprint():
    """The admission budget's per-job figure (footprint_bytes, built on
    tga_workspace_bytes and the allocators' 2 MiB granules) against the
    device memory a job really takes: the drop of free device memory when
    one job is admitted is at most its footprint and not far below it.  A
    footprint that missed the instance matrix or the position-ordered
    distance copy (each about 80-100 MB here) would fail.  The first
    admission of each kind is a warm-up (kernel code loaded on first use is
    not a per-job cost)."""
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    slack = 32 << 20
    for j, (n, tw) in enumerate([(4500, False), (4500, False), (5000, True), (5000, True)]):
        inst, sol = I.serving_job(j, n, tw, seed=12)
        req = S.Request(j, 0.0, inst, sol, I.mask_for(inst))
        pinned = S._Pinned(torch, req)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        free0 = torch.cuda.mem_get_info(dev)[0]
        job = S._Job(torch, dev, stream, req, pinned, 0, T.DESCENT_GRAPH)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info(dev)[0]
        need = S.footprint_bytes(n, int(np.asarray(sol.route_start).size - 1))
        while not job.done():
            pass
        st, _, _, _ = job.finish(False)
        assert st["status"] == 0
        used = free0 - free1
        if j % 2 == 0:
            continue                                     # warm-up admission
        assert used <= need, (n, used, need)
        assert used >= need - slack, (n, used, need)
