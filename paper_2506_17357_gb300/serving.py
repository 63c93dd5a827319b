"""Continuous-batching serving loop for local-search jobs over the C-ABI.

Requests (an instance plus an initial solution) arrive over time.  A request
is admitted as soon as a slot is free and its device footprint fits the
memory budget; admission copies its (pinned) host arrays to the device on
the slot's own CUDA stream, builds the attributes and enqueues the whole
descent (tga_descend_async: a CUDA graph with a device-driven loop, so
kernels of different jobs interleave on the SMs).  Jobs admitted while others
run overlap on the GPU; finished jobs are retired (a device-to-host read of
the final solution and counters), which frees their slot and budget for the
next arrivals.  ``max_slots=1`` is the one-at-a-time plain path: one job on
the GPU at a time, in arrival order, each descending along the library's
default (fastest single-job) path, which may claim every SM.

Admission is first-come first-served: a request that does not fit waits at
the head of the queue (no reordering, so no starvation).  Results do not
depend on the mix: each job runs the same kernels on its own state.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import List, Optional

import numpy as np

from . import tga as T


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    inst: object            # instances.Instance
    sol: object             # instances.Solution
    op_mask: int


@dataclasses.dataclass
class Result:
    rid: int
    n: int
    kind: str
    arrival_s: float
    admitted_s: float
    finished_s: float
    steps: int
    candidates: int
    initial_cost: int
    final_cost: int
    status: int
    tour: Optional[np.ndarray] = None
    route_start: Optional[np.ndarray] = None
    move_log: Optional[np.ndarray] = None

    @property
    def latency_s(self) -> float:
        return self.finished_s - self.arrival_s


# Device allocators hand out memory in 2 MiB granules: torch's caching
# allocator rounds each large block up to them (small arrays share 2 MiB
# segments) and so does the stream-ordered pool behind the library's
# workspace.  A job's descent graph and its streams take a little device
# memory of their own.
_GRANULE = 2 << 20
_GRAPH_ALLOWANCE = 16 << 20


def _granules(nbytes: int) -> int:
    return -(-int(nbytes) // _GRANULE) * _GRANULE


def footprint_bytes(n: int, m: int) -> int:
    """Device bytes one job holds while admitted: the instance matrix, the
    small instance and solution arrays (one shared 2 MiB segment counted per
    job), the context workspace and its tile list, each rounded up to the
    allocators' 2 MiB granules, plus an allowance for the descent graph."""
    matrix = _granules(4 * (n + 1) * (n + 1))
    small = _GRANULE
    tiles = _granules(8 * (-(-(n + m) // 8)) * (-(-(n + m) // 64)))     # largest tile list of the default shapes
    return matrix + small + _granules(T.tga_workspace_bytes(n, m)) + tiles + _GRAPH_ALLOWANCE


class _Pinned:
    """Host copy of a request in page-locked memory (what a real request
    payload would arrive in), so admission copies are asynchronous."""

    def __init__(self, torch, req: Request):
        inst, sol = req.inst, req.sol

        def pin(a):
            t = torch.empty(int(np.asarray(a).size), dtype=torch.int32).pin_memory()
            t.numpy()[:] = np.ascontiguousarray(a, dtype=np.int32).reshape(-1)
            return t
        self.arrays = [pin(inst.dist), pin(inst.demand), pin(inst.service), pin(inst.tw_early),
                       pin(inst.tw_late), pin(sol.tour), pin(sol.route_start)]


class _Job:
    def __init__(self, torch, device, stream, req: Request, pinned: _Pinned, log_capacity: int,
                 mode: int = T.DESCENT_AUTO):
        self.torch = torch
        self.req = req
        self.stream = stream
        inst = req.inst
        self.n = int(inst.n)
        self.m = int(np.asarray(req.sol.route_start).size - 1)
        with torch.cuda.stream(stream):
            self.dev = [torch.empty_like(h, device=device).copy_(h, non_blocking=True) for h in pinned.arrays]
            self.log = (torch.full((log_capacity,), -1, dtype=torch.int64, device=device)
                        if log_capacity else None)
        dist, demand, service, early, late, tour, rs = self.dev
        tw = bool(inst.has_tw)
        self.c_inst = T.tga_instance(self.n, self.m, int(inst.capacity), int(tw), int(inst.w_load),
                                     int(inst.w_tw), dist.data_ptr(), demand.data_ptr(),
                                     service.data_ptr() if tw else None, early.data_ptr() if tw else None,
                                     late.data_ptr() if tw else None)
        self.c_sol = T.tga_solution(tour.data_ptr(), rs.data_ptr())
        self.ctx = T.tga_create(self.c_inst, self.c_sol, req.op_mask, stream.cuda_stream)
        if self.log is not None:
            T.tga_set_move_log(self.ctx, self.log.data_ptr(), log_capacity)
        T.tga_set_descent_mode(self.ctx, mode)
        T.tga_build_attrs(self.ctx)
        T.tga_descend_async(self.ctx)

    def done(self) -> bool:
        return T.tga_query(self.ctx)

    def finish(self, keep_solution: bool):
        st = T.tga_get_stats(self.ctx)            # synchronises the slot's stream (already idle)
        tour = rs = log = None
        if keep_solution:
            torch = self.torch
            with torch.cuda.stream(self.stream):       # copy on the slot's own stream
                tour = self.dev[5].cpu().numpy().copy()
                rs = self.dev[6].cpu().numpy().copy()
                if self.log is not None:
                    k = min(int(st["evaluations"]), self.log.shape[0])
                    log = self.log[:k].cpu().numpy().view(np.uint64).copy()
        T.tga_destroy(self.ctx)
        self.ctx = None
        self.dev = None
        self.log = None
        return st, tour, rs, log


class Server:
    """Serve requests with at most ``max_slots`` jobs on the GPU and a device
    memory budget of ``budget_bytes`` for their footprints."""

    def __init__(self, budget_bytes: int = 1 << 30, max_slots: int = 32, device="cuda:0",
                 log_capacity: int = 0, keep_solutions: bool = True, poll_s: float = 50e-6):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(self.max_slots)]
        self.log_capacity = int(log_capacity)
        self.keep = keep_solutions
        self.poll_s = poll_s

    def serve(self, requests: List[Request], pinned: Optional[dict] = None) -> List[Result]:
        torch = self.torch
        if pinned is None:
            pinned = {r.rid: _Pinned(torch, r) for r in requests}
        for r in requests:
            need = footprint_bytes(int(r.inst.n), int(np.asarray(r.sol.route_start).size - 1))
            if need > self.budget:
                raise ValueError(f"request {r.rid} needs {need} bytes, above the budget {self.budget}")
        arrivals = collections.deque(sorted(requests, key=lambda r: (r.arrival_s, r.rid)))
        queue = collections.deque()
        free = list(range(self.max_slots))
        active = {}                      # slot -> (job, admitted_s, bytes)
        used = 0
        results = []
        t0 = time.perf_counter()
        while arrivals or queue or active:
            now = time.perf_counter() - t0
            while arrivals and arrivals[0].arrival_s <= now:
                queue.append(arrivals.popleft())
            # retire finished jobs
            for slot in list(active):
                job, adm, nbytes = active[slot]
                if job.done():
                    st, tour, rs, log = job.finish(self.keep)
                    fin = time.perf_counter() - t0
                    r = job.req
                    results.append(Result(r.rid, job.n, r.inst.kind, r.arrival_s, adm, fin, int(st["steps"]),
                                          int(st["candidates"]), int(st["initial_cost"]),
                                          int(st["final_cost"]), int(st["status"]), tour, rs, log))
                    del active[slot]
                    free.append(slot)
                    used -= nbytes
            # admit in arrival order while a slot and the budget allow
            while queue and free:
                r = queue[0]
                need = footprint_bytes(int(r.inst.n), int(np.asarray(r.sol.route_start).size - 1))
                if used + need > self.budget:
                    break
                queue.popleft()
                slot = free.pop()
                adm = time.perf_counter() - t0
                # a persistent descent claims every SM: concurrent jobs use the graph path
                mode = T.DESCENT_AUTO if self.max_slots == 1 else T.DESCENT_GRAPH
                active[slot] = (_Job(torch, self.device, self.streams[slot], r, pinned[r.rid], self.log_capacity,
                                     mode), adm, need)
                used += need
            if not queue and active:
                time.sleep(self.poll_s)
            elif not active and not queue and arrivals:
                time.sleep(max(0.0, min(self.poll_s * 20, arrivals[0].arrival_s - (time.perf_counter() - t0))))
        results.sort(key=lambda x: x.rid)
        return results


def summarize(results: List[Result]) -> dict:
    lat = np.array([r.latency_s for r in results])
    span = max(r.finished_s for r in results) - min(r.arrival_s for r in results)
    return {"jobs": len(results), "jobs_per_s": len(results) / span if span > 0 else None,
            "p50_latency_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_latency_ms": 1e3 * float(np.percentile(lat, 99)),
            "mean_latency_ms": 1e3 * float(lat.mean()), "makespan_s": span,
            "candidates": int(sum(r.candidates for r in results)),
            "status": sorted({r.status for r in results})}
