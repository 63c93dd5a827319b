"""Benchmark: best-improvement descent to a local optimum on one GB300.

One bench step = one whole pass of the hot path over one synthetic instance:
build the attribute representation from the initial solution, then evaluate
the full neighbourhood (relocate, swap, 2-opt, 2-opt*, or-opt), apply the best
move on the device, and repeat until no move improves (a local optimum).

Default run (no --workload): the headline is the largest single-GPU
workload, clustered CVRP with 1 depot + 10000 customers (relocate, swap,
2-opt*, or-opt; the distance matrix, 400 MB, exceeds L2), timed for --steps
descents after --warmup untimed ones.  The same JSON line carries, under
"configs", the other workloads measured in the same process: CVRP-100,
VRPTW-1000 (moves/s, time to the local optimum, roofline), the batched
launch of 256 jobs (jobs/s against 256 sequential descents) and the
continuous-batching server (jobs/s and p50/p99 latency against one job at a
time).

metric = candidate moves evaluated per second over the whole descent; the
line also carries time-to-local-optimum.  Inputs are device resident when the
timed region starts; L2 (129 MB) is flushed between timed steps by writing a
512 MB buffer.  ``e2e`` repeats the measurement through the public Python API
with host arrays: pinned H2D copies of the instance and solution, build,
descent, and a D2H read of the final tour, route boundaries and counters.

Roofline: the evaluation path is integer arithmetic (no dense contraction),
so its ceilings are the measured 32-bit integer issue rate of the GPU
(tga_measure_int_peak: a dependency-free add/max stream over every SM) and
the algorithmic bytes over the measured HBM bandwidth.

``cpu_baseline``: the CPU oracle (test infrastructure) on the host cores --
one core, and every core of the process's affinity set, where a pool of
processes splits the same evaluations into interleaved slices and the
smallest key is reduced exactly.  ``--impl reference`` times the oracle the
same way (all cores) on the headline workload.

Multi-GPU (torchrun): every rank runs an independent replica of the headline
on its own instance seed (replicas only; the path is not sharded); value is
the sum of all ranks' candidates over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2506_17357_gb300 import instances as I  # noqa: E402

WORKLOADS = {
    "vrptw1000": ("VRPTW 1 depot + 1000 customers, all five operators", I.config2, I.MASK_CONFIG2),
    "cvrp100": ("CVRP 1 depot + 100 customers, relocate/swap/2-opt/2-opt*", I.config1, I.MASK_CONFIG1),
    "cvrp10000": ("clustered CVRP 1 depot + 10000 customers, relocate/swap/2-opt*/or-opt", I.config3,
                  I.MASK_CONFIG3),
    "vrpspdtw1000": ("VRPSPDTW 1 depot + 1000 customers with pickups and deliveries, all five operators",
                     I.config_spd, I.MASK_ALL),
}
HEADLINE = "cvrp10000"

# Integer operations per inter-route candidate, counted from the delta
# expressions (adds/subs, min/max, multiplies, plus one compare for the
# running argmin).  Index: op rank.  CVRP and VRPTW (time-warp terms added);
# with pickups the load term of each new route is the three-way maximum of
# the largest-load constants instead of one sum (relocate/or-opt +5, swap +8,
# 2-opt* +4) and the intra-route 2-opt closes a load chain (+14).
# Ranks 6 and 7 (swaps of runs, --extended-swaps): two gap constants, two
# inserted pieces and two load terms, plus two time-warp chains of a piece
# each with time windows.
OPS_CVRP = {0: 8, 1: 13, 2: 6, 3: 13, 4: 8, 5: 8, 6: 15, 7: 15}
OPS_TW = {0: 20, 1: 36, 2: 22, 3: 22, 4: 20, 5: 20, 6: 39, 7: 39}
OPS_PD = {0: 25, 1: 44, 2: 36, 3: 26, 4: 25, 5: 25, 6: 0, 7: 0}      # ranks 6, 7 have no pickup variant

# Algorithmic bytes of one evaluation: every distance entry c(x, y) is
# needed by some candidate (relocate / swap pairs), 4 B each, plus the
# per-anchor records read once (64 B base + 128 B hoisted constants).
REC_BYTES_PER_ANCHOR = 192


def ops_table(inst):
    if getattr(inst, "pickup", None) is not None:
        return OPS_PD
    return OPS_TW if inst.has_tw else OPS_CVRP


def inter_candidates(n, lens, mask):
    """Valid inter-route candidates per op for route lengths ``lens``."""
    m = len(lens)
    A = n + m
    lens = np.asarray(lens, dtype=np.int64)
    other = A - (lens + 1)                      # anchors outside the route
    out = {}
    if mask & 1:
        out[0] = int((lens * other).sum())
    if mask & 2:
        out[1] = int((n * n - (lens * lens).sum()) // 2)
    if mask & 8:
        out[3] = int((A * A - ((lens + 1) ** 2).sum()) // 2)
    if mask & 16:
        out[4] = int((np.maximum(lens - 1, 0) * other).sum())
    if mask & 32:
        out[5] = int((np.maximum(lens - 2, 0) * other).sum())
    runs = np.maximum(lens - 1, 0)              # runs of two per route
    if mask & 64:                               # a run with a customer of another route
        out[6] = int((runs * (n - lens)).sum())
    if mask & 128:                              # two runs in different routes
        out[7] = int((runs.sum() ** 2 - (runs * runs).sum()) // 2)
    return out


def algorithmic_ops(n, lens, mask, table, ops=range(6)):
    """Integer operations of the inter-route candidates of ranks ``ops``."""
    return sum(table[op] * c for op, c in inter_candidates(n, lens, mask).items() if op in ops)


def descent_ops(op_candidates, table):
    """Integer operations of every candidate evaluated (per-operator totals
    from the device counters, weighted by the per-candidate counts above)."""
    return sum(table[op] * c for op, c in enumerate(op_candidates))


def evaluation_bytes(n, m):
    """Algorithmic bytes of one neighbourhood evaluation."""
    return 4 * (n + 1) ** 2 + REC_BYTES_PER_ANCHOR * (n + 1 + m)


def kernel_source_hash() -> str:
    """Hash of the kernel sources' code: comments and whitespace are removed
    first, so an edit of a comment keeps recorded counters valid."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("tga_kernels.cu", "tga_persist.cu", "tga_device.cuh", "tga_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2506_17357_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(re.sub(r"\s+", "", src).encode())
    return h.hexdigest()[:16]


def measured_traffic(workload, kernel):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary (profiles/dram_traffic.json), or None when the kernel sources
    changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    ent = rec.get(kernel, {}).get(workload)
    if not ent or ent.get("source_hash") != kernel_source_hash():
        return None
    return ent.get("dram_bytes_per_launch")


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)                                     # first sample lands before the region
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


def reduce_replicas(total_s, candidates, device):
    """Whole-job figures of N independent replicas (one per rank): the
    slowest rank's time and the candidates of all ranks.  Single process:
    the inputs themselves."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_s), float(candidates)
    t = torch.tensor([float(total_s)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(candidates)], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def replica_seed(base_seed, rank):
    """Instance seed of a rank's replica: every rank descends its own instance."""
    return base_seed + rank


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


OP_NAMES = ["relocate", "swap", "2-opt", "2-opt*", "or-opt-2", "or-opt-3", "swap-1-2", "swap-2-2"]
_T0 = time.time()


def progress(msg):
    """One line per bench phase on stderr (wall seconds since start), so a slow phase shows."""
    print(f"[bench {time.time() - _T0:7.1f}s] {msg}", file=sys.stderr, flush=True)


def workload(args, name=None):
    """(description, generator, operator mask) of the chosen workload;
    --extended-swaps adds ranks 6 and 7 (swaps of runs) to its mask."""
    desc, make, mask = WORKLOADS[name or args.workload]
    if getattr(args, "extended_swaps", False):
        desc, mask = desc + ", plus the swaps of runs (ranks 6, 7)", mask | I.MASK_EXT
    return desc, make, mask


def workload_name(args, name=None):
    return (name or args.workload) + ("-xswap" if getattr(args, "extended_swaps", False) else "")


def only_descent(args):
    """One build + descent of the workload and nothing else (no timing): the
    command profilers run to list the per-step kernel launches."""
    import torch
    from paper_2506_17357_gb300 import tga as T
    wl = HEADLINE if args.workload == "all" else args.workload
    desc, make, mask = workload(args, wl)
    inst, sol = make(args.seed)
    nbr = I.granular_neighbors(inst, args.granular) if args.granular else None
    ls = T.LocalSearch(inst, sol, mask, granular=nbr).build()
    if args.tile:
        tile = ls.set_tile(*[int(x) for x in args.tile.split(",")])
    else:
        tile = ls.set_tile(0, 0)                                   # autotune, as the timed bench does
    if args.persistent_shape:                                      # the persistent path under a set shape
        T.tga_set_persistent_shape(ls.ctx, *[int(x) for x in args.persistent_shape.split(",")])
        ls.set_descent_mode(T.DESCENT_PERSISTENT)
    st = ls.descend(max_steps=args.descent_steps) if args.descent_steps else ls.descend()
    torch.cuda.synchronize()
    mode_used, grid = T.tga_get_descent_mode(ls.ctx)
    print(json.dumps({"workload": workload_name(args, wl), "tile": list(tile), "steps": st["steps"],
                      "descent_path": T.DESCENT_NAMES[mode_used], "grid": grid,
                      "persistent_shape": list(T.tga_get_persistent_shape(ls.ctx)),
                      "evaluations": st["evaluations"],
                      "final_cost": st["final_cost"], "status": st["status"]}))
    ls.close()


# ---------------------------------------------------------------------------
# peaks

def measure_int_peak(dev_index=0):
    """Measured 32-bit integer rate of the GPU (tga_measure_int_peak) with the
    SM clock sampled during the measurement; the nominal issue rate from the
    device's SM count and clock is kept as a cross-check."""
    import torch
    from paper_2506_17357_gb300 import tga as T
    props = torch.cuda.get_device_properties(dev_index)
    nsm = int(props.multi_processor_count)
    s = torch.cuda.Stream()
    T.tga_measure_int_peak(0, s.cuda_stream, 64)              # load the code, ramp the clocks
    with ClockSampler(dev_index) as clk:
        add_max, ms0 = T.tga_measure_int_peak(0, s.cuda_stream, 4000)
        add3, ms1 = T.tga_measure_int_peak(1, s.cuda_stream, 4000)
        add_max2, _ = T.tga_measure_int_peak(0, s.cuda_stream, 4000)
    clocks = clk.summary()
    add_max = max(add_max, add_max2)
    peaks, _ = load_peaks()
    sm_max = float(clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0))
    nominal = nsm * 4 * 32 * sm_max * 1e6
    return {"ops_per_s": add_max, "kernel": "tga_measure_int_peak kind 0 (x = max(x + a, b), 8 independent "
                                            "chains per thread, every SM)",
            "add_max_ops_per_s": add_max, "add3_ops_per_s": add3, "ms": [ms0, ms1],
            "nominal_issue_ops_per_s": nominal, "measured_over_nominal": add_max / nominal,
            "sm_count": nsm, "clocks": clocks}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on one core and on all cores

_W = {}


def _cpu_worker_init(wl_name, seed, mask, states, granular):
    import oracle as O
    _, make, _ = WORKLOADS[wl_name]
    inst, _ = make(seed)
    _W.update(O=O, inst=inst, mask=mask, states=states,
              nbr=I.granular_neighbors(inst, granular) if granular else None)


def _cpu_worker_task(units):
    """units: [(state index, phase, stride)]; returns (min key, candidates,
    start, end) with host wall-clock times."""
    O, inst, mask, states, nbr = _W["O"], _W["inst"], _W["mask"], _W["states"], _W["nbr"]
    t0 = time.time()
    best, cands = O.NO_MOVE_KEY, 0
    for si, ph, st in units:
        tour, rs = states[si]
        r = O.best_move_slice(inst, I.Solution(tour, rs), mask, ph, st, "concat", granular=nbr)
        best = min(best, r["key"])
        cands += r["candidates"]
    return best, cands, t0, time.time()


def cpu_baseline(args, wl_name, seconds=15.0, all_core_target_s=5.0, per_op_seconds=1.0, pool_cores=None):
    """The oracle's concatenation evaluator (plain single-threaded C) on the
    host: best-improvement steps of the workload from its initial solution.
    One core: evaluations along the trajectory (each split into slices when
    one evaluation is long), as many as fit in ``seconds``.  All cores: the
    same slices (repeated to fill about ``all_core_target_s`` seconds of wall
    time) spread over a spawn pool of one process per core; the rate is the
    candidates over the wall time from the first slice's start to the last
    one's end."""
    import multiprocessing as mp
    import oracle as O
    desc, make, mask = workload(args, wl_name)
    inst, sol = make(args.seed)
    theta = getattr(args, "granular", 0)
    nbr = I.granular_neighbors(inst, theta) if theta else None
    est = O.count_candidates(inst, sol, mask, granular=nbr) / 1e7      # rough seconds per evaluation
    stride = max(1, int(math.ceil(est / 0.5)))
    # ---- one core
    states, units, unit_s = [(np.asarray(sol.tour, np.int32), np.asarray(sol.route_start, np.int32))], [], []
    cur, si = sol, 0
    cands, evals = 0, 0
    t0 = time.perf_counter()
    done = False
    while not done:
        best = None
        for ph in range(stride):
            t1 = time.perf_counter()
            r = O.best_move_slice(inst, cur, mask, ph, stride, "concat", granular=nbr)
            unit_s.append(time.perf_counter() - t1)
            units.append((si, ph, stride))
            cands += r["candidates"]
            if r["found"] and (best is None or r["key"] < best["key"]):
                best = r
            if time.perf_counter() - t0 >= seconds:
                done = True
                break
        if done:
            break
        evals += 1
        if best is None or best["delta"] >= 0:                 # local optimum: start the trajectory over
            cur = sol
            si = 0
        else:
            cur = O.apply_move(inst, cur, best["op"], best["a"], best["b"])
            states.append((np.asarray(cur.tour, np.int32), np.asarray(cur.route_start, np.int32)))
            si = len(states) - 1
    dt1 = time.perf_counter() - t0
    single = cands / dt1
    sample1 = (f"{len(units)} slices of 1/{stride} evaluation" if stride > 1 else f"{len(units)} evaluations") + \
        f" along the trajectory of {workload_name(args, wl_name)} seed {args.seed}, {dt1:.1f} s"
    # ---- all cores
    K = pool_cores or host_cores()
    reps = max(1, int(round(K * all_core_target_s / max(dt1, 1e-3))))
    work = [(u, t) for _ in range(reps) for u, t in zip(units, unit_s)]
    tasks, cur_task, acc = [], [], 0.0
    for u, t in work:                                          # chunks of about 0.25 s of one core
        cur_task.append(u)
        acc += t
        if acc >= 0.25:
            tasks.append(cur_task)
            cur_task, acc = [], 0.0
    if cur_task:
        tasks.append(cur_task)
    ctx = mp.get_context("spawn")
    with ctx.Pool(K, initializer=_cpu_worker_init,
                  initargs=(wl_name, args.seed, mask, states, theta)) as pool:
        pool.map(time.sleep, [0.05] * K)                       # every worker has started
        res = pool.map(_cpu_worker_task, tasks, chunksize=1)
    start = min(r[2] for r in res)
    end = max(r[3] for r in res)
    all_cands = sum(r[1] for r in res)
    allv = all_cands / (end - start)
    # per operator: the oracle's evaluation of the initial solution with only
    # that operator enabled (about a second each; long evaluations in slices)
    per_op = {}
    for op in range(8):
        if not (mask >> op) & 1 or per_op_seconds <= 0:
            continue
        t1 = time.perf_counter()
        reps1 = c1 = 0
        while time.perf_counter() - t1 < per_op_seconds:
            c1 += O.best_move_slice(inst, sol, 1 << op, reps1 % stride, stride, "concat",
                                    granular=nbr)["candidates"]
            reps1 += 1
        d1 = time.perf_counter() - t1
        per_op[OP_NAMES[op]] = {"ms_per_evaluation": 1e3 * d1 / reps1 * stride, "candidates_per_s": c1 / d1}
    return {"value": allv, "unit": "candidate moves/s", "cores": K, "kind": "oracle",
            "cores_used": K, "host_cores": host_cores(), "os_cpu_count": os.cpu_count(),
            "single_core": single, "all_cores": allv,
            "sample": f"one core: {sample1}; all {K} cores: the same slices x{reps} in {len(tasks)} tasks of a "
                      f"spawn pool, {end - start:.1f} s wall (concatenation evaluator"
                      f"{', granular mask theta=%d' % theta if theta else ''})",
            "per_operator": per_op}


# ---------------------------------------------------------------------------
# single-instance workloads

def breakdown(inst, sol, mask, dev, stream, reps=200, step_count=200):
    """Per-operator and per-step GPU times of the workload, outside the timed
    region (the paper's per-operator and key-step analyses, Sections 6.6 and
    6.7).  Per operator: one neighbourhood evaluation with only that operator
    enabled (tga_eval_best_move: its kernels, autotuned inter tile) on the
    initial solution, `reps` evaluations captured in one CUDA graph and
    replayed, so the figure is the device time of the operator's kernels
    without host launch gaps.  With one operator enabled the inter-route
    kernels run their gated variants, which skip the other operators'
    arithmetic, and an evaluation without an inter-route operator (2-opt)
    launches no inter-route kernel; every figure still includes the
    evaluation's fixed launches (begin, intra-route kernel, finalize), which
    the 2-opt figure is close to.  Per step: evaluation and
    update times of the first steps of the descent through
    tga_eval_best_move / tga_apply_move."""
    import torch
    from paper_2506_17357_gb300 import tga as T
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2 = torch.cuda.Event(enable_timing=True)
    per_op = {}
    for op in range(8):
        if not (mask >> op) & 1:
            continue
        ls = T.LocalSearch(inst, sol, 1 << op, device=dev, stream=stream).build()
        ls.set_descent_mode(T.DESCENT_GRAPH)
        ls.set_tile(0, 0)
        T.tga_eval_best_move(ls.ctx, ls.move.data_ptr())
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(reps):
                T.tga_eval_best_move(ls.ctx, ls.move.data_ptr())
        # a replay is launched on the current stream: make it the context's
        # stream, so the events bracket it and the context outlives it
        with torch.cuda.stream(stream):
            g.replay()                                          # warm
            torch.cuda.synchronize()
            st0 = ls.stats()
            e0.record(stream)
            g.replay()
            e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        us = 1e3 * e0.elapsed_time(e1) / reps
        st = ls.stats()
        cands = (st["candidates"] - st0["candidates"]) / max(1, st["evaluations"] - st0["evaluations"])
        per_op[OP_NAMES[op]] = {"us_per_evaluation": us, "candidates": int(cands),
                                "candidates_per_s": cands / (us * 1e-6)}
        progress(f"breakdown: {OP_NAMES[op]} {us:.1f} us")
        del g
        torch.cuda.synchronize()
        ls.close()
    ls = T.LocalSearch(inst, sol, mask, device=dev, stream=stream).build()
    ls.set_descent_mode(T.DESCENT_GRAPH)
    ls.set_tile(0, 0)
    ev, up = [], []
    for _ in range(step_count):
        e0.record(stream)
        T.tga_eval_best_move(ls.ctx, ls.move.data_ptr())
        e1.record(stream)
        ls.apply_current_move()
        e2.record(stream)
        e2.synchronize()
        ev.append(1e3 * e0.elapsed_time(e1))
        up.append(1e3 * e1.elapsed_time(e2))
        mv = ls.move.cpu().numpy()
        if not mv[5] or mv[0] >= 0:
            break
    ls.close()
    return {"per_operator": per_op,
            "per_operator_path": f"{reps} evaluations of the operator alone captured in one CUDA graph "
                                 "(begin + gated inter (none for 2-opt) + intra + finalize kernels each), replayed",
            "per_step": {"steps": len(ev), "evaluation_us_median": float(np.median(ev)),
                         "update_us_median": float(np.median(up)),
                         "path": "per-step kernels launched one call at a time (eval: begin + inter + intra + "
                                 "finalize; update: apply of the caller-given move + write-back)"}}


def run_single(args, wl_name, steps, warmup, peak, e2e_reps=None, with_breakdown=True, cpu=None):
    """Time `steps` whole descents of one workload (after `warmup` untimed
    ones); returns the record (the JSON line's body for the headline)."""
    import torch
    import torch.distributed as dist
    from paper_2506_17357_gb300 import tga as T

    ws, rank, local = dist_env()
    dev = torch.device("cuda", local)
    desc, make, mask = workload(args, wl_name)
    seed = replica_seed(args.seed, rank)
    inst, sol = make(seed)
    progress(f"{wl_name}: instance ready")
    nbr = I.granular_neighbors(inst, args.granular) if args.granular else None
    stream = torch.cuda.Stream(dev)
    ls = T.LocalSearch(inst, sol, mask, device=dev, stream=stream, granular=nbr).build()
    if args.tile:                                              # pinned shape (profiler runs)
        tile = ls.set_tile(*[int(x) for x in args.tile.split(",")])
    else:
        tile = ls.set_tile(0, 0)                               # autotune on the initial state
    torch.cuda.synchronize()
    progress(f"{wl_name}: tuned {tile}, path {T.DESCENT_NAMES[T.tga_get_descent_mode(ls.ctx)[0]]}")
    tour0 = ls.tour.clone()
    rs0 = ls.route_start.clone()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    def restore():
        with torch.cuda.stream(stream):
            ls.tour.copy_(tour0)
            ls.route_start.copy_(rs0)

    def one_step():
        T.tga_build_attrs(ls.ctx)
        return T.tga_descend(ls.ctx)

    for _ in range(warmup):                                    # untimed
        restore()
        one_step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    times, cands, nsteps, stats = [], 0, [], None
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for _ in range(steps):
            flush.fill_(1)                                      # evict L2 between timed steps
            restore()
            torch.cuda.synchronize()
            e0.record(stream)
            stats = one_step()                                  # synchronises at its end
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            cands += stats["candidates"]
            nsteps.append(stats["steps"])
        torch.cuda.synchronize()
    clocks = clk.summary()
    progress(f"{wl_name}: {steps} timed descents done")
    total = float(sum(times))
    t_max, c_all = reduce_replicas(total, cands, dev)
    value = c_all / t_max
    tlo_ms = 1e3 * total / steps
    evals = stats["evaluations"]
    mode_used, grid = T.tga_get_descent_mode(ls.ctx)
    persistent = mode_used == T.DESCENT_PERSISTENT
    # gpu launches per descent: build (check, positions, perm, routes, finish,
    # pcol init) + begin, then one persistent launch, or 3 per evaluation
    # (inter, intra, apply), and the write-back of the solution
    launches_per_step = 6 + 1 + (1 if persistent else 3 * evals) + 1
    op_cands = T.tga_get_op_candidates(ls.ctx)
    pshape = T.tga_get_persistent_shape(ls.ctx)

    # ---- end to end through the public API with host buffers
    e2e_reps = steps if e2e_reps is None else max(1, min(e2e_reps, steps))
    e2e_warm = min(warmup, 1) if e2e_reps < steps else warmup
    e2e_times = []
    h2d = d2h = 0
    for k in range(e2e_warm + e2e_reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2d = ls.reload(inst, sol)                         # pinned H2D + build
        st = T.tga_descend(ls.ctx)
        tour, rs = ls.solution()                           # D2H of the result
        t1 = time.perf_counter()
        d2h = (tour.nbytes + rs.nbytes + 48)
        if k >= e2e_warm:
            e2e_times.append(t1 - t0)
        assert st["candidates"] == stats["candidates"]
    e2e_value = stats["candidates"] * len(e2e_times) / sum(e2e_times)
    progress(f"{wl_name}: end-to-end done")

    # ---- roofline of the dominant kernel, timed live with CUDA events on the
    # context's stream.  Persistent path: the one launch that runs the whole
    # descent (k_persist); its algorithmic work is every candidate evaluated,
    # per operator.  Graph path: the inter-route evaluation kernel at states
    # along the trajectory.
    peaks, peak_src = load_peaks()
    peak_ops = peak["ops_per_s"]
    peak_desc = (f"measured: {peak['kernel']}, {peak_ops / 1e12:.2f} T ops/s on {peak['sm_count']} SMs at "
                 f"{peak['clocks'].get('sm_mhz')} MHz (nominal issue rate {peak['nominal_issue_ops_per_s'] / 1e12:.2f} T)")
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))

    def hbm_ceiling(bytes_per_launch, ms):
        gbs = bytes_per_launch / (ms * 1e-3) / 1e9
        return {"algorithmic_bytes": int(bytes_per_launch), "achieved_gbs": gbs, "peak_gbs": hbm_peak,
                "frac": gbs / hbm_peak, "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})"}

    def kept_inter_ops():
        """Edge-based extraction: integer ops of the inter-route candidates the
        mask keeps in the current state (one evaluation's per-operator
        counts minus the closed-form intra-route counts)."""
        before = T.tga_get_op_candidates(ls.ctx)
        T.tga_eval_best_move(ls.ctx, ls.move.data_ptr())
        after = T.tga_get_op_candidates(ls.ctx)
        tour_h, rs_h = ls.solution()
        L = np.diff(rs_h).astype(np.int64)
        intra = [int((L * (L - 1)).sum()), int((L * (L - 1) // 2).sum()), int((L * (L - 1) // 2).sum()), 0,
                 int((np.maximum(L - 1, 0) * np.maximum(L - 2, 0)).sum()),
                 int((np.maximum(L - 2, 0) * np.maximum(L - 3, 0)).sum())]
        table = ops_table(inst)
        return sum(table[op] * (after[op] - before[op] - (intra[op] if (mask >> op) & 1 else 0))
                   for op in range(6))     # the edge-based extraction has no ranks 6, 7

    def inter_kernel_roof():
        restore()
        T.tga_build_attrs(ls.ctx)
        total_ops = total_ms = 0.0
        x_ops = x_ms = 0.0                      # swaps of runs (ranks 6, 7)
        xs = bool(mask & 0xC0)
        probes = 5
        n_steps = nsteps[-1]
        for j in range(probes):
            ms = T.tga_profile_inter(ls.ctx, reps=20)
            if args.granular:
                total_ops += kept_inter_ops()
            else:
                tour_h, rs_h = ls.solution()
                lens = np.diff(rs_h)
                total_ops += algorithmic_ops(inst.n, lens, mask, ops_table(inst))
                if xs:
                    x_ms += T.tga_profile_xswap(ls.ctx, reps=20)
                    x_ops += algorithmic_ops(inst.n, lens, mask, ops_table(inst), ops=(6, 7))
            total_ms += ms
            if j + 1 < probes:
                T.tga_descend(ls.ctx, max_steps=max(1, n_steps // (probes - 1)))
        achieved = total_ops / (total_ms / 1e3)
        kname = "k_eval_edges" if args.granular else ("k_eval_strip" if tile[2] == 0 else "k_eval_inter")
        ms_l = total_ms / probes
        out = {"bound": "alu", "kernel": kname, "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
               "unit": "Tops/s (INT32 lane-ops)", "frac": achieved / peak_ops, "peak_source": peak_desc,
               "frac_of_nominal_issue": achieved / peak["nominal_issue_ops_per_s"],
               "ms_per_launch": ms_l, "ops_per_launch": total_ops / probes,
               "work": "inter-route candidates of the state (per-candidate integer ops x candidates), "
                       "mean over 5 states along the trajectory",
               "hbm": hbm_ceiling(evaluation_bytes(inst.n, ls.m), ms_l),
               "traffic": measured_traffic(workload_name(args, wl_name) +
                                           (f"-granular{args.granular}" if args.granular else ""), kname),
               "kernel_source_hash": kernel_source_hash()}
        if xs:
            xa = x_ops / (x_ms / 1e3)
            out["xswap_kernel"] = {"kernel": "k_eval_xswap", "achieved": xa / 1e12, "frac": xa / peak_ops,
                                   "ms_per_launch": x_ms / probes, "ops_per_launch": x_ops / probes,
                                   "traffic": measured_traffic(workload_name(args, wl_name), "k_eval_xswap")}
        return out

    inter_roof = inter_kernel_roof()
    progress(f"{wl_name}: inter-route kernel timed")
    if persistent:
        kms = []
        for _ in range(3):
            restore()
            T.tga_build_attrs(ls.ctx)
            torch.cuda.synchronize()
            e0.record(stream)
            T.tga_descend_async(ls.ctx)
            e1.record(stream)
            e1.synchronize()
            kms.append(e0.elapsed_time(e1))
        ops = descent_ops(op_cands, ops_table(inst))
        ms = float(np.mean(kms))
        achieved = ops / (ms / 1e3)
        roof = {"bound": "alu", "kernel": "k_persist", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                "unit": "Tops/s (INT32 lane-ops)", "frac": achieved / peak_ops, "peak_source": peak_desc,
                "frac_of_nominal_issue": achieved / peak["nominal_issue_ops_per_s"],
                "ms_per_launch": ms, "ops_per_launch": ops, "grid": grid,
                "work": "every candidate of every evaluation of the descent (per-operator device counters "
                        "x per-candidate integer ops); one launch = one whole descent",
                "hbm": hbm_ceiling(evaluation_bytes(inst.n, ls.m) * evals, ms),
                "traffic": measured_traffic(workload_name(args, wl_name), "k_persist"),
                "kernel_source_hash": kernel_source_hash(),
                "inter_kernel": {k: inter_roof[k] for k in ("kernel", "achieved", "frac", "ms_per_launch",
                                                             "ops_per_launch", "traffic", "hbm")}}
    else:
        roof = inter_roof
    m_routes = ls.m
    ls.close()
    del flush
    progress(f"{wl_name}: roofline done")
    brk = breakdown(inst, sol, mask, dev, stream) if (with_breakdown and rank == 0 and not args.granular) else None
    progress(f"{wl_name}: breakdown done")
    rec = {
        "metric": "move evals/s", "value": value, "unit": "candidate moves/s",
        "n_gpus": ws, "steps": steps, "warmup": warmup,
        "ms_per_step": 1e3 * t_max / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "time_to_local_optimum_ms": tlo_ms, "moves_applied": nsteps[-1], "evaluations": evals,
        "candidates_per_descent": stats["candidates"], "initial_cost": stats["initial_cost"],
        "final_cost": stats["final_cost"],
        "config": {"workload": workload_name(args, wl_name), "desc": desc, "instance_seed": seed,
                   "n_customers": int(inst.n), "n_routes": int(m_routes),
                   "op_mask": mask, "tile_rows_warps": list(tile), "parallelism": f"replicas x{ws}",
                   "descent_path": T.DESCENT_NAMES[mode_used],
                   "extraction": (f"edge-based, granular mask of the {args.granular} nearest customers"
                                  if args.granular else "node-based, full neighbourhood"),
                   "persistent_tile": list(pshape) if persistent else None,
                   "l2": "flushed between timed steps (512 MB write)"},
        "candidates_per_operator": op_cands,
        "e2e": {"value": e2e_value, "unit": "candidate moves/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "time_to_local_optimum_ms": 1e3 * float(np.mean(e2e_times)),
                "repeats": len(e2e_times),
                "note": None if len(e2e_times) == steps else
                f"{len(e2e_times)} timed end-to-end descents after {e2e_warm} untimed (each is a whole descent)"},
        "gpu_launches": int(launches_per_step * steps),
        "clocks": clocks,
        "roofline": roof,
        "breakdown": brk,
    }
    if cpu is not None and rank == 0 and ws == 1:
        rec["cpu_baseline"] = cpu_baseline(args, wl_name, **cpu)
        progress(f"{wl_name}: CPU baseline done")
    return rec


# ---------------------------------------------------------------------------
# batched and served workloads

def run_batch(args, steps, warmup):
    """Batched workload: 256 instances (sizes uniform in [100, 2000], half
    CVRP / half VRPTW) descended in one persistent launch, against 256
    sequential single-instance descents of the same jobs on the same GPU."""
    import torch
    from paper_2506_17357_gb300 import tga as T
    dev = torch.device("cuda", 0)
    count = args.batch_jobs
    jobs = I.batch_jobs(count=count, seed=4, lo=100, hi=2000)
    stream = torch.cuda.Stream(dev)
    lss = [T.LocalSearch(inst, sol, I.mask_for(inst), device=dev, stream=stream) for inst, sol in jobs]
    ctxs = [ls.ctx for ls in lss]
    progress("batch256: jobs ready")
    rows = T.tga_batch_autotune(ctxs)
    progress("batch256: tuned")
    init = [(ls.tour.clone(), ls.route_start.clone()) for ls in lss]
    torch.cuda.synchronize()

    def restore():
        with torch.cuda.stream(stream):
            for ls, (t0, r0) in zip(lss, init):
                ls.tour.copy_(t0)
                ls.route_start.copy_(r0)

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(warmup):
        restore()
        T.tga_descend_batch(ctxs)
    times, stats = [], None
    with ClockSampler(0) as clk:
        for _ in range(steps):
            restore()
            torch.cuda.synchronize()
            e0.record(stream)
            stats = T.tga_descend_batch(ctxs)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
    clocks = clk.summary()
    progress("batch256: timed")
    t_batch = float(np.mean(times))
    cands = sum(s["candidates"] for s in stats)
    # sequential single-instance descents of the same jobs
    restore()
    torch.cuda.synchronize()
    e0.record(stream)
    seq_stats = []
    for ls in lss:
        T.tga_build_attrs(ls.ctx)
        seq_stats.append(T.tga_descend(ls.ctx))
    e1.record(stream)
    e1.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3
    exact = all(a["final_cost"] == b["final_cost"] and a["steps"] == b["steps"] and
                a["candidates"] == b["candidates"] for a, b in zip(stats, seq_stats))
    # end to end: host instances/solutions -> batch -> host results
    t0 = time.perf_counter()
    h2d = 0
    for ls, (inst, sol) in zip(lss, jobs):
        h2d += ls.reload(inst, sol)
    T.tga_descend_batch(ctxs)
    d2h = 0
    for ls in lss:
        tour, rs = ls.solution()
        d2h += tour.nbytes + rs.nbytes + 48
    t_e2e = time.perf_counter() - t0
    sizes = [inst.n for inst, _ in jobs]
    for ls in lss:
        ls.close()
    return {"metric": "batched jobs/s", "value": count / t_batch, "unit": "jobs/s", "n_gpus": 1,
            "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * t_batch, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "sequential_jobs_per_s": count / t_seq, "speedup_vs_sequential": t_seq / t_batch,
            "move_evals_per_s": cands / t_batch, "bit_exact_vs_sequential": bool(exact),
            "config": {"workload": "batch256", "jobs": count, "sizes": [min(sizes), max(sizes)],
                       "mix": "alternating CVRP/VRPTW", "tile_rows_by_job": sorted(set(rows)),
                       "descent": "one persistent launch; the step loop runs on the device (no graph needed)",
                       "l2": "inputs (1.4 GB of matrices) exceed L2"},
            "e2e": {"value": count / t_e2e, "unit": "jobs/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "clocks": clocks}


def run_serve(args, warmup):
    """Serving workload: a seeded Poisson stream of jobs (sizes log-uniform in
    [100, 5000], 70% CVRP / 30% VRPTW) through the continuous-batching server
    (memory budget 1 GiB, up to 32 slots) against the one-at-a-time path on the
    same arrivals.  The arrival rate is set from the measured one-at-a-time
    capacity mu1: 0.8 mu1 (both keep up; latency differs) and 2 mu1 (the
    one-at-a-time queue grows)."""
    import torch
    from paper_2506_17357_gb300 import serving as S
    count = args.serve_jobs
    sizes, kinds = I.serving_sizes(count, seed=5)
    reqs = []
    for j in range(count):
        inst, sol = I.serving_job(j, int(sizes[j]), bool(kinds[j]), seed=5)
        reqs.append(S.Request(j, 0.0, inst, sol, I.mask_for(inst)))
    pinned = {r.rid: S._Pinned(torch, r) for r in reqs}
    budget = 1 << 30

    def run(slots, arrivals):
        rs = [S.Request(r.rid, float(a), r.inst, r.sol, r.op_mask) for r, a in zip(reqs, arrivals)]
        srv = S.Server(budget_bytes=budget, max_slots=slots, keep_solutions=False)
        return S.summarize(srv.serve(rs, pinned=pinned)), srv

    for _ in range(max(1, warmup)):
        S.Server(budget_bytes=budget, max_slots=4, keep_solutions=False).serve(
            [S.Request(r.rid, 0.0, r.inst, r.sol, r.op_mask) for r in reqs[:6]], pinned=pinned)
    zero = np.zeros(count)
    progress("serve: jobs ready")
    cap1, _ = run(1, zero)
    progress("serve: one-at-a-time capacity done")
    capN, _ = run(32, zero)
    progress("serve: continuous capacity done")
    mu1 = cap1["jobs_per_s"]
    sweep = {}
    with ClockSampler(0) as clk:
        for mult in (0.8, 2.0):
            arr = I.poisson_arrivals(count, mult * mu1, seed=5)
            one, _ = run(1, arr)
            cont, _ = run(32, arr)
            sweep[str(mult)] = {"rate_jobs_per_s": mult * mu1, "one_at_a_time": one, "continuous": cont}
            progress(f"serve: {mult}x rate done")
    clocks = clk.summary()
    head = sweep["2.0"]["continuous"]
    return {"metric": "served jobs/s", "value": head["jobs_per_s"], "unit": "jobs/s", "n_gpus": 1,
            "steps": 1, "warmup": warmup, "ms_per_step": 1e3 * head["makespan_s"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "p50_latency_ms": head["p50_latency_ms"], "p99_latency_ms": head["p99_latency_ms"],
            "one_at_a_time_at_2x": sweep["2.0"]["one_at_a_time"],
            "saturated_capacity_jobs_per_s": {"one_at_a_time": mu1, "continuous": capN["jobs_per_s"]},
            "sweep": sweep,
            "config": {"workload": "serve", "jobs": count, "sizes": "log-uniform [100, 5000]",
                       "mix": "70% CVRP / 30% VRPTW", "budget_bytes": budget, "max_slots": 32,
                       "arrivals": "seeded Poisson at 0.8x and 2x the one-at-a-time capacity"},
            "clocks": clocks}


# ---------------------------------------------------------------------------
# entry points

def _init_gpu():
    import torch
    import torch.distributed as dist
    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    return ws, rank, local


def bench_default(args):
    """Headline (clustered CVRP-10000) + the other workloads in one line."""
    import torch.distributed as dist
    ws, rank, local = _init_gpu()
    peak = measure_int_peak(local)
    line = run_single(args, HEADLINE, args.steps, args.warmup, peak, e2e_reps=args.e2e_reps,
                      cpu=None if args.no_cpu_baseline else dict(seconds=args.cpu_seconds))
    line["int32_peak"] = peak
    line["host"] = {"cpu_count": os.cpu_count(), "affinity_cores": host_cores(), "sm_count": peak["sm_count"]}
    if ws == 1 and not args.headline_only:
        cpu_small = None if args.no_cpu_baseline else dict(seconds=4.0, all_core_target_s=3.0, per_op_seconds=0.3)
        configs = {}
        for wl in ("cvrp100", "vrptw1000"):
            configs[wl] = run_single(args, wl, args.steps, args.warmup, peak, with_breakdown=(wl == "vrptw1000"),
                                     cpu=cpu_small)
        configs["batch256"] = run_batch(args, steps=min(args.steps, 3), warmup=1)
        configs["serve"] = run_serve(args, warmup=1)
        line["configs"] = configs
    if ws > 1:
        dist.barrier()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def bench_one(args):
    """One workload alone (--workload NAME): the profiling commands' form."""
    import torch.distributed as dist
    ws, rank, local = _init_gpu()
    if args.workload == "batch256":
        line = run_batch(args, args.steps, args.warmup)
    elif args.workload == "serve":
        line = run_serve(args, args.warmup)
    else:
        peak = measure_int_peak(local)
        line = run_single(args, args.workload, args.steps, args.warmup, peak, e2e_reps=args.e2e_reps,
                          cpu=None if args.no_cpu_baseline else dict(seconds=args.cpu_seconds))
        line["int32_peak"] = peak
    if ws > 1:
        dist.barrier()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def bench_reference(args):
    """The reference arm: the CPU oracle (there is no published code) on the
    host cores, on the headline workload.  Each step is one whole
    neighbourhood evaluation of the initial solution spread over a spawn
    pool of one process per core (interleaved slices, exact minimum key);
    warm-up steps evaluate one slice per process."""
    import multiprocessing as mp
    import oracle as O
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    wl = HEADLINE if args.workload == "all" else args.workload
    desc, make, mask = workload(args, wl)
    inst, sol = make(args.seed)
    K = host_cores()
    est = O.count_candidates(inst, sol, mask) / 1e7
    stride = max(K, K * int(math.ceil(est / (0.5 * K))))
    states = [(np.asarray(sol.tour, np.int32), np.asarray(sol.route_start, np.int32))]
    full = [[(0, ph, stride)] for ph in range(stride)]
    ctx = mp.get_context("spawn")
    vals, walls, key = [], [], None
    with ctx.Pool(K, initializer=_cpu_worker_init, initargs=(wl, args.seed, mask, states, 0)) as pool:
        pool.map(time.sleep, [0.05] * K)
        for k in range(args.warmup + args.steps):
            tasks = full[:K] if k < args.warmup else full
            res = pool.map(_cpu_worker_task, tasks, chunksize=1)
            wall = max(r[3] for r in res) - min(r[2] for r in res)
            if k >= args.warmup:
                vals.append(sum(r[1] for r in res) / wall)
                walls.append(wall)
                key = min(r[0] for r in res)
    value = float(sum(vals) / len(vals))
    dkey, didx = O.unpack_key(key)
    line = {"impl": "reference", "metric": "move evals/s", "value": value, "unit": "candidate moves/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(walls)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": workload_name(args, wl), "desc": desc,
                                            "instance_seed": args.seed, "op_mask": mask},
            "first_best_move": {"delta": dkey, "move_index": didx},
            "cpu_baseline": {"value": value, "unit": "candidate moves/s", "cores": K, "kind": "oracle",
                             "host_cores": host_cores(), "os_cpu_count": os.cpu_count(),
                             "sample": f"each step: one whole evaluation of the initial solution of "
                                       f"{workload_name(args, wl)} seed {args.seed} in {stride} interleaved slices "
                                       f"over a spawn pool of {K} processes (concatenation evaluator)"},
            "e2e": {"value": value, "unit": "candidate moves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tga", choices=["tga", "reference"])
    ap.add_argument("--workload", default="all", choices=["all"] + sorted(WORKLOADS) + ["batch256", "serve"],
                    help="all (default): the clustered CVRP-10000 headline plus every other workload in one line")
    ap.add_argument("--headline-only", action="store_true", help="with --workload all: skip the other workloads")
    ap.add_argument("--e2e-reps", type=int, default=3,
                    help="timed end-to-end descents of the headline (each a whole descent through the API)")
    ap.add_argument("--serve-jobs", type=int, default=120)
    ap.add_argument("--only-descent", action="store_true",
                    help="run one descent of the workload without timing (for profiler launch lists)")
    ap.add_argument("--descent-steps", type=int, default=0,
                    help="with --only-descent: stop after this many moves (0: run to the local optimum)")
    ap.add_argument("--tile", default="",
                    help="inter tile shape rows,warps,row_split (default: autotune on the initial state)")
    ap.add_argument("--persistent-shape", default="",
                    help="with --only-descent: run the persistent path under this shape rows,warps,row_split "
                         "(row_split 0: strip mode)")
    ap.add_argument("--extended-swaps", action="store_true",
                    help="add op ranks 6, 7 (a customer with a run of two, two runs of two) to the workload")
    ap.add_argument("--granular", type=int, default=0,
                    help="edge-based extraction with the THETA nearest customers per customer (0: full neighbourhood)")
    ap.add_argument("--batch-jobs", type=int, default=256)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.only_descent:
        only_descent(args)
    elif args.impl == "reference":
        bench_reference(args)
    elif args.workload == "all":
        bench_default(args)
    else:
        bench_one(args)


if __name__ == "__main__":
    main()
