"""Seeded synthetic VRP instances and initial solutions.

This module only produces *inputs*: customer coordinates, demands, service
times, time windows, the integer distance matrix and a random initial
solution.  It contains none of the local-search arithmetic (no route costs,
no segment concatenation, no move evaluation), so both the CUDA path and the
CPU oracle can consume its output without sharing any method code.

Problem statement followed: Section 2 of the paper (complete graph, depot 0,
customers 1..N, demands d_i, time windows [e_i, l_i], service times s_i,
distance matrix C; for the CVRP the time attributes are absent).  The
travel-time matrix T is taken equal to C.

Randomness: a counter-based splitmix64 generator (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014).  Every draw is
integer arithmetic or exactly rounded IEEE float64 add/mul, so x86 and Arm
hosts produce identical instances.

Workload recipes (sizes and distributions of the five benchmark workloads):

* ``cvrp_uniform(n)``: 1 depot + n customers, integer coordinates uniform in
  [0,1000]^2, demands uniform in [1,100], capacity ceil(sum d / 8).
* ``vrptw(n)``: coordinates uniform in [0,1000]^2, demands uniform in [1,50],
  capacity 200, service time 10 (depot 0), depot window [0,10000]; window
  centre uniform in [c(0,i), 10000 - c(i,0) - 10], width uniform in
  [60,400]; e = centre - floor(w/2), l = e + w, both clipped to [0,10000].
* ``vrpspdtw(n)``: the ``vrptw(n)`` recipe (same coordinates, deliveries,
  windows and service times for a given seed) plus pickup quantities
  uniform in [1,50] from their own stream (depot 0) -- the simultaneous
  pickup and delivery variant of Section 2.
* ``cvrp_clustered(n)``: depot uniform in [0,1000]^2; 50 cluster centres
  uniform in [0,1000]^2; each customer picks a centre uniformly and adds a
  zero-mean normal offset with sigma 40 per axis (Irwin-Hall sum of twelve
  uniforms), clipped to [0,1000] and rounded half away from zero; demands
  uniform in [1,100]; capacity 400.
* Distances: c_ij = round(sqrt(dx^2 + dy^2)) computed with an exact integer
  square root (round to nearest; ties cannot occur for integer dx^2+dy^2).
* Initial solution: a seeded Fisher-Yates permutation of the customers, split
  greedily into routes: a new route opens when the next customer's demand
  (or, with pickups, its delivery or its pickup) would take the route's
  total delivery (or total pickup) above the capacity.  Route count M is
  fixed from then on.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1

# Stream identifiers: each random quantity has its own counter stream, so a
# change to one recipe never shifts the draws of another.
S_COORD, S_DEMAND, S_TW_CENTRE, S_TW_WIDTH = 1, 2, 3, 4
S_CLUSTER_CENTRE, S_CLUSTER_PICK, S_GAUSS, S_PERM = 5, 6, 7, 8
S_BATCH_SIZE, S_BATCH_KIND, S_ARRIVAL = 9, 10, 11
S_PICKUP = 12

HORIZON = 10000
COORD_MAX = 1000


def splitmix64(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` outputs of splitmix64 for (seed, stream), counter-based.

    State for draw i is ``base + (i + 1) * golden`` with
    ``base = mix(seed) ^ (stream * golden)``; the output is the standard
    splitmix64 finaliser of that state.
    """
    base = (_mix_int(seed & _MASK64) ^ ((stream * 0x9E3779B97F4A7C15) & _MASK64)) & _MASK64
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(base) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _mix_int(x: int) -> int:
    x = (x + 0x9E3779B97F4A7C15) & _MASK64
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & _MASK64
    return x ^ (x >> 31)


def uniform_int(z: np.ndarray, lo, hi) -> np.ndarray:
    """Map 64-bit draws to integers in [lo, hi] (inclusive) by the
    multiply-shift rule ``lo + ((z >> 32) * (hi - lo + 1)) >> 32``.
    ``lo``/``hi`` may be arrays (per-draw bounds)."""
    lo = np.asarray(lo, dtype=np.int64)
    hi = np.asarray(hi, dtype=np.int64)
    span = (hi - lo + 1).astype(np.uint64)
    with np.errstate(over="ignore"):
        v = ((z >> np.uint64(32)) * span) >> np.uint64(32)
    return lo + v.astype(np.int64)


def uniform01(z: np.ndarray) -> np.ndarray:
    """53-bit uniform doubles in [0, 1) (exact: (z >> 11) * 2^-53)."""
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def round_sqrt(s: np.ndarray) -> np.ndarray:
    """Nearest integer to sqrt(s) for non-negative int64 s (s < 2^52).

    r = isqrt(s) exactly (float64 sqrt followed by integer correction), then
    c = r + (s - r^2 > r), i.e. round half up; no half can occur because
    sqrt(s) = r + 1/2 would need s = r^2 + r + 1/4."""
    s = np.asarray(s, dtype=np.int64)
    r = np.floor(np.sqrt(s.astype(np.float64))).astype(np.int64)
    r -= (r * r > s)
    r += ((r + 1) * (r + 1) <= s)
    return r + (s - r * r > r)


def rounded_euclidean(xy: np.ndarray) -> np.ndarray:
    """int32 matrix c_ij = nearest integer to the Euclidean distance."""
    xy = np.asarray(xy, dtype=np.int64)
    n1 = xy.shape[0]
    out = np.empty((n1, n1), dtype=np.int32)
    rows = max(1, (1 << 22) // max(n1, 1))
    for r0 in range(0, n1, rows):
        r1 = min(n1, r0 + rows)
        dx = xy[r0:r1, None, 0] - xy[None, :, 0]
        dy = xy[r0:r1, None, 1] - xy[None, :, 1]
        out[r0:r1] = round_sqrt(dx * dx + dy * dy).astype(np.int32)
    return out


def instance_from_arrays(name, dist, demand, capacity, service=None, tw_early=None,
                         tw_late=None, coords=None, w_load=100, w_tw=100, pickup=None) -> "Instance":
    """Wrap explicit arrays (e.g. a hand-made example) as an Instance."""
    dist = np.ascontiguousarray(dist, dtype=np.int32)
    n1 = dist.shape[0]
    has_tw = tw_early is not None
    svc = np.zeros(n1, np.int32) if service is None else np.asarray(service, np.int32)
    e = np.zeros(n1, np.int32) if tw_early is None else np.asarray(tw_early, np.int32)
    l = np.full(n1, HORIZON, np.int32) if tw_late is None else np.asarray(tw_late, np.int32)
    xy = np.zeros((n1, 2), np.int32) if coords is None else np.asarray(coords, np.int32)
    pk = None if pickup is None else np.asarray(pickup, np.int32)
    return Instance(name, n1 - 1, int(capacity), has_tw, xy, np.asarray(demand, np.int32),
                    svc, e, l, dist, w_load, w_tw, pk)


@dataclasses.dataclass
class Instance:
    """A VRP instance (host arrays, int32).  Index 0 is the depot."""
    name: str
    n: int
    capacity: int
    has_tw: bool
    coords: np.ndarray          # (n+1, 2)
    demand: np.ndarray          # (n+1,), demand[0] = 0
    service: np.ndarray         # (n+1,), zeros for CVRP
    tw_early: np.ndarray        # (n+1,)
    tw_late: np.ndarray         # (n+1,)
    dist: np.ndarray            # (n+1, n+1) row-major
    w_load: int = 100
    w_tw: int = 100
    pickup: Optional[np.ndarray] = None   # (n+1,), pickup[0] = 0; None: no pickups

    @property
    def has_pd(self) -> bool:
        return self.pickup is not None

    @property
    def kind(self) -> str:
        if self.pickup is not None:
            return "vrpspdtw" if self.has_tw else "vrpspd"
        return "vrptw" if self.has_tw else "cvrp"


@dataclasses.dataclass
class Solution:
    """Giant tour (customers in route order) plus route boundaries.

    Route r visits tour[route_start[r]:route_start[r+1]] between two depot
    visits; route_start has M+1 entries with route_start[0] = 0 and
    route_start[M] = n.  Empty routes are allowed."""
    tour: np.ndarray            # (n,) int32
    route_start: np.ndarray     # (M+1,) int32

    @property
    def n_routes(self) -> int:
        return int(self.route_start.shape[0] - 1)

    def routes(self):
        rs = self.route_start
        return [self.tour[rs[r]:rs[r + 1]].tolist() for r in range(len(rs) - 1)]

    def copy(self) -> "Solution":
        return Solution(self.tour.copy(), self.route_start.copy())


def _no_tw(n1: int):
    z = np.zeros(n1, dtype=np.int32)
    late = np.full(n1, HORIZON, dtype=np.int32)
    return z.copy(), z.copy(), late


def cvrp_uniform(n: int, seed: int) -> Instance:
    xy = uniform_int(splitmix64(seed, S_COORD, 2 * (n + 1)), 0, COORD_MAX).reshape(n + 1, 2)
    dem = np.zeros(n + 1, dtype=np.int64)
    dem[1:] = uniform_int(splitmix64(seed, S_DEMAND, n), 1, 100)
    cap = -(-int(dem.sum()) // 8)
    svc, early, late = _no_tw(n + 1)
    return Instance(f"cvrp_uniform_n{n}_s{seed}", n, cap, False, xy.astype(np.int32),
                    dem.astype(np.int32), svc, early, late, rounded_euclidean(xy))


def vrptw(n: int, seed: int) -> Instance:
    xy = uniform_int(splitmix64(seed, S_COORD, 2 * (n + 1)), 0, COORD_MAX).reshape(n + 1, 2)
    dist = rounded_euclidean(xy)
    dem = np.zeros(n + 1, dtype=np.int64)
    dem[1:] = uniform_int(splitmix64(seed, S_DEMAND, n), 1, 50)
    svc = np.full(n + 1, 10, dtype=np.int32)
    svc[0] = 0
    d0 = dist[0, 1:].astype(np.int64)
    centre = uniform_int(splitmix64(seed, S_TW_CENTRE, n), d0, HORIZON - d0 - 10)
    width = uniform_int(splitmix64(seed, S_TW_WIDTH, n), 60, 400)
    e = centre - width // 2
    l = e + width
    early = np.zeros(n + 1, dtype=np.int32)
    late = np.full(n + 1, HORIZON, dtype=np.int32)
    early[1:] = np.clip(e, 0, HORIZON)
    late[1:] = np.clip(l, 0, HORIZON)
    return Instance(f"vrptw_n{n}_s{seed}", n, 200, True, xy.astype(np.int32),
                    dem.astype(np.int32), svc, early, late, dist)


def vrpspdtw(n: int, seed: int) -> Instance:
    """VRPTW recipe plus pickups uniform in [1,50] (stream S_PICKUP)."""
    base = vrptw(n, seed)
    pk = np.zeros(n + 1, dtype=np.int64)
    pk[1:] = uniform_int(splitmix64(seed, S_PICKUP, n), 1, 50)
    base.name = f"vrpspdtw_n{n}_s{seed}"
    base.pickup = pk.astype(np.int32)
    return base


def _round_half_away(x: np.ndarray) -> np.ndarray:
    return (np.sign(x) * np.floor(np.abs(x) + 0.5)).astype(np.int64)


def cvrp_clustered(n: int, seed: int, n_clusters: int = 50, sigma: float = 40.0) -> Instance:
    depot = uniform_int(splitmix64(seed, S_COORD, 2), 0, COORD_MAX)
    centres = uniform_int(splitmix64(seed, S_CLUSTER_CENTRE, 2 * n_clusters), 0,
                          COORD_MAX).reshape(n_clusters, 2)
    pick = uniform_int(splitmix64(seed, S_CLUSTER_PICK, n), 0, n_clusters - 1)
    u = uniform01(splitmix64(seed, S_GAUSS, 24 * n)).reshape(n, 2, 12)
    g = u[:, :, 0].copy()
    for k in range(1, 12):            # fixed left-to-right summation order
        g = g + u[:, :, k]
    g = g - 6.0
    pos = centres[pick].astype(np.float64) + sigma * g
    pos = np.clip(pos, 0.0, float(COORD_MAX))
    xy = np.empty((n + 1, 2), dtype=np.int64)
    xy[0] = depot
    xy[1:] = _round_half_away(pos)
    dem = np.zeros(n + 1, dtype=np.int64)
    dem[1:] = uniform_int(splitmix64(seed, S_DEMAND, n), 1, 100)
    svc, early, late = _no_tw(n + 1)
    return Instance(f"cvrp_clustered_n{n}_s{seed}", n, 400, False, xy.astype(np.int32),
                    dem.astype(np.int32), svc, early, late, rounded_euclidean(xy))


def random_split_solution(inst: Instance, seed: int) -> Solution:
    """Seeded Fisher-Yates permutation of 1..n split greedily by capacity."""
    n = inst.n
    perm = list(range(1, n + 1))
    if n > 1:
        bounds = np.arange(n - 1, 0, -1, dtype=np.int64)          # i = n-1 .. 1
        js = uniform_int(splitmix64(seed, S_PERM, n - 1), 0, bounds).tolist()
        for i, j in zip(bounds.tolist(), js):
            perm[i], perm[j] = perm[j], perm[i]
    starts = [0]
    load = pick = 0
    pk = getattr(inst, "pickup", None)
    for t, c in enumerate(perm):
        d = int(inst.demand[c])
        p = 0 if pk is None else int(pk[c])
        if t > 0 and (load + d > inst.capacity or pick + p > inst.capacity):
            starts.append(t)
            load = pick = 0
        load += d
        pick += p
    starts.append(n)
    if n == 0:
        starts = [0, 0]
    return Solution(np.asarray(perm, dtype=np.int32), np.asarray(starts, dtype=np.int32))


def granular_neighbors(inst: Instance, theta: int) -> np.ndarray:
    """Granular mask of the edge-based extraction (Section 5.3.1; neighbour
    lists in the manner of Vidal et al. 2013): row x (customers 1..n) holds
    the theta customers y != x with the smallest (c(x, y), y); row 0 is unused
    (zeros).  An input, like the distance matrix: both evaluators read it."""
    n = int(inst.n)
    if not 1 <= theta <= n - 1:
        raise ValueError(f"theta must be in [1, n-1], got {theta}")
    d = np.asarray(inst.dist, dtype=np.int64)
    out = np.zeros((n + 1, theta), dtype=np.int32)
    ids = np.arange(1, n + 1, dtype=np.int64)
    for x in range(1, n + 1):
        key = d[x, 1:] * (n + 2) + ids            # distance first, then the smaller id
        key[x - 1] = np.iinfo(np.int64).max       # not its own neighbour
        out[x] = ids[np.argsort(key, kind="stable")[:theta]]
    return out


def solution_seed(instance_seed: int) -> int:
    return instance_seed + 1_000_000


# ---------------------------------------------------------------------------
# The five benchmark workloads.

def config1(seed: int = 1):
    """CVRP, 100 customers, uniform; relocate, swap, 2-opt, 2-opt*."""
    inst = cvrp_uniform(100, seed)
    return inst, random_split_solution(inst, solution_seed(seed))


def config2(seed: int = 1):
    """VRPTW, 1000 customers; all five operators."""
    inst = vrptw(1000, seed)
    return inst, random_split_solution(inst, solution_seed(seed))


def config_spd(seed: int = 1, n: int = 1000):
    """VRPSPDTW, 1000 customers (the VRPTW workload with pickups); all five
    operators."""
    inst = vrpspdtw(n, seed)
    return inst, random_split_solution(inst, solution_seed(seed))


def config3(seed: int = 1):
    """Large clustered CVRP, 10000 customers; relocate, swap, 2-opt*, or-opt."""
    inst = cvrp_clustered(10000, seed)
    return inst, random_split_solution(inst, solution_seed(seed))


# Operator ranks (move-index op field) and the per-workload operator masks.
OP_RELOCATE, OP_SWAP, OP_2OPT, OP_2OPT_STAR, OP_OROPT2, OP_OROPT3 = range(6)
# swaps with unequal or longer runs (Section 5.3.1 Swap with N1, N2 > 0): a
# customer with a run of two (rank 6), two runs of two (rank 7)
OP_SWAP12, OP_SWAP22 = 6, 7
MASK_ALL = 0x3F
MASK_EXT = 0xFF          # every rank, with the swaps of runs
MASK_CONFIG1 = (1 << OP_RELOCATE) | (1 << OP_SWAP) | (1 << OP_2OPT) | (1 << OP_2OPT_STAR)
MASK_CONFIG2 = MASK_ALL
MASK_CONFIG3 = MASK_ALL & ~(1 << OP_2OPT)
MASK_CVRP_MIXED = MASK_CONFIG1 | (1 << OP_OROPT2) | (1 << OP_OROPT3)


def mask_for(inst: Instance) -> int:
    """Operator mask for mixed (batched/served) jobs: CVRP gets relocate,
    swap, 2-opt, 2-opt* and or-opt; VRPTW gets all five operators (both
    cover all six move ranks)."""
    return MASK_CVRP_MIXED if not inst.has_tw else MASK_ALL


def batch_jobs(count: int = 256, seed: int = 4, lo: int = 100, hi: int = 2000):
    """Batched workload: ``count`` instances, sizes uniform in [lo, hi],
    alternating CVRP (uniform generator) / VRPTW, one random split each.
    Instance seeds are seed*100000 + j."""
    sizes = uniform_int(splitmix64(seed, S_BATCH_SIZE, count), lo, hi)
    jobs = []
    for j in range(count):
        s = seed * 100000 + j
        n = int(sizes[j])
        inst = cvrp_uniform(n, s) if j % 2 == 0 else vrptw(n, s)
        jobs.append((inst, random_split_solution(inst, solution_seed(s))))
    return jobs


def serving_sizes(count: int, seed: int = 5, lo: int = 100, hi: int = 5000):
    """Log-uniform sizes floor(exp(U[ln lo, ln hi])) and a 70/30 CVRP/VRPTW
    split (True = VRPTW)."""
    u = uniform01(splitmix64(seed, S_BATCH_SIZE, count))
    sizes = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    sizes = np.clip(sizes, lo, hi)
    kind = uniform01(splitmix64(seed, S_BATCH_KIND, count)) >= 0.7
    return sizes, kind


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 5) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: cumulative exponential gaps
    -ln(1-U)/rate.  Uses libm log, so times may differ in the last bit
    across hosts; they only schedule requests, never enter the arithmetic."""
    u = uniform01(splitmix64(seed, S_ARRIVAL, count))
    return np.cumsum(-np.log1p(-u) / rate_per_s)


def serving_job(j: int, size: int, is_tw: bool, seed: int = 5):
    s = seed * 100000 + j
    inst = vrptw(int(size), s) if is_tw else cvrp_uniform(int(size), s)
    return inst, random_split_solution(inst, solution_seed(s))
