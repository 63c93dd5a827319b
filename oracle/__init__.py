"""CPU oracle for best-improvement VRP local search -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU product path
(``paper_2506_17357_gb300``) never imports it, and the two share no code.

The arithmetic lives in ``tga_oracle.c`` (plain single-threaded C); this
module only compiles it (gcc) and marshals numpy arrays through ctypes.

Functions and the passages they follow:

* ``route_cost`` / ``solution_cost``: Section 2 objective with the penalised
  load excess and the time-warp relaxation (Section 4.3.3), by forward
  simulation; with pickups (VRPSPDTW, an instance whose ``pickup`` is not
  None) the load excess is that of the largest load on board
  (``route_peak_load``).
* ``best_move(method="def")``: the plain definition -- every candidate of
  relocate / swap / 2-opt / 2-opt* / or-opt (Section 4.1), and of the
  optional swaps of runs (ranks 6, 7: Section 5.3.1 Swap with run lengths 1
  and 2, or 2 and 2), is built by route surgery and costed from scratch; the
  smallest (delta, move index) wins (best improvement, Section 5.3.4, Eq.
  "min_obj").
* ``best_move(method="concat")``: the paper's sequence concatenation
  (Sections 4.2-4.3): per-route attribute matrices and the concatenation
  operator; must agree exactly with "def".
* ``best_move_slice``: ``best_move`` over one of several interleaved
  slices of the same candidate set (the harness spreads one evaluation over
  host processes with it; the arithmetic is unchanged).
* ``descend``: the feasible/infeasible search loop of the appendix algorithm
  with best improvement: accept iff delta < 0, stop at a local optimum.
* ``granular=nbr`` (every evaluating function): the edge-based extraction of
  Section 5.3.1 with a granular mask given as the theta nearest customers of
  each customer (rows of ``nbr``); the kept candidates are listed in
  ``tga_oracle.h``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tga_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libtga_oracle.so")
_lock = threading.Lock()
_lib = None

METHODS = {"def": 0, "concat": 1}
NO_MOVE_KEY = (1 << 64) - 1


class _Inst(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int32), ("capacity", ctypes.c_int32),
                ("has_tw", ctypes.c_int32), ("w_load", ctypes.c_int32), ("w_tw", ctypes.c_int32),
                ("dist", ctypes.c_void_p), ("demand", ctypes.c_void_p), ("service", ctypes.c_void_p),
                ("early", ctypes.c_void_p), ("late", ctypes.c_void_p),
                ("theta", ctypes.c_int32), ("nbr", ctypes.c_void_p), ("pickup", ctypes.c_void_p)]


class _Move(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_int64), ("idx", ctypes.c_uint64), ("op", ctypes.c_int32),
                ("a", ctypes.c_int32), ("b", ctypes.c_int32), ("found", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/libtga_oracle.so``."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
                os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "tga_oracle.h"))):
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.orc_route_cost.restype = ctypes.c_int64
        lib.orc_route_cost.argtypes = [ctypes.POINTER(_Inst), P, ctypes.c_int32]
        lib.orc_route_peak_load.restype = ctypes.c_int64
        lib.orc_route_peak_load.argtypes = [ctypes.POINTER(_Inst), P, ctypes.c_int32]
        lib.orc_route_warp.restype = ctypes.c_int64
        lib.orc_route_warp.argtypes = [ctypes.POINTER(_Inst), P, ctypes.c_int32]
        lib.orc_solution_cost.restype = ctypes.c_int64
        lib.orc_solution_cost.argtypes = [ctypes.POINTER(_Inst), P, P]
        lib.orc_check_solution.restype = ctypes.c_int
        lib.orc_check_solution.argtypes = [ctypes.POINTER(_Inst), P, P]
        lib.orc_count_candidates.restype = ctypes.c_int64
        lib.orc_count_candidates.argtypes = [ctypes.POINTER(_Inst), P, P, ctypes.c_uint32]
        lib.orc_best_move.restype = ctypes.c_int
        lib.orc_best_move.argtypes = [ctypes.POINTER(_Inst), P, P, ctypes.c_uint32, ctypes.c_int,
                                      ctypes.POINTER(_Move), ctypes.POINTER(ctypes.c_int64)]
        lib.orc_best_move_slice.restype = ctypes.c_int
        lib.orc_best_move_slice.argtypes = [ctypes.POINTER(_Inst), P, P, ctypes.c_uint32, ctypes.c_int,
                                            ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_Move),
                                            ctypes.POINTER(ctypes.c_int64)]
        lib.orc_list_moves.restype = ctypes.c_int64
        lib.orc_list_moves.argtypes = [ctypes.POINTER(_Inst), P, P, ctypes.c_uint32, ctypes.c_int,
                                       P, P, ctypes.c_int64]
        lib.orc_apply_move.restype = ctypes.c_int
        lib.orc_apply_move.argtypes = [ctypes.POINTER(_Inst), P, P, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32]
        lib.orc_descend.restype = ctypes.c_int64
        lib.orc_descend.argtypes = [ctypes.POINTER(_Inst), P, P, ctypes.c_uint32, ctypes.c_int,
                                    ctypes.c_int64, P, ctypes.c_int64,
                                    ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        lib.orc_seg_node.restype = None
        lib.orc_seg_node.argtypes = [ctypes.POINTER(_Inst), ctypes.c_int32, P]
        lib.orc_seg_concat.restype = None
        lib.orc_seg_concat.argtypes = [ctypes.POINTER(_Inst), P, P, P]
        _lib = lib
    return _lib


def _c32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


class OracleInstance:
    """Host copy of an instance laid out for the C oracle.  ``inst`` is any
    object with the fields of ``instances.Instance``."""

    def __init__(self, inst, n_routes: int, granular=None):
        self.n = int(inst.n)
        self.m = int(n_routes)
        self._arrs = [_c32(inst.dist).reshape(-1), _c32(inst.demand), _c32(inst.service),
                      _c32(inst.tw_early), _c32(inst.tw_late)]
        d, dem, svc, e, l = self._arrs
        theta, nbr_ptr = 0, None
        if granular is not None:
            self._nbr = _c32(granular)
            assert self._nbr.ndim == 2 and self._nbr.shape[0] == self.n + 1
            theta, nbr_ptr = int(self._nbr.shape[1]), self._nbr.ctypes.data
        pick = getattr(inst, "pickup", None)
        pick_ptr = None
        if pick is not None:
            self._pick = _c32(pick)
            assert self._pick.shape == (self.n + 1,)
            pick_ptr = self._pick.ctypes.data
        self.c = _Inst(self.n, self.m, int(inst.capacity), int(bool(inst.has_tw)), int(inst.w_load),
                       int(inst.w_tw), d.ctypes.data, dem.ctypes.data, svc.ctypes.data,
                       e.ctypes.data, l.ctypes.data, theta, nbr_ptr, pick_ptr)
        self.W = self.n + 1 + self.m

    def ref(self):
        return ctypes.byref(self.c)


def _oi(inst, sol, granular=None) -> OracleInstance:
    return OracleInstance(inst, int(np.asarray(sol.route_start).shape[0]) - 1, granular)


def route_cost(inst, nodes, n_routes: int = 1) -> int:
    oi = OracleInstance(inst, n_routes)
    a = _c32(nodes)
    return int(_load().orc_route_cost(oi.ref(), a.ctypes.data, a.shape[0]))


def route_peak_load(inst, nodes) -> int:
    """Largest load on board along the route (forward simulation)."""
    oi = OracleInstance(inst, 1)
    a = _c32(nodes)
    return int(_load().orc_route_peak_load(oi.ref(), a.ctypes.data, a.shape[0]))


def route_warp(inst, nodes) -> int:
    oi = OracleInstance(inst, 1)
    a = _c32(nodes)
    return int(_load().orc_route_warp(oi.ref(), a.ctypes.data, a.shape[0]))


def solution_cost(inst, sol) -> int:
    oi = _oi(inst, sol)
    t, rs = _c32(sol.tour), _c32(sol.route_start)
    return int(_load().orc_solution_cost(oi.ref(), t.ctypes.data, rs.ctypes.data))


def check_solution(inst, sol) -> int:
    oi = _oi(inst, sol)
    t, rs = _c32(sol.tour), _c32(sol.route_start)
    return int(_load().orc_check_solution(oi.ref(), t.ctypes.data, rs.ctypes.data))


def count_candidates(inst, sol, op_mask: int, granular=None) -> int:
    oi = _oi(inst, sol, granular)
    t, rs = _c32(sol.tour), _c32(sol.route_start)
    return int(_load().orc_count_candidates(oi.ref(), t.ctypes.data, rs.ctypes.data, op_mask))


def best_move(inst, sol, op_mask: int, method: str = "def", granular=None):
    """Returns dict(found, delta, idx, op, a, b, key, candidates)."""
    oi = _oi(inst, sol, granular)
    t, rs = _c32(sol.tour), _c32(sol.route_start)
    mv = _Move()
    nc = ctypes.c_int64(0)
    _load().orc_best_move(oi.ref(), t.ctypes.data, rs.ctypes.data, op_mask, METHODS[method],
                          ctypes.byref(mv), ctypes.byref(nc))
    return _move_dict(mv, nc.value)


def best_move_slice(inst, sol, op_mask: int, phase: int, stride: int, method: str = "concat", granular=None):
    """best_move over the slice `phase` of `stride` interleaved slices of
    the candidate set (split by the outermost enumeration index); the
    smallest key over all slices is best_move's."""
    oi = _oi(inst, sol, granular)
    t, rs = _c32(sol.tour), _c32(sol.route_start)
    mv = _Move()
    nc = ctypes.c_int64(0)
    rc = _load().orc_best_move_slice(oi.ref(), t.ctypes.data, rs.ctypes.data, op_mask, METHODS[method],
                                     int(phase), int(stride), ctypes.byref(mv), ctypes.byref(nc))
    if rc != 0:
        raise ValueError(f"bad slice {phase} of {stride}")
    return _move_dict(mv, nc.value)


def _move_dict(mv: _Move, cands: int):
    found = bool(mv.found)
    key = pack_key(mv.delta, mv.idx) if found else NO_MOVE_KEY
    return dict(found=found, delta=int(mv.delta), idx=int(mv.idx), op=int(mv.op), a=int(mv.a),
                b=int(mv.b), key=key, candidates=int(cands))


def pack_key(delta: int, idx: int) -> int:
    """((delta + 2^31) << 32) | idx, the packed (delta, move index) order."""
    return (((int(delta) + (1 << 31)) & 0xFFFFFFFF) << 32) | (int(idx) & 0xFFFFFFFF)


def unpack_key(key: int):
    return (int(key) >> 32) - (1 << 31), int(key) & 0xFFFFFFFF


def list_moves(inst, sol, op_mask: int, method: str = "def", granular=None):
    """All candidates as (idx array uint64, delta array int64)."""
    oi = _oi(inst, sol, granular)
    t, rs = _c32(sol.tour), _c32(sol.route_start)
    cnt = count_candidates(inst, sol, op_mask, granular)
    idx = np.zeros(max(cnt, 1), dtype=np.uint64)
    dl = np.zeros(max(cnt, 1), dtype=np.int64)
    got = _load().orc_list_moves(oi.ref(), t.ctypes.data, rs.ctypes.data, op_mask, METHODS[method],
                                 idx.ctypes.data, dl.ctypes.data, cnt)
    assert got == cnt, (got, cnt)
    return idx[:cnt], dl[:cnt]


def apply_move(inst, sol, op: int, a: int, b: int):
    """Route surgery on a copy of ``sol``; returns the new solution."""
    oi = _oi(inst, sol)
    new = sol.copy()
    new.tour = _c32(new.tour).copy()
    new.route_start = _c32(new.route_start).copy()
    rc = _load().orc_apply_move(oi.ref(), new.tour.ctypes.data, new.route_start.ctypes.data,
                                op, a, b)
    if rc != 0:
        raise ValueError(f"not a candidate move: op={op} a={a} b={b}")
    return new


def descend(inst, sol, op_mask: int, method: str = "def", max_steps: int = 1 << 62,
            log_cap: int = 1 << 20, granular=None):
    """Best-improvement descent on a copy of ``sol``.
    Returns (final solution, steps, key log (uint64 array), candidates)."""
    oi = _oi(inst, sol, granular)
    new = sol.copy()
    new.tour = _c32(new.tour).copy()
    new.route_start = _c32(new.route_start).copy()
    log = np.zeros(log_cap, dtype=np.uint64)
    cands = ctypes.c_int64(0)
    evals = ctypes.c_int64(0)
    steps = _load().orc_descend(oi.ref(), new.tour.ctypes.data, new.route_start.ctypes.data,
                                op_mask, METHODS[method], max_steps, log.ctypes.data, log_cap,
                                ctypes.byref(cands), ctypes.byref(evals))
    return new, int(steps), log[:min(evals.value, log_cap)].copy(), int(cands.value)


SEG_FIELDS = ("D", "LI", "LO", "LM", "TD", "TE", "TL", "TV", "first", "last")


def seg_node(inst, v: int):
    """Single-node segment as an int64 array with the fields SEG_FIELDS."""
    oi = OracleInstance(inst, 1)
    out = np.zeros(10, dtype=np.int64)
    _load().orc_seg_node(oi.ref(), v, out.ctypes.data)
    return out


def seg_concat(inst, s1, s2):
    oi = OracleInstance(inst, 1)
    a = np.ascontiguousarray(s1, dtype=np.int64)
    b = np.ascontiguousarray(s2, dtype=np.int64)
    out = np.zeros(10, dtype=np.int64)
    _load().orc_seg_concat(oi.ref(), a.ctypes.data, b.ctypes.data, out.ctypes.data)
    return out
